// lq_device.cuh -- device helpers shared by the lq kernels: complex
// arithmetic in the forms the tile ops use, sign-bit manipulation without
// FP64 instructions, bit deposit/insert, and the tile-op interpreter.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "lq_internal.h"
#include "lq_kernels.h"

namespace lq {

// Flip the sign of a double when `flip` is 0x80000000 (integer pipe only).
__device__ __forceinline__ double xsign(double x, uint32_t flip) {
  return __hiloint2double(__double2hiint(x) ^ (int)flip, __double2loint(x));
}

// v * i^k (k mod 4): register moves and sign flips, no FP64 instruction.
__device__ __forceinline__ double2 mul_ipow(double2 v, int k) {
  double re = (k & 1) ? v.y : v.x;
  double im = (k & 1) ? v.x : v.y;
  uint32_t sre = (uint32_t)((k + 1) & 2) << 30;
  uint32_t sim = (uint32_t)(k & 2) << 30;
  return make_double2(xsign(re, sre), xsign(im, sim));
}

__device__ __forceinline__ double2 cmul(double2 v, double wr, double wi) {
  return make_double2(fma(v.x, wr, -v.y * wi), fma(v.x, wi, v.y * wr));
}

// 16-byte asynchronous global -> shared copy (completion by
// cp.async.wait_group, a hardware wait: no spin loop).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Hint: bring the cache line holding gmem into L2 (no register result, no
// wait).  A tile kernel issues it for its next tile while it computes the
// current one, so that tile's synchronous load hits L2 instead of HBM.
__device__ __forceinline__ void prefetch_l2(const void* gmem) {
  asm volatile("prefetch.global.L2 [%0];\n" ::"l"(gmem));
}

// Insert a zero bit at position b of j.
__device__ __forceinline__ uint32_t insert0(uint32_t j, int b) {
  uint32_t lo = j & ((1u << b) - 1u);
  return ((j ^ lo) << 1) | lo;
}
__device__ __forceinline__ uint64_t insert0_64(uint64_t j, int b) {
  uint64_t lo = j & ((1ull << b) - 1ull);
  return ((j ^ lo) << 1) | lo;
}

// Expand j into a tile index whose bits in mask M take the values of V and
// whose other bits are the bits of j in order (so every lane of a loop over
// j < T >> popcount(M) lands on an amplitude the op changes).
__device__ __forceinline__ uint32_t expand(uint32_t j, uint32_t M, uint32_t V) {
  uint32_t s = j;
  while (M) {
    const int b = __ffs(M) - 1;
    M &= M - 1;
    s = insert0(s, b) | (V & (1u << b));
  }
  return s;
}

// Scatter the low bits of v onto the bit positions pos[0..cnt).
__device__ __forceinline__ uint64_t deposit(uint64_t v, const int8_t* pos, int cnt) {
  uint64_t r = 0;
  for (int i = 0; i < cnt; i++) r |= ((v >> i) & 1ull) << pos[i];
  return r;
}

// All threads of the block call it; the caller synchronises.
// Partial <H> of one thread over state `st` (shared or global memory): the
// thread visits amplitudes/pairs t0, t0 + nth, ...  Terms sharing an X mask
// form a group.  A group with x != 0 visits each unordered pair (i, i^x) once
// (i has the top bit of x clear) and adds 2 c_t Re(i^kk conj(psi_i) psi_j),
// kk = k0 + 2 parity(j & z), j = i^x (only the Re or Im part of
// conj(psi_i) psi_j when the group's terms allow).  The x == 0 group adds
// c_t (-1)^popcount(i & z_t) |psi_i|^2, terms inside one 8-bit index chunk
// through the tables `tab` (per chunk 256 entries, built by the caller;
// nullptr: all terms direct).
__device__ __forceinline__ double expval_partial(const double2* __restrict__ st, int n,
                                                 const ExpGroup* __restrict__ groups,
                                                 int ngroups, const ExpTerm* __restrict__ terms,
                                                 uint64_t t0, uint64_t nth,
                                                 const double* __restrict__ tab) {
  const uint64_t N = 1ull << n;
  const int nch = (n + EXP_CHUNK_BITS - 1) / EXP_CHUNK_BITS;
  double acc = 0.0;
  for (int g = 0; g < ngroups; g++) {
    const ExpGroup G = groups[g];
    if (G.x == 0) {
      for (uint64_t i = t0; i < N; i += nth) {
        const double2 v = st[i];
        const double p = fma(v.x, v.x, v.y * v.y);
        double d = 0.0;
        if (tab)
          for (int c = 0; c < nch; c++)
            d += tab[c * 256 + ((i >> (EXP_CHUNK_BITS * c)) & 255)];
        for (int t = G.first; t < G.first + G.count; t++) {
          if (tab && terms[t].chunk > 0) continue;
          const uint32_t f = (uint32_t)(__popcll(i & terms[t].z) & 1) << 31;
          d += xsign(terms[t].c, f);
        }
        acc = fma(d, p, acc);
      }
    } else {
      for (uint64_t j = t0; j < (N >> 1); j += nth) {
        const uint64_t i = insert0_64(j, G.h), l = i ^ G.x;
        const double2 a = st[i], b = st[l];
        const double vr = G.part == 2 ? 0.0 : fma(a.x, b.x, a.y * b.y);
        const double vi = G.part == 1 ? 0.0 : fma(a.x, b.y, -(a.y * b.x));
        for (int t = G.first; t < G.first + G.count; t++) {
          const int kk = (terms[t].k0 + 2 * (__popcll(l & terms[t].z) & 1)) & 3;
          // Re(i^kk v): vr, -vi, -vr, vi
          const double val = (kk & 1) ? vi : vr;
          const uint32_t f = (uint32_t)(((kk + 1) & 2) >> 1) << 31;
          acc = fma(xsign(terms[t].c2, f), val, acc);
        }
      }
    }
  }
  return acc;
}

// Build the diagonal-term chunk tables (nch x 256 doubles) in shared memory:
// tab[c][v] = sum over the x == 0 terms inside chunk c of c_t (-1)^popcount(v & z_t).
__device__ __forceinline__ void expval_tables(double* tab, int n, const ExpGroup* groups,
                                              int ngroups, const ExpTerm* terms) {
  const int nch = (n + EXP_CHUNK_BITS - 1) / EXP_CHUNK_BITS;
  for (int e = threadIdx.x; e < nch * 256; e += blockDim.x) {
    const int c = e >> 8, v = e & 255;
    double s = 0.0;
    for (int g = 0; g < ngroups; g++) {
      if (groups[g].x != 0) continue;
      for (int t = groups[g].first; t < groups[g].first + groups[g].count; t++) {
        if (terms[t].chunk != c + 1) continue;
        const uint32_t zl = (uint32_t)(terms[t].z >> (EXP_CHUNK_BITS * c)) & 255u;
        s += (__popc((uint32_t)v & zl) & 1) ? -terms[t].c : terms[t].c;
      }
    }
    tab[e] = s;
  }
}

// One-bit Pauli rotation with a uniform phase per side: x = 1 << h and the
// string's Z bits inside the tile are at most h, so for a pair (s0, s1 = s0 |
// x) the phases are w_A = i^kA (applied to psi_s1 in out_s0) and w_B = i^kB
// (applied to psi_s0 in out_s1), the same for every pair of the tile.  The
// powers' parities are template arguments; their signs are folded into the
// coefficients (tangent form: out = own + c * rot(other)) or applied as sign
// bits (cotangent form: out = a * own + sign * rot(other)), where rot is the
// identity for an even power and multiplication by i for an odd one.  Two
// pairs per thread and iteration: all four loads issue before any store.
template <bool ODD>
__device__ __forceinline__ double2 rot_fma(double c, double2 other, double2 own) {
  return ODD ? make_double2(fma(-c, other.y, own.x), fma(c, other.x, own.y))
             : make_double2(fma(c, other.x, own.x), fma(c, other.y, own.y));
}
template <bool ODD>
__device__ __forceinline__ double2 rot_cot(double a, double2 own, double2 other, uint32_t sg) {
  return ODD ? make_double2(fma(a, own.x, xsign(other.y, sg ^ 0x80000000u)),
                            fma(a, own.y, xsign(other.x, sg)))
             : make_double2(fma(a, own.x, xsign(other.x, sg)), fma(a, own.y, xsign(other.y, sg)));
}
template <bool ODD>
__device__ __forceinline__ double2 rot_perm(double2 other, uint32_t sg) {
  return ODD ? make_double2(xsign(other.y, sg ^ 0x80000000u), xsign(other.x, sg))
             : make_double2(xsign(other.x, sg), xsign(other.y, sg));
}
enum RotForm { ROT_COT = 0, ROT_TAN = 1, ROT_PERM = 2 };
template <int BLOCK, int FORM, bool OA, bool OB>
__device__ __forceinline__ void rot1_pairs(double2* __restrict__ sm, uint32_t cnt, uint32_t M,
                                           uint32_t cv, uint32_t x, double a, double cA,
                                           double cB, uint32_t sA, uint32_t sB) {
  const uint32_t tid = threadIdx.x;
  const int h = 31 - __clz(x);
  const bool plain = M == x;   // no tile-local condition
  auto idx = [&](uint32_t j) { return plain ? insert0(j, h) : expand(j, M, cv); };
  auto pair = [&](double2 A, double2 B, double2& o0, double2& o1) {
    if (FORM == ROT_TAN) {
      o0 = rot_fma<OA>(cA, B, A);
      o1 = rot_fma<OB>(cB, A, B);
    } else if (FORM == ROT_COT) {
      o0 = rot_cot<OA>(a, A, B, sA);
      o1 = rot_cot<OB>(a, B, A, sB);
    } else {
      o0 = rot_perm<OA>(B, sA);
      o1 = rot_perm<OB>(A, sB);
    }
  };
  if ((cnt & (2 * BLOCK - 1)) == 0) {
    for (uint32_t j = tid; j < cnt; j += 2 * BLOCK) {
      const uint32_t p0 = idx(j), q0 = idx(j + BLOCK);
      const double2 A = sm[p0], B = sm[p0 | x], C = sm[q0], D = sm[q0 | x];
      double2 o0, o1, o2, o3;
      pair(A, B, o0, o1);
      pair(C, D, o2, o3);
      sm[p0] = o0;
      sm[p0 | x] = o1;
      sm[q0] = o2;
      sm[q0 | x] = o3;
    }
  } else {
    for (uint32_t j = tid; j < cnt; j += BLOCK) {
      const uint32_t p0 = idx(j);
      const double2 A = sm[p0], B = sm[p0 | x];
      double2 o0, o1;
      pair(A, B, o0, o1);
      sm[p0] = o0;
      sm[p0 | x] = o1;
    }
  }
}

// Phase table of a table-mode OP_LPHASE (every factor's condition bit is a
// tile bit): tab[s] = product of the factors w_f whose condition holds for
// tile index s, s < 2^k.  Per tile bit b, c_b = product of the factors on b
// (a factor that needs s_b = 0 contributes w to the constant e0 and conj(w)
// to c_b); then tab is built by doubling from tab[0] = e0.  All threads call
// it; it ends with a barrier.
template <int BLOCK>
__device__ __forceinline__ void build_lphase_table(double2* tab, int k, const Op& op,
                                                   const double* __restrict__ coef) {
  __shared__ double2 lt_c[MAX_TILE_BITS + 1];
  const uint32_t tid = threadIdx.x;
  const int nf = (int)op.x_loc;
  const double* F = coef + op.cidx;
  if (tid <= (uint32_t)k) {
    double cr = 1, ci = 0;
    for (int f = 0; f < nf; f++) {
      const double* Ff = F + LPHASE_FAC * f;
      const uint64_t loc = (uint64_t)__double_as_longlong(Ff[0]);
      const uint32_t lm = (uint32_t)loc, lv = (uint32_t)(loc >> 32);
      double wr = Ff[3], wi = Ff[4];
      if (lm == 0) {
        if (tid != (uint32_t)k) continue;
      } else {
        const int b = __ffs(lm) - 1;
        if (tid == (uint32_t)k) {
          if (lv & lm) continue;
        } else {
          if (b != (int)tid) continue;
          if (!(lv & lm)) wi = -wi;
        }
      }
      const double nr = fma(cr, wr, -ci * wi), ni = fma(cr, wi, ci * wr);
      cr = nr;
      ci = ni;
    }
    lt_c[tid] = make_double2(cr, ci);
  }
  __syncthreads();
  if (tid == 0) tab[0] = lt_c[k];
  __syncthreads();
  for (int b = 0; b < k; b++) {
    const double2 c = lt_c[b];
    for (uint32_t s = tid; s < (1u << b); s += BLOCK) tab[s | (1u << b)] = cmul(tab[s], c.x, c.y);
    __syncthreads();
  }
}

// Diagonal update v <- f(s, v) of the cnt amplitudes s = expand(j, cm, cv),
// j < cnt; U amplitudes per thread and iteration, all loaded before any is
// stored.
template <int BLOCK, int U, typename F>
__device__ __forceinline__ void diag_apply(double2* __restrict__ sm, uint32_t cnt, uint32_t cm,
                                           uint32_t cv, F f) {
  const uint32_t tid = threadIdx.x;
  if (cnt % (U * BLOCK) == 0) {
    for (uint32_t j = tid; j < cnt; j += U * BLOCK) {
      uint32_t sx[U];
      double2 v[U];
#pragma unroll
      for (int u = 0; u < U; u++) {
        sx[u] = cm ? expand(j + u * BLOCK, cm, cv) : j + u * BLOCK;
        v[u] = sm[sx[u]];
      }
#pragma unroll
      for (int u = 0; u < U; u++) v[u] = f(sx[u], v[u]);
#pragma unroll
      for (int u = 0; u < U; u++) sm[sx[u]] = v[u];
    }
  } else {
    for (uint32_t j = tid; j < cnt; j += BLOCK) {
      const uint32_t sj = expand(j, cm, cv);
      sm[sj] = f(sj, sm[sj]);
    }
  }
}

// Per-CTA tables of a table-mode OP_DPHASE: at `out` (256 words) the two
// 128-entry partial sums of the tile-bit weights (entry 0 of the first also
// holds the weights that hold on every tile); at `triples` (CTA mask, CTA
// value, weight) of each factor decided by CTA bits alone.  A factor that needs
// s_b = 0 adds w to the constant and -w to c_b.  All threads call it; it
// ends with a barrier.
template <int BLOCK>
__device__ __forceinline__ void build_dphase_table(unsigned long long* out,
                                                   unsigned long long* triples, int k,
                                                   const Op& op,
                                                   const double* __restrict__ coef) {
  __shared__ unsigned long long dt_c[MAX_TILE_BITS + 1];
  const uint32_t tid = threadIdx.x;
  const int nf = (int)op.x_loc;
  const double* F = coef + op.cidx;
  const unsigned long long M34 = (1ull << DYADIC_BITS) - 1ull;
  if (tid <= (uint32_t)k) {
    unsigned long long acc = 0;
    for (int f = 0; f < nf; f++) {
      const uint64_t loc = (uint64_t)__double_as_longlong(F[4 * f]);
      const uint64_t gm = (uint64_t)__double_as_longlong(F[4 * f + 1]);
      const unsigned long long w = (unsigned long long)__double_as_longlong(F[4 * f + 3]);
      const uint32_t lm = (uint32_t)loc & ~op.cm_loc, lv = (uint32_t)(loc >> 32);
      if (lm == 0) {
        if (gm == 0 && tid == (uint32_t)k) acc += w;
        continue;
      }
      const uint32_t b = (uint32_t)(__ffs(lm) - 1);
      if (lv & lm) {
        if (tid == b) acc += w;
      } else {
        if (tid == (uint32_t)k) acc += w;
        if (tid == b) acc += (1ull << DYADIC_BITS) - w;
      }
    }
    dt_c[tid] = acc & M34;
  }
  __syncthreads();
  for (uint32_t v = tid; v < 256; v += BLOCK) {
    const int c = v >> 7;
    unsigned long long e = c ? 0ull : dt_c[k];
    for (int b = 0; b < 7; b++)
      if (((v & 127) >> b) & 1 && 7 * c + b < k) e += dt_c[7 * c + b];
    out[v] = e & M34;
  }
  if (tid == 0) {
    int q = 0;
    for (int f = 0; f < nf; f++) {
      const uint64_t loc = (uint64_t)__double_as_longlong(F[4 * f]);
      const uint64_t gm = (uint64_t)__double_as_longlong(F[4 * f + 1]);
      if (((uint32_t)loc & ~op.cm_loc) != 0 || gm == 0) continue;
      triples[3 * q] = gm;
      triples[3 * q + 1] = (uint64_t)__double_as_longlong(F[4 * f + 2]);
      triples[3 * q + 2] = (unsigned long long)__double_as_longlong(F[4 * f + 3]);
      q++;
    }
  }
  __syncthreads();
}

// exp(2 pi i E / 2^34) from the two-level dyadic tables dtab (hi: 2^17
// entries exp(2 pi i h / 2^17), lo: 2^17 entries exp(2 pi i l / 2^34)).
__device__ __forceinline__ double2 dyadic_phase(unsigned long long E,
                                                const double2* __restrict__ dtab) {
  if (E == 0) return make_double2(1.0, 0.0);
  double2 w = dtab[E >> DYADIC_HALF];
  const unsigned long long lo = E & ((1ull << DYADIC_HALF) - 1ull);
  if (lo) {
    const double2 wl = dtab[(1u << DYADIC_HALF) + lo];
    w = cmul(w, wl.x, wl.y);
  }
  return w;
}

// Full phase table of a full-mode OP_DPHASE: F[u] = exp(2 pi i (t0 + t1) /
// 2^34) at s = expand(u, cm, cv), from its partial-sum tables tb (the
// tile-invariant part of E).  No barrier: the caller synchronises.
template <int BLOCK>
__device__ __forceinline__ void build_dfull_table(double2* F, int k, const Op& op,
                                                  const unsigned long long* tb,
                                                  const double2* __restrict__ dtab) {
  const unsigned long long M34 = (1ull << DYADIC_BITS) - 1ull;
  const bool bf = (op.mode & DP_BFLY) != 0;
  const int lo = bf ? (int)op.a : 0;
  const uint32_t cnt = bf ? 1u << (int)op.b : 1u << (k - __popc(op.cm_loc));
  unsigned char* form = reinterpret_cast<unsigned char*>(F + cnt);   // DP_BFLY only
  for (uint32_t u = threadIdx.x; u < cnt; u += BLOCK) {
    // butterflies: the factor bits' run at u, the condition bit set
    const uint32_t s = bf ? (u << lo) | op.cm_loc : expand(u, op.cm_loc, op.cv_loc);
    const double2 w = dyadic_phase((tb[s & 127] + tb[128 + ((s >> 7) & 127)]) & M34, dtab);
    if (bf) {
      // w = Re w (1 + i Im w / Re w), or w = Im w (1 + i (-Re w / Im w)) i
      const bool cot = fabs(w.x) < fabs(w.y);
      F[u] = cot ? make_double2(w.y, -w.x / w.y) : make_double2(w.x, w.y / w.x);
      form[u] = cot;
    } else {
      F[u] = w;
    }
  }
}


// Per-tile constant of a table-mode OP_DPHASE: the sum of the weights of its
// `ncta` CTA-decided factors (triples at tr) that hold for the tile's CTA
// bits `base`; every warp computes it with shuffles.
__device__ __forceinline__ unsigned long long dphase_tile_sum(const unsigned long long* tr,
                                                              int ncta, uint64_t base) {
  unsigned long long e0 = 0;
  for (int q = (int)(threadIdx.x & 31); q < ncta; q += 32)
    if ((base & tr[3 * q]) == tr[3 * q + 1]) e0 += tr[3 * q + 2];
  for (int o = 16; o > 0; o >>= 1) e0 += __shfl_xor_sync(0xffffffffu, e0, o);
  return e0;
}

// Per-CTA tables of a pass (pass_kernel); a member is nullptr when absent.
struct PassTables {
  const double2* ltab;               // table-mode OP_LPHASE phase table
  const unsigned long long* dpt;     // table-mode OP_DPHASE partial sums
  const double2* dfull;              // full-mode OP_DPHASE phase tables
  unsigned long long* dfe;           // full mode: this tile's deferred sums
};

// A DP_BFLY op and the OP_H after it: for each pair (s0, s1 = s0 | 2^c),
// a' = a + w b, b' = a - w b with w = scale (1 + i s) applied to u = b or
// u = i b (form byte): t = u (1 + i s) in 2 FMAs, a +- scale t in 4.  The
// table index is the pair's factor-bit run (s0 >> a) mod 2^b (the condition
// bit c lies outside the run).
template <int BLOCK>
__device__ __forceinline__ void dphase_bfly_pairs(double2* __restrict__ sm, uint32_t T,
                                                  const Op& d, const PassTables* tabs) {
  const uint32_t tid = threadIdx.x;
  const uint32_t cnt = T >> 1;
  const int lo = (int)d.a;
  const uint32_t tmask = (1u << (int)d.b) - 1u;   // table: 2^b entries, then form bytes
  const double2* __restrict__ F = tabs->dfull + d.z_glob;
  const unsigned char* __restrict__ form = reinterpret_cast<const unsigned char*>(F + tmask + 1);
  const uint32_t xb = d.cm_loc;
  const int c = __ffs(xb) - 1;
  auto bfly = [&](double2 A, double2 B, double2 w, unsigned f, double2& o0, double2& o1) {
    const uint32_t neg = f ? 0x80000000u : 0u;
    const double ux = f ? xsign(B.y, neg) : B.x, uy = f ? B.x : B.y;
    const double tx = fma(-w.y, uy, ux), ty = fma(w.y, ux, uy);
    o0 = make_double2(fma(w.x, tx, A.x), fma(w.x, ty, A.y));
    o1 = make_double2(fma(-w.x, tx, A.x), fma(-w.x, ty, A.y));
  };
  if ((cnt & (2 * BLOCK - 1)) == 0) {
    for (uint32_t j = tid; j < cnt; j += 2 * BLOCK) {
      const uint32_t p0 = insert0(j, c), q0 = insert0(j + BLOCK, c);
      const double2 A = sm[p0], B = sm[p0 | xb], C = sm[q0], D = sm[q0 | xb];
      const uint32_t i0 = (p0 >> lo) & tmask, i1 = (q0 >> lo) & tmask;
      const double2 w0 = F[i0], w1 = F[i1];
      const unsigned f0 = form[i0], f1 = form[i1];
      double2 o0, o1, o2, o3;
      bfly(A, B, w0, f0, o0, o1);
      bfly(C, D, w1, f1, o2, o3);
      sm[p0] = o0;
      sm[p0 | xb] = o1;
      sm[q0] = o2;
      sm[q0 | xb] = o3;
    }
  } else {
    for (uint32_t j = tid; j < cnt; j += BLOCK) {
      const uint32_t s0 = insert0(j, c), i0 = (s0 >> lo) & tmask;
      double2 o0, o1;
      bfly(sm[s0], sm[s0 | xb], F[i0], form[i0], o0, o1);
      sm[s0] = o0;
      sm[s0 | xb] = o1;
    }
  }
}

// Apply one op to a shared-memory tile of T = 2^k amplitudes whose CTA bits
// are `base`; dtab: the dyadic phase tables; tabs: the pass's per-CTA tables
// (pass_kernel), or nullptr; pt: the circuit's patch (batched launches: the
// patched gate's factor of a merged one-bit phase op), or nullptr; sm2: a
// second tile that a per-tile-mode OP_LPHASE multiplies by the same phases
// (two-state passes), or nullptr.
template <int BLOCK>
__device__ __forceinline__ void apply_op(double2* __restrict__ sm, uint32_t T, const Op& op,
                                         const double* __restrict__ coef, uint64_t base,
                                         const double2* __restrict__ dtab,
                                         const PassTables* tabs = nullptr,
                                         const Patch* pt = nullptr,
                                         double2* __restrict__ sm2 = nullptr) {
  const uint32_t tid = threadIdx.x;
  // per-tile tables of OP_DPHASE (2 x 128 sums) or OP_LPHASE (2 x 128
  // phases); one op at a time uses it
  __shared__ __align__(16) double2 op_tab[2][128];
  if ((base & op.cm_glob) != op.cv_glob) return;  // CTA-level condition
  const int zs = __popcll(base & op.z_glob) & 1;
  const uint32_t cm = op.cm_loc, cv = op.cv_loc;
  switch (op.type) {
    case OP_PAULI: {
      const uint32_t x = op.x_loc, z = op.z_loc;
      const int h = 31 - __clz(x);
      const int k0 = op.mode >> 2, pm = op.mode & 3;
      const double a = op.a, b = op.b;
      const uint32_t M = cm | (1u << h);
      const uint32_t cnt = T >> __popc(M);
      if ((x & (x - 1)) == 0 && (z & ~x) == 0 && pm != PM_GEN) {
        // uniform phases: w_A = i^kA (pairs' s1 has the Z bit), w_B = i^kB
        const int kA = (k0 + 2 * (((z != 0) + zs) & 1)) & 3;
        const int kB = (k0 + 2 * (zs & 1)) & 3;
        // the signs as sign-bit flips (a double negation would take an FP64
        // instruction per thread and op)
        const uint32_t sA = (uint32_t)(kA & 2) << 30, sB = (uint32_t)(kB & 2) << 30;
        const double cA = xsign(a, sA), cB = xsign(a, sB);
        const int v = ((kA & 1) << 1) | (kB & 1);
#define LQ_ROT1(F, A_, B_) rot1_pairs<BLOCK, F, A_, B_>(sm, cnt, M, cv, x, a, cA, cB, sA, sB)
#define LQ_ROT1_FORM(F)                      \
  switch (v) {                               \
    case 0: LQ_ROT1(F, false, false); break; \
    case 1: LQ_ROT1(F, false, true); break;  \
    case 2: LQ_ROT1(F, true, false); break;  \
    default: LQ_ROT1(F, true, true); break;  \
  }
        if (pm == PM_TAN) {
          LQ_ROT1_FORM(ROT_TAN)
        } else if (pm == PM_COT) {
          LQ_ROT1_FORM(ROT_COT)
        } else {
          LQ_ROT1_FORM(ROT_PERM)
        }
#undef LQ_ROT1_FORM
#undef LQ_ROT1
        break;
      }
      for (uint32_t j = tid; j < cnt; j += BLOCK) {
        const uint32_t s0 = expand(j, M, cv);
        const uint32_t s1 = s0 ^ x;
        double2 A = sm[s0], B = sm[s1];
        int kA = (k0 + 2 * ((__popc(s1 & z) + zs) & 1)) & 3;
        int kB = (k0 + 2 * ((__popc(s0 & z) + zs) & 1)) & 3;
        double2 Bw = mul_ipow(B, kA), Aw = mul_ipow(A, kB);
        double2 o0, o1;
        if (pm == PM_TAN) {
          o0 = make_double2(fma(a, Bw.x, A.x), fma(a, Bw.y, A.y));
          o1 = make_double2(fma(a, Aw.x, B.x), fma(a, Aw.y, B.y));
        } else if (pm == PM_COT) {
          o0 = make_double2(fma(a, A.x, Bw.x), fma(a, A.y, Bw.y));
          o1 = make_double2(fma(a, B.x, Aw.x), fma(a, B.y, Aw.y));
        } else if (pm == PM_GEN) {
          o0 = make_double2(fma(b, Bw.x, a * A.x), fma(b, Bw.y, a * A.y));
          o1 = make_double2(fma(b, Aw.x, a * B.x), fma(b, Aw.y, a * B.y));
        } else {
          o0 = Bw;
          o1 = Aw;
        }
        sm[s0] = o0;
        sm[s1] = o1;
      }
      break;
    }
    case OP_H: {
      const int bb = op.b0;
      const uint32_t xb = 1u << bb;
      const uint32_t M = cm | xb;
      const uint32_t cnt = T >> __popc(M);
      if ((cnt & (2 * BLOCK - 1)) == 0) {
        for (uint32_t j = tid; j < cnt; j += 2 * BLOCK) {
          const uint32_t p0 = cm ? expand(j, M, cv) : insert0(j, bb);
          const uint32_t q0 = cm ? expand(j + BLOCK, M, cv) : insert0(j + BLOCK, bb);
          const double2 A = sm[p0], B = sm[p0 | xb], C = sm[q0], D = sm[q0 | xb];
          sm[p0] = make_double2(A.x + B.x, A.y + B.y);
          sm[p0 | xb] = make_double2(A.x - B.x, A.y - B.y);
          sm[q0] = make_double2(C.x + D.x, C.y + D.y);
          sm[q0 | xb] = make_double2(C.x - D.x, C.y - D.y);
        }
      } else {
        for (uint32_t j = tid; j < cnt; j += BLOCK) {
          const uint32_t s0 = expand(j, M, cv);
          const uint32_t s1 = s0 | xb;
          double2 A = sm[s0], B = sm[s1];
          sm[s0] = make_double2(A.x + B.x, A.y + B.y);
          sm[s1] = make_double2(A.x - B.x, A.y - B.y);
        }
      }
      break;
    }
    case OP_PAIR_GEN: {
      const int bb = op.b0;
      const double* M = coef + op.cidx;
      const double m00r = M[0], m00i = M[1], m01r = M[2], m01i = M[3];
      const double m10r = M[4], m10i = M[5], m11r = M[6], m11i = M[7];
      const uint32_t MM = cm | (1u << bb);
      const uint32_t cnt = T >> __popc(MM);
      for (uint32_t j = tid; j < cnt; j += BLOCK) {
        const uint32_t s0 = expand(j, MM, cv);
        const uint32_t s1 = s0 | (1u << bb);
        double2 A = sm[s0], B = sm[s1];
        double2 o0, o1;
        o0.x = fma(m00r, A.x, fma(-m00i, A.y, fma(m01r, B.x, -m01i * B.y)));
        o0.y = fma(m00r, A.y, fma(m00i, A.x, fma(m01r, B.y, m01i * B.x)));
        o1.x = fma(m10r, A.x, fma(-m10i, A.y, fma(m11r, B.x, -m11i * B.y)));
        o1.y = fma(m10r, A.y, fma(m10i, A.x, fma(m11r, B.y, m11i * B.x)));
        sm[s0] = o0;
        sm[s1] = o1;
      }
      break;
    }
    case OP_QUAD_GEN: {
      const int hb = op.b0, lb = op.b1;
      const double* M = coef + op.cidx;
      const uint32_t MM = cm | (1u << hb) | (1u << lb);
      const uint32_t cnt = T >> __popc(MM);
      for (uint32_t j = tid; j < cnt; j += BLOCK) {
        const uint32_t s = expand(j, MM, cv);
        uint32_t idx[4] = {s, s | (1u << lb), s | (1u << hb), s | (1u << hb) | (1u << lb)};
        double2 v[4];
#pragma unroll
        for (int c = 0; c < 4; c++) v[c] = sm[idx[c]];
#pragma unroll
        for (int r = 0; r < 4; r++) {
          double re = 0, im = 0;
#pragma unroll
          for (int c = 0; c < 4; c++) {
            double mr = M[2 * (4 * r + c)], mi = M[2 * (4 * r + c) + 1];
            re = fma(mr, v[c].x, fma(-mi, v[c].y, re));
            im = fma(mr, v[c].y, fma(mi, v[c].x, im));
          }
          sm[idx[r]] = make_double2(re, im);
        }
      }
      break;
    }
    case OP_SWAP: {
      const int b0 = op.b0, b1 = op.b1;
      const uint32_t MM = cm | (1u << b0) | (1u << b1);
      const uint32_t cnt = T >> __popc(MM);
      for (uint32_t j = tid; j < cnt; j += BLOCK) {
        const uint32_t s = expand(j, MM, cv);
        const uint32_t sa = s | (1u << b0), sb = s | (1u << b1);
        double2 A = sm[sa];
        sm[sa] = sm[sb];
        sm[sb] = A;
      }
      break;
    }
    case OP_PHASE: {
      const double wr = op.a, wi = op.b;
      diag_apply<BLOCK, 2>(sm, T >> __popc(cm), cm, cv,
                           [&](uint32_t, double2 v) { return cmul(v, wr, wi); });
      break;
    }
    case OP_SIGN: {
      diag_apply<BLOCK, 2>(sm, T >> __popc(cm), cm, cv, [&](uint32_t, double2 v) {
        return make_double2(xsign(v.x, 0x80000000u), xsign(v.y, 0x80000000u));
      });
      break;
    }
    case OP_MULI: {
      const int kk = op.mode & 3;
      diag_apply<BLOCK, 2>(sm, T >> __popc(cm), cm, cv,
                           [&](uint32_t, double2 v) { return mul_ipow(v, kk); });
      break;
    }
    case OP_PARITY: {
      // amplitudes with odd popcount(idx & z): pick the top free bit hz of z
      // and set it so the parity is odd
      const uint32_t z = op.z_loc, zf = z & ~cm;
      const double wr = op.a, wi = op.b;
      if (zf == 0) {  // parity fixed by the condition and CTA bits
        const uint32_t cnt = T >> __popc(cm);
        for (uint32_t j = tid; j < cnt; j += BLOCK) {
          const uint32_t s = expand(j, cm, cv);
          if (((__popc(s & z) + zs) & 1) == 0) continue;
          sm[s] = cmul(sm[s], wr, wi);
        }
      } else {
        const int hz = 31 - __clz(zf);
        const uint32_t M = cm | (1u << hz);
        const uint32_t cnt = T >> __popc(M);
        for (uint32_t j = tid; j < cnt; j += BLOCK) {
          uint32_t s = expand(j, M, cv);
          s |= (uint32_t)(((__popc(s & z) + zs) & 1) ^ 1) << hz;
          sm[s] = cmul(sm[s], wr, wi);
        }
      }
      break;
    }
    case OP_DPHASE: {
      // E(s) = sum of the weights of the factors whose conditions hold, mod
      // 2^34; phase exp(2 pi i E / 2^34) = hi[E >> 17] * lo[E & (2^17-1)].
      // When every factor has at most one tile bit beyond the op's common
      // condition, E is linear in the tile bits: E = e0 + sum_b c_b s_b,
      // evaluated per amplitude from two 7-bit partial-sum tables built per
      // tile; otherwise each amplitude sums its factors directly.
      __shared__ unsigned long long dp_e0, dp_c[MAX_TILE_BITS + 1];
      unsigned long long(*dp_t)[128] = reinterpret_cast<unsigned long long(*)[128]>(op_tab);
      __shared__ int dp_nonlin;
      const int nf = (int)op.x_loc;
      const double* F = coef + op.cidx;
      const uint32_t cnt = T >> __popc(cm);
      const unsigned long long M34 = (1ull << DYADIC_BITS) - 1ull, LOMASK = (1ull << DYADIC_HALF) - 1ull;
      if ((op.mode & DP_TABLE) && tabs && tabs->dpt) {
        const unsigned long long* tb = tabs->dpt + op.z_loc;
        if ((op.mode & DP_FULL) && tabs->dfull) {
          // tile-invariant part from the full table; e0 deferred to the store
          // (summed here) or to the load (summed when the tile started)
          if (!(op.mode & (DP_PRE | DP_NODEFER))) {
            const unsigned long long e0 = dphase_tile_sum(tb, (int)op.b1, base);   // triples
            if (tid == 0) tabs->dfe[op.b0] = e0;
          }
          const double2* __restrict__ F = tabs->dfull + op.z_glob;
          if ((cnt & (2 * BLOCK - 1)) == 0) {
            for (uint32_t j = tid; j < cnt; j += 2 * BLOCK) {
              const uint32_t s0 = expand(j, cm, cv), s1 = expand(j + BLOCK, cm, cv);
              const double2 a = sm[s0], b = sm[s1], w0 = F[j], w1 = F[j + BLOCK];
              sm[s0] = cmul(a, w0.x, w0.y);
              sm[s1] = cmul(b, w1.x, w1.y);
            }
          } else {
            for (uint32_t j = tid; j < cnt; j += BLOCK) {
              const uint32_t s = expand(j, cm, cv);
              const double2 w = F[j];
              sm[s] = cmul(sm[s], w.x, w.y);
            }
          }
          break;
        }
        // per-CTA partial sums; the per-tile constant summed by each warp
        const unsigned long long e0 = dphase_tile_sum(tb + 256, (int)op.b1, base);
        for (uint32_t j = tid; j < cnt; j += BLOCK) {
          const uint32_t s = expand(j, cm, cv);
          const unsigned long long e = (e0 + tb[s & 127] + tb[128 + ((s >> 7) & 127)]) & M34;
          if (e == 0) continue;
          double2 w = dtab[e >> DYADIC_HALF];
          const unsigned long long lo = e & LOMASK;
          if (lo) {
            const double2 wl = dtab[(1u << DYADIC_HALF) + lo];
            w = cmul(w, wl.x, wl.y);
          }
          sm[s] = cmul(sm[s], w.x, w.y);
        }
        break;
      }
      if (tid <= MAX_TILE_BITS) dp_c[tid] = 0;
      if (tid == 0) {
        dp_e0 = 0;
        dp_nonlin = 0;
      }
      __syncthreads();
      for (int f = tid; f < nf; f += BLOCK) {
        const uint64_t loc = (uint64_t)__double_as_longlong(F[4 * f]);
        const uint64_t gm = (uint64_t)__double_as_longlong(F[4 * f + 1]);
        const uint64_t gv = (uint64_t)__double_as_longlong(F[4 * f + 2]);
        const unsigned long long w = (unsigned long long)__double_as_longlong(F[4 * f + 3]);
        if ((base & gm) != gv) continue;                 // factor off for this tile
        const uint32_t lm = (uint32_t)loc & ~cm, lv = (uint32_t)(loc >> 32);
        if (lm == 0) {
          atomicAdd(&dp_e0, w);
        } else if ((lm & (lm - 1)) == 0) {
          const int b = __ffs(lm) - 1;
          if (lv & lm) {
            atomicAdd(&dp_c[b], w);
          } else {                                      // w (1 - s_b)
            atomicAdd(&dp_e0, w);
            atomicAdd(&dp_c[b], ((1ull << DYADIC_BITS) - w) & M34);
          }
        } else {
          dp_nonlin = 1;
        }
      }
      __syncthreads();
      if (!dp_nonlin) {
        for (uint32_t v = tid; v < 256; v += BLOCK) {
          const int c = v >> 7;
          unsigned long long e = 0;
          for (int b = 0; b < 7; b++)
            if (((v & 127) >> b) & 1 && 7 * c + b <= MAX_TILE_BITS) e += dp_c[7 * c + b];
          dp_t[c][v & 127] = e;
        }
        __syncthreads();
        const unsigned long long e0 = dp_e0;
        for (uint32_t j = tid; j < cnt; j += BLOCK) {
          const uint32_t s = expand(j, cm, cv);
          const unsigned long long e = (e0 + dp_t[0][s & 127] + dp_t[1][(s >> 7) & 127]) & M34;
          if (e == 0) continue;
          double2 w = dtab[e >> DYADIC_HALF];
          const unsigned long long lo = e & LOMASK;
          if (lo) {
            const double2 wl = dtab[(1u << DYADIC_HALF) + lo];
            w = cmul(w, wl.x, wl.y);
          }
          sm[s] = cmul(sm[s], w.x, w.y);
        }
      } else {
        for (uint32_t j = tid; j < cnt; j += BLOCK) {
          const uint32_t s = expand(j, cm, cv);
          unsigned long long e = 0;
          for (int f = 0; f < nf; f++) {
            const uint64_t loc = (uint64_t)__double_as_longlong(F[4 * f]);
            const uint64_t gm = (uint64_t)__double_as_longlong(F[4 * f + 1]);
            const uint64_t gv = (uint64_t)__double_as_longlong(F[4 * f + 2]);
            if ((s & (uint32_t)loc) == (uint32_t)(loc >> 32) && (base & gm) == gv)
              e += (unsigned long long)__double_as_longlong(F[4 * f + 3]);
          }
          e &= M34;
          if (e == 0) continue;
          double2 w = dtab[e >> DYADIC_HALF];
          const unsigned long long lo = e & LOMASK;
          if (lo) {
            const double2 wl = dtab[(1u << DYADIC_HALF) + lo];
            w = cmul(w, wl.x, wl.y);
          }
          sm[s] = cmul(sm[s], w.x, w.y);
        }
      }
      break;
    }
    case OP_LPHASE: {
      if ((op.mode & LP_TABLE) && tabs && tabs->ltab) {
        const double2* __restrict__ ltab = tabs->ltab;
        diag_apply<BLOCK, 4>(sm, T >> __popc(cm), cm, cv, [&](uint32_t s, double2 v) {
          const double2 w = ltab[s];
          return cmul(v, w.x, w.y);
        });
        break;
      }
      // phase(s) = prod_f w_f^[cond_f(s)] with one condition bit per factor:
      // per tile, e0 = product of the factors decided by CTA bits and, per
      // tile bit b, c_b = product of the factors on b (a factor that needs
      // s_b = 0 contributes w to e0 and conj(w) to c_b); then two 7-bit
      // tables of products (built by doubling, e0 folded into the first)
      // give phase(s) = t0[s & 127] * t1[s >> 7].
      __shared__ double2 lp_c[MAX_TILE_BITS + 1];
      double2(*lp_t)[128] = op_tab;
      const int nf = (int)op.x_loc;
      const double* F = coef + op.cidx;
      const int k = 31 - __clz(T);
      if (tid <= (uint32_t)k) {
        // thread b < k builds c_b; thread k builds e0
        double cr = 1, ci = 0;
        for (int f = 0; f < nf; f++) {
          const double* Ff = F + LPHASE_FAC * f;
          const uint64_t loc = (uint64_t)__double_as_longlong(Ff[0]);
          const uint64_t gm = (uint64_t)__double_as_longlong(Ff[1]);
          const uint64_t gv = (uint64_t)__double_as_longlong(Ff[2]);
          const uint32_t lm = (uint32_t)loc;
          uint32_t lv = (uint32_t)(loc >> 32);
          if (gv & kLphaseParity) {
            // parity factor: w where popcount(idx & mask) is odd, i.e. where
            // the tile bit (if any) differs from the parity of the CTA bits
            const uint32_t pg = (uint32_t)__popcll(base & gm) & 1u;
            if (lm == 0) {
              if (!pg) continue;
            } else {
              lv = pg ? 0u : lm;
            }
          } else if ((base & gm) != gv) {
            continue;
          }
          double wr = Ff[3], wi = Ff[4];
          if (pt && (int)__double_as_longlong(Ff[5]) == pt->gate) {   // shifted circuit
            wr = pt->a0;
            wi = pt->b0;
          }
          if (lm == 0) {
            if (tid != (uint32_t)k) continue;
          } else {
            const int b = __ffs(lm) - 1;
            if (tid == (uint32_t)k) {
              if (lv & lm) continue;         // e0 takes w of the s_b = 0 factors
            } else {
              if (b != (int)tid) continue;
              if (!(lv & lm)) wi = -wi;      // conj(w) on s_b = 1
            }
          }
          const double nr = fma(cr, wr, -ci * wi), ni = fma(cr, wi, ci * wr);
          cr = nr;
          ci = ni;
        }
        lp_c[tid] = make_double2(cr, ci);
      }
      __syncthreads();
      if (tid < 2) lp_t[tid][0] = tid == 0 ? lp_c[k] : make_double2(1.0, 0.0);
      __syncthreads();
      for (int r = 0; r < 7; r++) {
        for (uint32_t v = tid; v < 2u << r; v += BLOCK) {
          const int c = v >> r, lo = v & ((1u << r) - 1u);
          const int b = 7 * c + r;
          if (b < k) {
            const double2 x = lp_t[c][lo], y = lp_c[b];
            lp_t[c][lo | (1u << r)] = cmul(x, y.x, y.y);
          }
        }
        __syncthreads();
      }
      const uint32_t cnt = T >> __popc(cm);
      for (uint32_t j = tid; j < cnt; j += BLOCK) {
        const uint32_t s = expand(j, cm, cv);
        double2 w = lp_t[0][s & 127];
        if (k > 7) {
          const double2 w1 = lp_t[1][(s >> 7) & 127];
          w = cmul(w, w1.x, w1.y);
        }
        sm[s] = cmul(sm[s], w.x, w.y);
        if (sm2) sm2[s] = cmul(sm2[s], w.x, w.y);
      }
      break;
    }
    case OP_SCALE: {
      const double wr = op.a, wi = op.b;
      if (op.mode & 1) {
        diag_apply<BLOCK, 4>(sm, T, 0, 0,
                             [&](uint32_t, double2 v) { return make_double2(v.x * wr, v.y * wr); });
      } else {
        diag_apply<BLOCK, 4>(sm, T, 0, 0, [&](uint32_t, double2 v) { return cmul(v, wr, wi); });
      }
      break;
    }
    default:
      break;
  }
}

}  // namespace lq
