// lq_expval.cu -- tiled Pauli-sum expectation value E = sum_t c_t <psi|P_t|psi>
// (Sec. V, the observable of Eq. expval; Sec. VI's Hamiltonians) for large
// states.
//
// P_t |i> = i^{k0} (-1)^{popcount(i & z)} |i ^ x> (x: X and Y sites, z: Z and
// Y sites, k0 = number of Y factors), so a term with x != 0 pairs amplitude i
// with j = i ^ x and contributes 2 c_t Re(i^kk conj(psi_i) psi_j) per
// unordered pair (i has the top bit of x clear), kk = k0 + 2 parity(j & z);
// a diagonal term (x = 0) contributes c_t (-1)^{popcount(i & z)} |psi_i|^2.
//
// Terms are grouped by x.  The state is read in tile passes: a pass loads
// each 2^k-amplitude tile (bit set = the low m bits and bits covering the x
// masks of the pass's groups) into shared memory once, and every group of the
// pass is evaluated on the tile's pairs.  A group's per-pair coefficient
// depends on the parities of j & z_t:
//   * class mode (every z_t inside x, w = |x| <= 3 bits): the coefficient is
//     a function of the pair's lower x bits ("class", 2^{w-1} of them);
//     threads are split by class, each accumulates sum Re / Im of
//     conj(psi_i) psi_j over its pairs (2 FP64 FMAs per pair and part) and
//     folds its class coefficient in once per tile;
//   * table mode (up to 4 terms): the parities index a host-built table of
//     (coefficient of Re, coefficient of Im), one FMA per pair and part;
//   * the diagonal group sums |psi_i|^2 d(i) with d from per-CTA 8-bit chunk
//     tables over the global index (terms spanning chunks: directly).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <vector>

#include "lq_device.cuh"
#include "lq_internal.h"
#include "lq_kernels.h"
#include "lq_xplan.cuh"

namespace lq {

// ------------------------------------------------------------ host plan

static uint32_t xp_to_local(uint64_t mask, const int* pos) {
  uint32_t r = 0;
  while (mask) {
    const int b = __builtin_ctzll(mask);
    mask &= mask - 1;
    r |= 1u << pos[b];
  }
  return r;
}

static int pc64(uint64_t v) { return __builtin_popcountll(v); }

int build_xplans(int n, const lq_pauli_term* terms, int nt, int kt, std::vector<XPlan>& out,
                 std::vector<lq_pauli_term>& wide) {
  out.clear();
  wide.clear();
  if (kt > XP_TILE_BITS) kt = XP_TILE_BITS;
  const int k = n < kt ? n : kt;
  const int m0 = n < XP_LOW_BITS ? n : XP_LOW_BITS;
  const uint64_t low = (1ull << m0) - 1ull;

  // groups by X mask; groups with x != 0 that cannot use class mode are split
  // into table-mode groups of <= XP_TABLE_TERMS terms
  struct HG {
    uint64_t x;
    std::vector<int> t;
    int mode;
  };
  std::map<uint64_t, std::vector<int>> byx;
  for (int t = 0; t < nt; t++) byx[terms[t].xmask].push_back(t);
  std::vector<HG> groups;
  HG diag{0, {}, XG_DIAG};
  for (auto& kv : byx) {
    if (kv.first == 0) {
      diag.t = kv.second;
      continue;
    }
    if (pc64(kv.first | low) > k) {   // X mask wider than a tile: untiled kernel
      for (int t : kv.second) wide.push_back(terms[t]);
      continue;
    }
    bool cls = pc64(kv.first) <= 3;
    for (int t : kv.second)
      if (terms[t].zmask & ~kv.first) cls = false;
    if (cls) {   // class groups of the same mask add up: split long term lists
      for (std::size_t a = 0; a < kv.second.size(); a += XP_CLASS_TERMS) {
        HG g{kv.first, {}, XG_CLASS};
        for (std::size_t b = a; b < kv.second.size() && b < a + XP_CLASS_TERMS; b++)
          g.t.push_back(kv.second[b]);
        groups.push_back(g);
      }
    } else {
      for (std::size_t a = 0; a < kv.second.size(); a += XP_TABLE_TERMS) {
        HG g{kv.first, {}, XG_TABLE};
        for (std::size_t b = a; b < kv.second.size() && b < a + XP_TABLE_TERMS; b++)
          g.t.push_back(kv.second[b]);
        groups.push_back(g);
      }
    }
  }
  // a diagonal group too long for one plan goes to the untiled kernel
  if ((int)diag.t.size() > XP_MAX_TERMS / 2) {
    for (int t : diag.t) wide.push_back(terms[t]);
    diag.t.clear();
  }
  // what a group takes of an XPlan's groups, terms and coefficients
  auto coefs = [](const HG& G) {
    return G.mode == XG_CLASS ? 1 << (pc64(G.x) - 1)
                              : G.mode == XG_TABLE ? 1 << (int)G.t.size() : 0;
  };
  // passes: greedy, groups in ascending x, each pass within one XPlan's
  // capacity (a small state's tile holds every mask, so the tile bits alone
  // would put all groups into one pass)
  struct HP {
    uint64_t tile;
    std::vector<int> g;   // indices into groups; -1 = the diagonal group
  };
  std::vector<HP> passes;
  std::vector<int> pending;
  for (int g = 0; g < (int)groups.size(); g++) pending.push_back(g);
  if (!diag.t.empty()) passes.push_back(HP{low, {-1}});
  while (!pending.empty()) {
    HP P{low, {}};
    int ng = 0, ntm = 0, nco = 0;
    if (passes.size() == 1 && passes[0].g.size() == 1 && passes[0].g[0] == -1) {
      P = passes[0];   // the diagonal group shares the first pass
      passes.clear();
      ng = 1;
      ntm = (int)diag.t.size();
    }
    std::vector<int> rest;
    for (int g : pending) {
      const uint64_t t = P.tile | groups[g].x;
      const int tg = (int)groups[g].t.size(), cg = coefs(groups[g]);
      if (pc64(t) <= k && ng + 1 <= XP_MAX_GROUPS && ntm + tg <= XP_MAX_TERMS &&
          nco + cg <= XP_MAX_COEF) {
        P.tile = t;
        P.g.push_back(g);
        ng++;
        ntm += tg;
        nco += cg;
      } else {
        rest.push_back(g);
      }
    }
    if (P.g.empty()) return -1;   // cannot happen: every group fits a tile with the low bits
    passes.push_back(P);
    pending.swap(rest);
  }

  // fill XPlan chunks
  auto fresh = [&]() {
    out.emplace_back();
    XPlan& X = out.back();
    std::memset(&X, 0, sizeof X);
    X.n = n;
    X.diag = -1;
    return &out.back();
  };
  XPlan* X = fresh();
  for (const HP& P : passes) {
    // capacity of this pass: groups, terms and coefficients
    int ng = 0, ntm = 0, nco = 0;
    for (int g : P.g) {
      const HG& G = g < 0 ? diag : groups[g];
      ng++;
      ntm += (int)G.t.size();
      if (G.mode == XG_CLASS) nco += 1 << (pc64(G.x) - 1);
      if (G.mode == XG_TABLE) nco += 1 << G.t.size();
    }
    if (ng > XP_MAX_GROUPS || ntm > XP_MAX_TERMS || nco > XP_MAX_COEF) return -1;
    if (X->npass == XP_MAX_PASS || X->ngroups + ng > XP_MAX_GROUPS ||
        X->nterms + ntm > XP_MAX_TERMS || X->ncoef + nco > XP_MAX_COEF)
      X = fresh();
    XPass& Q = X->passes[X->npass++];
    uint64_t tile = P.tile;
    for (int bit = 0; bit < n && pc64(tile) < k; bit++) tile |= 1ull << bit;
    int pos[64];
    for (int i = 0; i < 64; i++) pos[i] = -1;
    int j = 0, o = 0;
    for (int bit = 0; bit < n; bit++) {
      if (tile >> bit & 1) {
        Q.tbits[j] = (int8_t)bit;
        pos[bit] = j++;
      } else {
        Q.obits[o++] = (int8_t)bit;
      }
    }
    int mm = 0;
    while (mm < k && Q.tbits[mm] == mm) mm++;
    Q.k = k;
    Q.m = mm;
    Q.nobits = o;
    Q.g0 = X->ngroups;
    for (int g : P.g) {
      const HG& G = g < 0 ? diag : groups[g];
      XGroup& D = X->groups[X->ngroups++];
      D.mode = (int8_t)G.mode;
      D.x = xp_to_local(G.x, pos);
      D.h = (int8_t)(G.x ? 31 - __builtin_clz(D.x) : 0);
      D.w = (int8_t)pc64(G.x);
      D.first = (int16_t)X->nterms;
      D.count = (int16_t)G.t.size();
      // diagonal group: terms inside one 8-bit index chunk (read from the
      // chunk tables) first, then the terms evaluated directly
      auto in_chunk = [&](int t) {
        const uint64_t z = terms[t].zmask;
        if (!z) return false;
        return __builtin_ctzll(z) / EXP_CHUNK_BITS == (63 - __builtin_clzll(z)) / EXP_CHUNK_BITS;
      };
      std::vector<int> order(G.t);
      // diagonal group: a few distinct coefficients (the ZZ couplings of a
      // chain) are cheaper as classes -- K - 1 adds per amplitude after a
      // table lookup each -- than chunk lookups plus direct terms
      std::vector<double> cls;
      bool classes = false;
      if (G.mode == XG_DIAG) {
        int chunks = 0, direct = 0;
        uint32_t used = 0;
        for (int t : order) {
          bool found = false;
          for (double c : cls) found |= c == terms[t].coeff;
          if (!found) cls.push_back(terms[t].coeff);
          if (in_chunk(t)) {
            const uint32_t cb = 1u << (__builtin_ctzll(terms[t].zmask) / EXP_CHUNK_BITS);
            chunks += (used & cb) == 0;
            used |= cb;
          } else if (terms[t].zmask) {
            direct++;
          }
        }
        classes = (int)cls.size() <= XP_DIAG_CLASSES && (int)cls.size() - 1 < chunks + direct &&
                  X->dcls == 0;
      }
      if (classes) {
        // per class: two-bit terms (b, b + delta) and one-bit terms (b,
        // delta 0) join a delta group while their low bit is new to it (at
        // most XP_DIAG_DELTAS groups); the others are counted one by one and
        // come first in the class
        std::vector<int> sorted;
        int at = D.first;
        for (std::size_t c = 0; c < cls.size(); c++) {
          std::vector<int> direct, paired;
          int nd = 0;
          int8_t del[XP_DIAG_DELTAS] = {0, 0};
          uint64_t msk[XP_DIAG_DELTAS] = {0, 0};
          for (int t : order) {
            if (terms[t].coeff != cls[c]) continue;
            const uint64_t z = terms[t].zmask;
            bool joined = false;
            if (pc64(z) == 2 || pc64(z) == 1) {   // delta 0: one-bit terms
              const int lo = __builtin_ctzll(z), dl = 63 - __builtin_clzll(z) - lo;
              for (int e = 0; e < nd && !joined; e++)
                if (del[e] == dl && !(msk[e] >> lo & 1)) {
                  msk[e] |= 1ull << lo;
                  joined = true;
                }
              if (!joined && nd < XP_DIAG_DELTAS) {
                del[nd] = (int8_t)dl;
                msk[nd++] = 1ull << lo;
                joined = true;
              }
            }
            (joined ? paired : direct).push_back(t);
          }
          X->dfirst[c] = (int16_t)at;
          X->dcount[c] = (int16_t)(direct.size() + paired.size());
          X->ddirect[c] = (int16_t)direct.size();
          X->dnd[c] = (int8_t)nd;
          for (int e = 0; e < XP_DIAG_DELTAS; e++) {
            X->ddel[c][e] = del[e];
            X->dmsk[c][e] = msk[e];
          }
          at += X->dcount[c];
          sorted.insert(sorted.end(), direct.begin(), direct.end());
          sorted.insert(sorted.end(), paired.begin(), paired.end());
        }
        order.swap(sorted);
        X->dcls = (int32_t)cls.size();
      } else if (G.mode == XG_DIAG) {
        std::stable_partition(order.begin(), order.end(), in_chunk);
      }
      D.direct = D.first;
      int odd = 0, even = 0;
      for (int t : order) {
        XTerm& T = X->terms[X->nterms++];
        const lq_pauli_term& src = terms[t];
        T.c = G.mode == XG_DIAG ? src.coeff : 2.0 * src.coeff;
        if (G.mode == XG_DIAG) {   // diagonal terms: the full global Z mask
          T.zl = 0;
          T.zg = src.zmask;
        } else {
          T.zl = xp_to_local(src.zmask & tile, pos);
          T.zg = src.zmask & ~tile;
        }
        T.k0 = pc64(src.xmask & src.zmask) & 3;
        T.chunk = 0;
        if (G.mode == XG_DIAG && src.zmask && !classes) {
          const int lo = __builtin_ctzll(src.zmask), hi = 63 - __builtin_clzll(src.zmask);
          if (lo / EXP_CHUNK_BITS == hi / EXP_CHUNK_BITS) T.chunk = 1 + lo / EXP_CHUNK_BITS;
        }
        if (T.chunk) D.direct = (int16_t)X->nterms;
        (T.k0 & 1 ? odd : even)++;
      }
      D.part = (int8_t)(G.mode == XG_DIAG ? 0 : odd == 0 ? 1 : even == 0 ? 2 : 0);
      D.coef = (int16_t)X->ncoef;
      // Re(i^kk v) = vr, -vi, -vr, vi for kk = 0..3: coefficient of vr and of vi
      auto add = [](double2& C, int kk, double c2) {
        switch (kk & 3) {
          case 0: C.x += c2; break;
          case 1: C.y -= c2; break;
          case 2: C.x -= c2; break;
          default: C.y += c2; break;
        }
      };
      if (G.mode == XG_CLASS) {
        // class c: the lower x bits of i are deposit(c); j = i ^ x
        const int W = pc64(G.x) - 1;
        const uint64_t xlo = G.x & ~(1ull << (63 - __builtin_clzll(G.x)));
        for (int c = 0; c < (1 << W); c++) {
          uint64_t dep = 0, mk = xlo;
          for (int b = 0; mk; b++) {
            const int bit = __builtin_ctzll(mk);
            mk &= mk - 1;
            if (c >> b & 1) dep |= 1ull << bit;
          }
          const uint64_t jx = dep ^ G.x;
          double2 C = make_double2(0.0, 0.0);
          for (int q = D.first; q < D.first + D.count; q++) {
            const lq_pauli_term& src = terms[order[q - D.first]];
            add(C, X->terms[q].k0 + 2 * (pc64(jx & src.zmask) & 1), X->terms[q].c);
          }
          X->coef[X->ncoef++] = C;
        }
        // an earlier class group of this plan with the same width, part
        // and coefficients: share its block, so that the kernel adds both
        // groups' class sums before applying the coefficients once
        const int nc = 1 << W;
        for (int e = 0; e < X->ngroups - 1; e++) {
          const XGroup& E = X->groups[e];
          if (E.mode != XG_CLASS || E.w != D.w || E.part != D.part) continue;
          bool same = true;
          for (int c = 0; c < nc && same; c++)
            same = X->coef[E.coef + c].x == X->coef[D.coef + c].x &&
                   X->coef[E.coef + c].y == X->coef[D.coef + c].y;
          if (same) {
            X->ncoef -= nc;
            D.coef = E.coef;
            break;
          }
        }
      } else if (G.mode == XG_TABLE) {
        // index bit t = parity(j & z_t)
        for (int idx = 0; idx < (1 << D.count); idx++) {
          double2 C = make_double2(0.0, 0.0);
          for (int q = 0; q < D.count; q++)
            add(C, X->terms[D.first + q].k0 + 2 * (idx >> q & 1), X->terms[D.first + q].c);
          X->coef[X->ncoef++] = C;
        }
      }
      if (G.mode == XG_DIAG) {
        X->diag = X->ngroups - 1;
        for (int q = D.first; q < D.first + D.count; q++)
          if (X->terms[q].chunk) X->tables = 1;
      }
    }
    Q.g1 = X->ngroups;
  }
  return (int)out.size();
}

// ---------------------------------------------------------------- kernel

// One CTA walks the tiles t = blockIdx.x, blockIdx.x + gridDim.x, ... of every
// pass of the plan (state blockIdx.y) and writes its partial sum.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, 4) expval_tile_kernel(const __grid_constant__ XPlan X,
                                                               const double2* __restrict__ states,
                                                               uint64_t stride,
                                                               double* __restrict__ partial) {
  // dynamic shared memory: the tile, then the coefficient table, then the
  // diagonal chunk tables
  extern __shared__ double2 xsm[];
  // global offsets (>> m) of the tile bits above the low run: off(j) =
  // hlo[j & 31] | hhi[j >> 5] (k - m <= XP_TILE_BITS - XP_LOW_BITS = 10 bits)
  __shared__ uint32_t hlo[32], hhi[1 << (XP_TILE_BITS - XP_LOW_BITS - 5)];
  __shared__ double red[BLOCK / 32];
  const uint32_t tid = threadIdx.x;
  const double2* __restrict__ st = states + blockIdx.y * stride;
  const int n = X.n;
  const uint32_t Tmax = X.npass ? 1u << X.passes[0].k : 0u;
  double2* coef = xsm + Tmax;
  double* tab = reinterpret_cast<double*>(coef + X.ncoef);
  for (int e = tid; e < X.ncoef; e += BLOCK) coef[e] = X.coef[e];
  xp_tables<BLOCK>(X, tab);
  double acc = 0.0;
  for (int p = 0; p < X.npass; p++) {
    const XPass& Q = X.passes[p];
    const int k = Q.k, m = Q.m;
    const uint32_t T = 1u << k, lowmask = (1u << m) - 1u;
    __syncthreads();
    xp_offsets(Q, hlo, hhi);
    __syncthreads();
    const uint64_t ntiles = 1ull << (n - k);
    for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
      const uint64_t base = deposit(t, Q.obits, Q.nobits);
      // the next tile of this pass (same tile index, its CTA bits) into L2:
      // one hint per run of 2^m amplitudes, at most one per 128-byte line
      const int64_t ahead =
          t + gridDim.x < ntiles ? (int64_t)(deposit(t + gridDim.x, Q.obits, Q.nobits) - base) : 0;
      const uint32_t pmask = ahead ? (1u << (m < 3 ? m : 3)) - 1u : ~0u;
      for (uint32_t s = tid; s < T; s += BLOCK) {
        const double2* src =
            st + (base | ((uint64_t)(hlo[(s >> m) & 31u] | hhi[(s >> m) >> 5]) << m) | (s & lowmask));
        xsm[s] = *src;
        if ((s & pmask) == 0) prefetch_l2(src + ahead);
      }
      __syncthreads();
      acc += xp_tile<BLOCK>(xsm, T, X, Q, base, hlo, hhi, coef, tab);
      __syncthreads();
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((tid & 31) == 0) red[tid >> 5] = acc;
  __syncthreads();
  if (tid == 0) {
    double s = 0;
    for (int w = 0; w < BLOCK / 32; w++) s += red[w];
    partial[blockIdx.y * gridDim.x + blockIdx.x] = s;
  }
}

static constexpr int kXBlock = 256;

cudaError_t launch_expval_tiled(const XPlan& X, const double2* states, uint64_t stride,
                                int nstates, double* partial, double* out, int accumulate,
                                cudaStream_t s) {
  (void)cudaGetLastError();  // report only this launcher's own errors
  const int k = X.npass ? X.passes[0].k : 0;
  const int nch = (X.n + EXP_CHUNK_BITS - 1) / EXP_CHUNK_BITS;
  int ctab = 0;   // class tables of the diagonal group
  for (int c = 0; c < X.dcls; c++) ctab += X.dcount[c] + 1;
  const size_t smem = (sizeof(double2) << k) + sizeof(double2) * X.ncoef +
                      (X.tables ? sizeof(double) * 256 * nch : 0) + sizeof(double) * ctab;
  static std::atomic<uint64_t> configured{0};
  cudaError_t ce = once_per_device(configured, [] {
    return cudaFuncSetAttribute(
        expval_tile_kernel<kXBlock>, cudaFuncAttributeMaxDynamicSharedMemorySize,
        (int)((sizeof(double2) << XP_TILE_BITS) + sizeof(double2) * XP_MAX_COEF +
              sizeof(double) * 256 * ((34 + EXP_CHUNK_BITS - 1) / EXP_CHUNK_BITS)));
  });
  if (ce != cudaSuccess) return ce;
  // one wave of resident CTAs (the launch bound allows 4 per SM; shared
  // memory, with ~1.5 KiB static and 1 KiB reserved, may allow fewer)
  int per_sm = (int)((228u << 10) / (smem + (3u << 10)));
  per_sm = per_sm < 1 ? 1 : per_sm > 4 ? 4 : per_sm;
  int gx = expval_grid(X.n);
  if (gx > sm_count() * per_sm) gx = sm_count() * per_sm;
  dim3 grid(gx, nstates);
  expval_tile_kernel<kXBlock><<<grid, kXBlock, smem, s>>>(X, states, stride, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_sum_partials(partial, gx, nstates, out, accumulate, s);
}

}  // namespace lq
