// lq_qft.cu -- the QFT of Sec. IV-B on the dense state, in FFT form (Alg. 2)
// and gate form (Alg. 3).
//
// FFT form.  QFT|x> = N^{-1/2} sum_k e^{2 pi i x k/N}|k> is the unitary inverse
// DFT.  Reading Alg. 3 per target qubit j: the controlled phases CP(pi/2^{j-q})
// from every earlier qubit q < j are applied before H(j), so stage j is a
// decimation-in-time butterfly on bit p = n-1-j,
//     (a, b) -> (a + w_j b, a - w_j b),   w_j = exp(2 pi i M_j / 2^{j+1}),
//     M_j = sum_{q<j} b_q 2^q   (b_q = bit n-1-q of the index),
// with 1/sqrt2 per stage deferred to one final scale, followed by the bit
// reversal of the index (the SWAPs).  Stages are grouped into shared-memory
// passes over d consecutive qubits [q0, q1).  Inside a pass the twiddle factors
// into a per-tile constant part (qubits q < q0 are fixed for the tile) and a
// local part that depends only on in-tile bits; the constant parts of all d
// stages commute to the start of the pass and form one diagonal
//     D(V) = exp(2 pi i M_out V / 2^{q1}),  V = the group's bits as an integer,
// applied by one table lookup and one complex multiply per amplitude
// (four-step FFT).  Local twiddles come from a constant table in tangent form
// (c, t = s/c) or cotangent form (s, u = c/s), so each butterfly costs
// 6 FP64 FMAs: b' = b + i t b (2), a +- c b' (4).
//
// Radix 4.  Stages r and r + 1 of a pass act on local bits p and p - 1; on a
// quad x_ab (a = bit p, b = bit p - 1, v = the in-tile bits above p,
// theta = pi bitrev_r(v) / 2^{r+1}) stage r's twiddle is W1 = e^{2 i theta}
// and stage r + 1's is W2 = e^{i theta} where a = 0 and i W2 where a = 1, so
//   z_00, z_01 = (x00 + W1 x10) +- (W2 x01 + W3 x11),
//   z_10, z_11 = (x00 - W1 x10) +- i (W2 x01 - W3 x11),   W3 = W1 W2,
// the classic radix-4 step.  With each W = c (1 + i sigma) applied to x or
// to i x (2 FMAs) and c1, c2, rho = c3 / c2 folded into the sums, a quad
// costs 22 FMAs instead of the 24 of two radix-2 stages, and one
// shared-memory round trip instead of two.  A pass's first two stages have
// unit twiddles (16 adds per quad); an odd last stage runs radix 2.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "lq_device.cuh"
#include "lq_internal.h"
#include "lq_kernels.h"

namespace lq {

constexpr int FFT_MAX_D = 12;                     // qubits per pass
constexpr int FFT_FULL_DIAG = 10;                 // largest group with a 2^d diagonal table
constexpr int FFT_TABLE = (1 << FFT_MAX_D) - 1;   // sum_{r<12} 2^r entries

// g_tw[(1 << r) - 1 + v]: twiddle w = exp(2 pi i u / 2^{r+1}) = exp(i pi u /
// 2^r) of the stage with r in-tile higher qubits, u = bit-reverse_r(v), as
// (scale, sigma): tangent form (scale c, sigma = -s/c) when the top two bits of
// u are equal (angle in [0, pi/4) or [3pi/4, pi), |sigma| <= 1), otherwise
// cotangent form (scale s, sigma = c/s).  The top bits of u are the low bits
// of v, so the form is cot(v) = (v ^ (v >> 1)) & 1.
__device__ double2 g_tw[FFT_TABLE];

__global__ void fft_table_kernel() {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= FFT_TABLE) return;
  int r = 31 - __clz(idx + 1);
  int v = idx + 1 - (1 << r);
  int u = r ? (int)(__brev((unsigned)v) >> (32 - r)) : 0;
  double s, c;
  sincospi((double)u / (double)(1 << r), &s, &c);
  const bool cot = ((v ^ (v >> 1)) & 1) != 0;
  g_tw[idx] = cot ? make_double2(s, c / s) : make_double2(c, -s / c);
}



// The twiddle table is filled once per device and complete before this
// returns (fill_table_once), whichever thread or stream asks first.
// g_tw4[3 ((1 << r) - 2 + v) + {0, 1, 2}]: the radix-4 twiddles of stages
// (r, r + 1), r = 1 .. FFT_MAX_D - 2, for the in-tile bits v above stage r's
// bit: (c1, sigma1) of W1, (c2, sigma2) of W2, (rho = c3 / c2, sigma3) of W3,
// W3's sign (e^{3 i theta} = -e^{i (3 theta - pi)} when 3 theta >= pi) in c3.
// With N = 2^{r+1} and u = bitrev_r(v) the angles are pi a / N for a = 2u, u
// and 3u mod N; a twiddle is in cotangent form (scale sin, sigma = -cot) when
// a lies in [N/4, 3N/4), else in tangent form (scale cos, sigma = tan), so
// |sigma| <= 1 and |scale| >= 1/sqrt2 (|rho| in [1/sqrt2, sqrt2]).
constexpr int FFT4_ENTRIES = (2 << (FFT_MAX_D - 2)) - 2;   // sum_{r=1}^{10} 2^r
__device__ double2 g_tw4[3 * FFT4_ENTRIES];

__host__ __device__ __forceinline__ bool fft4_cot(uint32_t a, uint32_t N) {
  return ((a + 3u * (N >> 2)) & (N - 1u)) < (N >> 1);
}

__global__ void fft4_table_kernel() {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= FFT4_ENTRIES) return;
  const int r = 31 - __clz(idx + 2);
  const uint32_t v = (uint32_t)(idx + 2 - (1 << r));
  const uint32_t u = __brev(v) >> (32 - r), N = 2u << r;
  auto form = [&](uint32_t a, double* scale, double* sig) {
    double sn, cs;
    sincospi((double)a / (double)N, &sn, &cs);
    if (fft4_cot(a, N)) {
      *scale = sn;
      *sig = -cs / sn;
    } else {
      *scale = cs;
      *sig = sn / cs;
    }
  };
  double c1, s1, c2, s2, c3, s3;
  form(2u * u, &c1, &s1);
  form(u, &c2, &s2);
  form((3u * u) & (N - 1u), &c3, &s3);
  if (3u * u >= N) c3 = -c3;
  g_tw4[3 * idx] = make_double2(c1, s1);
  g_tw4[3 * idx + 1] = make_double2(c2, s2);
  g_tw4[3 * idx + 2] = make_double2(c3 / c2, s3);
}

static cudaError_t fill_fft_table(cudaStream_t ps) {
  fft_table_kernel<<<(FFT_TABLE + 255) / 256, 256, 0, ps>>>();
  fft4_table_kernel<<<(FFT4_ENTRIES + 255) / 256, 256, 0, ps>>>();
  return cudaGetLastError();
}

cudaError_t fft_tables_init(cudaStream_t s) {
  (void)cudaGetLastError();  // report only this launcher's own errors
  static TableOnce once;
  return fill_table_once(once, &s, fill_fft_table);
}

struct FftParams {
  int n, q0, q1, d, ms, plo, k;
  int inverse;
  int scaled;     // scale != 1 (decided on the host: no per-tile FP64 compare)
  double scale;   // folded into the diagonal (or applied alone)
};

// Scaled radix-2 butterfly (a, b) -> (a + w b, a - w b), w = scale (1 + i
// sigma) applied to b (tangent form) or to i b (cotangent form; -i b for the
// inverse, whose twiddles are conjugated): with (p, q) = b or +-i b,
// b' = (p + sigma q, q - sigma p) and out = a +- scale b' -- 6 FP64 FMAs, no
// branch.  fpos/fneg: sign masks (inverse: flip sigma and pick -i b).
__device__ __forceinline__ void fft_bfly(double2& a, double2& b, double2 w, uint32_t v,
                                         uint32_t fpos, uint32_t fneg) {
  const bool cot = ((v ^ (v >> 1)) & 1u) != 0;
  const double p = cot ? xsign(b.y, fneg) : b.x;
  const double q = cot ? xsign(b.x, fpos) : b.y;
  const double sg = xsign(w.y, fpos);
  const double tr = fma(sg, q, p), ti = fma(-sg, p, q);
  b = make_double2(fma(-w.x, tr, a.x), fma(-w.x, ti, a.y));
  a = make_double2(fma(w.x, tr, a.x), fma(w.x, ti, a.y));
}

// x' with W x = scale x': W = scale (1 + i sigma) applied to x (tangent
// form) or to i x (cotangent form); the inverse transform takes conj(W)
// (sign masks fpos, fneg as in fft_bfly).  2 FMAs.
__device__ __forceinline__ double2 fft4_rot(double2 x, double sig, bool cot, uint32_t fpos,
                                            uint32_t fneg) {
  const double p = cot ? xsign(x.y, fneg) : x.x;
  const double q = cot ? xsign(x.x, fpos) : x.y;
  const double sg = xsign(sig, fpos);
  return make_double2(fma(-sg, q, p), fma(sg, p, q));
}

// A pass's first two stages (local bits lp and lp - 1; unit twiddles, and
// i on the second stage where bit lp is set): 16 adds per quad.
template <int BLOCK>
__device__ __forceinline__ void fft4_first(double2* __restrict__ sm, uint32_t T, int lp,
                                           uint32_t fpos, uint32_t fneg) {
  const uint32_t L = 1u << lp, H = L >> 1;
  for (uint32_t j = threadIdx.x; j < (T >> 2); j += BLOCK) {
    const uint32_t s = insert0(insert0(j, lp - 1), lp);
    const double2 x00 = sm[s], x01 = sm[s | H], x10 = sm[s | L], x11 = sm[s | L | H];
    const double2 A = make_double2(x00.x + x10.x, x00.y + x10.y);
    const double2 B = make_double2(x00.x - x10.x, x00.y - x10.y);
    const double2 F1 = make_double2(x01.x + x11.x, x01.y + x11.y);
    const double2 F2 = make_double2(x01.x - x11.x, x01.y - x11.y);
    const double ix = xsign(F2.y, fneg), iy = xsign(F2.x, fpos);   // (+-i) F2
    sm[s] = make_double2(A.x + F1.x, A.y + F1.y);
    sm[s | H] = make_double2(A.x - F1.x, A.y - F1.y);
    sm[s | L] = make_double2(B.x + ix, B.y + iy);
    sm[s | L | H] = make_double2(B.x - ix, B.y - iy);
  }
}

// Stages r and r + 1 (r >= 1) on local bits lp and lp - 1 as radix-4 steps
// with the g_tw4 twiddles of level r: 22 FMAs per quad.
template <int BLOCK>
__device__ __forceinline__ void fft4_step(double2* __restrict__ sm, uint32_t T, int lp, int r,
                                          uint32_t fpos, uint32_t fneg) {
  const uint32_t L = 1u << lp, H = L >> 1, N = 2u << r;
  const double2* __restrict__ t4 = g_tw4 + 3 * ((1 << r) - 2);
  for (uint32_t j = threadIdx.x; j < (T >> 2); j += BLOCK) {
    const uint32_t s = insert0(insert0(j, lp - 1), lp);
    const double2 x00 = sm[s], x01 = sm[s | H], x10 = sm[s | L], x11 = sm[s | L | H];
    const uint32_t v = s >> (lp + 1);
    const uint32_t u = __brev(v) >> (32 - r);
    const double2 e1 = t4[3 * v], e2 = t4[3 * v + 1], e3 = t4[3 * v + 2];
    const double2 a = fft4_rot(x10, e1.y, fft4_cot(2u * u, N), fpos, fneg);
    const double2 b = fft4_rot(x01, e2.y, fft4_cot(u, N), fpos, fneg);
    const double2 c = fft4_rot(x11, e3.y, fft4_cot(3u * u, N), fpos, fneg);
    const double c1 = e1.x, c2 = e2.x, rho = e3.x;
    const double2 A = make_double2(fma(c1, a.x, x00.x), fma(c1, a.y, x00.y));
    const double2 B = make_double2(fma(-c1, a.x, x00.x), fma(-c1, a.y, x00.y));
    const double2 F1 = make_double2(fma(rho, c.x, b.x), fma(rho, c.y, b.y));
    const double2 F2 = make_double2(fma(-rho, c.x, b.x), fma(-rho, c.y, b.y));
    const double cn = xsign(c2, fneg);   // B +- (+-i) c2 F2
    sm[s] = make_double2(fma(c2, F1.x, A.x), fma(c2, F1.y, A.y));
    sm[s | H] = make_double2(fma(-c2, F1.x, A.x), fma(-c2, F1.y, A.y));
    sm[s | L] = make_double2(fma(cn, F2.y, B.x), fma(-cn, F2.x, B.y));
    sm[s | L | H] = make_double2(fma(-cn, F2.y, B.x), fma(cn, F2.x, B.y));
  }
}

// One pass of the FFT form over the d qubits [q0, q1) (tile: those bits plus
// ms spectator low bits).  Two butterflies per thread and iteration, all four
// loads before any store.
template <int BLOCK, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) fft_pass_kernel(const FftParams F,
                                                               double2* __restrict__ state) {
  extern __shared__ double2 sm[];
  __shared__ double2 omega[FFT_MAX_D];
  const int k = F.k, ms = F.ms, d = F.d, plo = F.plo;
  const uint32_t T = 1u << k;
  // the diagonal's table after the tile: 2^d entries, or (groups of more
  // than FFT_FULL_DIAG qubits) two tables of 2^dl and 2^(d - dl)
  const bool split = d > FFT_FULL_DIAG;
  const int dl = d / 2;
  double2* dtab = sm + T;
  const uint64_t ntiles = 1ull << (F.n - k);
  const int nlow = plo - ms;               // CTA bits below the group: [ms, plo)
  // sign flips for the inverse transform (conjugate twiddles), integer only
  const uint32_t fpos = F.inverse ? 0x80000000u : 0u, fneg = fpos ^ 0x80000000u;
  const uint32_t tid = threadIdx.x;
  // each CTA takes a contiguous range of tiles: M_out (the top q0 index
  // bits) then stays the same over runs of tiles, and the diagonal's table
  // is rebuilt only when it changes
  const uint64_t per = (ntiles + gridDim.x - 1) / gridDim.x;
  const uint64_t t_end = (blockIdx.x + 1) * per < ntiles ? (blockIdx.x + 1) * per : ntiles;
  uint64_t have = ~0ull;   // M_out of the table in dtab (none yet)
  for (uint64_t t = blockIdx.x * per; t < t_end; t++) {
    // CTA bits: low part -> [ms, plo), high part -> [plo + d, n)
    const uint64_t tlo = t & ((1ull << nlow) - 1ull), thi = t >> nlow;
    const uint64_t base = (tlo << ms) | (thi << (plo + d));
    // M_out = sum_{q<q0} b_q 2^q over the high CTA bits: qubit q is bit n-1-q
    uint64_t mout = 0;
    for (int q = 0; q < F.q0; q++) mout |= ((base >> (F.n - 1 - q)) & 1ull) << q;
    const bool diag = (mout != 0) || F.scaled;
    if (diag && mout != have) {
      have = mout;
      // D(V) = scale * exp(sgn 2 pi i mout V / 2^{q1}), built by doubling from
      // directly evaluated factors exp(sgn 2 pi i (mout 2^r mod 2^{q1}) / 2^{q1})
      const uint64_t modmask = (F.q1 >= 64) ? ~0ull : ((1ull << F.q1) - 1ull);
      if (tid < (uint32_t)d) {
        const uint64_t e = (mout << tid) & modmask;
        double sn, cs;
        sincospi(2.0 * (double)e / (double)(1ull << F.q1), &sn, &cs);
        omega[tid] = make_double2(cs, xsign(sn, fpos));
      }
      if (tid == 0) dtab[0] = make_double2(F.scale, 0.0);
      if (split && tid == 1) dtab[1 << dl] = make_double2(1.0, 0.0);
      __syncthreads();
      if (split) {
        // D(V) = lo[V mod 2^dl] hi[V >> dl]: two tables of 2^dl and 2^(d-dl)
        // entries (the 2^d-entry one would take as much shared memory as the
        // tile, and cost one complex multiply per amplitude to build)
        double2* hi = dtab + (1 << dl);
        for (int r = 0; r < d - dl || r < dl; r++) {
          const double2 om = omega[r], oh = omega[dl + r < d ? dl + r : 0];
          for (uint32_t v = tid; v < (1u << r); v += BLOCK) {
            if (r < dl) dtab[v | (1u << r)] = cmul(dtab[v], om.x, om.y);
            if (r < d - dl) hi[v | (1u << r)] = cmul(hi[v], oh.x, oh.y);
          }
          __syncthreads();
        }
      } else {
        for (int r = 0; r < d; r++) {
          const double2 om = omega[r];
          for (uint32_t v = tid; v < (1u << r); v += BLOCK)
            dtab[v | (1u << r)] = cmul(dtab[v], om.x, om.y);
          __syncthreads();
        }
      }
    }
    const uint32_t lm = (1u << ms) - 1u;
    // the next tile's amplitude at the same tile index lies `ahead`
    // amplitudes further: one L2 hint per run of 2^ms amplitudes (ms <= 3)
    int64_t ahead = 0;
    if (t + 1 < t_end)
      ahead = (int64_t)((((t + 1) & ((1ull << nlow) - 1ull)) << ms) |
                        (((t + 1) >> nlow) << (plo + d))) - (int64_t)base;
    const uint32_t pmask = ahead ? lm : ~0u;
#pragma unroll 4
    for (uint32_t s = tid; s < T; s += BLOCK) {
      const uint64_t g = base | (s & lm) | ((uint64_t)(s >> ms) << plo);
      if ((s & pmask) == 0) prefetch_l2(state + g + ahead);
      double2 v = state[g];
      if (diag) {
        const uint32_t V = s >> ms;
        double2 w;
        if (split) {
          const double2 a = dtab[V & ((1u << dl) - 1u)], b = dtab[(1u << dl) + (V >> dl)];
          w = cmul(a, b.x, b.y);
        } else {
          w = dtab[V];
        }
        v = cmul(v, w.x, w.y);
      }
      sm[s] = v;
    }
    __syncthreads();
    // stage r: qubit q0 + r acts on local bit lp = ms + d - 1 - r; stages
    // in pairs as radix-4 steps, an odd last one radix 2
    int r = 0;
    if (d >= 2) {
      fft4_first<BLOCK>(sm, T, ms + d - 1, fpos, fneg);
      __syncthreads();
      r = 2;
    } else {
      const int lp = ms + d - 1;
      const uint32_t L = 1u << lp;
      for (uint32_t j = tid; j < (T >> 1); j += BLOCK) {
        const uint32_t s0 = insert0(j, lp);
        const double2 a = sm[s0], b = sm[s0 | L];
        sm[s0] = make_double2(a.x + b.x, a.y + b.y);
        sm[s0 | L] = make_double2(a.x - b.x, a.y - b.y);
      }
      __syncthreads();
      r = 1;
    }
    for (; r + 1 < d; r += 2) {
      fft4_step<BLOCK>(sm, T, ms + d - 1 - r, r, fpos, fneg);
      __syncthreads();
    }
    if (r < d) {
      const int lp = ms + d - 1 - r;
      const uint32_t L = 1u << lp;
      const double2* tw = g_tw + ((1 << r) - 1);
      if (((T >> 1) & (2 * BLOCK - 1)) == 0) {
        for (uint32_t j = tid; j < (T >> 1); j += 2 * BLOCK) {
          const uint32_t p0 = insert0(j, lp), p1 = insert0(j + BLOCK, lp);
          double2 a0 = sm[p0], b0 = sm[p0 | L], a1 = sm[p1], b1 = sm[p1 | L];
          const uint32_t v0 = p0 >> (lp + 1), v1 = p1 >> (lp + 1);
          fft_bfly(a0, b0, tw[v0], v0, fpos, fneg);
          fft_bfly(a1, b1, tw[v1], v1, fpos, fneg);
          sm[p0] = a0;
          sm[p0 | L] = b0;
          sm[p1] = a1;
          sm[p1 | L] = b1;
        }
      } else {
        for (uint32_t j = tid; j < (T >> 1); j += BLOCK) {
          const uint32_t p0 = insert0(j, lp);
          double2 a0 = sm[p0], b0 = sm[p0 | L];
          const uint32_t v0 = p0 >> (lp + 1);
          fft_bfly(a0, b0, tw[v0], v0, fpos, fneg);
          sm[p0] = a0;
          sm[p0 | L] = b0;
        }
      }
      __syncthreads();
    }
#pragma unroll 4
    for (uint32_t s = tid; s < T; s += BLOCK) {
      const uint64_t g = base | (s & lm) | ((uint64_t)(s >> ms) << plo);
      state[g] = sm[s];
    }
    __syncthreads();
  }
}

// Threads per CTA: CTAs per SM by shared memory (228 KiB), then threads so
// that the SM holds 1024 of them (64 registers each).
cudaError_t launch_fft_pass(double2* state, int n, int q0, int q1, int inverse, double scale,
                            cudaStream_t s) {
  (void)cudaGetLastError();  // report only this launcher's own errors
  static std::atomic<uint64_t> configured{0};
  cudaError_t ce = once_per_device(configured, [] {
    const int max_smem = (int)((sizeof(double2) << MAX_TILE_BITS) + (sizeof(double2) << FFT_MAX_D));
    cudaError_t e = cudaFuncSetAttribute(fft_pass_kernel<256, 4>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(fft_pass_kernel<512, 2>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(fft_pass_kernel<1024, 1>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    return e;
  });
  if (ce != cudaSuccess) return ce;
  FftParams F;
  F.n = n;
  F.q0 = q0;
  F.q1 = q1;
  F.d = q1 - q0;
  F.plo = n - q1;
  F.ms = F.plo < 3 ? F.plo : 3;   // spectator low bits for coalesced loads
  F.k = F.ms + F.d;
  F.inverse = inverse;
  F.scaled = scale != 1.0;
  F.scale = scale;
  size_t smem = (sizeof(double2) << F.k) +
                (F.d > FFT_FULL_DIAG ? sizeof(double2) * ((1u << (F.d / 2)) + (1u << (F.d - F.d / 2)))
                                     : sizeof(double2) << F.d);
  int per_sm = (int)((228u << 10) / (smem + (2u << 10)));
  per_sm = per_sm < 1 ? 1 : per_sm > 4 ? 4 : per_sm;
  if (per_sm == 3) per_sm = 2;
  const uint32_t T = 1u << F.k;
  uint64_t ntiles = 1ull << (n - F.k);
  uint64_t cap = (uint64_t)sm_count() * per_sm;
  int grid = (int)(ntiles < cap ? ntiles : cap);
  // small tiles take the smallest block
  if (per_sm >= 4 || T < 4096) {
    fft_pass_kernel<256, 4><<<grid, 256, smem, s>>>(F, state);
  } else if (per_sm == 2) {
    fft_pass_kernel<512, 2><<<grid, 512, smem, s>>>(F, state);
  } else {
    fft_pass_kernel<1024, 1><<<grid, 1024, smem, s>>>(F, state);
  }
  return cudaGetLastError();
}

// --------------------------------------------------------- bit reversal

// In-place index bit reversal i -> rev_n(i).  Tile bits are the low L and the
// high L bits; the middle bits M select the tile.  Tile c and tile rev_M(c)
// exchange contents, so one CTA handles the pair (c <= rev_M(c)) and no tile
// is read after another CTA wrote it.
template <int BLOCK, int L>
__global__ void __launch_bounds__(BLOCK) bitrev_kernel(double2* __restrict__ state, int n) {
  extern __shared__ double2 sm[];  // 2 * 2^{2L}
  constexpr uint32_t TL = 1u << L, T = TL * TL;
  static_assert(L >= 3, "the swizzle takes 3 row bits");
  const int M = n - 2 * L;
  double2* A = sm;
  double2* B = sm + T;
  const uint64_t ntiles = 1ull << M;
  // Tile rows are stored XOR-swizzled: (row r, column col) at r * TL + (col ^
  // ((r >> (L - 3)) & 7)).  The transposed read below takes rows r = rev(lo2)
  // for 8 consecutive lo2 per quarter warp; those rows differ exactly in bits
  // L-3..L-1, so the 8 accesses hit 8 different 16-byte bank slots (without
  // the swizzle all 8 hit the same one).
  for (uint64_t c = blockIdx.x; c < ntiles; c += gridDim.x) {
    const uint64_t cr = M ? (__brevll(c) >> (64 - M)) : 0;
    if (cr < c) continue;
    // element (hi, lo) of tile c: index hi << (n-L) | c << L | lo
#pragma unroll 4
    for (uint32_t s = threadIdx.x; s < T; s += BLOCK) {
      const uint32_t hi = s >> L, lo = s & (TL - 1);
      const uint32_t slot = hi * TL + (lo ^ ((hi >> (L - 3)) & 7u));
      A[slot] = state[((uint64_t)hi << (n - L)) | (c << L) | lo];
      if (cr != c) B[slot] = state[((uint64_t)hi << (n - L)) | (cr << L) | lo];
    }
    __syncthreads();
    // destination (hi', lo') of tile cr receives source (hi = rev(lo'), lo = rev(hi'))
#pragma unroll 4
    for (uint32_t s = threadIdx.x; s < T; s += BLOCK) {
      const uint32_t hi2 = s >> L, lo2 = s & (TL - 1);
      const uint32_t r = __brev(lo2) >> (32 - L), col = __brev(hi2) >> (32 - L);
      const uint32_t slot = r * TL + (col ^ ((r >> (L - 3)) & 7u));
      state[((uint64_t)hi2 << (n - L)) | (cr << L) | lo2] = A[slot];
      if (cr != c) state[((uint64_t)hi2 << (n - L)) | (c << L) | lo2] = B[slot];
    }
    __syncthreads();
  }
}

// Small states: the whole vector in one CTA.
__global__ void bitrev_small_kernel(double2* __restrict__ state, int n) {
  extern __shared__ double2 sm[];
  const uint32_t N = 1u << n;
  for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) sm[i] = state[i];
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < N; i += blockDim.x)
    state[i] = sm[n ? (__brev(i) >> (32 - n)) : 0];
}

cudaError_t launch_bitrev(double2* state, int n, cudaStream_t s) {
  (void)cudaGetLastError();  // report only this launcher's own errors
  if (n <= 12) {
    static std::atomic<uint64_t> conf{0};
    cudaError_t ce = once_per_device(conf, [] {
      return cudaFuncSetAttribute(bitrev_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(sizeof(double2) << 12));
    });
    if (ce != cudaSuccess) return ce;
    bitrev_small_kernel<<<1, 512, sizeof(double2) << n, s>>>(state, n);
    return cudaGetLastError();
  }
  // 32 x 32 tiles (512-byte runs), 32 KiB of shared memory per CTA: six
  // CTAs per SM (measured at n = 30: 6.6 ms against 8.0 ms with four)
  constexpr int L = 5;
  size_t smem = 2 * (sizeof(double2) << (2 * L));
  uint64_t ntiles = 1ull << (n - 2 * L);
  uint64_t cap = (uint64_t)sm_count() * 6;
  int grid = (int)(ntiles < cap ? ntiles : cap);
  bitrev_kernel<256, L><<<grid, 256, smem, s>>>(state, n);
  return cudaGetLastError();
}

}  // namespace lq

using namespace lq;

// Pass boundaries (qubit indices) of the FFT form: the lowest group takes up to
// 12 qubits, earlier groups up to 10 (tile = group + 3 spectator bits <= 13).
static std::vector<int> fft_bounds(int n) {
  std::vector<int> bounds;
  int rest = n;
  int last = n < 12 ? n : 12;
  rest -= last;
  int ng = (rest + 9) / 10;
  bounds.push_back(0);
  for (int i = 0; i < ng; i++)
    bounds.push_back(bounds.back() + (rest - bounds.back() + (ng - i) - 1) / (ng - i));
  if (bounds.back() != n) bounds.push_back(n);
  return bounds;
}

// Gates of Alg. 3 without its final swap network.  Alg. 3 applies, for i,
// H(i) then CP(pi / 2^{j-i}) with control i and target j > i.  CP(i, j) is
// diagonal: it commutes with every other CP and with the H of any qubit other
// than i and j, so it can move to just before H(j); from n = 24 on the
// forward list is, for j, the CP(i, j) with i < j, then H(j) -- the same
// gates, so the same unitary (smaller states keep Alg. 3's order, which
// schedules into cheaper passes there).  Then each qubit's phases (one merged op on its bit) stand right
// before its H, which runs them as butterflies (as in the inverse: the
// reversed Alg. 3 order with conjugated phases).  The floor(n/2)
// SWAP(i, n-1-i) gates reverse the bits of the index; they run as one
// bit-reversal pass (after the gates, or before them for the inverse).
// Default schedule of the gate form on large states (no tune-cache entry):
// 2^11-amplitude tiles with 6 contiguous low bits and the dyadic phase
// tables, the autotuner's choice for the n = 30 inverse transform (221.6 ms
// against 242.1 ms with the library default).
static const ScheduleOptions* qft_gate_schedule(int n, ScheduleOptions* opt) {
  if (n < 24) return nullptr;
  opt->k = 11;
  opt->m = 6;
  opt->lphase_table = true;
  return opt;
}

static std::vector<lq_gate> qft_gate_list(int n, int inverse) {
  const double PI = 3.14159265358979323846;
  std::vector<lq_gate> g;
  auto mk = [](int kind, int a, int b, double ang) {
    lq_gate G;
    std::memset(&G, 0, sizeof G);
    G.kind = kind;
    G.qubits[0] = a;
    G.qubits[1] = b;
    G.qubits[2] = -1;
    G.param = -1;
    G.angle = ang;
    return G;
  };
  if (!inverse && n >= 24) {   // measured: from n = 24 on the reordered list is faster
    for (int j = 0; j < n; j++) {
      for (int i = 0; i < j; i++) g.push_back(mk(LQ_CP, i, j, PI / std::ldexp(1.0, j - i)));
      g.push_back(mk(LQ_H, j, -1, 0));
    }
    return g;
  }
  for (int i = 0; i < n; i++) {
    g.push_back(mk(LQ_H, i, -1, 0));
    for (int j = i + 1; j < n; j++) g.push_back(mk(LQ_CP, i, j, PI / std::ldexp(1.0, j - i)));
  }
  if (inverse) {
    std::vector<lq_gate> r(g.rbegin(), g.rend());
    for (auto& G : r)
      if (G.kind == LQ_CP) G.angle = -G.angle;
    g.swap(r);
  }
  return g;
}

extern "C" lq_status lq_qft_plan_dir(int n, int method, int inverse, lq_plan_info* out) {
  lq_status st = check_n(n);
  if (st) return st;
  if (!out) return fail(LQ_ERR_INVALID_ARG, "out is NULL");
  if (method == LQ_QFT_GATES) {
    std::vector<lq_gate> g = qft_gate_list(n, inverse);
    ScheduleOptions def;
    st = circuit_plan_with(n, g.data(), (int)g.size(), nullptr, 0, out, qft_gate_schedule(n, &def));
    if (st) return st;
    if (n > 1) {   // the bit-reversal pass
      out->npasses += 1;
      out->dram_bytes += 32.0 * std::ldexp(1.0, n);
    }
    return LQ_OK;
  }
  if (method != LQ_QFT_FFT) return fail(LQ_ERR_INVALID_ARG, "unknown QFT method %d", method);
  std::vector<int> b = fft_bounds(n);
  const double N = std::ldexp(1.0, n);
  double fl = 0;
  int kmax = 0;
  for (std::size_t p = 0; p + 1 < b.size(); p++) {
    int d = b[p + 1] - b[p];
    int ms = (n - b[p + 1]) < 3 ? (n - b[p + 1]) : 3;
    kmax = kmax > d + ms ? kmax : d + ms;
    // butterflies: the first two stages 16 adds per quad, later pairs of
    // stages 22 FMA per quad (radix 4), an odd last stage 6 FMA per pair; a
    // one-stage pass 2 adds per amplitude
    fl += d == 1 ? 2.0 * N : N * (4.0 + 11.0 * ((d - 2) / 2) + 6.0 * ((d - 2) % 2));
    // diagonal of the pass (all but the first; the last also carries the
    // scale): a complex multiply, and for groups read from two tables the
    // product of the two entries
    if (p > 0 || b.size() == 2) fl += (d > FFT_FULL_DIAG ? 12.0 : 6.0) * N;
  }
  out->npasses = (int)b.size();   // FFT passes + the bit-reversal pass
  out->tile_bits = kmax;
  out->dp_flops = fl;
  out->dram_bytes = 32.0 * N * (double)b.size();
  return LQ_OK;
}

extern "C" lq_status lq_qft_plan(int n, int method, lq_plan_info* out) {
  return lq_qft_plan_dir(n, method, 0, out);
}

extern "C" lq_status lq_autotune_qft(void* scratch, int n, int inverse, lq_tune_result* out,
                                     lq_stream stream) {
  lq_status st = check_n(n);
  if (st) return st;
  std::vector<lq_gate> g = qft_gate_list(n, inverse);
  return lq_autotune_circuit(scratch, n, g.data(), (int)g.size(), nullptr, 0, out, stream);
}

extern "C" lq_status lq_qft(void* amps, int n, int inverse, int method, void* scratch,
                            size_t scratch_bytes, lq_stream stream) {
  (void)scratch;
  (void)scratch_bytes;
  lq_status st = check_n(n);
  if (st) return st;
  if (!amps) return fail(LQ_ERR_INVALID_ARG, "amps is NULL");
  if (method != LQ_QFT_FFT && method != LQ_QFT_GATES)
    return fail(LQ_ERR_INVALID_ARG, "unknown QFT method %d", method);
  cudaStream_t s = (cudaStream_t)stream;
  double2* psi = (double2*)amps;
  if (method == LQ_QFT_GATES) {
    // Alg. 3: for i: H(i), CP(pi/2^{j-i}) control i target j > i; then the
    // swaps (one bit-reversal pass).  The inverse is the reversed sequence
    // with conjugated phases.
    std::vector<lq_gate> g = qft_gate_list(n, inverse);
    cudaError_t e = cudaSuccess;
    if (inverse && n > 1 && (e = launch_bitrev(psi, n, s)) != cudaSuccess)
      return fail(LQ_ERR_CUDA, "bit reversal: %s", cudaGetErrorString(e));
    ScheduleOptions def;
    st = apply_circuit_with(amps, n, g.data(), (int)g.size(), nullptr, 0, stream,
                            qft_gate_schedule(n, &def));
    if (st) return st;
    if (!inverse && n > 1 && (e = launch_bitrev(psi, n, s)) != cudaSuccess)
      return fail(LQ_ERR_CUDA, "bit reversal: %s", cudaGetErrorString(e));
    return LQ_OK;
  }
  cudaError_t e = fft_tables_init(s);
  if (e == cudaErrorStreamCaptureUnsupported)
    return fail(LQ_ERR_CUDA, "fft tables: the first FFT-form QFT on a device fills its twiddle "
                "table and is refused while the stream is capturing; make one uncaptured call "
                "first");
  if (e != cudaSuccess) return fail(LQ_ERR_CUDA, "fft tables: %s", cudaGetErrorString(e));
  std::vector<int> bounds = fft_bounds(n);
  const double scale = std::ldexp(1.0, -n / 2) * ((n & 1) ? 0.70710678118654752440 : 1.0);
  int npass = (int)bounds.size() - 1;
  for (int p = 0; p < npass; p++) {
    e = launch_fft_pass(psi, n, bounds[p], bounds[p + 1], inverse,
                        p == npass - 1 ? scale : 1.0, s);
    if (e != cudaSuccess) return fail(LQ_ERR_CUDA, "fft pass: %s", cudaGetErrorString(e));
  }
  e = launch_bitrev(psi, n, s);
  if (e != cudaSuccess) return fail(LQ_ERR_CUDA, "bit reversal: %s", cudaGetErrorString(e));
  return LQ_OK;
}
