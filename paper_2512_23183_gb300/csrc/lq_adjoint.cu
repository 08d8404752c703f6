// lq_adjoint.cu -- exact gradients by reverse-mode (adjoint) differentiation.
//
// For E(theta) = <psi_L|H|psi_L>, psi_L = U_L ... U_1 |0>, and a gate
// U_k = exp(-i theta G_k / 2) (Sec. III-A form of the parametrised gates):
//     dE/dtheta_k = 2 Re <lambda_k| (-i G_k / 2) |psi_k> = Im <lambda_k|G_k|psi_k>,
// where psi_k = U_k ... U_1|0> and lambda_k = U_{k+1}^dag ... U_L^dag H psi_L.
// Starting from psi_L and lambda_L = H psi_L, the sweep for k = L..1 adds
// Im <lambda|G_k|psi> to the gradient of gate k's parameter and then applies
// U_k^dag to both states.  Phase gates P(theta) = exp(i theta |1><1|) and
// CP have G = -2 (projector), controlled rotations G = |1><1| (x) sigma.
//
// The sweep is lowered like a circuit: each U_k^dag becomes tile ops in
// tangent form with deferred scalars (the same scalar for both states, so
// <lambda|G|psi> carries the real factor |zeta|^2), and each gradient term
// becomes an OP_GRAD op whose per-warp sums collect in shared memory over a
// CTA's tiles; two-state tile passes hold psi and lambda in shared memory
// together, so each pass reads and writes each state once.  Two states are resident, no checkpoints are needed: U^dag
// uncomputes the forward states.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "lq_coefs.h"
#include "lq_device.cuh"
#include "lq_internal.h"
#include "lq_kernels.h"

namespace lq {

#define LQ_CUDA(expr)                                                                  \
  do {                                                                                 \
    cudaError_t e_ = (expr);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      (void)cudaGetLastError();                                                        \
      return fail(LQ_ERR_CUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, \
                  __LINE__);                                                           \
    }                                                                                  \
  } while (0)

static constexpr int kPassBlock = 256;

// ------------------------------------------------------- two-state passes

// Warp sums of gradient terms, four at a time: each lane holds its partial
// value of up to four consecutive terms; a transposing butterfly (lanes
// exchange the terms they do not keep) leaves lane t < 4 with term t's warp
// sum after 6 adds and 6 double shuffles, against 20 and 20 for four plain
// shuffle reductions.  gacc[term][warp] collects the sums over the tiles.
struct GradBatch {
  double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
  int n = 0, first = 0;
};

__device__ __forceinline__ void grad_flush(GradBatch& b, double* gacc, int nw, int warp) {
  if (b.n == 0) return;
  const uint32_t lane = threadIdx.x & 31;
  const bool o1 = lane & 1, o2 = lane & 2;
  // lanes with bit 0 set keep terms 1 and 3, the others 0 and 2
  const double k0 = (o1 ? b.v1 : b.v0) + __shfl_xor_sync(0xffffffffu, o1 ? b.v0 : b.v1, 1);
  const double k1 = (o1 ? b.v3 : b.v2) + __shfl_xor_sync(0xffffffffu, o1 ? b.v2 : b.v3, 1);
  // lanes with bit 1 set keep terms 2|3, the others 0|1: lane holds term lane & 3
  double kept = (o2 ? k1 : k0) + __shfl_xor_sync(0xffffffffu, o2 ? k0 : k1, 2);
  kept += __shfl_xor_sync(0xffffffffu, kept, 4);
  kept += __shfl_xor_sync(0xffffffffu, kept, 8);
  kept += __shfl_xor_sync(0xffffffffu, kept, 16);
  if (lane < (uint32_t)b.n) gacc[(b.first + (int)lane) * nw + warp] += kept;
  b = GradBatch();
}

// Add this thread's value v of gradient term gl (terms arrive in order).
__device__ __forceinline__ void grad_push(GradBatch& b, double v, int gl, double* gacc, int nw,
                                          int warp) {
  if (b.n == 0) b.first = gl;
  switch (b.n) {
    case 0: b.v0 = v; break;
    case 1: b.v1 = v; break;
    case 2: b.v2 = v; break;
    default: b.v3 = v; break;
  }
  if (++b.n == 4) grad_flush(b, gacc, nw, warp);
}

// A gradient op and the op after it fuse (grad_rot1_pairs) when both act on
// the same single tile bit without conditions, the generator's Z part lies
// on that bit, and the rotation is in tangent or cotangent form with phases
// of the parity opposite to the generator's.
__device__ __forceinline__ bool fusable_grad_rot(const Op& g, const Op& r) {
  if (r.type != OP_PAULI || g.x_loc == 0 || g.x_loc != r.x_loc || (g.x_loc & (g.x_loc - 1)) != 0)
    return false;
  if (g.cm_loc | r.cm_loc | g.cm_glob | r.cm_glob) return false;
  if ((g.z_loc & ~g.x_loc) | (r.z_loc & ~r.x_loc)) return false;
  const int pm = r.mode & 3;
  if (pm != PM_TAN && pm != PM_COT) return false;
  // rotation phase parity (r.mode >> 2) against the generator's (i^k0)
  return ((r.mode >> 2) & 1) != (g.mode & 1);
}

// Op o only reads the tiles: a gradient op not fused with the op after it.
__device__ __forceinline__ bool grad_reads_only(const Op* ops, int o, int nops) {
  return ops[o].type == OP_GRAD && !(o + 1 < nops && fusable_grad_rot(ops[o], ops[o + 1]));
}

// Gradient terms of a run of diagonal generators G_t (Z strings z_t under
// conditions cm_t/cv_t; x = 0, no factor i) on the two tiles A = psi,
// B = lambda: Im <lambda|G_t|psi> = sum_s G_t(s) q_s with
// q_s = Im(conj(lambda_s) psi_s).  Diagonal unitaries applied to both states
// leave q unchanged, which is why a run of diagonal gates of the reverse
// sweep can take all its gradients at one point.  A thread holds the
// amplitudes s = tid + i * BLOCK (i < 8, T <= 8 * BLOCK); after a Walsh-
// Hadamard transform over i, W[m] = sum_i (-1)^popcount(i & m) q_i, so
//   sum_s (-1)^popcount(s & M) q_s = (-1)^popcount(tid & M) W[M / BLOCK]
// over this thread's amplitudes, and a condition on the bits cm with values
// cv expands as prod_b (1 + (-1)^(s_b + cv_b)) / 2 over its bits:
//   sum_s [cond(s)] (-1)^popcount(s & z) q_s
//     = 2^-|cm| sum_{S subset of cm} (-1)^popcount(cv & S) W(z ^ S).
// Each term's value goes to the warp's gradient batch as term gl + t.
template <int BLOCK>
__device__ __forceinline__ void diag_grad_terms(const double2* __restrict__ A,
                                                const double2* __restrict__ B, uint32_t T,
                                                const Op* ops, int nterms, uint64_t base,
                                                GradBatch& gb, int gl, double* gacc, int nw) {
  constexpr int LB = BLOCK == 1024 ? 10 : BLOCK == 512 ? 9 : BLOCK == 256 ? 8 : 7;
  static_assert((1 << LB) == BLOCK, "BLOCK must be a power of two in 128..1024");
  const uint32_t tid = threadIdx.x;
  double q[8];
#pragma unroll
  for (int i = 0; i < 8; i++) {
    const uint32_t s = tid + (uint32_t)i * BLOCK;
    q[i] = 0.0;
    if (s < T) {
      const double2 l = B[s], v = A[s];
      q[i] = fma(l.x, v.y, -l.y * v.x);
    }
  }
#pragma unroll
  for (int h = 1; h < 8; h <<= 1)
#pragma unroll
    for (int i = 0; i < 8; i++)
      if (!(i & h)) {
        const double a = q[i], b = q[i | h];
        q[i] = a + b;
        q[i | h] = a - b;
      }
  for (int t = 0; t < nterms; t++) {
    const Op& d = ops[t];
    double v = 0.0;
    if ((base & d.cm_glob) == d.cv_glob) {
      const uint32_t cm = d.cm_loc, cv = d.cv_loc;
      uint32_t S = cm;
      while (true) {
        const uint32_t M = d.z_loc ^ S;
        const uint32_t mi = (M >> LB) & 7u;
        double w = q[0];
#pragma unroll
        for (int j = 1; j < 8; j++) w = (mi == (uint32_t)j) ? q[j] : w;
        const int neg = (__popc(tid & M & (BLOCK - 1)) + __popc(cv & S)) & 1;
        v += neg ? -w : w;
        if (S == 0) break;
        S = (S - 1) & cm;
      }
      v = ldexp(v, -__popc(cm));
      if (__popcll(base & d.z_glob) & 1) v = -v;
    }
    grad_push(gb, v, gl + t, gacc, nw, (int)(tid >> 5));
  }
}

// A one-bit rotation's gradient op fused with the rotation that follows it
// in the sweep (U_k^dag of the same gate, or any one-bit rotation on the same
// bit without conditions): one pass over the amplitude pairs (s0, s1 = s0|x)
// adds the gradient terms Im(conj(lambda_s0) i^gA psi_s1) and
// Im(conj(lambda_s1) i^gB psi_s0) and rotates both states' pairs.  For RY
// the gradient phases are odd and the rotation's even, for RX the reverse
// (ODD = rotation phases odd); the gradient signs (gA, gB & 2) are applied
// to the sums afterwards.  Same FP64 work as the separate ops, half the
// shared-memory reads and one barrier instead of two.
template <int BLOCK, int FORM, bool ODD>
__device__ __forceinline__ void grad_rot1_pairs(double2* __restrict__ A, double2* __restrict__ B,
                                                uint32_t T, uint32_t x, double a, double cA,
                                                double cB, uint32_t sA, uint32_t sB,
                                                double& accA, double& accB) {
  const uint32_t tid = threadIdx.x;
  const int h = 31 - __clz(x);
  // acc += Im(conj(l) i^g v) up to the sign of g
  auto term = [&](double& acc, double2 l, double2 v) {
    acc = ODD ? fma(l.x, v.y, fma(-l.y, v.x, acc)) : fma(l.x, v.x, fma(l.y, v.y, acc));
  };
  auto rot = [&](double2 u0, double2 u1, double2& o0, double2& o1) {
    if (FORM == ROT_TAN) {
      o0 = rot_fma<ODD>(cA, u1, u0);
      o1 = rot_fma<ODD>(cB, u0, u1);
    } else {
      o0 = rot_cot<ODD>(a, u0, u1, sA);
      o1 = rot_cot<ODD>(a, u1, u0, sB);
    }
  };
  for (uint32_t j = tid; j < (T >> 1); j += BLOCK) {
    const uint32_t s0 = insert0(j, h), s1 = s0 | x;
    const double2 p0 = A[s0], p1 = A[s1], l0 = B[s0], l1 = B[s1];
    term(accA, l0, p1);
    term(accB, l1, p0);
    double2 o0, o1;
    rot(p0, p1, o0, o1);
    A[s0] = o0;
    A[s1] = o1;
    rot(l0, l1, o0, o1);
    B[s0] = o0;
    B[s1] = o1;
  }
}

// Adjoint sweep: every op is applied to both tiles (psi in A, lambda in B);
// an OP_GRAD op instead adds Im <lambda| G |psi> over its amplitudes
// (G = condition projector x Pauli string: <i|P|j> = i^k0 (-1)^popcount(j & z),
// j = i ^ x).  Each warp keeps its own running sum per gradient op of the
// pass in shared memory (gacc[op][warp], no barrier, no global traffic per
// tile); at the end the CTA adds the warp sums, in warp order, into
// partial[slot * pstride + blockIdx.x] (one writer per entry, fixed
// reduction order).
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, 3) pass2_kernel(const __grid_constant__ PassParams P,
                                                      double2* __restrict__ psi,
                                                      double2* __restrict__ lam,
                                                      double* __restrict__ partial, int pstride,
                                                      int ngrad) {
  constexpr int NW = BLOCK / 32;
  extern __shared__ double2 sm[];
  __shared__ uint64_t hioff[256];
  const int k = P.h.k, m = P.h.m, nops = P.h.nops;
  const uint32_t T = 1u << k;
  double2* A = sm;
  double2* B = sm + T;
  double* gacc = (double*)(sm + 2 * T);
  const uint32_t lowmask = (1u << m) - 1u;
  const int kh = k - m;
  for (uint32_t j = threadIdx.x; j < (1u << kh); j += BLOCK)
    hioff[j] = deposit(j, P.h.tbits + m, kh);
  for (int j = threadIdx.x; j < ngrad * NW; j += BLOCK) gacc[j] = 0.0;
  const uint64_t ntiles = P.h.ntiles;
  const int warp = threadIdx.x >> 5;
  __syncthreads();
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint64_t base = deposit(t, P.h.obits, P.h.nobits);
    for (uint32_t s = threadIdx.x; s < T; s += BLOCK) {
      const uint64_t g = base | hioff[s >> m] | (s & lowmask);
      A[s] = psi[g];
      B[s] = lam[g];
    }
    __syncthreads();
    int gl = 0;
    GradBatch gb;
    for (int o = 0; o < nops; o++) {
      const Op& op = P.ops[o];
      if (op.type == OP_GRAD && op.x_loc == 0 && (op.mode & 3) == 0 && T <= 8 * BLOCK) {
        // a run of diagonal generators (Z strings under conditions): one
        // pass over the tile for all of them (see diag_grad_terms)
        int e = o + 1;
        while (e < nops && P.ops[e].type == OP_GRAD && P.ops[e].x_loc == 0 &&
               (P.ops[e].mode & 3) == 0)
          e++;
        diag_grad_terms<BLOCK>(A, B, T, P.ops + o, e - o, base, gb, gl, gacc, NW);
        gl += e - o;
        o = e - 1;
        // the next op may overwrite what this one read
        if (e < nops && !grad_reads_only(P.ops, e, nops)) __syncthreads();
      } else if (op.type == OP_GRAD && o + 1 < nops && fusable_grad_rot(op, P.ops[o + 1])) {
        const Op& r = P.ops[o + 1];
        double accA = 0.0, accB = 0.0;
        const int zsg = __popcll(base & op.z_glob) & 1, zsr = __popcll(base & r.z_glob) & 1;
        const int k0 = op.mode & 3;
        const int gA = (k0 + 2 * ((op.z_loc != 0) + zsg)) & 3, gB = (k0 + 2 * zsg) & 3;
        const int rk0 = r.mode >> 2;
        const int kA = (rk0 + 2 * ((r.z_loc != 0) + zsr)) & 3, kB = (rk0 + 2 * zsr) & 3;
        const double a = r.a, cA = xsign(a, (uint32_t)(kA & 2) << 30),
                     cB = xsign(a, (uint32_t)(kB & 2) << 30);
        const uint32_t sA = (uint32_t)(kA & 2) << 30, sB = (uint32_t)(kB & 2) << 30;
        const bool odd = kA & 1;
        if ((r.mode & 3) == PM_TAN) {
          if (odd)
            grad_rot1_pairs<BLOCK, ROT_TAN, true>(A, B, T, r.x_loc, a, cA, cB, sA, sB, accA, accB);
          else
            grad_rot1_pairs<BLOCK, ROT_TAN, false>(A, B, T, r.x_loc, a, cA, cB, sA, sB, accA, accB);
        } else {
          if (odd)
            grad_rot1_pairs<BLOCK, ROT_COT, true>(A, B, T, r.x_loc, a, cA, cB, sA, sB, accA, accB);
          else
            grad_rot1_pairs<BLOCK, ROT_COT, false>(A, B, T, r.x_loc, a, cA, cB, sA, sB, accA, accB);
        }
        grad_push(gb, ((gA & 2) ? -accA : accA) + ((gB & 2) ? -accB : accB), gl, gacc, NW, warp);
        gl++;
        o++;
        __syncthreads();
      } else if (op.type == OP_GRAD) {
        double acc = 0.0;
        if ((base & op.cm_glob) == op.cv_glob) {
          const int zs = __popcll(base & op.z_glob) & 1;
          const int k0 = op.mode & 3;
          for (uint32_t s = threadIdx.x; s < T; s += BLOCK) {
            if ((s & op.cm_loc) != op.cv_loc) continue;
            const uint32_t j = s ^ op.x_loc;
            const int kk = (k0 + 2 * ((__popc(j & op.z_loc) + zs) & 1)) & 3;
            const double2 v = mul_ipow(A[j], kk);
            const double2 l = B[s];
            acc = fma(l.x, v.y, fma(-l.y, v.x, acc));
          }
        }
        grad_push(gb, acc, gl, gacc, NW, warp);
        gl++;
        // the next op may overwrite what this one read
        if (o + 1 < nops && !grad_reads_only(P.ops, o + 1, nops)) __syncthreads();
      } else if (op.type == OP_LPHASE && !(op.mode & LP_TABLE)) {
        // the same per-tile phase tables serve both states
        apply_op<BLOCK>(A, T, op, P.coef, base, (const double2*)P.h.dtab, nullptr, nullptr, B);
        __syncthreads();
      } else {
        apply_op<BLOCK>(A, T, op, P.coef, base, (const double2*)P.h.dtab);
        apply_op<BLOCK>(B, T, op, P.coef, base, (const double2*)P.h.dtab);
        __syncthreads();
      }
    }
    grad_flush(gb, gacc, NW, warp);
    for (uint32_t s = threadIdx.x; s < T; s += BLOCK) {
      const uint64_t g = base | hioff[s >> m] | (s & lowmask);
      psi[g] = A[s];
      lam[g] = B[s];
    }
    __syncthreads();
  }
  int gl = 0;
  for (int o = 0; o < nops; o++) {
    if (P.ops[o].type != OP_GRAD) continue;
    if ((gl % BLOCK) == (int)threadIdx.x) {
      double sum = 0.0;
      for (int w = 0; w < NW; w++) sum += gacc[gl * NW + w];
      partial[(uint64_t)P.ops[o].cidx * pstride + blockIdx.x] += sum;
    }
    gl++;
  }
}

// Tile bits of the reverse sweep: two 32 KiB tiles per CTA (3 CTAs per SM)
// take fewer passes than 2^10-amplitude tiles: measured 11% faster at
// n = 24 and 6% at n = 18 (128 tiles); at n = 16 (32 tiles for 152 SMs)
// 2^10-amplitude tiles are 12% faster.
static int sweep_tile_bits(int n) { return n >= 18 ? 11 : n < 10 ? n : 10; }

// Largest grid of a two-state pass (the stride of the partial sums): tiles
// of 2^k amplitudes, up to 6 CTAs per SM; passes with wider tiles launch
// fewer CTAs.
int pass2_grid(int n, int k) {
  uint64_t ntiles = 1ull << (n - (k < n ? k : n));
  size_t smem = 2 * (sizeof(double2) << (k < n ? k : n));
  int per_sm = smem <= 32768 ? 6 : smem <= 65536 ? 3 : 1;
  uint64_t cap = (uint64_t)sm_count() * per_sm;
  return (int)(ntiles < cap ? ntiles : cap);
}

cudaError_t launch_pass2(const PassParams& P, double2* psi, double2* lam, double* partial,
                         int grid, cudaStream_t s) {
  (void)cudaGetLastError();  // report only this launcher's own errors
  constexpr int NW = kPassBlock / 32;
  static std::atomic<uint64_t> configured{0};
  cudaError_t ce = once_per_device(configured, [] {
    // two tiles of at most 2^12 amplitudes and one running sum per warp per op
    return cudaFuncSetAttribute(pass2_kernel<kPassBlock>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(2 * (sizeof(double2) << 12) + sizeof(double) * NW * MAX_OPS));
  });
  if (ce != cudaSuccess) return ce;
  if (P.h.k > 12) return cudaErrorInvalidValue;
  int ngrad = 0;
  for (int o = 0; o < P.h.nops; o++) ngrad += P.ops[o].type == OP_GRAD;
  const size_t smem = 2 * (sizeof(double2) << P.h.k) + sizeof(double) * NW * ngrad;
  // one wave of resident CTAs (registers and shared memory); with tiles of
  // at most 2^11 amplitudes two CTAs per SM always fit, so fewer tiles than
  // that need no occupancy query (it costs microseconds per launch, which
  // small states feel)
  uint64_t g = P.h.ntiles;
  if (P.h.k > 11 || g > 2 * (uint64_t)sm_count()) {
    int per_sm = 0;
    cudaError_t oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, pass2_kernel<kPassBlock>, kPassBlock, smem);
    if (oe != cudaSuccess) return oe;
    per_sm = per_sm < 1 ? 1 : per_sm;
    g = (uint64_t)sm_count() * per_sm;
    if (g > P.h.ntiles) g = P.h.ntiles;
  }
  const int pgrid = (int)g < grid ? (int)g : grid;
  if (P.h.flags & PF_DYADIC) {
    cudaError_t e;
    const double2* t = dyadic_tables(&e, &s);
    if (!t) return e;
    static thread_local PassParams Q;
    Q = P;
    Q.h.dtab = t;
    pass2_kernel<kPassBlock><<<pgrid, kPassBlock, smem, s>>>(Q, psi, lam, partial, grid, ngrad);
  } else {
    pass2_kernel<kPassBlock><<<pgrid, kPassBlock, smem, s>>>(P, psi, lam, partial, grid, ngrad);
  }
  return cudaGetLastError();
}

// grad[p] = sum over the slots of parameter p (in slot order) of
// factor[slot] * sum_b partial[slot][b].
__global__ void grad_reduce_kernel(const double* __restrict__ partial, int grid,
                                   const double* __restrict__ factor,
                                   const int* __restrict__ first, const int* __restrict__ count,
                                   int np, double* __restrict__ grad) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  double g = 0;
  for (int s = first[p]; s < first[p] + count[p]; s++) {
    double v = 0;
    for (int b = 0; b < grid; b++) v += partial[(uint64_t)s * grid + b];
    g += factor[s] * v;
  }
  grad[p] = g;
}

cudaError_t launch_grad_reduce(const double* partial, int grid, const double* factor,
                               const int* first, const int* count, int np, double* grad,
                               cudaStream_t s) {
  (void)cudaGetLastError();  // report only this launcher's own errors
  if (np <= 0) return cudaSuccess;
  grad_reduce_kernel<<<(np + 127) / 128, 128, 0, s>>>(partial, grid, factor, first, count, np,
                                                      grad);
  return cudaGetLastError();
}

static inline std::size_t align256(std::size_t b) { return (b + 255) & ~(std::size_t)255; }

// U^dag of a gate: rotations and phases at -theta, S <-> SDG, T <-> TDG,
// matrices conjugate-transposed, the rest self-inverse.
static lq_gate inverse_gate(const lq_gate& g) {
  lq_gate r = g;
  switch (g.kind) {
    case LQ_S: r.kind = LQ_SDG; break;
    case LQ_SDG: r.kind = LQ_S; break;
    case LQ_T: r.kind = LQ_TDG; break;
    case LQ_TDG: r.kind = LQ_T; break;
    case LQ_U1: case LQ_U2: {
      int d = g.kind == LQ_U1 ? 2 : 4;
      for (int i = 0; i < d; i++)
        for (int j = 0; j < d; j++) {
          r.mat[2 * (i * d + j)] = g.mat[2 * (j * d + i)];
          r.mat[2 * (i * d + j) + 1] = -g.mat[2 * (j * d + i) + 1];
        }
      break;
    }
    default: break;
  }
  return r;
}

// Gradient op (generator) of a parametrised gate and its factor f_gen.
static LOp grad_op(const lq_gate& g, int n, double* fgen) {
  LOp o;
  o.type = OP_GRAD;
  int b0 = n - 1 - g.qubits[0];
  int b1 = gate_arity(g.kind) > 1 ? n - 1 - g.qubits[1] : 0;
  uint64_t m0 = 1ull << b0, m1 = 1ull << b1;
  int ny = 0;
  *fgen = 1.0;
  switch (g.kind) {
    case LQ_RX: o.x = m0; break;
    case LQ_RY: o.x = m0; o.z = m0; ny = 1; break;
    case LQ_RZ: o.z = m0; break;
    case LQ_RXX: o.x = m0 | m1; break;
    case LQ_RYY: o.x = m0 | m1; o.z = m0 | m1; ny = 2; break;
    case LQ_RZZ: o.z = m0 | m1; break;
    case LQ_P: o.cm = o.cv = m0; *fgen = -2.0; break;
    case LQ_CP: o.cm = o.cv = m0 | m1; *fgen = -2.0; break;
    case LQ_CRX: o.cm = o.cv = m0; o.x = m1; break;
    case LQ_CRY: o.cm = o.cv = m0; o.x = m1; o.z = m1; ny = 1; break;
    case LQ_CRZ: o.cm = o.cv = m0; o.z = m1; break;
    default: break;
  }
  o.mode = (uint8_t)(ny & 3);
  return o;
}

}  // namespace lq

namespace lq {
// The reverse sweep as scheduled tile passes: for k = L..1 an OP_GRAD op
// (if gate k has a parameter), then the ops of U_k^dag.  Within a run of
// diagonal gates (diagonal generators and inverses: RZ, P, CP, RZZ, CRZ and
// the fixed phase gates) the gradient ops of the whole run come first: the
// run's inverses are diagonal unitaries applied to both states, which leave
// every Im(conj(lambda_s) psi_s) unchanged, so the gradients are the same at
// any point of the run; the run's phase ops then stand next to each other
// and merge into one op.  factor[slot] is the generator factor times
// |zeta|^2 at the gradient op's execution point.
static lq_status build_sweep(int n, const lq_gate* gates, int ng, const double* params,
                             std::vector<LOp>& ops, std::vector<double>& factor,
                             std::vector<int>& slot_param, Schedule& S, int tile_bits) {
  lq_status st;
  ops.clear();
  factor.clear();
  slot_param.clear();
  ops.reserve((std::size_t)ng * 2 + 8);
  std::vector<LOp> run_grads, run_ops;   // the current run of diagonal gates
  auto flush = [&]() {
    ops.insert(ops.end(), run_grads.begin(), run_grads.end());
    ops.insert(ops.end(), run_ops.begin(), run_ops.end());
    run_grads.clear();
    run_ops.clear();
  };
  double zr = 1, zi = 0;
  for (int gi = ng - 1; gi >= 0; gi--) {
    const lq_gate& G = gates[gi];
    double th = G.angle + (G.param >= 0 ? params[G.param] : 0.0);
    lq_gate inv = inverse_gate(G);
    Lowered L;
    st = lower_gate(inv, n, -th, L);
    if (st) return st;
    bool diagonal = true;
    for (int j = 0; j < L.nops; j++) diagonal = diagonal && L.op[j].mix() == 0;
    LOp go;
    if (G.param >= 0) {
      double fgen;
      go = grad_op(G, n, &fgen);
      go.slot = (int)factor.size();
      go.gate = gi;
      go.a = fgen;   // the |zeta|^2 part is added in execution order below
      factor.push_back(fgen);
      slot_param.push_back(G.param);
      diagonal = diagonal && go.x == 0;
    }
    if (!diagonal) flush();
    std::vector<LOp>& dst = diagonal ? run_ops : ops;
    if (G.param >= 0) (diagonal ? run_grads : ops).push_back(go);
    for (int j = 0; j < L.nops; j++) {
      L.op[j].gate = gi;
      if (j == 0) {
        L.op[j].fr = L.zr;
        L.op[j].fi = L.zi;
      }
      dst.push_back(L.op[j]);
    }
    double nr = zr * L.zr - zi * L.zi, ni = zr * L.zi + zi * L.zr;
    zr = nr;
    zi = ni;
    double mag = std::hypot(zr, zi);
    if (mag < 1e-100 || mag > 1e100) {
      LOp sc;
      sc.type = OP_SCALE;
      sc.mode = 1;
      sc.a = mag;
      sc.fr = 1.0 / mag;
      dst.push_back(sc);
      zr /= mag;
      zi /= mag;
    }
  }
  flush();
  ScheduleOptions sopt;
  sopt.k = tile_bits;
  // with two 32 KiB tiles, 56 gradient sums (8 warps, 3.5 KiB) keep three
  // CTAs resident per SM; smaller tiles leave room for a pass's every op
  sopt.max_grads = tile_bits >= 11 ? 56 : MAX_OPS;
  st = schedule_ops(n, ops.data(), ops.size(), zr, zi, sopt, S);
  if (st) return st;
  // A gradient op sees the states divided by the deferred scalar accumulated
  // over the ops executed before it; the scheduler may reorder commuting
  // ops, so accumulate in execution order.
  {
    double ar = 1, ai = 0;
    for (int ps = 0; ps < S.npasses; ps++)
      for (const LOp& l : S.pass_ops[ps]) {
        if (l.type == OP_GRAD) {
          factor[l.slot] = l.a * (ar * ar + ai * ai);
        } else if (!(l.type == OP_SCALE && (l.mode & 2))) {
          double nr2 = ar * l.fr - ai * l.fi, ni2 = ar * l.fi + ai * l.fr;
          ar = nr2;
          ai = ni2;
        }
      }
  }
  return LQ_OK;
}

}  // namespace lq

using namespace lq;

extern "C" {

lq_status lq_adjoint_plan(int n, const lq_gate* gates, int ng, const double* params, int np,
                          int nt, lq_plan_info* out) {
  lq_status st = check_n(n);
  if (st) return st;
  if (!out) return fail(LQ_ERR_INVALID_ARG, "out is NULL");
  st = check_gates(n, gates, ng, params, np);
  if (st) return st;
  lq_plan_info fwd;
  st = lq_circuit_plan(n, gates, ng, params, np, &fwd);
  if (st) return st;
  std::vector<LOp> ops;
  std::vector<double> factor;
  std::vector<int> slot_param;
  Schedule S;
  st = build_sweep(n, gates, ng, params, ops, factor, slot_param, S, sweep_tile_bits(n));
  if (st) return st;
  double fl = fwd.dp_flops;
  const double N = std::ldexp(1.0, n);
  int rev = 0;
  for (int p = 0; p < S.npasses; p++) {
    int nops = S.passes[p].h.nops;
    if (p == S.npasses - 1 && nops > 0 && S.passes[p].ops[nops - 1].type == OP_SCALE &&
        (S.passes[p].ops[nops - 1].mode & 2))
      nops--;
    if (nops == 0) continue;
    rev++;
    const std::vector<LOp>& L = S.pass_ops[p];
    for (std::size_t i = 0; i < L.size(); i++) {
      const LOp& l = L[i];
      if (l.type == OP_GRAD && l.x == 0 && (l.mode & 3) == 0 && S.passes[p].h.k <= 11) {
        // a run of diagonal generators: q_s (3 flops) and the Walsh-Hadamard
        // transform over a thread's 8 amplitudes (3 adds) per amplitude
        while (i + 1 < L.size() && L[i + 1].type == OP_GRAD && L[i + 1].x == 0 &&
               (L[i + 1].mode & 3) == 0)
          i++;
        fl += 6.0 * N;
      } else if (l.type == OP_GRAD) {
        fl += op_flops(l, n);
      } else if (l.type == OP_LPHASE && !(l.mode & LP_TABLE)) {
        fl += op_flops(l, n) + 6.0 * N;   // one phase per amplitude, two multiplies
      } else {
        fl += 2.0 * op_flops(l, n);
      }
    }
  }
  const int chunks = nt > 0 ? (nt + EXP_MAX_TERMS - 1) / EXP_MAX_TERMS : 0;
  // init, forward passes, <H> (2 per chunk), H psi (1 per chunk), reverse
  // passes, gradient reduction
  out->npasses = 1 + fwd.npasses + 2 * chunks + chunks + rev + (np > 0 ? 1 : 0);
  out->tile_bits = fwd.tile_bits;
  out->dp_flops = fl;
  out->dram_bytes = fwd.dram_bytes + 64.0 * std::ldexp(1.0, n) * rev;
  return LQ_OK;
}

size_t lq_adjoint_workspace_size(int n, int ng, int np, int nt) {
  if (n < 1 || n > 34 || ng < 0 || np < 0) return 0;
  int k = n < 10 ? n : 10;
  int grid = pass2_grid(n, k);
  std::size_t slots = (std::size_t)ng;   // at most one gradient op per gate
  return 2 * align256(sizeof(double2) << n) + align256(sizeof(double) * slots * grid) +
         align256(sizeof(double) * (slots + 1)) + 2 * align256(sizeof(int) * (np + 1)) +
         align256(sizeof(double) * (np + 1)) + lq_expval_workspace_size(n, nt);
}

lq_status lq_adjoint_grad(int n, const lq_gate* gates, int ng, const double* params, int np,
                          const lq_pauli_term* terms, int nt, double* energy, double* grad,
                          void* workspace, size_t ws_bytes, lq_stream stream) {
  lq_status st = check_n(n);
  if (st) return st;
  st = check_gates(n, gates, ng, params, np);
  if (st) return st;
  st = check_terms(n, terms, nt);
  if (st) return st;
  if (!energy || (np > 0 && !grad)) return fail(LQ_ERR_INVALID_ARG, "NULL output");
  std::size_t need = lq_adjoint_workspace_size(n, ng, np, nt);
  if (!workspace || ws_bytes < need)
    return fail(LQ_ERR_OOM, "workspace too small: %zu < %zu", ws_bytes, need);
  cudaStream_t s = (cudaStream_t)stream;
  const std::size_t sb = sizeof(double2) << n;
  const int grid = pass2_grid(n, n < 10 ? n : 10);   // stride of the partial sums

  // workspace layout
  char* p = (char*)workspace;
  double2* psi = (double2*)p;
  p += align256(sb);
  double2* lam = (double2*)p;
  p += align256(sb);
  double* partial = (double*)p;
  p += align256(sizeof(double) * (std::size_t)ng * grid);
  double* d_factor = (double*)p;
  p += align256(sizeof(double) * ((std::size_t)ng + 1));
  int* d_first = (int*)p;
  p += align256(sizeof(int) * (np + 1));
  int* d_count = (int*)p;
  p += align256(sizeof(int) * (np + 1));
  double* d_out = (double*)p;   // [0] = E, [1..np] = grad
  p += align256(sizeof(double) * (np + 1));
  char* ews = p;
  std::size_t ews_bytes = ws_bytes - (std::size_t)(p - (char*)workspace);

  // forward: psi_L = U|0>, E = <H>, lambda = H psi_L
  st = lq_state_init(psi, n, 0, stream);
  if (st) return st;
  st = lq_apply_circuit(psi, n, gates, ng, params, np, stream);
  if (st) return st;
  st = lq_expval_pauli_sum_async(psi, n, terms, nt, d_out, ews, ews_bytes, stream);
  if (st) return st;
  st = lq_apply_pauli_sum(lam, psi, n, terms, nt, stream);
  if (st) return st;

  std::vector<LOp> ops;
  std::vector<double> factor;
  std::vector<int> slot_param;
  Schedule S;
  st = build_sweep(n, gates, ng, params, ops, factor, slot_param, S, sweep_tile_bits(n));
  if (st) return st;
  const int nslots = (int)factor.size();
  // slots grouped by parameter, in slot order
  std::vector<int> first((std::size_t)np + 1, 0), count((std::size_t)np + 1, 0);
  std::vector<int> order;
  std::vector<double> fsorted;
  for (int pi = 0; pi < np; pi++) {
    first[pi] = (int)order.size();
    for (int sl = 0; sl < nslots; sl++)
      if (slot_param[sl] == pi) {
        order.push_back(sl);
        fsorted.push_back(factor[sl]);
      }
    count[pi] = (int)order.size() - first[pi];
  }
  // renumber slots so each parameter's slots are contiguous
  std::vector<int> newslot((std::size_t)nslots + 1, 0);
  for (std::size_t i = 0; i < order.size(); i++) newslot[order[i]] = (int)i;
  // renumber the gradient ops inside the scheduled passes
  for (int ps = 0; ps < S.npasses; ps++)
    for (int o = 0; o < S.passes[ps].h.nops; o++)
      if (S.passes[ps].ops[o].type == OP_GRAD)
        S.passes[ps].ops[o].cidx = (uint32_t)newslot[S.passes[ps].ops[o].cidx];
  if (nslots > 0) {
    LQ_CUDA(cudaMemsetAsync(partial, 0, sizeof(double) * (std::size_t)nslots * grid, s));
    LQ_CUDA(cudaMemcpyAsync(d_factor, fsorted.data(), sizeof(double) * nslots,
                            cudaMemcpyHostToDevice, s));
  }
  if (np > 0) {
    LQ_CUDA(cudaMemcpyAsync(d_first, first.data(), sizeof(int) * np, cudaMemcpyHostToDevice, s));
    LQ_CUDA(cudaMemcpyAsync(d_count, count.data(), sizeof(int) * np, cudaMemcpyHostToDevice, s));
  }
  for (int ps = 0; ps < S.npasses; ps++) {
    // the final scale would only rescale the uncomputed states: drop it
    PassParams& P = S.passes[ps];
    if (ps == S.npasses - 1 && P.h.nops > 0 && P.ops[P.h.nops - 1].type == OP_SCALE &&
        (P.ops[P.h.nops - 1].mode & 2))
      P.h.nops--;
    if (P.h.nops == 0) continue;
    LQ_CUDA(launch_pass2(P, psi, lam, partial, grid, s));
  }
  LQ_CUDA(launch_grad_reduce(partial, grid, d_factor, d_first, d_count, np, d_out + 1, s));
  std::vector<double> h((std::size_t)np + 1);
  LQ_CUDA(cudaMemcpyAsync(h.data(), d_out, sizeof(double) * (np + 1), cudaMemcpyDeviceToHost, s));
  LQ_CUDA(cudaStreamSynchronize(s));
  *energy = h[0];
  for (int i = 0; i < np; i++) grad[i] = h[1 + i];
  return LQ_OK;
}

}  // extern "C"
