// lq_probe.cu -- measured FP64 throughput of the current device: DFMA alone,
// and DFMA in the shared-memory tile sweeps the state-vector passes run.
//
// Every state-vector kernel of this library is bound by FP64 issue (a pass
// over a complex128 state needs more FP64 instructions per amplitude than
// the HBM time of its 32 bytes allows), so their roofline denominator is the
// device's FP64 FMA rate.  GB300's FP64 rate is far below its FP32 and
// tensor rates and is not a published constant of the part, so it is
// measured where the kernels run: independent DFMA chains, no memory
// traffic, every SM filled, timed with CUDA events on the caller's stream.
#include <cuda_runtime.h>

#include <cstdint>

#include "lq_internal.h"
#include "lq_kernels.h"

namespace lq {

constexpr int kProbeChains = 8;     // independent FMA chains per thread
constexpr int kProbeIters = 4096;   // FMAs per chain
constexpr int kProbeBlock = 256;

static __device__ double g_probe_sink;

// x <- x * y + z converges to z / (1 - y) (|y| < 1), so the chains stay
// finite and normal; the sum is stored only when it is impossible in
// practice, which keeps the loop live without memory traffic.
__global__ void __launch_bounds__(kProbeBlock) fp64_fma_probe_kernel(double y, double z) {
  double x[kProbeChains];
#pragma unroll
  for (int c = 0; c < kProbeChains; c++) x[c] = (double)(threadIdx.x + c);
  for (int i = 0; i < kProbeIters; i++) {
#pragma unroll
    for (int c = 0; c < kProbeChains; c++) x[c] = fma(x[c], y, z);
  }
  double s = 0;
#pragma unroll
  for (int c = 0; c < kProbeChains; c++) s += x[c];
  if (s == -1.0) g_probe_sink = s;
}

// Tile-sweep probe: the access pattern of every state-sized pass without
// its global traffic.  Each CTA keeps a 2^12-amplitude tile in shared memory
// and applies tangent-form rotations (a' = a - t b, b' = b + t a: 4 FMAs per
// pair) on tile bits 0, 1, ..., 11 in turn, one sweep per bit with a barrier
// after each: two loads, four FMAs and two stores per pair, as in the tile
// ops.  t is small, so the values stay finite.
constexpr int kSweepBits = 12;
constexpr int kSweepRounds = 200;    // sweeps = kSweepRounds * kSweepBits

__global__ void __launch_bounds__(kProbeBlock) fp64_sweep_probe_kernel(double t) {
  extern __shared__ double2 tile[];
  constexpr uint32_t T = 1u << kSweepBits;
  for (uint32_t s = threadIdx.x; s < T; s += kProbeBlock)
    tile[s] = make_double2(1.0 + 1e-3 * s, 0.5 - 1e-3 * s);
  __syncthreads();
  for (int r = 0; r < kSweepRounds; r++) {
    for (int b = 0; b < kSweepBits; b++) {
      const uint32_t xb = 1u << b;
      for (uint32_t j = threadIdx.x; j < T / 2; j += kProbeBlock) {
        const uint32_t lo = j & (xb - 1u), s0 = ((j - lo) << 1) | lo, s1 = s0 | xb;
        const double2 A = tile[s0], B = tile[s1];
        tile[s0] = make_double2(fma(-t, B.x, A.x), fma(-t, B.y, A.y));
        tile[s1] = make_double2(fma(t, A.x, B.x), fma(t, A.y, B.y));
      }
      __syncthreads();
    }
  }
  if (tile[threadIdx.x].x == -1.0) g_probe_sink = tile[threadIdx.x].y;
}

}  // namespace lq

using namespace lq;

namespace {

// Best of `reps` timed launches (after one warm-up) of launch() on s.
template <typename F>
cudaError_t best_launch_ms(int reps, cudaStream_t s, F launch, float* best) {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e;
  if ((e = cudaEventCreate(&a)) != cudaSuccess || (e = cudaEventCreate(&b)) != cudaSuccess) {
    if (a) cudaEventDestroy(a);
    return e;
  }
  launch();
  e = cudaGetLastError();
  *best = 0;
  for (int r = 0; r < reps && e == cudaSuccess; r++) {
    e = cudaEventRecord(a, s);
    launch();
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(b, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float t = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
    if (e == cudaSuccess && (r == 0 || t < *best)) *best = t;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return e;
}

}  // namespace

extern "C" lq_status lq_measure_fp64_fma(int reps, double* tflops, double* ms_best,
                                         lq_stream stream) {
  if (!tflops) return fail(LQ_ERR_INVALID_ARG, "tflops is NULL");
  if (reps < 1 || reps > 1000) return fail(LQ_ERR_INVALID_ARG, "reps %d not in [1, 1000]", reps);
  (void)cudaGetLastError();
  cudaStream_t s = (cudaStream_t)stream;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fp64_fma_probe_kernel,
                                                                kProbeBlock, 0);
  if (e != cudaSuccess) return fail(LQ_ERR_CUDA, "occupancy: %s", cudaGetErrorString(e));
  const int grid = sm_count() * (per_sm > 0 ? per_sm : 1);
  float best = 0;
  e = best_launch_ms(reps, s, [&] {
    fp64_fma_probe_kernel<<<grid, kProbeBlock, 0, s>>>(0.9999999, 1e-3);
  }, &best);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(LQ_ERR_CUDA, "fp64 probe: %s", cudaGetErrorString(e));
  }
  const double flops = 2.0 * kProbeChains * (double)kProbeIters * grid * kProbeBlock;
  *tflops = flops / (best * 1e-3) / 1e12;
  if (ms_best) *ms_best = best;
  return LQ_OK;
}

extern "C" lq_status lq_measure_fp64_tile_sweep(int reps, double* tflops, double* ms_best,
                                                lq_stream stream) {
  if (!tflops) return fail(LQ_ERR_INVALID_ARG, "tflops is NULL");
  if (reps < 1 || reps > 1000) return fail(LQ_ERR_INVALID_ARG, "reps %d not in [1, 1000]", reps);
  (void)cudaGetLastError();
  cudaStream_t s = (cudaStream_t)stream;
  const size_t smem = sizeof(double2) << kSweepBits;
  cudaError_t e = cudaFuncSetAttribute(fp64_sweep_probe_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fp64_sweep_probe_kernel,
                                                      kProbeBlock, smem);
  if (e != cudaSuccess) return fail(LQ_ERR_CUDA, "sweep probe set-up: %s", cudaGetErrorString(e));
  const int grid = sm_count() * (per_sm > 0 ? per_sm : 1);
  float best = 0;
  e = best_launch_ms(reps, s, [&] {
    fp64_sweep_probe_kernel<<<grid, kProbeBlock, smem, s>>>(1e-3);
  }, &best);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(LQ_ERR_CUDA, "sweep probe: %s", cudaGetErrorString(e));
  }
  const double flops = 2.0 * 4 * (double)(1u << (kSweepBits - 1)) * kSweepRounds * kSweepBits * grid;
  *tflops = flops / (best * 1e-3) / 1e12;
  if (ms_best) *ms_best = best;
  return LQ_OK;
}
