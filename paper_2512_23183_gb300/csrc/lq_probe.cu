// lq_probe.cu -- measured FP64 FMA throughput of the current device.
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

}  // namespace lq

using namespace lq;

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
  cudaEvent_t a = nullptr, b = nullptr;
  if ((e = cudaEventCreate(&a)) != cudaSuccess || (e = cudaEventCreate(&b)) != cudaSuccess) {
    if (a) cudaEventDestroy(a);
    (void)cudaGetLastError();
    return fail(LQ_ERR_CUDA, "event: %s", cudaGetErrorString(e));
  }
  fp64_fma_probe_kernel<<<grid, kProbeBlock, 0, s>>>(0.9999999, 1e-3);   // warm-up
  float best = 0;
  for (int r = 0; r < reps && e == cudaSuccess; r++) {
    e = cudaEventRecord(a, s);
    fp64_fma_probe_kernel<<<grid, kProbeBlock, 0, s>>>(0.9999999, 1e-3);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(b, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float t = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
    if (e == cudaSuccess && (r == 0 || t < best)) best = t;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(LQ_ERR_CUDA, "fp64 probe: %s", cudaGetErrorString(e));
  }
  const double flops = 2.0 * kProbeChains * (double)kProbeIters * grid * kProbeBlock;
  *tflops = flops / (best * 1e-3) / 1e12;
  if (ms_best) *ms_best = best;
  return LQ_OK;
}
