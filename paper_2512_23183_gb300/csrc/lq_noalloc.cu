// lq_noalloc.cu -- <H> for callers that cannot allocate device memory.
//
// lq_expval_pauli_sum needs a small device workspace for its per-block
// partial sums, which the caller normally provides (cudaMalloc, a torch
// tensor, a pool allocator).  Some callers cannot allocate device memory at
// all: code embedded in a host application whose device memory belongs to an
// allocator it has no access to, plugins that are handed only the state's
// pointer, or loops that must not allocate.  lq_expval_pauli_sum_noalloc
// serves them: its scratch is one array compiled into this library
// (`g_noalloc_scratch`, 4096 doubles = 32 KiB), which every GPU that loads
// the library holds until the process exits.
//
// In host code the array's name is only a host-side stand-in for the
// symbol, not a device address, so the address is fetched with
// cudaGetSymbolAddress once per device (with that device current) on the
// first call on that device, and cached.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "lq_internal.h"
#include "lq_kernels.h"

namespace lq {

constexpr int NOALLOC_DOUBLES = 4096;   // [0] result, [1..] per-block partial sums
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_DOUBLES];

static double* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {nullptr};
static std::mutex g_noalloc_mu;
static ExpParams g_noalloc_terms;   // host staging of the grouped terms (under the mutex)

// Group the terms by X mask into one ExpParams without any heap allocation
// (an insertion sort of term indices on the stack).  nt <= EXP_MAX_TERMS.
static void group_terms_fixed(int n, const lq_pauli_term* terms, int nt, ExpParams& E) {
  int order[EXP_MAX_TERMS];
  for (int t = 0; t < nt; t++) {
    int j = t;
    while (j > 0 && terms[order[j - 1]].xmask > terms[t].xmask) {
      order[j] = order[j - 1];
      j--;
    }
    order[j] = t;
  }
  std::memset(&E, 0, sizeof E);
  E.n = n;
  for (int i = 0; i < nt; i++) {
    const lq_pauli_term& P = terms[order[i]];
    if (E.ngroups == 0 || E.groups[E.ngroups - 1].x != P.xmask) {
      ExpGroup& G = E.groups[E.ngroups++];
      G.x = P.xmask;
      G.h = P.xmask ? 63 - __builtin_clzll(P.xmask) : 0;
      G.first = i;
      G.count = 0;
    }
    ExpTerm& T = E.terms[i];
    T.c = P.coeff;
    T.c2 = 2.0 * P.coeff;
    T.z = P.zmask;
    T.k0 = __builtin_popcountll(P.xmask & P.zmask) & 3;
    E.groups[E.ngroups - 1].count++;
  }
}

}  // namespace lq

using namespace lq;

extern "C" lq_status lq_expval_pauli_sum_noalloc(const void* amps, int n,
                                                 const lq_pauli_term* terms, int nt,
                                                 double* out, lq_stream stream) {
  lq_status st = check_n(n);
  if (st) return st;
  if (!amps || !out) return fail(LQ_ERR_INVALID_ARG, "NULL pointer");
  st = check_terms(n, terms, nt);
  if (st) return st;
  if (nt > EXP_MAX_TERMS)
    return fail(LQ_ERR_INVALID_ARG,
                "lq_expval_pauli_sum_noalloc takes at most %d terms (got %d); use "
                "lq_expval_pauli_sum with a workspace", EXP_MAX_TERMS, nt);
  // distinct X masks also bound the group table
  {
    int groups = 0;
    for (int t = 0; t < nt; t++) {
      bool seen = false;
      for (int u = 0; u < t && !seen; u++) seen = terms[u].xmask == terms[t].xmask;
      groups += !seen;
    }
    if (groups > EXP_MAX_GROUPS)
      return fail(LQ_ERR_INVALID_ARG,
                  "lq_expval_pauli_sum_noalloc takes at most %d distinct X masks (got %d)",
                  EXP_MAX_GROUPS, groups);
  }
  const int grid = expval_grid(n);
  if (1 + grid > NOALLOC_DOUBLES)
    return fail(LQ_ERR_INVALID_ARG,
                "fixed scratch holds %d partial sums, this device needs %d", NOALLOC_DOUBLES - 1,
                grid);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(LQ_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  }
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES)
    return fail(LQ_ERR_INVALID_ARG, "device %d beyond the %d supported", dev, NOALLOC_MAX_DEVICES);
  cudaStream_t s = (cudaStream_t)stream;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      // first call on this device: resolve the array's device address
      e = cudaGetSymbolAddress((void**)&g_noalloc_ptr[dev], g_noalloc_scratch);
      if (e != cudaSuccess) {
        g_noalloc_ptr[dev] = nullptr;
        (void)cudaGetLastError();
        return fail(LQ_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      }
    }
    double* d_out = g_noalloc_ptr[dev];
    double* partial = d_out + 1;
    if (nt == 0) {
      e = cudaMemsetAsync(d_out, 0, sizeof(double), s);
    } else {
      // every block overwrites its partial sum and the result slot is
      // written (not accumulated), so nothing in the array has to start at
      // zero; the kernel parameters are copied at launch, so the staging
      // buffer is free again once the launch returns
      group_terms_fixed(n, terms, nt, g_noalloc_terms);
      e = launch_expval(g_noalloc_terms, (const double2*)amps, 0, 1, partial, d_out, 0, s);
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(out, d_out, sizeof(double), cudaMemcpyDeviceToHost, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(LQ_ERR_CUDA, "noalloc <H>: %s", cudaGetErrorString(e));
  }
  return LQ_OK;
}
