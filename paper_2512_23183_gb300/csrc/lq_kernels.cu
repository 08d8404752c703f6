// lq_kernels.cu -- state initialisation, the shared-memory tile-pass kernel
// that executes lowered gate ops (Sec. IV-A direct state-vector updates, Alg. 1,
// Alg. 4), and the Pauli-sum kernels (<H>, H psi; Sec. VI-A, Sec. VII-A-2).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "lq_device.cuh"
#include "lq_kernels.h"

namespace lq {

// ------------------------------------------------------------------ init

__global__ void init_basis_kernel(double2* __restrict__ amps, uint64_t N, uint64_t basis) {
  uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (; i < N; i += stride) amps[i] = make_double2(i == basis ? 1.0 : 0.0, 0.0);
}

cudaError_t launch_init_basis(double2* amps, int n, uint64_t basis, cudaStream_t s) {
  (void)cudaGetLastError();  // report only this launcher's own errors
  uint64_t N = 1ull << n;
  uint64_t blocks = (N + 255) / 256;
  int grid = (int)(blocks < (uint64_t)sm_count() * 16 ? blocks : (uint64_t)sm_count() * 16);
  init_basis_kernel<<<grid, 256, 0, s>>>(amps, N, basis);
  return cudaGetLastError();
}

// ---------------------------------------------------- dyadic phase tables

// g_dyadic[h] = exp(2 pi i h / 2^17), g_dyadic[2^17 + l] = exp(2 pi i l / 2^34),
// so exp(2 pi i E / 2^34) = g_dyadic[E >> 17] * g_dyadic[2^17 + (E & (2^17-1))].
__device__ double2 g_dyadic[2 << DYADIC_HALF];

__global__ void dyadic_table_kernel() {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (2u << DYADIC_HALF)) return;
  const uint32_t j = i & ((1u << DYADIC_HALF) - 1u);
  // angle / pi = 2 j / 2^17 (high table) or 2 j / 2^34 (low table), exact
  const double x = (i >> DYADIC_HALF) ? std::ldexp((double)j, 1 - DYADIC_BITS)
                                      : std::ldexp((double)j, 1 - DYADIC_HALF);
  double sn, cs;
  sincospi(x, &sn, &cs);
  g_dyadic[i] = make_double2(cs, sn);
}

// Constant device tables (the dyadic phase tables here, the FFT twiddles of
// the QFT) are filled once per device before the first kernel that reads them
// is enqueued.  The fill runs under a mutex on a private non-blocking stream
// and only that stream is synchronised, so other streams keep running and a
// caller's stream capture is not disturbed; the device is marked done only
// after the fill has completed, so a launch enqueued on any stream after the
// mark (or after another thread's fill returned) reads a finished table.  A
// first fill requested from a stream that is being captured is refused, since
// the caller would then record kernels that read a table this call has not
// filled yet.
cudaError_t fill_table_once(TableOnce& t, const cudaStream_t* caller,
                            cudaError_t (*fill)(cudaStream_t)) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  const uint64_t bit = 1ull << dev;
  if (t.done.load(std::memory_order_acquire) & bit) return cudaSuccess;
  if (caller) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(*caller, &cs);
    if (e != cudaSuccess) return e;
    if (cs != cudaStreamCaptureStatusNone) return cudaErrorStreamCaptureUnsupported;
  }
  std::lock_guard<std::mutex> lock(t.mu);
  if (t.done.load(std::memory_order_acquire) & bit) return cudaSuccess;
  cudaStream_t ps = nullptr;
  e = cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  e = fill(ps);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ps);
  cudaStreamDestroy(ps);
  if (e == cudaSuccess) t.done.fetch_or(bit, std::memory_order_release);
  return e;
}

static cudaError_t fill_dyadic(cudaStream_t ps) {
  dyadic_table_kernel<<<(2u << DYADIC_HALF) / 256, 256, 0, ps>>>();
  return cudaGetLastError();
}

// Device address of the tables of the current device, filling them on first
// use (see fill_table_once).
const double2* dyadic_tables(cudaError_t* err, const cudaStream_t* caller) {
  static TableOnce once;
  static std::atomic<const double2*> ptr[64];
  int dev = 0;
  *err = cudaGetDevice(&dev);
  if (*err != cudaSuccess) return nullptr;
  if (dev < 0 || dev >= 64) {
    *err = cudaErrorInvalidDevice;
    return nullptr;
  }
  const double2* p = ptr[dev].load(std::memory_order_acquire);
  if (p) return p;
  *err = fill_table_once(once, caller, fill_dyadic);
  if (*err != cudaSuccess) return nullptr;
  void* a = nullptr;
  *err = cudaGetSymbolAddress(&a, g_dyadic);
  if (*err != cudaSuccess) return nullptr;
  ptr[dev].store((const double2*)a, std::memory_order_release);
  return (const double2*)a;
}

// ----------------------------------------------------------- tile passes

// One CTA processes tiles w = blockIdx.x, blockIdx.x + gridDim.x, ... of the
// `nstates` states (stride `stride` amplitudes apart); a tile is the 2^k
// amplitudes base | deposit(s, tbits), s < 2^k.  Tile loads and stores are
// coalesced runs of 2^m contiguous amplitudes.  With `dbuf`, the next tile is
// copied into a second buffer (cp.async) while the current one is computed,
// so the CTAs of an SM do not all wait on HBM at the same time.  With
// PF_LTAB, the phase table of the pass's table-mode OP_LPHASE (every factor
// on a tile bit) is built once per CTA, after the tile buffers, and serves
// every tile.
// Deferred per-tile phase table of a pass: dD[v] = exp(2 pi i E(v) / 2^34),
// E(v) = sum of the deferred sums (the pre-load ones, or the store ones) whose
// conditions the index-bit pattern v meets; with PF_DSCALE, times the
// circuit's final scalar in the table applied first (the pre-load one when
// the pass has one).  No barrier.
template <int BLOCK>
__device__ __forceinline__ void build_deferred(double2* dD, const PassHeader& h,
                                               const double* __restrict__ coef,
                                               const unsigned long long* dfe, bool pre) {
  const unsigned long long M34 = (1ull << DYADIC_BITS) - 1ull;
  const bool scaled = (h.flags & PF_DSCALE) && (pre || h.dpre == 0);
  for (uint32_t v = threadIdx.x; v < (1u << h.ndbits); v += BLOCK) {
    unsigned long long E = 0;
    for (int q = 0; q < h.ndefer; q++)
      if ((((h.dpre >> q) & 1) != 0) == pre && (v & h.dmask[q]) == h.dval[q]) E += dfe[q];
    const double2 w = dyadic_phase(E & M34, (const double2*)h.dtab);
    dD[v] = scaled ? cmul(w, coef[h.dsc], coef[h.dsc + 1]) : w;
  }
}

// BF: the pass has DP_BFLY ops (separate instantiation, so the other passes
// keep their code and registers).
template <int BLOCK, bool BF>
__global__ void __launch_bounds__(BLOCK, 4) pass_kernel(const __grid_constant__ PassParams P,
                                                        double2* __restrict__ state,
                                                        uint64_t stride, int nstates, int dbuf) {
  extern __shared__ double2 smem_tiles[];
  __shared__ uint32_t hioff[1 << PASS_HI_BITS];   // high tile bits' global offsets >> m
  const int k = P.h.k, m = P.h.m, nops = P.h.nops;
  const uint32_t T = 1u << k;
  const uint32_t lowmask = (1u << m) - 1u;
  const int kh = k - m;
  for (uint32_t j = threadIdx.x; j < (1u << kh); j += BLOCK)
    hioff[j] = (uint32_t)(deposit(j, P.h.tbits + m, kh) >> m);
  // dynamic shared memory: tile buffer(s), [phase table], [dyadic partial
  // sums], [full dyadic phase tables]
  __shared__ unsigned long long dfe[8];   // this tile's deferred dyadic sums
  __shared__ double2 dD[64];              // this tile's deferred phase table
  PassTables tabs = {nullptr, nullptr, nullptr, dfe};
  double2* area = smem_tiles + (dbuf ? 2 * T : T);
  if (P.h.flags & PF_LTAB) {
    build_lphase_table<BLOCK>(area, k, P.ops[P.h.ltab_op], P.coef);
    tabs.ltab = area;
    area += T;
  }
  // full-mode ops build their partial sums in the tile buffer (slot b0),
  // which is not in use before the first tile
  unsigned long long* scratch_tabs = reinterpret_cast<unsigned long long*>(smem_tiles);
  if (P.h.flags & PF_DTAB) {
    unsigned long long* d = reinterpret_cast<unsigned long long*>(area);
    for (int o = 0; o < nops; o++) {
      const Op& op = P.ops[o];
      if (op.type != OP_DPHASE || !(op.mode & DP_TABLE)) continue;
      if (op.mode & DP_FULL)
        build_dphase_table<BLOCK>(scratch_tabs + 256 * op.b0, d + op.z_loc, k, op, P.coef);
      else
        build_dphase_table<BLOCK>(d + op.z_loc, d + op.z_loc + 256, k, op, P.coef);
    }
    tabs.dpt = d;
    area += (P.h.dtab_words + 1) / 2;
  }
  const bool deferred = (P.h.flags & PF_DFULL) != 0;
  // deferred sums applied at the store (the others after the load)
  const bool post = deferred && ((((1u << P.h.ndefer) - 1u) & ~(uint32_t)P.h.dpre) != 0);
  if (deferred) {
    for (int o = 0; o < nops; o++)
      if (P.ops[o].type == OP_DPHASE && (P.ops[o].mode & DP_FULL))
        build_dfull_table<BLOCK>(area + P.ops[o].z_glob, k, P.ops[o],
                                 scratch_tabs + 256 * P.ops[o].b0, (const double2*)P.h.dtab);
    tabs.dfull = area;
  }
  const uint64_t ntiles = P.h.ntiles;
  const uint64_t total = ntiles * (uint64_t)nstates;
  const bool zero = (P.h.flags & PF_INIT_ZERO) != 0;
  const bool store = !(P.h.flags & PF_NO_STORE);
  __syncthreads();
  const int lgt = __ffsll((long long)ntiles) - 1;   // ntiles = 2^(n - k)
  auto tile_of = [&](uint64_t w, uint64_t* base) -> double2* {
    const uint64_t si = w >> lgt, t = w & (ntiles - 1ull);
    *base = deposit(t, P.h.obits, P.h.nobits);
    return state + si * stride;
  };
  auto issue = [&](uint64_t w, double2* buf) {
    uint64_t base;
    const double2* st = tile_of(w, &base);
    for (uint32_t s = threadIdx.x; s < T; s += BLOCK)
      cp_async16(buf + s, st + (base | ((uint64_t)hioff[s >> m] << m) | (s & lowmask)));
    cp_async_commit();
  };
  int cur = 0;
  if (dbuf && blockIdx.x < total) issue(blockIdx.x, smem_tiles);
  for (uint64_t w = blockIdx.x; w < total; w += gridDim.x, cur ^= 1) {
    double2* __restrict__ sm = smem_tiles + (dbuf ? cur * T : 0);
    uint64_t base;
    double2* __restrict__ st = tile_of(w, &base);
    // deferred sums applied after the load: they depend on the tile's CTA
    // bits alone, so their table is built before the load and applied to the
    // amplitudes as they arrive (a plain load; with zero-initialised tiles
    // and cp.async buffers, in a sweep after it)
    const bool pre = deferred && P.h.dpre;
    const bool pre_at_load = pre && !zero && !dbuf;
    if (threadIdx.x < 8 && !((P.h.dpre >> threadIdx.x) & 1u)) dfe[threadIdx.x] = 0;
    if (pre) {
      // per-tile parts hoisted to the load: warp w sums the (w mod 8)-th such
      // ops (0 where the op's CTA condition fails)
      int wi = 0;
      for (int o = 0; o < nops; o++) {
        const Op& d = P.ops[o];
        if (d.type != OP_DPHASE || !(d.mode & DP_PRE)) continue;
        if ((int)(threadIdx.x >> 5) == (wi++ % (BLOCK / 32))) {
          const unsigned long long e0 = (base & d.cm_glob) == d.cv_glob
                                            ? dphase_tile_sum(tabs.dpt + d.z_loc, (int)d.b1, base)
                                            : 0ull;
          if ((threadIdx.x & 31) == 0) dfe[d.b0] = e0;
        }
      }
      __syncthreads();
      build_deferred<BLOCK>(dD, P.h, P.coef, dfe, true);
      __syncthreads();
    }
    if (zero) {
      for (uint32_t s = threadIdx.x; s < T; s += BLOCK)
        sm[s] = make_double2((base == 0 && s == 0) ? 1.0 : 0.0, 0.0);
    } else if (dbuf) {
      if (w + gridDim.x < total) {
        issue(w + gridDim.x, smem_tiles + (cur ^ 1) * T);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
    } else {
      // the next tile's amplitude at the same tile index lies `ahead`
      // amplitudes further (its CTA bits replace this tile's): one L2 hint
      // per 128-byte line (or per run of 2^m amplitudes when runs are shorter)
      int64_t ahead = 0;
      if (w + gridDim.x < total) {
        uint64_t b2;
        const double2* st2 = tile_of(w + gridDim.x, &b2);
        ahead = (st2 + b2) - (st + base);
      }
      const uint32_t pmask = ahead ? (1u << (m < 3 ? m : 3)) - 1u : ~0u;
      if (pre_at_load) {
        const int nb = P.h.ndbits;
        for (uint32_t s = threadIdx.x; s < T; s += BLOCK) {
          const double2* src = st + (base | ((uint64_t)hioff[s >> m] << m) | (s & lowmask));
          uint32_t idx = 0;
          for (int i = 0; i < nb; i++) idx |= ((s >> P.h.dbits[i]) & 1u) << i;
          const double2 v = *src, wd = dD[idx];
          if ((s & pmask) == 0) prefetch_l2(src + ahead);
          sm[s] = cmul(v, wd.x, wd.y);
        }
      } else {
        for (uint32_t s = threadIdx.x; s < T; s += BLOCK) {
          const double2* src = st + (base | ((uint64_t)hioff[s >> m] << m) | (s & lowmask));
          sm[s] = *src;
          if ((s & pmask) == 0) prefetch_l2(src + ahead);
        }
      }
    }
    __syncthreads();
    if (pre && !pre_at_load) {
      const int nb = P.h.ndbits;
      for (uint32_t s = threadIdx.x; s < T; s += BLOCK) {
        uint32_t idx = 0;
        for (int i = 0; i < nb; i++) idx |= ((s >> P.h.dbits[i]) & 1u) << i;
        const double2 wd = dD[idx];
        sm[s] = cmul(sm[s], wd.x, wd.y);
      }
      __syncthreads();
    }
    for (int o = 0; o < nops; o++) {
      if constexpr (BF) {
        if (P.ops[o].type == OP_DPHASE && (P.ops[o].mode & DP_BFLY)) {
          dphase_bfly_pairs<BLOCK>(sm, T, P.ops[o], &tabs);   // with the H after it
          o++;
          __syncthreads();
          continue;
        }
      }
      apply_op<BLOCK>(sm, T, P.ops[o], P.coef, base, (const double2*)P.h.dtab, &tabs);
      __syncthreads();
    }
    if (post) {
      build_deferred<BLOCK>(dD, P.h, P.coef, dfe, false);
      __syncthreads();
    }
    if (store) {
      if (post) {
        const int nb = P.h.ndbits;
        for (uint32_t s = threadIdx.x; s < T; s += BLOCK) {
          uint32_t idx = 0;
          for (int i = 0; i < nb; i++) idx |= ((s >> P.h.dbits[i]) & 1u) << i;
          const double2 w = dD[idx];
          st[base | ((uint64_t)hioff[s >> m] << m) | (s & lowmask)] = cmul(sm[s], w.x, w.y);
        }
      } else {
        for (uint32_t s = threadIdx.x; s < T; s += BLOCK)
          st[base | ((uint64_t)hioff[s >> m] << m) | (s & lowmask)] = sm[s];
      }
    }
    __syncthreads();
  }
  if (dbuf) cp_async_wait<0>();
}

static constexpr int kPassBlock = 256;

cudaError_t launch_pass(const PassParams& P, double2* state, uint64_t stride, int nstates,
                        cudaStream_t s) {
  (void)cudaGetLastError();  // report only this launcher's own errors
  static std::atomic<uint64_t> configured{0};
  const size_t tile = sizeof(double2) << P.h.k;
  // double buffering for passes that load from HBM with tiles of <= 2^11
  const int dbuf = (P.h.k <= 11 && !(P.h.flags & (PF_INIT_ZERO | PF_DFULL))) ? 1 : 0;
  const size_t smem = tile * ((dbuf ? 2 : 1) + ((P.h.flags & PF_LTAB) ? 1 : 0)) +
                      ((P.h.flags & PF_DTAB) ? sizeof(double2) * ((P.h.dtab_words + 1) / 2) : 0) +
                      ((P.h.flags & PF_DFULL) ? sizeof(double2) * P.h.dfull_entries : 0);
  cudaError_t ce = once_per_device(configured, [] {
    cudaError_t e = cudaFuncSetAttribute(pass_kernel<kPassBlock, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(200u << 10));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(pass_kernel<kPassBlock, true>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(200u << 10));
    return e;
  });
  if (ce != cudaSuccess) return ce;
  uint64_t total = P.h.ntiles * (uint64_t)nstates;
  // resident CTAs per SM (the launch bound allows 4; dynamic and static
  // shared memory may allow fewer): a grid of more CTAs than fit would run
  // its last CTAs as a second wave.  Four CTAs with up to 46 KiB of dynamic
  // shared memory each always fit (static ~8 KiB and 1 KiB reserved per CTA
  // of 228 KiB); above that the occupancy query decides (it costs
  // microseconds, which launches on small states feel)
  int per_sm = 4;
  if (total > (uint64_t)sm_count() && smem > (46u << 10)) {
    int occ = 0;
    const bool bf = (P.h.flags & PF_DYADIC) && (P.h.flags & PF_BFLY);
    cudaError_t oe =
        bf ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pass_kernel<kPassBlock, true>,
                                                           kPassBlock, smem)
           : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pass_kernel<kPassBlock, false>,
                                                           kPassBlock, smem);
    if (oe != cudaSuccess) return oe;
    per_sm = occ < 1 ? 1 : occ > 4 ? 4 : occ;
  }
  uint64_t cap = (uint64_t)sm_count() * per_sm;
  int grid = (int)(total < cap ? total : cap);
  if (P.h.flags & PF_DYADIC) {
    cudaError_t e;
    const double2* t = dyadic_tables(&e, &s);
    if (!t) return e;
    static thread_local PassParams Q;   // launch copy carrying the table address
    Q = P;
    Q.h.dtab = t;
    if (P.h.flags & PF_BFLY)
      pass_kernel<kPassBlock, true><<<grid, kPassBlock, smem, s>>>(Q, state, stride, nstates, dbuf);
    else
      pass_kernel<kPassBlock, false><<<grid, kPassBlock, smem, s>>>(Q, state, stride, nstates, dbuf);
  } else {
    pass_kernel<kPassBlock, false><<<grid, kPassBlock, smem, s>>>(P, state, stride, nstates, dbuf);
  }
  return cudaGetLastError();
}


// ------------------------------------------------------------ Pauli sums

// <H> over grouped terms.  Terms sharing an X mask form a group; a group with
// x != 0 visits each unordered pair (i, i^x) once (i has the top bit of x
// clear) and adds 2 c_t Re(conj(psi_i) <i|P_t|i^x> psi_{i^x}); the x == 0 group
// adds c_t (-1)^popcount(i & z_t) |psi_i|^2.  <i|P|j> = i^k0 (-1)^popcount(j&z).
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) expval_kernel(const __grid_constant__ ExpParams E,
                                                       const double2* __restrict__ state,
                                                       uint64_t stride,
                                                       double* __restrict__ partial) {
  __shared__ double tab[((34 + EXP_CHUNK_BITS - 1) / EXP_CHUNK_BITS) * 256];
  const double2* __restrict__ st = state + blockIdx.y * stride;
  if (E.tables) expval_tables(tab, E.n, E.groups, E.ngroups, E.terms);
  __syncthreads();
  const uint64_t nthreads = (uint64_t)gridDim.x * BLOCK;
  const uint64_t t0 = blockIdx.x * (uint64_t)BLOCK + threadIdx.x;
  double acc = expval_partial(st, E.n, E.groups, E.ngroups, E.terms, t0, nthreads,
                              E.tables ? tab : nullptr);
  // block reduction in a fixed order
  __shared__ double red[BLOCK / 32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0;
    for (int w = 0; w < BLOCK / 32; w++) s += red[w];
    partial[blockIdx.y * gridDim.x + blockIdx.x] = s;
  }
}

// Sum the partials of each state in a fixed order (deterministic), add into
// out[state] when `accumulate`, else overwrite.
__global__ void sum_partials_kernel(const double* __restrict__ partial, int nparts,
                                    int nstates, double* __restrict__ out, int accumulate) {
  int sidx = blockIdx.x * blockDim.x + threadIdx.x;
  if (sidx >= nstates) return;
  double s = 0;
  for (int p = 0; p < nparts; p++) s += partial[(uint64_t)sidx * nparts + p];
  out[sidx] = accumulate ? out[sidx] + s : s;
}

cudaError_t launch_sum_partials(const double* partial, int nparts, int nstates, double* out,
                                int accumulate, cudaStream_t s) {
  sum_partials_kernel<<<(nstates + 127) / 128, 128, 0, s>>>(partial, nparts, nstates, out,
                                                             accumulate);
  return cudaGetLastError();
}

static constexpr int kExpBlock = 256;

int expval_grid(int n) {
  uint64_t pairs = 1ull << (n > 0 ? n - 1 : 0);
  uint64_t blocks = (pairs + kExpBlock - 1) / kExpBlock;
  uint64_t cap = (uint64_t)sm_count() * 4;
  return (int)(blocks < cap ? blocks : cap);
}

cudaError_t launch_expval(const ExpParams& E, const double2* state, uint64_t stride,
                          int nstates, double* partial, double* out, int accumulate,
                          cudaStream_t s) {
  (void)cudaGetLastError();  // report only this launcher's own errors
  int gx = expval_grid(E.n);
  dim3 grid(gx, nstates);
  expval_kernel<kExpBlock><<<grid, kExpBlock, 0, s>>>(E, state, stride, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  sum_partials_kernel<<<(nstates + 127) / 128, 128, 0, s>>>(partial, gx, nstates, out,
                                                             accumulate);
  return cudaGetLastError();
}

// out_i (+)= sum_t c_t <i|P_t|i^x> psi_{i^x}, i.e. out (+)= H psi, one element per
// thread iteration; `accumulate` adds into out (chunked term lists).
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) apply_pauli_sum_kernel(
    const __grid_constant__ ExpParams E, const double2* __restrict__ in,
    double2* __restrict__ out, int accumulate) {
  const uint64_t N = 1ull << E.n;
  const uint64_t nthreads = (uint64_t)gridDim.x * BLOCK;
  for (uint64_t i = blockIdx.x * (uint64_t)BLOCK + threadIdx.x; i < N; i += nthreads) {
    double re = 0, im = 0;
    if (accumulate) {
      double2 o = out[i];
      re = o.x;
      im = o.y;
    }
    for (int g = 0; g < E.ngroups; g++) {
      const ExpGroup G = E.groups[g];
      const uint64_t l = i ^ G.x;
      const double2 v = in[l];
      for (int t = G.first; t < G.first + G.count; t++) {
        int kk = (E.terms[t].k0 + 2 * (__popcll(l & E.terms[t].z) & 1)) & 3;
        double2 w = mul_ipow(v, kk);
        re = fma(E.terms[t].c, w.x, re);
        im = fma(E.terms[t].c, w.y, im);
      }
    }
    out[i] = make_double2(re, im);
  }
}

cudaError_t launch_apply_pauli_sum(const ExpParams& E, const double2* in, double2* out,
                                   int accumulate, cudaStream_t s) {
  (void)cudaGetLastError();  // report only this launcher's own errors
  uint64_t N = 1ull << E.n;
  uint64_t blocks = (N + 255) / 256;
  uint64_t cap = (uint64_t)sm_count() * 8;
  int grid = (int)(blocks < cap ? blocks : cap);
  apply_pauli_sum_kernel<256><<<grid, 256, 0, s>>>(E, in, out, accumulate);
  return cudaGetLastError();
}

}  // namespace lq
