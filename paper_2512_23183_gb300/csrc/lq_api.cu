// lq_api.cu -- the extern "C" entry points declared in include/lq.h:
// argument validation, lowering/scheduling on the host, kernel launches on
// the caller's stream.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <vector>

#include "lq_coefs.h"
#include "lq_internal.h"
#include "lq_kernels.h"

namespace lq {

const char* last_error();
void clear_error();

int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (cached[dev] == 0) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = v > 0 ? v : 1;
  }
  return cached[dev];
}

#define LQ_CUDA(expr)                                                                  \
  do {                                                                                 \
    cudaError_t e_ = (expr);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      (void)cudaGetLastError();                                                        \
      return fail(LQ_ERR_CUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, \
                  __LINE__);                                                           \
    }                                                                                  \
  } while (0)

static inline std::size_t align256(std::size_t b) { return (b + 255) & ~(std::size_t)255; }

// ------------------------------------------------------- Pauli-term chunks

int exp_chunk_count(const lq_pauli_term* terms, int nt) {
  std::map<uint64_t, int> groups;
  for (int t = 0; t < nt; t++) groups[terms[t].xmask]++;
  int chunks = 1, g = 0, c = 0;
  for (auto& kv : groups) {
    int left = kv.second;
    while (left > 0) {
      if (g == EXP_MAX_GROUPS || c == EXP_MAX_TERMS) {
        chunks++;
        g = 0;
        c = 0;
      }
      int take = left < EXP_MAX_TERMS - c ? left : EXP_MAX_TERMS - c;
      g++;
      c += take;
      left -= take;
    }
  }
  return chunks;
}

int build_exp_chunks(int n, const lq_pauli_term* terms, int nt, ExpParams* chunks,
                     int max_chunks) {
  std::map<uint64_t, std::vector<int>> groups;
  for (int t = 0; t < nt; t++) groups[terms[t].xmask].push_back(t);
  int ci = 0;
  std::memset(&chunks[0], 0, sizeof(ExpParams));
  chunks[0].n = n;
  for (auto& kv : groups) {
    const uint64_t x = kv.first;
    std::size_t done = 0;
    while (done < kv.second.size()) {
      ExpParams* E = &chunks[ci];
      int used = 0;
      for (int g = 0; g < E->ngroups; g++) used += E->groups[g].count;
      if (E->ngroups == EXP_MAX_GROUPS || used == EXP_MAX_TERMS) {
        if (++ci >= max_chunks) return -1;
        E = &chunks[ci];
        std::memset(E, 0, sizeof(ExpParams));
        E->n = n;
        used = 0;
      }
      ExpGroup& G = E->groups[E->ngroups++];
      G.x = x;
      G.h = x ? 63 - __builtin_clzll(x) : 0;
      G.first = used;
      G.count = 0;
      while (done < kv.second.size() && used < EXP_MAX_TERMS) {
        const lq_pauli_term& P = terms[kv.second[done++]];
        ExpTerm& T = E->terms[used++];
        T.c = P.coeff;
        T.c2 = 2.0 * P.coeff;
        T.z = P.zmask;
        T.k0 = __builtin_popcountll(P.xmask & P.zmask) & 3;
        T.chunk = 0;
        if (x == 0 && P.zmask) {
          const int lo = __builtin_ctzll(P.zmask), hi = 63 - __builtin_clzll(P.zmask);
          if (lo / EXP_CHUNK_BITS == hi / EXP_CHUNK_BITS) {
            T.chunk = 1 + lo / EXP_CHUNK_BITS;
            E->tables = 1;
          }
        }
        G.count++;
      }
    }
  }
  // groups whose terms all have the same parity of Y factors need only one
  // component of conj(psi_i) psi_j
  for (int c = 0; c <= ci; c++) {
    ExpParams& E = chunks[c];
    for (int g = 0; g < E.ngroups; g++) {
      ExpGroup& G = E.groups[g];
      G.part = 0;
      if (G.x == 0 || G.count == 0) continue;
      int odd = 0, even = 0;
      for (int t = G.first; t < G.first + G.count; t++) (E.terms[t].k0 & 1 ? odd : even)++;
      G.part = odd == 0 ? 1 : even == 0 ? 2 : 0;
    }
  }
  return ci + 1;
}

// The tiled <H> plans of a term list: 2^12 tiles (3 CTAs/SM) when class-mode
// groups (2 FMAs per pair, little integer work) dominate, 2^11 tiles (4
// CTAs/SM) when table-mode groups (parity index per pair) do -- measured on
// the XYZ chain and on random 50-term sums at n = 28, 30.
static int plan_expval_tiled(int n, const lq_pauli_term* terms, int nt,
                             std::vector<XPlan>& xp, std::vector<lq_pauli_term>& wide) {
  int r = build_xplans(n, terms, nt, 12, xp, wide);
  int ncls = 0, ntab = 0;
  for (const XPlan& X : xp)
    for (int g = 0; g < X.ngroups; g++) {
      ncls += X.groups[g].mode == XG_CLASS;
      ntab += X.groups[g].mode == XG_TABLE;
    }
  if (r >= 0 && ntab > ncls) r = build_xplans(n, terms, nt, 11, xp, wide);
  return r;
}

// <H> of nstates states (stride apart) into out_dev[0..nstates).  partial:
// expval_grid(n) * nstates doubles.
lq_status expval_states(const double2* states, uint64_t stride, int nstates, int n,
                               const lq_pauli_term* terms, int nt, double* partial,
                               double* out_dev, cudaStream_t s) {
  if (nt == 0) {
    LQ_CUDA(cudaMemsetAsync(out_dev, 0, sizeof(double) * nstates, s));
    return LQ_OK;
  }
  bool acc = false;
  std::vector<lq_pauli_term> wide;
  if (n >= kTiledExpvalMinN) {   // tiled passes: each tile read once per pass of groups
    std::vector<XPlan> xp;
    if (plan_expval_tiled(n, terms, nt, xp, wide) < 0)
      return fail(LQ_ERR_INVALID_ARG, "internal: term plan");
    for (std::size_t c = 0; c < xp.size(); c++) {
      LQ_CUDA(launch_expval_tiled(xp[c], states, stride, nstates, partial, out_dev, acc, s));
      acc = true;
    }
    if (wide.empty()) {
      if (!acc) LQ_CUDA(cudaMemsetAsync(out_dev, 0, sizeof(double) * nstates, s));
      return LQ_OK;
    }
    terms = wide.data();   // X masks wider than a tile: the untiled kernel
    nt = (int)wide.size();
  }
  int nch = exp_chunk_count(terms, nt);
  std::vector<ExpParams> ch((std::size_t)nch);
  int got = build_exp_chunks(n, terms, nt, ch.data(), nch);
  if (got < 0) return fail(LQ_ERR_INVALID_ARG, "internal: term chunking");
  for (int c = 0; c < got; c++)
    LQ_CUDA(launch_expval(ch[c], states, stride, nstates, partial, out_dev, acc || c > 0, s));
  return LQ_OK;
}

// Run a lowered op list on nstates states; flags of the first pass may ask
// for a |0...0> start.
static lq_status run_ops(double2* states, uint64_t stride, int nstates, int n, const LOp* ops,
                         std::size_t nops, double zr, double zi, bool init_zero,
                         cudaStream_t s, const ScheduleOptions* tuned = nullptr) {
  ScheduleOptions opt;
  opt.lphase_table = true;   // run by pass_kernel
  if (tuned) opt = *tuned;
  opt.max_hi = PASS_HI_BITS;
  opt.sink_phases = true;
  Schedule S;
  lq_status st = schedule_ops(n, ops, nops, zr, zi, opt, S);
  if (st) return st;
  if (S.npasses == 0) {
    if (init_zero)
      for (int i = 0; i < nstates; i++)
        LQ_CUDA(launch_init_basis(states + (uint64_t)i * stride, n, 0, s));
    return LQ_OK;
  }
  for (int p = 0; p < S.npasses; p++) {
    if (p == 0 && init_zero) S.passes[p].h.flags |= PF_INIT_ZERO;
    LQ_CUDA(launch_pass(S.passes[p], states, stride, nstates, s));
  }
  return LQ_OK;
}

}  // namespace lq

using namespace lq;

// =================================================================== C ABI

extern "C" {

const char* lq_last_error(void) { return lq::last_error(); }

const char* lq_version(void) { return "lq 0.1 (sm_103a)"; }

lq_status lq_pauli_from_string(const char* s, int n, double coeff, lq_pauli_term* out) {
  if (!s || !out) return fail(LQ_ERR_INVALID_ARG, "NULL argument");
  lq_status st = check_n(n);
  if (st) return st;
  if ((int)std::strlen(s) != n) return fail(LQ_ERR_INVALID_ARG, "Pauli string length != n");
  if (!std::isfinite(coeff)) return fail(LQ_ERR_NONFINITE, "coefficient not finite");
  uint64_t x = 0, z = 0;
  for (int q = 0; q < n; q++) {
    uint64_t b = 1ull << (n - 1 - q);
    switch (s[q]) {
      case 'I': break;
      case 'X': x |= b; break;
      case 'Y': x |= b; z |= b; break;
      case 'Z': z |= b; break;
      default: return fail(LQ_ERR_INVALID_ARG, "bad Pauli character '%c'", s[q]);
    }
  }
  out->coeff = coeff;
  out->xmask = x;
  out->zmask = z;
  return LQ_OK;
}

lq_status lq_state_init(void* amps, int n, uint64_t basis, lq_stream stream) {
  lq_status st = check_n(n);
  if (st) return st;
  if (!amps) return fail(LQ_ERR_INVALID_ARG, "amps is NULL");
  if (basis >> n) return fail(LQ_ERR_INVALID_ARG, "basis index >= 2^n");
  LQ_CUDA(launch_init_basis((double2*)amps, n, basis, (cudaStream_t)stream));
  return LQ_OK;
}

lq_status lq_apply_circuit(void* amps, int n, const lq_gate* gates, int ng,
                           const double* params, int np, lq_stream stream) {
  return apply_circuit_with(amps, n, gates, ng, params, np, stream, nullptr);
}

}  // extern "C"

namespace lq {

lq_status apply_circuit_with(void* amps, int n, const lq_gate* gates, int ng,
                             const double* params, int np, lq_stream stream,
                             const ScheduleOptions* fallback) {
  lq_status st = check_n(n);
  if (st) return st;
  if (!amps) return fail(LQ_ERR_INVALID_ARG, "amps is NULL");
  LOp* ops = nullptr;
  std::size_t nops = 0;
  double zr, zi;
  st = lower_circuit(n, gates, ng, params, np, &ops, &nops, &zr, &zi, true);
  if (st) return st;
  // the autotuner's choice for this (GPU, n, circuit structure), if any,
  // else the caller's default
  ScheduleOptions tuned;
  tuned.lphase_table = true;
  bool has = tuned_options(n, gates, ng, &tuned);
  if (!has && fallback) {
    tuned = *fallback;
    has = true;
  }
  st = run_ops((double2*)amps, 0, 1, n, ops, nops, zr, zi, false, (cudaStream_t)stream,
               has ? &tuned : nullptr);
  delete[] ops;
  return st;
}

}  // namespace lq

extern "C" {

lq_status lq_expval_plan(int n, const lq_pauli_term* terms, int nt, lq_plan_info* out) {
  lq_status st = check_n(n);
  if (st) return st;
  if (!out) return fail(LQ_ERR_INVALID_ARG, "out is NULL");
  st = check_terms(n, terms, nt);
  if (st) return st;
  const double N = std::ldexp(1.0, n);
  std::vector<lq_pauli_term> rest(terms, terms + nt);
  int reads = 0, tb = 0;
  double fl = 0;
  if (n >= kTiledExpvalMinN && nt > 0) {
    std::vector<XPlan> xp;
    if (plan_expval_tiled(n, terms, nt, xp, rest) < 0)
      return fail(LQ_ERR_INVALID_ARG, "internal: term plan");
    for (const XPlan& X : xp) {
      reads += X.npass;
      const int nch = (n + EXP_CHUNK_BITS - 1) / EXP_CHUNK_BITS;
      for (int g = 0; g < X.ngroups; g++) {
        const XGroup& G = X.groups[g];
        const int parts = G.part == 0 ? 2 : 1;
        if (G.mode == XG_CLASS) {
          fl += 2.0 * parts * N;                  // 2 FMA per pair and part
        } else if (G.mode == XG_TABLE) {
          fl += 2.5 * parts * N;                  // MUL + FMA, then FMA, per pair and part
        } else {
          if (X.dcls) {   // |psi|^2, the classes' table values, FMA
            fl += (5.0 + (X.dcls - 1)) * N;
          } else {
            const int direct = X.tables ? G.first + G.count - G.direct : G.count;
            fl += (5.0 + (X.tables ? nch : 0) + direct) * N;   // |psi|^2, d(i), FMA
          }
        }
      }
      if (X.npass) tb = X.passes[0].k;
    }
  }
  // untiled kernel: one read of the state per X-mask group
  std::map<uint64_t, int> groups;
  for (const lq_pauli_term& t : rest) groups[t.xmask]++;
  for (auto& kv : groups) {
    reads++;
    fl += kv.first ? (3.0 + kv.second) * N : (3.0 + 2.0 * kv.second) * N;
  }
  out->npasses = reads;
  out->tile_bits = tb;
  out->dp_flops = fl;
  out->dram_bytes = 16.0 * N * reads;
  return LQ_OK;
}

lq_status lq_circuit_plan(int n, const lq_gate* gates, int ng, const double* params, int np,
                          lq_plan_info* out) {
  return circuit_plan_with(n, gates, ng, params, np, out, nullptr);
}

}  // extern "C"

namespace lq {

lq_status circuit_plan_with(int n, const lq_gate* gates, int ng, const double* params, int np,
                            lq_plan_info* out, const ScheduleOptions* fallback) {
  lq_status st = check_n(n);
  if (st) return st;
  if (!out) return fail(LQ_ERR_INVALID_ARG, "out is NULL");
  LOp* ops = nullptr;
  std::size_t nops = 0;
  double zr, zi;
  st = lower_circuit(n, gates, ng, params, np, &ops, &nops, &zr, &zi, true);
  if (st) return st;
  ScheduleOptions opt;
  opt.lphase_table = true;   // run by pass_kernel
  // the schedule apply_circuit_with would use
  if (!tuned_options(n, gates, ng, &opt) && fallback) opt = *fallback;
  opt.max_hi = PASS_HI_BITS;
  opt.sink_phases = true;
  Schedule S;
  st = schedule_ops(n, ops, nops, zr, zi, opt, S);
  delete[] ops;
  if (st) return st;
  out->npasses = S.npasses;
  out->tile_bits = S.npasses ? S.passes[0].h.k : 0;
  double fl = 0;
  for (int p = 0; p < S.npasses; p++) {
    const PassParams& P = S.passes[p];
    for (int o = 0; o < P.h.nops; o++) {
      const Op& d = P.ops[o];
      LOp l;
      l.type = d.type;
      l.mode = d.mode;
      // condition width: tile-local and CTA bits together
      uint64_t cmbits = (uint64_t)__builtin_popcountll(d.cm_glob) + __builtin_popcount(d.cm_loc);
      l.cm = cmbits ? ((1ull << cmbits) - 1) : 0;
      fl += op_flops(l, n);
    }
    // deferred per-tile phases: one complex multiply per amplitude after the
    // load and/or at the store
    if (P.h.flags & PF_DFULL) {
      const uint32_t all = (1u << P.h.ndefer) - 1u;
      if (P.h.dpre) fl += 6.0 * std::ldexp(1.0, n);
      if (all & ~(uint32_t)P.h.dpre) fl += 6.0 * std::ldexp(1.0, n);
    }
  }
  out->dp_flops = fl;
  out->dram_bytes = 32.0 * std::ldexp(1.0, n) * S.npasses;
  return LQ_OK;
}

}  // namespace lq

extern "C" {

size_t lq_expval_workspace_size(int n, int nt) {
  (void)nt;
  if (n < 1 || n > 34) return 0;
  return align256(sizeof(double)) + align256(sizeof(double) * (std::size_t)expval_grid(n));
}

lq_status lq_expval_pauli_sum_async(const void* amps, int n, const lq_pauli_term* terms,
                                    int nt, double* out_dev, void* workspace,
                                    size_t ws_bytes, lq_stream stream) {
  lq_status st = check_n(n);
  if (st) return st;
  if (!amps || !out_dev) return fail(LQ_ERR_INVALID_ARG, "NULL device pointer");
  st = check_terms(n, terms, nt);
  if (st) return st;
  if (!workspace || ws_bytes < lq_expval_workspace_size(n, nt))
    return fail(LQ_ERR_OOM, "workspace too small: %zu < %zu", ws_bytes,
                lq_expval_workspace_size(n, nt));
  cudaStream_t s = (cudaStream_t)stream;
  double* partial = (double*)((char*)workspace + align256(sizeof(double)));
  return expval_states((const double2*)amps, 0, 1, n, terms, nt, partial, out_dev, s);
}

lq_status lq_expval_pauli_sum(const void* amps, int n, const lq_pauli_term* terms, int nt,
                              double* out, void* workspace, size_t ws_bytes,
                              lq_stream stream) {
  if (!out) return fail(LQ_ERR_INVALID_ARG, "out is NULL");
  if (!workspace) return fail(LQ_ERR_OOM, "workspace is NULL");
  double* d_out = (double*)workspace;
  lq_status st = lq_expval_pauli_sum_async(amps, n, terms, nt, d_out, workspace, ws_bytes,
                                           stream);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  LQ_CUDA(cudaMemcpyAsync(out, d_out, sizeof(double), cudaMemcpyDeviceToHost, s));
  LQ_CUDA(cudaStreamSynchronize(s));
  return LQ_OK;
}

lq_status lq_apply_pauli_sum(void* out, const void* in, int n, const lq_pauli_term* terms,
                             int nt, lq_stream stream) {
  lq_status st = check_n(n);
  if (st) return st;
  if (!out || !in) return fail(LQ_ERR_INVALID_ARG, "NULL device pointer");
  if (out == in) return fail(LQ_ERR_INVALID_ARG, "out must differ from in");
  st = check_terms(n, terms, nt);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if (nt == 0) {
    LQ_CUDA(cudaMemsetAsync(out, 0, sizeof(double2) << n, s));
    return LQ_OK;
  }
  int nch = exp_chunk_count(terms, nt);
  std::vector<ExpParams> ch((std::size_t)nch);
  int got = build_exp_chunks(n, terms, nt, ch.data(), nch);
  if (got < 0) return fail(LQ_ERR_INVALID_ARG, "internal: term chunking");
  for (int c = 0; c < got; c++)
    LQ_CUDA(launch_apply_pauli_sum(ch[c], (const double2*)in, (double2*)out, c > 0, s));
  return LQ_OK;
}

}  // extern "C"
