// lq_tune.cu -- the schedule autotuner: per (GPU, n, circuit structure) it
// times the tile-pass schedules of lq_apply_circuit over tile width k,
// contiguous low bits m and the per-CTA phase-table option, and keeps the
// fastest in a process-wide cache that lq_apply_circuit (and lq_circuit_plan)
// consult.  It also keeps, per batch structure, the tile width of the
// persistent batched launch for states larger than shared memory
// (lq_autotune_batch, n = 0 in the key).  The cache can be written to and
// read from a text file, one line per entry:
//   <gpu> <n> <structure hash, 16 hex digits> <k> <m> <table> <ms> <ms_default>
// The structure hash covers n and, per gate, its kind, qubits, whether it
// takes a parameter and (for fixed gates) its angle: everything the schedule
// depends on apart from the parameter values.
#include <cuda_runtime.h>

#include <cinttypes>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "lq_internal.h"
#include "lq_kernels.h"

namespace lq {

namespace {

struct TuneEntry {
  int k, m, table;
  double ms, ms_default;
};

std::mutex g_tune_mu;
std::map<std::string, TuneEntry>& tune_cache() {
  static std::map<std::string, TuneEntry> m;
  return m;
}

uint64_t fnv(uint64_t h, const void* p, std::size_t n) {
  const unsigned char* b = (const unsigned char*)p;
  for (std::size_t i = 0; i < n; i++) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  return h;
}

}  // namespace

uint64_t circuit_structure_hash(int n, const lq_gate* gates, int ng) {
  uint64_t h = 1469598103934665603ull;
  h = fnv(h, &n, sizeof n);
  for (int i = 0; i < ng; i++) {
    const lq_gate& g = gates[i];
    const int32_t rec[5] = {g.kind, g.qubits[0], g.qubits[1], g.qubits[2], g.param >= 0};
    h = fnv(h, rec, sizeof rec);
    if (g.param < 0) h = fnv(h, &g.angle, sizeof g.angle);
    if (g.kind == LQ_U1 || g.kind == LQ_U2) h = fnv(h, g.mat, sizeof g.mat);
  }
  return h;
}

namespace {

// "<device name>|<SM count>" with blanks replaced, for the current device.
std::string gpu_id() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return "unknown";
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
  std::string s = p.name;
  for (char& c : s)
    if (c == ' ' || c == '\t') c = '_';
  return s + "|" + std::to_string(p.multiProcessorCount);
}

std::string key_of(const std::string& gpu, int n, uint64_t h) {
  char buf[64];
  std::snprintf(buf, sizeof buf, " %d %016" PRIx64, n, h);
  return gpu + buf;
}

const std::string& current_gpu() {
  static thread_local std::string gpu;
  static thread_local int gpu_dev = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != gpu_dev) {
    gpu = gpu_id();
    gpu_dev = dev;
  }
  return gpu;
}

}  // namespace

// Batch entries use n = 0 in the key (the structure hash covers every
// problem's n).
bool tuned_batch_tile(uint64_t structure, int* k) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (tune_cache().empty()) return false;
  auto it = tune_cache().find(key_of(current_gpu(), 0, structure));
  if (it == tune_cache().end()) return false;
  *k = it->second.k;
  return true;
}

void record_batch_tile(uint64_t structure, int k, double ms, double ms_default) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_cache()[key_of(current_gpu(), 0, structure)] = TuneEntry{k, 5, 0, ms, ms_default};
}

bool tuned_options(int n, const lq_gate* gates, int ng, ScheduleOptions* opt) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (tune_cache().empty()) return false;
  auto it = tune_cache().find(key_of(current_gpu(), n, circuit_structure_hash(n, gates, ng)));
  if (it == tune_cache().end()) return false;
  opt->k = it->second.k;
  opt->m = it->second.m;
  opt->lphase_table = it->second.table != 0;
  return true;
}

}  // namespace lq

using namespace lq;

extern "C" {

lq_status lq_autotune_circuit(void* scratch, int n, const lq_gate* gates, int ng,
                              const double* params, int np, lq_tune_result* out,
                              lq_stream stream) {
  lq_status st = check_n(n);
  if (st) return st;
  if (!scratch || !out) return fail(LQ_ERR_INVALID_ARG, "NULL argument");
  LOp* ops = nullptr;
  std::size_t nops = 0;
  double zr, zi;
  st = lower_circuit(n, gates, ng, params, np, &ops, &nops, &zr, &zi, true);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    delete[] ops;
    (void)cudaGetLastError();
    return fail(LQ_ERR_CUDA, "event creation failed");
  }
  struct Cand {
    int k, m, table;
  };
  std::vector<Cand> cands;
  const int kmax = n < MAX_TILE_BITS - 1 ? n : MAX_TILE_BITS - 1;   // up to 2^12
  // low runs of 5 and 6 bits; with 2^11 and 2^12 tiles also 3 and 4 (more
  // high bits per pass: at n = 30 a layer of one-qubit rotations takes 3
  // passes at k = 12, m = 3 instead of 4 at m = 5, the inverse gate-form QFT
  // 4 at k = 11, m = 4 instead of 5 at m = 5)
  for (int k = kmax < 9 ? kmax : 9; k <= kmax; k++)
    for (int m = k >= 11 ? 3 : 5; m <= 6; m++)
      // the option switches the per-CTA tables: a one-bit phase op's table
      // (tiles of up to 2^LTAB_MAX_BITS amplitudes) and the merged dyadic
      // phases' partial-sum and full tables (any tile; the gate-form QFT's
      // butterflies need them).  Above 2^LTAB_MAX_BITS the option only
      // changes the dyadic tables, which are never slower: only "on" is timed
      for (int table = 1; table >= (k <= LTAB_MAX_BITS ? 0 : 1); table--) {
        const int mm = m < k ? m : k;
        bool dup = false;
        for (const Cand& c : cands) dup |= c.k == k && c.m == mm && c.table == table;
        if (!dup) cands.push_back(Cand{k, mm, table});
      }
  double best = 1e300, def_ms = -1;
  Cand bestc{10, 5, 1};
  lq_status err = LQ_OK;
  for (const Cand& c : cands) {
    ScheduleOptions opt;
    opt.k = c.k;
    opt.m = c.m;
    opt.max_hi = PASS_HI_BITS;
    opt.lphase_table = c.table != 0;
    opt.sink_phases = true;   // as lq_apply_circuit schedules
    Schedule S;
    st = schedule_ops(n, ops, nops, zr, zi, opt, S);
    if (st) {
      err = st;
      break;
    }
    float ms = 0, msmin = 1e30f;
    cudaError_t e = cudaSuccess;
    for (int rep = 0; rep < 3 && e == cudaSuccess; rep++) {
      e = launch_init_basis((double2*)scratch, n, 0, s);
      if (e == cudaSuccess) e = cudaEventRecord(e0, s);
      for (int p = 0; p < S.npasses && e == cudaSuccess; p++)
        e = launch_pass(S.passes[p], (double2*)scratch, 0, 1, s);
      if (e == cudaSuccess) e = cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0 && ms < msmin) msmin = ms;   // the first run warms up
    }
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      err = fail(LQ_ERR_CUDA, "autotune: %s", cudaGetErrorString(e));
      break;
    }
    if (c.k == 10 && c.m == 5 && c.table == 1) def_ms = msmin;
    if (msmin < best) {
      best = msmin;
      bestc = c;
    }
  }
  delete[] ops;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err) return err;
  if (def_ms < 0) def_ms = best;   // small n: no k = 10 candidate
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_cache()[key_of(gpu_id(), n, circuit_structure_hash(n, gates, ng))] =
        TuneEntry{bestc.k, bestc.m, bestc.table, best, def_ms};
  }
  out->tile_bits = bestc.k;
  out->low_bits = bestc.m;
  out->phase_table = bestc.table;
  out->candidates = (int32_t)cands.size();
  out->ms = best;
  out->ms_default = def_ms;
  return LQ_OK;
}

lq_status lq_tune_cache_save(const char* path) {
  if (!path) return fail(LQ_ERR_INVALID_ARG, "path is NULL");
  FILE* f = std::fopen(path, "w");
  if (!f) return fail(LQ_ERR_INVALID_ARG, "cannot open %s for writing", path);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  std::fprintf(f, "# lq autotune cache v1: gpu n hash k m table ms ms_default\n");
  for (auto& kv : tune_cache())
    std::fprintf(f, "%s %d %d %d %.6f %.6f\n", kv.first.c_str(), kv.second.k, kv.second.m,
                 kv.second.table, kv.second.ms, kv.second.ms_default);
  const bool ok = std::ferror(f) == 0;
  std::fclose(f);
  return ok ? LQ_OK : fail(LQ_ERR_INVALID_ARG, "write error on %s", path);
}

lq_status lq_tune_cache_load(const char* path) {
  if (!path) return fail(LQ_ERR_INVALID_ARG, "path is NULL");
  FILE* f = std::fopen(path, "r");
  if (!f) return fail(LQ_ERR_INVALID_ARG, "cannot open %s", path);
  char line[512];
  int lineno = 0;
  std::map<std::string, TuneEntry> got;
  lq_status st = LQ_OK;
  while (std::fgets(line, sizeof line, f)) {
    lineno++;
    if (line[0] == '#' || line[0] == '\n') continue;
    char gpu[256];
    int n, k, m, table;
    char hash[32];
    double ms, msd;
    if (std::sscanf(line, "%255s %d %31s %d %d %d %lf %lf", gpu, &n, hash, &k, &m, &table, &ms,
                    &msd) != 8 ||
        n < 0 || n > 34 || k < 1 || k > MAX_TILE_BITS || m < 1 || m > k || std::strlen(hash) != 16) {
      st = fail(LQ_ERR_INVALID_ARG, "%s:%d: malformed autotune entry", path, lineno);
      break;
    }
    const uint64_t h = std::strtoull(hash, nullptr, 16);
    got[key_of(gpu, n, h)] = TuneEntry{k, m, table != 0, ms, msd};
  }
  std::fclose(f);
  if (st) return st;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (auto& kv : got) tune_cache()[kv.first] = kv.second;
  return LQ_OK;
}

lq_status lq_tune_cache_clear(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_cache().clear();
  return LQ_OK;
}

int lq_tune_cache_size(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return (int)tune_cache().size();
}

}  // extern "C"
