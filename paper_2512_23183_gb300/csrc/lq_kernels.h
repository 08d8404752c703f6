// lq_kernels.h -- kernel launchers and kernel-parameter structs of the lq
// library (internal).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <mutex>
#include <utility>
#include <vector>

#include "lq_internal.h"

namespace lq {

// ------------------------------------------------------- Pauli-sum params

struct ExpTerm {
  double c;      // coefficient
  double c2;     // 2 * coefficient (pair form of <H>)
  uint64_t z;    // Z mask (global bits)
  int32_t k0;    // number of Y factors mod 4
  int32_t chunk; // diagonal terms: 1 + the 8-bit index chunk holding z (read
                 // from a table), 0: applied directly
};
struct ExpGroup {
  uint64_t x;    // common X mask
  int32_t h;     // top bit of x (pair enumeration), 0 for x == 0
  int32_t first, count;
  int32_t part;  // x != 0: 0 needs Re and Im of conj(psi_i) psi_j, 1 only Re, 2 only Im
};
constexpr int EXP_CHUNK_BITS = 8;  // diagonal terms inside one 8-bit chunk use a table
constexpr int EXP_MAX_TERMS = 640;
constexpr int EXP_MAX_GROUPS = 240;
struct ExpParams {
  int32_t n, ngroups;
  int32_t tables;   // nonzero: some diagonal terms are read from chunk tables
  int32_t pad;
  ExpGroup groups[EXP_MAX_GROUPS];
  ExpTerm terms[EXP_MAX_TERMS];
};
static_assert(sizeof(ExpParams) < 32000, "ExpParams exceeds the kernel parameter budget");

// Tiled <H> (lq_expval.cu): terms grouped by X mask, groups packed into tile
// passes whose tile bits cover their X masks.
constexpr int XP_TILE_BITS = 12;   // largest tile (the plan picks 11 or 12)
constexpr int XP_LOW_BITS = 2;     // contiguous low bits in every tile (64-byte runs)
constexpr int kTiledExpvalMinN = 12;   // smaller states use the untiled kernel
constexpr int XP_MAX_PASS = 48;
constexpr int XP_MAX_GROUPS = 192;
constexpr int XP_MAX_TERMS = 512;
constexpr int XP_MAX_COEF = 384;
constexpr int XP_TABLE_TERMS = 4;   // terms per table-mode group
constexpr int XP_CLASS_TERMS = 128; // terms per class-mode group (longer lists are split)
enum XGroupMode : int8_t { XG_DIAG = 0, XG_CLASS = 1, XG_TABLE = 2 };
struct XTerm {
  double c;        // c_t (diagonal) or 2 c_t (pair terms)
  uint64_t zg;     // Z mask outside the tile (diagonal terms: the whole Z mask)
  uint32_t zl;     // Z mask inside the tile (tile-local bits)
  int16_t k0;      // number of Y factors mod 4
  int16_t chunk;   // diagonal terms: 1 + the 8-bit index chunk holding z, or 0
};
struct XGroup {
  uint32_t x;        // X mask (tile-local bits); 0 for the diagonal group
  int16_t first, count;
  int16_t coef;      // class mode: 2^{w-1} entries; table mode: 2^count entries
  int8_t h, w;       // top bit of x, number of x bits
  int8_t mode, part; // XGroupMode; part 1: only Re, 2: only Im, 0: both
  int16_t direct;    // diagonal group: first term not read from a chunk table
};
struct XPass {
  int32_t k, m, nobits, g0, g1, pad;
  int8_t tbits[16];
  int8_t obits[48];
};
constexpr int XP_DIAG_CLASSES = 4;   // coefficient classes of a diagonal group
constexpr int XP_DIAG_DELTAS = 2;    // pair-term groups per class
struct XPlan {
  int32_t n, npass, ngroups, nterms, ncoef, tables, diag;
  // nonzero: the diagonal group's terms form dcls classes of equal
  // coefficient, terms [dfirst[c], dfirst[c] + dcount[c]); an amplitude's
  // class-c value c (count - 2 #odd) is read from a per-CTA table by its
  // number of odd parities, counted with integer operations: the first
  // ddirect[c] terms one by one, the class's two-bit terms (b, b + delta)
  // in groups of one delta as popcount((i ^ (i >> delta)) & mask), one-bit
  // terms as the group of delta 0, popcount(i & mask)
  int32_t dcls;
  int16_t dfirst[XP_DIAG_CLASSES], dcount[XP_DIAG_CLASSES], ddirect[XP_DIAG_CLASSES];
  int8_t dnd[XP_DIAG_CLASSES], ddel[XP_DIAG_CLASSES][XP_DIAG_DELTAS];
  uint64_t dmsk[XP_DIAG_CLASSES][XP_DIAG_DELTAS];
  XPass passes[XP_MAX_PASS];
  XGroup groups[XP_MAX_GROUPS];
  XTerm terms[XP_MAX_TERMS];
  double2 coef[XP_MAX_COEF];   // (coefficient of Re, coefficient of Im) per entry
};
static_assert(sizeof(XPlan) < 32000, "XPlan exceeds the kernel parameter budget");
// Build the tile-pass plans (one or more launches) of a term list with 2^k
// tiles; terms whose X mask does not fit a tile go to `wide`.  Returns the
// number of plans, or -1 on an internal limit.
int build_xplans(int n, const lq_pauli_term* terms, int nt, int k, std::vector<XPlan>& out,
                 std::vector<lq_pauli_term>& wide);
cudaError_t launch_expval_tiled(const XPlan& X, const double2* states, uint64_t stride,
                                int nstates, double* partial, double* out, int accumulate,
                                cudaStream_t s);
cudaError_t launch_sum_partials(const double* partial, int nparts, int nstates, double* out,
                                int accumulate, cudaStream_t s);

// Group a term list by X mask into chunks that fit ExpParams.  Returns the
// number of chunks written to `chunks` (caller-allocated with capacity
// `max_chunks`), or -1 when max_chunks is too small.
int build_exp_chunks(int n, const lq_pauli_term* terms, int nt, ExpParams* chunks,
                     int max_chunks);
int exp_chunk_count(const lq_pauli_term* terms, int nt);

// <H> of nstates states (stride amplitudes apart) into out_dev[0..nstates);
// partial holds expval_grid(n) * nstates doubles.
lq_status expval_states(const double2* states, uint64_t stride, int nstates, int n,
                        const lq_pauli_term* terms, int nt, double* partial, double* out_dev,
                        cudaStream_t s);

// ------------------------------------------------- persistent batch runner

// One problem as the batch runner sees it: circuit, Hamiltonian, the patch
// of every circuit (index 0 = unshifted), and per parameter the (circuit,
// weight) pairs of its shift rule.
struct HostProblem {
  int n = 0, ng = 0, np = 0, nt = 0;
  const lq_gate* gates = nullptr;
  const double* params = nullptr;
  const lq_pauli_term* terms = nullptr;
  std::vector<Patch> patches;
  std::vector<std::vector<std::pair<int, double>>> comb;
};

lq_status make_problem(int n, const lq_gate* gates, int ng, const double* params, int np,
                       const lq_pauli_term* terms, int nt, bool want_grad, bool general,
                       HostProblem& hp);
std::size_t batch_workspace_for(const std::vector<HostProblem>& hps, lq_status* st);
// Runs every circuit of every problem in one persistent launch; out holds
// per problem E then its np gradient entries.
lq_status batch_run(const std::vector<HostProblem>& hps, void* ws, std::size_t ws_bytes,
                    cudaStream_t s, std::vector<double>& out);
// Times the batch for every tile width of its larger-than-shared-memory
// states and records the fastest for this batch structure.
lq_status batch_autotune(const std::vector<HostProblem>& hps, void* ws, std::size_t ws_bytes,
                         cudaStream_t s, lq_tune_result* res);

// Run `set` (a kernel's cudaFuncSetAttribute calls) once per device; the
// calling threads may race, the attribute calls are idempotent.
template <typename F>
cudaError_t once_per_device(std::atomic<uint64_t>& done, F set) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
  e = set();
  if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_release);
  return e;
}

// --------------------------------------------------------------- launchers

int sm_count();

// Once-per-device fill of a constant device table (lq_kernels.cu).
struct TableOnce {
  std::mutex mu;
  std::atomic<uint64_t> done{0};
};
// Runs fill(private stream) once per device and waits for it; `caller`, when
// not null, is the stream of the launch that needs the table: a first fill
// while it is being captured returns cudaErrorStreamCaptureUnsupported.
cudaError_t fill_table_once(TableOnce& t, const cudaStream_t* caller,
                            cudaError_t (*fill)(cudaStream_t));
const double2* dyadic_tables(cudaError_t* err, const cudaStream_t* caller);
int expval_grid(int n);

cudaError_t launch_init_basis(double2* amps, int n, uint64_t basis, cudaStream_t s);
cudaError_t launch_pass(const PassParams& P, double2* state, uint64_t stride, int nstates,
                        cudaStream_t s);
int pass2_grid(int n, int k);
cudaError_t launch_pass2(const PassParams& P, double2* psi, double2* lam, double* partial,
                         int grid, cudaStream_t s);
cudaError_t launch_grad_reduce(const double* partial, int grid, const double* factor,
                               const int* first, const int* count, int np, double* grad,
                               cudaStream_t s);
cudaError_t launch_psr_grad(const double* E, int np, double* out, cudaStream_t s);
cudaError_t launch_fft_pass(double2* state, int n, int q0, int q1, int inverse, double scale,
                            cudaStream_t s);
cudaError_t launch_bitrev(double2* state, int n, cudaStream_t s);
cudaError_t fft_tables_init(cudaStream_t s);   // fills the twiddle table once per device
cudaError_t launch_expval(const ExpParams& E, const double2* state, uint64_t stride,
                          int nstates, double* partial, double* out, int accumulate,
                          cudaStream_t s);
cudaError_t launch_apply_pauli_sum(const ExpParams& E, const double2* in, double2* out,
                                   int accumulate, cudaStream_t s);

}  // namespace lq
