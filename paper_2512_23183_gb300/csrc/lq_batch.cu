// lq_batch.cu -- batched gradients in one persistent launch.
//
// The circuits of a parameter-shift gradient (Sec. III-A Eq. parameter_shift:
// the base circuit and the +-s shifted copies per parameter, each run from
// |0...0>, Sec. III-C) -- and, for uneven batches, the circuits of many
// independent problems -- are work items of one persistent kernel.  Each
// CTA takes the next circuit from an atomic work counter (items in
// decreasing cost order, largest first), runs all of its tile passes on it,
// evaluates <H>, and writes the energy; the last CTA to finish combines the
// energies into gradients with the shift-rule weights.  No CTA waits on
// another, so the launch has no inter-CTA spin-waits.
//
// A circuit whose state fits a tile (n <= 12) lives in shared memory from
// |0...0> to <H> and never touches HBM; a larger one uses a per-CTA scratch
// state in the workspace.  Circuits of one problem share one op program
// lowered at the base angles; a circuit differs only in the coefficients of
// its shifted gate and in the deferred scalar (a Patch).
#include <cuda.h>
#include <cuda_runtime.h>

#include <chrono>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "lq_coefs.h"
#include "lq_device.cuh"
#include "lq_internal.h"
#include "lq_kernels.h"
#include "lq_xplan.cuh"

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

static inline std::size_t align256(std::size_t b) { return (b + 255) & ~(std::size_t)255; }

constexpr int BATCH_SMEM_BITS = 12;   // whole-state tiles up to n = 12
constexpr int BATCH_TILE_BITS = 12;   // tile width of larger states (the autotuner's
                                      // choice on the n = 16 and uneven batches)

struct BPass {
  PassHeader h;
  int32_t op_first, coef_first;
};

struct BProb {
  int32_t n, k, npasses, pass_first;
  int32_t ngroups, group_first;
  int32_t circ_first, ncirc;
  int32_t tables, xplan;        // xplan: index of its tiled <H> plan, or -1
  int32_t np, out_first;
  int32_t comb_first, pad;
};

struct BatchArgs {
  const BProb* probs;
  const BPass* passes;
  const Op* ops;
  const double* coef;
  const ExpGroup* groups;
  const ExpTerm* terms;
  const Patch* patches;        // per circuit
  const int32_t* circ_prob;    // per circuit
  const int32_t* items;        // circuits in execution order
  const int32_t* comb_first;   // per (problem, parameter): first combine entry
  const int32_t* comb_count;
  const int32_t* comb_circ;    // circuit offset within the problem
  const double* comb_w;
  double* E;                   // per circuit
  double* out;                 // per problem: E, grad[np]
  int32_t* counters;           // [0] next item, [1] finished CTAs
  const XPlan* xplans;         // tiled <H> plans (BProb::xplan)
  double2* scratch;            // per-CTA scratch states
  uint64_t scratch_stride;     // amplitudes
  int32_t nitems, nprobs;
  uint32_t tile_amps;          // amplitudes of the shared-memory tile area; the
                               // <H> tables follow it
};

template <int BLOCK>
__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0;
  for (int w = 0; w < BLOCK / 32; w++) s += red[w];
  return s;
}

// <H> of one state (shared or global memory) by one block.
template <int BLOCK>
__device__ double expval_block(const double2* st, int n, const ExpGroup* groups, int ngroups,
                               const ExpTerm* terms, double* red, double* tab, int tables) {
  if (tables) expval_tables(tab, n, groups, ngroups, terms);
  __syncthreads();
  const double acc = expval_partial(st, n, groups, ngroups, terms, threadIdx.x, BLOCK,
                                    tables ? tab : nullptr);
  return block_sum<BLOCK>(acc, red);
}

// The op with the circuit's patch applied (shifted gate coefficients, final
// scale times the ratio of deferred factors).
__device__ __forceinline__ Op patched(const Op& src, const Patch& pt) {
  Op op = src;
  if ((int)op.cidx == pt.gate &&
      (op.type == OP_PAULI || op.type == OP_PHASE || op.type == OP_PARITY)) {
    if (op.b1 == 0) {
      op.a = pt.a0;
      op.b = pt.b0;
      if (op.type == OP_PAULI) op.mode = (uint8_t)((op.mode & ~3) | pt.mode0);
    } else {
      op.a = pt.a1;
      op.b = pt.b1;
    }
  } else if (op.type == OP_SCALE && (op.mode & 2)) {
    const double ar = op.a, ai = op.b;
    op.a = ar * pt.zr - ai * pt.zi;
    op.b = ar * pt.zi + ai * pt.zr;
    op.mode &= ~1;
  }
  return op;
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, 3) batch_kernel(const __grid_constant__ BatchArgs A) {
  // dynamic shared memory: the tile area (a whole small state or one tile of
  // a scratch state), then the <H> tables of the problem being run
  extern __shared__ double2 sm[];
  __shared__ uint64_t hioff[256];
  __shared__ uint32_t xhlo[32], xhhi[1 << (XP_TILE_BITS - XP_LOW_BITS - 5)];
  __shared__ double red[BLOCK / 32];
  __shared__ int s_item, s_last;
  double* etab = reinterpret_cast<double*>(sm + A.tile_amps);
  double2* __restrict__ scratch = A.scratch + (uint64_t)blockIdx.x * A.scratch_stride;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(&A.counters[0], 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= A.nitems) break;
    const int c = A.items[it];
    const BProb P = A.probs[A.circ_prob[c]];
    const Patch pt = A.patches[c];
    const int n = P.n;
    double e;
    if (n <= P.k) {
      // whole state in shared memory
      const uint32_t T = 1u << n;
      for (uint32_t s = threadIdx.x; s < T; s += BLOCK)
        sm[s] = make_double2(s == 0 ? 1.0 : 0.0, 0.0);
      __syncthreads();
      for (int p = 0; p < P.npasses; p++) {
        const BPass& B = A.passes[P.pass_first + p];
        for (int o = 0; o < B.h.nops; o++) {
          const Op op = patched(A.ops[B.op_first + o], pt);
          apply_op<BLOCK>(sm, T, op, A.coef + B.coef_first, 0, (const double2*)B.h.dtab, nullptr,
                          &pt);
          __syncthreads();
        }
      }
      e = expval_block<BLOCK>(sm, n, A.groups + P.group_first, P.ngroups, A.terms, red, etab,
                              P.tables);
    } else {
      // tile passes over the CTA's scratch state
      for (int p = 0; p < P.npasses; p++) {
        const BPass& B = A.passes[P.pass_first + p];
        const int k = B.h.k, m = B.h.m, kh = k - m;
        const uint32_t T = 1u << k, lowmask = (1u << m) - 1u;
        for (uint32_t j = threadIdx.x; j < (1u << kh); j += BLOCK)
          hioff[j] = deposit(j, B.h.tbits + m, kh);
        __syncthreads();
        for (uint64_t t = 0; t < B.h.ntiles; t++) {
          const uint64_t base = deposit(t, B.h.obits, B.h.nobits);
          if (p == 0) {
            for (uint32_t s = threadIdx.x; s < T; s += BLOCK)
              sm[s] = make_double2((base == 0 && s == 0) ? 1.0 : 0.0, 0.0);
          } else {
            // the next tile of this pass (same tile index, its CTA bits) into
            // L2: one hint per run of 2^m amplitudes, at most one per line
            const int64_t ahead =
                t + 1 < B.h.ntiles
                    ? (int64_t)(deposit(t + 1, B.h.obits, B.h.nobits) - base) : 0;
            const uint32_t pmask = ahead ? (1u << (m < 3 ? m : 3)) - 1u : ~0u;
            for (uint32_t s = threadIdx.x; s < T; s += BLOCK) {
              const double2* src = scratch + (base | hioff[s >> m] | (s & lowmask));
              sm[s] = *src;
              if ((s & pmask) == 0) prefetch_l2(src + ahead);
            }
          }
          __syncthreads();
          for (int o = 0; o < B.h.nops; o++) {
            const Op op = patched(A.ops[B.op_first + o], pt);
            apply_op<BLOCK>(sm, T, op, A.coef + B.coef_first, base, (const double2*)B.h.dtab,
                            nullptr, &pt);
            __syncthreads();
          }
          for (uint32_t s = threadIdx.x; s < T; s += BLOCK)
            scratch[base | hioff[s >> m] | (s & lowmask)] = sm[s];
          __syncthreads();
        }
      }
      if (P.xplan >= 0) {
        // tiled <H> plan: its passes over the scratch state's tiles
        const XPlan& X = A.xplans[P.xplan];
        xp_tables<BLOCK>(X, etab);
        double acc = 0.0;
        for (int q = 0; q < X.npass; q++) {
          const XPass& Q = X.passes[q];
          const int m = Q.m;
          const uint32_t T = 1u << Q.k, lowmask = (1u << m) - 1u;
          __syncthreads();
          xp_offsets(Q, xhlo, xhhi);
          __syncthreads();
          const uint64_t ntiles = 1ull << (n - Q.k);
          for (uint64_t t = 0; t < ntiles; t++) {
            const uint64_t base = deposit(t, Q.obits, Q.nobits);
            const int64_t ahead =
                t + 1 < ntiles ? (int64_t)(deposit(t + 1, Q.obits, Q.nobits) - base) : 0;
            const uint32_t pmask = ahead ? (1u << (m < 3 ? m : 3)) - 1u : ~0u;
            for (uint32_t s = threadIdx.x; s < T; s += BLOCK) {
              const double2* src =
                  scratch + (base | ((uint64_t)(xhlo[(s >> m) & 31u] | xhhi[(s >> m) >> 5]) << m) |
                             (s & lowmask));
              sm[s] = *src;
              if ((s & pmask) == 0) prefetch_l2(src + ahead);
            }
            __syncthreads();
            acc += xp_tile<BLOCK>(sm, T, X, Q, base, xhlo, xhhi, X.coef, etab);
            __syncthreads();
          }
        }
        e = block_sum<BLOCK>(acc, red);
      } else {
        e = expval_block<BLOCK>(scratch, n, A.groups + P.group_first, P.ngroups, A.terms, red,
                                etab, P.tables);
      }
    }
    if (threadIdx.x == 0) A.E[c] = e;
  }
  // the last CTA to finish combines energies into gradients
  __threadfence();
  if (threadIdx.x == 0) s_last = (atomicAdd(&A.counters[1], 1) == (int)gridDim.x - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const volatile double* E = A.E;
  for (int pi = 0; pi < A.nprobs; pi++) {
    const BProb P = A.probs[pi];
    if (threadIdx.x == 0) A.out[P.out_first] = E[P.circ_first];
    for (int i = threadIdx.x; i < P.np; i += BLOCK) {
      double g = 0;
      const int f = A.comb_first[P.comb_first + i], cnt = A.comb_count[P.comb_first + i];
      for (int q = f; q < f + cnt; q++) g += A.comb_w[q] * E[P.circ_first + A.comb_circ[q]];
      A.out[P.out_first + 1 + i] = g;
    }
  }
}

// ---------------------------------------------------------- host side

static const double kPi = 3.14159265358979323846;

static bool two_term_kind(int kind) {
  switch (kind) {
    case LQ_RX: case LQ_RY: case LQ_RZ: case LQ_P: case LQ_CP: case LQ_RXX: case LQ_RYY:
    case LQ_RZZ:
      return true;
    default:
      return false;
  }
}

static Patch patch_for(const lq_gate& G, int g, double theta_base, double theta) {
  Patch p;
  std::memset(&p, 0, sizeof p);
  AngleCoefs a0, a1;
  angle_coefs(G.kind, theta_base, a0);
  angle_coefs(G.kind, theta, a1);
  p.gate = g;
  p.mode0 = a1.mode0;
  p.mode1 = a1.mode1;
  p.a0 = a1.a0;
  p.b0 = a1.b0;
  p.a1 = a1.a1;
  p.b1 = a1.b1;
  double den = a0.zr * a0.zr + a0.zi * a0.zi;
  p.zr = (a1.zr * a0.zr + a1.zi * a0.zi) / den;
  p.zi = (a1.zi * a0.zr - a1.zr * a0.zi) / den;
  return p;
}

static Patch unpatched() {
  Patch p;
  std::memset(&p, 0, sizeof p);
  p.gate = -2;
  p.zr = 1.0;
  return p;
}

// Build the circuits of a problem.  general = 0: two-term rule, every
// parameter on at most one gate (else LQ_ERR_UNSUPPORTED); general = 1:
// four-term rule for controlled rotations, shared parameters summed.
lq_status make_problem(int n, const lq_gate* gates, int ng, const double* params, int np,
                       const lq_pauli_term* terms, int nt, bool want_grad, bool general,
                       HostProblem& hp) {
  lq_status st = check_n(n);
  if (st) return st;
  st = check_gates(n, gates, ng, params, np);
  if (st) return st;
  st = check_terms(n, terms, nt);
  if (st) return st;
  hp.n = n;
  hp.ng = ng;
  hp.np = np;
  hp.nt = nt;
  hp.gates = gates;
  hp.params = params;
  hp.terms = terms;
  hp.patches.assign(1, unpatched());
  hp.comb.assign((std::size_t)np, {});
  if (!want_grad) return LQ_OK;
  std::vector<int> uses((std::size_t)np, 0);
  for (int g = 0; g < ng; g++) {
    const lq_gate& G = gates[g];
    if (G.param < 0) continue;
    const bool two = two_term_kind(G.kind);
    const bool four = G.kind == LQ_CRX || G.kind == LQ_CRY || G.kind == LQ_CRZ;
    if (!general) {
      if (!two)
        return fail(LQ_ERR_UNSUPPORTED,
                    "gate %d (kind %d) needs a generalised shift rule; use "
                    "lq_param_shift_grad_general or lq_adjoint_grad", g, G.kind);
      if (uses[G.param]++)
        return fail(LQ_ERR_UNSUPPORTED,
                    "parameter %d drives several gates; use lq_param_shift_grad_general",
                    G.param);
    }
    double th = G.angle + params[G.param];
    double sh[4], w[4];
    int cnt = 0;
    if (two) {
      sh[0] = kPi / 2; w[0] = 0.5;
      sh[1] = -kPi / 2; w[1] = -0.5;
      cnt = 2;
    } else if (four) {
      const double r2 = std::sqrt(2.0);
      const double d1 = (r2 + 1) / (4 * r2), d2 = (r2 - 1) / (4 * r2);
      sh[0] = kPi / 2; w[0] = d1;
      sh[1] = -kPi / 2; w[1] = -d1;
      sh[2] = 3 * kPi / 2; w[2] = -d2;
      sh[3] = -3 * kPi / 2; w[3] = d2;
      cnt = 4;
    }
    for (int j = 0; j < cnt; j++) {
      hp.comb[G.param].push_back({(int)hp.patches.size(), w[j]});
      hp.patches.push_back(patch_for(G, g, th, th + sh[j]));
    }
  }
  return LQ_OK;
}

// Device layout of a batch run, computed on the host.
struct BatchPlan {
  std::vector<BProb> probs;
  std::vector<BPass> passes;
  std::vector<Op> ops;
  std::vector<double> coef;
  std::vector<ExpGroup> groups;
  std::vector<ExpTerm> terms;
  std::vector<Patch> patches;
  std::vector<int32_t> circ_prob, items, comb_first, comb_count, comb_circ;
  std::vector<double> comb_w;
  std::vector<XPlan> xplans;
  int kmax = 0, nmax_scratch = 0, nout = 0;
  int etab_words = 0;   // doubles of <H> tables after the tile area
  std::size_t program_bytes = 0;
};

// The largest <H> table area a launch reserves: chunk tables of a 34-qubit
// diagonal group (class tables of a plan are smaller).
constexpr int BATCH_MAX_TABLE_WORDS = 256 * ((34 + EXP_CHUNK_BITS - 1) / EXP_CHUNK_BITS);

// Dynamic shared memory of a launch: the tile area and the <H> tables.
static std::size_t batch_smem(const BatchPlan& B) {
  return (sizeof(double2) << B.kmax) + sizeof(double) * (std::size_t)B.etab_words;
}

static lq_status plan_batch(const std::vector<HostProblem>& hps, BatchPlan& B,
                            int tile_bits = BATCH_TILE_BITS) {
  std::vector<double> cost;
  for (std::size_t pi = 0; pi < hps.size(); pi++) {
    const HostProblem& hp = hps[pi];
    const int n = hp.n;
    LOp* ops = nullptr;
    std::size_t nops = 0;
    double zr, zi;
    lq_status st = lower_circuit(n, hp.gates, hp.ng, hp.params, hp.np, &ops, &nops, &zr, &zi);
    if (st) return st;
    ScheduleOptions opt;
    opt.k = n <= BATCH_SMEM_BITS ? n : tile_bits;
    opt.force_scale = true;
    // one-bit phases of parametrised gates merge too: a shifted circuit's
    // patch replaces its gate's factor when the kernel builds the tables
    opt.merge_params = true;
    // phases move to fewer merge points (each factor keeps its gate, so the
    // patch still finds it); the schedule is built once per problem, so the
    // host time of the search does not count against small states
    opt.sink_phases = true;
    opt.sink_min_qubits = 0;
    Schedule S;
    st = schedule_ops(n, ops, nops, zr, zi, opt, S);
    double flops = 0;
    for (std::size_t i = 0; i < nops; i++) flops += op_flops(ops[i], n);
    delete[] ops;
    if (st) return st;
    BProb P;
    std::memset(&P, 0, sizeof P);
    P.n = n;
    P.k = opt.k < n ? opt.k : n;
    P.npasses = S.npasses;
    P.pass_first = (int)B.passes.size();
    for (int p = 0; p < S.npasses; p++) {
      BPass bp;
      bp.h = S.passes[p].h;
      if (bp.h.flags & PF_DYADIC) {
        cudaError_t e;
        bp.h.dtab = dyadic_tables(&e, nullptr);
        if (!bp.h.dtab) return fail(LQ_ERR_CUDA, "dyadic tables: %s", cudaGetErrorString(e));
      }
      bp.op_first = (int)B.ops.size();
      bp.coef_first = (int)B.coef.size();
      for (int o = 0; o < bp.h.nops; o++) B.ops.push_back(S.passes[p].ops[o]);
      int ncoef = 0;
      for (int o = 0; o < bp.h.nops; o++) {
        const Op& d = S.passes[p].ops[o];
        if (d.type == OP_PAIR_GEN) ncoef = std::max(ncoef, (int)d.cidx + 8);
        if (d.type == OP_QUAD_GEN) ncoef = std::max(ncoef, (int)d.cidx + 32);
        if (d.type == OP_DPHASE) ncoef = std::max(ncoef, (int)d.cidx + 4 * (int)d.x_loc);
        if (d.type == OP_LPHASE) ncoef = std::max(ncoef, (int)d.cidx + LPHASE_FAC * (int)d.x_loc);
      }
      for (int c = 0; c < ncoef; c++) B.coef.push_back(S.passes[p].coef[c]);
      B.passes.push_back(bp);
    }
    // Hamiltonian groups (absolute term indices)
    int nch = exp_chunk_count(hp.terms, hp.nt);
    std::vector<ExpParams> ch((std::size_t)nch);
    int got = hp.nt ? build_exp_chunks(n, hp.terms, hp.nt, ch.data(), nch) : 0;
    P.group_first = (int)B.groups.size();
    for (int c = 0; c < got; c++) {
      int tbase = (int)B.terms.size();
      int used = 0;
      for (int g = 0; g < ch[c].ngroups; g++) used += ch[c].groups[g].count;
      for (int t = 0; t < used; t++) B.terms.push_back(ch[c].terms[t]);
      for (int g = 0; g < ch[c].ngroups; g++) {
        ExpGroup G = ch[c].groups[g];
        G.first += tbase;
        B.groups.push_back(G);
      }
    }
    P.ngroups = (int)B.groups.size() - P.group_first;
    for (int c = 0; c < got; c++) P.tables |= ch[c].tables;
    // a state wider than the tile area takes the tiled <H> plan when its
    // terms fit one plan (else the per-group sweeps of expval_block)
    P.xplan = -1;
    int words = P.tables ? 256 * ((n + EXP_CHUNK_BITS - 1) / EXP_CHUNK_BITS) : 0;
    if (n > P.k && hp.nt > 0) {
      std::vector<XPlan> xp;
      std::vector<lq_pauli_term> wide;
      const int kt = P.k < XP_TILE_BITS ? P.k : XP_TILE_BITS;
      if (build_xplans(n, hp.terms, hp.nt, kt, xp, wide) == 1 && wide.empty() &&
          xp_table_words(xp[0]) <= BATCH_MAX_TABLE_WORDS) {
        P.xplan = (int)B.xplans.size();
        B.xplans.push_back(xp[0]);
        words = xp_table_words(xp[0]);
      }
    }
    B.etab_words = std::max(B.etab_words, words);
    P.circ_first = (int)B.patches.size();
    P.ncirc = (int)hp.patches.size();
    P.np = hp.np;
    P.out_first = B.nout;
    B.nout += 1 + hp.np;
    P.comb_first = (int)B.comb_first.size();
    for (int i = 0; i < hp.np; i++) {
      B.comb_first.push_back((int)B.comb_circ.size());
      B.comb_count.push_back((int)hp.comb[i].size());
      for (auto& cw : hp.comb[i]) {
        B.comb_circ.push_back(cw.first);
        B.comb_w.push_back(cw.second);
      }
    }
    double ecost = 0;
    for (int t = 0; t < hp.nt; t++) ecost += 2.0;
    double per = flops + (ecost + 6.0) * std::ldexp(1.0, n);
    for (std::size_t c = 0; c < hp.patches.size(); c++) {
      B.patches.push_back(hp.patches[c]);
      B.circ_prob.push_back((int)pi);
      cost.push_back(per);
    }
    B.kmax = std::max(B.kmax, P.k);
    if (n > P.k) B.nmax_scratch = std::max(B.nmax_scratch, n);
    B.probs.push_back(P);
  }
  // largest circuits first
  B.items.resize(B.patches.size());
  for (std::size_t i = 0; i < B.items.size(); i++) B.items[i] = (int)i;
  std::stable_sort(B.items.begin(), B.items.end(),
                   [&](int a, int b) { return cost[a] > cost[b]; });
  return LQ_OK;
}

// Device memory the per-CTA scratch states of one launch may take: 40% of
// the device's memory (115 GB on a GB300), at least 4 GiB.
static std::size_t scratch_budget() {
  static std::size_t cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    (void)cudaGetLastError();
    return (std::size_t)48 << 30;
  }
  if (!cached[dev]) {
    cudaDeviceProp pr;
    std::size_t total = 0;
    if (cudaGetDeviceProperties(&pr, dev) == cudaSuccess) total = pr.totalGlobalMem;
    (void)cudaGetLastError();
    std::size_t b = total / 10 * 4;
    cached[dev] = b < ((std::size_t)4 << 30) ? ((std::size_t)4 << 30) : b;
  }
  return cached[dev];
}

// The kernel's shared-memory limit: the largest tile area and table area.
static cudaError_t configure_batch_kernel() {
  static std::atomic<uint64_t> configured{0};
  return once_per_device(configured, [] {
    return cudaFuncSetAttribute(batch_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)((sizeof(double2) << BATCH_SMEM_BITS) +
                                      sizeof(double) * BATCH_MAX_TABLE_WORDS));
  });
}

static int batch_grid(const BatchPlan& B) {
  const std::size_t smem = batch_smem(B);
  // resident CTAs per SM from the occupancy query (registers, static and
  // dynamic shared memory); without a device, an estimate from shared memory
  static const bool have_device = [] {
    int c = 0;
    const bool ok = cudaGetDeviceCount(&c) == cudaSuccess && c > 0;
    (void)cudaGetLastError();
    return ok;
  }();
  int per_sm = 0;
  if (!have_device || configure_batch_kernel() != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<256>, 256, smem) !=
          cudaSuccess ||
      per_sm < 1) {
    (void)cudaGetLastError();
    per_sm = (int)((228u << 10) / (smem + (8u << 10)));
    per_sm = per_sm < 1 ? 1 : per_sm > 3 ? 3 : per_sm;
  }
  int g = sm_count() * per_sm;
  if ((int)B.items.size() < g) g = (int)B.items.size();
  if (B.nmax_scratch > 0) {
    // keep the scratch states within the device's scratch budget
    std::size_t sb = sizeof(double2) << B.nmax_scratch;
    std::size_t cap = scratch_budget() / sb;
    if (cap < 1) cap = 1;
    if ((std::size_t)g > cap) g = (int)cap;
  }
  return g < 1 ? 1 : g;
}

template <typename T>
static std::size_t vbytes(const std::vector<T>& v) {
  return align256(sizeof(T) * (v.size() > 0 ? v.size() : 1));
}

static std::size_t batch_bytes(const BatchPlan& B, int grid) {
  std::size_t b = 0;
  b += vbytes(B.probs) + vbytes(B.passes) + vbytes(B.ops) + vbytes(B.coef) + vbytes(B.groups) +
       vbytes(B.terms) + vbytes(B.patches) + vbytes(B.circ_prob) + vbytes(B.items) +
       vbytes(B.comb_first) + vbytes(B.comb_count) + vbytes(B.comb_circ) + vbytes(B.comb_w) +
       vbytes(B.xplans);
  b += align256(sizeof(double) * B.patches.size());   // E
  b += align256(sizeof(double) * (std::size_t)B.nout); // out
  b += align256(sizeof(int32_t) * 2);                  // counters
  if (B.nmax_scratch > 0) b += (sizeof(double2) << B.nmax_scratch) * (std::size_t)grid;
  return b;
}

// ------------------------------------------------------ graph replay
//
// A batch run is four stream operations: upload the program image, reset the
// two counters, the persistent kernel, download the results.  They are
// captured once per layout (workspace allocation, section sizes, grid) into
// a CUDA graph on an internal stream of the device and replayed; a replay
// only rewrites the pinned staging image (new angles give new coefficients,
// never a new layout).  Events order the replay after the caller's stream
// work and the caller's stream after the replay.
//
// A graph's copy and memset nodes belong to the allocation they were
// captured on, not just to its address: after the caller frees a workspace,
// a new allocation can come back at the same address (a caching allocator
// returning memory to the driver and taking it again does this), and
// replaying the old graph on it faulted or left the upload in the freed
// memory.  So an entry also records the allocation's process-wide buffer id
// and is used only while the workspace is that same allocation; when the id
// cannot be read, the graph is not kept.

// Process-wide unique id of the device allocation holding p, 0 if unknown.
static unsigned long long allocation_id(const void* p) {
  using GetAttr = CUresult (*)(void*, CUpointer_attribute, CUdeviceptr);
  static GetAttr fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuPointerGetAttribute", &f, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    (void)cudaGetLastError();
    return reinterpret_cast<GetAttr>(f);
  }();
  if (!fn) return 0;
  unsigned long long id = 0;
  if (fn(&id, CU_POINTER_ATTRIBUTE_BUFFER_ID, (CUdeviceptr)(uintptr_t)p) != CUDA_SUCCESS) return 0;
  return id;
}

struct GraphEntry {
  int device = -1;
  void* ws = nullptr;
  unsigned long long ws_id = 0;   // buffer id of the workspace allocation
  std::vector<std::size_t> key;
  cudaGraphExec_t exec = nullptr;
  char* h_image = nullptr;      // pinned
  double* h_out = nullptr;      // pinned
  std::size_t image = 0, nout = 0;
  uint64_t last_use = 0;
};

static std::mutex g_graph_mu;
static std::vector<GraphEntry> g_graphs;
static uint64_t g_graph_clock = 0;
static cudaStream_t g_graph_stream[64] = {nullptr};
static cudaEvent_t g_ev_in[64] = {nullptr}, g_ev_out[64] = {nullptr};
constexpr std::size_t kMaxGraphs = 8;

static void drop_entry(GraphEntry& e) {
  if (e.exec) cudaGraphExecDestroy(e.exec);
  if (e.h_image) cudaFreeHost(e.h_image);
  if (e.h_out) cudaFreeHost(e.h_out);
  e = GraphEntry();
}

// Run the batch; results (per problem E then grad) into host vector `out`.
static lq_status run_batch(const BatchPlan& B, void* workspace, std::size_t ws_bytes,
                           cudaStream_t s, std::vector<double>& out) {
  const int grid = batch_grid(B);
  if (!workspace || ws_bytes < batch_bytes(B, grid))
    return fail(LQ_ERR_OOM, "workspace too small: %zu < %zu", ws_bytes, batch_bytes(B, grid));
  char* p = (char*)workspace;
  BatchArgs A;
  std::memset(&A, 0, sizeof A);
  std::vector<std::size_t> key;
  std::size_t off = 0;
  struct Sec { const void* src; std::size_t n, cap; };
  std::vector<Sec> secs;
  auto place = [&](const void* src, std::size_t n, std::size_t cap) {
    std::size_t at = off;
    secs.push_back({src, n, cap});
    key.push_back(cap);
    off += cap;
    return p + at;
  };
#define LQ_PLACE(vec, field, type) \
  A.field = (type)place(vec.data(), sizeof(vec[0]) * vec.size(), vbytes(vec))
  LQ_PLACE(B.probs, probs, const BProb*);
  LQ_PLACE(B.passes, passes, const BPass*);
  LQ_PLACE(B.ops, ops, const Op*);
  LQ_PLACE(B.coef, coef, const double*);
  LQ_PLACE(B.groups, groups, const ExpGroup*);
  LQ_PLACE(B.terms, terms, const ExpTerm*);
  LQ_PLACE(B.patches, patches, const Patch*);
  LQ_PLACE(B.circ_prob, circ_prob, const int32_t*);
  LQ_PLACE(B.items, items, const int32_t*);
  LQ_PLACE(B.comb_first, comb_first, const int32_t*);
  LQ_PLACE(B.comb_count, comb_count, const int32_t*);
  LQ_PLACE(B.comb_circ, comb_circ, const int32_t*);
  LQ_PLACE(B.comb_w, comb_w, const double*);
  LQ_PLACE(B.xplans, xplans, const XPlan*);
#undef LQ_PLACE
  const std::size_t image = off;
  A.E = (double*)(p + off);
  off += align256(sizeof(double) * B.patches.size());
  A.out = (double*)(p + off);
  off += align256(sizeof(double) * (std::size_t)B.nout);
  A.counters = (int32_t*)(p + off);
  off += align256(sizeof(int32_t) * 2);
  A.scratch = (double2*)(p + off);
  A.scratch_stride = B.nmax_scratch > 0 ? (1ull << B.nmax_scratch) : 0;
  A.nitems = (int)B.items.size();
  A.nprobs = (int)B.probs.size();
  A.tile_amps = 1u << B.kmax;
  const std::size_t smem = batch_smem(B);
  key.push_back(B.patches.size());
  key.push_back((std::size_t)B.nout);
  key.push_back((std::size_t)grid);
  key.push_back(smem);
  key.push_back((std::size_t)A.scratch_stride);
  key.push_back((std::size_t)A.nitems);
  key.push_back((std::size_t)A.nprobs);
  int dev = 0;
  LQ_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(LQ_ERR_INVALID_ARG, "device %d", dev);
  LQ_CUDA(configure_batch_kernel());
  std::lock_guard<std::mutex> lock(g_graph_mu);
  if (!g_graph_stream[dev]) {
    LQ_CUDA(cudaStreamCreateWithFlags(&g_graph_stream[dev], cudaStreamNonBlocking));
    LQ_CUDA(cudaEventCreateWithFlags(&g_ev_in[dev], cudaEventDisableTiming));
    LQ_CUDA(cudaEventCreateWithFlags(&g_ev_out[dev], cudaEventDisableTiming));
  }
  cudaStream_t gs = g_graph_stream[dev];
  const unsigned long long ws_id = allocation_id(workspace);
  // entries on a freed workspace (the address now names another allocation),
  // or left by a run whose allocation was unknown
  for (std::size_t i = 0; i < g_graphs.size();) {
    if (g_graphs[i].device == dev && g_graphs[i].ws == workspace &&
        (g_graphs[i].ws_id != ws_id || ws_id == 0)) {
      drop_entry(g_graphs[i]);
      g_graphs.erase(g_graphs.begin() + (long)i);
    } else {
      i++;
    }
  }
  GraphEntry* E = nullptr;
  for (auto& e : g_graphs)
    if (e.device == dev && e.ws == workspace && e.ws_id == ws_id && e.key == key) E = &e;
  if (!E) {
    // capture a new graph for this layout (evict the least recently used)
    if (g_graphs.size() >= kMaxGraphs) {
      std::size_t lru = 0;
      for (std::size_t i = 1; i < g_graphs.size(); i++)
        if (g_graphs[i].last_use < g_graphs[lru].last_use) lru = i;
      drop_entry(g_graphs[lru]);
      g_graphs.erase(g_graphs.begin() + (long)lru);
    }
    GraphEntry ne;
    ne.device = dev;
    ne.ws = workspace;
    ne.ws_id = ws_id;
    ne.key = key;
    ne.image = image;
    ne.nout = (std::size_t)B.nout;
    LQ_CUDA(cudaHostAlloc((void**)&ne.h_image, image > 0 ? image : 256, cudaHostAllocPortable));
    LQ_CUDA(cudaHostAlloc((void**)&ne.h_out, sizeof(double) * (ne.nout > 0 ? ne.nout : 1),
                          cudaHostAllocPortable));
    cudaGraph_t graph;
    LQ_CUDA(cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal));
    cudaMemcpyAsync(p, ne.h_image, image, cudaMemcpyHostToDevice, gs);
    cudaMemsetAsync(A.counters, 0, sizeof(int32_t) * 2, gs);
    batch_kernel<256><<<grid, 256, smem, gs>>>(A);
    cudaMemcpyAsync(ne.h_out, A.out, sizeof(double) * B.nout, cudaMemcpyDeviceToHost, gs);
    cudaError_t ce = cudaStreamEndCapture(gs, &graph);
    if (ce == cudaSuccess) {
      ce = cudaGraphInstantiate(&ne.exec, graph, 0);
      cudaGraphDestroy(graph);
    }
    if (ce != cudaSuccess) {
      drop_entry(ne);
      (void)cudaGetLastError();
      return fail(LQ_ERR_CUDA, "batch graph capture: %s", cudaGetErrorString(ce));
    }
    g_graphs.push_back(ne);
    E = &g_graphs.back();
  }
  E->last_use = ++g_graph_clock;
  std::size_t at = 0;
  for (const Sec& sc : secs) {
    if (sc.n) std::memcpy(E->h_image + at, sc.src, sc.n);
    at += sc.cap;
  }
  LQ_CUDA(cudaEventRecord(g_ev_in[dev], s));
  LQ_CUDA(cudaStreamWaitEvent(gs, g_ev_in[dev], 0));
  LQ_CUDA(cudaGraphLaunch(E->exec, gs));
  LQ_CUDA(cudaEventRecord(g_ev_out[dev], gs));
  LQ_CUDA(cudaStreamWaitEvent(s, g_ev_out[dev], 0));
  LQ_CUDA(cudaStreamSynchronize(gs));
  out.assign(E->h_out, E->h_out + B.nout);
  if (ws_id == 0) {   // allocation unknown: do not keep the graph
    drop_entry(*E);
    g_graphs.erase(g_graphs.begin() + (E - g_graphs.data()));
  }
  return LQ_OK;
}

// The tile widths the autotuner may pick for states larger than shared
// memory; the workspace size covers every one of them.
static const int kBatchTileChoices[] = {9, 10, 11, 12};

static bool batch_has_tiles(const std::vector<HostProblem>& hps) {
  for (const HostProblem& hp : hps)
    if (hp.n > BATCH_SMEM_BITS) return true;
  return false;
}

// Structure of a batch for the autotuner's cache: per problem n, the gate
// structure, the number of circuits and of terms.
static uint64_t batch_structure(const std::vector<HostProblem>& hps) {
  uint64_t h = 0x6c71626174636821ull;
  for (const HostProblem& hp : hps) {
    const uint64_t rec[3] = {circuit_structure_hash(hp.n, hp.gates, hp.ng),
                             (uint64_t)hp.patches.size(), (uint64_t)hp.nt};
    for (uint64_t r : rec) h = (h ^ r) * 1099511628211ull + (h >> 29);
  }
  return h;
}

std::size_t batch_workspace_for(const std::vector<HostProblem>& hps, lq_status* st_out) {
  std::size_t need = 0;
  for (int k : kBatchTileChoices) {
    BatchPlan B;
    lq_status st = plan_batch(hps, B, k);
    if (st_out) *st_out = st;
    if (st) return 0;
    need = std::max(need, batch_bytes(B, batch_grid(B)));
    if (!batch_has_tiles(hps)) break;   // the tile width does not matter
  }
  return need;
}

lq_status batch_run(const std::vector<HostProblem>& hps, void* ws, std::size_t ws_bytes,
                    cudaStream_t s, std::vector<double>& out) {
  BatchPlan B;
  int k = BATCH_TILE_BITS;
  if (batch_has_tiles(hps)) tuned_batch_tile(batch_structure(hps), &k);
  lq_status st = plan_batch(hps, B, k);
  if (st) return st;
  return run_batch(B, ws, ws_bytes, s, out);
}

// Time the persistent batched launch for every tile width (host wall clock
// around the graph-replayed run, which synchronises) and record the fastest.
lq_status batch_autotune(const std::vector<HostProblem>& hps, void* ws, std::size_t ws_bytes,
                         cudaStream_t s, lq_tune_result* res) {
  double best = 1e300, def_ms = -1;
  int bestk = BATCH_TILE_BITS, cands = 0;
  const bool tiles = batch_has_tiles(hps);
  for (int k : kBatchTileChoices) {
    if (!tiles && k != BATCH_TILE_BITS) continue;
    BatchPlan B;
    lq_status st = plan_batch(hps, B, k);
    if (st) return st;
    std::vector<double> out;
    double ms = 1e300;
    for (int rep = 0; rep < 3; rep++) {
      const auto t0 = std::chrono::steady_clock::now();
      st = run_batch(B, ws, ws_bytes, s, out);
      if (st) return st;
      const double t = std::chrono::duration<double, std::milli>(
                           std::chrono::steady_clock::now() - t0).count();
      if (rep > 0 && t < ms) ms = t;   // the first run captures the graph
    }
    cands++;
    if (k == BATCH_TILE_BITS) def_ms = ms;
    if (ms < best) {
      best = ms;
      bestk = k;
    }
  }
  if (tiles) record_batch_tile(batch_structure(hps), bestk, best, def_ms);
  res->tile_bits = bestk;
  res->low_bits = 5;
  res->phase_table = 0;
  res->candidates = cands;
  res->ms = best;
  res->ms_default = def_ms;
  return LQ_OK;
}

}  // namespace lq

using namespace lq;

extern "C" {

size_t lq_batch_workspace_size(const lq_problem* problems, int count) {
  if (!problems || count <= 0) return 0;
  std::vector<HostProblem> hps((std::size_t)count);
  for (int i = 0; i < count; i++) {
    const lq_problem& q = problems[i];
    if (make_problem(q.n, q.gates, q.ng, q.params, q.np, q.terms, q.nt, q.want_grad != 0, false,
                     hps[i]))
      return 0;
  }
  return batch_workspace_for(hps, nullptr);
}

lq_status lq_autotune_batch(const lq_problem* problems, int count, void* workspace,
                            size_t ws_bytes, lq_tune_result* out, lq_stream stream) {
  if (!problems || count <= 0 || !out) return fail(LQ_ERR_INVALID_ARG, "no problems");
  std::vector<HostProblem> hps((std::size_t)count);
  for (int i = 0; i < count; i++) {
    const lq_problem& q = problems[i];
    lq_status st = make_problem(q.n, q.gates, q.ng, q.params, q.np, q.terms, q.nt,
                                q.want_grad != 0, false, hps[i]);
    if (st) return st;
  }
  return batch_autotune(hps, workspace, ws_bytes, (cudaStream_t)stream, out);
}

lq_status lq_batch_param_shift(const lq_problem* problems, int count, void* workspace,
                               size_t ws_bytes, lq_stream stream) {
  if (!problems || count <= 0) return fail(LQ_ERR_INVALID_ARG, "no problems");
  std::vector<HostProblem> hps((std::size_t)count);
  for (int i = 0; i < count; i++) {
    const lq_problem& q = problems[i];
    if (!q.energy || (q.want_grad && q.np > 0 && !q.grad))
      return fail(LQ_ERR_INVALID_ARG, "problem %d: NULL output", i);
    lq_status st = make_problem(q.n, q.gates, q.ng, q.params, q.np, q.terms, q.nt,
                                q.want_grad != 0, false, hps[i]);
    if (st) return st;
  }
  std::vector<double> out;
  lq_status st = batch_run(hps, workspace, ws_bytes, (cudaStream_t)stream, out);
  if (st) return st;
  std::size_t at = 0;
  for (int i = 0; i < count; i++) {
    const lq_problem& q = problems[i];
    *q.energy = out[at];
    if (q.want_grad)
      for (int j = 0; j < q.np; j++) q.grad[j] = out[at + 1 + j];
    at += 1 + q.np;
  }
  return LQ_OK;
}

}  // extern "C"
