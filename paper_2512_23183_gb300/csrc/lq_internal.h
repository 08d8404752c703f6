// lq_internal.h -- internal data structures of the lq library: the lowered
// "op" encoding of gates executed by the tile-pass kernels, the pass
// descriptors, and the host-side compiler interface.
//
// A gate of the circuit (Sec. II-A) is lowered into ops that work on a
// shared-memory tile of 2^k amplitudes whose index bits are a chosen set of
// k state-index bits ("tile bits"; the lowest m are always the contiguous low
// bits so tile loads are coalesced).  Every other bit of the index is fixed
// for the tile ("CTA bits").  Mixing ops (pairs/quads of amplitudes) need
// their mixing bits inside the tile; diagonal ops and control conditions may
// use any bit: for CTA bits they reduce to per-tile constants.
//
// FP64 economy.  On GB300 an FP64 instruction costs ~1/3 of a 32-byte HBM pass
// per amplitude (1.19 TFLOP/s FP64 against 6.8 TB/s), so ops are encoded in
// the forms with the fewest FP64 instructions:
//   * Pauli rotations exp(-i theta P / 2) in tangent form
//       out_i = c (psi_i + t w_i psi_{i^x}),  t = tan(theta/2)
//     (or cotangent form when |t| > 1) with the real factor c deferred into a
//     global scalar: 2 FP64 FMAs per amplitude;
//   * H as (a + b, a - b) with 1/sqrt2 deferred: 2 FP64 adds per amplitude;
//   * permutations, signs and multiplications by +-i (X, Y, Z, S, CNOT, CY,
//     CZ, SWAP, CCX) move or flip sign bits only: no FP64 instruction;
//   * diagonal phases (RZ, P, CP, T, RZZ) multiply only the amplitudes they
//     change, with global phases deferred.
// The deferred scalar is applied once, by an OP_SCALE at the end.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include "../../include/lq.h"

#if defined(__CUDACC__)
#define LQ_HD __host__ __device__
#else
#define LQ_HD
#endif

namespace lq {

// ------------------------------------------------------------------ ops

enum OpType : uint8_t {
  OP_PAULI = 0,   // out_i = alpha psi_i + beta w_i psi_{i^x}  (see PauliMode)
  OP_H,           // (a, b) -> (a + b, a - b) on tile bit b0
  OP_PAIR_GEN,    // 2x2 complex matrix on tile bit b0 (coef pool)
  OP_QUAD_GEN,    // 4x4 complex matrix on tile bits b0 (high), b1 (low)
  OP_SWAP,        // exchange tile bits b0 and b1
  OP_PHASE,       // multiply matching amplitudes by (a + i b)
  OP_SIGN,        // negate matching amplitudes
  OP_MULI,        // multiply matching amplitudes by i^mode
  OP_PARITY,      // multiply amplitudes with odd popcount(idx & z) by (a + i b)
  OP_SCALE,       // multiply every amplitude by (a + i b) (mode 1: b == 0)
  OP_GRAD,        // adjoint: accumulate Im <lam| G |psi> into slot cidx
  OP_DPHASE,      // merged dyadic phases: exp(2 pi i E(idx) / 2^34), E = sum of
                  // integer weights of the factors whose conditions hold
                  // (x_loc factors at coef[cidx..], 4 doubles each)
  OP_LPHASE,      // merged one-bit phases: product of the unit factors w_f whose
                  // single condition bit holds (x_loc factors at coef[cidx..],
                  // LPHASE_FAC doubles each)
  OP_TYPE_COUNT
};

// OP_PAULI sub-modes (low 2 bits of Op::mode; bits 2-3 hold k0, the power of
// i of the fixed phase, w_i = i^k0 (-1)^popcount((i ^ x) & z)).
enum PauliMode : uint8_t {
  PM_TAN = 0,   // alpha = 1, beta = a     (deferred factor cos)
  PM_COT = 1,   // alpha = a, beta = 1     (deferred factor sin)
  PM_GEN = 2,   // alpha = a, beta = b     (controlled rotations)
  PM_PERM = 3   // alpha = 0, beta = 1     (X, Y, CNOT, CY, CCX)
};

// A condition is "(idx & cm) == cv"; split into tile-local bits (cm_loc,
// cv_loc: positions are tile-local bit numbers) and CTA bits (cm_glob,
// cv_glob: global bit positions).
struct Op {
  uint8_t type;
  uint8_t mode;       // Pauli mode | k0 << 2; OP_MULI: power of i; OP_SCALE:
                      // bit 0 real factor, bit 1 final scale of the circuit
  uint8_t b0, b1;     // tile-local bit positions (b1 of a diagonal or Pauli
                      // op: index of the op among its gate's ops)
  uint32_t cidx;      // coef-pool index (PAIR_GEN/QUAD_GEN), grad slot
                      // (OP_GRAD), else source gate index
  uint32_t cm_loc, cv_loc;
  uint32_t x_loc, z_loc;
  uint64_t cm_glob, cv_glob;
  uint64_t z_glob;
  double a, b;
};
static_assert(sizeof(Op) == 64, "Op must stay 64 bytes");

constexpr int DYADIC_BITS = 34;    // dyadic phases are multiples of 2 pi / 2^34
constexpr int LPHASE_FAC = 6;      // doubles per OP_LPHASE factor: tile-local cm | cv << 32,
                                   // CTA cm, CTA cv, re, im, source gate
// Marker in an OP_LPHASE factor's CTA cv: a parity factor, w on the
// amplitudes with odd popcount(idx & mask) (mask = its tile-local cm, at most
// one bit, and CTA cm), instead of the condition (idx & cm) == cv.
constexpr uint64_t kLphaseParity = 1ull << 63;
constexpr int DYADIC_HALF = 17;    // two-level table: 2^17 + 2^17 entries
constexpr int MAX_TILE_BITS = 13;   // 2^13 amplitudes = 128 KiB of shared memory
constexpr int PASS_HI_BITS = 9;    // pass_kernel maps up to 9 tile bits above the
                                   // contiguous low run (a 512-entry offset table)
constexpr int MAX_OPS = 384;        // per pass (kernel-parameter budget)
constexpr int MAX_COEF = 1000;      // doubles per pass coefficient pool (the
                                    // pass stays within the 32764-byte limit
                                    // of a kernel parameter)

// Everything a tile pass needs; passed by value as a __grid_constant__
// kernel parameter (< 32 KiB), so a pass needs no device allocation.
struct PassHeader {
  int32_t n, k, m, nops;
  int32_t nobits;
  int32_t flags;          // PF_* below
  int32_t ltab_op;        // PF_LTAB: index of the table-mode OP_LPHASE
  int32_t dtab_words;     // PF_DTAB: 64-bit words of the per-CTA dyadic tables
  int32_t dfull_entries;  // PF_DFULL: double2 entries of the per-CTA full phase tables
  int8_t ndefer;          // PF_DFULL: deferred per-tile phase sums (<= 8)
  int8_t ndbits;          // bits of the deferred phase table's index (<= 6)
  int8_t dbits[6];        // their tile-local positions, ascending
  uint8_t dmask[8], dval[8];   // per deferred sum: condition over the index bits
  uint8_t dpre;           // deferred sums applied after the load (bit per slot);
                          // the others are applied at the store
  uint16_t dsc;           // PF_DSCALE: coef[dsc], coef[dsc + 1] = the circuit's
                          // final scalar (re, im)
  uint64_t ntiles;        // 2^(n-k)
  const void* dtab;       // dyadic phase tables (device), set at launch
  int8_t tbits[16];       // tile-local bit j -> global bit position
  int8_t obits[48];       // CTA bits (global positions), ascending
};
enum PassFlags : int32_t {
  PF_INIT_ZERO = 1,       // do not load: start from |0...0> (whole-state tile)
  PF_NO_STORE = 2,        // do not store the tile back
  PF_DYADIC = 4,          // the pass has OP_DPHASE ops (needs dtab)
  PF_LTAB = 8,            // ops[ltab_op] is a table-mode OP_LPHASE: its 2^k-entry
                          // phase table is built once per CTA (pass_kernel only)
  PF_DTAB = 16,           // some OP_DPHASE ops are in table mode (pass_kernel only)
  PF_BFLY = 64,           // some full-mode OP_DPHASE ops run as butterflies with the
                          // OP_H after them (DP_BFLY; pass_kernel's butterfly variant)
  PF_DFULL = 32,          // some table-mode OP_DPHASE ops use full phase tables and
                          // defer their per-tile phases to the store (pass_kernel only)
  PF_DSCALE = 128,        // the circuit's final scalar (coef[dsc..]) is a factor of every
                          // entry of the deferred phase table applied after the load
                          // (dpre != 0) or else at the store, instead of an OP_SCALE
};

// OP_DPHASE in table mode (Op::mode bit): every factor has at most one tile
// bit beyond the op's common condition, and a factor with a tile bit has no
// CTA-bit condition.  Then E(s) = e0(tile) + t0[s & 127] + t1[s >> 7] where
// the two 128-entry partial-sum tables are the same for every tile: they are
// built once per CTA (at word offset z_loc of the pass's dyadic-table area),
// followed by the (CTA mask, CTA value, weight) triples of the b1 factors
// decided by CTA bits alone, which each warp sums per tile with shuffles.
constexpr uint8_t DP_TABLE = 0x80;
constexpr uint32_t DTAB_MAX_WORDS = 4096;   // per pass (32 KiB of shared memory)

// A table-mode OP_DPHASE in full mode (Op::mode bit): its tile-invariant
// phase exp(2 pi i (t0 + t1) / 2^34) is one complex table over the op's free
// tile bits (index = the op's loop index, at double2 offset z_glob of the
// pass's full-table area), built once per CTA, so an affected amplitude costs
// one complex multiply.  The per-tile part e0 is a phase on the amplitudes
// meeting the op's condition; no later op of the pass mixes a condition bit,
// so it commutes to the end of the pass: the op stores e0 in deferred slot b0,
// and the store multiplies every amplitude by the phase of the sum of the
// slots whose conditions (dmask, dval over the header's dbits) it meets.
// When a later op mixes a condition bit but no earlier one does (the inverse
// QFT: the phases of qubit i precede its H), e0 commutes to the start of the
// pass instead (DP_PRE): it is summed when the tile starts and applied right
// after the load.
constexpr uint8_t DP_FULL = 0x40;
constexpr uint8_t DP_PRE = 0x20;
// A full-mode, per-tile-part-at-the-load OP_DPHASE on one condition bit c
// (set) followed by an OP_H on bit c (the inverse gate-form QFT: qubit i's
// phases, then its H): the two ops form the butterfly (a + w b, a - w b) of
// the pair (s0, s1 = s0 | 2^c), w the phase of s1 (table entry of the pair
// index).  Its table holds w as (scale, s) with w = scale (1 + i s) applied
// to b, or, when |Re w| < |Im w|, w = scale (1 + i s) applied to i b
// (|s| <= 1 either way), followed by one form byte per entry: 6 FMAs per
// pair instead of a complex multiply and four adds.  The phase depends on the
// factors' tile bits only, which form one run of tile-local positions
// [a, a + b) (Op::a, Op::b): the table has 2^b entries, index (s >> a) mod 2^b.
constexpr uint8_t DP_BFLY = 0x10;
// A full-mode OP_DPHASE with no CTA-decided factor and no CTA-bit condition:
// its phase is the same for every tile, so it has no per-tile part and takes
// no deferred slot (Op::b0 is then only its scratch slot for the table build).
constexpr uint8_t DP_NODEFER = 0x08;
constexpr int DFULL_MAX_ENTRIES = 3072;     // per pass (48 KiB of shared memory)

// OP_LPHASE in table mode (Op::mode bit): every factor's condition bit is a
// tile bit, so phase(s) is the same for every tile and one 2^k-entry table,
// built once per CTA, gives it with one complex multiply per amplitude.
constexpr uint8_t LP_TABLE = 0x80;
constexpr int LTAB_MAX_BITS = 10;   // table-mode tiles: 2^10 entries, 16 KiB

struct PassParams {
  PassHeader h;
  Op ops[MAX_OPS];
  double coef[MAX_COEF];
};
static_assert(sizeof(PassParams) <= 32764, "a pass must fit one kernel parameter");

// ----------------------------------------------------- host-side compiler

// A lowered op with global bit positions, before tile assignment.
struct LOp {
  uint8_t type = 0, mode = 0;
  int g0 = -1, g1 = -1;          // global mixing bits
  uint64_t cm = 0, cv = 0;       // condition (global bits)
  uint64_t x = 0, z = 0;         // Pauli masks (global bits)
  double a = 0, b = 0;
  int ncoef = 0;
  double coef[32];
  int gate = -1;                 // source gate index (-1: synthetic)
  int sub = 0;                   // index of this op among its gate's ops
  int slot = -1;                 // gradient slot (OP_GRAD)
  double fr = 1, fi = 0;         // deferred factor this op contributes to the
                                 // global scalar (first op of a gate)
  int64_t dy = -1;               // dyadic phase weight (angle = 2 pi dy / 2^34) of a
                                 // fixed diagonal op, -1 if not dyadic
  bool fixed = false;            // from a gate without a parameter
  // OP_DPHASE factors: (cm, cv, weight) triples, global bits
  std::vector<uint64_t> dfac;
  uint64_t mix() const;          // bits that must lie inside the tile
  uint64_t diag() const;         // bits only read (conditions, phases)
};

// Result of lowering one gate at a given angle.
struct Lowered {
  int nops = 0;
  LOp op[2];
  double zr = 1, zi = 0;         // deferred scalar factor
};

// Lower one gate (kind, global bits derived from qubits) at angle theta.
// Returns LQ_OK or an error status (message set).
lq_status lower_gate(const lq_gate& g, int n, double theta, Lowered& out);

// Pass schedule: one PassParams per tile pass, in execution order.
struct ScheduleOptions {
  int k = 10;                // tile bits
  int m = 5;                 // contiguous low bits always in the tile (raised
                             // to k - max_hi when smaller)
  int max_hi = 8;            // tile bits above the low run that the launching
                             // kernel's offset table maps (2^max_hi entries;
                             // pass_kernel: PASS_HI_BITS)
  bool force_scale = false;  // always end with a (final) OP_SCALE
  bool merge_params = true;  // merge one-bit phases of parametrised gates too
  int max_grads = 1 << 30;   // OP_GRAD ops per pass (two-state passes keep a
                             // shared-memory sum per gradient op and warp)
  bool lphase_table = false; // mark one OP_LPHASE per pass for a per-CTA table,
                             // and OP_DPHASE ops for per-CTA partial-sum tables
                             // (schedules run by pass_kernel only)
  bool sink_phases = false;  // move one-bit phases across passes to fewer merge
                             // points (parity factors through CNOTs) and fold the
                             // final scalar into a merged phase op of the last
                             // pass (schedules run by pass_kernel only), for
                             // states of at least sink_min_qubits qubits
  int sink_min_qubits = 18;  // below it the search costs more host time than
                             // the moved phases save on the device
};

// Per-state replacement of one gate's coefficients (shifted circuits of the
// parameter-shift rule).  The final OP_SCALE is multiplied by (zr, zi), the
// ratio of the shifted to the unshifted deferred factor.
struct Patch {
  int32_t gate;
  uint8_t mode0, mode1, pad0, pad1;
  double a0, b0, a1, b1;
  double zr, zi;
};

struct Schedule {
  int n = 0;
  int npasses = 0;
  PassParams* passes = nullptr;   // host array (npasses)
  int* op_src = nullptr;          // npasses * MAX_OPS: index of the source LOp (-1:
                                  // synthetic or merged)
  std::vector<std::vector<LOp>> pass_ops;   // the final ops of each pass
  Schedule() = default;
  Schedule(const Schedule&) = delete;
  Schedule& operator=(const Schedule&) = delete;
  ~Schedule();
};

// Greedily pack `ops` (in order) into tile passes of opt.k bits; an op may
// move ahead of ops it commutes with.  The deferred scalar (zr, zi) is
// appended as an OP_SCALE to the last pass (no pass is added for an empty
// circuit with a unit scalar).
lq_status schedule_ops(int n, const LOp* ops, std::size_t nops, double zr, double zi,
                       const ScheduleOptions& opt, Schedule& out);

// Merge runs of fixed dyadic diagonal ops into OP_DPHASE, and runs of
// one-bit phase ops into OP_LPHASE, where cheaper (full_tables: the ops will
// run in pass_kernel, where a dyadic op with a common control bit costs one
// complex multiply per affected amplitude).  With params = false, ops
// of parametrised gates are left alone (per-circuit patches address them).
void merge_dyadic(std::vector<LOp>& ops, int n, bool full_tables = false);
// tile (nonzero): the pass's tile bits; parity phases (OP_PARITY) with at
// most one tile bit then merge too, as parity factors.
void merge_linear(std::vector<LOp>& ops, int n, bool params, std::vector<int>* src,
                  int coef_budget, uint64_t tile = 0);

// Validate and lower a whole circuit at the given parameters.  The caller
// owns *ops_out (delete[]).  (*zr, *zi) is the product of deferred factors.
lq_status lower_circuit(int n, const lq_gate* gates, int ng, const double* params, int np,
                        LOp** ops_out, std::size_t* nops_out, double* zr, double* zi,
                        bool full_tables = false);

// FP64 flops one op executes on a 2^n state (FMA = 2), in the op forms of the
// tile kernels.
double op_flops(const LOp& o, int n);

// The autotuner's schedule options for this circuit structure on the current
// GPU (lq_tune.cu); false (opt untouched) when it has not been tuned.
bool tuned_options(int n, const lq_gate* gates, int ng, ScheduleOptions* opt);

// lq_apply_circuit and lq_circuit_plan with a default schedule for when the
// tune cache has no entry for the circuit (nullptr: the library default).
lq_status apply_circuit_with(void* amps, int n, const lq_gate* gates, int ng,
                             const double* params, int np, lq_stream stream,
                             const ScheduleOptions* fallback);
lq_status circuit_plan_with(int n, const lq_gate* gates, int ng, const double* params, int np,
                            lq_plan_info* out, const ScheduleOptions* fallback);
// Structure hash of a circuit (n; per gate kind, qubits, whether it takes a
// parameter, fixed angle / matrix) and the autotuner's batch entries.
uint64_t circuit_structure_hash(int n, const lq_gate* gates, int ng);
bool tuned_batch_tile(uint64_t structure, int* k);
void record_batch_tile(uint64_t structure, int k, double ms, double ms_default);

// Validation helpers.
lq_status check_n(int n);
lq_status check_gates(int n, const lq_gate* gates, int ng, const double* params, int np);
lq_status check_terms(int n, const lq_pauli_term* terms, int nt);
bool gate_takes_angle(int kind);
int gate_arity(int kind);

// ------------------------------------------------------------ utilities

void set_error(const char* fmt, ...);
lq_status fail(lq_status st, const char* fmt, ...);

}  // namespace lq
