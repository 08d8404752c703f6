// lq_compile.cpp -- host side of lq_apply_circuit and friends: validation,
// lowering of gates into tile ops, and greedy packing of ops into
// shared-memory tile passes.
//
// Lowering follows the gate definitions of the paper (rotations
// exp(-i theta sigma/2), Sec. III-A; CNOT and Toffoli as the bit-mask swaps of
// Alg. 1 and Alg. 4; CP as diag(1,1,1,e^{i theta}), Alg. 3) with qubit q at bit
// n-1-q of the amplitude index (MSB-first).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "lq_coefs.h"
#include "lq_internal.h"

namespace lq {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}

lq_status fail(lq_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return st;
}

const char* last_error() { return g_err; }
void clear_error() { g_err[0] = 0; }

static inline int popc64(uint64_t v) { return __builtin_popcountll(v); }

// ------------------------------------------------------------- validation

int gate_arity(int kind) {
  switch (kind) {
    case LQ_H: case LQ_X: case LQ_Y: case LQ_Z: case LQ_S: case LQ_SDG: case LQ_T:
    case LQ_TDG: case LQ_RX: case LQ_RY: case LQ_RZ: case LQ_P: case LQ_U1:
      return 1;
    case LQ_CNOT: case LQ_CY: case LQ_CZ: case LQ_CP: case LQ_SWAP: case LQ_CRX:
    case LQ_CRY: case LQ_CRZ: case LQ_RXX: case LQ_RYY: case LQ_RZZ: case LQ_U2:
      return 2;
    case LQ_CCX:
      return 3;
    default:
      return 0;
  }
}

bool gate_takes_angle(int kind) {
  switch (kind) {
    case LQ_RX: case LQ_RY: case LQ_RZ: case LQ_P: case LQ_CP: case LQ_CRX: case LQ_CRY:
    case LQ_CRZ: case LQ_RXX: case LQ_RYY: case LQ_RZZ:
      return true;
    default:
      return false;
  }
}

lq_status check_n(int n) {
  if (n < 1 || n > 34) return fail(LQ_ERR_INVALID_ARG, "n=%d outside [1, 34]", n);
  return LQ_OK;
}

lq_status check_gates(int n, const lq_gate* gates, int ng, const double* params, int np) {
  if (ng < 0 || np < 0) return fail(LQ_ERR_INVALID_ARG, "negative gate or parameter count");
  if (ng > 0 && !gates) return fail(LQ_ERR_INVALID_ARG, "gates is NULL");
  if (np > 0 && !params) return fail(LQ_ERR_INVALID_ARG, "params is NULL");
  for (int i = 0; i < np; i++)
    if (!std::isfinite(params[i]))
      return fail(LQ_ERR_NONFINITE, "params[%d] is not finite", i);
  for (int g = 0; g < ng; g++) {
    const lq_gate& G = gates[g];
    int k = gate_arity(G.kind);
    if (k == 0) return fail(LQ_ERR_INVALID_ARG, "gate %d: unknown kind %d", g, G.kind);
    for (int j = 0; j < k; j++) {
      if (G.qubits[j] < 0 || G.qubits[j] >= n)
        return fail(LQ_ERR_INVALID_ARG, "gate %d: qubit %d outside [0, %d)", g, G.qubits[j], n);
      for (int l = 0; l < j; l++)
        if (G.qubits[l] == G.qubits[j])
          return fail(LQ_ERR_INVALID_ARG, "gate %d: qubit %d repeated", g, G.qubits[j]);
    }
    if (G.param >= 0) {
      if (!gate_takes_angle(G.kind))
        return fail(LQ_ERR_INVALID_ARG, "gate %d: kind %d takes no parameter", g, G.kind);
      if (G.param >= np)
        return fail(LQ_ERR_INVALID_ARG, "gate %d: parameter index %d >= np=%d", g, G.param, np);
    } else if (G.param < -1) {
      return fail(LQ_ERR_INVALID_ARG, "gate %d: parameter index %d", g, G.param);
    }
    if (!std::isfinite(G.angle)) return fail(LQ_ERR_NONFINITE, "gate %d: angle not finite", g);
    int nm = G.kind == LQ_U1 ? 8 : G.kind == LQ_U2 ? 32 : 0;
    for (int i = 0; i < nm; i++)
      if (!std::isfinite(G.mat[i])) return fail(LQ_ERR_NONFINITE, "gate %d: matrix not finite", g);
  }
  return LQ_OK;
}

lq_status check_terms(int n, const lq_pauli_term* terms, int nt) {
  if (nt < 0) return fail(LQ_ERR_INVALID_ARG, "negative term count");
  if (nt > 0 && !terms) return fail(LQ_ERR_INVALID_ARG, "terms is NULL");
  uint64_t lim = n >= 64 ? ~0ull : ((1ull << n) - 1);
  for (int t = 0; t < nt; t++) {
    if (!std::isfinite(terms[t].coeff))
      return fail(LQ_ERR_NONFINITE, "term %d: coefficient not finite", t);
    if ((terms[t].xmask | terms[t].zmask) & ~lim)
      return fail(LQ_ERR_INVALID_ARG, "term %d: mask has bits >= n=%d", t, n);
  }
  return LQ_OK;
}

// ---------------------------------------------------------------- lowering

uint64_t LOp::mix() const {
  switch (type) {
    case OP_PAULI: case OP_GRAD: return x;
    case OP_H: case OP_PAIR_GEN: return 1ull << g0;
    case OP_QUAD_GEN: case OP_SWAP: return (1ull << g0) | (1ull << g1);
    default: return 0;
  }
}

uint64_t LOp::diag() const { return cm | z; }

static LOp pauli_op(uint64_t x, uint64_t z, int ny, uint8_t pmode) {
  LOp o;
  o.type = OP_PAULI;
  o.x = x;
  o.z = z;
  // w_i = (-i)^{rotations} i^{ny}: rotations carry the -i of c - i s P
  int k0 = (pmode == PM_PERM) ? (ny & 3) : ((3 + ny) & 3);
  o.mode = (uint8_t)(pmode | (k0 << 2));
  return o;
}

static LOp diag_op(uint8_t type, uint64_t cm, uint64_t cv, double a, double b) {
  LOp o;
  o.type = type;
  o.cm = cm;
  o.cv = cv;
  o.a = a;
  o.b = b;
  return o;
}

// Weight w with angle = 2 pi w / 2^34 (mod 2^34) if the angle is an exact
// dyadic multiple of 2 pi / 2^34, else -1.
static int64_t dyadic_weight(double angle) {
  const double PI = 3.14159265358979323846;
  double w = angle / PI * std::ldexp(1.0, DYADIC_BITS - 1);
  if (!(std::fabs(w) < std::ldexp(1.0, 60)) || w != std::floor(w)) return -1;
  int64_t iw = (int64_t)w;
  const int64_t M = (int64_t)1 << DYADIC_BITS;
  iw %= M;
  if (iw < 0) iw += M;
  return iw;
}

lq_status lower_gate(const lq_gate& g, int n, double theta, Lowered& L) {
  L = Lowered();
  int b[3] = {0, 0, 0};
  int k = gate_arity(g.kind);
  for (int j = 0; j < k; j++) b[j] = n - 1 - g.qubits[j];
  const uint64_t m0 = 1ull << b[0], m1 = k > 1 ? 1ull << b[1] : 0, m2 = k > 2 ? 1ull << b[2] : 0;
  const double R2 = 0.70710678118654752440;
  AngleCoefs ac;
  if (gate_takes_angle(g.kind)) angle_coefs(g.kind, theta, ac);
  L.zr = ac.zr;
  L.zi = ac.zi;
  LOp& o = L.op[0];
  L.nops = 1;
  switch (g.kind) {
    case LQ_H:
      o.type = OP_H; o.g0 = b[0];
      L.zr = R2; L.zi = 0;
      break;
    case LQ_X: o = pauli_op(m0, 0, 0, PM_PERM); break;
    case LQ_Y: o = pauli_op(m0, m0, 1, PM_PERM); break;
    case LQ_Z: o = diag_op(OP_SIGN, m0, m0, 0, 0); o.dy = (int64_t)1 << 33; break;
    case LQ_S: o = diag_op(OP_MULI, m0, m0, 0, 0); o.mode = 1; o.dy = (int64_t)1 << 32; break;
    case LQ_SDG: o = diag_op(OP_MULI, m0, m0, 0, 0); o.mode = 3; o.dy = (int64_t)3 << 32; break;
    case LQ_T: o = diag_op(OP_PHASE, m0, m0, R2, R2); o.dy = (int64_t)1 << 31; break;
    case LQ_TDG: o = diag_op(OP_PHASE, m0, m0, R2, -R2); o.dy = (int64_t)7 << 31; break;
    case LQ_RX: o = pauli_op(m0, 0, 0, ac.mode0); o.a = ac.a0; o.b = ac.b0; break;
    case LQ_RY: o = pauli_op(m0, m0, 1, ac.mode0); o.a = ac.a0; o.b = ac.b0; break;
    case LQ_RZ: case LQ_P:
      o = diag_op(OP_PHASE, m0, m0, ac.a0, ac.b0);
      o.dy = dyadic_weight(theta);
      break;
    case LQ_U1:
      o.type = OP_PAIR_GEN; o.g0 = b[0]; o.ncoef = 8;
      for (int i = 0; i < 8; i++) o.coef[i] = g.mat[i];
      break;
    case LQ_CNOT: o = pauli_op(m1, 0, 0, PM_PERM); o.cm = m0; o.cv = m0; break;
    case LQ_CY: o = pauli_op(m1, m1, 1, PM_PERM); o.cm = m0; o.cv = m0; break;
    case LQ_CZ: o = diag_op(OP_SIGN, m0 | m1, m0 | m1, 0, 0); o.dy = (int64_t)1 << 33; break;
    case LQ_CP:
      o = diag_op(OP_PHASE, m0 | m1, m0 | m1, ac.a0, ac.b0);
      o.dy = dyadic_weight(theta);
      break;
    case LQ_SWAP: o.type = OP_SWAP; o.g0 = b[0]; o.g1 = b[1]; break;
    case LQ_CRX:
      o = pauli_op(m1, 0, 0, PM_GEN); o.a = ac.a0; o.b = ac.b0; o.cm = m0; o.cv = m0;
      break;
    case LQ_CRY:
      o = pauli_op(m1, m1, 1, PM_GEN); o.a = ac.a0; o.b = ac.b0; o.cm = m0; o.cv = m0;
      break;
    case LQ_CRZ:
      o = diag_op(OP_PHASE, m0 | m1, m0, ac.a0, ac.b0);
      L.op[1] = diag_op(OP_PHASE, m0 | m1, m0 | m1, ac.a1, ac.b1);
      L.op[1].sub = 1;
      L.nops = 2;
      break;
    case LQ_RXX: o = pauli_op(m0 | m1, 0, 0, ac.mode0); o.a = ac.a0; o.b = ac.b0; break;
    case LQ_RYY:
      o = pauli_op(m0 | m1, m0 | m1, 2, ac.mode0); o.a = ac.a0; o.b = ac.b0;
      break;
    case LQ_RZZ:
      o = diag_op(OP_PARITY, 0, 0, ac.a0, ac.b0); o.z = m0 | m1;
      break;
    case LQ_CCX: o = pauli_op(m2, 0, 0, PM_PERM); o.cm = m0 | m1; o.cv = m0 | m1; break;
    case LQ_U2:
      o.type = OP_QUAD_GEN; o.g0 = b[0]; o.g1 = b[1]; o.ncoef = 32;
      for (int i = 0; i < 32; i++) o.coef[i] = g.mat[i];
      break;
    default:
      return fail(LQ_ERR_INVALID_ARG, "unknown gate kind %d", g.kind);
  }
  return LQ_OK;
}

static uint64_t dbits_u(double v) {
  uint64_t u;
  std::memcpy(&u, &v, sizeof u);
  return u;
}

// Merge runs of consecutive fixed dyadic diagonal ops (phases that are exact
// multiples of 2 pi / 2^34: CP(pi/2^k), T, S, Z, CZ, ...) into one OP_DPHASE
// when that needs fewer FP64 operations: the merged op costs at most two
// complex multiplies on the amplitudes meeting the factors' common
// condition, a separate phase op one complex multiply on its own fraction.
static bool dyadic_diag(const LOp& o) {
  return o.fixed && o.dy >= 0 && (o.type == OP_PHASE || o.type == OP_SIGN || o.type == OP_MULI);
}

void merge_dyadic(std::vector<LOp>& ops, int n, bool full_tables) {
  std::vector<LOp> out;
  out.reserve(ops.size());
  std::size_t i = 0;
  while (i < ops.size()) {
    if (!dyadic_diag(ops[i])) {
      out.push_back(ops[i++]);
      continue;
    }
    std::size_t j = i;
    while (j < ops.size() && dyadic_diag(ops[j])) j++;
    // common condition: bits every factor requires with the same value
    uint64_t cm = ~0ull, cv = 0, all = 0;
    double separate = 0;
    for (std::size_t k = i; k < j; k++) {
      cm &= ops[k].cm;
      all |= ops[k].cm;
      separate += op_flops(ops[k], n);
    }
    for (std::size_t k = i; k < j; k++) cm &= ~(ops[k].cv ^ ops[i].cv);
    cv = ops[i].cv & cm;
    LOp m;
    m.type = OP_DPHASE;
    m.cm = cm;
    m.cv = cv;
    m.z = all & ~cm;
    m.fixed = true;
    for (std::size_t k = i; k < j; k++) {
      m.dfac.push_back(ops[k].cm);
      m.dfac.push_back(ops[k].cv);
      m.dfac.push_back((uint64_t)ops[k].dy);
    }
    m.ncoef = 4 * (int)(j - i);
    // cost of the merged op: with per-CTA full tables (pass_kernel, a common
    // control bit) one complex multiply per affected amplitude, else two
    double merged = op_flops(m, n);
    if (full_tables && cm) merged *= 0.5;
    // followed by the H on its one common condition bit, a merged op runs as
    // a butterfly with that H on large states (6 FMAs per pair for both, vs
    // 4 adds for the H and a complex multiply per factor on a quarter of the
    // pairs): take it from two factors on
    const bool before_h = full_tables && n >= 24 && j < ops.size() && ops[j].type == OP_H &&
                          ops[j].cm == 0 && cm != 0 && (cm & (cm - 1)) == 0 && cv == cm &&
                          ops[j].g0 == __builtin_ctzll(cm);
    if (j - i >= 2 && m.ncoef <= MAX_COEF / 2 && (merged < separate || before_h)) {
      out.push_back(m);
    } else {
      for (std::size_t k = i; k < j; k++) out.push_back(ops[k]);
    }
    i = j;
  }
  ops.swap(out);
}

// A phase op conditioned on exactly one bit (RZ, P, T, Z, S, ...).
static bool one_bit_phase(const LOp& o, bool params) {
  if (!(o.type == OP_PHASE || o.type == OP_SIGN || o.type == OP_MULI)) return false;
  if (!params && !o.fixed) return false;
  return o.cm != 0 && (o.cm & (o.cm - 1)) == 0;
}

static void phase_value(const LOp& o, double* a, double* b) {
  if (o.type == OP_PHASE || o.type == OP_PARITY) {
    *a = o.a;
    *b = o.b;
  } else if (o.type == OP_SIGN) {
    *a = -1;
    *b = 0;
  } else {  // i^mode
    const double re[4] = {1, 0, -1, 0}, im[4] = {0, 1, 0, -1};
    *a = re[o.mode & 3];
    *b = im[o.mode & 3];
  }
}

// A parity phase (w on the amplitudes with odd popcount(idx & z)) with at
// most one of its bits in the pass's tile: a factor of a merged one-bit phase
// op, its other bits giving a per-tile constant.
static bool tile_parity_phase(const LOp& o, bool params, uint64_t tile) {
  if (!tile || o.type != OP_PARITY || o.cm != 0 || o.z == 0) return false;
  if (!params && !o.fixed) return false;
  return popc64(o.z & tile) <= 1;
}

void merge_linear(std::vector<LOp>& ops, int n, bool params, std::vector<int>* src,
                  int coef_budget, uint64_t tile) {
  std::vector<LOp> out;
  std::vector<int> osrc;
  out.reserve(ops.size());
  auto mergeable = [&](const LOp& o) {
    return one_bit_phase(o, params) || tile_parity_phase(o, params, tile);
  };
  std::size_t i = 0;
  while (i < ops.size()) {
    if (!mergeable(ops[i])) {
      if (src) osrc.push_back((*src)[i]);
      out.push_back(ops[i++]);
      continue;
    }
    std::size_t j = i;
    while (j < ops.size() && mergeable(ops[j])) j++;
    double separate = 0;
    uint64_t all = 0;
    for (std::size_t k = i; k < j; k++) {
      separate += op_flops(ops[k], n);
      all |= ops[k].cm | (ops[k].type == OP_PARITY ? ops[k].z : 0);
    }
    LOp m;
    m.type = OP_LPHASE;
    m.z = all;
    m.fixed = true;
    for (std::size_t k = i; k < j; k++) {
      const double fr = m.fr * ops[k].fr - m.fi * ops[k].fi;
      m.fi = m.fr * ops[k].fi + m.fi * ops[k].fr;
      m.fr = fr;
    }
    for (std::size_t k = i; k < j; k++) {
      double a, b;
      phase_value(ops[k], &a, &b);
      if (ops[k].type == OP_PARITY) {   // condition: odd parity of idx & z
        m.dfac.push_back(ops[k].z);
        m.dfac.push_back(ops[k].z | kLphaseParity);
      } else {
        m.dfac.push_back(ops[k].cm);
        m.dfac.push_back(ops[k].cv);
      }
      m.dfac.push_back(dbits_u(a));
      m.dfac.push_back(dbits_u(b));
      m.dfac.push_back((uint64_t)(int64_t)ops[k].gate);   // for per-circuit patches
    }
    m.ncoef = LPHASE_FAC * (int)(j - i);
    // merged: about 12 flops per amplitude plus per-tile tables
    if (j - i >= 3 && m.ncoef <= coef_budget && 13.0 * std::ldexp(1.0, n) < separate) {
      coef_budget -= m.ncoef;
      out.push_back(m);
      if (src) osrc.push_back(-1);
    } else {
      for (std::size_t k = i; k < j; k++) {
        out.push_back(ops[k]);
        if (src) osrc.push_back((*src)[k]);
      }
    }
    i = j;
  }
  ops.swap(out);
  if (src) src->swap(osrc);
}

// Magnitude window of the deferred scalar; outside it the magnitude is applied
// by an explicit OP_SCALE so stored amplitudes stay far from overflow.
static const double kScaleLo = 1e-100, kScaleHi = 1e100;

lq_status lower_circuit(int n, const lq_gate* gates, int ng, const double* params, int np,
                        LOp** ops_out, std::size_t* nops_out, double* zr_out, double* zi_out,
                        bool full_tables) {
  lq_status st = check_gates(n, gates, ng, params, np);
  if (st) return st;
  std::vector<LOp> ops;
  ops.reserve((std::size_t)ng + 8);
  double zr = 1, zi = 0;
  for (int g = 0; g < ng; g++) {
    double th = gates[g].angle + (gates[g].param >= 0 ? params[gates[g].param] : 0.0);
    Lowered L;
    st = lower_gate(gates[g], n, th, L);
    if (st) return st;
    for (int j = 0; j < L.nops; j++) {
      L.op[j].gate = g;
      L.op[j].fixed = gates[g].param < 0;
      ops.push_back(L.op[j]);
    }
    double nr = zr * L.zr - zi * L.zi, ni = zr * L.zi + zi * L.zr;
    zr = nr;
    zi = ni;
    double mag = std::hypot(zr, zi);
    if (mag < kScaleLo || mag > kScaleHi) {
      LOp s;
      s.type = OP_SCALE;
      s.mode = 1;
      s.a = mag;
      ops.push_back(s);
      zr /= mag;
      zi /= mag;
    }
  }
  merge_dyadic(ops, n, full_tables);
  LOp* out = new LOp[ops.size() > 0 ? ops.size() : 1];
  for (std::size_t i = 0; i < ops.size(); i++) out[i] = ops[i];
  *ops_out = out;
  *nops_out = ops.size();
  *zr_out = zr;
  *zi_out = zi;
  return LQ_OK;
}

// ------------------------------------------------------------ cost model

double op_flops(const LOp& o, int n) {
  const double N = std::ldexp(1.0, n);
  const double frac = std::ldexp(1.0, -popc64(o.cm));  // amplitudes meeting the condition
  switch (o.type) {
    case OP_PAULI:
      switch (o.mode & 3) {
        case PM_TAN: case PM_COT: return 4.0 * N * frac;   // 2 FMA per amplitude
        case PM_GEN: return 6.0 * N * frac;                // MUL + FMA per component
        default: return 0.0;                               // permutation
      }
    case OP_H: return 2.0 * N * frac;                      // 2 adds per amplitude
    case OP_PAIR_GEN: return 14.0 * N * frac;              // 1 MUL + 3 FMA per component
    case OP_QUAD_GEN: return 32.0 * N * frac;              // 8 FMA per component
    case OP_PHASE: return 6.0 * N * frac;                  // complex multiply
    case OP_PARITY: return 6.0 * N * 0.5 * frac;
    case OP_SCALE: return ((o.mode & 1) ? 2.0 : 6.0) * N;
    case OP_GRAD: return 4.0 * N;
    case OP_DPHASE:   // (table combine +) multiply; a butterfly: 6 FMA per pair with its H
      return ((o.mode & DP_BFLY) ? 8.0 : (o.mode & DP_FULL) ? 6.0 : 12.0) * N * frac;
    case OP_LPHASE:                                        // (table combine +) multiply
      return ((o.mode & LP_TABLE) ? 6.0 : 12.0) * N * frac;
    default: return 0.0;                                   // sign flips, i^k, swaps
  }
}

// -------------------------------------------------------------- scheduling

Schedule::~Schedule() {
  delete[] passes;
  delete[] op_src;
}

static uint32_t to_local(uint64_t mask, const int* pos) {
  uint32_t r = 0;
  while (mask) {
    int b = __builtin_ctzll(mask);
    mask &= mask - 1;
    r |= 1u << pos[b];
  }
  return r;
}

static uint64_t dbits(double v) {
  uint64_t u;
  std::memcpy(&u, &v, sizeof u);
  return u;
}
static double bitsd(uint64_t u) {
  double v;
  std::memcpy(&v, &u, sizeof v);
  return v;
}

// Factor list of an OP_DPHASE in the pass coefficient pool: per factor
// (tile-local cm | cv << 32, CTA-bit cm, CTA-bit cv, weight), as raw bits.
static void fill_dphase(double* pool, const LOp& s, uint64_t tile, const int* pos) {
  const std::size_t nf = s.dfac.size() / 3;
  for (std::size_t f = 0; f < nf; f++) {
    uint64_t cm = s.dfac[3 * f], cv = s.dfac[3 * f + 1], w = s.dfac[3 * f + 2];
    uint64_t loc = (uint64_t)to_local(cm & tile, pos) | ((uint64_t)to_local(cv & tile, pos) << 32);
    pool[4 * f + 0] = bitsd(loc);
    pool[4 * f + 1] = bitsd(cm & ~tile);
    pool[4 * f + 2] = bitsd(cv & ~tile);
    pool[4 * f + 3] = bitsd(w);
  }
}

// Factor list of an OP_LPHASE: per factor (tile-local cm | cv << 32, CTA cm,
// CTA cv, re, im, source gate index).
static void fill_lphase(double* pool, const LOp& s, uint64_t tile, const int* pos) {
  const std::size_t nf = s.dfac.size() / 5;
  for (std::size_t f = 0; f < nf; f++) {
    uint64_t cm = s.dfac[5 * f], cv = s.dfac[5 * f + 1];
    uint64_t loc = (uint64_t)to_local(cm & tile, pos) | ((uint64_t)to_local(cv & tile, pos) << 32);
    double* q = pool + LPHASE_FAC * f;
    q[0] = bitsd(loc);
    q[1] = bitsd(cm & ~tile);
    q[2] = bitsd(cv & ~tile);
    q[3] = bitsd(s.dfac[5 * f + 2]);
    q[4] = bitsd(s.dfac[5 * f + 3]);
    q[5] = bitsd(s.dfac[5 * f + 4]);
  }
}

// Tile-local bits an op mixes (pairs or quads of amplitudes differing in them).
static uint32_t op_mixing_bits(const Op& d) {
  switch (d.type) {
    case OP_PAULI: case OP_GRAD: return d.x_loc;
    case OP_H: case OP_PAIR_GEN: return 1u << d.b0;
    case OP_QUAD_GEN: case OP_SWAP: return (1u << d.b0) | (1u << d.b1);
    default: return 0;   // diagonal ops
  }
}

static void fill_op(Op& d, const LOp& s, uint64_t tile, const int* pos, int coef_at) {
  std::memset(&d, 0, sizeof d);
  d.type = s.type;
  d.mode = s.mode;
  d.b0 = s.g0 >= 0 ? (uint8_t)pos[s.g0] : 0;
  d.b1 = s.g1 >= 0 ? (uint8_t)pos[s.g1] : (uint8_t)s.sub;
  if (s.type == OP_GRAD)
    d.cidx = (uint32_t)s.slot;
  else if (s.type == OP_PAIR_GEN || s.type == OP_QUAD_GEN || s.type == OP_DPHASE ||
           s.type == OP_LPHASE)
    d.cidx = (uint32_t)coef_at;
  else
    d.cidx = (uint32_t)s.gate;
  d.cm_loc = to_local(s.cm & tile, pos);
  d.cv_loc = to_local(s.cv & tile, pos);
  d.cm_glob = s.cm & ~tile;
  d.cv_glob = s.cv & ~tile;
  d.x_loc = s.type == OP_DPHASE   ? (uint32_t)(s.dfac.size() / 3)
            : s.type == OP_LPHASE ? (uint32_t)(s.dfac.size() / 5)
                                  : to_local(s.x, pos);
  d.z_loc = to_local(s.z & tile, pos);
  d.z_glob = s.z & ~tile;
  d.a = s.a;
  d.b = s.b;
}

// ------------------------------------------------------------ phase sinking
//
// A one-bit phase (RZ, P, T on one qubit: the amplitudes with bit b set
// times w) is diagonal, so it commutes with every op that does not mix bit b.
// Moved past a CNOT-type permutation (X on target t under one control c,
// y -> y ^ (y_c ? 2^t : 0)) it becomes a parity phase, w on the amplitudes
// with odd popcount(y & M), where M gains or loses c when t is in M; a swap
// exchanges the two bits of M.  So a hardware-efficient layer's RZ factors
// need not be applied in every pass that holds some of them: moved forward
// to the last pass they are parities of CTA bits there (per-tile constants)
// or one-bit phases on its tile bits, and one merged phase op serves them
// all.

// A phase op that sinking may move: OP_PHASE on the amplitudes with one bit set.
static bool sinkable_phase(const LOp& o) {
  return o.type == OP_PHASE && o.cm != 0 && (o.cm & (o.cm - 1)) == 0 && o.cv == o.cm;
}

// Moves a parity phase with mask M from before op o to after it: false when
// o mixes a bit of M other than as a CNOT-type target or a swap.
static bool sink_past(const LOp& o, uint64_t& M) {
  const uint64_t mx = o.mix();
  if ((mx & M) == 0) return true;   // diagonal, or acts on other bits
  if (o.type == OP_PAULI && (o.mode & 3) == PM_PERM && (mx & (mx - 1)) == 0 && o.cm != 0 &&
      (o.cm & (o.cm - 1)) == 0 && o.cv == o.cm && (o.cm & mx) == 0) {
    M ^= o.cm;   // CNOT, CY: parity(y' & M) = parity(y & (M ^ c)) for t in M
    return true;
  }
  if (o.type == OP_SWAP) {
    const uint64_t a = 1ull << o.g0, b = 1ull << o.g1;
    if (((M & a) != 0) != ((M & b) != 0)) M ^= a | b;
    return true;
  }
  return false;
}

// plists: the passes' ops in execution order (tiles: their tile bits).  Each
// one-bit phase moves forward until an op mixes one of its bits; a point on
// the way is usable when at most one bit of its mask there is a tile bit of
// that point's pass.  Points are fixed greedily: the phase whose last usable
// point comes first fixes a point there, and every phase usable at it joins
// it.  The phases are re-inserted at their points (one-bit masks as OP_PHASE,
// wider ones as OP_PARITY) when that leaves fewer points than passes with
// phases; otherwise nothing changes.  A point is (pass, position in the
// pass's list): before the op at that position, or at the end of the pass;
// the phases themselves are diagonal and commute, so a moving phase skips
// the others.
static void sink_phases(const std::vector<uint64_t>& tiles, std::vector<std::vector<LOp>>& plists,
                        std::vector<std::vector<int>>& psrcs) {
  const int P = (int)plists.size();
  if (P < 2) return;
  struct Fac {
    int p, q;        // the phase op: plists[p][q]
    int first, cnt;  // its usable points in `pts`
  };
  struct Pt {
    int key;         // off[p] + position
    uint64_t M;
  };
  std::vector<int> off(P + 1, 0);
  std::vector<Fac> facs;
  int before = 0;
  for (int p = 0; p < P; p++) {
    off[p + 1] = off[p] + (int)plists[p].size() + 1;
    bool any = false;
    for (int q = 0; q < (int)plists[p].size(); q++)
      if (sinkable_phase(plists[p][q])) {
        facs.push_back(Fac{p, q, 0, 0});
        any = true;
      }
    before += any;
  }
  if (before < 2) return;
  std::vector<Pt> pts;
  pts.reserve(facs.size() * 16);
  for (Fac& f : facs) {
    uint64_t M = plists[f.p][f.q].cm;
    int p = f.p, q = f.q + 1;
    f.first = (int)pts.size();
    for (;;) {
      if (popc64(M & tiles[p]) <= 1) pts.push_back(Pt{off[p] + q, M});
      if (q == (int)plists[p].size()) {
        if (p + 1 == P) break;
        p++;
        q = 0;
        continue;
      }
      const LOp& o = plists[p][q];
      if (!sinkable_phase(o) && !sink_past(o, M)) break;
      q++;
    }
    f.cnt = (int)pts.size() - f.first;
  }
  // greedy points
  std::vector<int> at(facs.size(), -1);
  std::vector<uint64_t> mask(facs.size(), 0);
  std::size_t left = facs.size();
  int npoints = 0;
  while (left && npoints < before) {
    int x = 1 << 30;
    for (std::size_t f = 0; f < facs.size(); f++)
      if (at[f] < 0) x = std::min(x, pts[(std::size_t)(facs[f].first + facs[f].cnt - 1)].key);
    npoints++;
    for (std::size_t f = 0; f < facs.size(); f++) {
      if (at[f] >= 0) continue;
      const Pt* b = pts.data() + facs[f].first;
      const Pt* e = b + facs[f].cnt;
      const Pt* it = std::lower_bound(b, e, x, [](const Pt& a, int v) { return a.key < v; });
      if (it != e && it->key == x) {
        at[f] = x;
        mask[f] = it->M;
        left--;
      }
    }
  }
  if (left || npoints >= before) return;
  // rebuild the passes that lose or gain phases
  std::vector<int> order(facs.size());
  for (std::size_t f = 0; f < facs.size(); f++) order[f] = (int)f;
  std::sort(order.begin(), order.end(), [&](int a, int b) {
    return at[a] != at[b] ? at[a] < at[b] : a < b;
  });
  // the phase ops themselves (their passes' lists are rebuilt below)
  std::vector<LOp> fop;
  std::vector<int> fsrc;
  fop.reserve(facs.size());
  for (const Fac& f : facs) {
    fop.push_back(plists[f.p][f.q]);
    fsrc.push_back(psrcs[f.p][f.q]);
  }
  std::vector<char> touched(P, 0);
  for (const Fac& f : facs) touched[f.p] = 1;
  for (std::size_t f = 0; f < facs.size(); f++) {
    const int p = (int)(std::upper_bound(off.begin(), off.end(), at[f]) - off.begin()) - 1;
    touched[p] = 1;
  }
  std::size_t next = 0;   // into order, by point
  for (int p = 0; p < P; p++) {
    if (!touched[p]) continue;
    std::vector<LOp> out;
    std::vector<int> osrc;
    out.reserve(plists[p].size() + 8);
    osrc.reserve(plists[p].size() + 8);
    while (next < order.size() && at[order[next]] < off[p]) next++;
    for (int q = 0; q <= (int)plists[p].size(); q++) {
      for (; next < order.size() && at[order[next]] == off[p] + q; next++) {
        LOp o = fop[(std::size_t)order[next]];
        const uint64_t M = mask[order[next]];
        if ((M & (M - 1)) == 0) {
          osrc.push_back(M == o.cm ? fsrc[(std::size_t)order[next]] : -1);
          o.cm = o.cv = M;
        } else {
          o.type = OP_PARITY;
          o.cm = o.cv = 0;
          o.z = M;
          o.dy = -1;
          osrc.push_back(-1);
        }
        out.push_back(std::move(o));
      }
      if (q < (int)plists[p].size() && !sinkable_phase(plists[p][q])) {
        out.push_back(plists[p][q]);
        osrc.push_back(psrcs[p][q]);
      }
    }
    plists[p].swap(out);
    psrcs[p].swap(osrc);
  }
}

lq_status schedule_ops(int n, const LOp* ops, std::size_t nops, double zr, double zi,
                       const ScheduleOptions& opt, Schedule& out) {
  const int k = opt.k < n ? opt.k : n;
  int m = opt.m < k ? opt.m : k;
  if (k > MAX_TILE_BITS || k < 1) return fail(LQ_ERR_INVALID_ARG, "tile bits %d", k);
  // the kernels map the tile bits above the low run through a table of
  // 2^max_hi offsets: a smaller low run is widened to fit it
  if (opt.max_hi < 0) return fail(LQ_ERR_INVALID_ARG, "internal: max_hi %d", opt.max_hi);
  if (k - m > opt.max_hi) m = k - opt.max_hi;
  // pass_kernel keeps those offsets shifted right by the low run in 32 bits
  if (m < n - 32) m = n - 32;
  const uint64_t low = (m >= 64) ? ~0ull : ((1ull << m) - 1);
  const bool need_scale = opt.force_scale || !(zr == 1.0 && zi == 0.0);

  struct Built {
    uint64_t tile;
    std::vector<int> idx;
  };
  std::vector<Built> passes;
  std::vector<int> pending(nops);
  for (std::size_t i = 0; i < nops; i++) pending[i] = (int)i;

  while (!pending.empty()) {
    Built B;
    B.tile = low;
    int coefs = 0, grads = 0;
    std::vector<int> skipped;
    uint64_t blocked_mix = 0, blocked_all = 0;
    // a merged dyadic phase on one condition bit c that can no longer join
    // this pass's tile, whose next op on c is the H on c: in the pass that
    // holds c the two run
    // as one butterfly (or at least as a full-table phase op), here it would
    // run on every amplitude of half the tiles; it waits for that pass
    auto waits_for_h = [&](std::size_t pi) {
      const LOp& o = ops[pending[pi]];
      if (!opt.lphase_table || B.idx.empty() || o.type != OP_DPHASE || o.cm == 0 ||
          (o.cm & (o.cm - 1)) != 0 || o.cv != o.cm || popc64(B.tile | o.cm) <= k)
        return false;
      for (std::size_t pj = pi + 1; pj < pending.size(); pj++) {
        const LOp& h = ops[pending[pj]];
        if (!(h.mix() & o.cm)) continue;
        return h.type == OP_H && h.cm == 0 && (1ull << h.g0) == o.cm;
      }
      return false;
    };
    for (std::size_t pi = 0; pi < pending.size(); pi++) {
      const int idx = pending[pi];
      const LOp& o = ops[idx];
      uint64_t mx = o.mix(), dg = o.diag();
      bool commutes = !(mx & blocked_all) && !(dg & blocked_mix);
      bool room = (int)B.idx.size() < MAX_OPS - 1 && coefs + o.ncoef <= MAX_COEF &&
                  (o.type != OP_GRAD || grads < opt.max_grads);
      if (commutes && room && !waits_for_h(pi)) {
        uint64_t t = B.tile | mx;
        if (popc64(t) <= k) {
          B.tile = t;
          B.idx.push_back(idx);
          coefs += o.ncoef;
          grads += o.type == OP_GRAD;
          continue;
        }
      }
      skipped.push_back(idx);
      blocked_mix |= mx;
      blocked_all |= mx | dg;
    }
    if (B.idx.empty()) return fail(LQ_ERR_INVALID_ARG, "internal: op cannot be scheduled");
    passes.push_back(std::move(B));
    pending.swap(skipped);
  }
  if (passes.empty() && need_scale) passes.push_back(Built{low, {}});

  out.n = n;
  out.npasses = (int)passes.size();
  delete[] out.passes;
  delete[] out.op_src;
  out.passes = new PassParams[passes.size() > 0 ? passes.size() : 1];
  out.pass_ops.clear();
  out.op_src = new int[(passes.size() > 0 ? passes.size() : 1) * MAX_OPS];
  // the passes' ops in order, tiles filled up to k bits with the lowest
  // unused bits (larger contiguous loads, fewer tiles)
  std::vector<uint64_t> tiles(passes.size());
  std::vector<std::vector<LOp>> plists(passes.size());
  std::vector<std::vector<int>> psrcs(passes.size());
  for (std::size_t p = 0; p < passes.size(); p++) {
    Built& B = passes[p];
    for (int bit = 0; bit < n && popc64(B.tile) < k; bit++) B.tile |= 1ull << bit;
    tiles[p] = B.tile;
    for (int idx : B.idx) {
      plists[p].push_back(ops[idx]);
      psrcs[p].push_back(idx);
    }
  }
  // the moved phases save FP64 work in proportion to the state, the search
  // costs host time in proportion to the circuit: from 2^18 amplitudes on
  // the first outweighs the second (at n = 16 they were about equal)
  const bool sink = opt.sink_phases && n >= opt.sink_min_qubits;
  if (sink) sink_phases(tiles, plists, psrcs);
  for (std::size_t p = 0; p < passes.size(); p++) {
    Built& B = passes[p];
    // runs of one-bit (and, in the pass's tile, parity) phases merge within
    // the pass
    std::vector<LOp>& plist = plists[p];
    std::vector<int>& psrc = psrcs[p];
    {
      int used = 0;
      for (const LOp& l : plist) used += l.ncoef;
      merge_linear(plist, n, opt.merge_params, &psrc, MAX_COEF - used, sink ? B.tile : 0);
    }
    // the circuit's final scalar as an unconditional factor of a merged
    // phase op of the last pass instead of a separate scale op
    bool folded = false;
    if (sink && !opt.force_scale && p + 1 == passes.size() && need_scale) {
      int used = 0;
      for (const LOp& l : plist) used += l.ncoef;
      for (LOp& l : plist) {
        if (l.type != OP_LPHASE || used + LPHASE_FAC > MAX_COEF) continue;
        l.dfac.push_back(0);
        l.dfac.push_back(0);
        l.dfac.push_back(dbits_u(zr));
        l.dfac.push_back(dbits_u(zi));
        l.dfac.push_back((uint64_t)(int64_t)-1);
        l.ncoef += LPHASE_FAC;
        folded = true;
        break;
      }
    }
    PassParams& P = out.passes[p];
    std::memset(&P.h, 0, sizeof P.h);
    P.h.n = n;
    P.h.k = k;
    P.h.m = m;
    int pos[64];
    for (int i = 0; i < 64; i++) pos[i] = -1;
    int j = 0, o = 0;
    for (int bit = 0; bit < n; bit++) {
      if (B.tile >> bit & 1) {
        P.h.tbits[j] = (int8_t)bit;
        pos[bit] = j++;
      } else {
        P.h.obits[o++] = (int8_t)bit;
      }
    }
    // contiguous low run: tile bits 0..m'-1 where every lower bit is in
    int mm = 0;
    while (mm < k && P.h.tbits[mm] == mm) mm++;
    P.h.m = mm;
    P.h.nobits = o;
    P.h.ntiles = 1ull << (n - k);
    int coef_at = 0, cnt = 0;
    for (std::size_t q = 0; q < plist.size(); q++) {
      const LOp& l = plist[q];
      fill_op(P.ops[cnt], l, B.tile, pos, coef_at);
      if (l.type == OP_DPHASE) {
        fill_dphase(P.coef + coef_at, l, B.tile, pos);
        P.h.flags |= PF_DYADIC;
      } else if (l.type == OP_LPHASE) {
        fill_lphase(P.coef + coef_at, l, B.tile, pos);
        if (opt.lphase_table && k <= LTAB_MAX_BITS && !(P.h.flags & PF_LTAB)) {
          bool local = true;   // every factor's condition on a tile bit (or none)
          for (std::size_t f = 0; f < l.dfac.size() / 5; f++)
            if (l.dfac[5 * f] & ~B.tile) local = false;
          if (local) {
            P.ops[cnt].mode |= LP_TABLE;
            P.h.flags |= PF_LTAB;
            P.h.ltab_op = cnt;
            plist[q].mode |= LP_TABLE;
          }
        }
      } else {
        for (int c = 0; c < l.ncoef; c++) P.coef[coef_at + c] = l.coef[c];
      }
      coef_at += l.ncoef;
      out.op_src[p * MAX_OPS + cnt] = psrc[q];
      cnt++;
    }
    if (opt.lphase_table) {
      // table-mode dyadic ops: per-CTA partial-sum tables (256 words) and the
      // CTA-decided factors (3 words each) in the pass's dyadic-table area
      uint32_t words = 0;
      for (int o = 0; o < cnt; o++) {
        Op& d = P.ops[o];
        if (d.type != OP_DPHASE) continue;
        const double* F = P.coef + d.cidx;
        bool ok = true;
        int ncta = 0;
        for (uint32_t f = 0; f < d.x_loc; f++) {
          const uint64_t loc = dbits(F[4 * f]), gm = dbits(F[4 * f + 1]);
          const uint32_t lm = (uint32_t)loc & ~d.cm_loc;
          if (lm & (lm - 1)) ok = false;
          if (lm && gm) ok = false;
          if (!lm && gm) ncta++;
        }
        if (!ok || ncta > 255 || words + 256 + 3 * (uint32_t)ncta > DTAB_MAX_WORDS) continue;
        d.mode |= DP_TABLE;
        d.z_loc = words;
        d.b1 = (uint8_t)ncta;
        words += 256 + 3 * (uint32_t)ncta;
      }
      if (words) {
        P.h.flags |= PF_DTAB;
        P.h.dtab_words = (int32_t)words;
      }
      // full tables with the per-tile phases deferred to the store or the load;
      // a full-mode op's partial sums are built in the (still unused) tile
      // buffer, so only its CTA-decided factor triples stay resident
      int entries = 0, nd = 0, nfull = 0;
      uint32_t ubits = 0;
      const int scratch_slots = (2 << k) / 256;   // 256-word tables the tile buffer holds
      for (int o = 0; o < cnt && (P.h.flags & PF_DTAB); o++) {
        Op& d = P.ops[o];
        if (d.type != OP_DPHASE || !(d.mode & DP_TABLE) || nfull >= scratch_slots) continue;
        const int c = __builtin_popcount(d.cm_loc);
        if (c < 1) continue;
        // no CTA-decided factor and no CTA-bit condition: the phase is the
        // same for every tile, there is no per-tile part to defer, and the op
        // needs no deferred slot
        const bool local = d.b1 == 0 && d.cm_glob == 0;
        if (!local && nd == 8) continue;
        const int sz = 1 << (k - c);
        // the per-tile part commutes to the store if no later op of the pass
        // mixes a condition bit, else to the load if no earlier op does
        bool later = false, earlier = false;
        for (int o2 = o + 1; o2 < cnt; o2++) later |= (op_mixing_bits(P.ops[o2]) & d.cm_loc) != 0;
        for (int o2 = 0; o2 < o; o2++) earlier |= (op_mixing_bits(P.ops[o2]) & d.cm_loc) != 0;
        if (later && earlier && !local) continue;
        // butterfly with the H on its condition bit right after it (DP_BFLY):
        // the table is followed by one form byte per entry; its per-CTA build
        // (a division per entry) pays off from 2^12 tiles on (measured:
        // slower at n = 18-20 with 2^10-amplitude tiles, faster from n = 22)
        bool bfly = later && n - k >= 12 && c == 1 && d.cv_loc == d.cm_loc && d.cm_glob == 0 &&
                    o + 1 < cnt && P.ops[o + 1].type == OP_H &&
                    (1u << P.ops[o + 1].b0) == d.cm_loc && P.ops[o + 1].cm_loc == 0 &&
                    P.ops[o + 1].cm_glob == 0;
        // a butterfly's phase depends on its factors' tile bits only: when
        // they form one run [lo, lo + width) of tile-local positions (both
        // QFT directions), its table is indexed by that run alone
        int bsz = sz, lo = 0, width = k - c;
        if (bfly) {
          uint32_t fl = 0;
          const double* Fc = P.coef + d.cidx;
          for (uint32_t f = 0; f < d.x_loc; f++) fl |= (uint32_t)dbits(Fc[4 * f]) & ~d.cm_loc;
          if (fl == 0) {
            width = 0;
          } else {
            lo = __builtin_ctz(fl);
            width = 32 - __builtin_clz(fl) - lo;
            if (fl != (((1u << width) - 1u) << lo)) bfly = false;   // not one run
          }
          if (bfly) bsz = 1 << width;
        }
        const int need = bfly ? bsz + (bsz + 15) / 16 : sz;
        if (entries + need > DFULL_MAX_ENTRIES ||
            (!local && __builtin_popcount(ubits | d.cm_loc) > 6))
          continue;
        d.mode |= DP_FULL;
        if (local) {
          d.mode |= DP_NODEFER;
        } else if (later) {
          d.mode |= DP_PRE;
          P.h.dpre |= (uint8_t)(1u << nd);
        }
        if (bfly) {
          d.mode |= DP_BFLY;
          P.h.flags |= PF_BFLY;
          d.a = lo;      // table index = (s >> lo) & (2^width - 1)
          d.b = width;
        }
        d.z_glob = (uint64_t)entries;
        d.b0 = (uint8_t)nd;   // deferred slot (local ops: renumbered below)
        entries += need;
        if (!local) {
          ubits |= d.cm_loc;
          nd++;
        }
        nfull++;
      }
      // b0 is also the op's scratch slot for building its table in the tile
      // buffer: the deferred ops keep their slots 0..nd-1, local ones follow
      for (int o = 0, sl = nd; o < cnt; o++)
        if (P.ops[o].type == OP_DPHASE && (P.ops[o].mode & DP_NODEFER)) P.ops[o].b0 = (uint8_t)sl++;
      if (entries) {
        // re-lay the resident area: full-mode ops keep their triples only
        uint32_t w2 = 0;
        for (int o = 0; o < cnt; o++) {
          Op& d = P.ops[o];
          if (d.type != OP_DPHASE || !(d.mode & DP_TABLE)) continue;
          d.z_loc = w2;
          w2 += ((d.mode & DP_FULL) ? 0u : 256u) + 3u * d.b1;
        }
        P.h.dtab_words = (int32_t)w2;
        P.h.flags |= PF_DFULL;
        P.h.dfull_entries = entries;
        P.h.ndefer = (int8_t)nd;
        int nb = 0;
        for (uint32_t u = ubits; u; u &= u - 1) P.h.dbits[nb++] = (int8_t)__builtin_ctz(u);
        P.h.ndbits = (int8_t)nb;
        auto squeeze = [&](uint32_t v) {   // bits of v at dbits -> index bits
          uint32_t r = 0;
          for (int i = 0; i < nb; i++) r |= ((v >> P.h.dbits[i]) & 1u) << i;
          return (uint8_t)r;
        };
        for (int o = 0; o < cnt; o++) {
          const Op& d = P.ops[o];
          if (d.type != OP_DPHASE || !(d.mode & DP_FULL) || (d.mode & DP_NODEFER)) continue;
          P.h.dmask[d.b0] = squeeze(d.cm_loc);
          P.h.dval[d.b0] = squeeze(d.cv_loc);
        }
      }
    }
    if (p + 1 == passes.size() && need_scale && !folded) {
      LOp s;
      s.type = OP_SCALE;
      s.mode = (uint8_t)((zi == 0.0 ? 1 : 0) | 2);
      s.a = zr;
      s.b = zi;
      plist.push_back(s);
      if ((P.h.flags & PF_DFULL) && P.h.ndefer > 0 && !opt.force_scale &&
          coef_at + 2 <= MAX_COEF) {
        // every amplitude of the pass is multiplied by an entry of its
        // deferred phase table: the scalar joins those entries (a complex
        // multiply per entry and tile) instead of costing a sweep
        P.h.flags |= PF_DSCALE;
        P.h.dsc = (uint16_t)coef_at;
        P.coef[coef_at] = zr;
        P.coef[coef_at + 1] = zi;
        coef_at += 2;
      } else {
        fill_op(P.ops[cnt], s, B.tile, pos, 0);
        out.op_src[p * MAX_OPS + cnt] = -1;
        cnt++;
      }
    }
    P.h.nops = cnt;
    out.pass_ops.push_back(plist);
  }
  return LQ_OK;
}

}  // namespace lq
