// lq_psr.cu -- parameter-shift gradients (Sec. III-A Eq. parameter_shift,
// Sec. III-C ParameterShift::compute_gradient) and first-order Trotter
// evolution (Sec. VII-A, Eq. trotter).
//
// Plain method: exactly the paper's loop -- for every parameter, two fresh
// |0...0> states, the circuit at theta +- pi/2, <H>, and (E+ - E-)/2 -- issued as
// separate library calls.
//
// Batched method: the 2P+1 circuits (base, then +pi/2 and -pi/2 per parameter)
// share one pass schedule lowered at the base angles.  A circuit differs from
// the base only in the coefficients of its shifted gate and in the deferred
// scalar, so each circuit carries a small Patch (new coefficients, ratio of
// deferred factors) and every pass runs all circuits in one launch; the first
// pass starts from |0...0> in shared memory without reading HBM.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "lq_coefs.h"
#include "lq_internal.h"
#include "lq_kernels.h"

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

static const double kPi = 3.14159265358979323846;

// Two-term shift rule applies: generator with two eigenvalues one apart.
static bool two_term(int kind) {
  switch (kind) {
    case LQ_RX: case LQ_RY: case LQ_RZ: case LQ_P: case LQ_CP: case LQ_RXX: case LQ_RYY:
    case LQ_RZZ:
      return true;
    default:
      return false;
  }
}

// For each parameter, the single gate it drives (-1 if unused).
static lq_status psr_param_gates(const lq_gate* gates, int ng, int np, std::vector<int>& pg) {
  pg.assign((std::size_t)np, -1);
  for (int g = 0; g < ng; g++) {
    int p = gates[g].param;
    if (p < 0) continue;
    if (!two_term(gates[g].kind))
      return fail(LQ_ERR_UNSUPPORTED,
                  "gate %d (kind %d) needs a generalised shift rule; use "
                  "lq_param_shift_grad_general or lq_adjoint_grad", g, gates[g].kind);
    if (pg[p] >= 0)
      return fail(LQ_ERR_UNSUPPORTED,
                  "parameter %d drives several gates; use lq_param_shift_grad_general", p);
    pg[p] = g;
  }
  return LQ_OK;
}

__global__ void psr_grad_kernel(const double* __restrict__ E, int np, double* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) out[0] = E[0];
  if (i < np) out[1 + i] = 0.5 * (E[1 + 2 * i] - E[2 + 2 * i]);
}

cudaError_t launch_psr_grad(const double* E, int np, double* out, cudaStream_t s) {
  (void)cudaGetLastError();  // report only this launcher's own errors
  int n = np > 0 ? np : 1;
  psr_grad_kernel<<<(n + 127) / 128, 128, 0, s>>>(E, np, out);
  return cudaGetLastError();
}

}  // namespace lq

using namespace lq;

extern "C" {

static std::size_t batched_workspace_size(int n, int np, int nt) {
  // an HEA-shaped stand-in with np single-use rotations sizes the batch: the
  // workspace depends on n, the number of circuits and the program size
  std::vector<lq_gate> g((std::size_t)np);
  std::vector<double> p((std::size_t)np, 0.0);
  std::vector<lq_pauli_term> t((std::size_t)(nt > 0 ? nt : 0));
  for (int i = 0; i < np; i++) {
    std::memset(&g[i], 0, sizeof(lq_gate));
    g[i].kind = LQ_RY;
    g[i].qubits[0] = i % n;
    g[i].qubits[1] = g[i].qubits[2] = -1;
    g[i].param = i;
  }
  for (int i = 0; i < nt; i++) {
    t[i].coeff = 1.0;
    t[i].xmask = (uint64_t)(i % n);
    t[i].zmask = 0;
  }
  HostProblem hp;
  if (make_problem(n, g.data(), np, p.data(), np, t.data(), nt, true, false, hp)) return 0;
  std::vector<HostProblem> v(1, hp);
  // room for larger op programs than the stand-in: 1 MiB
  return batch_workspace_for(v, nullptr) + ((std::size_t)1 << 20);
}

size_t lq_param_shift_workspace_size(int n, int np, int nt, int method) {
  if (n < 1 || n > 34 || np < 0) return 0;
  if (method == LQ_PSR_PLAIN)
    return align256(sizeof(double2) << n) + lq_expval_workspace_size(n, nt);
  // the batched size depends on (n, np, nt) only; planning the stand-in takes
  // tens to hundreds of microseconds, and every batched call checks its
  // workspace against it, so sizes are kept
  static std::mutex mu;
  static std::map<std::tuple<int, int, int>, std::size_t> sizes;
  const auto key = std::make_tuple(n, np, nt);
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = sizes.find(key);
    if (it != sizes.end()) return it->second;
  }
  const std::size_t sz = batched_workspace_size(n, np, nt);
  if (sz) {
    std::lock_guard<std::mutex> lk(mu);
    if (sizes.size() > 256) sizes.clear();
    sizes[key] = sz;
  }
  return sz;
}


lq_status lq_param_shift_grad(int n, const lq_gate* gates, int ng, const double* params,
                              int np, const lq_pauli_term* terms, int nt, int method,
                              double* energy, double* grad, void* workspace, size_t ws_bytes,
                              lq_stream stream) {
  lq_status st = check_n(n);
  if (st) return st;
  st = check_gates(n, gates, ng, params, np);
  if (st) return st;
  st = check_terms(n, terms, nt);
  if (st) return st;
  if (!energy || (np > 0 && !grad)) return fail(LQ_ERR_INVALID_ARG, "NULL output");
  if (method != LQ_PSR_PLAIN && method != LQ_PSR_BATCHED)
    return fail(LQ_ERR_INVALID_ARG, "unknown method %d", method);
  std::vector<int> pg;
  st = psr_param_gates(gates, ng, np, pg);
  if (st) return st;
  std::size_t need = lq_param_shift_workspace_size(n, np, nt, method);
  if (!workspace || ws_bytes < need)
    return fail(LQ_ERR_OOM, "workspace too small: %zu < %zu", ws_bytes, need);
  cudaStream_t s = (cudaStream_t)stream;

  if (method == LQ_PSR_PLAIN) {
    // the paper's loop: fresh state, circuit, expectation, per evaluation
    void* psi = workspace;
    char* ews = (char*)workspace + align256(sizeof(double2) << n);
    std::size_t ews_bytes = ws_bytes - align256(sizeof(double2) << n);
    std::vector<double> p(params, params + np);
    auto eval = [&](double* out) -> lq_status {
      lq_status r = lq_state_init(psi, n, 0, stream);
      if (r) return r;
      r = lq_apply_circuit(psi, n, gates, ng, p.data(), np, stream);
      if (r) return r;
      return lq_expval_pauli_sum(psi, n, terms, nt, out, ews, ews_bytes, stream);
    };
    st = eval(energy);
    if (st) return st;
    for (int i = 0; i < np; i++) {
      double fp, fm;
      p[i] = params[i] + kPi / 2;
      st = eval(&fp);
      if (st) return st;
      p[i] = params[i] - kPi / 2;
      st = eval(&fm);
      if (st) return st;
      p[i] = params[i];
      grad[i] = 0.5 * (fp - fm);
    }
    return LQ_OK;
  }

  // batched: every circuit in one persistent launch
  HostProblem hp;
  st = make_problem(n, gates, ng, params, np, terms, nt, true, false, hp);
  if (st) return st;
  std::vector<HostProblem> v(1, hp);
  std::vector<double> out;
  st = batch_run(v, workspace, ws_bytes, s, out);
  if (st) return st;
  *energy = out[0];
  for (int i = 0; i < np; i++) grad[i] = out[1 + i];
  return LQ_OK;
}

lq_status lq_autotune_param_shift(int n, const lq_gate* gates, int ng, const double* params,
                                  int np, const lq_pauli_term* terms, int nt, void* workspace,
                                  size_t ws_bytes, lq_tune_result* out, lq_stream stream) {
  lq_status st = check_n(n);
  if (st) return st;
  st = check_gates(n, gates, ng, params, np);
  if (st) return st;
  st = check_terms(n, terms, nt);
  if (st) return st;
  if (!out) return fail(LQ_ERR_INVALID_ARG, "out is NULL");
  std::vector<int> pg;
  st = psr_param_gates(gates, ng, np, pg);
  if (st) return st;
  std::size_t need = lq_param_shift_workspace_size(n, np, nt, LQ_PSR_BATCHED);
  if (!workspace || ws_bytes < need)
    return fail(LQ_ERR_OOM, "workspace too small: %zu < %zu", ws_bytes, need);
  HostProblem hp;
  st = make_problem(n, gates, ng, params, np, terms, nt, true, false, hp);
  if (st) return st;
  std::vector<HostProblem> v(1, hp);
  return batch_autotune(v, workspace, ws_bytes, (cudaStream_t)stream, out);
}

// ------------------------------------------------------------- Trotter

lq_status lq_trotter_evolve(void* amps, int n, const lq_pauli_term* terms, int nt,
                            const lq_pauli_term* field, int nf, double A, double omega,
                            double dt, int steps, lq_stream stream) {
  lq_status st = check_n(n);
  if (st) return st;
  if (!amps) return fail(LQ_ERR_INVALID_ARG, "amps is NULL");
  st = check_terms(n, terms, nt);
  if (st) return st;
  st = check_terms(n, field, nf);
  if (st) return st;
  if (steps < 0) return fail(LQ_ERR_INVALID_ARG, "steps < 0");
  if (!std::isfinite(A) || !std::isfinite(omega) || !std::isfinite(dt))
    return fail(LQ_ERR_NONFINITE, "A, omega or dt not finite");
  // exp(-i phi P): x == 0 -> parity phase e^{-i phi} (even) / e^{+i phi} (odd);
  // x != 0 -> Pauli rotation with theta/2 = phi, tangent or cotangent form
  std::vector<LOp> ops;
  ops.reserve((std::size_t)steps * (nt + nf) + 8);
  double zr = 1, zi = 0;
  auto push = [&](const lq_pauli_term& P, double phi) {
    double c = std::cos(phi), s = std::sin(phi);
    double fr, fi;
    LOp o;
    if (P.xmask == 0) {
      fr = c;
      fi = -s;  // e^{-i phi}
      if (P.zmask && (P.zmask & (P.zmask - 1)) == 0) {
        // one Z: e^{-i phi} diag(1, e^{2 i phi}) on its bit, a one-bit phase
        // that merges with the step's other field terms into one table op
        o.type = OP_PHASE;
        o.cm = o.cv = P.zmask;
        o.a = std::cos(2 * phi);
        o.b = std::sin(2 * phi);
        ops.push_back(o);
      } else if (P.zmask) {
        o.type = OP_PARITY;
        o.z = P.zmask;
        o.a = std::cos(2 * phi);
        o.b = std::sin(2 * phi);
        ops.push_back(o);
      }
    } else {
      int ny = __builtin_popcountll(P.xmask & P.zmask);
      o.type = OP_PAULI;
      o.x = P.xmask;
      o.z = P.zmask;
      if (std::fabs(c) >= std::fabs(s)) {
        o.mode = (uint8_t)(PM_TAN | (((3 + ny) & 3) << 2));
        o.a = s / c;
        fr = c;
      } else {
        o.mode = (uint8_t)(PM_COT | (((3 + ny) & 3) << 2));
        o.a = c / s;
        fr = s;
      }
      fi = 0;
      ops.push_back(o);
    }
    double nr = zr * fr - zi * fi, ni = zr * fi + zi * fr;
    zr = nr;
    zi = ni;
    double mag = std::hypot(zr, zi);
    if (mag < 1e-100 || mag > 1e100) {
      LOp sc;
      sc.type = OP_SCALE;
      sc.mode = 1;
      sc.a = mag;
      ops.push_back(sc);
      zr /= mag;
      zi /= mag;
    }
  };
  for (int j = 0; j < steps; j++) {
    double tj = j * dt, h = A * std::sin(omega * tj);
    for (int k = 0; k < nt; k++) push(terms[k], terms[k].coeff * dt);
    for (int f = 0; f < nf; f++) push(field[f], h * field[f].coeff * dt);
  }
  ScheduleOptions opt;
  opt.lphase_table = true;   // run by pass_kernel
  opt.max_hi = PASS_HI_BITS;
  opt.sink_phases = true;
  Schedule S;
  st = schedule_ops(n, ops.data(), ops.size(), zr, zi, opt, S);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  for (int p = 0; p < S.npasses; p++) LQ_CUDA(launch_pass(S.passes[p], (double2*)amps, 0, 1, s));
  return LQ_OK;
}

// ------------------------------------------------- not yet implemented

size_t lq_param_shift_general_workspace_size(int n, const lq_gate* gates, int ng, int np,
                                             int nt) {
  if (n < 1 || n > 34 || np < 0 || ng < 0 || (ng > 0 && !gates)) return 0;
  // sizes depend on the circuit's structure only: evaluate at zero parameters
  std::vector<double> p((std::size_t)(np > 0 ? np : 1), 0.0);
  std::vector<lq_pauli_term> t((std::size_t)(nt > 0 ? nt : 1));
  for (int i = 0; i < nt; i++) {
    t[i].coeff = 1.0;
    t[i].xmask = (uint64_t)(i % n);
    t[i].zmask = 0;
  }
  HostProblem hp;
  if (make_problem(n, gates, ng, p.data(), np, t.data(), nt, true, true, hp)) return 0;
  std::vector<HostProblem> v(1, hp);
  return batch_workspace_for(v, nullptr) + ((std::size_t)1 << 20);
}

lq_status lq_param_shift_grad_general(int n, const lq_gate* gates, int ng,
                                      const double* params, int np,
                                      const lq_pauli_term* terms, int nt, double* energy,
                                      double* grad, void* workspace, size_t ws_bytes,
                                      lq_stream stream) {
  if (!energy || (np > 0 && !grad)) return fail(LQ_ERR_INVALID_ARG, "NULL output");
  HostProblem hp;
  lq_status st = make_problem(n, gates, ng, params, np, terms, nt, true, true, hp);
  if (st) return st;
  std::vector<HostProblem> v(1, hp);
  std::vector<double> out;
  st = batch_run(v, workspace, ws_bytes, (cudaStream_t)stream, out);
  if (st) return st;
  *energy = out[0];
  for (int i = 0; i < np; i++) grad[i] = out[1 + i];
  return LQ_OK;
}

}  // extern "C"
