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
#include <vector>

#include "lq_coefs.h"
#include "lq_internal.h"
#include "lq_kernels.h"

namespace lq {

#define LQ_CUDA(expr)                                                                  \
  do {                                                                                 \
    cudaError_t e_ = (expr);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(LQ_ERR_CUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, \
                  __LINE__);                                                           \
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
  int n = np > 0 ? np : 1;
  psr_grad_kernel<<<(n + 127) / 128, 128, 0, s>>>(E, np, out);
  return cudaGetLastError();
}

// Patch of circuit (gate g shifted to angle theta): new op coefficients and
// the ratio new/old of the gate's deferred factor.
static Patch make_patch(const lq_gate& G, int g, double theta_base, double theta) {
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
  // (a1.z) / (a0.z)
  double den = a0.zr * a0.zr + a0.zi * a0.zi;
  p.zr = (a1.zr * a0.zr + a1.zi * a0.zi) / den;
  p.zi = (a1.zi * a0.zr - a1.zr * a0.zi) / den;
  return p;
}

static Patch no_patch() {
  Patch p;
  std::memset(&p, 0, sizeof p);
  p.gate = -2;
  p.zr = 1.0;
  return p;
}

// Expectation workspace layout helper (partials for `nstates`).
static std::size_t exp_partials(int n, int nstates) {
  return align256(sizeof(double) * (std::size_t)expval_grid(n) * (std::size_t)nstates);
}

// How many circuits the batched method runs per launch.
static int psr_chunk(int n, int C) {
  std::size_t sb = sizeof(double2) << n;
  std::size_t cap = ((std::size_t)4 << 30) / sb;  // about 4 GiB of states per chunk
  if (cap < 1) cap = 1;
  return (int)((std::size_t)C < cap ? (std::size_t)C : cap);
}

static std::size_t batched_ws(int n, int C, int np) {
  int chunk = psr_chunk(n, C);
  return align256((sizeof(double2) << n) * (std::size_t)chunk) +
         align256(sizeof(Patch) * (std::size_t)chunk) + exp_partials(n, chunk) +
         align256(sizeof(double) * (std::size_t)C) + align256(sizeof(double) * (np + 1));
}

// Energies of C circuits that share the lowered schedule of (gates at
// params), each modified by patches[c].  Writes E[0..C) (device).
lq_status run_patched_energies(int n, const lq_gate* gates, int ng, const double* params,
                               int np, const lq_pauli_term* terms, int nt,
                               const std::vector<Patch>& patches, double* E_dev,
                               char* ws, std::size_t ws_bytes, cudaStream_t s) {
  const int C = (int)patches.size();
  LOp* ops = nullptr;
  std::size_t nops = 0;
  double zr, zi;
  lq_status st = lower_circuit(n, gates, ng, params, np, &ops, &nops, &zr, &zi);
  if (st) return st;
  ScheduleOptions opt;
  opt.force_scale = true;
  Schedule S;
  st = schedule_ops(n, ops, nops, zr, zi, opt, S);
  delete[] ops;
  if (st) return st;
  const int chunk = psr_chunk(n, C);
  const std::size_t sb = sizeof(double2) << n;
  char* p = ws;
  double2* states = (double2*)p;
  p += align256(sb * (std::size_t)chunk);
  Patch* d_patch = (Patch*)p;
  p += align256(sizeof(Patch) * (std::size_t)chunk);
  double* partial = (double*)p;
  p += exp_partials(n, chunk);
  if ((std::size_t)(p - ws) > ws_bytes) return fail(LQ_ERR_OOM, "workspace too small");
  for (int c0 = 0; c0 < C; c0 += chunk) {
    int cnt = C - c0 < chunk ? C - c0 : chunk;
    LQ_CUDA(cudaMemcpyAsync(d_patch, patches.data() + c0, sizeof(Patch) * cnt,
                            cudaMemcpyHostToDevice, s));
    for (int ps = 0; ps < S.npasses; ps++) {
      PassParams& P = S.passes[ps];
      if (ps == 0) P.h.flags |= PF_INIT_ZERO;
      LQ_CUDA(launch_pass(P, states, (uint64_t)1 << n, cnt, s, d_patch));
    }
    // expectation of every state of the chunk
    st = expval_states(states, (uint64_t)1 << n, cnt, n, terms, nt, partial, E_dev + c0, s);
    if (st) return st;
    // the chunk's passes must finish before the patches buffer is reused
    if (c0 + chunk < C) LQ_CUDA(cudaStreamSynchronize(s));
  }
  return LQ_OK;
}

}  // namespace lq

using namespace lq;

extern "C" {

size_t lq_param_shift_workspace_size(int n, int np, int nt, int method) {
  (void)nt;
  if (n < 1 || n > 34 || np < 0) return 0;
  if (method == LQ_PSR_PLAIN)
    return align256(sizeof(double2) << n) + lq_expval_workspace_size(n, nt);
  return batched_ws(n, 2 * np + 1, np);
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

  // batched
  const int C = 2 * np + 1;
  std::vector<Patch> patches((std::size_t)C);
  patches[0] = no_patch();
  for (int i = 0; i < np; i++) {
    int g = pg[i];
    if (g < 0) {
      patches[1 + 2 * i] = no_patch();
      patches[2 + 2 * i] = no_patch();
      continue;
    }
    double th = gates[g].angle + params[i];
    patches[1 + 2 * i] = make_patch(gates[g], g, th, th + kPi / 2);
    patches[2 + 2 * i] = make_patch(gates[g], g, th, th - kPi / 2);
  }
  char* ws = (char*)workspace;
  const int chunk = psr_chunk(n, C);
  std::size_t off = align256((sizeof(double2) << n) * (std::size_t)chunk) +
                    align256(sizeof(Patch) * (std::size_t)chunk) + exp_partials(n, chunk);
  double* E = (double*)(ws + off);
  double* out = (double*)(ws + off + align256(sizeof(double) * (std::size_t)C));
  st = run_patched_energies(n, gates, ng, params, np, terms, nt, patches, E, ws, off, s);
  if (st) return st;
  LQ_CUDA(launch_psr_grad(E, np, out, s));
  std::vector<double> h((std::size_t)np + 1);
  LQ_CUDA(cudaMemcpyAsync(h.data(), out, sizeof(double) * (np + 1), cudaMemcpyDeviceToHost, s));
  LQ_CUDA(cudaStreamSynchronize(s));
  *energy = h[0];
  for (int i = 0; i < np; i++) grad[i] = h[1 + i];
  return LQ_OK;
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
      if (P.zmask) {
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
  (void)n; (void)gates; (void)ng; (void)np; (void)nt;
  return 256;
}

lq_status lq_param_shift_grad_general(int n, const lq_gate* gates, int ng,
                                      const double* params, int np,
                                      const lq_pauli_term* terms, int nt, double* energy,
                                      double* grad, void* workspace, size_t ws_bytes,
                                      lq_stream stream) {
  (void)n; (void)gates; (void)ng; (void)params; (void)np; (void)terms; (void)nt;
  (void)energy; (void)grad; (void)workspace; (void)ws_bytes; (void)stream;
  return fail(LQ_ERR_UNSUPPORTED, "not built yet");
}

size_t lq_adjoint_workspace_size(int n, int ng, int np, int nt) {
  (void)n; (void)ng; (void)np; (void)nt;
  return 256;
}

lq_status lq_adjoint_grad(int n, const lq_gate* gates, int ng, const double* params, int np,
                          const lq_pauli_term* terms, int nt, double* energy, double* grad,
                          void* workspace, size_t ws_bytes, lq_stream stream) {
  (void)n; (void)gates; (void)ng; (void)params; (void)np; (void)terms; (void)nt;
  (void)energy; (void)grad; (void)workspace; (void)ws_bytes; (void)stream;
  return fail(LQ_ERR_UNSUPPORTED, "not built yet");
}

size_t lq_batch_workspace_size(const lq_problem* problems, int count) {
  (void)problems; (void)count;
  return 256;
}

lq_status lq_batch_param_shift(const lq_problem* problems, int count, void* workspace,
                               size_t ws_bytes, lq_stream stream) {
  (void)problems; (void)count; (void)workspace; (void)ws_bytes; (void)stream;
  return fail(LQ_ERR_UNSUPPORTED, "not built yet");
}

}  // extern "C"
