// lq_vqe.cpp -- the VQE outer loop of Sec. VI-B: minimise E(theta) =
// <psi(theta)|H|psi(theta)> with Adam (learning rate 1e-2, at most 350
// iterations, stop when the energy changes by less than 1e-7), each gradient
// computed on the GPU by the adjoint method or the batched parameter-shift
// rule.  The optimiser is the Adam update of Kingma and Ba (2015):
//   m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,
//   theta -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
#include <cmath>
#include <vector>

#include "../../include/lq.h"
#include "lq_internal.h"

using namespace lq;

extern "C" {

size_t lq_vqe_workspace_size(int n, int ng, int np, int nt, int method) {
  if (method == 0) return lq_adjoint_workspace_size(n, ng, np, nt);
  return lq_param_shift_workspace_size(n, np, nt, LQ_PSR_BATCHED);
}

lq_status lq_vqe_adam(int n, const lq_gate* gates, int ng, double* params, int np,
                      const lq_pauli_term* terms, int nt, const lq_adam_options* opt,
                      double* energies, int* iters, void* workspace, size_t ws_bytes,
                      lq_stream stream) {
  if (!opt || !params || !energies || !iters) return fail(LQ_ERR_INVALID_ARG, "NULL argument");
  if (opt->max_iters < 1) return fail(LQ_ERR_INVALID_ARG, "max_iters < 1");
  if (!(opt->lr > 0) || !(opt->beta1 >= 0 && opt->beta1 < 1) ||
      !(opt->beta2 >= 0 && opt->beta2 < 1) || !(opt->eps > 0) || !(opt->tol >= 0))
    return fail(LQ_ERR_INVALID_ARG, "bad Adam options");
  if (opt->method != 0 && opt->method != 1)
    return fail(LQ_ERR_INVALID_ARG, "method must be 0 (adjoint) or 1 (batched shift)");
  std::vector<double> g((std::size_t)(np > 0 ? np : 1)), m(g.size(), 0.0), v(g.size(), 0.0);
  double prev = 0;
  int t = 0;
  for (t = 1; t <= opt->max_iters; t++) {
    double e;
    lq_status st = opt->method == 0
                       ? lq_adjoint_grad(n, gates, ng, params, np, terms, nt, &e, g.data(),
                                         workspace, ws_bytes, stream)
                       : lq_param_shift_grad(n, gates, ng, params, np, terms, nt, LQ_PSR_BATCHED,
                                             &e, g.data(), workspace, ws_bytes, stream);
    if (st) return st;
    energies[t - 1] = e;
    if (t > 1 && std::fabs(e - prev) < opt->tol) break;
    prev = e;
    const double c1 = 1.0 - std::pow(opt->beta1, t), c2 = 1.0 - std::pow(opt->beta2, t);
    for (int i = 0; i < np; i++) {
      m[i] = opt->beta1 * m[i] + (1.0 - opt->beta1) * g[i];
      v[i] = opt->beta2 * v[i] + (1.0 - opt->beta2) * g[i] * g[i];
      params[i] -= opt->lr * (m[i] / c1) / (std::sqrt(v[i] / c2) + opt->eps);
    }
  }
  *iters = t > opt->max_iters ? opt->max_iters : t;
  return LQ_OK;
}

}  // extern "C"
