// lq_coefs.h -- angle-dependent coefficients of the parametrised gates, in
// the FP64-economical forms of the tile ops.  Shared by the host lowering and
// by kernels that re-derive a gate's coefficients for a shifted angle.
//
// Rotations R_P(theta) = exp(-i theta P / 2) (Sec. III-A):
//   exp(-i theta P/2) psi = c psi - i s P psi,  c = cos(theta/2), s = sin(theta/2)
//   tangent form   (|c| >= |s|): c (psi + t (-i P) psi),  t = s/c, factor c deferred
//   cotangent form (|c| <  |s|): s (u psi + (-i P) psi),  u = c/s, factor s deferred
// so |t|, |u| <= 1 and every deferred factor has magnitude >= 1/sqrt2.
#pragma once

#include <math.h>

#include "lq_internal.h"

namespace lq {

struct AngleCoefs {
  uint8_t mode0 = 0, mode1 = 0;  // Pauli modes of op 0 / op 1
  double a0 = 0, b0 = 0, a1 = 0, b1 = 0;
  double zr = 1, zi = 0;         // deferred factor
};

LQ_HD inline void angle_coefs(int kind, double theta, AngleCoefs& c) {
  double h = 0.5 * theta;
  double ch = cos(h), sh = sin(h);
  c = AngleCoefs();
  switch (kind) {
    case LQ_RX: case LQ_RY: case LQ_RXX: case LQ_RYY:
      if (fabs(ch) >= fabs(sh)) {
        c.mode0 = PM_TAN; c.a0 = sh / ch; c.zr = ch;
      } else {
        c.mode0 = PM_COT; c.a0 = ch / sh; c.zr = sh;
      }
      break;
    case LQ_CRX: case LQ_CRY:
      c.mode0 = PM_GEN; c.a0 = ch; c.b0 = sh;
      break;
    case LQ_RZ: case LQ_RZZ:
      // diag(e^{-i theta/2}, e^{i theta/2}) = e^{-i theta/2} diag(1, e^{i theta})
      c.a0 = cos(theta); c.b0 = sin(theta);
      c.zr = ch; c.zi = -sh;
      break;
    case LQ_P: case LQ_CP:
      c.a0 = cos(theta); c.b0 = sin(theta);
      break;
    case LQ_CRZ:
      // control set: target 0 -> e^{-i theta/2}, target 1 -> e^{+i theta/2}
      c.a0 = ch; c.b0 = -sh;
      c.a1 = ch; c.b1 = sh;
      break;
    default:
      break;
  }
}

}  // namespace lq
