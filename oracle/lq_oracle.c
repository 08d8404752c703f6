/*
 * lq_oracle.c -- plain, slow CPU oracle for the dense state-vector method of
 * arXiv 2512.23183 ("LogosQ").
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and the cpu
 * baseline of bench.py may load or call this library.  It shares no code,
 * header, table or constant with the CUDA path.
 *
 * Everything is complex128 (C99 `double complex`), which matches the paper's
 * Complex64 = two f64 state vector (Sec. II, "Dense State Vector
 * Representation").  Each routine is the plain definition of what it
 * computes, written out with no blocking, fusion or reordering:
 *
 *   - index convention: qubit q is bit n-1-q of the amplitude index
 *     (MSB-first, Alg. 1 and Alg. 4, App. A/B worked examples);
 *   - a k-qubit gate is its 2^k x 2^k matrix, the first listed qubit being the
 *     most significant bit of the gate's local index (the two-qubit matrix
 *     index (s1, s2) of Sec. II-C, Eq. for the MPS two-site gate), applied to
 *     every group of 2^k amplitudes that differ only in the gate's bits;
 *   - rotations are R_P(theta) = exp(-i theta sigma_P / 2) (Sec. III-A);
 *   - a circuit applies its operations in list order (Sec. II-A, execute);
 *   - <H> = sum_t c_t <psi|P_t|psi>, each P_t applied to a copy of psi as a
 *     product of one-qubit Pauli matrices (Sec. VI-A, Sec. VII-A-2);
 *   - the parameter-shift gradient restarts from |0...0> for every shifted
 *     evaluation (Sec. III-A Eq. parameter_shift, Sec. III-C listing);
 *   - QFT in FFT form: unitary inverse DFT, a plain iterative radix-2 FFT with
 *     the + sign followed by 1/sqrt(N) (Sec. IV-B, Alg. 2 and the QFT formula);
 *   - QFT in gate form: H, then CP(pi/2^(j-i)) controlled by i on every
 *     later j, then the swaps (Alg. 3);
 *   - first-order Trotter evolution: exp(-i c_k P_k dt) factors in term order
 *     for every step t_j = j dt (Sec. VII-A-1, Eq. trotter).
 *
 * Parity pins for every function live in tests/test_oracle_pins.py.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* Oracle-private gate codes; the Python wrapper maps gate names onto them. */
enum {
  OG_H = 0, OG_X, OG_Y, OG_Z, OG_S, OG_SDG, OG_T, OG_TDG, OG_RX, OG_RY, OG_RZ,
  OG_P, OG_U1, OG_CNOT, OG_CY, OG_CZ, OG_CP, OG_SWAP, OG_CRX, OG_CRY, OG_CRZ,
  OG_RXX, OG_RYY, OG_RZZ, OG_CCX, OG_U2, OG_COUNT
};

#define OR_OK 0
#define OR_EINVAL 1
#define OR_EUNSUPPORTED 2

static const double OR_PI = 3.14159265358979323846264338327950288;

int or_arity(int g) {
  switch (g) {
    case OG_H: case OG_X: case OG_Y: case OG_Z: case OG_S: case OG_SDG:
    case OG_T: case OG_TDG: case OG_RX: case OG_RY: case OG_RZ: case OG_P:
    case OG_U1:
      return 1;
    case OG_CNOT: case OG_CY: case OG_CZ: case OG_CP: case OG_SWAP:
    case OG_CRX: case OG_CRY: case OG_CRZ: case OG_RXX: case OG_RYY:
    case OG_RZZ: case OG_U2:
      return 2;
    case OG_CCX:
      return 3;
    default:
      return 0;
  }
}

/* 1 if the gate takes an angle (fixed or from the parameter vector). */
int or_takes_angle(int g) {
  switch (g) {
    case OG_RX: case OG_RY: case OG_RZ: case OG_P: case OG_CP: case OG_CRX:
    case OG_CRY: case OG_CRZ: case OG_RXX: case OG_RYY: case OG_RZZ:
      return 1;
    default:
      return 0;
  }
}

/* Pauli matrices by letter: 0=I, 1=X, 2=Y, 3=Z. */
static void pauli2(int p, cplx M[4]) {
  M[0] = M[1] = M[2] = M[3] = 0;
  switch (p) {
    case 0: M[0] = 1; M[3] = 1; break;
    case 1: M[1] = 1; M[2] = 1; break;
    case 2: M[1] = -I; M[2] = I; break;
    case 3: M[0] = 1; M[3] = -1; break;
  }
}

/* exp(-i theta/2 sigma) = cos(theta/2) I - i sin(theta/2) sigma, for a
 * Pauli (or tensor product of two Paulis) sigma with sigma^2 = I. */
static void pauli_rotation(const cplx* sigma, int d, double theta, cplx* M) {
  double c = cos(theta / 2), s = sin(theta / 2);
  for (int r = 0; r < d; r++)
    for (int k = 0; k < d; k++)
      M[r * d + k] = (r == k ? c : 0.0) - I * s * sigma[r * d + k];
}

static void kron2(const cplx A[4], const cplx B[4], cplx M[16]) {
  for (int r = 0; r < 4; r++)
    for (int k = 0; k < 4; k++)
      M[r * 4 + k] = A[(r >> 1) * 2 + (k >> 1)] * B[(r & 1) * 2 + (k & 1)];
}

/* Controlled version: block-diag(I, U) over (control, target). */
static void controlled(const cplx U[4], cplx M[16]) {
  for (int i = 0; i < 16; i++) M[i] = 0;
  M[0] = 1; M[5] = 1;
  M[10] = U[0]; M[11] = U[1]; M[14] = U[2]; M[15] = U[3];
}

/* Fill the 2^k x 2^k row-major matrix of gate g.  `um` holds the
 * row-major (re, im) pairs for U1 (8 doubles) and U2 (32 doubles). */
int or_gate_matrix(int g, double theta, const double* um, double* out) {
  cplx* M = (cplx*)out;
  cplx P[4], Q[4], R[4], K[16];
  int k = or_arity(g);
  if (k == 0) return OR_EINVAL;
  int d = 1 << k;
  for (int i = 0; i < d * d; i++) M[i] = 0;
  double c = cos(theta / 2), s = sin(theta / 2);
  switch (g) {
    case OG_H: {
      double r = 1.0 / sqrt(2.0);
      M[0] = r; M[1] = r; M[2] = r; M[3] = -r;
      break;
    }
    case OG_X: pauli2(1, M); break;
    case OG_Y: pauli2(2, M); break;
    case OG_Z: pauli2(3, M); break;
    case OG_S: M[0] = 1; M[3] = I; break;
    case OG_SDG: M[0] = 1; M[3] = -I; break;
    case OG_T: M[0] = 1; M[3] = cexp(I * OR_PI / 4); break;
    case OG_TDG: M[0] = 1; M[3] = cexp(-I * OR_PI / 4); break;
    case OG_RX: pauli2(1, P); pauli_rotation(P, 2, theta, M); break;
    case OG_RY: pauli2(2, P); pauli_rotation(P, 2, theta, M); break;
    case OG_RZ: pauli2(3, P); pauli_rotation(P, 2, theta, M); break;
    case OG_P: M[0] = 1; M[3] = cexp(I * theta); break;
    case OG_U1:
      for (int i = 0; i < 4; i++) M[i] = um[2 * i] + I * um[2 * i + 1];
      break;
    case OG_CNOT: pauli2(1, P); controlled(P, M); break;
    case OG_CY: pauli2(2, P); controlled(P, M); break;
    case OG_CZ: pauli2(3, P); controlled(P, M); break;
    case OG_CP: M[0] = 1; M[5] = 1; M[10] = 1; M[15] = cexp(I * theta); break;
    case OG_SWAP: M[0] = 1; M[6] = 1; M[9] = 1; M[15] = 1; break;
    case OG_CRX: pauli2(1, P); pauli_rotation(P, 2, theta, R); controlled(R, M); break;
    case OG_CRY: pauli2(2, P); pauli_rotation(P, 2, theta, R); controlled(R, M); break;
    case OG_CRZ: pauli2(3, P); pauli_rotation(P, 2, theta, R); controlled(R, M); break;
    case OG_RXX: pauli2(1, P); pauli2(1, Q); kron2(P, Q, K); pauli_rotation(K, 4, theta, M); break;
    case OG_RYY: pauli2(2, P); pauli2(2, Q); kron2(P, Q, K); pauli_rotation(K, 4, theta, M); break;
    case OG_RZZ: pauli2(3, P); pauli2(3, Q); kron2(P, Q, K); pauli_rotation(K, 4, theta, M); break;
    case OG_CCX:
      /* identity except |110> <-> |111> (both controls set, target flipped) */
      for (int i = 0; i < 6; i++) M[i * 8 + i] = 1;
      M[6 * 8 + 7] = 1; M[7 * 8 + 6] = 1;
      break;
    case OG_U2:
      for (int i = 0; i < 16; i++) M[i] = um[2 * i] + I * um[2 * i + 1];
      break;
  }
  (void)c; (void)s;
  return OR_OK;
}

/* Apply a 2^k x 2^k matrix on qubits q[0..k-1] (q[0] = most significant bit
 * of the local index).  Qubit q lives at bit n-1-q of the amplitude index. */
void or_apply_matrix(double* state, int n, const int* q, int k, const double* mat) {
  cplx* psi = (cplx*)state;
  const cplx* M = (const cplx*)mat;
  int d = 1 << k;
  uint64_t N = 1ull << n, masks[3] = {0, 0, 0}, allm = 0;
  for (int j = 0; j < k; j++) {
    masks[j] = 1ull << (n - 1 - q[j]);
    allm |= masks[j];
  }
#pragma omp parallel for schedule(static)
  for (int64_t b = 0; b < (int64_t)N; b++) {
    uint64_t base = (uint64_t)b;
    if (base & allm) continue;
    cplx in[8], out[8];
    uint64_t idx[8];
    for (int l = 0; l < d; l++) {
      uint64_t i = base;
      for (int j = 0; j < k; j++)
        if ((l >> (k - 1 - j)) & 1) i |= masks[j];
      idx[l] = i;
      in[l] = psi[i];
    }
    for (int r = 0; r < d; r++) {
      cplx acc = 0;
      for (int c = 0; c < d; c++) acc += M[r * d + c] * in[c];
      out[r] = acc;
    }
    for (int l = 0; l < d; l++) psi[idx[l]] = out[l];
  }
}

/* |x>: amplitude x is 1, every other amplitude 0 (DenseState::zero_state for
 * x = 0, Sec. II-B). */
void or_state_basis(double* state, int n, uint64_t x) {
  cplx* psi = (cplx*)state;
  uint64_t N = 1ull << n;
  for (uint64_t i = 0; i < N; i++) psi[i] = 0;
  psi[x] = 1;
}

/* Alg. 1: direct CNOT.  For every index with the control bit set and the
 * target bit clear, swap it with the index whose target bit is flipped. */
void or_cnot_alg1(double* state, int n, int c, int t) {
  cplx* psi = (cplx*)state;
  uint64_t cmask = 1ull << (n - 1 - c), tmask = 1ull << (n - 1 - t);
  uint64_t N = 1ull << n;
  for (uint64_t i = 0; i < N; i++) {
    if ((i & cmask) != 0 && (i & tmask) == 0) {
      uint64_t j = i ^ tmask;
      cplx tmp = psi[i];
      psi[i] = psi[j];
      psi[j] = tmp;
    }
  }
}

/* Alg. 4 (App. B): direct Toffoli with the combined control mask. */
void or_toffoli_alg4(double* state, int n, int c1, int c2, int t) {
  cplx* psi = (cplx*)state;
  uint64_t both = (1ull << (n - 1 - c1)) | (1ull << (n - 1 - c2));
  uint64_t tmask = 1ull << (n - 1 - t);
  uint64_t N = 1ull << n;
  for (uint64_t i = 0; i < N; i++) {
    if ((i & both) == both && (i & tmask) == 0) {
      uint64_t j = i ^ tmask;
      cplx tmp = psi[i];
      psi[i] = psi[j];
      psi[j] = tmp;
    }
  }
}

/* One gate of a circuit.  The angle used is params[pidx] + angle when
 * pidx >= 0, else the fixed angle. */
static int apply_gate(double* state, int n, int g, const int* q, int pidx,
                      double angle, const double* um, const double* params, int np) {
  int k = or_arity(g);
  if (k == 0) return OR_EINVAL;
  for (int j = 0; j < k; j++) {
    if (q[j] < 0 || q[j] >= n) return OR_EINVAL;
    for (int l = 0; l < j; l++)
      if (q[l] == q[j]) return OR_EINVAL;
  }
  double theta = angle;
  if (pidx >= 0) {
    if (pidx >= np || !or_takes_angle(g)) return OR_EINVAL;
    theta += params[pidx];
  }
  double M[2 * 64];
  or_gate_matrix(g, theta, um, M);
  or_apply_matrix(state, n, q, k, M);
  return OR_OK;
}

/* Apply a gate list in order (Circuit::execute).  qubits: 3 ints per gate;
 * mats: 32 doubles per gate (read for U1/U2 only). */
int or_apply_circuit(double* state, int n, const int* kinds, const int* qubits,
                     const int* pidx, const double* angles, const double* mats,
                     int ng, const double* params, int np) {
  for (int g = 0; g < ng; g++) {
    int rc = apply_gate(state, n, kinds[g], qubits + 3 * g, pidx[g], angles[g],
                        mats + 32 * g, params, np);
    if (rc) return rc;
  }
  return OR_OK;
}

/* <psi|P|psi> for one Pauli string (chars 'I','X','Y','Z'; char q acts on
 * qubit q), by applying P to a copy of psi and taking the inner product. */
static double pauli_expval(const cplx* psi, cplx* work, int n, const char* s) {
  uint64_t N = 1ull << n;
  memcpy(work, psi, N * sizeof(cplx));
  for (int q = 0; q < n; q++) {
    int p = s[q] == 'X' ? 1 : s[q] == 'Y' ? 2 : s[q] == 'Z' ? 3 : 0;
    if (p == 0) continue;
    cplx M[4];
    pauli2(p, M);
    or_apply_matrix((double*)work, n, &q, 1, (const double*)M);
  }
  double re = 0;
#pragma omp parallel for reduction(+ : re) schedule(static)
  for (int64_t i = 0; i < (int64_t)N; i++) re += creal(conj(psi[i]) * work[i]);
  return re;
}

/* <H> = sum_t c_t <psi|P_t|psi>.  paulis: nt strings of n chars each. */
int or_expval(const double* state, int n, const char* paulis, const double* coeffs,
              int nt, double* out) {
  uint64_t N = 1ull << n;
  cplx* work = (cplx*)malloc(N * sizeof(cplx));
  if (!work) return OR_EINVAL;
  double e = 0;
  for (int t = 0; t < nt; t++)
    e += coeffs[t] * pauli_expval((const cplx*)state, work, n, paulis + (size_t)t * n);
  free(work);
  *out = e;
  return OR_OK;
}

/* E(theta): fresh |0...0>, the circuit, then <H>. */
static int energy(int n, const int* kinds, const int* qubits, const int* pidx,
                  const double* angles, const double* mats, int ng,
                  const double* params, int np, const char* paulis,
                  const double* coeffs, int nt, cplx* psi, double* out) {
  or_state_basis((double*)psi, n, 0);
  int rc = or_apply_circuit((double*)psi, n, kinds, qubits, pidx, angles, mats,
                            ng, params, np);
  if (rc) return rc;
  return or_expval((const double*)psi, n, paulis, coeffs, nt, out);
}

int or_energy(int n, const int* kinds, const int* qubits, const int* pidx,
              const double* angles, const double* mats, int ng, const double* params,
              int np, const char* paulis, const double* coeffs, int nt, double* out) {
  cplx* psi = (cplx*)malloc((1ull << n) * sizeof(cplx));
  if (!psi) return OR_EINVAL;
  int rc = energy(n, kinds, qubits, pidx, angles, mats, ng, params, np, paulis,
                  coeffs, nt, psi, out);
  free(psi);
  return rc;
}

/* Shift rule that applies to the generator of gate g:
 *   1: two-term rule, shift pi/2, factor 1/2 (generator with two eigenvalues
 *      a distance 1 apart: Pauli rotations RX/RY/RZ/RXX/RYY/RZZ, and the
 *      phase gates P and CP whose generator is a projector; Sec. III-A);
 *   2: four-term rule for the controlled rotations CRX/CRY/CRZ, whose
 *      generator |1><1| (x) sigma/2 has the three eigenvalues -1/2, 0, 1/2
 *      (the generalised rules the paper cites in Sec. III-A);
 *   0: not a parametrised gate. */
static int shift_rule(int g) {
  switch (g) {
    case OG_RX: case OG_RY: case OG_RZ: case OG_P: case OG_CP:
    case OG_RXX: case OG_RYY: case OG_RZZ:
      return 1;
    case OG_CRX: case OG_CRY: case OG_CRZ:
      return 2;
    default:
      return 0;
  }
}

/* Parameter-shift gradient, Eq. parameter_shift with s = pi/2:
 *   g_i = ( E(theta + s e_i) - E(theta - s e_i) ) / 2,
 * each evaluation from a fresh |0...0> (Sec. III-C, ParameterShift).
 * With general=0 every parameter must drive exactly one gate whose rule is
 * the two-term rule (else OR_EUNSUPPORTED, the paper's setting).  With
 * general=1 a parameter may drive several gates (the derivative is the sum
 * over its occurrences, each occurrence shifted on its own) and controlled
 * rotations use the four-term rule
 *   d1 [f(+pi/2) - f(-pi/2)] - d2 [f(+3pi/2) - f(-3pi/2)],
 *   d1 = (sqrt2 + 1) / (4 sqrt2),  d2 = (sqrt2 - 1) / (4 sqrt2).
 * Also returns E(theta) in *e0. */
int or_param_shift(int n, const int* kinds, const int* qubits, const int* pidx,
                   const double* angles, const double* mats, int ng,
                   const double* params, int np, const char* paulis,
                   const double* coeffs, int nt, int general, double* e0, double* grad) {
  int* uses = (int*)calloc(np > 0 ? np : 1, sizeof(int));
  for (int g = 0; g < ng; g++) {
    if (pidx[g] < 0) continue;
    if (pidx[g] >= np) { free(uses); return OR_EINVAL; }
    int rule = shift_rule(kinds[g]);
    if (rule == 0) { free(uses); return OR_EINVAL; }
    if (!general && rule != 1) { free(uses); return OR_EUNSUPPORTED; }
    uses[pidx[g]]++;
  }
  if (!general)
    for (int i = 0; i < np; i++)
      if (uses[i] > 1) { free(uses); return OR_EUNSUPPORTED; }
  free(uses);

  cplx* psi = (cplx*)malloc((1ull << n) * sizeof(cplx));
  double* ang = (double*)malloc((ng > 0 ? ng : 1) * sizeof(double));
  int* pid = (int*)malloc((ng > 0 ? ng : 1) * sizeof(int));
  if (!psi || !ang || !pid) { free(psi); free(ang); free(pid); return OR_EINVAL; }
  int rc = energy(n, kinds, qubits, pidx, angles, mats, ng, params, np, paulis,
                  coeffs, nt, psi, e0);
  for (int i = 0; i < np && rc == OR_OK; i++) grad[i] = 0;
  /* Each occurrence g of parameter i: freeze every gate to its own angle
   * (pidx = -1, angle = params + offset), then shift occurrence g only. */
  for (int g = 0; g < ng && rc == OR_OK; g++) {
    if (pidx[g] < 0) continue;
    for (int h = 0; h < ng; h++) {
      pid[h] = -1;
      ang[h] = angles[h] + (pidx[h] >= 0 ? params[pidx[h]] : 0.0);
    }
    double base = ang[g], fp, fm, d;
    ang[g] = base + OR_PI / 2;
    rc |= energy(n, kinds, qubits, pid, ang, mats, ng, NULL, 0, paulis, coeffs, nt, psi, &fp);
    ang[g] = base - OR_PI / 2;
    rc |= energy(n, kinds, qubits, pid, ang, mats, ng, NULL, 0, paulis, coeffs, nt, psi, &fm);
    if (shift_rule(kinds[g]) == 1) {
      d = 0.5 * (fp - fm);
    } else {
      double f3p, f3m;
      ang[g] = base + 3 * OR_PI / 2;
      rc |= energy(n, kinds, qubits, pid, ang, mats, ng, NULL, 0, paulis, coeffs, nt, psi, &f3p);
      ang[g] = base - 3 * OR_PI / 2;
      rc |= energy(n, kinds, qubits, pid, ang, mats, ng, NULL, 0, paulis, coeffs, nt, psi, &f3m);
      double r2 = sqrt(2.0);
      double d1 = (r2 + 1) / (4 * r2), d2 = (r2 - 1) / (4 * r2);
      d = d1 * (fp - fm) - d2 * (f3p - f3m);
    }
    grad[pidx[g]] += d;
  }
  free(psi); free(ang); free(pid);
  return rc;
}

/* Central finite differences: (E(theta + h e_i) - E(theta - h e_i)) / (2h)
 * for the parameters listed in `which` (nw of them). */
int or_finite_diff(int n, const int* kinds, const int* qubits, const int* pidx,
                   const double* angles, const double* mats, int ng,
                   const double* params, int np, const char* paulis,
                   const double* coeffs, int nt, double h, const int* which, int nw,
                   double* grad) {
  cplx* psi = (cplx*)malloc((1ull << n) * sizeof(cplx));
  double* p = (double*)malloc((np > 0 ? np : 1) * sizeof(double));
  if (!psi || !p) { free(psi); free(p); return OR_EINVAL; }
  int rc = OR_OK;
  for (int w = 0; w < nw && rc == OR_OK; w++) {
    int i = which[w];
    double fp, fm;
    memcpy(p, params, np * sizeof(double));
    p[i] = params[i] + h;
    rc |= energy(n, kinds, qubits, pidx, angles, mats, ng, p, np, paulis, coeffs, nt, psi, &fp);
    p[i] = params[i] - h;
    rc |= energy(n, kinds, qubits, pidx, angles, mats, ng, p, np, paulis, coeffs, nt, psi, &fm);
    grad[w] = (fp - fm) / (2 * h);
  }
  free(psi); free(p);
  return rc;
}

static uint64_t bitrev(uint64_t x, int n) {
  uint64_t r = 0;
  for (int b = 0; b < n; b++)
    if ((x >> b) & 1) r |= 1ull << (n - 1 - b);
  return r;
}

/* Alg. 2: QFT = InverseFFT(psi) / sqrt(N), with
 * QFT|x> = N^{-1/2} sum_k exp(+2 pi i x k / N)|k>.  A plain iterative
 * radix-2 Cooley-Tukey (bit reversal, then log2 N butterfly stages).  The
 * twiddle of stage length L and offset j is exp(sign 2 pi i j / L),
 * evaluated directly (no recurrence).  inverse=1 gives the inverse QFT
 * (sign -). */
int or_qft_fft(double* state, int n, int inverse) {
  cplx* a = (cplx*)state;
  uint64_t N = 1ull << n;
  double sign = inverse ? -1.0 : 1.0;
  for (uint64_t i = 0; i < N; i++) {
    uint64_t j = bitrev(i, n);
    if (i < j) { cplx t = a[i]; a[i] = a[j]; a[j] = t; }
  }
  /* twiddles of the longest stage, w[j] = exp(sign 2 pi i j / N); a stage of
   * length L uses w[j N / L] = exp(sign 2 pi i j / L) exactly (the argument
   * differs only by a power-of-two scaling). */
  uint64_t half = N / 2 > 0 ? N / 2 : 1;
  cplx* w = (cplx*)malloc(half * sizeof(cplx));
  if (!w) return OR_EINVAL;
  for (uint64_t j = 0; j < half; j++) w[j] = cexp(I * sign * 2.0 * OR_PI * (double)j / (double)N);
  for (uint64_t L = 2; L <= N; L <<= 1) {
    uint64_t h = L / 2, step = N / L;
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < (int64_t)N; s += (int64_t)L) {
      for (uint64_t j = 0; j < h; j++) {
        cplx u = a[s + j], v = a[s + j + h] * w[j * step];
        a[s + j] = u + v;
        a[s + j + h] = u - v;
      }
    }
  }
  free(w);
  double r = 1.0 / sqrt((double)N);
  for (uint64_t i = 0; i < N; i++) a[i] *= r;
  return OR_OK;
}

/* Alg. 3: gate-sequence QFT on the dense state. */
int or_qft_gates(double* state, int n) {
  double M[2 * 16];
  for (int i = 0; i < n; i++) {
    int q = i;
    or_gate_matrix(OG_H, 0, NULL, M);
    or_apply_matrix(state, n, &q, 1, M);
    for (int j = i + 1; j < n; j++) {
      int qq[2] = {i, j};
      or_gate_matrix(OG_CP, OR_PI / ldexp(1.0, j - i), NULL, M);
      or_apply_matrix(state, n, qq, 2, M);
    }
  }
  for (int i = 0; i < n / 2; i++) {
    int qq[2] = {i, n - 1 - i};
    or_gate_matrix(OG_SWAP, 0, NULL, M);
    or_apply_matrix(state, n, qq, 2, M);
  }
  return OR_OK;
}

/* One QFT output amplitude by its definition: sum_x psi[x] e^{2 pi i x k/N}
 * / sqrt(N), with the phase index (x k mod N) formed exactly in integers. */
int or_qft_amplitude(const double* state, int n, uint64_t k, double* out) {
  const cplx* psi = (const cplx*)state;
  uint64_t N = 1ull << n, mask = N - 1;
  double re = 0, im = 0;
#pragma omp parallel for reduction(+ : re, im) schedule(static)
  for (int64_t x = 0; x < (int64_t)N; x++) {
    uint64_t r = ((uint64_t)x * k) & mask;
    cplx v = psi[x] * cexp(I * 2.0 * OR_PI * (double)r / (double)N);
    re += creal(v);
    im += cimag(v);
  }
  double s = 1.0 / sqrt((double)N);
  out[0] = re * s;
  out[1] = im * s;
  return OR_OK;
}

/* exp(-i theta P) psi = cos(theta) psi - i sin(theta) P psi for a Pauli
 * string P (P^2 = I). */
static void pauli_exp(cplx* psi, cplx* work, int n, const char* s, double theta) {
  uint64_t N = 1ull << n;
  memcpy(work, psi, N * sizeof(cplx));
  for (int q = 0; q < n; q++) {
    int p = s[q] == 'X' ? 1 : s[q] == 'Y' ? 2 : s[q] == 'Z' ? 3 : 0;
    if (p == 0) continue;
    cplx M[4];
    pauli2(p, M);
    or_apply_matrix((double*)work, n, &q, 1, (const double*)M);
  }
  double c = cos(theta), sn = sin(theta);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < (int64_t)N; i++) psi[i] = c * psi[i] - I * sn * work[i];
}

/* First-order Trotter-Suzuki evolution (Eq. trotter) of
 *   H(t) = sum_k c_k P_k + h(t) sum_f d_f F_f,   h(t) = A sin(omega t),
 * for `steps` steps of dt: step j applies exp(-i c_k P_k dt) for every
 * static term in order, then exp(-i h(t_j) d_f F_f dt) for every field term
 * in order, with t_j = j dt. */
int or_trotter(double* state, int n, const char* paulis, const double* coeffs, int nt,
               const char* fpaulis, const double* fcoeffs, int nf, double A,
               double omega, double dt, int steps) {
  uint64_t N = 1ull << n;
  cplx* work = (cplx*)malloc(N * sizeof(cplx));
  if (!work) return OR_EINVAL;
  cplx* psi = (cplx*)state;
  for (int j = 0; j < steps; j++) {
    double tj = j * dt, h = A * sin(omega * tj);
    for (int k = 0; k < nt; k++)
      pauli_exp(psi, work, n, paulis + (size_t)k * n, coeffs[k] * dt);
    for (int f = 0; f < nf; f++)
      pauli_exp(psi, work, n, fpaulis + (size_t)f * n, h * fcoeffs[f] * dt);
  }
  free(work);
  return OR_OK;
}

/* Norm sum |psi_i|^2 (used by invariants in the tests). */
double or_norm2(const double* state, int n) {
  const cplx* psi = (const cplx*)state;
  uint64_t N = 1ull << n;
  double s = 0;
  for (uint64_t i = 0; i < N; i++) s += creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
  return s;
}
