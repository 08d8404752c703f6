// Host-side check of the tile-pass scheduler (no GPU): random circuits are
// lowered and scheduled with small tiles (many passes), with and without
// phase sinking, and the scheduled ops are applied on the CPU with the
// semantics the pass kernels give them (global bit positions; the merged
// phase op's AND and parity factors, the dyadic op's integer weights).  The
// result must equal a plain gate-by-gate simulation of the circuit (each
// gate's 2x2 matrix, or its permutation / phase on the amplitudes it moves)
// to 1e-12, and sinking must never leave more phase ops than it found.
//
// Usage: sched_interp TRIALS SEED; prints "ok ..." and exits 0 on success.
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>
#include <vector>

#include "lq_internal.h"

using namespace lq;
using cplx = std::complex<double>;

static int popc(uint64_t v) { return __builtin_popcountll(v); }
static double as_double(uint64_t u) {
  double d;
  std::memcpy(&d, &u, sizeof d);
  return d;
}
static cplx ipow(int k) {
  static const cplx t[4] = {cplx(1, 0), cplx(0, 1), cplx(-1, 0), cplx(0, -1)};
  return t[k & 3];
}

// One lowered op on the whole state.
static bool apply_lop(std::vector<cplx>& s, int n, const LOp& o) {
  const uint64_t N = 1ull << n;
  auto cond = [&](uint64_t i) { return (i & o.cm) == o.cv; };
  switch (o.type) {
    case OP_PAULI: {   // out_i = alpha psi_i + beta w_i psi_{i^x}
      std::vector<cplx> t = s;
      const int pm = o.mode & 3, k0 = (o.mode >> 2) & 3;
      cplx al = 0, be = 1;
      if (pm == PM_TAN) { al = 1; be = o.a; }
      else if (pm == PM_COT) { al = o.a; be = 1; }
      else if (pm == PM_GEN) { al = o.a; be = o.b; }
      for (uint64_t i = 0; i < N; i++) {
        if (!cond(i)) continue;
        const uint64_t j = i ^ o.x;
        const cplx w = ipow(k0) * ((popc(j & o.z) & 1) ? -1.0 : 1.0);
        t[i] = al * s[i] + be * w * s[j];
      }
      s.swap(t);
      return true;
    }
    case OP_H: {
      const uint64_t b = 1ull << o.g0;
      for (uint64_t i = 0; i < N; i++)
        if (!(i & b) && cond(i)) {
          const cplx a = s[i], c = s[i | b];
          s[i] = a + c;
          s[i | b] = a - c;
        }
      return true;
    }
    case OP_SWAP: {
      const uint64_t a = 1ull << o.g0, b = 1ull << o.g1;
      for (uint64_t i = 0; i < N; i++)
        if ((i & a) && !(i & b) && cond(i)) std::swap(s[i], s[i ^ a ^ b]);
      return true;
    }
    case OP_PHASE:
      for (uint64_t i = 0; i < N; i++) if (cond(i)) s[i] *= cplx(o.a, o.b);
      return true;
    case OP_SIGN:
      for (uint64_t i = 0; i < N; i++) if (cond(i)) s[i] = -s[i];
      return true;
    case OP_MULI:
      for (uint64_t i = 0; i < N; i++) if (cond(i)) s[i] *= ipow(o.mode);
      return true;
    case OP_PARITY:
      for (uint64_t i = 0; i < N; i++)
        if (cond(i) && (popc(i & o.z) & 1)) s[i] *= cplx(o.a, o.b);
      return true;
    case OP_SCALE:
      for (uint64_t i = 0; i < N; i++) s[i] *= cplx(o.a, (o.mode & 1) ? 0.0 : o.b);
      return true;
    case OP_LPHASE: {   // factors: (cm, cv, re bits, im bits, gate)
      const std::size_t nf = o.dfac.size() / 5;
      for (uint64_t i = 0; i < N; i++) {
        if (!cond(i)) continue;
        cplx w = 1;
        for (std::size_t f = 0; f < nf; f++) {
          const uint64_t cm = o.dfac[5 * f], cv = o.dfac[5 * f + 1];
          const bool on = (cv & kLphaseParity) ? (popc(i & cm) & 1) != 0 : (i & cm) == cv;
          if (on) w *= cplx(as_double(o.dfac[5 * f + 2]), as_double(o.dfac[5 * f + 3]));
        }
        s[i] *= w;
      }
      return true;
    }
    case OP_DPHASE: {   // factors: (cm, cv, weight); phase exp(2 pi i E / 2^34)
      const std::size_t nf = o.dfac.size() / 3;
      for (uint64_t i = 0; i < N; i++) {
        if (!cond(i)) continue;
        unsigned long long E = 0;
        for (std::size_t f = 0; f < nf; f++)
          if ((i & o.dfac[3 * f]) == o.dfac[3 * f + 1]) E += o.dfac[3 * f + 2];
        E &= (1ull << DYADIC_BITS) - 1;
        s[i] *= std::polar(1.0, 2 * M_PI * (double)E / std::ldexp(1.0, DYADIC_BITS));
      }
      return true;
    }
    default:
      std::printf("op type %d not interpreted\n", o.type);
      return false;
  }
}

// One gate of the circuit, by its definition.
static void apply_gate(std::vector<cplx>& s, int n, const lq_gate& g, double th) {
  const uint64_t N = 1ull << n;
  auto bit = [&](int q) { return 1ull << (n - 1 - q); };
  const double c = std::cos(th / 2), sn = std::sin(th / 2), r = 1 / std::sqrt(2.0);
  cplx M[4];
  bool one = true;
  switch (g.kind) {
    case LQ_H: M[0] = M[1] = M[2] = r; M[3] = -r; break;
    case LQ_RX: M[0] = c; M[1] = cplx(0, -sn); M[2] = cplx(0, -sn); M[3] = c; break;
    case LQ_RY: M[0] = c; M[1] = -sn; M[2] = sn; M[3] = c; break;
    case LQ_RZ: M[0] = std::polar(1.0, -th / 2); M[1] = M[2] = 0; M[3] = std::polar(1.0, th / 2); break;
    case LQ_P: M[0] = 1; M[1] = M[2] = 0; M[3] = std::polar(1.0, th); break;
    case LQ_T: M[0] = 1; M[1] = M[2] = 0; M[3] = std::polar(1.0, M_PI / 4); break;
    default: one = false;
  }
  if (one) {
    const uint64_t b = bit(g.qubits[0]);
    for (uint64_t i = 0; i < N; i++)
      if (!(i & b)) {
        const cplx a = s[i], d = s[i | b];
        s[i] = M[0] * a + M[1] * d;
        s[i | b] = M[2] * a + M[3] * d;
      }
    return;
  }
  const uint64_t cb = bit(g.qubits[0]), tb = bit(g.qubits[1]);
  for (uint64_t i = 0; i < N; i++) {
    if (g.kind == LQ_CNOT && (i & cb) && !(i & tb)) {
      std::swap(s[i], s[i | tb]);
    } else if (g.kind == LQ_CY && (i & cb) && !(i & tb)) {
      const cplx a = s[i], d = s[i | tb];
      s[i] = cplx(0, -1) * d;
      s[i | tb] = cplx(0, 1) * a;
    } else if (g.kind == LQ_SWAP && (i & cb) && !(i & tb)) {
      std::swap(s[i], s[i ^ cb ^ tb]);
    } else if (g.kind == LQ_CZ && (i & cb) && (i & tb)) {
      s[i] = -s[i];
    } else if (g.kind == LQ_CP && (i & cb) && (i & tb)) {
      s[i] *= std::polar(1.0, th);
    }
  }
}

static lq_gate make_gate(int kind, int q0, int q1, int param) {
  lq_gate x;
  std::memset(&x, 0, sizeof x);
  x.kind = kind;
  x.qubits[0] = q0;
  x.qubits[1] = q1;
  x.qubits[2] = -1;
  x.param = param;
  return x;
}

int main(int argc, char** argv) {
  const int trials = argc > 1 ? std::atoi(argv[1]) : 200;
  std::mt19937_64 rng(argc > 2 ? std::strtoull(argv[2], nullptr, 10) : 1);
  const int kinds[] = {LQ_RY, LQ_RZ, LQ_RZ, LQ_RZ, LQ_P, LQ_T, LQ_CNOT, LQ_CNOT, LQ_CNOT,
                       LQ_CY, LQ_SWAP, LQ_CZ, LQ_H, LQ_RX, LQ_CP};
  double worst = 0;
  int fewer = 0;
  for (int t = 0; t < trials; t++) {
    const int n = 8 + (int)(rng() % 5), k = 4 + (int)(rng() % 4);   // small states: sinking is forced below
    int m = 1 + (int)(rng() % 3);
    if (m > k - 2) m = k - 2;
    std::vector<lq_gate> g;
    std::vector<double> p;
    auto angle = [&]() { return (double)(rng() % 20000) / 2000.0 - 5.0; };
    if (t % 6 == 1) {   // Alg. 3 (H, then CP(pi/2^(j-i)) from i to j > i), forward or reversed
      std::vector<lq_gate> f;
      for (int i = 0; i < n; i++) {
        f.push_back(make_gate(LQ_H, i, -1, -1));
        for (int j = i + 1; j < n; j++) {
          lq_gate c = make_gate(LQ_CP, i, j, -1);
          c.angle = M_PI / std::ldexp(1.0, j - i);
          f.push_back(c);
        }
      }
      if (t % 12 == 7)
        for (int i = (int)f.size() - 1; i >= 0; i--) {
          lq_gate c = f[i];
          c.angle = -c.angle;
          g.push_back(c);
        }
      else
        g = f;
    } else if (t % 3 == 0) {   // hardware-efficient layers: RY, RZ on every qubit, CNOT ladder or ring
      const int depth = 1 + (int)(rng() % 3);
      for (int l = 0; l < depth; l++) {
        for (int r = 0; r < 2; r++)
          for (int q = 0; q < n; q++) {
            g.push_back(make_gate(r ? LQ_RZ : LQ_RY, q, -1, (int)p.size()));
            p.push_back(angle());
          }
        for (int q = 0; q + 1 < n + (t % 2); q++) g.push_back(make_gate(LQ_CNOT, q, (q + 1) % n, -1));
      }
    } else {
      const int ng = 20 + (int)(rng() % 60);
      for (int i = 0; i < ng; i++) {
        const int kind = kinds[rng() % (sizeof kinds / sizeof kinds[0])];
        const int q0 = (int)(rng() % n);
        int q1 = -1;
        if (kind == LQ_CNOT || kind == LQ_CY || kind == LQ_SWAP || kind == LQ_CZ || kind == LQ_CP)
          do q1 = (int)(rng() % n); while (q1 == q0);
        const bool ang = gate_takes_angle(kind);
        g.push_back(make_gate(kind, q0, q1, ang ? (int)p.size() : -1));
        if (ang) p.push_back(angle());
      }
    }
    const uint64_t N = 1ull << n;
    std::vector<cplx> ref(N, 0.0);
    ref[0] = 1;
    for (const lq_gate& x : g) apply_gate(ref, n, x, x.param >= 0 ? p[x.param] : x.angle);
    int phases[2] = {0, 0};
    for (int sink = 0; sink < 2; sink++) {
      LOp* ops = nullptr;
      std::size_t nops = 0;
      double zr, zi;
      if (lower_circuit(n, g.data(), (int)g.size(), p.data(), (int)p.size(), &ops, &nops, &zr,
                        &zi, true)) {
        std::printf("lowering failed: %s\n", lq_last_error());
        return 1;
      }
      ScheduleOptions opt;
      opt.lphase_table = true;
      opt.sink_phases = sink != 0;
      opt.sink_min_qubits = 0;
      opt.k = k;
      opt.m = m;
      opt.max_hi = PASS_HI_BITS;
      Schedule S;
      if (schedule_ops(n, ops, nops, zr, zi, opt, S)) {
        std::printf("scheduling failed: %s\n", lq_last_error());
        return 1;
      }
      delete[] ops;
      std::vector<cplx> st(N, 0.0);
      st[0] = 1;
      for (int ps = 0; ps < S.npasses; ps++)
        for (const LOp& o : S.pass_ops[ps]) {
          if (!apply_lop(st, n, o)) return 1;
          phases[sink] += o.type == OP_LPHASE || o.type == OP_PHASE || o.type == OP_PARITY;
        }
      double err = 0;
      for (uint64_t i = 0; i < N; i++) err = std::max(err, std::abs(st[i] - ref[i]));
      worst = std::max(worst, err);
      if (err > 1e-12) {
        std::printf("trial %d (sinking %d, n=%d k=%d m=%d, %d passes): error %.3g\n", t, sink, n,
                    k, m, S.npasses, err);
        return 1;
      }
    }
    if (phases[1] > phases[0]) {
      std::printf("trial %d: sinking left %d phase ops, %d before\n", t, phases[1], phases[0]);
      return 1;
    }
    fewer += phases[1] < phases[0];
  }
  std::printf("ok %d trials, worst error %.3g, fewer phase ops in %d\n", trials, worst, fewer);
  return 0;
}
