"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and bench.py.

This module holds circuit and Hamiltonian *descriptions* (gate lists, Pauli
strings) and seeded random draws only: it performs none of the simulation
arithmetic, and imports neither the oracle nor the CUDA library.

Conventions used by every description here:
  * a gate is ``Gate(name, qubits, param, angle, mat)``; the angle a
    parametrised gate uses is ``params[param] + angle`` (param >= 0) or the
    fixed ``angle`` (param = -1); ``mat`` is a row-major complex matrix for the
    ``U1`` (2x2) and ``U2`` (4x4) gates, else None;
  * the first listed qubit of a controlled gate is its control;
  * a Pauli sum is a list of ``(coeff, string)`` where character q of the
    string acts on qubit q (qubit 0 is the most significant bit of an
    amplitude index, Alg. 1);
  * random draws use numpy's PCG64 ``default_rng(seed)``.
"""
from collections import namedtuple

import numpy as np

Gate = namedtuple("Gate", "name qubits param angle mat")

PI = np.pi


def G(name, *qubits, param=-1, angle=0.0, mat=None):
    return Gate(name, tuple(int(q) for q in qubits), int(param), float(angle), mat)


# ----------------------------------------------------------------- circuits

def hea(n, depth, entangler="ladder", rotations=("RY", "RZ")):
    """Hardware-efficient ansatz (Sec. VI-B): per layer one rotation of each
    kind on every qubit (all RY, then all RZ), then a CNOT ladder
    0->1->...->n-1 (``ring`` appends n-1->0).  Parameter index of rotation r
    on qubit q in layer l is l*len(rotations)*n + r*n + q.
    Returns (gates, number_of_parameters)."""
    gates, p = [], 0
    for _ in range(depth):
        for r in rotations:
            for q in range(n):
                gates.append(G(r, q, param=p))
                p += 1
        if n > 1:
            for q in range(n - 1):
                gates.append(G("CNOT", q, q + 1))
            if entangler == "ring":
                gates.append(G("CNOT", n - 1, 0))
    return gates, p


def appd_circuit():
    """Edge-case circuit of App. D: RX(t0) on q0, RY(t1) on q1, RZ(t2) on q0,
    CNOT(0 -> 1), CRY(t3) with control q1 and target q0; observable Z0."""
    gates = [
        G("RX", 0, param=0),
        G("RY", 1, param=1),
        G("RZ", 0, param=2),
        G("CNOT", 0, 1),
        G("CRY", 1, 0, param=3),
    ]
    return gates, 4, [(1.0, "ZI")]


APPD_ANGLE_SETS = {
    "normal": [0.5, 0.3, 0.2, 0.1],
    "large": [10.0, 5.0, 3.0, 2.0],
    "near_zero": [1e-8, 1e-7, 1e-6, 1e-5],
    "pi_2": [PI / 2] * 4,
    "pi": [PI] * 4,
}


def random_circuit(n, ngates, rng, kinds=None, parametrised=True):
    """A random gate list over a mixed gate set, for parity tests.  Every
    angle-taking gate gets its own parameter when ``parametrised``."""
    one = ["H", "X", "Y", "Z", "S", "SDG", "T", "TDG", "RX", "RY", "RZ", "P", "U1"]
    two = ["CNOT", "CY", "CZ", "CP", "SWAP", "CRX", "CRY", "CRZ", "RXX", "RYY", "RZZ", "U2"]
    three = ["CCX"]
    pool = kinds or (one + (two if n >= 2 else []) + (three if n >= 3 else []))
    angle_kinds = {"RX", "RY", "RZ", "P", "CP", "CRX", "CRY", "CRZ", "RXX", "RYY", "RZZ"}
    gates, p = [], 0
    for _ in range(ngates):
        name = pool[rng.integers(len(pool))]
        k = 3 if name == "CCX" else 2 if name in two else 1
        qs = rng.choice(n, size=k, replace=False)
        mat = None
        if name in ("U1", "U2"):
            d = 2 if name == "U1" else 4
            z = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
            q_, r_ = np.linalg.qr(z)
            mat = q_ * (np.diag(r_) / np.abs(np.diag(r_)))
        if name in angle_kinds:
            if parametrised:
                gates.append(G(name, *qs, param=p, angle=float(rng.uniform(-0.3, 0.3))))
                p += 1
            else:
                gates.append(G(name, *qs, angle=float(rng.uniform(-PI, PI))))
        else:
            gates.append(G(name, *qs, mat=mat))
    return gates, p


# -------------------------------------------------------------- hamiltonians

def heisenberg(n, J=(1.0, 0.5, 0.25), ring=False):
    """XYZ Heisenberg couplings sum_<ij> (Jx XiXj + Jy YiYj + Jz ZiZj) on the
    open chain (pairs (i, i+1)), plus (n-1, 0) for a ring.  Term order: per
    pair XX, YY, ZZ."""
    pairs = [(i, i + 1) for i in range(n - 1)]
    if ring and n > 2:
        pairs.append((n - 1, 0))
    terms = []
    for a, b in pairs:
        for j, ch in zip(J, "XYZ"):
            s = ["I"] * n
            s[a] = ch
            s[b] = ch
            terms.append((float(j), "".join(s)))
    return terms


def z_field(n, coeff=1.0):
    """sum_i coeff Z_i."""
    out = []
    for i in range(n):
        s = ["I"] * n
        s[i] = "Z"
        out.append((float(coeff), "".join(s)))
    return out


def random_pauli_sum(n, nterms, rng, kmin=2, kmax=4):
    """nterms random k-local Pauli strings: k ~ U{kmin..min(kmax, n)}, k
    distinct qubits, each operator ~ U{X, Y, Z}; coefficients ~ N(0, 1)."""
    terms = []
    for _ in range(nterms):
        k = int(rng.integers(kmin, min(kmax, n) + 1))
        qs = rng.choice(n, size=k, replace=False)
        s = ["I"] * n
        for q in qs:
            s[q] = "XYZ"[rng.integers(3)]
        terms.append((float(rng.standard_normal()), "".join(s)))
    return terms


# ------------------------------------------------------------------- draws

def angles(count, seed):
    """count angles uniform in [-pi, pi)."""
    return np.random.default_rng(seed).uniform(-PI, PI, count)


def gaussian_state(n, seed):
    """2^n i.i.d. complex Gaussian amplitudes (re, im ~ N(0, 1)), L2-normalised."""
    rng = np.random.default_rng(seed)
    N = 1 << n
    psi = np.empty(N, np.complex128)
    v = psi.view(np.float64)
    chunk = 1 << 24
    for s in range(0, 2 * N, chunk):
        v[s: s + chunk] = rng.standard_normal(min(chunk, 2 * N - s))
    psi /= np.sqrt(np.vdot(psi, psi).real)
    return psi


def basis_index(n, seed):
    return int(np.random.default_rng(seed).integers(0, 1 << n))


# ------------------------------------------------------------------ configs
# Seeded workloads named by what they are, with their sizes.

def vqe_chain(n=10, depth=4, seed=1):
    """HEA depth `depth` (RY, RZ, CNOT ladder) on n qubits, 2*n*depth angles
    U[-pi, pi) from `seed`, open-chain XYZ Heisenberg (1.0, 0.5, 0.25)."""
    gates, P = hea(n, depth, "ladder")
    return gates, angles(P, seed), heisenberg(n)


def vqe_ring(n=16, depth=8, seed=3):
    """HEA with a CNOT ring, XYZ Heisenberg ring."""
    gates, P = hea(n, depth, "ring")
    return gates, angles(P, seed), heisenberg(n, ring=True)


def uneven_batch(count=64, seed=4, nmin=8, nmax=20, dmin=2, dmax=12, nterms=50):
    """`count` instances: n ~ U{nmin..nmax}, depth ~ U{dmin..dmax}, ring HEA,
    random 2-4-local Pauli sum of `nterms` terms; angles U[-pi, pi)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.integers(nmin, nmax + 1))
        d = int(rng.integers(dmin, dmax + 1))
        gates, P = hea(n, d, "ring")
        th = rng.uniform(-PI, PI, P)
        terms = random_pauli_sum(n, nterms, rng)
        out.append((n, gates, th, terms))
    return out


def xyz_trotter(n, J=(1.0, 1.0, 1.0)):
    """Time-dependent XYZ model of Sec. VII-A:
    H(t) = -sum(Jx XX + Jy YY + Jz ZZ) - h(t) sum Z,  h(t) = A sin(omega t),
    A = 2, omega = 1, initial state |1...1>.  Returns (static terms, field
    terms with unit h, A, omega, initial basis index)."""
    static = [(-c, s) for c, s in heisenberg(n, J)]
    field = z_field(n, -1.0)
    return static, field, 2.0, 1.0, (1 << n) - 1


def serve_requests(count, seed=6, rate=None, nmin=8, nmax=28, dmin=2, dmax=20):
    """Poisson request stream: arrival gaps ~ Exp(rate) (seconds), kind 50/50
    energy-only / energy+gradient, n ~ U{nmin..nmax}, depth ~ U{dmin..dmax}
    (ladder HEA), Hamiltonian 50/50 Heisenberg chain / random 50-term."""
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    for i in range(count):
        if rate:
            t += float(rng.exponential(1.0 / rate))
        n = int(rng.integers(nmin, nmax + 1))
        d = int(rng.integers(dmin, dmax + 1))
        grad = bool(rng.integers(2))
        gates, P = hea(n, d, "ladder")
        th = rng.uniform(-PI, PI, P)
        terms = heisenberg(n) if rng.integers(2) == 0 else random_pauli_sum(n, 50, rng)
        reqs.append(dict(id=i, t=t, n=n, depth=d, grad=grad, gates=gates, params=th, terms=terms))
    return reqs
