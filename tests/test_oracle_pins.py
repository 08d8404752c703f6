"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here retypes the oracle's formulas: gate matrices are pinned by
matrix exponentials of their generators (scipy.linalg.expm) and by algebraic
identities; the gate-application loop by an independent numpy tensor
contraction; the index convention by the paper's worked examples
(App. A, App. B, App. C); <H> by dense Kronecker-product Hamiltonians and
closed forms; the QFT by its closed form on basis states and by numpy's FFT;
the parameter-shift gradient by the App. D table, closed forms and central
finite differences; Trotter evolution by dense products of exponentials.
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")
R2 = 1 / np.sqrt(2)
PX = np.array([[0, 1], [1, 0]], complex)
PY = np.array([[0, -1j], [1j, 0]], complex)
PZ = np.array([[1, 0], [0, -1]], complex)
I2 = np.eye(2)
P1 = np.array([[0, 0], [0, 1]], complex)  # |1><1|
PAULI = {"I": I2, "X": PX, "Y": PY, "Z": PZ}


# ------------------------------------------------------------ helpers (test)

def read_golden(name):
    rows = {}
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            rows[key] = vals
    return rows


def tensor_apply(psi, n, qubits, M):
    """Independent application route: view psi as an n-axis tensor (axis q
    = qubit q, C order makes axis 0 the most significant index bit), move
    the gate's axes to the front and contract with M."""
    k = len(qubits)
    t = psi.reshape([2] * n)
    t = np.moveaxis(t, list(qubits), list(range(k)))
    shp = t.shape
    t = (M @ t.reshape(1 << k, -1)).reshape(shp)
    t = np.moveaxis(t, list(range(k)), list(qubits))
    return np.ascontiguousarray(t.reshape(-1))


def dense_pauli(s):
    m = np.array([[1.0 + 0j]])
    for ch in s:
        m = np.kron(m, PAULI[ch])
    return m


def dense_h(terms):
    return sum(c * dense_pauli(s) for c, s in terms)


def rand_state(n, seed):
    return W.gaussian_state(n, seed)


# ------------------------------------------------------- worked examples

def test_appA_cnot_example():
    g = read_golden("appA_cnot.txt")
    n = int(g["n"][0])
    c, t = int(g["gate"][1]), int(g["gate"][2])
    psi = np.array([float(v) for v in g["in"]], complex) * R2
    want = np.array([float(v) for v in g["out"]], complex) * R2
    np.testing.assert_array_equal(oracle.cnot_alg1(psi.copy(), n, c, t), want)
    out = oracle.apply_circuit(psi.copy(), n, [W.G("CNOT", c, t)])
    np.testing.assert_allclose(out, want, atol=0)


def test_appB_toffoli_example():
    g = read_golden("appB_toffoli.txt")
    n = int(g["n"][0])
    c1, c2, t = (int(v) for v in g["gate"][1:4])
    m = [int(v) for v in g["masks"]]
    # masks of Alg. 4 for this example: 2^(n-1-q)
    assert [1 << (n - 1 - q) for q in (c1, c2, t)] == m[:3] and (m[0] | m[1]) == m[3]
    psi = np.array([float(v) for v in g["in"]], complex) * R2
    want = np.array([float(v) for v in g["out"]], complex) * R2
    np.testing.assert_array_equal(oracle.toffoli_alg4(psi.copy(), n, c1, c2, t), want)
    out = oracle.apply_circuit(psi.copy(), n, [W.G("CCX", c1, c2, t)])
    np.testing.assert_allclose(out, want, atol=0)


def test_appC_hadamard_example():
    g = read_golden("appC_hadamard.txt")
    n = int(g["n"][0])
    psi = oracle.basis_state(n, 0)
    out = oracle.apply_circuit(psi, n, [W.G("H", int(g["gate"][1]))])
    want = np.array([float(v) for v in g["out"]], complex) * R2
    np.testing.assert_allclose(out, want, atol=1e-16)


@pytest.mark.parametrize("n", [3, 5])
def test_alg1_alg4_match_matrix_route(n):
    for c in range(n):
        for t in range(n):
            if c == t:
                continue
            psi = rand_state(n, 10 + c * n + t)
            a = oracle.cnot_alg1(psi.copy(), n, c, t)
            b = oracle.apply_circuit(psi.copy(), n, [W.G("CNOT", c, t)])
            np.testing.assert_array_equal(a, b)
            for c2 in range(n):
                if c2 in (c, t):
                    continue
                a = oracle.toffoli_alg4(psi.copy(), n, c, c2, t)
                b = oracle.apply_circuit(psi.copy(), n, [W.G("CCX", c, c2, t)])
                np.testing.assert_array_equal(a, b)


# ------------------------------------------------------------ gate matrices

@pytest.mark.parametrize("theta", [0.0, 0.37, -2.1, np.pi, 7.5])
def test_rotation_matrices_are_exponentials(theta):
    # R_P(theta) = exp(-i theta sigma_P / 2), Sec. III-A
    for name, s in (("RX", PX), ("RY", PY), ("RZ", PZ)):
        np.testing.assert_allclose(oracle.gate_matrix(name, theta), sla.expm(-0.5j * theta * s), atol=1e-14)
    for name, s in (("RXX", PX), ("RYY", PY), ("RZZ", PZ)):
        np.testing.assert_allclose(oracle.gate_matrix(name, theta), sla.expm(-0.5j * theta * np.kron(s, s)), atol=1e-14)
    # phase gates: exp(i phi |1><1|) and exp(i phi |11><11|)
    np.testing.assert_allclose(oracle.gate_matrix("P", theta), sla.expm(1j * theta * P1), atol=1e-14)
    np.testing.assert_allclose(oracle.gate_matrix("CP", theta), sla.expm(1j * theta * np.kron(P1, P1)), atol=1e-14)
    # controlled rotations: exp(-i theta/2 |1><1| (x) sigma) on (control, target)
    for name, s in (("CRX", PX), ("CRY", PY), ("CRZ", PZ)):
        np.testing.assert_allclose(oracle.gate_matrix(name, theta), sla.expm(-0.5j * theta * np.kron(P1, s)), atol=1e-14)


def test_fixed_gate_identities():
    m = oracle.gate_matrix
    H, X, Y, Z = m("H"), m("X"), m("Y"), m("Z")
    np.testing.assert_allclose(H @ H, I2, atol=1e-15)
    np.testing.assert_allclose(H @ X @ H, Z, atol=1e-15)
    np.testing.assert_allclose(H @ Z @ H, X, atol=1e-15)
    np.testing.assert_allclose(X @ Y, 1j * Z, atol=0)  # Pauli algebra fixes Y's sign
    np.testing.assert_allclose(m("S") @ m("S"), Z, atol=0)
    np.testing.assert_allclose(m("T") @ m("T"), m("S"), atol=1e-15)
    np.testing.assert_allclose(m("T") @ m("TDG"), I2, atol=1e-15)
    np.testing.assert_allclose(m("S") @ m("SDG"), I2, atol=0)
    IH = np.kron(I2, H)
    np.testing.assert_allclose(IH @ m("CNOT") @ IH, m("CZ"), atol=1e-15)
    IS, ISd = np.kron(I2, m("S")), np.kron(I2, m("SDG"))
    np.testing.assert_allclose(IS @ m("CNOT") @ ISd, m("CY"), atol=1e-15)
    np.testing.assert_allclose(m("CP", np.pi), m("CZ"), atol=1e-15)
    # SWAP = CNOT(a,b) CNOT(b,a) CNOT(a,b) on a random 2-qubit state
    psi = rand_state(2, 3)
    a = oracle.apply_circuit(psi.copy(), 2, [W.G("SWAP", 0, 1)])
    b = oracle.apply_circuit(psi.copy(), 2, [W.G("CNOT", 0, 1), W.G("CNOT", 1, 0), W.G("CNOT", 0, 1)])
    np.testing.assert_allclose(a, b, atol=0)
    np.testing.assert_allclose(a, psi[[0, 2, 1, 3]], atol=0)


def test_all_gate_matrices_unitary():
    rng = np.random.default_rng(0)
    for name in oracle.GATE_CODES:
        mat = None
        if name in ("U1", "U2"):
            d = 2 if name == "U1" else 4
            q, r = np.linalg.qr(rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d)))
            mat = q
        M = oracle.gate_matrix(name, 0.731, mat)
        np.testing.assert_allclose(M.conj().T @ M, np.eye(M.shape[0]), atol=1e-14)
        if mat is not None:
            np.testing.assert_array_equal(M, mat)


# ------------------------------------------------- application of a circuit

@pytest.mark.parametrize("n,seed", [(1, 1), (2, 2), (3, 3), (5, 4), (7, 5), (10, 6)])
def test_circuit_matches_tensor_contraction(n, seed):
    rng = np.random.default_rng(seed)
    gates, P = W.random_circuit(n, 40 if n < 10 else 25, rng)
    params = rng.uniform(-np.pi, np.pi, P)
    psi = rand_state(n, 100 + seed)
    got = oracle.apply_circuit(psi.copy(), n, gates, params)
    want = psi.copy()
    for g in gates:
        th = g.angle + (params[g.param] if g.param >= 0 else 0.0)
        want = tensor_apply(want, n, g.qubits, oracle.gate_matrix(g.name, th, g.mat))
    np.testing.assert_allclose(got, want, atol=1e-13)
    assert abs(oracle.norm2(got, n) - 1) < 1e-13


@pytest.mark.parametrize("n", [4, 6])
def test_circuit_matches_dense_unitary_product(n):
    """2^n x 2^n products built from Kronecker products of expm generators."""
    rng = np.random.default_rng(7)
    th = rng.uniform(-np.pi, np.pi, 3 * n)
    gates, U = [], np.eye(1 << n, dtype=complex)

    def emb(ops):  # Kronecker product over all qubits, qubit 0 leftmost
        m = np.array([[1.0 + 0j]])
        for q in range(n):
            m = np.kron(m, ops.get(q, I2))
        return m

    for q in range(n):
        gates.append(W.G("RY", q, angle=th[q]))
        U = emb({q: sla.expm(-0.5j * th[q] * PY)}) @ U
        gates.append(W.G("RZ", q, angle=th[n + q]))
        U = emb({q: sla.expm(-0.5j * th[n + q] * PZ)}) @ U
    for q in range(n - 1):
        gates.append(W.G("CNOT", q, q + 1))
        U = (emb({q: np.diag([1.0, 0]) + 0j}) + emb({q: P1, q + 1: PX})) @ U
    for q in range(n):
        gates.append(W.G("RX", q, angle=th[2 * n + q]))
        U = emb({q: sla.expm(-0.5j * th[2 * n + q] * PX)}) @ U
    psi = rand_state(n, 8)
    np.testing.assert_allclose(oracle.apply_circuit(psi.copy(), n, gates), U @ psi, atol=1e-13)


def test_invariants_and_ghz():
    n = 6
    psi = rand_state(n, 11)
    for gs in (
        [W.G("H", 2), W.G("H", 2)],
        [W.G("X", 4), W.G("X", 4)],
        [W.G("CNOT", 1, 3), W.G("CNOT", 1, 3)],
        [W.G("RZ", 0, angle=0.8), W.G("RZ", 0, angle=-0.8)],
        [W.G("CCX", 5, 0, 2), W.G("CCX", 5, 0, 2)],
    ):
        np.testing.assert_allclose(oracle.apply_circuit(psi.copy(), n, gs), psi, atol=1e-15)
    ghz = oracle.basis_state(n)
    oracle.apply_circuit(ghz, n, [W.G("H", 0)] + [W.G("CNOT", q, q + 1) for q in range(n - 1)])
    want = np.zeros(1 << n, complex)
    want[0] = want[-1] = R2
    np.testing.assert_allclose(ghz, want, atol=1e-16)
    bell = oracle.apply_circuit(oracle.basis_state(2), 2, [W.G("H", 0), W.G("CNOT", 0, 1)])
    np.testing.assert_allclose(bell, [R2, 0, 0, R2], atol=1e-16)


# ----------------------------------------------------------------- <H>

@pytest.mark.parametrize("theta", [0.0, 0.4, -1.3, 2.9])
def test_expval_closed_forms(theta):
    # <Z> after RY(theta)|0> = cos(theta), <X> = sin(theta); after RX: <Y> = -sin
    psi = oracle.apply_circuit(oracle.basis_state(1), 1, [W.G("RY", 0, angle=theta)])
    assert abs(oracle.expval(psi, 1, [(1.0, "Z")]) - np.cos(theta)) < 1e-15
    assert abs(oracle.expval(psi, 1, [(1.0, "X")]) - np.sin(theta)) < 1e-15
    psi = oracle.apply_circuit(oracle.basis_state(1), 1, [W.G("RX", 0, angle=theta)])
    assert abs(oracle.expval(psi, 1, [(1.0, "Y")]) + np.sin(theta)) < 1e-15


@pytest.mark.parametrize("n", [2, 5, 10])
def test_heisenberg_on_basis_states(n):
    terms = W.heisenberg(n)
    # |0...0>: only ZZ contributes, each pair +Jz
    assert abs(oracle.expval(oracle.basis_state(n), n, terms) - 0.25 * (n - 1)) < 1e-15
    x = W.basis_index(n, 3)
    bits = [(x >> (n - 1 - q)) & 1 for q in range(n)]
    want = sum(0.25 * (1 if bits[i] == bits[i + 1] else -1) for i in range(n - 1))
    assert abs(oracle.expval(oracle.basis_state(n, x), n, terms) - want) < 1e-15


@pytest.mark.parametrize("n,seed", [(3, 1), (6, 2), (8, 3)])
def test_expval_matches_dense_hamiltonian(n, seed):
    rng = np.random.default_rng(seed)
    terms = W.random_pauli_sum(n, 12, rng, kmin=1, kmax=min(4, n)) + W.heisenberg(n, ring=True)
    psi = rand_state(n, seed)
    want = np.vdot(psi, dense_h(terms) @ psi).real
    assert abs(oracle.expval(psi, n, terms) - want) < 1e-13


@pytest.mark.parametrize("n", [4, 6, 8])
def test_variational_bound(n):
    terms = W.heisenberg(n)
    e0 = np.linalg.eigvalsh(dense_h(terms)).min()
    gates, P = W.hea(n, 3)
    for s in range(4):
        e = oracle.energy(n, gates, W.angles(P, 50 + s), terms)
        assert e >= e0 - 1e-12


# -------------------------------------------------------------------- QFT

@pytest.mark.parametrize("n", [1, 2, 3, 8, 12])
def test_qft_closed_form_basis(n):
    N = 1 << n
    for x in sorted({0, 1, N - 1, W.basis_index(n, 2000 + n)}):
        k = np.arange(N, dtype=np.int64)
        r = (x * k) % N  # exact integer phase index
        want = np.exp(2j * np.pi * r / N) / np.sqrt(N)
        got = oracle.qft_fft(oracle.basis_state(n, x), n)
        np.testing.assert_allclose(got, want, atol=1e-14)
        got = oracle.qft_gates(oracle.basis_state(n, x), n)
        np.testing.assert_allclose(got, want, atol=1e-14)


@pytest.mark.parametrize("n", [4, 10, 16])
def test_qft_matches_numpy_ifft(n):
    psi = W.gaussian_state(n, 1000 + n)
    want = np.fft.ifft(psi, norm="ortho")
    np.testing.assert_allclose(oracle.qft_fft(psi.copy(), n), want, atol=1e-14)
    back = oracle.qft_fft(want.copy(), n, inverse=True)
    np.testing.assert_allclose(back, psi, atol=1e-14)
    if n <= 10:
        np.testing.assert_allclose(oracle.qft_gates(psi.copy(), n), want, atol=1e-13)
    for k in (0, 1, (1 << n) - 1, 12345 % (1 << n)):
        assert abs(oracle.qft_amplitude(psi, n, k) - want[k]) < 1e-14


def test_qft_invariants():
    n, N = 9, 512
    psi = W.gaussian_state(n, 77)
    q1 = oracle.qft_fft(psi.copy(), n)
    q2 = oracle.qft_fft(q1.copy(), n)
    np.testing.assert_allclose(q2, psi[(-np.arange(N)) % N], atol=1e-14)  # QFT^2: x -> -x
    q4 = oracle.qft_fft(oracle.qft_fft(q2.copy(), n), n)
    np.testing.assert_allclose(q4, psi, atol=1e-14)
    u = oracle.qft_fft(oracle.basis_state(n, 0), n)
    np.testing.assert_allclose(u, np.full(N, 1 / np.sqrt(N)), atol=1e-15)
    assert abs(oracle.norm2(q1, n) - 1) < 1e-14


# ------------------------------------------------------ gradients (PSR/FD)

def _table_value(tok):
    return float(tok)


def _angles(toks):
    out = []
    for t in toks:
        out.append({"pi": np.pi, "pi/2": np.pi / 2}.get(t, None) if t in ("pi", "pi/2") else float(t))
    return out


def test_appD_table():
    gates, P, H = W.appd_circuit()
    with open(os.path.join(GOLD, "appD_psr_table.txt")) as f:
        rows = [ln for ln in f if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 5
    for ln in rows:
        left, right = ln.split("|")
        name, *th = left.split()
        th = _angles(th)
        assert th == W.APPD_ANGLE_SETS[name]
        want = [float(v) for v in right.split()]
        e, g = oracle.param_shift(2, gates, th, H, general=True)
        fd = oracle.finite_diff(2, gates, th, H, h=1e-5)
        np.testing.assert_allclose(g, fd, atol=1e-9)
        # printed to 4 decimals (the near-zero first entry as -1.0e-8)
        tol = 2e-10 if name == "near_zero" else 5e-5
        np.testing.assert_allclose(g, want, atol=tol)


def test_psr_closed_form_one_qubit():
    gates = [W.G("RY", 0, param=0)]
    for th in (-2.0, 0.3, 1.1):
        e, g = oracle.param_shift(1, gates, [th], [(1.0, "Z")])
        assert abs(e - np.cos(th)) < 1e-15 and abs(g[0] + np.sin(th)) < 1e-15


@pytest.mark.parametrize("n,depth", [(3, 2), (4, 3)])
def test_psr_matches_finite_differences(n, depth):
    gates, P = W.hea(n, depth, "ring")
    th = W.angles(P, 9)
    terms = W.heisenberg(n)
    e, g = oracle.param_shift(n, gates, th, terms)
    fd = oracle.finite_diff(n, gates, th, terms, h=1e-4)
    np.testing.assert_allclose(g, fd, atol=1e-7)
    assert abs(e - oracle.energy(n, gates, th, terms)) < 1e-15


def test_psr_general_rules_match_finite_differences():
    # controlled rotations (four-term rule) and a parameter shared by 3 gates
    n = 3
    gates = [
        W.G("H", 0), W.G("RX", 1, param=0), W.G("CRY", 0, 1, param=1),
        W.G("CRX", 1, 2, param=2), W.G("CRZ", 2, 0, param=1, angle=0.3),
        W.G("RYY", 0, 2, param=0), W.G("CP", 1, 0, param=2), W.G("RZZ", 1, 2, param=0, angle=-0.2),
    ]
    terms = [(0.7, "XIZ"), (-1.1, "YXI"), (0.4, "ZZZ"), (0.9, "IXY")]
    th = np.array([0.41, -1.3, 2.2])
    e, g = oracle.param_shift(n, gates, th, terms, general=True)
    fd = oracle.finite_diff(n, gates, th, terms, h=1e-4)
    np.testing.assert_allclose(g, fd, atol=1e-7)
    # a mistake the four-term rule guards against: the two-term rule on CRY
    # is wrong here, so the two-term mode must refuse this circuit
    with pytest.raises(oracle.OracleUnsupported):
        oracle.param_shift(n, gates, th, terms)


def test_psr_rejects_shared_parameter_in_paper_mode():
    gates = [W.G("RX", 0, param=0), W.G("RY", 0, param=0)]
    with pytest.raises(oracle.OracleUnsupported):
        oracle.param_shift(1, gates, [0.1], [(1.0, "Z")])


# ---------------------------------------------------------------- Trotter

def test_trotter_matches_dense_exponential_product():
    n, dt, steps = 4, 0.05, 7
    static, field, A, omega, x0 = W.xyz_trotter(n)
    psi = oracle.basis_state(n, x0)
    got = oracle.trotter(psi.copy(), n, static, field, A, omega, dt, steps)
    want = psi.copy()
    for j in range(steps):
        h = A * np.sin(omega * j * dt)
        for c, s in static:
            want = sla.expm(-1j * c * dt * dense_pauli(s)) @ want
        for c, s in field:
            want = sla.expm(-1j * h * c * dt * dense_pauli(s)) @ want
    np.testing.assert_allclose(got, want, atol=1e-13)
    # first-order convergence to the exact time-ordered evolution: from a
    # non-eigenstate, quartering dt cuts the error about four times
    x0 = 0b0110
    psi = oracle.basis_state(n, x0)
    H0, Hf = dense_h(static), dense_h(field)
    T, m = 0.4, 2000
    exact = psi.copy()
    for j in range(m):
        t = (j + 0.5) * T / m
        exact = sla.expm(-1j * (H0 + A * np.sin(omega * t) * Hf) * (T / m)) @ exact
    errs = []
    for steps in (10, 40):
        got = oracle.trotter(psi.copy(), n, static, field, A, omega, T / steps, steps)
        errs.append(np.abs(got - exact).max())
    assert errs[1] < errs[0] / 3.0 and errs[1] < 0.05
