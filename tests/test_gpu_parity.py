"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bars: 1e-12 absolute per amplitude; energies and gradients within
1e-10 * max(1, |value|); permutation-only circuits and basis-state set-up
bit-exact.  Sizes span one tile (n <= 10), several tiles (n = 11..17) and
the edge cases n = 1, n below the contiguous-run width, and n = tile width.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

ATOL = 1e-12
RTOL = 1e-10


@pytest.fixture(scope="module")
def lq():
    import paper_2512_23183_gb300 as m

    m.load()
    return m


def dev(psi):
    import torch

    return torch.from_numpy(np.ascontiguousarray(psi)).cuda()


def host(t):
    import torch

    torch.cuda.synchronize()
    return t.cpu().numpy()


def close_e(a, b):
    return abs(a - b) <= RTOL * max(1.0, abs(b))


# --------------------------------------------------------------- states

@pytest.mark.parametrize("n", [1, 2, 5, 10, 13, 20])
def test_state_init_bit_exact(lq, n):
    x = W.basis_index(n, 7)
    t = lq.new_state(n, x)
    np.testing.assert_array_equal(host(t), oracle.basis_state(n, x))


def test_paper_worked_examples(lq):
    s = np.zeros(4, complex)
    s[0] = s[3] = 1 / np.sqrt(2)
    t = dev(s)
    lq.apply_circuit(t, 2, [W.G("CNOT", 0, 1)])
    np.testing.assert_array_equal(host(t), oracle.cnot_alg1(s.copy(), 2, 0, 1))
    s = np.zeros(8, complex)
    s[5] = s[6] = 1 / np.sqrt(2)
    t = dev(s)
    lq.apply_circuit(t, 3, [W.G("CCX", 0, 1, 2)])
    np.testing.assert_array_equal(host(t), oracle.toffoli_alg4(s.copy(), 3, 0, 1, 2))


# ------------------------------------------------------------- circuits

@pytest.mark.parametrize("n,seed,ng", [(1, 1, 30), (2, 2, 40), (3, 3, 60), (4, 4, 80), (6, 5, 80),
                                       (9, 6, 80), (10, 7, 100), (11, 8, 100), (12, 9, 80),
                                       (14, 10, 80), (17, 11, 60)])
def test_random_circuit(lq, n, seed, ng):
    rng = np.random.default_rng(seed)
    gates, P = W.random_circuit(n, ng, rng)
    params = rng.uniform(-np.pi, np.pi, P)
    psi = W.gaussian_state(n, 100 + seed)
    want = oracle.apply_circuit(psi.copy(), n, gates, params)
    t = dev(psi)
    lq.apply_circuit(t, n, gates, params)
    np.testing.assert_allclose(host(t), want, rtol=0, atol=ATOL)


@pytest.mark.parametrize("n,k,m,table,seed", [(18, 6, 2, 0, 1), (18, 8, 3, 1, 2), (19, 9, 4, 0, 3),
                                              (18, 7, 5, 1, 4), (20, 10, 3, 0, 5)])
def test_phase_sinking_across_many_passes(lq, tune_entry, n, k, m, table, seed):
    # small forced tiles give many passes: one-bit phases (RZ, P, T) move
    # forward across passes, through CNOT and CY targets and swaps as parity
    # phases, and merge where at most one of their bits is a tile bit
    rng = np.random.default_rng(900 + seed)
    kinds = ["RY", "RZ", "RZ", "RZ", "P", "T", "CNOT", "CNOT", "CY", "SWAP", "CZ", "H", "RX", "CP"]
    gates, P = W.random_circuit(n, 150, rng, kinds=kinds)
    params = rng.uniform(-np.pi, np.pi, P)
    psi = W.gaussian_state(n, 700 + seed)
    want = oracle.apply_circuit(psi.copy(), n, gates, params)
    tune_entry(n, gates, k, m, table)
    t = dev(psi)
    lq.apply_circuit(t, n, gates, params)
    np.testing.assert_allclose(host(t), want, rtol=0, atol=ATOL)


@pytest.mark.parametrize("n,depth,ent,k,m", [(18, 2, "ladder", 8, 3), (18, 3, "ring", 9, 2),
                                             (22, 1, "ladder", 12, 3), (22, 2, "ring", 12, 3)])
def test_hea_phases_merged_once_per_layer(lq, tune_entry, n, depth, ent, k, m):
    # a layer's RZ factors reach its last pass as CTA-bit parities and
    # one-bit tile phases, one merged op with the circuit's final scalar
    rng = np.random.default_rng(n + depth)
    gates, P = W.hea(n, depth, ent)
    params = rng.uniform(-np.pi, np.pi, P)
    psi = W.gaussian_state(n, 800 + n)
    want = oracle.apply_circuit(psi.copy(), n, gates, params)
    tune_entry(n, gates, k, m, 0)
    t = dev(psi)
    lq.apply_circuit(t, n, gates, params)
    np.testing.assert_allclose(host(t), want, rtol=0, atol=ATOL)


@pytest.mark.parametrize("name", sorted(oracle.GATE_CODES))
def test_each_gate_kind_on_every_qubit_tuple(lq, name):
    n = 4
    rng = np.random.default_rng(abs(hash(name)) % 1000)
    k = 3 if name == "CCX" else 2 if name in (
        "CNOT", "CY", "CZ", "CP", "SWAP", "CRX", "CRY", "CRZ", "RXX", "RYY", "RZZ", "U2") else 1
    import itertools

    gates = []
    for qs in itertools.permutations(range(n), k):
        mat = None
        if name in ("U1", "U2"):
            d = 2 if name == "U1" else 4
            q, _ = np.linalg.qr(rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d)))
            mat = q
        gates.append(W.G(name, *qs, angle=float(rng.uniform(-7, 7)), mat=mat))
    psi = W.gaussian_state(n, 3)
    for g in gates:
        want = oracle.apply_circuit(psi.copy(), n, [g])
        t = dev(psi)
        lq.apply_circuit(t, n, [g])
        np.testing.assert_allclose(host(t), want, rtol=0, atol=ATOL, err_msg=str(g))


@pytest.mark.parametrize("n,depth,ent", [(10, 4, "ladder"), (16, 3, "ring"), (20, 2, "ladder")])
def test_hea(lq, n, depth, ent):
    gates, P = W.hea(n, depth, ent)
    th = W.angles(P, 5)
    want = oracle.apply_circuit(oracle.basis_state(n), n, gates, th)
    t = lq.new_state(n)
    lq.apply_circuit(t, n, gates, th)
    np.testing.assert_allclose(host(t), want, rtol=0, atol=ATOL)


def test_permutation_circuit_bit_exact(lq):
    n = 15
    rng = np.random.default_rng(3)
    gates, _ = W.random_circuit(n, 200, rng, kinds=["X", "Y", "Z", "S", "SDG", "CNOT", "CY", "CZ",
                                                     "SWAP", "CCX"])
    psi = W.gaussian_state(n, 4)
    want = oracle.apply_circuit(psi.copy(), n, gates)
    t = dev(psi)
    lq.apply_circuit(t, n, gates)
    np.testing.assert_array_equal(host(t), want)


def test_long_circuit_rescales(lq):
    # thousands of tangent-form rotations: the deferred scalar is renormalised
    n = 6
    rng = np.random.default_rng(9)
    gates = [W.G("RX", q % n, angle=float(rng.uniform(1.2, 1.9))) for q in range(3000)]
    psi = W.gaussian_state(n, 1)
    want = oracle.apply_circuit(psi.copy(), n, gates)
    t = dev(psi)
    lq.apply_circuit(t, n, gates)
    np.testing.assert_allclose(host(t), want, rtol=0, atol=1e-11)


# ----------------------------------------------------------------- <H>

@pytest.mark.parametrize("n,seed", [(1, 1), (3, 2), (8, 3), (12, 4), (16, 5), (20, 6)])
def test_expval(lq, n, seed):
    rng = np.random.default_rng(seed)
    terms = W.random_pauli_sum(n, 50, rng, kmin=1, kmax=min(4, n))
    if n >= 2:
        terms += W.heisenberg(n, ring=n > 2)
    psi = W.gaussian_state(n, seed)
    want = oracle.expval(psi, n, terms)
    got = lq.expval_pauli_sum(dev(psi), n, terms)
    assert close_e(got, want), (got, want)


def test_expval_many_terms_chunked(lq):
    n = 9
    rng = np.random.default_rng(11)
    terms = W.random_pauli_sum(n, 1500, rng, kmin=1, kmax=5)
    psi = W.gaussian_state(n, 2)
    assert close_e(lq.expval_pauli_sum(dev(psi), n, terms), oracle.expval(psi, n, terms))
    assert lq.expval_pauli_sum(dev(psi), n, []) == 0.0


@pytest.mark.parametrize("n,masks,diag,dup", [(12, 240, 5, 0), (14, 400, 0, 0), (12, 20, 300, 0),
                                              (13, 3, 10, 300)])
def test_expval_tiled_beyond_one_plan(lq, n, masks, diag, dup):
    # more X-mask groups, terms or coefficients than one tiled plan holds: a
    # small state is one tile, so the passes are split by capacity; a long
    # diagonal group and a long class group (the same XX term repeated) too
    rng = np.random.default_rng(n + masks + diag)
    terms = []
    for m in rng.choice(np.arange(1, 1 << n), size=masks, replace=False):
        s = ["XY"[rng.integers(2)] if (int(m) >> (n - 1 - q)) & 1 else "IZ"[rng.integers(2)]
             for q in range(n)]
        terms.append((float(rng.standard_normal()), "".join(s)))
    terms += [(float(rng.standard_normal()),
               "".join("Z" if rng.random() < 0.3 else "I" for _ in range(n))) for _ in range(diag)]
    terms += [(float(rng.standard_normal()), "XX" + "I" * (n - 2)) for _ in range(dup)]
    psi = W.gaussian_state(n, 60 + n)
    assert close_e(lq.expval_pauli_sum(dev(psi), n, terms), oracle.expval(psi, n, terms))


def _pauli(n, ops, c=1.0):
    """(c, string) with ops = {qubit: 'X'|'Y'|'Z'}."""
    s = ["I"] * n
    for q, ch in ops.items():
        s[q] = ch
    return (float(c), "".join(s))


@pytest.mark.parametrize("n,ring", [(12, False), (13, True), (16, True), (18, False)])
def test_expval_tiled_heisenberg(lq, n, ring):
    # XX + YY share an X mask with Z inside it (class mode); ZZ is diagonal
    terms = W.heisenberg(n, ring=ring) + W.z_field(n, 0.3)
    psi = W.gaussian_state(n, 40 + n)
    assert close_e(lq.expval_pauli_sum(dev(psi), n, terms), oracle.expval(psi, n, terms))


@pytest.mark.parametrize("n,seed", [(12, 1), (14, 2), (17, 3)])
def test_expval_tiled_random(lq, n, seed):
    # table mode: Z factors outside the X mask, every Y parity mix
    rng = np.random.default_rng(100 + seed)
    terms = W.random_pauli_sum(n, 80, rng, kmin=1, kmax=4)
    psi = W.gaussian_state(n, 50 + seed)
    assert close_e(lq.expval_pauli_sum(dev(psi), n, terms), oracle.expval(psi, n, terms))


def test_expval_tiled_group_shapes(lq):
    n = 15
    rng = np.random.default_rng(7)
    terms = []
    # eleven terms on one X mask (split into table-mode groups of four)
    for _ in range(11):
        ops = {0: "X", 9: "Y"}
        for q in rng.choice([2, 3, 5, 12, 14], size=2, replace=False):
            ops[int(q)] = "Z"
        terms.append(_pauli(n, ops, rng.normal()))
    # class mode with an odd Y count (only Im) and with both parities (Re and Im)
    terms.append(_pauli(n, {3: "X", 4: "Y"}, 0.7))
    terms.append(_pauli(n, {3: "Y", 4: "X"}, -0.4))
    terms.append(_pauli(n, {6: "X", 7: "X"}, 0.9))
    terms.append(_pauli(n, {6: "X", 7: "Y"}, 0.5))
    terms.append(_pauli(n, {1: "Y", 8: "Y", 13: "X"}, -1.1))   # three X bits, four classes
    terms.append(_pauli(n, {11: "X"}, 0.25))                     # one X bit
    terms.append(_pauli(n, {10: "Y"}, -0.35))
    # X masks wider than a tile (the untiled kernel) and diagonal terms across chunks
    terms.append((0.6, "X" * n))
    terms.append((-0.2, "XY" * (n // 2) + "Z"))
    terms.append(_pauli(n, {0: "Z", 14: "Z"}, 0.8))
    terms.append(_pauli(n, {2: "Z", 5: "Z", 9: "Z"}, -0.45))
    psi = W.gaussian_state(n, 77)
    assert close_e(lq.expval_pauli_sum(dev(psi), n, terms), oracle.expval(psi, n, terms))
    # diagonal only, and wide only
    for sub in (terms[-2:] + W.z_field(n, 0.1), terms[-4:-2]):
        assert close_e(lq.expval_pauli_sum(dev(psi), n, sub), oracle.expval(psi, n, sub))


@pytest.mark.parametrize("n", [2, 7, 13])
def test_apply_pauli_sum(lq, n):
    import torch

    rng = np.random.default_rng(n)
    terms = W.random_pauli_sum(n, 30, rng, kmin=1, kmax=min(3, n))
    psi = W.gaussian_state(n, 8)
    want = np.zeros_like(psi)
    for c, s in terms:
        gs = [W.G(ch, q) for q, ch in enumerate(s) if ch != "I"]
        want += c * oracle.apply_circuit(psi.copy(), n, gs)
    out = torch.empty(1 << n, dtype=torch.complex128, device="cuda")
    lq.apply_pauli_sum(out, dev(psi), n, terms)
    np.testing.assert_allclose(host(out), want, rtol=0, atol=ATOL * 10)


# ------------------------------------------------------------------ QFT

@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 11, 12, 13, 14, 17, 20])
def test_qft_fft_gaussian(lq, n):
    psi = W.gaussian_state(n, 1000 + n)
    want = oracle.qft_fft(psi.copy(), n)
    t = dev(psi)
    lq.qft(t, n)
    np.testing.assert_allclose(host(t), want, rtol=0, atol=ATOL)
    lq.qft(t, n, inverse=True)
    np.testing.assert_allclose(host(t), psi, rtol=0, atol=ATOL)


@pytest.mark.parametrize("n", [1, 4, 9, 12, 15])
def test_qft_gate_form(lq, n):
    psi = W.gaussian_state(n, 2000 + n)
    want = oracle.qft_gates(psi.copy(), n)
    t = dev(psi)
    lq.qft(t, n, method=lq.QFT_GATES)
    np.testing.assert_allclose(host(t), want, rtol=0, atol=ATOL)
    lq.qft(t, n, inverse=True, method=lq.QFT_GATES)
    np.testing.assert_allclose(host(t), psi, rtol=0, atol=ATOL)


@pytest.mark.parametrize("n", [22, 24])
def test_qft_gate_form_large_against_fft_form(lq, n):
    # from 2^12 tiles on the gate form runs butterflies, and from n = 24 the
    # forward list has each CP moved before its target's H: both forms agree
    # element-wise (the FFT form is pinned to the oracle), and the inverse
    # gate form undoes the forward FFT form
    psi = W.gaussian_state(n, 3000 + n)
    a, b = dev(psi), dev(psi)
    lq.qft(a, n, method=lq.QFT_GATES)
    lq.qft(b, n, method=lq.QFT_FFT)
    assert float((a - b).abs().max()) < ATOL
    lq.qft(b, n, inverse=True, method=lq.QFT_GATES)
    np.testing.assert_allclose(host(b), psi, rtol=0, atol=ATOL)


@pytest.mark.parametrize("n", [20, 22, 24, 28])
def test_qft_basis_closed_form_sampled(lq, n):
    # QFT|x> = N^{-1/2} sum_k e^{2 pi i x k / N}|k>, phase index x k mod N in
    # integers; both forms, at the basis inputs of the QFT workload sizes
    import torch

    N = 1 << n
    x = W.basis_index(n, 2000 + n)
    k = np.random.default_rng(n).integers(0, N, 4096)
    want = np.exp(2j * np.pi * ((x * k) % N) / N) / np.sqrt(N)
    for meth in (lq.QFT_FFT, lq.QFT_GATES):
        t = lq.new_state(n, x)
        lq.qft(t, n, method=meth)
        got = t[torch.from_numpy(k).cuda()].cpu().numpy()
        np.testing.assert_allclose(got, want, rtol=0, atol=ATOL)
        del t


def test_qft_n24_gaussian_both_forms_against_oracle(lq):
    # the seeded Gaussian input of the QFT workload at n = 24, where the
    # forward gate form uses its reordered list: both forms and both
    # directions element-wise against the oracle's plain radix-2 inverse DFT
    n = 24
    psi = W.gaussian_state(n, 1000 + n)
    want = {False: oracle.qft_fft(psi.copy(), n), True: oracle.qft_fft(psi.copy(), n, inverse=True)}
    for meth in (lq.QFT_FFT, lq.QFT_GATES):
        for inverse in (False, True):
            t = dev(psi)
            lq.qft(t, n, inverse=inverse, method=meth)
            err = float(np.abs(host(t) - want[inverse]).max())
            assert err < ATOL, (meth, inverse, err)
            del t


# ------------------------------------------------------------ gradients

@pytest.mark.parametrize("method", [0, 1])
@pytest.mark.parametrize("n,depth,ent", [(1, 2, "ladder"), (4, 3, "ring"), (10, 4, "ladder"),
                                         (12, 2, "ring")])
def test_param_shift(lq, method, n, depth, ent):
    gates, P = W.hea(n, depth, ent)
    th = W.angles(P, 1 + n)
    terms = W.heisenberg(n) if n > 1 else [(1.0, "Z"), (0.5, "X")]
    e_w, g_w = oracle.param_shift(n, gates, th, terms)
    e, g = lq.param_shift_grad(n, gates, th, terms, method=method)
    assert close_e(e, e_w)
    np.testing.assert_allclose(g, g_w, rtol=0, atol=RTOL * max(1.0, np.abs(g_w).max()))


def test_param_shift_all_two_term_kinds(lq):
    n = 4
    gates = [W.G("H", 0), W.G("RX", 0, param=0), W.G("RY", 1, param=1), W.G("RZ", 2, param=2),
             W.G("P", 3, param=3), W.G("CNOT", 0, 2), W.G("CP", 1, 3, param=4),
             W.G("RXX", 0, 3, param=5), W.G("RYY", 2, 1, param=6), W.G("RZZ", 3, 0, param=7)]
    th = W.angles(8, 17)
    terms = W.random_pauli_sum(n, 20, np.random.default_rng(5), kmin=1, kmax=4)
    e_w, g_w = oracle.param_shift(n, gates, th, terms)
    for method in (0, 1):
        e, g = lq.param_shift_grad(n, gates, th, terms, method=method)
        assert close_e(e, e_w)
        np.testing.assert_allclose(g, g_w, rtol=0, atol=RTOL)


# -------------------------------------------------------------- Trotter

@pytest.mark.parametrize("n,steps", [(3, 5), (8, 12), (12, 4), (16, 3), (20, 2)])
def test_trotter(lq, n, steps):
    static, field, A, omega, x0 = W.xyz_trotter(n, J=(1.0, 0.7, 0.4))
    dt = 0.07
    want = oracle.trotter(oracle.basis_state(n, x0), n, static, field, A, omega, dt, steps)
    t = lq.new_state(n, x0)
    lq.trotter_evolve(t, n, static, field, A, omega, dt, steps)
    np.testing.assert_allclose(host(t), want, rtol=0, atol=ATOL)


@pytest.mark.parametrize("n,seed", [(12, 1), (15, 2), (17, 3), (20, 4)])
def test_dyadic_runs_with_one_common_control(lq, n, seed):
    # QFT-like blocks: H(i), then CP(i, j) on a random set of other qubits
    # (one common control bit, phases deferred to the store or the load of
    # the pass), sometimes with H(i) again after the run (the per-tile part
    # must then stay in place or move to the load) or before the block's H
    rng = np.random.default_rng(500 + seed)
    gates = []
    for _ in range(3 * n):
        i = int(rng.integers(n))
        if rng.random() < 0.3:
            gates.append(W.G("H", i))
        gates.append(W.G("H", i))
        others = [j for j in range(n) if j != i]
        for j in rng.choice(others, size=int(rng.integers(2, min(8, n - 1))), replace=False):
            k = int(rng.integers(1, 25))
            gates.append(W.G("CP", i, int(j), angle=float(rng.choice([1, -1]) * np.pi / 2 ** k)))
        if rng.random() < 0.3:
            gates.append(W.G("H", i))
        if rng.random() < 0.2:
            gates.append(W.G("RY", int(rng.integers(n)), angle=float(rng.uniform(-3, 3))))
    psi = W.gaussian_state(n, 70 + seed)
    want = oracle.apply_circuit(psi.copy(), n, gates)
    t = dev(psi)
    lq.apply_circuit(t, n, gates)
    np.testing.assert_allclose(host(t), want, rtol=0, atol=ATOL)


@pytest.mark.parametrize("n,seed", [(3, 1), (9, 2), (14, 3), (16, 4)])
def test_fixed_dyadic_phase_runs(lq, n, seed):
    # runs of fixed dyadic diagonal gates (merged into one table-driven phase
    # op when cheaper) between H layers, with controls on tile and CTA bits
    rng = np.random.default_rng(seed)
    gates = []
    for layer in range(4):
        for q in range(n):
            gates.append(W.G("H", q))
        for _ in range(3 * n):
            kind = ["CP", "CP", "P", "T", "TDG", "S", "Z", "CZ", "RZ"][rng.integers(9)]
            k = int(rng.integers(1, 12))
            ang = float(rng.choice([1, -1]) * np.pi / 2 ** k)
            if kind in ("CP", "CZ"):
                a, b = rng.choice(n, 2, replace=False) if n > 1 else (0, 0)
                gates.append(W.G(kind, a, b, angle=ang if kind == "CP" else 0.0))
            else:
                gates.append(W.G(kind, int(rng.integers(n)),
                                 angle=ang if kind in ("P", "RZ") else 0.0))
    gates = [g for g in gates if len(set(g.qubits)) == len(g.qubits)]
    psi = W.gaussian_state(n, 60 + seed)
    want = oracle.apply_circuit(psi.copy(), n, gates)
    t = dev(psi)
    lq.apply_circuit(t, n, gates)
    np.testing.assert_allclose(host(t), want, rtol=0, atol=ATOL)
