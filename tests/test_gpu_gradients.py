"""Gradients on the GPU: adjoint (reverse-mode) and generalised parameter
shift, against the oracle's parameter-shift rule (1e-10) and central finite
differences (h = 1e-4, 1e-6), the App. D table, and the autograd wrapper."""
import os

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-10


@pytest.fixture(scope="module")
def lq():
    import paper_2512_23183_gb300 as m

    m.load()
    return m


def general_circuit(n, rng, ngates=40, nparams=6):
    kinds = ["H", "RX", "RY", "RZ", "P", "CP", "CRX", "CRY", "CRZ", "RXX", "RYY", "RZZ", "CNOT",
             "CZ", "SWAP", "S", "T", "CCX", "U2"]
    gates, _ = W.random_circuit(n, ngates, rng, kinds=kinds, parametrised=False)
    out = []
    for g in gates:
        if g.name in ("RX", "RY", "RZ", "P", "CP", "CRX", "CRY", "CRZ", "RXX", "RYY", "RZZ"):
            out.append(W.G(g.name, *g.qubits, param=int(rng.integers(nparams)), angle=g.angle))
        else:
            out.append(g)
    return out


@pytest.mark.parametrize("n,depth,ent", [(1, 3, "ladder"), (4, 3, "ring"), (10, 4, "ladder"),
                                         (12, 3, "ring"), (14, 2, "ladder")])
def test_adjoint_matches_parameter_shift(lq, n, depth, ent):
    gates, P = W.hea(n, depth, ent)
    th = W.angles(P, 40 + n)
    terms = W.heisenberg(n) if n > 1 else [(1.0, "Z"), (0.3, "Y")]
    e_w, g_w = oracle.param_shift(n, gates, th, terms)
    e, g = lq.adjoint_grad(n, gates, th, terms)
    assert abs(e - e_w) <= RTOL * max(1, abs(e_w))
    np.testing.assert_allclose(g, g_w, rtol=0, atol=RTOL * max(1.0, np.abs(g_w).max()))


@pytest.mark.parametrize("n,seed", [(2, 1), (3, 2), (5, 3), (11, 4)])
def test_adjoint_general_gates_vs_finite_differences(lq, n, seed):
    rng = np.random.default_rng(seed)
    gates = general_circuit(n, rng, ngates=30 if n < 11 else 60)
    th = rng.uniform(-np.pi, np.pi, 6)
    terms = W.random_pauli_sum(n, 15, rng, kmin=1, kmax=min(3, n))
    e_w, g_w = oracle.param_shift(n, gates, th, terms, general=True)
    fd = oracle.finite_diff(n, gates, th, terms, h=1e-4)
    e, g = lq.adjoint_grad(n, gates, th, terms)
    assert abs(e - e_w) <= RTOL * max(1, abs(e_w))
    np.testing.assert_allclose(g, g_w, rtol=0, atol=RTOL * max(1.0, np.abs(g_w).max()))
    np.testing.assert_allclose(g, fd, rtol=0, atol=1e-6)


def diagonal_run_circuit(n, rng, layers=3):
    """RY layers separated by long runs of diagonal gates (RZ, P, CP, CRZ,
    RZZ with parameters, some shared; S, T, CZ fixed): the reverse sweep
    takes each run's gradients together."""
    gates, p = [], 0
    for _ in range(layers):
        for q in range(n):
            gates.append(W.G("RY", q, param=p)); p += 1
        for q in range(n):
            gates.append(W.G("RZ", q, param=p)); p += 1
            a, b = q, (q + 1 + int(rng.integers(n - 1))) % n
            kind = ["P", "CP", "CRZ", "RZZ", "S", "T", "CZ"][int(rng.integers(7))]
            if kind == "P":
                gates.append(W.G("P", a, param=int(rng.integers(p))))   # shared parameter
            elif kind in ("CP", "CRZ", "RZZ"):
                gates.append(W.G(kind, a, b, param=p)); p += 1
            else:
                gates.append(W.G(kind, *((a, b) if kind == "CZ" else (a,))))
        for q in range(n - 1):
            gates.append(W.G("CNOT", q, q + 1))
    return gates, p


@pytest.mark.parametrize("n", [18, 20])
def test_adjoint_wide_sweep_tiles_match_oracle(lq, n):
    # from n = 18 the reverse sweep runs 2^11-amplitude tiles: every entry of
    # the gradient against the oracle's parameter-shift rule
    gates, P = W.hea(n, 2, "ladder")
    th = W.angles(P, 60 + n)
    terms = W.heisenberg(n)
    e_w, g_w = oracle.param_shift(n, gates, th, terms)
    e, g = lq.adjoint_grad(n, gates, th, terms)
    assert abs(e - e_w) <= RTOL * max(1, abs(e_w))
    np.testing.assert_allclose(g, g_w, rtol=0, atol=RTOL * max(1.0, np.abs(g_w).max()))


@pytest.mark.parametrize("n,seed", [(9, 5), (13, 6), (16, 7), (18, 8)])
def test_adjoint_diagonal_runs(lq, n, seed):
    rng = np.random.default_rng(seed)
    gates, P = diagonal_run_circuit(n, rng, layers=3 if n < 16 else 2 if n < 18 else 1)
    th = rng.uniform(-np.pi, np.pi, P)
    terms = W.random_pauli_sum(n, 20, rng, kmin=1, kmax=3)
    e_w, g_w = oracle.param_shift(n, gates, th, terms, general=True)
    e, g = lq.adjoint_grad(n, gates, th, terms)
    assert abs(e - e_w) <= RTOL * max(1, abs(e_w))
    np.testing.assert_allclose(g, g_w, rtol=0, atol=RTOL * max(1.0, np.abs(g_w).max()))
    if n == 13:
        idx = rng.choice(P, 12, replace=False)
        fd = oracle.finite_diff(n, gates, th, terms, h=1e-4, which=idx)
        np.testing.assert_allclose(g[idx], fd, rtol=0, atol=1e-6)


def _appd_rows():
    rows = []
    with open(os.path.join(os.path.dirname(__file__), "golden", "appD_psr_table.txt")) as f:
        for ln in f:
            if ln.strip() and not ln.startswith("#"):
                left, right = ln.split("|")
                name = left.split()[0]
                rows.append((name, [float(v) for v in right.split()]))
    return rows


@pytest.mark.parametrize("name,want", _appd_rows())
def test_appD_table_on_gpu(lq, name, want):
    gates, P, H = W.appd_circuit()
    th = W.APPD_ANGLE_SETS[name]
    tol = 2e-10 if name == "near_zero" else 5e-5
    e, g = lq.adjoint_grad(2, gates, th, H)
    np.testing.assert_allclose(g, want, rtol=0, atol=tol)
    e2, g2 = lq.param_shift_grad_general(2, gates, th, H)
    np.testing.assert_allclose(g2, want, rtol=0, atol=tol)
    _, g_w = oracle.param_shift(2, gates, th, H, general=True)
    np.testing.assert_allclose(g, g_w, rtol=0, atol=1e-12)
    np.testing.assert_allclose(g2, g_w, rtol=0, atol=1e-12)


@pytest.mark.parametrize("n,seed", [(3, 5), (6, 6), (11, 7)])
def test_general_parameter_shift(lq, n, seed):
    rng = np.random.default_rng(seed)
    gates = general_circuit(n, rng, ngates=25)
    th = rng.uniform(-np.pi, np.pi, 6)
    terms = W.random_pauli_sum(n, 12, rng, kmin=1, kmax=min(3, n))
    e_w, g_w = oracle.param_shift(n, gates, th, terms, general=True)
    e, g = lq.param_shift_grad_general(n, gates, th, terms)
    assert abs(e - e_w) <= RTOL * max(1, abs(e_w))
    np.testing.assert_allclose(g, g_w, rtol=0, atol=RTOL * max(1.0, np.abs(g_w).max()))


def test_autograd_function(lq):
    import torch

    n = 6
    gates, P = W.hea(n, 2, "ring")
    th = torch.tensor(W.angles(P, 8), dtype=torch.float64, requires_grad=True)
    terms = W.heisenberg(n)
    e = lq.energy(th, n, gates, terms)
    e.backward()
    e_w, g_w = oracle.param_shift(n, gates, th.detach().numpy(), terms)
    assert abs(e.item() - e_w) <= RTOL * max(1, abs(e_w))
    np.testing.assert_allclose(th.grad.numpy(), g_w, rtol=0, atol=RTOL)
    # chain rule through a downstream op
    th.grad = None
    (3.0 * lq.energy(th, n, gates, terms)).backward()
    np.testing.assert_allclose(th.grad.numpy(), 3.0 * g_w, rtol=0, atol=3 * RTOL)


def test_adjoint_vs_batched_psr_on_gpu(lq):
    # the configuration shape of the n=24 adjoint workload, at n=16: ladder
    # HEA, open-chain Heisenberg; adjoint vs batched PSR (1e-10), FD (1e-6)
    n, depth = 16, 3
    gates, P = W.hea(n, depth, "ladder")
    th = W.angles(P, 5)
    terms = W.heisenberg(n)
    e_a, g_a = lq.adjoint_grad(n, gates, th, terms)
    e_b, g_b = lq.param_shift_grad(n, gates, th, terms, method=lq.PSR_BATCHED)
    assert abs(e_a - e_b) <= RTOL * max(1, abs(e_b))
    np.testing.assert_allclose(g_a, g_b, rtol=0, atol=RTOL * max(1.0, np.abs(g_b).max()))
    which = list(range(0, P, 7))
    fd = oracle.finite_diff(n, gates, th, terms, h=1e-4, which=which)
    np.testing.assert_allclose(g_a[which], fd, rtol=0, atol=1e-6)
