"""Parity at the workloads' full sizes, in the launch configuration bench.py
times: sampled outputs the oracle computes one by one, closed forms, and
properties that hold at any size.

  - QFT n = 28 (Gaussian input: sampled amplitudes by the oracle's
    one-amplitude DFT) and n = 30 (basis input: closed form; Gaussian input:
    sampled amplitudes of both forms by the oracle's one-amplitude DFT,
    inverse round trip, norm);
  - VQE n = 10 depth 4, 80 angles seed 1: energy and full gradient;
  - batched PSR n = 16 depth 8 ring, 256 angles seed 3: energy by the oracle,
    sampled gradient entries by oracle energies at +-pi/2;
  - adjoint n = 24 depth 10, 480 angles seed 5: energy and the first and
    last gradient entries by the oracle, sampled entries against GPU
    parameter shift (1e-10) and central differences (h = 1e-4, 1e-6), every
    entry against the batched parameter-shift launch;
  - uneven batch: a sample of the 64 seeded instances against the oracle.
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


def _close(a, b, tol=RTOL):
    return abs(a - b) <= tol * max(1.0, abs(b))


def test_qft_n28_gaussian_sampled(lq):
    import torch

    n = 28
    psi = W.gaussian_state(n, 1000 + n)
    t = torch.from_numpy(psi).cuda()
    lq.qft(t, n)
    ks = [0, 1, 12345678, (1 << n) - 1]
    got = t[ks].cpu().numpy()
    for k, g in zip(ks, got):
        assert abs(g - oracle.qft_amplitude(psi, n, k)) < ATOL, k
    del t


def test_qft_n30_basis_closed_form_and_properties(lq):
    import torch

    n = 30
    N = 1 << n
    x = W.basis_index(n, 2000 + n)
    t = lq.new_state(n, x)
    lq.qft(t, n)
    k = np.random.default_rng(n).integers(0, N, 8192)
    got = t[torch.from_numpy(k).cuda()].cpu().numpy()
    want = np.exp(2j * np.pi * ((x * k) % N) / N) / np.sqrt(N)
    np.testing.assert_allclose(got, want, rtol=0, atol=ATOL)
    # gate form on the same input agrees with the FFT form, element-wise
    t2 = lq.new_state(n, x)
    lq.qft(t2, n, method=lq.QFT_GATES)
    assert float((t2 - t).abs().max()) < ATOL
    del t2
    # inverse round trip restores the basis state; norm is preserved
    lq.qft(t, n, inverse=True)
    assert abs(float(torch.linalg.vector_norm(t)) - 1.0) < 1e-12
    t[x] -= 1.0
    assert float(t.abs().max()) < ATOL
    del t


def _device_gaussian(n, seed):
    """The n-qubit seeded Gaussian input drawn on the device (i.i.d. N(0, 1)
    real and imaginary parts from a seeded torch CUDA generator, then
    L2-normalised), as the benchmark draws its 16 GiB input."""
    import torch

    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    v = torch.randn(2 << n, dtype=torch.float64, device="cuda", generator=g)
    psi = torch.view_as_complex(v.view(-1, 2))
    psi /= torch.linalg.vector_norm(psi)
    return psi


def test_qft_n30_gaussian_sampled_both_forms(lq):
    # n = 30 Gaussian input: amplitudes of both forms (forward) against the
    # oracle's one-amplitude DFT on a host copy of the same input
    import torch

    n = 30
    psi = _device_gaussian(n, 1000 + n)
    x = psi.cpu().numpy()
    del psi
    ks = [0, 1, 0x2AAAAAAB, (1 << n) - 1]
    want = np.array([oracle.qft_amplitude(x, n, k) for k in ks])
    idx = torch.tensor(ks, device="cuda")
    for meth in (lq.QFT_FFT, lq.QFT_GATES):
        t = torch.from_numpy(x).cuda()
        lq.qft(t, n, method=meth)
        got = t[idx].cpu().numpy()
        del t
        np.testing.assert_allclose(got, want, rtol=0, atol=ATOL, err_msg=str(meth))


def test_qft_n30_gaussian_round_trip(lq):
    import torch

    n = 30
    psi = _device_gaussian(n, 1000 + n)
    ref = psi.clone()
    lq.qft(psi, n)
    assert abs(float(torch.linalg.vector_norm(psi)) - 1.0) < 1e-12
    lq.qft(psi, n, inverse=True, method=lq.QFT_GATES)
    assert float((psi - ref).abs().max()) < ATOL
    del psi, ref


def test_vqe_n10_config_exact(lq):
    gates, th, terms = W.vqe_chain(10, 4, 1)
    e_w, g_w = oracle.param_shift(10, gates, th, terms)
    for meth in (lq.PSR_PLAIN, lq.PSR_BATCHED):
        e, g = lq.param_shift_grad(10, gates, th, terms, method=meth)
        assert _close(e, e_w)
        np.testing.assert_allclose(g, g_w, rtol=0, atol=RTOL * max(1.0, np.abs(g_w).max()))
    e, g = lq.adjoint_grad(10, gates, th, terms)
    assert _close(e, e_w)
    np.testing.assert_allclose(g, g_w, rtol=0, atol=RTOL * max(1.0, np.abs(g_w).max()))


def test_batched_psr_n16_ring_config_sampled(lq):
    gates, th, terms = W.vqe_ring(16, 8, 3)
    e, g = lq.param_shift_grad(16, gates, th, terms, method=lq.PSR_BATCHED)
    assert _close(e, oracle.energy(16, gates, th, terms))
    for i in (0, 77, 255):
        p = th.copy()
        p[i] += np.pi / 2
        ep = oracle.energy(16, gates, p, terms)
        p[i] -= np.pi
        em = oracle.energy(16, gates, p, terms)
        assert abs(g[i] - 0.5 * (ep - em)) <= RTOL * max(1.0, abs(g[i])), i


def test_adjoint_n24_config_sampled(lq):
    import torch

    n = 24
    gates, P = W.hea(n, 10, "ladder")
    th = W.angles(P, 5)
    terms = W.heisenberg(n)
    e, g = lq.adjoint_grad(n, gates, th, terms)
    ws = torch.empty(lq.load().lq_expval_workspace_size(n, len(terms)), dtype=torch.uint8,
                     device="cuda")

    def energy(p):
        t = lq.new_state(n)
        lq.apply_circuit(t, n, gates, p)
        return lq.expval_pauli_sum(t, n, terms, workspace=ws)

    assert _close(e, energy(th))
    # RY and RZ gates of first, middle and last layers (local and CTA bits)
    for i in (0, 191, 250, 325, 479):
        p = th.copy()
        p[i] += np.pi / 2
        ep = energy(p)
        p[i] -= np.pi
        em = energy(p)
        assert abs(g[i] - 0.5 * (ep - em)) <= RTOL * max(1.0, abs(g[i])), i
        p = th.copy()
        p[i] += 1e-4
        fp = energy(p)
        p[i] -= 2e-4
        fm = energy(p)
        assert abs(g[i] - (fp - fm) / 2e-4) < 1e-6, i
    # the energy itself by the oracle (one evaluation at 2^24 amplitudes), and
    # the first and last gradient entries by the oracle's energies at +-pi/2
    assert _close(e, oracle.energy(n, gates, th, terms))
    for i in (0, P - 1):
        p = th.copy()
        p[i] += np.pi / 2
        ep = oracle.energy(n, gates, p, terms)
        p[i] -= np.pi
        em = oracle.energy(n, gates, p, terms)
        assert abs(g[i] - 0.5 * (ep - em)) <= RTOL * max(1.0, abs(g[i])), i


def test_uneven_batch_config_sample(lq):
    inst = W.uneven_batch(count=64, seed=4)
    probs = [lq.BatchProblem(n, g, th, t) for n, g, th, t in inst]
    lq.batch_param_shift(probs)
    small = [i for i, (n, _, _, _) in enumerate(inst) if n <= 9][:3]
    for i in small:
        n, g, th, t = inst[i]
        e_w, g_w = oracle.param_shift(n, g, th, t)
        assert _close(probs[i].energy, e_w)
        np.testing.assert_allclose(probs[i].grad, g_w, rtol=0,
                                   atol=RTOL * max(1.0, np.abs(g_w).max()))
    # the largest instance: energy by the oracle, one gradient entry
    j = max(range(len(inst)), key=lambda i: inst[i][0])
    n, g, th, t = inst[j]
    assert _close(probs[j].energy, oracle.energy(n, g, th, t))
    p = th.copy()
    p[3] += np.pi / 2
    ep = oracle.energy(n, g, p, t)
    p[3] -= np.pi
    em = oracle.energy(n, g, p, t)
    assert abs(probs[j].grad[3] - 0.5 * (ep - em)) <= RTOL * max(1.0, abs(probs[j].grad[3]))


def test_adjoint_vs_batched_psr_n24_config(lq):
    # the adjoint workload as configured (n = 24, depth-10 ladder, 480 angles
    # seed 5, open chain): the adjoint gradient against the batched
    # parameter-shift gradient (all 961 circuits in one persistent launch) on
    # every entry, and the batched energy against the oracle
    import torch

    n = 24
    gates, P = W.hea(n, 10, "ladder")
    th = W.angles(P, 5)
    terms = W.heisenberg(n)
    ea, ga = lq.adjoint_grad(n, gates, th, terms)
    ws = torch.empty(lq.load().lq_param_shift_workspace_size(n, P, len(terms), lq.PSR_BATCHED),
                     dtype=torch.uint8, device="cuda")
    eb, gb = lq.param_shift_grad(n, gates, th, terms, method=lq.PSR_BATCHED, workspace=ws)
    del ws
    torch.cuda.empty_cache()
    assert _close(ea, eb)
    np.testing.assert_allclose(ga, gb, rtol=0, atol=RTOL * max(1.0, np.abs(gb).max()))
    assert _close(eb, oracle.energy(n, gates, th, terms))
