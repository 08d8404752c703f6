"""The schedule autotuner on the GPU: the chosen schedule is at least as
fast as the default on the same call, is used by apply_circuit and
circuit_plan for every circuit of the same structure, gives results equal to
the oracle's, and survives a save / clear / load of the cache."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

ATOL = 1e-12


@pytest.fixture(scope="module")
def lq():
    import paper_2512_23183_gb300 as m

    m.load()
    m.tune_cache_clear()
    yield m
    m.tune_cache_clear()


def _dev(psi):
    import torch

    return torch.from_numpy(np.ascontiguousarray(psi)).cuda()


@pytest.mark.parametrize("n,depth", [(14, 2), (18, 1)])
def test_autotune_choice_and_parity(lq, n, depth, tmp_path):
    gates, P = W.hea(n, depth, "ring")
    r = lq.autotune(n, gates, W.angles(P, 3))
    assert r["candidates"] >= 4
    assert 9 <= r["tile_bits"] <= 12 and r["low_bits"] in (3, 4, 5, 6)
    assert r["low_bits"] >= 5 or r["tile_bits"] >= 11   # short low runs with 2^11, 2^12 tiles
    assert r["ms"] <= r["ms_default"]
    assert lq.circuit_plan(n, gates, W.angles(P, 4))["tile_bits"] == r["tile_bits"]
    # the tuned schedule serves other parameter values of the same structure
    for seed in (4, 5):
        th = W.angles(P, seed)
        psi = W.gaussian_state(n, seed)
        t = _dev(psi)
        lq.apply_circuit(t, n, gates, th)
        want = oracle.apply_circuit(psi.copy(), n, gates, th)
        np.testing.assert_allclose(t.cpu().numpy(), want, rtol=0, atol=ATOL)
    # save, clear, load: the same choice comes back
    f = tmp_path / "tune.txt"
    lq.tune_cache_save(str(f))
    lq.tune_cache_clear()
    assert lq.tune_cache_size() == 0
    lq.tune_cache_load(str(f))
    assert lq.circuit_plan(n, gates, W.angles(P, 4))["tile_bits"] == r["tile_bits"]


@pytest.mark.parametrize("m", [1, 3, 4])
def test_short_low_runs_parity(lq, tune_entry, m):
    """Schedules with 2^12 tiles and short contiguous low runs (m = 1 is
    widened to 3 by the pass kernel's 9-bit offset table): 2^9 tiles of an
    n = 21 state whose passes map up to 9 tile bits above the low run,
    results equal to the oracle's."""
    n = 21
    gates, P = W.hea(n, 2, "ring")
    tune_entry(n, gates, 12, m, 0)
    assert lq.circuit_plan(n, gates, W.angles(P, 7))["tile_bits"] == 12
    th = W.angles(P, 7)
    psi = W.gaussian_state(n, 11)
    t = _dev(psi)
    lq.apply_circuit(t, n, gates, th)
    want = oracle.apply_circuit(psi.copy(), n, gates, th)
    np.testing.assert_allclose(t.cpu().numpy(), want, rtol=0, atol=ATOL)


@pytest.mark.parametrize("m", [3, 4])
def test_short_low_runs_inverse_gate_qft(lq, tune_entry, m):
    """The inverse gate-form QFT (butterfly passes) with 2^11 tiles and a 3-
    or 4-bit low run, n = 22: equal to the oracle's inverse DFT."""
    from conftest import inverse_qft_gates

    n = 22
    tune_entry(n, inverse_qft_gates(n), 11, m, 1)
    assert lq.qft_plan(n, lq.QFT_GATES, inverse=True)["tile_bits"] == 11
    psi = W.gaussian_state(n, 5000 + m)
    t = _dev(psi)
    lq.qft(t, n, inverse=True, method=lq.QFT_GATES)
    want = oracle.qft_fft(psi.copy(), n, inverse=True)
    np.testing.assert_allclose(t.cpu().numpy(), want, rtol=0, atol=ATOL)


def test_autotune_qft_gate_circuit(lq):
    # a circuit with merged dyadic and one-bit phases
    n = 15
    gates = []
    for i in range(n):
        gates.append(W.G("H", i))
        for j in range(i + 1, min(n, i + 5)):
            gates.append(W.G("CP", i, j, angle=np.pi / 2 ** (j - i)))
        gates.append(W.G("RZ", i, param=i))
    th = W.angles(n, 9)
    r = lq.autotune(n, gates, th)
    psi = W.gaussian_state(n, 12)
    t = _dev(psi)
    lq.apply_circuit(t, n, gates, th)
    want = oracle.apply_circuit(psi.copy(), n, gates, th)
    np.testing.assert_allclose(t.cpu().numpy(), want, rtol=0, atol=ATOL)
    assert r["ms"] <= r["ms_default"]


def test_autotune_param_shift_batch_tiles(lq):
    # n = 14 > shared memory: the batched launch runs tiles of the tuned width
    gates, th, terms = W.vqe_ring(14, 3, 2)
    e0, g0 = lq.param_shift_grad(14, gates, th, terms, method=lq.PSR_BATCHED)
    r = lq.autotune_param_shift(14, gates, th, terms)
    assert r["candidates"] == 4 and 9 <= r["tile_bits"] <= 12
    assert r["ms"] <= r["ms_default"]
    e, g = lq.param_shift_grad(14, gates, th, terms, method=lq.PSR_BATCHED)
    assert abs(e - e0) <= 1e-10 * max(1.0, abs(e0))
    np.testing.assert_allclose(g, g0, rtol=0, atol=1e-10 * max(1.0, np.abs(g0).max()))
    assert abs(e - oracle.energy(14, gates, th, terms)) <= 1e-10 * max(1.0, abs(e))
    for i in (0, len(th) - 1):
        p = th.copy()
        p[i] += np.pi / 2
        ep = oracle.energy(14, gates, p, terms)
        p[i] -= np.pi
        em = oracle.energy(14, gates, p, terms)
        assert abs(g[i] - 0.5 * (ep - em)) <= 1e-10 * max(1.0, abs(g[i]))


def test_autotune_uneven_batch(lq):
    inst = W.uneven_batch(count=12, seed=9)
    probs = [lq.BatchProblem(n, g, th, t) for n, g, th, t in inst]
    r = lq.autotune_batch(probs)
    big = any(n > 12 for n, _, _, _ in inst)
    assert r["candidates"] == (4 if big else 1)
    lq.batch_param_shift(probs)
    for i, (n, g, th, t) in enumerate(inst):
        if n <= 9:
            e_w, g_w = oracle.param_shift(n, g, th, t)
            assert abs(probs[i].energy - e_w) <= 1e-10 * max(1.0, abs(e_w))
            np.testing.assert_allclose(probs[i].grad, g_w, rtol=0,
                                       atol=1e-10 * max(1.0, np.abs(g_w).max()))
    # a batch of small states has nothing to tune
    small = [lq.BatchProblem(n, g, th, t) for n, g, th, t in inst if n <= 12][:3]
    assert lq.autotune_batch(small)["candidates"] == 1


def test_autotune_qft_gate_form(lq):
    import torch

    n = 16
    r = lq.autotune_qft(n, inverse=True)
    assert r["ms"] <= r["ms_default"]
    psi = W.gaussian_state(n, 21)
    t = _dev(psi)
    lq.qft(t, n, inverse=True, method=lq.QFT_GATES)
    want = np.fft.fft(psi, norm="ortho")   # the inverse QFT: e^{-2 pi i xk/N} / sqrt(N)
    np.testing.assert_allclose(t.cpu().numpy(), want, rtol=0, atol=ATOL)
    assert lq.qft_plan(n, lq.QFT_GATES)["npasses"] >= 2
    del torch


def test_autotune_inverse_gate_qft_keeps_dyadic_tables(lq):
    # the table option also switches the merged dyadic phases' tables (the
    # gate-form QFT's butterflies); the tuner must time 2^11 and 2^12 tiles
    # with them: at n = 26 the best schedule keeps them, beats the default,
    # and the transform still equals the oracle's inverse DFT
    n = 26
    r = lq.autotune_qft(n, inverse=True)
    lq_plan = lq.qft_plan(n, lq.QFT_GATES, inverse=True)
    assert r["phase_table"] == 1 and r["ms"] <= r["ms_default"]
    assert lq_plan["tile_bits"] == r["tile_bits"]
    psi = W.gaussian_state(n, 1000 + n)
    t = _dev(psi)
    lq.qft(t, n, inverse=True, method=lq.QFT_GATES)
    want = oracle.qft_fft(psi.copy(), n, inverse=True)
    np.testing.assert_allclose(t.cpu().numpy(), want, rtol=0, atol=ATOL)
    lq.tune_cache_clear()
