"""Uneven batches in one persistent launch: every problem's energy and
parameter-shift gradient against the oracle (1e-10)."""
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


def test_uneven_batch_small(lq):
    rng = np.random.default_rng(21)
    probs, wants = [], []
    for i, (n, d) in enumerate([(1, 2), (3, 1), (8, 2), (11, 2), (12, 1), (13, 1), (14, 1),
                                (5, 3)]):
        gates, P = W.hea(n, d, "ring")
        th = rng.uniform(-np.pi, np.pi, P)
        terms = W.random_pauli_sum(n, 20, rng, kmin=1, kmax=min(4, n)) if n > 1 else \
            [(0.7, "Z"), (-0.2, "X")]
        want_grad = i % 3 != 2
        probs.append(lq.BatchProblem(n, gates, th, terms, want_grad=want_grad))
        if want_grad:
            wants.append(oracle.param_shift(n, gates, th, terms))
        else:
            wants.append((oracle.energy(n, gates, th, terms), None))
    lq.batch_param_shift(probs)
    for pb, (e_w, g_w) in zip(probs, wants):
        assert abs(pb.energy - e_w) <= RTOL * max(1, abs(e_w)), (pb.n, pb.energy, e_w)
        if g_w is not None:
            np.testing.assert_allclose(pb.grad, g_w, rtol=0,
                                       atol=RTOL * max(1.0, np.abs(g_w).max()))


def test_uneven_batch_generator_shape(lq):
    # the seeded 64-instance generator, restricted to small n so the oracle
    # stays fast; checks a sample of the instances
    inst = W.uneven_batch(count=12, seed=4, nmin=4, nmax=12, dmin=1, dmax=3, nterms=50)
    probs = [lq.BatchProblem(n, g, th, t) for n, g, th, t in inst]
    lq.batch_param_shift(probs)
    for (n, g, th, t), pb in list(zip(inst, probs))[::3]:
        e_w, g_w = oracle.param_shift(n, g, th, t)
        assert abs(pb.energy - e_w) <= RTOL * max(1, abs(e_w))
        np.testing.assert_allclose(pb.grad, g_w, rtol=0, atol=RTOL * max(1.0, np.abs(g_w).max()))


def test_batched_psr_n16_ring(lq):
    n, depth = 16, 1
    gates, P = W.hea(n, depth, "ring")
    th = W.angles(P, 3)
    terms = W.heisenberg(n, ring=True)
    e_w, g_w = oracle.param_shift(n, gates, th, terms)
    e, g = lq.param_shift_grad(n, gates, th, terms, method=lq.PSR_BATCHED)
    assert abs(e - e_w) <= RTOL * max(1, abs(e_w))
    np.testing.assert_allclose(g, g_w, rtol=0, atol=RTOL * max(1.0, np.abs(g_w).max()))


@pytest.mark.parametrize("n,depth,kind", [(13, 3, "ring"), (14, 2, "ladder")])
def test_batched_psr_tiled_multilayer(lq, n, depth, kind):
    # states wider than the 2^12 shared-memory tile run as tile passes over a
    # scratch state; several layers let the phases sink across passes, and
    # every shifted circuit's patch must still reach its own gate's factor
    gates, P = W.hea(n, depth, kind)
    th = W.angles(P, 40 + n)
    terms = W.heisenberg(n, ring=kind == "ring")
    e_w, g_w = oracle.param_shift(n, gates, th, terms)
    e, g = lq.param_shift_grad(n, gates, th, terms, method=lq.PSR_BATCHED)
    assert abs(e - e_w) <= RTOL * max(1, abs(e_w))
    np.testing.assert_allclose(g, g_w, rtol=0, atol=RTOL * max(1.0, np.abs(g_w).max()))


def test_batched_after_workspace_reallocation(lq):
    """A replayed launch must follow its workspace: free the workspace and
    hand the memory back to the driver, allocate again (the address usually
    repeats) and the batched gradient still matches the oracle."""
    import torch

    n, depth = 10, 4
    gates, P = W.hea(n, depth, "ladder")
    terms = W.heisenberg(n)
    need = lq.load().lq_param_shift_workspace_size(n, P, len(terms), lq.PSR_BATCHED)
    addrs = []
    for rep in range(4):
        th = W.angles(P, 60 + rep)
        ws = torch.empty(need, dtype=torch.uint8, device="cuda")
        addrs.append(ws.data_ptr())
        e, g = lq.param_shift_grad(n, gates, th, terms, method=lq.PSR_BATCHED, workspace=ws)
        e_w, g_w = oracle.param_shift(n, gates, th, terms)
        assert abs(e - e_w) <= RTOL * max(1, abs(e_w)), rep
        np.testing.assert_allclose(g, g_w, rtol=0, atol=RTOL * max(1.0, np.abs(g_w).max()))
        del ws
        # other allocations come and go, then the cache is returned to the driver
        big = torch.empty(1 << 28, dtype=torch.uint8, device="cuda")
        del big
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    assert len(addrs) == 4
