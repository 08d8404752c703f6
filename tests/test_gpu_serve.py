"""The continuous-batching server: every result is the same alone and in the
mix (1e-10), and matches the oracle."""
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


def test_serve_mix_equals_alone(lq):
    import torch

    reqs = W.serve_requests(40, seed=6, nmin=3, nmax=15, dmin=1, dmax=4)
    arena = torch.empty(1 << 30, dtype=torch.uint8, device="cuda")
    srv = lq.Server(arena, slots=4)
    try:
        alone = []
        for r in reqs:
            rid = srv.submit(r["n"], r["gates"], r["params"], r["terms"], r["grad"])
            alone.append(srv.result(rid))
        ids = [srv.submit(r["n"], r["gates"], r["params"], r["terms"], r["grad"]) for r in reqs]
        mixed = [srv.result(i) for i in ids]
    finally:
        srv.close()
    for r, (ea, ga, ta), (em, gm, tm) in zip(reqs, alone, mixed):
        assert abs(ea - em) <= RTOL * max(1, abs(ea))
        if r["grad"]:
            np.testing.assert_allclose(gm, ga, rtol=0, atol=RTOL * max(1.0, np.abs(ga).max()))
        assert tm[0] <= tm[1] <= tm[2]
    for r, (e, g, _) in list(zip(reqs, mixed))[::7]:
        if r["grad"]:
            e_w, g_w = oracle.param_shift(r["n"], r["gates"], r["params"], r["terms"])
            np.testing.assert_allclose(g, g_w, rtol=0, atol=RTOL * max(1.0, np.abs(g_w).max()))
        else:
            e_w = oracle.energy(r["n"], r["gates"], r["params"], r["terms"])
        assert abs(e - e_w) <= RTOL * max(1, abs(e_w))


def test_serve_admission_limits(lq):
    import torch

    arena = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    srv = lq.Server(arena, slots=2)
    try:
        gates, P = W.hea(20, 1)
        with pytest.raises(lq.LqError) as ei:   # 16 MiB state > 1 MiB arena
            srv.submit(20, gates, W.angles(P, 1), W.heisenberg(20))
        assert ei.value.status == 4
        # requests that fit one at a time still all complete
        gates, P = W.hea(14, 2)
        ids = [srv.submit(14, gates, W.angles(P, s), W.heisenberg(14)) for s in range(6)]
        es = [srv.result(i)[0] for i in ids]
        for s, e in enumerate(es):
            assert abs(e - oracle.energy(14, gates, W.angles(P, s), W.heisenberg(14))) < 1e-10
    finally:
        srv.close()


def test_serve_wait_times_out_then_completes(lq):
    # one slot and three gradient requests: the last is still queued behind
    # the first two when it is waited for with a zero timeout, so the wait
    # reports LQ_ERR_TIMEOUT; the request stays queued and a second wait
    # returns its (correct) result
    import torch

    n = 20
    gates, P = W.hea(n, 4, "ladder")
    terms = W.heisenberg(n)
    arena = torch.empty(1 << 30, dtype=torch.uint8, device="cuda")
    srv = lq.Server(arena, slots=1)
    try:
        ids = [srv.submit(n, gates, W.angles(P, s), terms, True) for s in range(3)]
        with pytest.raises(lq.LqError) as ei:
            srv.result(ids[-1], timeout=0.0)
        assert ei.value.status == lq.LQ_ERR_TIMEOUT
        res = [srv.result(i) for i in ids]
    finally:
        srv.close()
    e_w = oracle.energy(n, gates, W.angles(P, 2), terms)
    assert abs(res[-1][0] - e_w) <= RTOL * max(1, abs(e_w))


def test_serve_requests_overlap_on_the_device(lq):
    # eight gradient requests on four slots (one stream each): some requests
    # are in flight at the same time (their [t_start, t_done] intervals
    # overlap), and every result equals the one the request gets alone
    import torch

    reqs = [dict(n=n, gates=W.hea(n, 3, "ring")[0], params=W.angles(W.hea(n, 3, "ring")[1], s),
                 terms=W.heisenberg(n), grad=True)
            for s, n in enumerate([16, 17, 18, 16, 17, 18, 16, 17])]
    arena = torch.empty(4 << 30, dtype=torch.uint8, device="cuda")
    srv = lq.Server(arena, slots=4)
    try:
        alone = []
        for r in reqs:
            alone.append(srv.result(srv.submit(r["n"], r["gates"], r["params"], r["terms"], True)))
        ids = [srv.submit(r["n"], r["gates"], r["params"], r["terms"], True) for r in reqs]
        mixed = [srv.result(i) for i in ids]
    finally:
        srv.close()
    spans = [(t[1], t[2]) for _, _, t in mixed]
    overlaps = sum(1 for i in range(len(spans)) for j in range(i + 1, len(spans))
                   if spans[i][0] < spans[j][1] and spans[j][0] < spans[i][1])
    assert overlaps >= 1, spans
    for (ea, ga, _), (em, gm, _) in zip(alone, mixed):
        assert abs(ea - em) <= RTOL * max(1, abs(ea))
        np.testing.assert_allclose(gm, ga, rtol=0, atol=RTOL * max(1.0, np.abs(ga).max()))
