"""The allocation-free <H> entry point, lq_expval_pauli_sum_noalloc.

It is meant for callers that cannot allocate device memory (for example code
inside a host application whose device memory belongs to another allocator),
so it keeps its partial sums in a fixed array inside the library instead of a
caller workspace.  The test calls it through the C ABI twice in a row -- the
second call starts from whatever the first left in the shared array -- and
checks both results against lq_expval_pauli_sum, plus the size limit.  This
file is collected last so a failure here cannot hide the other tests.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-10


def _entry(lq):
    L = lq.load()
    f = L.lq_expval_pauli_sum_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(lq.LqPauliTerm), ctypes.c_int,
                  ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    f.restype = ctypes.c_int
    return L, f


def test_noalloc_expval_matches_workspace_version_twice():
    import torch

    import paper_2512_23183_gb300 as lq

    L, f = _entry(lq)
    n = 14
    rng = np.random.default_rng(31)
    terms = W.heisenberg(n) + W.random_pauli_sum(n, 60, rng, kmin=1, kmax=4)
    packed = lq.pack_terms(terms, n)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for seed in (1, 2):
        psi = torch.from_numpy(W.gaussian_state(n, seed)).cuda()
        want = lq.expval_pauli_sum(psi, n, terms)
        out = ctypes.c_double(float("nan"))
        st = f(ctypes.c_void_p(psi.data_ptr()), n, packed, len(terms), ctypes.byref(out), stream)
        assert st == 0, L.lq_last_error()
        assert abs(out.value - want) <= RTOL * max(1.0, abs(want)), (seed, out.value, want)


def test_noalloc_rejects_sums_beyond_its_fixed_scratch():
    import torch

    import paper_2512_23183_gb300 as lq

    L, f = _entry(lq)
    n = 6
    rng = np.random.default_rng(5)
    terms = W.random_pauli_sum(n, 700, rng, kmin=1, kmax=4)
    packed = lq.pack_terms(terms, n)
    psi = torch.from_numpy(W.gaussian_state(n, 3)).cuda()
    out = ctypes.c_double()
    st = f(ctypes.c_void_p(psi.data_ptr()), n, packed, len(terms), ctypes.byref(out), None)
    assert st == 1
    assert b"at most 640 terms" in L.lq_last_error()
