"""The allocation-free <H> entry point, lq_expval_pauli_sum_noalloc.

It is meant for callers that cannot allocate device memory (for example code
inside a host application whose device memory belongs to another allocator),
so it keeps its partial sums in a fixed array inside the library instead of a
caller workspace.  The tests call it through the C ABI twice in a row -- the
second call starts from whatever the first left in the shared array -- and
check both results against lq_expval_pauli_sum and against the oracle's
per-term <H> (Sec. VI-A), for a mixed sum, a sum of diagonal terms only, and
a sum at the entry point's limit of distinct X masks; plus the size limits.
This file is collected last so a failure here cannot hide the other tests.
"""
import ctypes

import numpy as np
import pytest

import oracle
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


def _diagonal_sum(n, count, rng):
    """Z strings only (one group, X mask 0), coefficients N(0, 1)."""
    return [(float(rng.standard_normal()),
             "".join("Z" if rng.random() < 0.4 else "I" for _ in range(n)))
            for _ in range(count)]


def _many_x_masks(n, groups, rng):
    """One term per distinct nonzero X mask (groups - 1 of them, qubits of the
    mask carrying X or Y, the others I or Z) plus a few diagonal terms: a sum
    with exactly `groups` distinct X masks."""
    masks = rng.choice(np.arange(1, 1 << n), size=groups - 1, replace=False)
    terms = []
    for m in masks:
        s = []
        for q in range(n):
            if (int(m) >> (n - 1 - q)) & 1:
                s.append("XY"[rng.integers(2)])
            else:
                s.append("IZ"[rng.integers(2)])
        terms.append((float(rng.standard_normal()), "".join(s)))
    return terms + _diagonal_sum(n, 5, rng)


def _sums():
    rng = np.random.default_rng(31)
    return {
        "mixed": (14, W.heisenberg(14) + W.random_pauli_sum(14, 60, rng, kmin=1, kmax=4)),
        "diagonal": (12, _diagonal_sum(12, 40, rng)),
        "240_x_masks": (12, _many_x_masks(12, 240, rng)),
    }


@pytest.mark.parametrize("case", ["mixed", "diagonal", "240_x_masks"])
def test_noalloc_expval_matches_workspace_version_and_oracle_twice(case):
    import torch

    import paper_2512_23183_gb300 as lq

    L, f = _entry(lq)
    n, terms = _sums()[case]
    packed = lq.pack_terms(terms, n)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for seed in (1, 2):
        x = W.gaussian_state(n, seed)
        psi = torch.from_numpy(x).cuda()
        want = lq.expval_pauli_sum(psi, n, terms)
        exact = oracle.expval(x, n, terms)
        out = ctypes.c_double(float("nan"))
        st = f(ctypes.c_void_p(psi.data_ptr()), n, packed, len(terms), ctypes.byref(out), stream)
        assert st == 0, L.lq_last_error()
        assert abs(out.value - want) <= RTOL * max(1.0, abs(want)), (seed, out.value, want)
        assert abs(out.value - exact) <= RTOL * max(1.0, abs(exact)), (seed, out.value, exact)


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


def test_noalloc_rejects_more_distinct_x_masks_than_its_group_table():
    import torch

    import paper_2512_23183_gb300 as lq

    L, f = _entry(lq)
    n = 12
    terms = _many_x_masks(n, 242, np.random.default_rng(9))
    packed = lq.pack_terms(terms, n)
    psi = torch.from_numpy(W.gaussian_state(n, 4)).cuda()
    out = ctypes.c_double()
    st = f(ctypes.c_void_p(psi.data_ptr()), n, packed, len(terms), ctypes.byref(out), None)
    assert st == 1
    assert b"at most 240 distinct X masks" in L.lq_last_error()
