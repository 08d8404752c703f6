"""VQE outer loop (Sec. VI-B): the library's Adam loop follows, iteration by
iteration, an independent Adam (Kingma & Ba) written here and fed with the
oracle's parameter-shift gradients; energies stay above the exact ground
energy (variational bound) and decrease."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


def reference_adam(n, gates, theta, terms, iters, lr=1e-2, b1=0.9, b2=0.999, eps=1e-8):
    th = np.array(theta, float)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    es = []
    for t in range(1, iters + 1):
        e, g = oracle.param_shift(n, gates, th, terms)
        es.append(e)
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g * g
        th = th - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
    return th, np.array(es)


@pytest.mark.parametrize("method", [0, 1])
def test_vqe_adam_follows_reference(method):
    import paper_2512_23183_gb300 as lq

    n, depth = 4, 2
    gates, P = W.hea(n, depth, "ladder")
    th0 = W.angles(P, 12)
    terms = W.heisenberg(n)
    th, es = lq.vqe_adam(n, gates, th0, terms, max_iters=40, tol=0.0, method=method)
    th_w, es_w = reference_adam(n, gates, th0, terms, 40)
    assert es.size == 40
    # energies within the 1e-10 relative energy tolerance; the parameters
    # Adam derives from the gradients within the same bound
    np.testing.assert_allclose(es, es_w, rtol=0, atol=1e-10 * max(1.0, np.abs(es_w).max()))
    np.testing.assert_allclose(th, th_w, rtol=0, atol=1e-10)


def test_vqe_adam_converges_above_ground_energy():
    import paper_2512_23183_gb300 as lq

    n, depth = 6, 3
    gates, P = W.hea(n, depth, "ladder")
    terms = W.heisenberg(n)
    from functools import reduce

    PAULI = {"I": np.eye(2), "X": np.array([[0, 1], [1, 0]]), "Y": np.array([[0, -1j], [1j, 0]]),
             "Z": np.diag([1.0, -1.0])}
    H = sum(c * reduce(np.kron, [PAULI[ch] for ch in s]) for c, s in terms)
    e0 = np.linalg.eigvalsh(H).min()
    th, es = lq.vqe_adam(n, gates, W.angles(P, 3), terms, max_iters=350, tol=1e-7)
    assert 1 < es.size <= 350
    assert es.min() >= e0 - 1e-12
    assert es[-1] < es[0] - 0.5
    # the returned parameters reproduce the last energy's neighbourhood
    e_final = oracle.energy(n, gates, th, terms)
    assert e_final >= e0 - 1e-12 and abs(e_final - es[-1]) < 1e-2
