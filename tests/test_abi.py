"""The C-ABI library builds, loads and exports every symbol include/lq.h
declares; host-side validation answers without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "lq.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lq_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    import paper_2512_23183_gb300 as lq

    return lq.load()


def test_exports_every_declared_symbol(L):
    names = header_functions()
    assert len(names) >= 18
    for name in names:
        assert hasattr(L, name), name
    import paper_2512_23183_gb300 as lq

    assert sorted(lq.EXPORTS) == names


def test_binding_gate_kinds_match_header():
    import paper_2512_23183_gb300 as lq

    src = open(os.path.join(ROOT, "include", "lq.h")).read()
    body = src[src.index("typedef enum {\n  LQ_H = 0"):]
    body = body[: body.index("} lq_gate_kind;")]
    names = re.findall(r"\bLQ_([A-Z0-9]+)\b", body)
    names = [n for n in names if n != "GATE_KIND_COUNT"]
    assert [lq.KINDS[n] for n in names] == list(range(len(names)))


def test_version_and_pauli_parsing(L):
    import paper_2512_23183_gb300 as lq

    assert b"sm_103a" in L.lq_version()
    t = lq.LqPauliTerm()
    assert L.lq_pauli_from_string(b"XIYZ", 4, 0.5, ctypes.byref(t)) == 0
    # qubit q is bit n-1-q: X on q0 -> bit 3, Y on q2 -> bit 1, Z on q3 -> bit 0
    assert (t.coeff, t.xmask, t.zmask) == (0.5, 0b1010, 0b0011)
    assert L.lq_pauli_from_string(b"XQ", 2, 1.0, ctypes.byref(t)) == 1
    assert L.lq_pauli_from_string(b"XX", 3, 1.0, ctypes.byref(t)) == 1
    assert L.lq_pauli_from_string(b"XX", 2, float("nan"), ctypes.byref(t)) == 3
    assert b"not finite" in L.lq_last_error()


def _gate(name, *qubits, param=-1, angle=0.0):
    from workloads import G

    return G(name, *qubits, param=param, angle=angle)


@pytest.mark.parametrize(
    "gates,params,status",
    [
        ([("RX", (5,), -1, 0.1)], [], 1),          # qubit out of range
        ([("CNOT", (1, 1), -1, 0.0)], [], 1),      # repeated qubit
        ([("RY", (0,), 3, 0.0)], [0.1], 1),        # parameter index >= np
        ([("H", (0,), 0, 0.0)], [0.1], 1),         # parameter on a fixed gate
        ([("RZ", (0,), 0, 0.0)], [float("nan")], 3),  # non-finite parameter
        ([("RZ", (0,), -1, float("inf"))], [], 3),    # non-finite angle
    ],
)
def test_apply_circuit_validation_on_host(L, gates, params, status):
    import paper_2512_23183_gb300 as lq

    gl = [_gate(n, *q, param=p, angle=a) for n, q, p, a in gates]
    g = lq.pack_gates(gl)
    p = np.asarray(params, np.float64)
    pp = p.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    # a non-NULL dummy pointer: validation must fail before any device access
    st = L.lq_apply_circuit(ctypes.c_void_p(16), 3, g, len(gl), pp, p.size, None)
    assert st == status, L.lq_last_error()


def test_n_range_and_null_pointers(L):
    assert L.lq_state_init(ctypes.c_void_p(16), 0, 0, None) == 1
    assert L.lq_state_init(ctypes.c_void_p(16), 35, 0, None) == 1
    assert L.lq_state_init(None, 3, 0, None) == 1
    assert L.lq_state_init(ctypes.c_void_p(16), 3, 8, None) == 1  # basis >= 2^n
    assert L.lq_qft(ctypes.c_void_p(16), 3, 0, 7, None, 0, None) == 1
    assert L.lq_expval_workspace_size(10, 3) > 0


def test_batched_workspace_sizing_on_host(L):
    # sizing a batched launch plans every problem on the host (lowering,
    # tile passes, the tiled <H> plan of states wider than a tile) and needs
    # no device: without one the grid is an estimate, with one the occupancy
    # query decides; the scratch states make the size grow with n
    import paper_2512_23183_gb300 as lq

    sizes = [L.lq_param_shift_workspace_size(n, 4 * n, 3 * (n - 1), lq.PSR_BATCHED)
             for n in (10, 13, 16, 20)]
    assert all(s > 0 for s in sizes), sizes
    assert sizes == sorted(sizes) and sizes[-1] > sizes[0], sizes


def test_probes_reject_bad_arguments_on_host(L):
    tf = ctypes.c_double()
    for fn in (L.lq_measure_fp64_fma, L.lq_measure_fp64_tile_sweep):
        assert fn(0, ctypes.byref(tf), None, None) == 1       # reps < 1
        assert fn(1001, ctypes.byref(tf), None, None) == 1    # reps > 1000
        assert fn(1, None, None, None) == 1                   # no output


def test_psr_rejects_unsupported_on_host(L):
    import paper_2512_23183_gb300 as lq

    terms = lq.pack_terms([(1.0, "ZI")], 2)
    p = np.array([0.1])
    pp = p.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    e = ctypes.c_double()
    gr = np.zeros(1)
    grp = gr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    # CRY needs the four-term rule
    g = lq.pack_gates([_gate("CRY", 0, 1, param=0)])
    st = L.lq_param_shift_grad(2, g, 1, pp, 1, terms, 1, 1, ctypes.byref(e), grp,
                               ctypes.c_void_p(256), 1 << 30, None)
    assert st == 2 and b"generalised" in L.lq_last_error()
    # a parameter shared by two gates
    g = lq.pack_gates([_gate("RX", 0, param=0), _gate("RY", 1, param=0)])
    st = L.lq_param_shift_grad(2, g, 2, pp, 1, terms, 1, 1, ctypes.byref(e), grp,
                               ctypes.c_void_p(256), 1 << 30, None)
    assert st == 2
    # workspace too small
    g = lq.pack_gates([_gate("RX", 0, param=0)])
    st = L.lq_param_shift_grad(2, g, 1, pp, 1, terms, 1, 1, ctypes.byref(e), grp,
                               ctypes.c_void_p(256), 8, None)
    assert st == 4


def test_gate_packing_layout_and_cache():
    """pack_gates fills the lq_gate layout (numpy columns viewed by ctypes),
    including matrices, and returns the same packing for an equal gate list."""
    import paper_2512_23183_gb300 as lq
    import workloads as W

    assert lq._GATE_DTYPE.itemsize == ctypes.sizeof(lq.LqGate)
    for name, _ctype in lq.LqGate._fields_:
        assert lq._GATE_DTYPE.fields[name][1] == getattr(lq.LqGate, name).offset, name
    rng = np.random.default_rng(5)
    gates, _ = W.random_circuit(6, 40, rng)
    arr = lq.pack_gates(gates)
    for i, g in enumerate(gates):
        assert arr[i].kind == lq.KINDS[g.name]
        q = list(arr[i].qubits)
        assert q[: len(g.qubits)] == list(g.qubits) and all(v == -1 for v in q[len(g.qubits):])
        assert arr[i].param == g.param and arr[i].angle == g.angle
        if g.mat is not None:
            m = np.asarray(g.mat, np.complex128).reshape(-1).view(np.float64)
            assert np.array_equal(np.array(arr[i].mat[: m.size]), m)
    hea, _ = W.hea(5, 2, "ring")
    a1 = lq.pack_gates(hea)
    assert lq.pack_gates(list(hea)) is a1          # equal sequence: kept packing
    assert lq.pack_gates(hea[:-1]) is not a1
    t1 = lq.pack_terms(W.heisenberg(5), 5)
    assert lq.pack_terms(W.heisenberg(5), 5) is t1
    assert lq.pack_terms(W.heisenberg(5, ring=True), 5) is not t1
