"""Python binding of liblq, the sm_103a state-vector library of include/lq.h.

Argument marshalling only: gate lists and Pauli sums are packed into the C
structs of the ABI, torch tensors supply device memory and streams, and every
step of the computation runs in the library's CUDA kernels.  There is no CPU
fallback: if liblq.so cannot be loaded, ``lib()`` raises.

Gates are any objects with fields ``name, qubits, param, angle, mat`` (for
example ``workloads.Gate``); Pauli sums are lists of ``(coeff, "XYZI...")``
with character q acting on qubit q (qubit 0 = most significant index bit).
States are contiguous ``torch.complex128`` CUDA tensors of 2^n amplitudes.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblq.so")

c_int32, c_uint64, c_double, c_size_t = ctypes.c_int32, ctypes.c_uint64, ctypes.c_double, ctypes.c_size_t
c_void_p = ctypes.c_void_p


class LqGate(ctypes.Structure):
    _fields_ = [("kind", c_int32), ("qubits", c_int32 * 3), ("param", c_int32),
                ("reserved", c_int32), ("angle", c_double), ("mat", c_double * 32)]


class LqPauliTerm(ctypes.Structure):
    _fields_ = [("coeff", c_double), ("xmask", c_uint64), ("zmask", c_uint64)]


class LqTuneResult(ctypes.Structure):
    _fields_ = [("tile_bits", ctypes.c_int32), ("low_bits", ctypes.c_int32),
                ("phase_table", ctypes.c_int32), ("candidates", ctypes.c_int32),
                ("ms", c_double), ("ms_default", c_double)]


class LqPlanInfo(ctypes.Structure):
    _fields_ = [("npasses", c_int32), ("tile_bits", c_int32), ("dp_flops", c_double),
                ("dram_bytes", c_double)]


class LqProblem(ctypes.Structure):
    _fields_ = [("n", c_int32), ("ng", c_int32), ("np", c_int32), ("nt", c_int32),
                ("want_grad", c_int32), ("reserved", c_int32),
                ("gates", ctypes.POINTER(LqGate)), ("params", ctypes.POINTER(c_double)),
                ("terms", ctypes.POINTER(LqPauliTerm)), ("energy", ctypes.POINTER(c_double)),
                ("grad", ctypes.POINTER(c_double))]


class LqAdamOptions(ctypes.Structure):
    _fields_ = [("lr", c_double), ("beta1", c_double), ("beta2", c_double), ("eps", c_double),
                ("tol", c_double), ("max_iters", c_int32), ("method", c_int32)]


class LqRequest(ctypes.Structure):
    _fields_ = [("n", c_int32), ("ng", c_int32), ("np", c_int32), ("nt", c_int32),
                ("want_grad", c_int32), ("reserved", c_int32),
                ("gates", ctypes.POINTER(LqGate)), ("params", ctypes.POINTER(c_double)),
                ("terms", ctypes.POINTER(LqPauliTerm))]


class LqResult(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("status", c_int32), ("np", c_int32),
                ("energy", c_double), ("t_submit", c_double), ("t_start", c_double),
                ("t_done", c_double)]


# lq_gate_kind values of include/lq.h
KINDS = {name: i for i, name in enumerate(
    "H X Y Z S SDG T TDG RX RY RZ P U1 CNOT CY CZ CP SWAP CRX CRY CRZ RXX RYY RZZ CCX U2".split())}

LQ_ERR_TIMEOUT = 6
STATUS = {0: "LQ_OK", 1: "LQ_ERR_INVALID_ARG", 2: "LQ_ERR_UNSUPPORTED", 3: "LQ_ERR_NONFINITE",
          4: "LQ_ERR_OOM", 5: "LQ_ERR_CUDA", 6: "LQ_ERR_TIMEOUT"}
PSR_PLAIN, PSR_BATCHED = 0, 1
QFT_FFT, QFT_GATES = 0, 1


class LqError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


_lib = None

EXPORTS = [
    "lq_last_error", "lq_version", "lq_pauli_from_string", "lq_state_init", "lq_apply_circuit",
    "lq_qft", "lq_expval_workspace_size", "lq_expval_pauli_sum", "lq_expval_pauli_sum_async",
    "lq_apply_pauli_sum", "lq_param_shift_workspace_size", "lq_param_shift_grad",
    "lq_param_shift_general_workspace_size", "lq_param_shift_grad_general",
    "lq_adjoint_workspace_size", "lq_adjoint_grad", "lq_trotter_evolve",
    "lq_batch_workspace_size", "lq_batch_param_shift", "lq_circuit_plan", "lq_qft_plan", "lq_qft_plan_dir",
    "lq_expval_pauli_sum_noalloc", "lq_server_footprint", "lq_server_create",
    "lq_server_submit", "lq_server_wait", "lq_server_destroy", "lq_vqe_workspace_size",
    "lq_vqe_adam", "lq_adjoint_plan", "lq_expval_plan", "lq_autotune_circuit",
    "lq_tune_cache_save", "lq_tune_cache_load", "lq_tune_cache_clear", "lq_tune_cache_size",
    "lq_autotune_batch", "lq_autotune_param_shift", "lq_autotune_qft", "lq_measure_fp64_fma",
    "lq_measure_fp64_tile_sweep",
]


def load(build_if_missing=True):
    """Load liblq.so (building it in-tree with nvcc when it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        if not build_if_missing:
            raise ImportError("liblq.so is missing; run __graft_entry__.build()")
        _build.build()
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    L.lq_last_error.restype = ctypes.c_char_p
    L.lq_version.restype = ctypes.c_char_p
    L.lq_pauli_from_string.argtypes = [ctypes.c_char_p, ctypes.c_int, c_double, P(LqPauliTerm)]
    L.lq_state_init.argtypes = [c_void_p, ctypes.c_int, c_uint64, c_void_p]
    L.lq_apply_circuit.argtypes = [c_void_p, ctypes.c_int, P(LqGate), ctypes.c_int, P(c_double),
                                   ctypes.c_int, c_void_p]
    L.lq_qft.argtypes = [c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, c_void_p, c_size_t,
                         c_void_p]
    L.lq_expval_workspace_size.argtypes = [ctypes.c_int, ctypes.c_int]
    L.lq_expval_workspace_size.restype = c_size_t
    L.lq_expval_pauli_sum.argtypes = [c_void_p, ctypes.c_int, P(LqPauliTerm), ctypes.c_int,
                                      P(c_double), c_void_p, c_size_t, c_void_p]
    L.lq_expval_pauli_sum_async.argtypes = [c_void_p, ctypes.c_int, P(LqPauliTerm), ctypes.c_int,
                                            c_void_p, c_void_p, c_size_t, c_void_p]
    L.lq_apply_pauli_sum.argtypes = [c_void_p, c_void_p, ctypes.c_int, P(LqPauliTerm),
                                     ctypes.c_int, c_void_p]
    L.lq_param_shift_workspace_size.argtypes = [ctypes.c_int] * 4
    L.lq_param_shift_workspace_size.restype = c_size_t
    L.lq_param_shift_grad.argtypes = [ctypes.c_int, P(LqGate), ctypes.c_int, P(c_double),
                                      ctypes.c_int, P(LqPauliTerm), ctypes.c_int, ctypes.c_int,
                                      P(c_double), P(c_double), c_void_p, c_size_t, c_void_p]
    L.lq_param_shift_general_workspace_size.argtypes = [ctypes.c_int, P(LqGate), ctypes.c_int,
                                                        ctypes.c_int, ctypes.c_int]
    L.lq_param_shift_general_workspace_size.restype = c_size_t
    L.lq_param_shift_grad_general.argtypes = [ctypes.c_int, P(LqGate), ctypes.c_int, P(c_double),
                                              ctypes.c_int, P(LqPauliTerm), ctypes.c_int,
                                              P(c_double), P(c_double), c_void_p, c_size_t,
                                              c_void_p]
    L.lq_adjoint_workspace_size.argtypes = [ctypes.c_int] * 4
    L.lq_adjoint_workspace_size.restype = c_size_t
    L.lq_adjoint_grad.argtypes = [ctypes.c_int, P(LqGate), ctypes.c_int, P(c_double),
                                  ctypes.c_int, P(LqPauliTerm), ctypes.c_int, P(c_double),
                                  P(c_double), c_void_p, c_size_t, c_void_p]
    L.lq_trotter_evolve.argtypes = [c_void_p, ctypes.c_int, P(LqPauliTerm), ctypes.c_int,
                                    P(LqPauliTerm), ctypes.c_int, c_double, c_double, c_double,
                                    ctypes.c_int, c_void_p]
    L.lq_batch_workspace_size.argtypes = [P(LqProblem), ctypes.c_int]
    L.lq_batch_workspace_size.restype = c_size_t
    L.lq_batch_param_shift.argtypes = [P(LqProblem), ctypes.c_int, c_void_p, c_size_t, c_void_p]
    L.lq_vqe_workspace_size.argtypes = [ctypes.c_int] * 5
    L.lq_vqe_workspace_size.restype = c_size_t
    L.lq_vqe_adam.argtypes = [ctypes.c_int, P(LqGate), ctypes.c_int, P(c_double), ctypes.c_int,
                              P(LqPauliTerm), ctypes.c_int, P(LqAdamOptions), P(c_double),
                              P(ctypes.c_int), c_void_p, c_size_t, c_void_p]
    L.lq_server_footprint.argtypes = [ctypes.c_int] * 5
    L.lq_server_footprint.restype = c_size_t
    L.lq_server_create.argtypes = [c_void_p, c_size_t, ctypes.c_int, P(c_void_p)]
    L.lq_server_submit.argtypes = [c_void_p, P(LqRequest), P(ctypes.c_int64)]
    L.lq_server_wait.argtypes = [c_void_p, ctypes.c_int64, c_double, P(LqResult), P(c_double)]
    L.lq_server_destroy.argtypes = [c_void_p]
    L.lq_circuit_plan.argtypes = [ctypes.c_int, P(LqGate), ctypes.c_int, P(c_double), ctypes.c_int,
                                  P(LqPlanInfo)]
    L.lq_qft_plan.argtypes = [ctypes.c_int, ctypes.c_int, P(LqPlanInfo)]
    L.lq_qft_plan_dir.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P(LqPlanInfo)]
    L.lq_expval_plan.argtypes = [ctypes.c_int, P(LqPauliTerm), ctypes.c_int, P(LqPlanInfo)]
    L.lq_autotune_circuit.argtypes = [c_void_p, ctypes.c_int, P(LqGate), ctypes.c_int,
                                      P(c_double), ctypes.c_int, P(LqTuneResult), c_void_p]
    L.lq_autotune_batch.argtypes = [P(LqProblem), ctypes.c_int, c_void_p, c_size_t,
                                    P(LqTuneResult), c_void_p]
    L.lq_autotune_param_shift.argtypes = [ctypes.c_int, P(LqGate), ctypes.c_int, P(c_double),
                                          ctypes.c_int, P(LqPauliTerm), ctypes.c_int, c_void_p,
                                          c_size_t, P(LqTuneResult), c_void_p]
    L.lq_autotune_qft.argtypes = [c_void_p, ctypes.c_int, ctypes.c_int, P(LqTuneResult), c_void_p]
    L.lq_tune_cache_save.argtypes = [ctypes.c_char_p]
    L.lq_tune_cache_load.argtypes = [ctypes.c_char_p]
    L.lq_tune_cache_clear.argtypes = []
    L.lq_tune_cache_size.argtypes = []
    L.lq_tune_cache_size.restype = ctypes.c_int
    L.lq_measure_fp64_fma.argtypes = [ctypes.c_int, P(c_double), P(c_double), c_void_p]
    L.lq_measure_fp64_tile_sweep.argtypes = [ctypes.c_int, P(c_double), P(c_double), c_void_p]
    L.lq_adjoint_plan.argtypes = [ctypes.c_int, P(LqGate), ctypes.c_int, P(c_double), ctypes.c_int,
                                  ctypes.c_int, P(LqPlanInfo)]
    _lib = L
    return L


lib = load


def _check(st):
    if st != 0:
        raise LqError(st, load().lq_last_error().decode())


def version():
    return load().lq_version().decode()


def measure_fp64_fma(reps=5, stream=None):
    """Measured FP64 FMA rate of the current device: (TFLOP/s, ms of the best
    launch)."""
    tf, ms = c_double(), c_double()
    _check(load().lq_measure_fp64_fma(int(reps), ctypes.byref(tf), ctypes.byref(ms),
                                      _stream(stream)))
    return tf.value, ms.value


def measure_fp64_tile_sweep(reps=5, stream=None):
    """Measured FP64 rate of shared-memory tile sweeps (rotations on a
    2^12-amplitude tile, the tile passes' access pattern): (TFLOP/s, ms of the
    best launch)."""
    tf, ms = c_double(), c_double()
    _check(load().lq_measure_fp64_tile_sweep(int(reps), ctypes.byref(tf), ctypes.byref(ms),
                                             _stream(stream)))
    return tf.value, ms.value


# ------------------------------------------------------------- marshalling

# numpy layout of lq_gate (the struct is filled column-wise, then viewed by ctypes)
_GATE_DTYPE = np.dtype([("kind", "<i4"), ("qubits", "<i4", (3,)), ("param", "<i4"),
                        ("reserved", "<i4"), ("angle", "<f8"), ("mat", "<f8", (32,))])


_GATE_CACHE = {}


def pack_gates(gates):
    """The gate list as a ctypes lq_gate array (sharing one numpy buffer); the
    packing of a given gate sequence is kept (gates carry no parameter
    values, so an optimisation loop passes the same sequence every call)."""
    try:
        key = tuple(gates)
        hash(key)
    except TypeError:   # a gate with a matrix (numpy array) is not hashable
        key = None
    if key is not None:
        hit = _GATE_CACHE.get(key)
        if hit is not None:
            return hit
    arr = _pack_gates(gates)
    if key is not None:
        if len(_GATE_CACHE) > 64:
            _GATE_CACHE.clear()
        _GATE_CACHE[key] = arr
    return arr


def _pack_gates(gates):
    m = len(gates)
    a = np.zeros(max(m, 1), _GATE_DTYPE)
    if m:
        a["kind"][:m] = [KINDS[g.name] for g in gates]
        a["qubits"][:m] = [tuple(g.qubits) + (-1,) * (3 - len(g.qubits)) for g in gates]
        a["param"][:m] = [g.param for g in gates]
        a["angle"][:m] = [g.angle for g in gates]
        for i, g in enumerate(gates):
            if g.mat is not None:
                v = np.ascontiguousarray(np.asarray(g.mat, np.complex128).reshape(-1)).view(np.float64)
                a["mat"][i, : v.size] = v
    return (LqGate * a.size).from_buffer(a)


_TERM_CACHE = {}


def pack_terms(terms, n):
    """The Pauli sum as a ctypes lq_pauli_term array; the packing of a given
    (terms, n) is kept (a VQE loop passes the same Hamiltonian every call)."""
    try:
        key = (n, tuple((float(c), str(s)) for c, s in terms))
    except (TypeError, ValueError):
        key = None
    if key is not None and key in _TERM_CACHE:
        return _TERM_CACHE[key]
    arr = (LqPauliTerm * max(len(terms), 1))()
    L = load()
    for i, (c, s) in enumerate(terms):
        _check(L.lq_pauli_from_string(s.encode(), n, float(c), ctypes.byref(arr[i])))
    if key is not None:
        if len(_TERM_CACHE) > 64:
            _TERM_CACHE.clear()
        _TERM_CACHE[key] = arr
    return arr


def _params(params):
    p = np.ascontiguousarray(np.asarray(params if params is not None else [], np.float64))
    return p, p.ctypes.data_as(ctypes.POINTER(c_double)), int(p.size)


def _stream(stream):
    import torch

    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _check_state(amps, n):
    import torch

    if not (amps.is_cuda and amps.dtype == torch.complex128 and amps.is_contiguous()):
        raise ValueError("state must be a contiguous complex128 CUDA tensor")
    if amps.numel() != (1 << n):
        raise ValueError("state has %d amplitudes, expected 2^%d" % (amps.numel(), n))


def _workspace(nbytes, device):
    import torch

    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


# --------------------------------------------------------------- entry points

def new_state(n, basis=0, device="cuda", stream=None):
    import torch

    amps = torch.empty(1 << n, dtype=torch.complex128, device=device)
    state_init(amps, n, basis, stream)
    return amps


def state_init(amps, n, basis=0, stream=None):
    _check_state(amps, n)
    _check(load().lq_state_init(_ptr(amps), n, int(basis), _stream(stream)))
    return amps


def apply_circuit(amps, n, gates, params=None, stream=None):
    _check_state(amps, n)
    g = pack_gates(gates)
    p, pp, np_ = _params(params)
    _check(load().lq_apply_circuit(_ptr(amps), n, g, len(gates), pp, np_, _stream(stream)))
    return amps


def qft(amps, n, inverse=False, method=QFT_FFT, stream=None):
    _check_state(amps, n)
    _check(load().lq_qft(_ptr(amps), n, int(inverse), int(method), None, 0, _stream(stream)))
    return amps


def expval_pauli_sum(amps, n, terms, stream=None, workspace=None):
    _check_state(amps, n)
    L = load()
    t = pack_terms(terms, n)
    need = L.lq_expval_workspace_size(n, len(terms))
    ws = workspace if workspace is not None else _workspace(need, amps.device)
    out = c_double(0.0)
    _check(L.lq_expval_pauli_sum(_ptr(amps), n, t, len(terms), ctypes.byref(out), _ptr(ws),
                                 ws.numel(), _stream(stream)))
    return out.value


def apply_pauli_sum(out, amps, n, terms, stream=None):
    _check_state(amps, n)
    _check_state(out, n)
    t = pack_terms(terms, n)
    _check(load().lq_apply_pauli_sum(_ptr(out), _ptr(amps), n, t, len(terms), _stream(stream)))
    return out


def param_shift_grad(n, gates, params, terms, method=PSR_BATCHED, device="cuda", stream=None,
                     workspace=None):
    """(E, grad) by the parameter-shift rule (two-term rule, single-use
    parameters)."""
    L = load()
    g = pack_gates(gates)
    t = pack_terms(terms, n)
    p, pp, np_ = _params(params)
    need = L.lq_param_shift_workspace_size(n, np_, len(terms), int(method))
    ws = workspace if workspace is not None else _workspace(need, device)
    e = c_double(0.0)
    grad = np.zeros(max(np_, 1))
    _check(L.lq_param_shift_grad(n, g, len(gates), pp, np_, t, len(terms), int(method),
                                 ctypes.byref(e), grad.ctypes.data_as(ctypes.POINTER(c_double)),
                                 _ptr(ws), ws.numel(), _stream(stream)))
    return e.value, grad[:np_].copy()


def param_shift_grad_general(n, gates, params, terms, device="cuda", stream=None):
    """(E, grad) with shared parameters and four-term rules for controlled
    rotations."""
    L = load()
    g = pack_gates(gates)
    t = pack_terms(terms, n)
    p, pp, np_ = _params(params)
    need = L.lq_param_shift_general_workspace_size(n, g, len(gates), np_, len(terms))
    ws = _workspace(need, device)
    e = c_double(0.0)
    grad = np.zeros(max(np_, 1))
    _check(L.lq_param_shift_grad_general(n, g, len(gates), pp, np_, t, len(terms), ctypes.byref(e),
                                         grad.ctypes.data_as(ctypes.POINTER(c_double)), _ptr(ws),
                                         ws.numel(), _stream(stream)))
    return e.value, grad[:np_].copy()


def adjoint_grad(n, gates, params, terms, device="cuda", stream=None, workspace=None):
    """(E, grad) by reverse-mode (adjoint) differentiation."""
    L = load()
    g = pack_gates(gates)
    t = pack_terms(terms, n)
    p, pp, np_ = _params(params)
    need = L.lq_adjoint_workspace_size(n, len(gates), np_, len(terms))
    ws = workspace if workspace is not None else _workspace(need, device)
    e = c_double(0.0)
    grad = np.zeros(max(np_, 1))
    _check(L.lq_adjoint_grad(n, g, len(gates), pp, np_, t, len(terms), ctypes.byref(e),
                             grad.ctypes.data_as(ctypes.POINTER(c_double)), _ptr(ws), ws.numel(),
                             _stream(stream)))
    return e.value, grad[:np_].copy()


def trotter_evolve(amps, n, terms, field_terms, A, omega, dt, steps, stream=None):
    _check_state(amps, n)
    t = pack_terms(terms, n)
    f = pack_terms(field_terms, n)
    _check(load().lq_trotter_evolve(_ptr(amps), n, t, len(terms), f, len(field_terms), float(A),
                                    float(omega), float(dt), int(steps), _stream(stream)))
    return amps


def circuit_plan(n, gates, params=None):
    """dict(npasses, tile_bits, dp_flops, dram_bytes) of lq_apply_circuit."""
    g = pack_gates(gates)
    p, pp, np_ = _params(params)
    info = LqPlanInfo()
    _check(load().lq_circuit_plan(n, g, len(gates), pp, np_, ctypes.byref(info)))
    return dict(npasses=info.npasses, tile_bits=info.tile_bits, dp_flops=info.dp_flops,
                dram_bytes=info.dram_bytes)


def adjoint_plan(n, gates, params, nt):
    g = pack_gates(gates)
    p, pp, np_ = _params(params)
    info = LqPlanInfo()
    _check(load().lq_adjoint_plan(n, g, len(gates), pp, np_, int(nt), ctypes.byref(info)))
    return dict(npasses=info.npasses, tile_bits=info.tile_bits, dp_flops=info.dp_flops,
                dram_bytes=info.dram_bytes)


def autotune(n, gates, params=None, scratch=None, stream=None):
    """Time the tile schedules of apply_circuit for this circuit on a scratch
    state (allocated when not given) and record the fastest for every circuit
    of the same structure on this GPU; returns the choice and its timing."""
    if scratch is None:
        scratch = new_state(n)
    _check_state(scratch, n)
    g = pack_gates(gates)
    p, pp, np_ = _params(params)
    r = LqTuneResult()
    _check(load().lq_autotune_circuit(_ptr(scratch), n, g, len(gates), pp, np_, ctypes.byref(r),
                                      _stream(stream)))
    return dict(tile_bits=r.tile_bits, low_bits=r.low_bits, phase_table=r.phase_table,
                candidates=r.candidates, ms=r.ms, ms_default=r.ms_default)


def _tune_dict(r):
    return dict(tile_bits=r.tile_bits, low_bits=r.low_bits, phase_table=r.phase_table,
                candidates=r.candidates, ms=r.ms, ms_default=r.ms_default)


def autotune_batch(problems, device="cuda", stream=None, workspace=None):
    """Pick the tile width of the persistent batched launch for this batch
    structure (states larger than shared memory); returns the choice."""
    L = load()
    arr, keep = _problem_array(problems)
    need = L.lq_batch_workspace_size(arr, len(problems))
    ws = workspace if workspace is not None else _workspace(need, device)
    r = LqTuneResult()
    _check(L.lq_autotune_batch(arr, len(problems), _ptr(ws), ws.numel(), ctypes.byref(r),
                               _stream(stream)))
    return _tune_dict(r)


def autotune_param_shift(n, gates, params, terms, device="cuda", stream=None, workspace=None):
    """Pick the tile width of the batched parameter-shift launch of this
    circuit structure; returns the choice."""
    L = load()
    g = pack_gates(gates)
    t = pack_terms(terms, n)
    p, pp, np_ = _params(params)
    need = L.lq_param_shift_workspace_size(n, np_, len(terms), PSR_BATCHED)
    ws = workspace if workspace is not None else _workspace(need, device)
    r = LqTuneResult()
    _check(L.lq_autotune_param_shift(n, g, len(gates), pp, np_, t, len(terms), _ptr(ws),
                                     ws.numel(), ctypes.byref(r), _stream(stream)))
    return _tune_dict(r)


def autotune_qft(n, inverse=False, scratch=None, stream=None):
    """Pick the schedule of the gate-form QFT (forward or inverse) on this
    GPU; qft(..., method=QFT_GATES) then uses it."""
    if scratch is None:
        scratch = new_state(n)
    _check_state(scratch, n)
    r = LqTuneResult()
    _check(load().lq_autotune_qft(_ptr(scratch), n, int(inverse), ctypes.byref(r),
                                  _stream(stream)))
    return _tune_dict(r)


def tune_cache_save(path):
    _check(load().lq_tune_cache_save(os.fsencode(path)))


def tune_cache_load(path):
    _check(load().lq_tune_cache_load(os.fsencode(path)))


def tune_cache_clear():
    _check(load().lq_tune_cache_clear())


def tune_cache_size():
    return int(load().lq_tune_cache_size())


def expval_plan(n, terms):
    """dict(npasses, tile_bits, dp_flops, dram_bytes) of lq_expval_pauli_sum."""
    pt = pack_terms(terms, n)
    info = LqPlanInfo()
    _check(load().lq_expval_plan(n, pt, len(terms), ctypes.byref(info)))
    return dict(npasses=info.npasses, tile_bits=info.tile_bits, dp_flops=info.dp_flops,
                dram_bytes=info.dram_bytes)


def qft_plan(n, method=QFT_FFT, inverse=False):
    info = LqPlanInfo()
    _check(load().lq_qft_plan_dir(n, int(method), int(inverse), ctypes.byref(info)))
    return dict(npasses=info.npasses, tile_bits=info.tile_bits, dp_flops=info.dp_flops,
                dram_bytes=info.dram_bytes)


class BatchProblem:
    """One problem of an uneven batch: its circuit, parameters and Pauli sum."""

    def __init__(self, n, gates, params, terms, want_grad=True):
        self.n, self.gates, self.terms, self.want_grad = n, gates, terms, want_grad
        self.params = np.ascontiguousarray(np.asarray(params, np.float64))
        self.energy = None
        self.grad = None


def _problem_array(problems):
    arr = (LqProblem * len(problems))()
    keep = []
    for i, pb in enumerate(problems):
        g = pack_gates(pb.gates)
        t = pack_terms(pb.terms, pb.n)
        e = np.zeros(1)
        gr = np.zeros(max(pb.params.size, 1))
        keep.append((g, t, e, gr, pb.params))
        P = arr[i]
        P.n, P.ng, P.np, P.nt = pb.n, len(pb.gates), pb.params.size, len(pb.terms)
        P.want_grad = int(pb.want_grad)
        P.gates = g
        P.params = pb.params.ctypes.data_as(ctypes.POINTER(c_double))
        P.terms = t
        P.energy = e.ctypes.data_as(ctypes.POINTER(c_double))
        P.grad = gr.ctypes.data_as(ctypes.POINTER(c_double))
    return arr, keep


def batch_param_shift(problems, device="cuda", stream=None, workspace=None):
    """Run many (n, circuit, H) problems' parameter-shift circuits in one
    batched launch; fills problem.energy / problem.grad."""
    L = load()
    arr, keep = _problem_array(problems)
    need = L.lq_batch_workspace_size(arr, len(problems))
    ws = workspace if workspace is not None else _workspace(need, device)
    _check(L.lq_batch_param_shift(arr, len(problems), _ptr(ws), ws.numel(), _stream(stream)))
    for pb, (g, t, e, gr, _) in zip(problems, keep):
        pb.energy = float(e[0])
        pb.grad = gr[: pb.params.size].copy()
    return problems


def vqe_adam(n, gates, params, terms, lr=1e-2, max_iters=350, tol=1e-7, method=0,
             beta1=0.9, beta2=0.999, eps=1e-8, device="cuda", stream=None):
    """Minimise E(theta) with Adam (Sec. VI-B settings by default).  Returns
    (final params, energies per iteration)."""
    L = load()
    g = pack_gates(gates)
    t = pack_terms(terms, n)
    p = np.array(params, np.float64, copy=True)
    need = L.lq_vqe_workspace_size(n, len(gates), p.size, len(terms), int(method))
    ws = _workspace(need, device)
    opt = LqAdamOptions(lr, beta1, beta2, eps, tol, int(max_iters), int(method))
    es = np.zeros(max_iters)
    it = ctypes.c_int(0)
    _check(L.lq_vqe_adam(n, g, len(gates), p.ctypes.data_as(ctypes.POINTER(c_double)), p.size, t,
                         len(terms), ctypes.byref(opt), es.ctypes.data_as(ctypes.POINTER(c_double)),
                         ctypes.byref(it), _ptr(ws), ws.numel(), _stream(stream)))
    return p, es[: it.value].copy()


class Server:
    """Continuous-batching request server over a device arena (a torch uint8
    CUDA tensor the caller keeps alive).  submit() queues a request and
    returns its id; result(id) waits and returns (energy, grad or None,
    (t_submit, t_start, t_done))."""

    def __init__(self, arena, slots=4):
        self.arena = arena
        h = c_void_p()
        _check(load().lq_server_create(_ptr(arena), arena.numel(), int(slots), ctypes.byref(h)))
        self.h = h
        self._np = {}

    def submit(self, n, gates, params, terms, want_grad=False):
        L = load()
        g = pack_gates(gates)
        t = pack_terms(terms, n)
        p = np.ascontiguousarray(np.asarray(params, np.float64))
        q = LqRequest(n, len(gates), p.size, len(terms), int(want_grad), 0, g,
                      p.ctypes.data_as(ctypes.POINTER(c_double)), t)
        rid = ctypes.c_int64()
        _check(L.lq_server_submit(self.h, ctypes.byref(q), ctypes.byref(rid)))
        self._np[rid.value] = (p.size, want_grad)
        return rid.value

    def result(self, rid, timeout=600.0):
        """Waits up to `timeout` seconds; LqError with LQ_ERR_TIMEOUT when the
        request is not done by then (it stays queued: wait again later)."""
        np_, want_grad = self._np[rid]
        res = LqResult()
        grad = np.zeros(max(np_, 1))
        st = load().lq_server_wait(self.h, rid, float(timeout), ctypes.byref(res),
                                   grad.ctypes.data_as(ctypes.POINTER(c_double)))
        if st != LQ_ERR_TIMEOUT:
            del self._np[rid]
        _check(st)
        return res.energy, (grad[:np_].copy() if want_grad else None), (res.t_submit, res.t_start,
                                                                       res.t_done)

    def close(self):
        if getattr(self, "h", None):
            load().lq_server_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()


def server_footprint(n, want_grad, ng, np_, nt):
    return load().lq_server_footprint(n, int(want_grad), ng, np_, nt)


from .autograd import AdjointEnergy, energy  # noqa: E402,F401
