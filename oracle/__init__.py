"""ctypes wrapper of the plain CPU oracle (lq_oracle.c).

TEST INFRASTRUCTURE.  Only tests/, ``__graft_entry__.smoke()`` and the cpu
baseline of ``bench.py`` may import this package.  It shares no code with the
CUDA library and never imports it.

Circuits are lists of ``workloads.Gate`` (name, qubits, param, angle, mat);
Pauli sums are lists of ``(coeff, "XYZI...")`` with character q acting on
qubit q.  States are C-contiguous numpy complex128 arrays of 2^n amplitudes,
qubit q at bit n-1-q of the index (MSB-first, Alg. 1).
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lq_oracle.c")
_LIB = os.path.join(_HERE, "liblq_oracle.so")

# Oracle-private gate codes (same order as the enum in lq_oracle.c).
GATE_CODES = {
    name: i
    for i, name in enumerate(
        "H X Y Z S SDG T TDG RX RY RZ P U1 CNOT CY CZ CP SWAP CRX CRY CRZ "
        "RXX RYY RZZ CCX U2".split()
    )
}

OK, EINVAL, EUNSUPPORTED = 0, 1, 2


class OracleError(RuntimeError):
    pass


class OracleUnsupported(OracleError):
    pass


def build(force=False):
    """Compile lq_oracle.c into liblq_oracle.so with gcc (-fopenmp)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-std=gnu11", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.or_gate_matrix.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp]
        L.or_apply_matrix.argtypes = [_dp, ctypes.c_int, _ip, ctypes.c_int, _dp]
        L.or_state_basis.argtypes = [_dp, ctypes.c_int, ctypes.c_uint64]
        L.or_cnot_alg1.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.or_toffoli_alg4.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        circ = [_ip, _ip, _ip, _dp, _dp, ctypes.c_int]
        L.or_apply_circuit.argtypes = [_dp, ctypes.c_int] + circ + [_dp, ctypes.c_int]
        L.or_expval.argtypes = [_dp, ctypes.c_int, ctypes.c_char_p, _dp, ctypes.c_int, _dp]
        ham = [ctypes.c_char_p, _dp, ctypes.c_int]
        L.or_energy.argtypes = [ctypes.c_int] + circ + [_dp, ctypes.c_int] + ham + [_dp]
        L.or_param_shift.argtypes = [ctypes.c_int] + circ + [_dp, ctypes.c_int] + ham + [ctypes.c_int, _dp, _dp]
        L.or_finite_diff.argtypes = (
            [ctypes.c_int] + circ + [_dp, ctypes.c_int] + ham + [ctypes.c_double, _ip, ctypes.c_int, _dp]
        )
        L.or_qft_fft.argtypes = [_dp, ctypes.c_int, ctypes.c_int]
        L.or_qft_gates.argtypes = [_dp, ctypes.c_int]
        L.or_qft_amplitude.argtypes = [_dp, ctypes.c_int, ctypes.c_uint64, _dp]
        L.or_trotter.argtypes = (
            [_dp, ctypes.c_int] + ham + ham
            + [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int]
        )
        L.or_norm2.argtypes = [_dp, ctypes.c_int]
        L.or_norm2.restype = ctypes.c_double
        _lib = L
    return _lib


def _check(rc):
    if rc == EUNSUPPORTED:
        raise OracleUnsupported("oracle: unsupported gradient setting")
    if rc != OK:
        raise OracleError("oracle: invalid argument (rc=%d)" % rc)


def _dptr(a):
    return a.ctypes.data_as(_dp)


def _iptr(a):
    return a.ctypes.data_as(_ip)


def _state_ptr(psi):
    assert psi.dtype == np.complex128 and psi.flags.c_contiguous
    return psi.ctypes.data_as(_dp)


def _circuit(gates):
    ng = len(gates)
    kinds = np.zeros(max(ng, 1), np.int32)
    qubits = np.full(3 * max(ng, 1), -1, np.int32)
    pidx = np.full(max(ng, 1), -1, np.int32)
    angles = np.zeros(max(ng, 1), np.float64)
    mats = np.zeros(32 * max(ng, 1), np.float64)
    for i, g in enumerate(gates):
        kinds[i] = GATE_CODES[g.name]
        for j, q in enumerate(g.qubits):
            qubits[3 * i + j] = q
        pidx[i] = g.param
        angles[i] = g.angle
        if g.mat is not None:
            m = np.asarray(g.mat, np.complex128).reshape(-1)
            mats[32 * i: 32 * i + 2 * m.size] = m.view(np.float64)
    keep = (kinds, qubits, pidx, angles, mats)
    args = [_iptr(kinds), _iptr(qubits), _iptr(pidx), _dptr(angles), _dptr(mats), ng]
    return keep, args


def _hamiltonian(terms, n):
    for c, s in terms:
        assert len(s) == n, "Pauli string length must equal n"
    strs = "".join(s for _, s in terms).encode()
    coeffs = np.array([c for c, _ in terms] or [0.0], np.float64)
    return (strs, coeffs), [strs, _dptr(coeffs), len(terms)]


def _params(params):
    p = np.ascontiguousarray(np.asarray(params if params is not None else [], np.float64))
    if p.size == 0:
        p = np.zeros(1)
        return p, 0
    return p, int(np.asarray(params).size)


def gate_matrix(name, theta=0.0, mat=None):
    code = GATE_CODES[name]
    um = np.zeros(32)
    if mat is not None:
        m = np.asarray(mat, np.complex128).reshape(-1)
        um[: 2 * m.size] = m.view(np.float64)
    out = np.zeros(2 * 64)
    rc = lib().or_gate_matrix(code, theta, _dptr(um), _dptr(out))
    _check(rc)
    arity = 3 if name == "CCX" else (2 if name in ("CNOT", "CY", "CZ", "CP", "SWAP", "CRX", "CRY", "CRZ", "RXX", "RYY", "RZZ", "U2") else 1)
    d = 1 << arity
    return out[: 2 * d * d].view(np.complex128).reshape(d, d).copy()


def basis_state(n, x=0):
    psi = np.empty(1 << n, np.complex128)
    lib().or_state_basis(_state_ptr(psi), n, x)
    return psi


def apply_matrix(psi, n, qubits, M):
    q = np.array(qubits, np.int32)
    M = np.ascontiguousarray(np.asarray(M, np.complex128))
    lib().or_apply_matrix(_state_ptr(psi), n, _iptr(q), len(qubits), M.ctypes.data_as(_dp))
    return psi


def cnot_alg1(psi, n, c, t):
    lib().or_cnot_alg1(_state_ptr(psi), n, c, t)
    return psi


def toffoli_alg4(psi, n, c1, c2, t):
    lib().or_toffoli_alg4(_state_ptr(psi), n, c1, c2, t)
    return psi


def apply_circuit(psi, n, gates, params=None):
    keep, cargs = _circuit(gates)
    p, np_ = _params(params)
    _check(lib().or_apply_circuit(_state_ptr(psi), n, *cargs, _dptr(p), np_))
    return psi


def expval(psi, n, terms):
    keep, hargs = _hamiltonian(terms, n)
    out = np.zeros(1)
    _check(lib().or_expval(_state_ptr(psi), n, *hargs, _dptr(out)))
    return float(out[0])


def energy(n, gates, params, terms):
    keep, cargs = _circuit(gates)
    hk, hargs = _hamiltonian(terms, n)
    p, np_ = _params(params)
    out = np.zeros(1)
    _check(lib().or_energy(n, *cargs, _dptr(p), np_, *hargs, _dptr(out)))
    return float(out[0])


def param_shift(n, gates, params, terms, general=False):
    """(E, grad) by the parameter-shift rule; general=True enables the
    four-term rule for controlled rotations and shared parameters."""
    keep, cargs = _circuit(gates)
    hk, hargs = _hamiltonian(terms, n)
    p, np_ = _params(params)
    grad = np.zeros(max(np_, 1))
    e0 = np.zeros(1)
    _check(lib().or_param_shift(n, *cargs, _dptr(p), np_, *hargs, int(general), _dptr(e0), _dptr(grad)))
    return float(e0[0]), grad[:np_].copy()


def finite_diff(n, gates, params, terms, h=1e-4, which=None):
    keep, cargs = _circuit(gates)
    hk, hargs = _hamiltonian(terms, n)
    p, np_ = _params(params)
    w = np.array(range(np_) if which is None else which, np.int32)
    out = np.zeros(max(w.size, 1))
    _check(lib().or_finite_diff(n, *cargs, _dptr(p), np_, *hargs, h, _iptr(w), int(w.size), _dptr(out)))
    return out[: w.size].copy()


def qft_fft(psi, n, inverse=False):
    _check(lib().or_qft_fft(_state_ptr(psi), n, int(inverse)))
    return psi


def qft_gates(psi, n):
    _check(lib().or_qft_gates(_state_ptr(psi), n))
    return psi


def qft_amplitude(psi, n, k):
    out = np.zeros(2)
    _check(lib().or_qft_amplitude(_state_ptr(psi), n, int(k), _dptr(out)))
    return complex(out[0], out[1])


def trotter(psi, n, terms, field_terms, A, omega, dt, steps):
    hk, hargs = _hamiltonian(terms, n)
    fk, fargs = _hamiltonian(field_terms, n)
    _check(lib().or_trotter(_state_ptr(psi), n, *hargs, *fargs, A, omega, dt, steps))
    return psi


def norm2(psi, n):
    return lib().or_norm2(_state_ptr(psi), n)
