import os
import struct
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def gpu_available():
    try:
        import torch

        return torch.cuda.is_available()
    except Exception:
        return False


def pytest_collection_modifyitems(config, items):
    if gpu_available():
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


def _gpu_key():
    """The autotune cache's device key: "<name>|<SM count>" of the current
    device, or "unknown" without one."""
    import torch

    if not torch.cuda.is_available():
        return "unknown"
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return p.name.replace(" ", "_").replace("\t", "_") + "|%d" % p.multi_processor_count


def _structure_hash(n, packed):
    """FNV-1a (64-bit) over n and each gate's (kind, qubits, has-parameter)
    record, plus the angle of a gate without a parameter: the cache's key for
    a circuit structure (gates with a matrix are not handled here)."""
    h = 1469598103934665603

    def fnv(h, data):
        for byte in data:
            h ^= byte
            h = (h * 1099511628211) & 0xFFFFFFFFFFFFFFFF
        return h

    h = fnv(h, struct.pack("<i", n))
    for g in packed:
        h = fnv(h, struct.pack("<5i", g.kind, g.qubits[0], g.qubits[1], g.qubits[2],
                               1 if g.param >= 0 else 0))
        if g.param < 0:
            h = fnv(h, struct.pack("<d", g.angle))
    return h


def inverse_qft_gates(n):
    """The gate list the library schedules for the inverse gate-form QFT:
    Alg. 3 (H(i), then CP(pi / 2^(j-i)) from control i to each j > i) in
    reverse order with negated angles, without the swap network (one
    bit-reversal pass)."""
    import math

    import workloads as W

    g = []
    for i in range(n):
        g.append(W.G("H", i))
        for j in range(i + 1, n):
            g.append(W.G("CP", i, j, angle=math.pi / 2.0 ** (j - i)))
    return [W.G("CP", x.qubits[0], x.qubits[1], angle=-x.angle) if x.name == "CP" else x
            for x in reversed(g)]


@pytest.fixture()
def tune_entry(tmp_path):
    """Replace the autotune cache by one entry (k, m, table) for this circuit
    structure on the current device, through the cache file loader."""
    import paper_2512_23183_gb300 as lq

    def put(n, gates, k, m, table):
        lq.tune_cache_clear()
        f = tmp_path / "entry.txt"
        f.write_text("%s %d %016x %d %d %d 1.0 2.0\n"
                     % (_gpu_key(), n, _structure_hash(n, lq.pack_gates(gates)), k, m, table))
        lq.tune_cache_load(str(f))

    yield put
    lq.tune_cache_clear()
