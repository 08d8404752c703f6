"""The autotuner's cache file (host only, no GPU): entries load, save and
merge; a malformed file is rejected and leaves the cache unchanged."""
import os

import pytest

import paper_2512_23183_gb300 as lq

GOOD = """# lq autotune cache v1: gpu n hash k m table ms ms_default
NVIDIA_GB300|152 24 00000000deadbeef 11 5 1 3.250000 3.900000
NVIDIA_GB300|152 30 0123456789abcdef 10 6 0 210.500000 222.000000
"""


@pytest.fixture()
def L():
    lib = lq.load()
    lq.tune_cache_clear()
    yield lib
    lq.tune_cache_clear()


def test_load_save_round_trip(L, tmp_path):
    src = tmp_path / "tune.txt"
    src.write_text(GOOD)
    lq.tune_cache_load(str(src))
    assert lq.tune_cache_size() == 2
    out = tmp_path / "out.txt"
    lq.tune_cache_save(str(out))
    lines = [ln for ln in out.read_text().splitlines() if not ln.startswith("#")]
    assert sorted(lines) == sorted(ln for ln in GOOD.splitlines() if not ln.startswith("#"))
    # loading the same file again merges (no duplicates)
    lq.tune_cache_load(str(out))
    assert lq.tune_cache_size() == 2


@pytest.mark.parametrize("bad", [
    "NVIDIA_GB300|152 24 00000000deadbeef 11 5 1 3.25\n",          # missing field
    "NVIDIA_GB300|152 40 00000000deadbeef 11 5 1 3.25 3.9\n",      # n out of range
    "NVIDIA_GB300|152 24 deadbeef 11 5 1 3.25 3.9\n",              # short hash
    "NVIDIA_GB300|152 24 00000000deadbeef 14 5 1 3.25 3.9\n",      # k too large
    "NVIDIA_GB300|152 24 00000000deadbeef 9 10 1 3.25 3.9\n",      # m > k
])
def test_malformed_rejected(L, tmp_path, bad):
    good = tmp_path / "good.txt"
    good.write_text(GOOD)
    lq.tune_cache_load(str(good))
    f = tmp_path / "bad.txt"
    f.write_text(GOOD + bad)
    with pytest.raises(lq.LqError):
        lq.tune_cache_load(str(f))
    assert lq.tune_cache_size() == 2
    with pytest.raises(lq.LqError):
        lq.tune_cache_load(str(tmp_path / "missing.txt"))


def test_plan_unaffected_by_other_gpus_entries(L, tmp_path):
    import workloads as W

    n = 16
    gates, P = W.hea(n, 2, "ladder")
    before = lq.circuit_plan(n, gates, W.angles(P, 1))
    f = tmp_path / "t.txt"
    f.write_text("Some_Other_GPU|1 16 %016x 12 6 0 1.0 2.0\n" % 0x1234)
    lq.tune_cache_load(str(f))
    assert lq.circuit_plan(n, gates, W.angles(P, 1)) == before


def test_low_run_widened_to_the_offset_table(L, tmp_path, tune_entry):
    """A cached low run that leaves more tile bits above it than the pass
    kernel's offset table maps (9) is widened: k = 12 with m = 1 plans as
    m = 3.  With 2^12 tiles an n = 30 layer of one-qubit rotations and a CNOT
    ladder takes 3 passes at m = 3 (12 + 9 + 9 qubits) and 4 at m = 5."""
    import workloads as W

    n = 30
    gates, P = W.hea(n, 1, "ladder")
    th = W.angles(P, 1)

    def plan_with(m):
        tune_entry(n, gates, 12, m, 0)
        return lq.circuit_plan(n, gates, th)

    p1, p3, p5 = plan_with(1), plan_with(3), plan_with(5)
    assert p3["tile_bits"] == 12 and p5["tile_bits"] == 12   # the entry applies
    assert p1 == p3
    assert p3["npasses"] == 3 and p5["npasses"] == 4


def test_short_low_run_for_the_inverse_gate_qft(L, tune_entry):
    """The inverse gate-form QFT at n = 30: with 2^11 tiles a 4-bit low run
    leaves 7 new qubits per pass (11 + 7 + 7 + 5: 4 passes) where a 5-bit run
    leaves 6 (5 passes); the plan adds the bit-reversal pass.  The entry is
    keyed by the structure of the gate list the library builds."""
    from conftest import inverse_qft_gates

    n = 30
    g = inverse_qft_gates(n)
    tune_entry(n, g, 11, 4, 1)
    p4 = lq.qft_plan(n, lq.QFT_GATES, inverse=True)
    tune_entry(n, g, 11, 5, 1)
    p5 = lq.qft_plan(n, lq.QFT_GATES, inverse=True)
    assert p4["tile_bits"] == p5["tile_bits"] == 11
    assert p4["npasses"] == 4 + 1 and p5["npasses"] == 5 + 1
