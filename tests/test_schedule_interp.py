"""The tile-pass scheduler's output on the CPU (no GPU): tests/native/
sched_interp.cpp lowers and schedules random circuits with small tiles (many
passes), with and without phase sinking, applies the scheduled ops with the
semantics the pass kernels give them, and compares with a plain gate-by-gate
simulation (1e-12).  This checks the compiler (op forms, pass packing,
phase sinking through CNOT/CY/SWAP as parity phases, merged phase factors,
the folded final scalar) independently of the kernels."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2512_23183_gb300")


@pytest.fixture(scope="module")
def interp(tmp_path_factory):
    import paper_2512_23183_gb300 as lq

    lq.load()   # builds liblq.so when missing
    exe = str(tmp_path_factory.mktemp("interp") / "sched_interp")
    cmd = ["g++", "-std=c++17", "-O2", "-I", os.path.join(PKG, "csrc"), "-I",
           os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "native", "sched_interp.cpp"),
           "-o", exe, "-L", PKG, "-llq", "-Wl,-rpath," + PKG]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_scheduled_ops_equal_the_circuit(interp, seed):
    r = subprocess.run([interp, "150", str(seed)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
