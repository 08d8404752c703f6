"""First use of the library's constant device tables (QFT twiddles, dyadic
phase tables of merged phase gates), each case in a fresh process so that the
call under test really is the process's first (Sec. IV-B QFT in FFT and gate
form, compared with the oracle's plain inverse DFT)."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_PRELUDE = r"""
import sys, threading
sys.path.insert(0, %r)
import numpy as np
import torch
import oracle
import paper_2512_23183_gb300 as lq
import workloads as W
torch.cuda.set_device(0)
""" % ROOT

# Two host threads, each with its own stream, make the process's first lq_qft
# call at the same moment; both results must equal the oracle's.
_TWO_THREADS = _PRELUDE + r"""
method = int(sys.argv[1])
n = 18
xs = [W.gaussian_state(n, 1000 + n + i) for i in range(2)]
ts = [torch.from_numpy(x).cuda() for x in xs]
streams = [torch.cuda.Stream() for _ in range(2)]
torch.cuda.synchronize()
gate = threading.Barrier(2)
errs = [None, None]

def run(i):
    try:
        gate.wait()
        lq.qft(ts[i], n, method=method, stream=streams[i])
        streams[i].synchronize()
    except Exception as e:  # reported below
        errs[i] = repr(e)

th = [threading.Thread(target=run, args=(i,)) for i in range(2)]
for t in th:
    t.start()
for t in th:
    t.join()
assert errs == [None, None], errs
for i in range(2):
    want = oracle.qft_fft(xs[i].copy(), n)
    err = float(np.abs(ts[i].cpu().numpy() - want).max())
    assert err < 1e-12, (i, err)
print("ok")
"""

# The first lq_qft of the process is made while its stream is being captured:
# it is refused (nothing is enqueued), and the same call outside the capture
# then fills the table and matches the oracle.
_UNDER_CAPTURE = _PRELUDE + r"""
n = 14
x = W.gaussian_state(n, 1000 + n)
t = torch.from_numpy(x).cuda()
s = torch.cuda.Stream()
torch.cuda.synchronize()
g = torch.cuda.CUDAGraph()
refused = None
with torch.cuda.graph(g, stream=s):
    try:
        lq.qft(t, n, method=lq.QFT_FFT, stream=s)
    except lq.LqError as e:
        refused = e
assert refused is not None and refused.status == 5, refused
assert "captur" in str(refused), str(refused)
lq.qft(t, n, method=lq.QFT_FFT)
torch.cuda.synchronize()
err = float(np.abs(t.cpu().numpy() - oracle.qft_fft(x.copy(), n)).max())
assert err < 1e-12, err
print("ok")
"""


def _run(script, *args):
    r = subprocess.run([sys.executable, "-c", script] + [str(a) for a in args],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr


@pytest.mark.gpu
@pytest.mark.parametrize("method", [0, 1], ids=["fft", "gates"])
def test_first_qft_on_two_threads(method):
    _run(_TWO_THREADS, method)


@pytest.mark.gpu
def test_first_qft_under_capture_is_refused():
    _run(_UNDER_CAPTURE)
