"""bench.py on the CPU: the max-over-ranks aggregation with two gloo ranks,
and the reference arm's JSON line (the oracle timed on host cores), alone
and under a two-rank torchrun (only rank 0 prints)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, ms, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, v = bench.aggregate(ms[rank], 1e9, world, "cpu")
    out.put((rank, t, v))
    dist.destroy_process_group()


def test_aggregate_max_over_two_gloo_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ms = [10.0, 25.0]
    ps = [ctx.Process(target=_rank, args=(r, 2, port, ms, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in res:
        assert t == 25.0                       # max over ranks
        assert abs(v - 2 * 1e9 / 25e-3 / 1e9) < 1e-9   # both ranks' bytes


def _json_lines(out):
    return [json.loads(ln) for ln in out.splitlines() if ln.startswith("{")]


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--cpu-n", "12"], cwd=ROOT, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["unit"] == "GB/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_reference_arm_two_ranks_prints_once():
    port = _free_port()
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
                        "--nproc-per-node", "2", "--master-addr", "127.0.0.1", "--master-port",
                        str(port), "bench.py", "--impl", "reference", "--gpus", "2", "--steps",
                        "1", "--warmup", "0", "--cpu-n", "12"], cwd=ROOT, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1 and lines[0]["n_gpus"] == 2


def test_oracle_arm_pass_table_matches_library_plans():
    # the oracle arm counts its bytes from a pass table so that it never loads
    # the CUDA library; the table must be the library's own default schedules
    sys.path.insert(0, ROOT)
    import bench
    import paper_2512_23183_gb300 as lq
    import workloads as W

    lq.tune_cache_clear()
    for n, passes in bench.ORACLE_STEP_PASSES.items():
        layer, P = W.hea(n, 1, "ladder")
        th = W.angles(P, 2000 + n)
        N = 2.0 ** n
        got = (lq.circuit_plan(n, layer, th)["dram_bytes"] / (32 * N),
               lq.qft_plan(n, lq.QFT_FFT)["dram_bytes"] / (32 * N),
               lq.qft_plan(n, lq.QFT_GATES, inverse=True)["dram_bytes"] / (32 * N),
               lq.expval_plan(n, W.heisenberg(n))["dram_bytes"] / (16 * N))
        assert got == passes, n
        want = (32 * N + lq.circuit_plan(n, layer, th)["dram_bytes"]
                + lq.qft_plan(n, lq.QFT_FFT)["dram_bytes"]
                + lq.qft_plan(n, lq.QFT_GATES, inverse=True)["dram_bytes"]
                + lq.expval_plan(n, W.heisenberg(n))["dram_bytes"])
        assert bench.step_bytes(n, passes) == want


def test_reference_arm_loads_no_product_library():
    # the reference arm runs the oracle only: the CUDA library is not mapped
    code = ("import sys, runpy; sys.argv = ['bench.py', '--impl', 'reference', '--steps', '1', "
            "'--warmup', '0', '--cpu-n', '12']; runpy.run_path('bench.py', run_name='__main__'); "
            "maps = open('/proc/self/maps').read(); "
            "assert 'liblq.so' not in maps, 'liblq.so mapped'; "
            "assert 'liblq_oracle.so' in maps; print('maps ok')")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0 and "maps ok" in r.stdout, r.stdout + r.stderr
