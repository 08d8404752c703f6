#!/usr/bin/env python3
"""Benchmark of the GB300 dense state-vector hot path (arXiv 2512.23183 method).

One step runs every row of the hot path once:
  a1  state set-up: the synthetic input state is copied into the working state
  a2-a4  one hardware-efficient layer (RY, RZ on every qubit, CNOT ladder),
      lowered to fused shared-memory tile passes
  a5  QFT, FFT form (Alg. 2)
  a6  inverse QFT, gate form (Alg. 3)
  a7  <H> of the open-chain XYZ Heisenberg model
  a8  batched parameter-shift energy + gradient of the n=10, depth-4 VQE
      problem (161 circuits in shared memory)
  a9  adjoint energy + gradient of the same VQE problem (when built)
on an n-qubit complex128 state (default n = 30: 16 GiB, inputs larger than L2,
so no flush is needed).  `value` is the step's state-vector DRAM bytes as the
library's plans give them (32 B per amplitude per tile pass, 16 B per amplitude
per read-only <H> pass; ncu confirms the kernels move exactly these) divided by
the step time measured with CUDA events.  Fewer passes for the same work lower
this figure while the step gets faster, so `ms_per_step` is the figure to
compare between versions.  `e2e` is the same step through the library's
public API with the input state copied from pinned host memory and the energy
read back inside the timed region.

Prints one JSON line (rank 0).  Multi-GPU runs are independent replicas (no
collective on the data path); value = all ranks' bytes / max rank time.
`--impl reference` times the CPU oracle on a bounded sample of the same step.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "state-vector HBM GB/s (% peak); VQE grads/s plain vs batched; serve p50/p99"
UNIT = "GB/s"
# nominal GB300 FP64 from unit counts and clock: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz
FP64_NOMINAL_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12

# State passes of the step's rows (HEA layer, FFT-form QFT with its bit
# reversal, inverse gate-form QFT with its bit reversal, <H> reads) under the
# library's default (untuned) schedules, at the sizes the oracle sample runs:
# the oracle arm counts its bytes with these, so it never loads the CUDA
# library.  tests/test_bench_cpu.py checks them against the library's plans.
ORACLE_STEP_PASSES = {10: (1, 2, 2, 10), 11: (2, 2, 3, 11), 12: (2, 2, 3, 1), 13: (2, 3, 3, 2),
                      14: (2, 3, 3, 2), 15: (2, 3, 3, 2), 16: (3, 3, 4, 2), 17: (3, 3, 4, 2),
                      18: (3, 3, 4, 2), 19: (3, 3, 4, 2), 20: (3, 3, 4, 2), 21: (4, 3, 5, 2),
                      22: (4, 3, 5, 3), 23: (4, 4, 5, 3), 24: (4, 4, 5, 3)}


def step_bytes(n, passes):
    """Algorithmic state bytes of one step at n qubits: the copy-in (read and
    write), 32 B per amplitude per tile pass, 16 B per amplitude per
    read-only <H> pass."""
    N = float(1 << n)
    hea, fft, gates, reads = passes
    return 32 * N * (1 + hea + fft + gates) + 16 * N * reads


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lq", choices=["lq", "reference"])
    ap.add_argument("--n", type=int, default=30)
    ap.add_argument("--no-extras", action="store_true", help="skip the VQE/serve side measurements")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-n", type=int, default=23, help="qubits of the bounded oracle sample")
    ap.add_argument("--cpu-s", type=float, default=10.0,
                    help="seconds of CPU work the oracle sample spans at least")
    ap.add_argument("--serve-requests", type=int, default=48,
                    help="requests of the serving measurement (Poisson pass)")
    ap.add_argument("--serve-only", action="store_true",
                    help="run only the serving measurement and print its JSON")
    ap.add_argument("--psr-batched-only", action="store_true",
                    help="run only the n=16 depth-8 ring batched parameter-shift gradient "
                         "(--steps timed runs after one untimed) and print its JSON")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while active."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


class nvtx_range:
    """An NVTX push/pop range (a no-op when torch has no NVTX support)."""

    def __init__(self, name):
        import torch

        try:
            torch.cuda.nvtx.range_push(name)
            self.ok = True
        except (RuntimeError, AttributeError):
            self.ok = False

    def close(self):
        import torch

        if self.ok:
            torch.cuda.nvtx.range_pop()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def fp64_roof(gpu_index, reps=30):
    """The FP64 roof of this GPU, measured in set-up: the library's DFMA
    throughput probe (independent FMA chains, every SM filled; best of
    `reps` launches timed with CUDA events) with nvidia-smi clocks sampled
    meanwhile."""
    import paper_2512_23183_gb300 as lq

    clocks = ClockSampler(gpu_index)
    clocks.start()
    t0 = time.perf_counter()
    tf, ms = 0.0, 0.0
    while time.perf_counter() - t0 < 0.6:   # long enough for a few clock samples
        t, m = lq.measure_fp64_fma(reps=reps)
        if t > tf:
            tf, ms = t, m
    sw, sw_ms = lq.measure_fp64_tile_sweep(reps=5)
    clk = clocks.stop()
    return {"tflops": round(tf, 4), "ms_per_launch": round(ms, 3),
            "nominal_tflops": round(FP64_NOMINAL_TFLOPS, 4), "clocks": clk,
            "how": "lq_measure_fp64_fma: 8 independent DFMA chains per thread, 4096 FMAs each, "
                   "every SM filled, best launch by CUDA events",
            "tile_sweep_tflops": round(sw, 4), "tile_sweep_ms": round(sw_ms, 3),
            "tile_sweep_frac_of_dfma": round(sw / tf, 4) if tf else None,
            "tile_sweep_how": "lq_measure_fp64_tile_sweep: tangent-form rotations on a "
                              "2^12-amplitude shared-memory tile per CTA (2 loads, 4 FMAs, "
                              "2 stores per pair, a barrier per sweep), as many CTAs as fit "
                              "per SM: the tile passes' access pattern without global traffic"}


def profiled_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if the
    kernel sources are unchanged since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f).get(kernel)
    except (OSError, ValueError):
        return None
    if not rec:
        return None
    import hashlib

    h = hashlib.sha256()
    for rel in rec.get("sources", []):
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return rec.get("bytes_per_launch") if h.hexdigest() == rec.get("sha256") else None


# -------------------------------------------------------------- the step

class Step:
    """All hot-path rows on an n-qubit state (see module docstring)."""

    def __init__(self, n, device):
        import numpy as np
        import torch

        import paper_2512_23183_gb300 as lq
        import workloads as W

        self.lq, self.n, self.dev = lq, n, device
        g = torch.Generator(device=device)
        g.manual_seed(1000 + n)
        v = torch.randn(2 << n, dtype=torch.float64, device=device, generator=g)
        self.inp = torch.view_as_complex(v.view(-1, 2))
        self.inp /= torch.linalg.vector_norm(self.inp)
        del v
        self.work = torch.empty_like(self.inp)
        self.layer, P = W.hea(n, 1, "ladder")
        self.theta = W.angles(P, 2000 + n)
        self.terms = W.heisenberg(n)
        # schedule autotuning of the layer (set-up, untimed): apply_circuit then
        # uses the chosen tile width / low bits / phase-table option
        self.tune = lq.autotune(n, self.layer, self.theta, scratch=self.work)
        self.tune_qft = lq.autotune_qft(n, inverse=True, scratch=self.work)
        self.exp_ws = torch.empty(lq.load().lq_expval_workspace_size(n, len(self.terms)),
                                  dtype=torch.uint8, device=device)
        self.e_dev = torch.zeros(1, dtype=torch.float64, device=device)
        self.packed_terms = lq.pack_terms(self.terms, n)
        # a8/a9: VQE problem, n=10, depth 4, 80 parameters
        self.vn = 10
        self.vgates, self.vth, self.vterms = W.vqe_chain(10, 4, 1)
        self.psr_ws = torch.empty(lq.load().lq_param_shift_workspace_size(10, len(self.vth),
                                                                          len(self.vterms), 1),
                                  dtype=torch.uint8, device=device)
        self.has_adjoint = True
        try:
            lq.adjoint_grad(10, self.vgates, self.vth, self.vterms, device=device)
        except lq.LqError:
            self.has_adjoint = False
        plan_l = lq.circuit_plan(n, self.layer, self.theta)
        plan_f = lq.qft_plan(n, lq.QFT_FFT)
        plan_g = lq.qft_plan(n, lq.QFT_GATES, inverse=True)
        plan_e = lq.expval_plan(n, self.terms)
        N = float(1 << n)
        self.rows = {
            "a1_init": dict(bytes=32 * N, flops=0.0, launches=0),
            "a2_a4_hea_layer": dict(bytes=plan_l["dram_bytes"], flops=plan_l["dp_flops"],
                                    launches=plan_l["npasses"], kernel="pass_kernel"),
            "a5_qft_fft": dict(bytes=plan_f["dram_bytes"], flops=plan_f["dp_flops"],
                               launches=plan_f["npasses"], kernel="fft_pass_kernel"),
            "a6_qft_gates_inverse": dict(bytes=plan_g["dram_bytes"], flops=plan_g["dp_flops"],
                                         launches=plan_g["npasses"], kernel="pass_kernel"),
            # tiled <H>: the state is read once per tile pass of X-mask groups
            "a7_expval": dict(bytes=plan_e["dram_bytes"], flops=plan_e["dp_flops"],
                              launches=2, kernel="expval_tile_kernel"),
            # one persistent batch_kernel launch (graph-replayed with its copies)
            "a8_psr_batched_n10": dict(bytes=0.0, flops=0.0, launches=1),
        }
        if self.has_adjoint:
            ap = lq.adjoint_plan(10, self.vgates, self.vth, len(self.vterms))
            self.rows["a9_adjoint_n10"] = dict(bytes=0.0, flops=ap["dp_flops"],
                                               launches=ap["npasses"])
        self.bytes = sum(r["bytes"] for r in self.rows.values())

    def run(self, events=None, host_in=None, work=None):
        """One step; `events` (list of CUDA events, len 8) marks the rows.
        host_in: pinned host tensor to copy in (e2e); work: a device state
        that already holds the step's input (e2e with the copy issued
        earlier on a copy stream), used in place of the copy-in."""
        import ctypes

        import torch

        lq, n = self.lq, self.n
        s = torch.cuda.current_stream()
        ev = events or [None] * 8

        def mark(i):
            if ev[i] is not None:
                ev[i].record(s)

        mark(0)
        if work is None:
            work = self.work
            if host_in is not None:
                work.copy_(host_in, non_blocking=True)
            else:
                work.copy_(self.inp)
        mark(1)
        lq.apply_circuit(work, n, self.layer, self.theta)
        mark(2)
        lq.qft(work, n, method=lq.QFT_FFT)
        mark(3)
        lq.qft(work, n, inverse=True, method=lq.QFT_GATES)
        mark(4)
        lq._check(lq.load().lq_expval_pauli_sum_async(
            lq._ptr(work), n, self.packed_terms, len(self.terms),
            ctypes.c_void_p(self.e_dev.data_ptr()), lq._ptr(self.exp_ws), self.exp_ws.numel(),
            ctypes.c_void_p(s.cuda_stream)))
        mark(5)
        e8, g8 = lq.param_shift_grad(self.vn, self.vgates, self.vth, self.vterms,
                                     method=lq.PSR_BATCHED, workspace=self.psr_ws)
        mark(6)
        if self.has_adjoint:
            lq.adjoint_grad(self.vn, self.vgates, self.vth, self.vterms, device=self.dev)
        mark(7)
        return e8, g8


def aggregate(ms_local, bytes_local, world, device):
    """Step time = max over ranks (all ranks run the same step on their own
    GPU: replicas, no data-path collective); value = all ranks' bytes / that
    time, in GB/s."""
    import torch

    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist

        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    return ms, world * bytes_local / (ms * 1e-3) / 1e9


def bench_lq(a, rank, world, device):
    import torch

    import paper_2512_23183_gb300 as lq

    lq.load()
    step = Step(a.n, device)
    gpu_index = torch.cuda.current_device() if world == 1 else int(os.environ.get("LOCAL_RANK", 0))
    roof = fp64_roof(gpu_index)
    fp64_peak = roof["tflops"]
    sweep = roof.get("tile_sweep_tflops")
    for _ in range(a.warmup):
        step.run()
    torch.cuda.synchronize()
    names = list(step.rows)
    seg_ms = {k: 0.0 for k in names}
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(8)] for _ in range(a.steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(gpu_index)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    # the timed steps form one NVTX range "lq_step" (profilers can select the
    # step's launches with it, skipping set-up and autotuning launches)
    nvtx = nvtx_range("lq_step")
    t0.record()
    for k in range(a.steps):
        step.run(evs[k])
    t1.record()
    nvtx.close()
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    total_ms = t0.elapsed_time(t1)
    for k in range(a.steps):
        e = evs[k]
        for i, nm in enumerate(names):
            if i + 1 < 8:
                seg_ms[nm] += e[i].elapsed_time(e[i + 1])
    ms, value = aggregate(total_ms / a.steps, step.bytes, world, device)
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    rows = {}
    for nm in names:
        r = step.rows[nm]
        t = seg_ms[nm] / a.steps
        tf = r["flops"] / (t * 1e-3) / 1e12 if t else None
        rows[nm] = dict(ms=round(t, 3), gbs=round(r["bytes"] / (t * 1e-3) / 1e9, 1) if t else None,
                        fp64_tflops=round(tf, 4) if t else None,
                        fp64_frac=round(tf / fp64_peak, 4) if t else None,
                        fp64_frac_of_tile_sweep=round(tf / sweep, 4) if t and sweep else None,
                        launches=r["launches"])
    # dominant kernel: the kernel family with the largest share of the step
    fam = {}
    for nm in names:
        kern = step.rows[nm].get("kernel")
        if kern:
            f = fam.setdefault(kern, dict(ms=0.0, flops=0.0, bytes=0.0, launches=0))
            f["ms"] += seg_ms[nm] / a.steps
            f["flops"] += step.rows[nm]["flops"]
            f["bytes"] += step.rows[nm]["bytes"]
            f["launches"] += step.rows[nm]["launches"]
    dom = max(fam, key=lambda k: fam[k]["ms"])
    f = fam[dom]
    per_launch_s = f["ms"] * 1e-3 / max(f["launches"], 1)
    flops_pl = f["flops"] / max(f["launches"], 1)
    bytes_pl = f["bytes"] / max(f["launches"], 1)
    ach_tf = flops_pl / per_launch_s / 1e12
    ach_gbs = bytes_pl / per_launch_s / 1e9
    roofline = {"bound": "alu", "achieved": round(ach_tf, 4), "peak": fp64_peak,
                "unit": "TFLOP/s", "frac": round(ach_tf / fp64_peak, 4),
                "tile_sweep_ceiling": sweep,
                "frac_of_tile_sweep": round(ach_tf / sweep, 4) if sweep else None,
                "traffic": profiled_traffic(dom), "kernel": dom,
                "peak_note": "measured on this GPU in set-up (DFMA probe, fp64_roof); nominal "
                             "%.3f TFLOP/s from 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz, frac "
                             "of nominal %.4f" % (FP64_NOMINAL_TFLOPS, ach_tf / FP64_NOMINAL_TFLOPS),
                "peak_nominal": round(FP64_NOMINAL_TFLOPS, 4),
                "flops_note": "achieved counts the plans' flops (FMA = 2, add/multiply = 1); "
                              "a DADD or DMUL takes an FP64 issue slot like a DFMA; ncu counts "
                              "exactly the planned 2 DFMA per amplitude and rotation on the HEA "
                              "passes, at 74-85% FP64-pipe activity (profiles/fp64_mix_n24.md); "
                              "tile_sweep_ceiling is the measured rate of the same shared-memory "
                              "access pattern without global traffic",
                "hbm": {"achieved_gbs": round(ach_gbs, 1), "peak_gbs": hbm_peak,
                        "frac": round(ach_gbs / hbm_peak, 4),
                        "algorithmic_bytes_per_launch": bytes_pl},
                "algorithmic_flops_per_launch": flops_pl}
    kernels = {k: dict(ms_per_step=round(v["ms"], 3), launches=v["launches"],
                       fp64_tflops=round(v["flops"] / (v["ms"] * 1e-3) / 1e12, 4),
                       hbm_gbs=round(v["bytes"] / (v["ms"] * 1e-3) / 1e9, 1))
               for k, v in fam.items()}
    launches = sum(r["launches"] for r in step.rows.values())
    out = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(ms, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "sv_step_n%d" % a.n, "n_qubits": a.n,
                   "state_bytes": 16 << a.n, "input": "complex Gaussian from seed %d (torch cuda "
                   "generator), L2-normalised" % (1000 + a.n),
                   "rows": "a1 copy-in, a2-a4 HEA layer, a5 FFT-QFT, a6 gate-QFT^-1, a7 <H> "
                           "XYZ chain; a8 batched PSR + a9 adjoint of HEA n=10 d=4 (80 params)",
                   "l2": "inputs larger than L2 (state %d GiB), no flush" % ((16 << a.n) >> 30)
                   if a.n >= 24 else "state smaller than L2",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "hbm_frac": round(value / hbm_peak, 4),
        "rows": rows, "kernels": kernels, "roofline": roofline,
        "fp64_roof": roof,
        "autotune_hea_layer": step.tune,
        "autotune_qft_gates_inverse": step.tune_qft,
        "gpu_launches": launches * a.steps,
        "clocks": clk,
    }
    if not a.no_e2e and rank == 0:
        out["e2e"] = e2e(step, a)
    return out, step


def e2e(step, a):
    """The same step through the public API with host buffers: every step's
    input state is copied from pinned host memory and its energy read back
    (a synchronous device-to-host copy).  The copies run one step ahead on a
    copy stream into a second device state, so step k+1's 16 GiB copy
    overlaps step k's kernels; a device state is refilled only after the step
    that used it has finished.  The pipeline runs through the warm-up steps
    into the timed ones, and the timed region ends when the last copy it
    issued has arrived: it holds exactly K copies and K steps (steady state).
    `serial_ms_per_step` is the same loop with each copy issued on the compute
    stream right before its step."""
    import torch

    host = torch.empty(step.inp.shape, dtype=step.inp.dtype, pin_memory=True)
    host.copy_(step.inp)
    out_host = torch.empty(1, dtype=torch.float64, pin_memory=True)
    bufs = [step.work, torch.empty_like(step.work)]
    cs = torch.cuda.Stream()
    main = torch.cuda.current_stream()
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    free = [None, None]

    def prefetch(j):   # the input of a step that will use bufs[j]
        with torch.cuda.stream(cs):
            if free[j] is not None:
                cs.wait_event(free[j])
            bufs[j].copy_(host, non_blocking=True)
            copied[j].record(cs)

    def pipelined_step(i):   # uses bufs[i % 2]; prefetches the next step's input
        prefetch((i + 1) % 2)
        main.wait_event(copied[i % 2])
        step.run(work=bufs[i % 2])
        free[i % 2] = torch.cuda.Event()
        free[i % 2].record(main)
        out_host.copy_(step.e_dev)   # synchronous device->host read of <H>

    k = max(3, a.steps)
    w = max(3, a.warmup)   # the first copies from a fresh pinned buffer can be slower
    prefetch(0)
    for i in range(w):
        pipelined_step(i)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(w, w + k):
        pipelined_step(i)
    cs.synchronize()   # the last copy issued inside the timed region
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / k
    for _ in range(w):
        step.run(host_in=host)
        out_host.copy_(step.e_dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(k):
        step.run(host_in=host)
        out_host.copy_(step.e_dev)
    torch.cuda.synchronize()
    ds = (time.perf_counter() - t0) / k
    del host, bufs
    return {"value": round(step.bytes / dt / 1e9, 2), "unit": UNIT,
            "h2d_bytes_per_step": int(step.inp.numel() * 16), "d2h_bytes_per_step": 8 + 8 * 81,
            "ms_per_step": round(dt * 1e3, 3), "steps": k,
            "serial_ms_per_step": round(ds * 1e3, 3),
            "how": "host-timed over %d steps in steady state: each step's 16 GiB input copied "
                   "one step ahead on a copy stream (double-buffered device state), energy read "
                   "back every step; the timed region holds %d copies and %d steps" % (k, k, k)}


# ------------------------------------------------------- side measurements

def psr_batched_only(device, steps):
    """The n=16 depth-8 ring batched parameter-shift gradient alone (one
    untimed run, then `steps` host-timed runs): the problem of vqe_extras'
    vqe_n16_d8_ring_256p row, for profiling its persistent launch."""
    import torch

    import paper_2512_23183_gb300 as lq
    import workloads as W

    n = 16
    gates, th, terms = W.vqe_ring(16, 8, 3)
    ws = torch.empty(lq.load().lq_param_shift_workspace_size(n, len(th), len(terms),
                                                             lq.PSR_BATCHED),
                     dtype=torch.uint8, device=device)
    lq.param_shift_grad(n, gates, th, terms, method=lq.PSR_BATCHED, workspace=ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        e, _g = lq.param_shift_grad(n, gates, th, terms, method=lq.PSR_BATCHED, workspace=ws)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / max(steps, 1)
    return {"ms": round(dt * 1e3, 3), "grads_per_s": round(1.0 / dt, 3), "energy": e,
            "circuits": 2 * len(th) + 1}


def vqe_extras(device):
    """Gradients per second, plain (per-circuit library calls) vs batched vs
    adjoint, on the n=10 depth-4 ladder problem and the n=16 depth-8 ring
    problem; the adjoint on the n=24 depth-10 problem."""
    import torch

    import paper_2512_23183_gb300 as lq
    import workloads as W

    res = {}
    for name, (gates, th, terms, n, reps_p, reps_b) in {
        "vqe_n10_d4_80p": W.vqe_chain(10, 4, 1) + (10, 2, 10),
        "vqe_n16_d8_ring_256p": W.vqe_ring(16, 8, 3) + (16, 1, 3),
    }.items():
        r = {}
        if n > 12:   # tile width of the batched launch (set-up, untimed)
            r["autotune_batched"] = lq.autotune_param_shift(n, gates, th, terms, device=device)
        for meth, reps in ((lq.PSR_PLAIN, reps_p), (lq.PSR_BATCHED, reps_b)):
            ws = torch.empty(lq.load().lq_param_shift_workspace_size(n, len(th), len(terms), meth),
                             dtype=torch.uint8, device=device)
            lq.param_shift_grad(n, gates, th, terms, method=meth, workspace=ws)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                lq.param_shift_grad(n, gates, th, terms, method=meth, workspace=ws)
            torch.cuda.synchronize()
            dt = (time.perf_counter() - t0) / reps
            r["plain" if meth == 0 else "batched"] = {"grads_per_s": round(1.0 / dt, 3),
                                                      "ms": round(dt * 1e3, 3)}
            del ws
        try:
            lq.adjoint_grad(n, gates, th, terms, device=device)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps_b):
                lq.adjoint_grad(n, gates, th, terms, device=device)
            torch.cuda.synchronize()
            dt = (time.perf_counter() - t0) / reps_b
            r["adjoint"] = {"grads_per_s": round(1.0 / dt, 3), "ms": round(dt * 1e3, 3)}
        except lq.LqError:
            pass
        r["circuits_per_grad"] = 2 * len(th) + 1
        res[name] = r
    # adjoint workload: n=24, depth-10 ladder, 480 angles (seed 5), open chain:
    # the adjoint gradient, the batched parameter-shift gradient (all 961
    # circuits in one persistent launch, one timed run), their agreement, and
    # one plain circuit (|0..0> -> <H>) for the plain method's rate
    n = 24
    gates, P = W.hea(n, 10, "ladder")
    th = W.angles(P, 5)
    terms = W.heisenberg(n)
    r = {}
    lq.adjoint_grad(n, gates, th, terms, device=device)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(3):
        ea, ga = lq.adjoint_grad(n, gates, th, terms, device=device)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / 3
    r["adjoint"] = {"grads_per_s": round(1.0 / dt, 3), "ms": round(dt * 1e3, 3)}
    ws = torch.empty(lq.load().lq_param_shift_workspace_size(n, P, len(terms), lq.PSR_BATCHED),
                     dtype=torch.uint8, device=device)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    eb, gb = lq.param_shift_grad(n, gates, th, terms, method=lq.PSR_BATCHED, workspace=ws)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    r["batched"] = {"grads_per_s": round(1.0 / dt, 4), "ms": round(dt * 1e3, 1),
                    "workspace_gb": round(ws.numel() / 1e9, 1),
                    "note": "one run (the graph capture, a few ms, included)"}
    tol = 1e-10 * max(1.0, float(abs(gb).max()))
    r["adjoint_vs_batched"] = {"max_abs_dgrad": float(abs(ga - gb).max()),
                               "abs_denergy": abs(ea - eb), "tolerance": tol,
                               "agree": bool(abs(ga - gb).max() <= tol
                                             and abs(ea - eb) <= 1e-10 * max(1.0, abs(eb)))}
    del ws
    torch.cuda.empty_cache()
    psi = lq.new_state(n)
    ws = torch.empty(lq.load().lq_expval_workspace_size(n, len(terms)), dtype=torch.uint8,
                     device=device)

    def circuit():
        lq.state_init(psi, n)
        lq.apply_circuit(psi, n, gates, th)
        return lq.expval_pauli_sum(psi, n, terms, workspace=ws)

    circuit()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(3):
        circuit()
    dt1 = (time.perf_counter() - t0) / 3
    r["one_circuit_ms"] = round(dt1 * 1e3, 3)
    r["plain_grads_per_s_from_one_circuit"] = round(1.0 / (dt1 * (2 * P + 1)), 4)
    r["circuits_per_grad"] = 2 * P + 1
    res["adjoint_n24_d10_480p"] = r
    del psi, ws
    # uneven batch: 64 instances (seed 4), n ~ U{8..20}, depth ~ U{2..12},
    # ring HEA, random 50-term sums; every instance's energy and gradient in
    # one persistent launch (one warm-up run, one timed)
    inst = W.uneven_batch(count=64, seed=4)
    probs = [lq.BatchProblem(n, g, th, t) for n, g, th, t in inst]
    lq.batch_param_shift(probs, device=device)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lq.batch_param_shift(probs, device=device)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    ncirc = sum(2 * len(th) + 1 for _, _, th, _ in inst)
    res["uneven_batch_64"] = {"s": round(dt, 3), "problem_grads_per_s": round(64 / dt, 3),
                              "circuits": ncirc, "circuits_per_s": round(ncirc / dt, 1)}
    return res


def next_rows_extras(device):
    """The rows after the hot path: first-order Trotter evolution of the
    time-dependent XYZ model (Sec. VII-A: J = 1, h(t) = 2 sin t, from
    |1...1>) at n = 24 and 28, and the VQE Adam loop (Sec. VI-B settings:
    lr 1e-2, at most 350 iterations, tolerance 1e-7) on the n = 10 depth-4
    problem with adjoint and batched parameter-shift gradients."""
    import numpy as np
    import torch

    import paper_2512_23183_gb300 as lq
    import workloads as W

    out = {}
    dt, steps = 0.05, 20
    for n in (24, 28):
        static, field, A, om, x0 = W.xyz_trotter(n)
        psi = lq.new_state(n, x0)
        lq.trotter_evolve(psi, n, static, field, A, om, dt, 2)   # warm-up
        lq.state_init(psi, n, x0)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        lq.trotter_evolve(psi, n, static, field, A, om, dt, steps)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        # E(t) with the field at t = steps * dt
        ht = A * np.sin(om * steps * dt)
        e = lq.expval_pauli_sum(psi, n, static + [(c * ht, f) for c, f in field])
        out["trotter_n%d" % n] = {"steps": steps, "dt": dt, "ms_per_step": round(ms / steps, 3),
                                  "E_t": e}
        del psi
        torch.cuda.empty_cache()
    gates, th, terms = W.vqe_chain(10, 4, 1)
    for meth, name in ((0, "adjoint"), (1, "batched_psr")):
        t0 = time.perf_counter()
        p, es = lq.vqe_adam(10, gates, th, terms, method=meth)
        dt_s = time.perf_counter() - t0
        out["vqe_adam_n10_" + name] = {"iterations": int(es.size), "s": round(dt_s, 3),
                                       "iters_per_s": round(es.size / dt_s, 1),
                                       "E_first": float(es[0]), "E_last": float(es[-1])}
    return out


def qft_extras(device, fp64_peak, sizes=(20, 24, 28, 30), reps=3):
    """The QFT workload as configured: FFT form and gate form at n = 20, 24,
    28, 30 on seeded Gaussian inputs, each timed with CUDA events (mean of
    `reps` after a warm-up): ms, state-vector GB/s by the plan's algorithmic
    bytes, FP64 TFLOP/s by the plan's flops."""
    import torch

    import paper_2512_23183_gb300 as lq

    out = {}
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    for n in sizes:
        g = torch.Generator(device=device)
        g.manual_seed(1000 + n)
        v = torch.randn(2 << n, dtype=torch.float64, device=device, generator=g)
        psi = torch.view_as_complex(v.view(-1, 2))
        psi /= torch.linalg.vector_norm(psi)
        r = {}
        for name, meth in (("fft", lq.QFT_FFT), ("gates", lq.QFT_GATES)):
            plan = lq.qft_plan(n, meth)
            lq.qft(psi, n, method=meth)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(reps):
                lq.qft(psi, n, method=meth)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            gbs = plan["dram_bytes"] / (ms * 1e-3) / 1e9
            tf = plan["dp_flops"] / (ms * 1e-3) / 1e12
            r[name] = {"ms": round(ms, 3), "gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm, 4),
                       "fp64_tflops": round(tf, 4), "fp64_frac": round(tf / fp64_peak, 4),
                       "launches": plan["npasses"]}
        out["n%d" % n] = r
        del psi, v
        torch.cuda.empty_cache()
    return out


def serve_extras(device, count=48, slots=8, closed=48):
    """Serving workload: seeded request stream (n ~ U{8..28}, depth ~
    U{2..20}, 50/50 energy / energy+gradient, Heisenberg chain or random
    50-term sums), admitted by footprint against a device arena of up to
    150 GB.  A closed-loop pass over the first `closed` requests measures
    capacity; then `count` requests arrive as a Poisson stream at 70% of it.
    Reports throughput, p50/p99 latency (submit -> done) with the number of
    samples behind them, and how many requests were in flight together."""
    import numpy as np
    import torch

    import paper_2512_23183_gb300 as lq
    import workloads as W

    free, _ = torch.cuda.mem_get_info()
    budget = int(min(150e9, free - 8e9))
    arena = torch.empty(budget, dtype=torch.uint8, device=device)
    reqs = W.serve_requests(count, seed=6)
    closed = min(closed, count)
    srv = lq.Server(arena, slots=slots)
    try:
        t0 = time.perf_counter()
        ids = [srv.submit(r["n"], r["gates"], r["params"], r["terms"], r["grad"])
               for r in reqs[:closed]]
        for i in ids:
            srv.result(i)
        cap = closed / (time.perf_counter() - t0)
        rate = 0.7 * cap
        gaps = np.random.default_rng(6).exponential(1.0 / rate, count)
        arrivals = np.cumsum(gaps)
        start = time.perf_counter()
        ids = []
        for r, ta in zip(reqs, arrivals):
            dt = start + ta - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            ids.append(srv.submit(r["n"], r["gates"], r["params"], r["terms"], r["grad"]))
        res = [srv.result(i) for i in ids]
        end = max(t[2] for _, _, t in res)
        first = min(t[0] for _, _, t in res)
        lat = np.array([t[2] - t[0] for _, _, t in res])
        # requests in flight together: the largest number of overlapping
        # [t_start, t_done] intervals (one stream per slot)
        ev = sorted([(t[1], 1) for _, _, t in res] + [(t[2], -1) for _, _, t in res])
        cur = peak = 0
        for _, d in ev:
            cur += d
            peak = max(peak, cur)
    finally:
        srv.close()
        del arena
    return {"requests": count, "slots": slots, "arena_gb": round(budget / 1e9, 1),
            "closed_loop_requests": closed,
            "closed_loop_req_per_s": round(cap, 3), "poisson_rate_req_per_s": round(rate, 3),
            "throughput_req_per_s": round(count / (end - first), 3),
            "p50_ms": round(float(np.percentile(lat, 50)) * 1e3, 2),
            "p99_ms": round(float(np.percentile(lat, 99)) * 1e3, 2),
            "latency_samples": int(lat.size),
            "p99_note": "p99 of %d samples%s" % (lat.size, " (= the largest latency)"
                                                 if lat.size < 100 else ""),
            "max_in_flight": peak,
            "workload": "seed 6: n~U{8..28}, depth~U{2..20}, 50/50 energy/grad (adjoint), "
                        "Heisenberg chain or random 50-term"}


# ----------------------------------------------------------- CPU baseline

def oracle_sample_rate(n):
    """The oracle, as it stands, on the same step at n qubits: returns
    (GB/s by the step's algorithmic-bytes formula, seconds, threads)."""
    import numpy as np

    import oracle
    import workloads as W

    oracle.build()
    psi0 = W.gaussian_state(n, 1000 + n)
    layer, P = W.hea(n, 1, "ladder")
    th = W.angles(P, 2000 + n)
    terms = W.heisenberg(n)
    t0 = time.perf_counter()
    work = psi0.copy()                                   # a1
    oracle.apply_circuit(work, n, layer, th)             # a2-a4
    oracle.qft_fft(work, n)                              # a5
    oracle.qft_gates(work, n)                            # a6 (forward gate form, same cost)
    e = oracle.expval(work, n, terms)                    # a7
    dt = time.perf_counter() - t0
    if n not in ORACLE_STEP_PASSES:
        raise SystemExit("no pass counts for an oracle sample at n=%d (have %s)"
                         % (n, sorted(ORACLE_STEP_PASSES)))
    byts = step_bytes(n, ORACLE_STEP_PASSES[n])
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    del e, np
    return byts / dt / 1e9, dt, threads


def cpu_baseline(n, min_s):
    """The oracle's step at n qubits, repeated until it has run for at least
    min_s seconds; the rate is total bytes over total time."""
    steps, byts, total = 0, 0.0, 0.0
    while steps == 0 or total < min_s:
        gbs, dt, threads = oracle_sample_rate(n)
        byts += gbs * dt * 1e9
        total += dt
        steps += 1
    return {"value": round(byts / total / 1e9, 3), "unit": UNIT, "cores": threads,
            "kind": "oracle",
            "sample": "%d step(s) (a1-a7) at n=%d (%.1f s of CPU work; a8/a9 excluded), "
                      "same algorithmic-bytes formula; a rate at n=%d, not the GPU's size"
                      % (steps, n, total, n)}


def run_reference(a, rank, world):
    if rank != 0:
        return None
    n = a.cpu_n - 2
    for _ in range(a.warmup):
        oracle_sample_rate(n)
    rates, times = [], []
    for _ in range(a.steps):
        g, dt, threads = oracle_sample_rate(n)
        rates.append(g)
        times.append(dt)
    value = sum(rates) / len(rates)
    ms = 1e3 * sum(times) / len(times)
    return {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(ms, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": "sv_step_n%d" % a.n,
                       "sample": "oracle step a1-a7 at n=%d per step (a rate comparison at a "
                                 "different n: the oracle's whole step at n=%d would take hours)"
                                 % (n, a.n)},
            "cpu_baseline": {"value": round(value, 3), "unit": UNIT, "cores": threads,
                             "kind": "oracle", "sample": "step a1-a7 at n=%d" % n},
            "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    a = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if a.impl == "reference":
        out = run_reference(a, rank, world)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    import torch

    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    device = "cuda:%d" % local
    if a.psr_batched_only:
        if rank == 0:
            print(json.dumps({"psr_batched_n16": psr_batched_only(device, a.steps)}), flush=True)
        return
    if a.serve_only:
        if rank == 0:
            import paper_2512_23183_gb300 as lq

            lq.load()
            print(json.dumps({"serve": serve_extras(device, count=a.serve_requests)}), flush=True)
        return
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device(device))
    out, step = bench_lq(a, rank, world, device)
    del step
    torch.cuda.empty_cache()
    if rank == 0:
        if not a.no_extras:
            out["qft"] = qft_extras(device, out["fp64_roof"]["tflops"])
            out["vqe"] = vqe_extras(device)
            torch.cuda.empty_cache()
            out["next_rows"] = next_rows_extras(device)
            torch.cuda.empty_cache()
            out["serve"] = serve_extras(device, count=a.serve_requests)
        out["cpu_baseline"] = cpu_baseline(a.cpu_n, a.cpu_s)
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
