"""The FP64 probes behind the bench's roofline denominators: the DFMA rate
and the shared-memory tile-sweep rate are positive, the sweep (two loads and
two stores per four FMAs) does not beat bare DFMA chains, and both stay
below the part's nominal FP64 rate (152 SMs x 2 DFMA/clk x 2 flops at the
largest SM clock), so neither probe can time less work than it counts."""
import pytest


@pytest.mark.gpu
def test_fp64_probes_are_consistent():
    import torch
    import paper_2512_23183_gb300 as lq

    props = torch.cuda.get_device_properties(0)
    nominal = props.multi_processor_count * 2 * 2 * 2.2e9 / 1e12   # 2.2 GHz bound
    dfma, ms = lq.measure_fp64_fma(reps=5)
    sweep, sms = lq.measure_fp64_tile_sweep(reps=3)
    assert ms > 0 and sms > 0
    assert 0 < dfma <= nominal, (dfma, nominal)
    assert 0 < sweep <= 1.02 * dfma, (sweep, dfma)
