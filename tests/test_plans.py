"""Pass structure of the bench's rows, from the host-side plans (no GPU):
how many state passes each row takes and the bytes it moves, at the sizes
the bench runs.  The counts follow from the tile geometry alone."""
import pytest

import paper_2512_23183_gb300 as lq
import workloads as W


@pytest.fixture(scope="module", autouse=True)
def L():
    lib = lq.load()
    lq.tune_cache_clear()
    yield lib


def test_hea_layer_default_schedule_n30():
    # default tiles: k = 10 with the 5 low bits always in the tile, so each
    # pass brings 5 new qubits and the last one 10: 5 + 5 + 5 + 5 + 10 = 30
    n = 30
    gates, P = W.hea(n, 1, "ladder")
    p = lq.circuit_plan(n, gates, W.angles(P, 1))
    assert p["tile_bits"] == 10 and p["npasses"] == 5
    assert p["dram_bytes"] == 5 * 32 * 2.0 ** n


@pytest.mark.parametrize("n,passes", [(20, 2), (24, 3), (30, 3)])
def test_fft_qft_passes(n, passes):
    # groups of at most 10 qubits, the last (lowest) of at most 12, plus the
    # bit-reversal pass; each pass reads and writes the state once
    p = lq.qft_plan(n, lq.QFT_FFT)
    assert p["npasses"] == passes + 1
    assert p["dram_bytes"] == (passes + 1) * 32 * 2.0 ** n


@pytest.mark.parametrize("n,reads", [(20, 2), (24, 3), (30, 3)])
def test_xyz_chain_expval_reads(n, reads):
    # 3(n-1) terms: one diagonal group (ZZ) and n-1 X-mask groups (XX+YY on a
    # bond); a tile holds 12 bits, the 2 low ones fixed, so the first pass
    # covers the 11 bonds inside bits 0-11 and each later one the 9 bonds
    # inside 10 further bits: 11 + 9 + 9 = 29 at n = 30
    terms = W.heisenberg(n)
    assert len(terms) == 3 * (n - 1)
    p = lq.expval_plan(n, terms)
    assert p["npasses"] == reads
    assert p["dram_bytes"] == reads * 16 * 2.0 ** n


def test_inverse_gate_qft_default_schedule_n30():
    # the phases need no tile bits; the 30 H do: the gate form's default on
    # large states, 2^11-amplitude tiles with 6 fixed low bits, takes
    # 11 + 5 + 5 + 5 + 4 qubits in 5 passes, then the bit reversal
    n = 30
    p = lq.qft_plan(n, lq.QFT_GATES, inverse=True)
    assert p["tile_bits"] == 11 and p["npasses"] == 5 + 1
    assert p["dram_bytes"] == 6 * 32 * 2.0 ** n


def test_gate_qft_small_states_keep_the_library_schedule():
    # below 24 qubits the gate form keeps the library default (2^10 tiles)
    p = lq.qft_plan(20, lq.QFT_GATES)
    assert p["tile_bits"] == 10


@pytest.mark.parametrize("n,masks,diag", [(12, 240, 5), (14, 400, 0), (12, 20, 300)])
def test_expval_plan_splits_passes_beyond_one_plan(n, masks, diag):
    # a 2^12-amplitude state is one tile, so every X mask fits the first pass;
    # the passes must still respect one plan's group/term/coefficient
    # capacity (and a diagonal group of hundreds of terms goes to the untiled
    # kernel) instead of failing
    import numpy as np

    rng = np.random.default_rng(n + masks)
    terms = []
    for m in rng.choice(np.arange(1, 1 << n), size=masks, replace=False):
        s = ["XY"[rng.integers(2)] if (int(m) >> (n - 1 - q)) & 1 else "IZ"[rng.integers(2)]
             for q in range(n)]
        terms.append((float(rng.standard_normal()), "".join(s)))
    terms += [(1.0, "".join("Z" if rng.random() < 0.3 else "I" for _ in range(n)))
              for _ in range(diag)]
    p = lq.expval_plan(n, terms)
    assert p["npasses"] >= 2


@pytest.mark.parametrize("k,m,passes", [(12, 3, 3), (10, 5, 5)])
def test_hea_layer_one_merged_phase_op(tune_entry, k, m, passes):
    # the layer's 30 RZ factors are applied once, in its last pass, as one
    # merged phase op (12 flops per amplitude) that also takes the final
    # scalar: 30 RY x 4 flops + 12 per amplitude, whatever the pass count
    n = 30
    gates, P = W.hea(n, 1, "ladder")
    tune_entry(n, gates, k, m, 0)
    p = lq.circuit_plan(n, gates, W.angles(P, 2030))
    assert p["npasses"] == passes and p["tile_bits"] == k
    assert p["dp_flops"] == (30 * 4 + 12) * 2.0 ** n
