"""Host logic of bench.py (CPU only): the algorithmic byte counts of the roofline, the DRAM traffic
read back from the committed ncu summaries and scaled to a batch, and the learned-initialisation
summaries carried into the bench line."""
import os
import re

import pytest

import bench


def _summary_values(kernel):
    vals = {}
    for line in open(os.path.join(bench.ROOT, "profiles", f"{kernel}_train_step_1M.md")):
        m = re.match(r"^- ([a-z_]+): (.*)$", line.strip())
        if m:
            vals[m.group(1)] = m.group(2)
    return vals


def test_algorithmic_bytes_per_unit():
    I, R, P, n, V = 1000, 300, 50, 200, 4
    assert bench.algorithmic_bytes("render_bwd", n, V, I, R, P, 6) == 4 * I + 72 * R + 20 * P
    assert bench.algorithmic_bytes("render_fwd", n, V, I, R, P, 6) == 4 * I + 36 * R + 24 * P
    assert bench.algorithmic_bytes("slice_project", n, V, I, R, P, 6) == 80 * n + 4 * V * n + 64 * R
    assert bench.algorithmic_bytes("adam", n, V, I, R, P, 6) == 560 * n
    assert bench.FLOPS_PER_BLENDED_PAIR == {"render_fwd": 12.0, "render_bwd": 40.0}


@pytest.mark.parametrize("kernel", ["render_bwd", "render_fwd"])
def test_stored_traffic_scales_with_the_batch(kernel):
    vals = _summary_values(kernel)
    measured = float(vals["dram_bytes_per_launch"])
    captured = float(vals["algorithmic_bytes_per_launch"].split()[0])
    assert measured == int(vals["dram_read_bytes_per_launch"]) + int(vals["dram_write_bytes_per_launch"])
    if vals["source_hash"] != bench.source_hash():
        assert bench.stored_traffic(kernel, captured) is None     # counters of other kernel sources
        return
    assert bench.stored_traffic(kernel, captured) == pytest.approx(measured)
    assert bench.stored_traffic(kernel, 0.5 * captured) == pytest.approx(0.5 * measured)
    # the committed traffic stays within 3x of the algorithmic bytes
    assert measured < 3.0 * captured


def test_learned_init_summaries():
    out = bench.learned_init_summary()
    assert set(out) == {"reduced", "full"}
    for size, d in out.items():
        s = d["summary"]
        assert "learned_half" in s and s["learned_half"]["of"] == d["scenes"]["test"]
        assert s["learned_half"]["reached"] <= s["learned_half"]["of"]
