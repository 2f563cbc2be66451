"""Host logic of bench.py that needs no GPU: the staleness guard of the
committed DRAM-traffic figure and the CPU baseline's layer sample."""
import re

import numpy as np
import pytest

import bench
import oracle


def test_kernel_source_hash_is_stable_and_covers_existing_files():
    h = bench.kernel_source_hash()
    assert re.fullmatch(r"[0-9a-f]{64}", h)
    assert h == bench.kernel_source_hash()
    assert "kernels.h" in bench.KERNEL_SOURCES and "epilogue.cuh" in bench.KERNEL_SOURCES


def test_traffic_figure_is_used_only_for_the_profiled_source(monkeypatch):
    text = open(bench.os.path.join(bench.ROOT, "profiles", "syrk_tc2_split_n16384.md")).read()
    want = float(re.search(r"dram_bytes_per_launch_n16384:\s*([0-9.eE+]+)", text).group(1))
    recorded = re.search(r"kernel_source_sha256:\s*([0-9a-f]{64})", text).group(1)
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: recorded)
    assert bench._traffic_from_profile(16384) == want
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 64)
    assert bench._traffic_from_profile(16384) is None


@pytest.mark.parametrize("rows", [1, 7, 64, 96])
def test_layer_sample_checksum_is_the_rows_of_the_layer(rows):
    """The CPU baseline times one SP2 layer restricted to a block of rows and
    returns a checksum of it: the trace of the leading rows x rows block of
    the sigma = -1 layer 2S - S^2, which pins the sample to that work."""
    rng = np.random.default_rng(5)
    A = rng.uniform(-1, 1, (96, 96))
    S = (A + A.T) / 2
    want = float(np.trace((2.0 * S - S @ S)[:rows, :rows]))
    assert abs(oracle.sp2_layer_sample(S, rows) - want) <= 1e-10 * max(1.0, abs(want))


def test_energy_from_sampled_power():
    """Energy of a solve = median sampled board power x time-to-D; per layer
    divided by the squaring layers; nothing when no power was sampled."""
    e = bench.energy_of(1400.0, 400.0, 50)
    assert e["power_w_median"] == 1400.0
    assert abs(e["joules_per_solve"] - 560.0) < 1e-9
    assert abs(e["joules_per_layer"] - 11.2) < 1e-9
    assert bench.energy_of(None, 400.0, 50) is None
    assert bench.energy_of(1400.0, 400.0, 0) is None
