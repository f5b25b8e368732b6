"""Host logic of the benchmark (CPU): the algorithmic work each roofline credits a phase with,
worked out by hand on a three-box tree, and the clock record read from nvidia-smi rows.

Tree: box 0 at level 2 (split; targets 0..8, sources 0..4) with two level-3 leaves, box 1
(targets 0..4, sources 0..2) and box 2 (targets 4..8, sources 2..4); U lists pair each leaf
with both leaves; no V or W entries.  Chebyshev order 5: n = 125 nodes, rows padded to 128.
"""
import os
import sys
import types

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

TREE = {
    "level": np.array([2, 3, 3]),
    "leaf": np.array([False, True, True]),
    "trg_begin": np.array([0, 0, 4]), "trg_end": np.array([8, 4, 8]),
    "src_begin": np.array([0, 0, 2]), "src_end": np.array([4, 2, 4]),
    "V": [],
    "U": np.array([[1, 1], [1, 2], [2, 1], [2, 2]]),
    "W": np.zeros((0, 2), np.int64),
}
PEAKS = {"bf16_tflops": 1000.0, "hbm_gbs": 5000.0, "source": "test"}
PIPES = {"ffma_flops": 60e12, "ex2_per_s": 4e12, "rsqrt_per_s": 8e12, "n_sm": 152, "source": "test"}
ARGS = types.SimpleNamespace(order=5, m2l="bf16x3")


def _stats(fused):
    base = {"ms_m2l": 0.01, "ms_l2l": 0.004, "ms_l2p": 0.006, "ms_l2lp": 0.004 if fused else 0.0,
            "ms_near": 0.003, "ms_select": 0.002, "l2lp_fused": 1 if fused else 0}
    other = dict(base, ms_select=0.004, ms_near=0.005)
    slow = dict(base, ms_select=0.009, ms_near=0.009)
    return [base, other, slow]            # phase times: medians over the steps


def test_fused_deepest_level():
    r = bench.rooflines(TREE, _stats(True), ARGS, nt=8, ns=4, ncell=1000, peaks=PEAKS, pipes=PIPES,
                        traffic_ok=False)
    # fused level: parent box 0 read (128 x 4 B); leaves 1, 2 have no V or X entries, so no own
    # local terms to read; 8 targets written
    assert r["l2lp"]["work_per_launch"] == 512 + 8 * 4
    assert r["l2lp"]["achieved"] == pytest.approx(544 / 0.004e-3 / 1e9)
    # with a V entry into leaf 2 (and one X entry into leaf 2 too) the fused kernel's work is the
    # same; the own-term L2P reads leaf 2's row and reads and writes S at its 4 targets, in the
    # L2P phase time left after the fused kernel (0.006 - 0.004 ms)
    tv = dict(TREE, V=np.array([[2, 1]]), X=np.array([[2, 1]]))
    r2 = bench.rooflines(tv, _stats(True), ARGS, nt=8, ns=4, ncell=1000, peaks=PEAKS, pipes=PIPES,
                         traffic_ok=False)
    assert r2["l2lp"]["work_per_launch"] == 512 + 8 * 4
    assert r2["l2p"]["kernel"].startswith("k_l2p_own")
    assert r2["l2p"]["work_per_launch"] == 512 + 4 * 8
    assert r2["l2p"]["ms_per_launch"] == pytest.approx(0.002)
    assert r["l2lp"]["traffic"] is None   # ncu traffic only where it was measured on this workload
    # nothing left for the separate L2L (both level-3 boxes are fused) or L2P: no entries
    assert "l2l" not in r and "l2p" not in r
    # near field: 4 x 2 source cells for each of the 4 (leaf, leaf) pairs, median time 0.005 ms;
    # MUFU bound: 1 / (2 / ex2 + 1 / rsqrt) = 1 / (0.5e-12 + 0.125e-12) = 1.6e12 evaluations/s
    assert r["near"]["work_per_launch"] == 32
    assert r["near"]["achieved"] == pytest.approx(32 / 0.005e-3)
    assert r["near"]["peak"] == pytest.approx(1.6e12)
    # selection: q and |E| read once (8 B per cell), 4 B per selected index (8 targets, 4 sources)
    assert r["select"]["work_per_launch"] == 8 * 1000 + 4 * (8 + 4)
    assert r["select"]["frac"] == pytest.approx(8048 / 0.004e-3 / 1e9 / 5000.0)
    assert r["m2l"]["work_per_launch"] == 0
    # the dominant single kernel: m2l (0.01 ms) over l2lp (0.004) and near (0.005)
    assert bench.dominant_kernel(r) == "m2l"
    assert not r["select"]["single_kernel"]


def test_separate_deepest_level():
    r = bench.rooflines(TREE, _stats(False), ARGS, nt=8, ns=4, ncell=1000, peaks=PEAKS, pipes=PIPES,
                        traffic_ok=True)
    assert "l2lp" not in r
    # both leaves get an L2L from box 0: 2 n^2 flops each
    assert r["l2l"]["work_per_launch"] == 2 * 2 * 125 ** 2
    assert r["l2l"]["achieved"] == pytest.approx(62500 / 0.004e-3 / 1e12)
    assert r["l2l"]["peak"] == 1000.0
    # both leaves' expansions read, 8 targets written
    assert r["l2p"]["work_per_launch"] == 2 * 512 + 8 * 4
    assert r["m2l"]["peak"] == 1000.0 and r["m2l"]["bound"] == "tensor"
    r32 = bench.rooflines(TREE, _stats(False), types.SimpleNamespace(order=5, m2l="f32"), nt=8, ns=4,
                          ncell=1000, peaks=PEAKS, pipes=PIPES)
    assert r32["m2l"]["peak"] == pytest.approx(60.0) and r32["m2l"]["bound"] == "alu"


def test_clock_summary_from_nvidia_smi_rows(tmp_path):
    """The clock record of the timed region: median SM clock under load, the highest maximum
    clock seen, and every throttle reason that was active in any sample."""
    f = tmp_path / "clocks.csv"
    f.write_text(
        "0, 2070, 2070, 801.25, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
        "0, 1995, 2070, 1391.00, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n"
        "[N/A], [N/A]\n"
        "0, 2040, 2070, 1200.00, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n")
    s = bench.ClockSampler(0)
    s.path = str(f)
    c = s.summary()
    assert c == {"sm_mhz": 2040.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_clock_summary_flags_hardware_slowdown_and_no_samples(tmp_path):
    f = tmp_path / "clocks.csv"
    f.write_text("0, 1500, 2070, 900.0, 0x0000000000000008, Active, Not Active, Active, Not Active\n")
    s = bench.ClockSampler(0)
    s.path = str(f)
    assert s.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    s.path = str(tmp_path / "missing.csv")
    assert s.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
