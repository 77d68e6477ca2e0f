"""Host-side arithmetic of bench.py's whole-build roofline (no GPU).

The whole build's roofline time is the sum over kernels of each kernel's
roofline time: the larger of its algorithmic bytes at the measured HBM
bandwidth and its arithmetic at the peak of its kind.
"""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _st(launches, bytes_, flops=0.0, ms=1.0):
    return {"launches": launches, "ms": ms, "bytes": bytes_, "flops": flops, "items": 0.0}


def test_hbm_kernel_at_peak_is_one(bench):
    peaks, _ = bench.measured_peaks()
    bw = float(peaks["hbm_gbs"]) * 1e9
    # two builds, each moving exactly 1 ms worth of bytes at the measured bandwidth
    stats = {"k4_merge": _st(8, 2 * bw * 1e-3)}
    r = bench.whole_build_roofline(stats, None, 2, 1.0)
    assert r["roofline_ms_per_step"] == pytest.approx(1.0, rel=1e-6)
    assert r["frac"] == pytest.approx(1.0, rel=1e-6)
    assert r["roofline_ms_by_bound"]["hbm"] == pytest.approx(1.0, rel=1e-6)
    # the same kernel measured at four times its roofline time
    assert bench.whole_build_roofline(stats, None, 2, 4.0)["frac"] == pytest.approx(0.25, rel=1e-6)


def test_kernel_takes_the_larger_of_bytes_and_arithmetic(bench):
    peaks, _ = bench.measured_peaks()
    bw = float(peaks["hbm_gbs"]) * 1e9
    tc = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))) * 1e12
    # a tensor kernel whose arithmetic takes 3 ms and whose bytes take 1 ms
    t, bound = bench.kernel_roofline_ms("k2_leaf_bf16", _st(1, bw * 1e-3, 3e-3 * tc), None, peaks)
    assert bound == "tensor" and t == pytest.approx(3.0, rel=1e-6)
    # FP8 runs at twice the BF16 rate
    t8, _ = bench.kernel_roofline_ms("k2_leaf_fp8", _st(1, bw * 1e-3, 3e-3 * tc), None, peaks)
    assert t8 == pytest.approx(1.5, rel=1e-6)
    # bytes dominate: the same kernel with 5 ms of bytes
    t, bound = bench.kernel_roofline_ms("k2_leaf_bf16", _st(1, 5 * bw * 1e-3, 3e-3 * tc), None, peaks)
    assert bound == "hbm" and t == pytest.approx(5.0, rel=1e-6)
    # an FP32 kernel: flops are counted 3 per pair and dim, two issue slots
    ops = 152 * 128 * 2000e6  # issue slots per second at 2000 MHz
    t, bound = bench.kernel_roofline_ms("k5_join", _st(1, 0.0, 1.5 * ops * 2e-3), {"sm_mhz": 2000.0}, peaks)
    assert bound == "alu" and t == pytest.approx(2.0, rel=1e-6)


def test_sum_over_kernels_and_unlaunched_kernels(bench):
    peaks, _ = bench.measured_peaks()
    bw = float(peaks["hbm_gbs"]) * 1e9
    stats = {"k1_project": _st(65, bw * 2e-3), "k5_join_tc": _st(8, bw * 3e-3), "k6_fill": _st(0, 1e12)}
    r = bench.whole_build_roofline(stats, None, 1, 10.0)
    assert r["roofline_ms_per_step"] == pytest.approx(5.0, rel=1e-6)
    assert r["frac"] == pytest.approx(0.5, rel=1e-6)


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` times the CPU oracle on the headline's
    recipe and prints one JSON line with the same metric, unit and config as
    the GPU arm would, its sample stated in cpu_baseline."""
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    spec = importlib.util.spec_from_file_location("bench_cfg", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    assert line["impl"] == "reference"
    assert line["metric"] == "kNN-graph build points/s at recall@k vs exact" and line["unit"] == "points/s"
    assert line["higher_is_better"] is True and line["steps"] == 1
    # the GPU arm's default precision is BF16: the two lines carry one config
    assert line["config"] == mod.workload_config(mod.DEFAULT_WORKLOAD, "bf16")
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def test_profiled_traffic_only_for_the_same_sources(bench, tmp_path, monkeypatch):
    """The committed ncu summary gives a kernel's DRAM bytes per algorithmic
    byte only while the sources it was captured on are unchanged; for the
    tensor-core join those are join_tc.cu and join.cu (which sets its node
    order)."""
    import hashlib
    csrc = tmp_path / "paper_1701_08475_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (csrc / "join_tc.cu").write_text("// kernel\n")
    (csrc / "join.cu").write_text("// order\n")
    h = hashlib.sha256(b"// kernel\n// order\n").hexdigest()[:16]
    (tmp_path / "profiles" / "k5_join_tc_sift-like-300k.md").write_text(
        "# summary\n\n- source_sha256_16: `%s`\n- dram_bytes_per_alg_byte: 0.25\n" % h)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # a smaller case of the same recipe stands in for the full-size workload
    assert bench.profiled_traffic("k5_join_tc", "sift-like-1m-d128") == 0.25
    (csrc / "join.cu").write_text("// another order\n")
    assert bench.profiled_traffic("k5_join_tc", "sift-like-1m-d128") is None
    assert bench.profiled_traffic("k4_merge", "sift-like-1m-d128") is None   # no summary at all


def test_autotuner_keeps_the_fastest_within_the_recall_slack():
    from paper_1701_08475_gb300.autotune import pick
    rows = [(64, 2, 4.8, 0.9917), (128, 2, 4.5, 0.9947), (128, 3, 5.1, 0.9945), (256, 2, 4.1, 0.9920),
            (256, 4, 3.9, 0.9900)]
    # best recall 0.9947: within 0.002 are the rows of recall >= 0.9927, the fastest of them (128, 2)
    assert pick(rows, 0.002)[:2] == (128, 2)
    # a looser slack admits (256, 2) at 4.1 ms and (256, 4) at 3.9 ms
    assert pick(rows, 0.003)[:2] == (256, 2)
    assert pick(rows, 0.005)[:2] == (256, 4)
    # equal times: the first row wins
    assert pick([(64, 2, 1.0, 0.5), (128, 2, 1.0, 0.5)], 0.0)[:2] == (64, 2)
