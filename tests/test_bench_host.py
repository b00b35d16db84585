"""Host-side logic of bench.py that needs no GPU.

* The DRAM-traffic figure of the roofline is taken from the committed ncu record only
  while the kernel source still hashes to the value recorded with it; any edit makes
  it null.
* The measured unit peaks are read by key; a missing key or file gives None.
* The product-equivalents of one evaluation (the CPU baseline's multiplier) follow
  CG iterations + residual recomputes + 2 (p - 1) derivative passes.
"""
import hashlib
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture()
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _fake_root(tmp_path, src_text, recorded_hash):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "src").mkdir()
    (tmp_path / "src" / "k.cu").write_text(src_text)
    (tmp_path / "profiles" / "dram_traffic.txt").write_text(
        "# comment line\n"
        f"ktag 12345 src/k.cu {recorded_hash}\n")
    (tmp_path / "profiles" / "unit_peaks_gb300.txt").write_text(
        "# comment\nex2_f32_per_s 1.5e13 results/s\nbroken notanumber\n")


def test_traffic_only_while_source_unchanged(bench, tmp_path):
    text = "__global__ void k() {}\n"
    h = hashlib.sha256(text.encode()).hexdigest()[:16]
    _fake_root(tmp_path, text, h)
    bench.ROOT = str(tmp_path)
    assert bench._traffic_from_profiles("ktag") == 12345.0
    assert bench._traffic_from_profiles("other") is None
    (tmp_path / "src" / "k.cu").write_text(text + "// edited\n")
    assert bench._traffic_from_profiles("ktag") is None


def test_unit_peaks_by_key(bench, tmp_path):
    _fake_root(tmp_path, "", "0" * 16)
    bench.ROOT = str(tmp_path)
    assert bench._unit_peak("ex2_f32_per_s") == 1.5e13
    assert bench._unit_peak("broken") is None
    assert bench._unit_peak("missing") is None
    (tmp_path / "profiles" / "unit_peaks_gb300.txt").unlink()
    assert bench._unit_peak("ex2_f32_per_s") is None


def test_committed_records_are_readable(bench):
    # the committed records parse; the traffic entry matches the current product source
    assert bench._unit_peak("ex2_f32_per_s") > 0
    assert bench._unit_peak("fp32_fma_flops") > 0
    t = bench._traffic_from_profiles("kmvm_tc_bf16")
    assert t is None or t > 0


def test_products_per_eval(bench):
    # 334 iterations, a recompute every 25 (14), and 2 (18 - 1) derivative passes
    assert bench.products_per_eval(334, 25, 18) == 334 + 14 + 34
    assert bench.products_per_eval(25, 25, 1) == 25 + 1


def test_extrapolation_scales_by_size_and_products(bench):
    """The oracle's subsample time scales with n^2 per product and with the ratio of
    product-equivalents per evaluation."""
    t = bench.extrapolate(2.0, 20, 300, n_full=4000, n_sub=2000, n_hyper=18)
    ratio = bench.products_per_eval(300, 25, 18) / bench.products_per_eval(20, 25, 18)
    assert t == pytest.approx(2.0 * 4.0 * ratio)
    assert bench.extrapolate(1.0, 50, 50, n_full=2000, n_sub=2000) == pytest.approx(1.0)


def test_cpu_info_reports_cores_and_threads(bench):
    info = bench._cpu_info()
    assert info["nproc"] >= 1 and info["threads"] >= 1
