"""Host-side arithmetic of the workload lines' roofline objects (no GPU)."""
import bench
import bench_workloads as bw


def test_roofline_reports_dominant_group():
    peak, _ = bench.measured_peak_hbm()
    r = bw._roofline({"a": (1e9, 2.0), "b": (6e9, 3.0)}, {"b": "k_b"})
    assert r["kernel"] == "k_b"
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert abs(r["achieved"] - 6e9 / 3e-3 / 1e9) < 1e-9
    assert abs(r["frac"] - r["achieved"] / peak) < 1e-12
    assert r["traffic"] is None
    assert r["phase_ms"] == {"a": 2.0, "b": 3.0}


def test_column_groups_sum_over_multiplies():
    st = {"nnzC_heavy": 10, "nnzB_heavy": 4, "gathered_nnz_exact": 20, "heavy_columns": 2, "nnzC": 30, "nnzB": 9,
          "light_columns": 5, "ms_num_heavy": 1.0, "ms_num_light": 0.5, "ms_sym_heavy": 0.25, "ms_sym_light": 0.1,
          "ms_gather": 0.05}
    g = bw._column_groups([st, st])
    assert g["num_heavy"] == (2 * (12 * (10 + 4 + 20) + 8 * 2), 2.0)
    assert g["num_light"] == (2 * (12 * (20 + 5 + 20) + 8 * 5), 1.0)
    assert g["gather"] == (2 * 24 * 20, 0.1)


def test_cpu_baseline_skipped_on_request():
    class A:
        no_cpu_baseline = True
    assert bw._cpu_baseline(A(), lambda: 1, "x") is None


def test_cpu_baseline_value():
    class A:
        no_cpu_baseline = False
    r = bw._cpu_baseline(A(), lambda: 10 ** 6, "sample", cores=1, min_seconds=0.01)
    assert r["kind"] == "oracle" and r["cores"] == 1
    products = r["value"] * r["seconds"] * 1e9 / 2
    reps = round(products / 1e6)
    assert reps >= 1 and abs(products - reps * 1e6) < 1e-3 * products
    assert r["seconds"] >= 0.01
