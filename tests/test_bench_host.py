"""Host logic of bench.py (no GPU): the roofline object built from a launch's statistics, the traffic figure
taken from the committed ncu summary only while the kernel's source is unchanged, and the byte formulas."""
import json

import pytest

import bench


def _res(iters=50.0, ms=3.0, refine=1.0):
    N, nnz = 2_097_152, 31_065_598
    return {"N": N, "nnz": nnz,
            "trace": {"steps": 10, "ms_solve_V": 10 * ms, "iters_V": 10 * iters, "refine_V": 10 * refine},
            "layout": {"column_bytes": 2, "kernel_code": 2, "nnz_stored": nnz}}


def test_roofline_divides_algorithmic_bytes_by_the_launch_time():
    peaks = {"hbm_gbs": 6500.0}
    r = bench.roofline(_res(), True, peaks, "measured")
    alg = bench.alg_bytes_mixed(2_097_152, 31_065_598, 50.0, 1.0, 2)
    assert r["alg_bytes_per_launch"] == pytest.approx(alg)
    assert r["achieved"] == pytest.approx(alg / 3.0e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6500.0)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and "of measured" in r["peak_kind"]
    f = bench.roofline(_res(iters=40.0, ms=6.0, refine=0.0), False, peaks, "fallback")
    assert f["kernel"].startswith("k_cg64") and "of fallback" in f["peak_kind"] and f["fp64_pipe"]["bound"] == "alu"


def test_traffic_only_for_the_captured_source(tmp_path, monkeypatch):
    """The committed DRAM-per-algorithmic-byte ratio scales the launch's bytes while the source hash matches;
    any other source gives null."""
    src = tmp_path / "paper_2409_13036_b300" / "csrc"
    src.mkdir(parents=True)
    (src / "krylov.cu").write_text("// kernel source\n")
    (tmp_path / "profiles").mkdir()
    entry = {"source": "krylov.cu", "source_sha256": bench._source_hash(str(src / "krylov.cu")),
             "dram_per_alg_byte": 0.6}
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps({"k_cg_mixed<2>": entry}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    r = bench.roofline(_res(), True, {"hbm_gbs": 6500.0}, "measured")
    assert r["traffic"] == pytest.approx(0.6 * r["alg_bytes_per_launch"])
    (src / "krylov.cu").write_text("// kernel source, changed\n")
    assert bench.roofline(_res(), True, {"hbm_gbs": 6500.0}, "measured")["traffic"] is None


def test_handed_over_residual_saves_one_matrix_stream():
    """A residual handed over by the projection replaces the first FP64 residual SpMV: (8 + column bytes) per
    nonzero less, in both CG byte counts."""
    N, nnz = 1000, 15000
    for cb in (2, 4):
        assert (bench.alg_bytes_mixed(N, nnz, 30, 1, cb, given_r0=False) - bench.alg_bytes_mixed(N, nnz, 30, 1, cb)
                == (8 + cb) * nnz)
        assert (bench.alg_bytes_cg64(N, nnz, 30, cb, given_r0=False) - bench.alg_bytes_cg64(N, nnz, 30, cb)
                == (8 + cb) * nnz)
    # one more inner iteration streams the FP32 matrix once more
    assert bench.alg_bytes_mixed(N, nnz, 31, 1, 2) - bench.alg_bytes_mixed(N, nnz, 30, 1, 2) == 6 * nnz + 56 * N


def test_cpu_baseline_line_from_timed_steps():
    """steps/s over the steps after the first (which also factors the constant thermal matrix), the 60-step run
    extrapolated from them, the host recorded, the GPU's rate on the same workload carried beside it."""
    t = {"setup_s": 10.0, "nodes": 117649, "step_s": [200.0, 100.0, 110.0]}
    c1 = {"steps_per_s": 50.0}
    small = {"fp64_cg": {"steps_per_s": 1500.0}, "mixed": {"steps_per_s": 1700.0}}
    out = bench.cpu_baseline_line(t, c1, small)
    assert out["value"] == pytest.approx(2 / 210.0)
    assert out["extrapolated_60_step_run_s"] == pytest.approx(10.0 + 200.0 + 59 * 105.0)
    assert out["cores"] == 1 and out["kind"] == "oracle" and "48^3" in out["config"]
    assert out["host"]["nproc"] >= 1 and out["c1_8"] == c1
    assert out["gpu_same_config_steps_per_s"] == {"fp64_cg": 1500.0, "mixed": 1700.0}
    one = bench.cpu_baseline_line({"setup_s": 1.0, "nodes": 1, "step_s": [4.0]}, None, None)
    assert one["value"] == pytest.approx(0.25)
    none = bench.cpu_baseline_line({"setup_s": None, "nodes": None, "step_s": []}, None, None)
    assert none["value"] is None


def test_accuracy_headline_picks_the_configured_arms():
    arm = lambda **kw: {"rel_err_T_max": 1.0, "rel_err_V_max": 2.0, "psnr_T_db_min": 3.0, "steps_per_s": 4.0,
                        "status": "OK", **kw}
    acc = {"steps": 900, "reference": {"tol": 1e-13},
           "mixed": [arm(tol=t, rel_err_V_max=t) for t in (1e-6, 1e-8, 1e-10, 1e-12)],
           "fp64": [arm(arm="fp64 double-word elements", tol=1e-10, rel_err_T_max=7.0),
                    arm(arm="fp64 FP64 elements", tol=1e-10, rel_err_T_max=8.0),
                    arm(arm="fp64 double-word elements", tol=1e-13, rel_err_T_max=9.0)]}
    h = bench.accuracy_headline(acc)
    assert h["mixed_tol_1e-10"]["rel_err_V_max"] == 1e-10
    assert h["fp64_tol_1e-10"]["rel_err_T_max"] == 7.0
    assert h["fp64_fp64_elements_tol_1e-10"]["rel_err_T_max"] == 8.0
    assert h["double_word_vs_fp64_elements_tol_1e-13"]["rel_err_T_max"] == 9.0


def test_dram_fraction_from_traffic(tmp_path, monkeypatch):
    """dram_frac = measured DRAM bytes per launch / launch time / peak, beside the algorithmic fraction."""
    src = tmp_path / "paper_2409_13036_b300" / "csrc"
    src.mkdir(parents=True)
    (src / "krylov.cu").write_text("// kernel source\n")
    (tmp_path / "profiles").mkdir()
    entry = {"source": "krylov.cu", "source_sha256": bench._source_hash(str(src / "krylov.cu")),
             "dram_per_alg_byte": 0.5}
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps({"k_cg_mixed<2>": entry}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    r = bench.roofline(_res(ms=3.0), True, {"hbm_gbs": 6500.0}, "measured")
    assert r["dram_achieved"] == pytest.approx(r["traffic"] / 3.0e-3 / 1e9)
    assert r["dram_frac"] == pytest.approx(0.5 * r["frac"])


def test_gmres_fp64_accounting():
    """GMRES's FP64 work counts its SpMVs and a few operations per row (the Gram-Schmidt runs on the FP32 pipes);
    the FP64-pipe line divides by 2 FMA/clk/SM x 148 SMs x 2.032 GHz."""
    import bench
    N, nnz = 1000, 15000
    assert bench.alg_fma_gmres(N, nnz, 10, 1) == 10 * (nnz + 5 * N) + (nnz + 2 * N)
    assert bench.alg_fma_gmres(N, nnz, 10, 0) == bench.alg_fma_gmres(N, nnz, 10, 1)  # at least one cycle
    line = bench.fp64_pipe_line(148 * 2 * 2.032e9 * 1e-3, 1.0)  # one millisecond at the peak rate
    assert abs(line["frac"] - 1.0) < 1e-12 and line["bound"] == "alu"
