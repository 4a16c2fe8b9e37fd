"""Host logic of bench.py (no GPU): the per-phase roofline table, the
source-hash guard of the measured DRAM traffic and the accuracy report
against the oracle's stored samples."""
import bench


def _prof():
    return {"schur": {"ms": 2.0, "flops": 40e9, "bytes": 1e9, "launches": 9},
            "apply": {"ms": 4.0, "flops": 1e9, "bytes": 8e9, "launches": 8},
            "cpqr": {"ms": 10.0, "flops": 20e9, "bytes": 6e8, "launches": 212}}


def test_phase_rooflines_bounds_and_fractions():
    peaks = {"hbm_gbs": 8000.0, "bf16_tflops": 2000.0, "_source": "test"}
    r = bench.phase_rooflines(_prof(), peaks, "tf32")
    assert r["apply"]["bound"] == "hbm" and abs(r["apply"]["achieved"] - 2000.0) < 1e-9
    assert abs(r["apply"]["frac"] - 0.25) < 1e-9
    assert r["schur"]["bound"] == "tensor" and r["schur"]["peak"] == bench.TF32_TENSOR_TFLOPS
    assert abs(r["schur"]["achieved"] - 20.0) < 1e-9
    assert r["cpqr"]["bound"] == "alu" and r["cpqr"]["peak"] == bench.FP32_ALU_TFLOPS
    rb = bench.phase_rooflines(_prof(), peaks, "bf16")
    assert rb["schur"]["peak"] == 2000.0 and abs(rb["schur"]["frac"] - 0.01) < 1e-9
    rf = bench.phase_rooflines(_prof(), peaks, "fp32")
    assert rf["schur"]["bound"] == "alu"  # SIMT Schur in the FP32 form


def test_measured_traffic_tied_to_source_hash(tmp_path, monkeypatch):
    src = tmp_path / "k.cuh"
    src.write_text("kernel")
    import hashlib
    good = hashlib.sha256(b"kernel").hexdigest()
    monkeypatch.setattr(bench, "MEASURED_TRAFFIC", {"x": {"bytes_per_launch": 5.0, "src": [str(src)], "sha256": [good]}})
    assert bench.measured_traffic("x", bench.GRID) == 5.0
    assert bench.measured_traffic("x", bench.GRID + 1) is None  # another workload size
    src.write_text("kernel changed")
    assert bench.measured_traffic("x", bench.GRID) is None


def test_x_vs_oracle_against_stored_samples():
    """The benchmark's accuracy report reads the oracle's stored samples: an
    x that carries exactly those samples (and the stored norm) reports zero
    sampled error; a perturbed one reports the perturbation."""
    import json
    import os

    import numpy as np
    g = json.load(open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                    bench.ORACLE_GOLDEN)))
    n = 64 ** 3
    idx = np.asarray(g["sample_idx"])
    x = np.zeros(n)
    x[idx] = g["sample_x"]
    rest = np.setdiff1d(np.arange(n), idx)
    # fill the other entries so that ||x|| equals the stored norm
    x[rest[0]] = np.sqrt(g["x_norm"] ** 2 - np.sum(np.square(g["sample_x"])))
    r = bench.x_vs_oracle({"a": x, "b": x * (1 + 1e-6)})
    assert r["samples"] == 256 and r["oracle_iters"] == g["iters"]
    assert r["a"]["sampled_rel_err"] == 0.0 and r["a"]["norm_rel_err"] < 1e-14
    assert abs(r["b"]["sampled_rel_err"] - 1e-6) < 1e-12


def test_measured_traffic_per_step_divided_by_live_launches(tmp_path, monkeypatch):
    """A family measured per factorization (all its launches in one capture)
    reports that total over the launch count of the profiled run, so the
    per-launch figure follows a change of launch grouping; the roofline line
    carries it."""
    src = tmp_path / "q.cuh"
    src.write_text("qr")
    import hashlib
    good = hashlib.sha256(b"qr").hexdigest()
    monkeypatch.setattr(bench, "MEASURED_TRAFFIC",
                        {"cpqr": {"bytes_per_step": 600e6, "src": [str(src)], "sha256": [good]}})
    assert bench.measured_traffic("cpqr", bench.GRID, 240) == 2.5e6
    assert bench.measured_traffic("cpqr", bench.GRID, 300) == 2e6
    peaks = {"hbm_gbs": 8000.0, "bf16_tflops": 2000.0, "_source": "test"}
    prof = _prof()
    prof["cpqr"]["launches"] = 240
    r = bench.make_roofline(prof, peaks, grid=bench.GRID)
    assert r["kernel"] == "cpqr" and r["traffic"] == 2.5e6 and r["launches"] == 240
    assert abs(r["achieved"] - 2.0) < 1e-12 and r["bound"] == "alu"


def test_oracle_runs_all_core_leg_matches_single_core():
    """The all-core leg of the CPU baseline (the oracle's factorization on a
    process pool) runs through the same subprocess recipe as the single-core
    leg and reaches the same iterations, rank structure and memory."""
    one = bench.oracle_phases(bench.oracle_runs(grid=12, levels=4))
    two = bench.oracle_phases(bench.oracle_runs(grid=12, levels=4, workers=2))
    assert (one["n_cg"], one["size_top"], one["mem_f"]) == (two["n_cg"], two["size_top"], two["mem_f"])
    assert one["relres"] <= 1e-10 and two["relres"] <= 1e-10
