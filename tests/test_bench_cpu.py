"""Host-side pieces of bench.py that run after the timed region: they must
not fail on a missing, stale or old-format traffic record."""
import json

import bench


def test_kernel_traffic_record_forms(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "profiles").mkdir()
    (tmp_path / "k.cu").write_text("kernel source")
    path = tmp_path / "profiles" / "traffic.txt"
    assert bench.kernel_traffic("sap_f32") is None                      # no file
    path.write_text(json.dumps({"sap_f32": {"source": "k.cu", "source_sha": "x"}}))
    assert bench.kernel_traffic("sap_f32") is None                      # old form
    rec = {"sources": ["k.cu"], "source_sha": bench.sources_sha(["k.cu"]), "bytes_per_alg_byte": 1.5}
    path.write_text(json.dumps({"sap_f32": rec}))
    assert bench.kernel_traffic("sap_f32")["bytes_per_alg_byte"] == 1.5  # current
    (tmp_path / "k.cu").write_text("changed kernel source")
    assert bench.kernel_traffic("sap_f32") is None                      # stale
    path.write_text("not json")
    assert bench.kernel_traffic("sap_f32") is None


def test_committed_traffic_record_parses():
    bench.kernel_traffic("sap_f32")       # current or stale, never an exception


def test_roofline_record():
    pk = bench.peaks()
    assert pk["hbm_gbs"] > 0
    prof = {"sap_f32": {"ms": 2000.0, "bytes": 4e12, "flops": 8e13, "launches": 1000},
            "blas": {"ms": 500.0, "bytes": 3e12, "flops": 1e11, "launches": 4000}}
    r = bench.roofline(prof, 3000.0, {"sm_mhz": 2070.0}, pk, sms=152)
    assert r["kernel"] == "sap_f32" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert abs(r["achieved"] - 40.0) < 1e-6 and abs(r["share_of_step"] - 0.667) < 1e-3
    assert r["algorithmic_bytes_per_launch"] == 4_000_000_000
    prof["sap_f32"]["flops"] = 1e12        # below the ridge: HBM-bound
    r = bench.roofline(prof, 3000.0, None, pk, sms=152)
    assert r["bound"] == "hbm" and abs(r["achieved"] - 2000.0) < 1e-6


def test_iteration_counts_record_and_cpu_sample():
    """The committed iteration counts (written by oracle/gcr_iteration_counts.py)
    carry what the CPU baseline needs, and a one-iteration sample of it runs."""
    import os
    counts = json.load(open(os.path.join(bench.ROOT, "oracle", "gcr_iteration_counts.json")))
    for key in ("dims", "eps", "csw", "kappa", "seed", "iters_sloppy", "iters_exact_from_sloppy"):
        assert key in counts
    assert counts["residual_sloppy"] <= counts["sloppy_tol"] and counts["residual_exact"] <= counts["exact_tol"]
    v, desc, cores, v1 = bench.oracle_sample(max_iter=1, parallel=False)
    assert v > 0 and v1 > 0 and cores == 1
    assert bench.lattice_label(counts["dims"]) in desc
