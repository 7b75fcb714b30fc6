"""Host-side pieces of bench.py that need no GPU: the kernel name reported
for each step-a variant (it must match ncu's name for the same kernel) and the
rule that a recorded DRAM-traffic figure is reported only for the kernel
sources it was measured on."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.mark.parametrize("var,name", [
    (0, "cg_step_a_kernel<float, 12, 0>"),
    (4, "cg_step_a_kernel<float, 12, 4>"),
    (5, "cg_step_a_staged_kernel<float, 12, 2, 0, 0>"),
    (6, "cg_step_a_staged_kernel<float, 12, 4, 0, 0>"),
    (7, "cg_step_a_staged_kernel<float, 12, 2, 1, 0>"),
    (8, "cg_step_a_staged_kernel<float, 12, 3, 0, 1>"),
    (9, "cg_step_a_pg_staged_kernel<float, 12, 2, 0>"),
    (10, "cg_step_a_pg_staged_kernel<float, 12, 3, 0>"),
    (11, "cg_step_a_pg_kernel<float, 12>"),
    (12, "cg_step_a_pg_staged_kernel<float, 12, 2, 1>"),
    (13, "cg_step_a_pg_staged_kernel<float, 12, 3, 1>"),
    (14, "cg_step_a_pg2_kernel<float, 12, 2>"),
    (15, "cg_step_a_pg2_kernel<float, 12, 1>"),
])
def test_kernel_name_per_variant(var, name):
    assert bench.step_a_kernel_name({"step_a_variant": var, "k_bucket": 12}) == name


def test_recorded_traffic_needs_matching_kernel_and_sources(tmp_path, monkeypatch):
    import json
    rec = tmp_path / "traffic.json"
    h = bench.kernel_source_hash()
    rec.write_text(json.dumps({"records": [{"kernel": "K<float, 12, 4, 0, 0>", "bytes_per_launch": 123,
                                            "source_sha256": h}]}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path.parent))
    monkeypatch.setattr(bench, "TRAFFIC_RECORDS", os.path.join(tmp_path.name, "traffic.json"))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: h)
    assert bench.recorded_traffic("K<float, 12, 4, 0, 0>") == 123
    assert bench.recorded_traffic("K<float, 12, 2, 0, 0>") is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.recorded_traffic("K<float, 12, 4, 0, 0>") is None


def test_committed_traffic_records_parse():
    """The committed ncu traffic records are well-formed JSON."""
    import json
    with open(os.path.join(ROOT, bench.TRAFFIC_RECORDS)) as f:
        recs = json.load(f)["records"]
    assert recs
    for r in recs:
        assert {"kernel", "bytes_per_launch", "source_sha256", "workload"} <= set(r)
        assert int(r["bytes_per_launch"]) > 0 and len(r["source_sha256"]) == 16


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` times the oracle on the arm's own workload
    and prints one JSON line with the keys the benchmark contract names."""
    import json
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "lap2d_64", "--steps", "2", "--warmup", "3"], capture_output=True, text=True,
                         timeout=600, check=True).stdout.strip().splitlines()
    line = json.loads(out[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 3
    assert line["value"] > 0 and line["unit"] == "solves/s" and line["higher_is_better"] is True
    assert line["config"]["workload"].startswith("lap2d_64x64_k4")
    import oracle as O
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == O.threads_available()
    # the whole 64 x 64 solve fits a step: nothing is extrapolated, and ms_per_step is the solve's real time
    assert line["value_extrapolated"] is False
    assert abs(line["ms_per_step"] - 1000.0 / line["value"]) <= 0.5 * line["ms_per_step"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_cpu_baseline_scales_only_by_the_oracles_own_count(monkeypatch):
    """A sampled baseline is scaled by the inner-iteration count of a whole
    oracle solve recorded by oracle/record_counts.py, never by anything else:
    with no record its value is None."""
    from gen import lap2d_64_k4
    p = lap2d_64_k4()
    monkeypatch.setattr(bench, "full_solve_inner_iters", lambda name, mcg="identity": None)
    big = type("P", (), {})()
    for a in ("rowptr", "colind", "val", "V", "lam", "b", "k"):
        setattr(big, a, getattr(p, a))
    big.n, big.name = 200_000, p.name  # past the whole-solve threshold: sampled
    import oracle as O
    monkeypatch.setattr(O.System, "from_problem", classmethod(
        lambda cls, q: cls(p.rowptr, p.colind, p.val, p.V, p.lam)))
    cb = bench.cpu_baseline(big)
    assert cb["value"] is None and "no whole oracle solve" in cb["sample"]
    assert cb["serial"]["value"] is None
    monkeypatch.setattr(bench, "full_solve_inner_iters", lambda name, mcg="identity": 815)
    cb = bench.cpu_baseline(big)
    assert cb["value"] > 0 and "scaled by the 815 inner iterations" in cb["sample"]
    assert cb["serial"]["value"] > 0 and cb["serial"]["cores"] == 1 and cb["extrapolated"] is True
    assert cb["cores"] == O.threads_available() and cb["cpu_model"]


def test_reference_arm_follows_the_inner_tolerance():
    import json
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "lap2d_64", "--steps", "1", "--warmup", "3", "--inner-tol", "1e-2"], capture_output=True,
                         text=True, timeout=600, check=True).stdout.strip().splitlines()
    line = json.loads(out[-1])
    assert line["config"]["inner_tol"] == 1e-2 and line["value"] > 0


def test_inner_bytes_of_the_one_gather_iteration():
    """Step a of the one-gather iteration streams A (values and 16-bit deltas),
    V_hat and three vectors; step b seven vectors.  With V_hat in BF16 only
    V_hat's term halves."""
    n, nnz, k = 1000, 6800, 10
    cfg = {"step_a_variant": 14, "index_bytes": 2}
    a, b = bench.inner_bytes(cfg, n, nnz, k, 4, "identity")
    assert a == nnz * (4 + 2) + k * n * 4 + 3 * n * 4 and b == 7 * n * 4
    a16, b16 = bench.inner_bytes(cfg, n, nnz, k, 4, "identity", vw=2)
    assert a - a16 == k * n * 2 and b16 == b
    a64, _ = bench.inner_bytes({"step_a_variant": 9, "index_bytes": 4}, n, nnz, k, 8, "jacobi")
    assert a64 == nnz * 12 + k * n * 8 + 3 * n * 8 + n * 8
