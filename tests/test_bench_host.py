"""bench.py's host side on CPU: the reference arm (the oracle timed on the
host cores) prints one JSON line with the benchmark contract's keys for
every workload, and ranks other than 0 of a multi-rank launch exit without
work."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

KEYS = ["impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
        "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"]


def _bench(args, env=None):
    e = dict(os.environ)
    e.update(env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                          timeout=600, cwd=ROOT, env=e)


@pytest.mark.parametrize("name", bench.WORKLOAD_NAMES)
def test_reference_arm_prints_one_contract_line(name):
    r = _bench(["--impl", "reference", "--workload", name, "--steps", "3", "--warmup", "3"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert all(k in d for k in KEYS), sorted(set(KEYS) - set(d))
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 3 and d["warmup"] == 3
    assert d["n_gpus"] == 1 and d["higher_is_better"] is True and d["data"] == "synthetic"
    assert d["config"]["workload"] == bench.full_size_desc(name)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_without_output():
    r = _bench(["--impl", "reference", "--steps", "3", "--warmup", "3"],
               env={"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


def test_every_workload_has_a_full_size_description():
    for name in bench.WORKLOAD_NAMES:
        assert bench.full_size_desc(name)


@pytest.mark.parametrize("name", ["quat", "ragged_f64"])
def test_cpu_baseline_reports_all_cores_and_one_thread(name):
    cb = bench.cpu_baseline(name, seconds=0.5, single_seconds=0.5)
    assert cb["kind"] == "oracle" and cb["unit"] == "vectors/s" and cb["value"] > 0 and cb["GB_per_s"] > 0
    assert cb["cores"] == bench.cpu_threads()
    st = cb["single_thread"]
    assert st["cores"] == 1 and st["value"] > 0 and st["GB_per_s"] > 0


def test_exact_error_report_on_oracle_outputs():
    """The bench's error report (oracle/exact.py) on the oracle's own results:
    every vector within the paper's bounds, the 64 binary64 edge vectors
    included; a result pushed 4 ulps off in one component is reported as
    outside the bound with its ulp error."""
    import numpy as np
    import oracle
    from oracle import exact
    from paper_1606_06508_gb300 import synth
    q = synth.quaternions_f32(300, seed=1)
    y, r, _, _ = oracle.normalize(q.reshape(-1), dim=4)
    y = y.reshape(-1, 4)
    rep = bench._exact_errors([(q[i], y[i], r[i]) for i in range(q.shape[0])], exact.F32)
    assert rep["all_within_bounds"] and rep["vectors_checked"] == 300
    assert 0 < rep["direction"]["max_u"] <= 5.001 and rep["direction"]["n_at_max"] == 4
    assert 0 <= rep["norm"]["max_u"] <= 3 and rep["component_ulp_max"] > 0
    e = synth.edge_vectors_d3_f64()
    ye, re_, _, _ = oracle.normalize(e.reshape(-1), dim=3)
    ye = ye.reshape(-1, 3)
    rep = bench._exact_errors([(e[i], ye[i], re_[i]) for i in range(64)], exact.F64)
    assert rep["all_within_bounds"] and rep["vectors_checked"] == 64 - 4  # the four zero vectors are skipped
    assert rep["sin_phi"]["max_u"] <= 1.001
    bad = y[0].copy()
    k = int(np.argmax(np.abs(bad)))
    bad[k] = np.float32(bad[k] + np.float32(4) * np.spacing(bad[k]))
    rep = bench._exact_errors([(q[0], bad, r[0])], exact.F32)
    assert not rep["all_within_bounds"] and rep["component_ulp_max"] >= 3.5
