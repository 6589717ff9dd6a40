"""The default bench line's short runs of the other workloads, on CPU: the
child runs are replaced by fakes, and the record keeps each run's rate,
quality and roofline, and records a failed or silent run instead of
raising."""
import json
import subprocess
import types

import bench


def _fake_run(outputs):
    calls = []

    def run(cmd, capture_output, text, timeout, cwd):
        calls.append(cmd)
        rc, stdout = outputs[len(calls) - 1]
        return types.SimpleNamespace(returncode=rc, stdout=stdout, stderr="boom")
    return run, calls


def test_other_workloads_record_parses_and_records_failures(monkeypatch):
    line = {"metric": "m", "value": 12.5, "unit": "columns/s", "ms_per_step": 3.0,
            "steps": 3, "warmup": 2, "dtype": "f64", "quality": {"max_over_n": 0.01},
            "config": {"workload": "w"}, "extra": 1,
            "roofline": {"kernel": "k", "bound": "alu", "achieved": 1.0, "peak": 1.2,
                         "unit": "TFLOP/s", "frac": 0.83, "traffic": 5}}
    entries = [("a", ["--x"], "first"), ("b", [], "second"), ("c", [], "third")]
    outputs = [(0, "noise\n" + json.dumps(line) + "\n"), (1, ""), (0, "no json here")]
    run, calls = _fake_run(outputs)
    monkeypatch.setattr(bench, "OTHER_WORKLOADS", entries)
    monkeypatch.setattr(subprocess, "run", run)
    rec = bench.other_workloads_record(steps=3, warmup=2)
    assert len(calls) == 3
    assert "--no-cpu-baseline" in calls[0] and "--x" in calls[0]
    assert calls[0][calls[0].index("--steps") + 1] == "3"
    a = rec["a"]
    assert a["value"] == 12.5 and a["unit"] == "columns/s" and a["workload"] == "w"
    assert a["roofline"]["frac"] == 0.83 and "traffic" not in a["roofline"]
    assert "extra" not in a and a["what"] == "first"
    assert rec["b"]["error"] == "exit 1"
    assert rec["c"]["error"] == "exit 0"


def test_other_workloads_cover_every_workload_kind():
    # the n = 4096 forms (config-0 and clustered), the pencil, and the
    # triangular-solve, left, batched-pencil, reordering and Hessenberg runs
    names = [n for n, _, _ in bench.OTHER_WORKLOADS]
    for prefix in ("n4096_fp64", "n4096_split", "n4096_clustered", "pencil_n8192", "trsolve",
                   "left", "batched_pencils", "window", "hessenberg"):
        assert any(n.startswith(prefix) for n in names), prefix
    args = {n: a for n, a, _ in bench.OTHER_WORKLOADS}
    assert "adversarial" in args["n4096_clustered_fp64"]
