"""bench.py's command-line contract on the CPU: every workload it dispatches to exists, and the
reference arm (the CPU oracle) prints one well-formed JSON line."""
import argparse
import json

import bench


def test_every_dispatch_target_exists():
    for name in ("run_gpu", "run_sk", "run_vb_batch", "run_sk_batch", "run_rrbg", "run_e6", "run_vb_windows", "run_aging",
                 "run_reference", "run_profile_case", "main"):
        assert callable(getattr(bench, name, None)), name


def test_reference_arm_prints_one_line(monkeypatch, capsys):
    monkeypatch.setattr(bench, "N_VERTS", 1 << 12)  # a small graph of the same ensemble
    args = argparse.Namespace(steps=3, warmup=1, gpus=1)
    assert bench.run_reference(args) == 0
    lines = [l for l in capsys.readouterr().out.splitlines() if l.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["metric"] == "spin updates/ns"
    assert line["value"] > 0 and line["steps"] == 3 and line["warmup"] == 1
    assert line["higher_is_better"] is True and line["unit"] == "spin updates/ns"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_all_core_cpu_sample_runs_one_process_per_core():
    # spawned processes re-import bench; a small graph keeps the sample to a fraction of a second
    out = bench.cpu_baseline_all_cores(budget_lanes=2, n_verts=1 << 12)
    assert out["kind"] == "oracle" and out["unit"] == "spin updates/ns"
    assert out["cores"] >= 1 and out["value"] > 0
