"""The run CLI (paper_1905_04065_gb300.run): JSON-lines log with throughput, energy and the drift
of each chunk's full recompute, checkpoints, and a resumed run that continues the same trajectory
(a chunk ends with a full recompute, which is also what a resume does, so both runs hold the same
state at every chunk boundary)."""
import json

import pytest

pytestmark = pytest.mark.gpu


def _lines(path):
    return [json.loads(x) for x in open(path)]


def test_run_log_and_resume(tmp_path):
    from paper_1905_04065_gb300 import run
    straight = tmp_path / "straight.jsonl"
    assert run.main(["--workload", "small", "--steps", "60", "--recompute-every", "20", "--precision", "fp64",
                     "--log", str(straight)]) == 0
    rec = _lines(straight)
    assert [r["event"] for r in rec] == ["start", "chunk", "chunk", "chunk"]
    assert [r["step"] for r in rec[1:]] == [20, 40, 60]
    for r in rec[1:]:
        assert r["kmc_steps_per_s"] > 0 and r["dU_evals_per_s"] > 0 and r["sim_time"] > 0
        assert r["drift_potential"] < 1e-4 and r["drift_energy"] < 1e-4
    ck = tmp_path / "ck.npz"
    first = tmp_path / "first.jsonl"
    assert run.main(["--workload", "small", "--steps", "40", "--recompute-every", "20", "--precision", "fp64",
                     "--log", str(first), "--checkpoint", str(ck)]) == 0
    second = tmp_path / "second.jsonl"
    assert run.main(["--steps", "20", "--recompute-every", "20", "--precision", "fp64", "--log", str(second),
                     "--resume", str(ck)]) == 0
    r2 = _lines(second)
    assert r2[0]["resumed"] and r2[0]["step"] == 40 and r2[-1]["step"] == 60
    assert abs(r2[-1]["energy"] - rec[-1]["energy"]) < 1e-9 * abs(rec[-1]["energy"])
    assert abs(r2[-1]["sim_time"] - rec[-1]["sim_time"]) < 1e-9 * rec[-1]["sim_time"]
