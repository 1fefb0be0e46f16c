"""Per-step JSON-line records of a run (paper_1704_01888_gb300.log)."""
import io
import json

import pytest

from paper_1704_01888_gb300 import log


def _obs(beta, R, lnQ, lnZ, meanE, meanM):
    return {"beta": beta, "lnQ": lnQ, "lnZ": lnZ, "meanE": meanE, "meanE2": meanE * meanE, "C": 0.5,
            "meanM": meanM, "S_f": 1.25, "R": R, "n_families": 7, "sumE": 0, "sumE2": 0, "sumMt": 0,
            "n_near_ties": 0}


def test_step_records_and_jsonl(tmp_path):
    N = 256
    obs = [_obs(0.1, 1000, -3.0, 100.0, -51.2, 12.8), _obs(0.25, 998, -5.0, 95.0, -128.0, 25.6)]
    recs = log.step_records(obs, N, 0.0, seconds_per_step=0.002, overlap_target=0.85)
    assert [r["dbeta"] for r in recs] == [pytest.approx(0.1), pytest.approx(0.15)]
    assert recs[0]["e"] == pytest.approx(-0.2) and recs[1]["m"] == pytest.approx(0.1)
    assert recs[1]["R"] == 998 and recs[0]["lnZ"] == 100.0 and recs[0]["S_f"] == 1.25
    assert all(r["overlap_target"] == 0.85 and r["seconds_per_step"] == 0.002 for r in recs)
    assert "overlap_target" not in log.step_records(obs, N, 0.0)[0]
    buf = io.StringIO()
    log.write_jsonl(buf, recs)
    lines = buf.getvalue().splitlines()
    assert len(lines) == 2 and json.loads(lines[1]) == recs[1]
    path = tmp_path / "run.jsonl"
    log.write_jsonl(str(path), recs[:1])
    log.write_jsonl(str(path), recs[1:])  # appends
    assert [json.loads(x) for x in path.read_text().splitlines()] == recs
