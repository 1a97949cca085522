"""Disorder averages of a run's JSON lines (report.py), on a synthetic file."""
import json

import numpy as np

from paper_2605_25872_gb300.analysis import append_jsonl
from paper_2605_25872_gb300.report import disorder_averages, load, main


def test_disorder_averages_and_errors(tmp_path, capsys):
    rng = np.random.default_rng(3)
    recs = []
    e = {}
    for b in (0, 1):
        for s in range(5):
            for k, T in enumerate((0.2, 1.0)):
                v = float(rng.normal(-1.5, 0.1))
                e.setdefault((b, k), []).append(v)
                recs.append({"bin": b, "sample": s, "k": k, "T": T, "n": 8, "e": v, "e2": v * v, "q": 0.0,
                             "q2": 0.3, "q4": 0.1, "ql": 0.7, "S": 0.0, "rule": "metropolis"})
    path = tmp_path / "r.jsonl"
    append_jsonl(path, recs)
    append_jsonl(path, [{"summary": True, "L": 4, "samples": 5, "emcs": 16, "tau_trw_median": None,
                         "spin_updates_per_ns": 1.0}])
    got, summ = load(path)
    assert len(got) == 20 and len(summ) == 1
    rows = disorder_averages(got)
    assert [(r["bin"], r["k"]) for r in rows] == [(1, 0), (1, 1), (0, 0), (0, 1)]   # earliest bin first
    for r in rows:
        v = np.array(e[(r["bin"], r["k"])])
        assert r["samples"] == 5 and r["e"] == v.mean()
        assert abs(r["e_err"] - v.std(ddof=1) / np.sqrt(5)) < 1e-15
        assert r["q2"] == 0.3 and r["q2_err"] == 0.0
    assert main([str(path)]) == 0
    out = capsys.readouterr().out
    assert "summary: L=4" in out and len(out.splitlines()) == 1 + 4 + 1
    assert main([str(path), "--json"]) == 0
    lines = capsys.readouterr().out.splitlines()
    assert json.loads(lines[0])["bin"] == 1 and json.loads(lines[-1])["summary"]
