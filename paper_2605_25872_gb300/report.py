"""Disorder averages of a command-line run's JSON lines (run.py): for every
log2 bin and temperature, the mean over samples of the thermal averages with
its standard error (samples are independent disorder realisations, Sec. 2),
plus the run's summary.

    python -m paper_2605_25872_gb300.report run.jsonl [--json]
"""
from __future__ import annotations

import argparse
import json
import sys

import numpy as np

FIELDS = ("e", "e2", "q", "q2", "q4", "ql", "S")


def load(path):
    """(per-(bin, sample, T) records, summary records) of a run file."""
    recs, summaries = [], []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line:
                continue
            r = json.loads(line)
            (summaries if r.get("summary") else recs).append(r)
    return recs, summaries


def disorder_averages(recs, fields=FIELDS) -> list:
    """One row per (bin, k): T, number of samples, and for each field the
    mean over samples and its standard error (sample std / sqrt(n))."""
    groups = {}
    for r in recs:
        groups.setdefault((r["bin"], r["k"]), []).append(r)
    out = []
    for (b, k) in sorted(groups, key=lambda x: (-x[0], x[1])):
        rs = groups[(b, k)]
        row = {"bin": b, "k": k, "T": rs[0]["T"], "samples": len(rs), "rule": rs[0].get("rule")}
        for name in fields:
            v = np.array([r[name] for r in rs if r.get(name) is not None], dtype=np.float64)
            if v.size == 0:
                continue
            row[name] = float(v.mean())
            row[name + "_err"] = float(v.std(ddof=1) / np.sqrt(v.size)) if v.size > 1 else None
        out.append(row)
    return out


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("path")
    ap.add_argument("--json", action="store_true", help="print JSON lines instead of a table")
    args = ap.parse_args(argv)
    recs, summaries = load(args.path)
    rows = disorder_averages(recs)
    if args.json:
        for r in rows:
            print(json.dumps(r))
        for s in summaries:
            print(json.dumps(s))
        return 0
    print(f"{'bin':>3} {'T':>6} {'n':>5}  {'<e>':>18}  {'<q2>':>16}  {'<ql>':>16}  {'<S>':>16}")
    for r in rows:
        def f(name):
            err = r.get(name + "_err")
            return f"{r[name]:.5f}({err:.5f})" if err is not None else f"{r[name]:.5f}"
        print(f"{r['bin']:>3} {r['T']:6.3f} {r['samples']:>5}  {f('e'):>18}  {f('q2'):>16}  "
              f"{f('ql'):>16}  {f('S'):>16}")
    for s in summaries:
        print(f"summary: L={s['L']} samples={s['samples']} emcs={s['emcs']} "
              f"tau_TRW median={s.get('tau_trw_median')} updates/ns={s.get('spin_updates_per_ns'):.1f}")
    return 0


if __name__ == "__main__":
    sys.exit(main())
