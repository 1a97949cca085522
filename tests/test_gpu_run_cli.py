"""The command-line run (python -m paper_2605_25872_gb300.run): its JSON-lines
records per (bin, sample, temperature) equal the thermal averages of the same
run stepped call by call through analysis.run_binned, and the summary record
closes the file."""
import json

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2605_25872_gb300")
from paper_2605_25872_gb300 import Batch, BatchConfig  # noqa: E402
from paper_2605_25872_gb300.analysis import run_binned, thermal_averages  # noqa: E402
from paper_2605_25872_gb300.build import build  # noqa: E402
from paper_2605_25872_gb300.run import main  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build()


@pytest.mark.parametrize("layout", ["bytes", "bits"])
def test_cli_records_equal_the_binned_run(tmp_path, layout):
    out = tmp_path / "run.jsonl"
    args = ["--L", "6", "--samples", "3", "--temps", "6", "--res", "2", "--sweeps", "2",
            "--res-sweeps", "8", "--pretherm", "16", "--emcs", "40", "--bins", "3", "--seed", "11",
            "--spin-layout", layout, "--out", str(out)]
    assert main(args) == 0
    lines = [json.loads(x) for x in out.read_text().splitlines()]
    summary = lines[-1]
    recs = lines[:-1]
    assert summary["summary"] and summary["records"] == len(recs) == 3 * 3 * 6
    assert summary["status"] == 0 and summary["emcs"] == 40
    # the same run through the analysis helper, one call per step
    cfg = BatchConfig(L=6, n_samples=3, n_temps=6, n_replicas=4, n_res=2, sweeps_per_emcs=2,
                      res_sweeps_per_emcs=8, seed=11, spin_layout=layout)
    b = Batch(cfg)
    b.prethermalize(16)
    ref = run_binned(b, 40, 3)
    for r in recs:
        avg = thermal_averages(ref[r["bin"]][0], cfg.n_replicas)
        for name in ("e", "e2", "q", "q2", "q4", "ql", "S"):
            assert r[name] == pytest.approx(float(avg[name][r["sample"], r["k"]]), rel=0, abs=0), name
        assert r["n"] == int(ref[r["bin"]][0][r["sample"], r["k"], 0])
    bins = {tuple(x) for x in summary["bins"]}
    assert bins == {(21, 40), (11, 20), (6, 10)}
    assert np.isfinite(summary["spin_updates_per_ns"])


def test_cli_pthr_star_switches_to_micsa_for_the_late_bins(tmp_path):
    out = tmp_path / "star.jsonl"
    args = ["--L", "8", "--samples", "2", "--temps", "8", "--res", "2", "--sweeps", "2",
            "--res-sweeps", "8", "--pretherm", "16", "--emcs", "64", "--bins", "3", "--micsa-bins", "2",
            "--out", str(out)]
    assert main(args) == 0
    recs = [json.loads(x) for x in out.read_text().splitlines()][:-1]
    rules = {r["bin"]: r["rule"] for r in recs}
    assert rules == {2: "metropolis", 1: "micsa", 0: "micsa"}
    # the same schedule through the library calls, one call per step: log2 bins
    # of 64 EMCS are 33..64 (bin 0), 17..32 (bin 1), 9..16 (bin 2); MicSA from 17
    cfg = BatchConfig(L=8, n_samples=2, n_temps=8, n_replicas=4, n_res=2, sweeps_per_emcs=2,
                      res_sweeps_per_emcs=8, seed=1)
    b = Batch(cfg)
    b.prethermalize(16)
    ref = {}
    for t in range(1, 65):
        if t == 17:
            b.set_rule("micsa")
        if t in (9, 17, 33):
            b.reset_observables()
        b.sweep(2, 8)
        b.houdayer()
        b.swap(True, True)
        b.measure()
        if t in (16, 32, 64):
            b.synchronize()
            ref[{16: 2, 32: 1, 64: 0}[t]] = thermal_averages(b.obs.cpu().numpy().copy(), cfg.n_replicas)
    for r in recs:
        for name in ("e", "q2", "ql", "S"):
            assert r[name] == float(ref[r["bin"]][name][r["sample"], r["k"]]), (r["bin"], name)
