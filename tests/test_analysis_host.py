"""Analysis helpers against the definitions of Secs. 2, 4 and 5."""
import numpy as np
import pytest

from paper_2605_25872_gb300 import analysis as A


def test_log2_bins_match_the_paper_statement():
    """Sec. 4: bin 0 is the second half of the simulation, bin 1 the second
    quarter, bin 2 the second eighth; bins tile (t_max/2^B, t_max]."""
    t_max = 2 ** 10
    bins = A.log2_bins(t_max, 4)
    assert bins[0] == (513, 1024)
    assert bins[1] == (257, 512)
    assert bins[2] == (129, 256)
    assert bins[3] == (65, 128)
    covered = sorted(t for lo, hi in bins for t in range(lo, hi + 1))
    assert covered == list(range(65, 1025))


def test_tau_trw_and_zeff():
    # every clone of 2 groups x 10 temperatures made 5 round trips in 1000 EMCS
    tau = A.tau_trw(2, 10, 1000, 2 * 10 * 5)
    assert tau == pytest.approx(1000 / 5)
    assert A.z_eff(6105.0, 3871.0, 16, 14) == pytest.approx(np.log(6105 / 3871) / np.log(16 / 14))


def test_chaos_parameter_limits():
    assert A.chaos_parameter(0.5, 0.5, 0.5) == pytest.approx(1.0)
    assert A.chaos_parameter(0.0, 0.5, 0.3) == 0.0


def test_thermal_averages_and_sdy():
    obs = np.zeros((1, 2, 8))
    obs[0, :, 0] = 10            # measurements
    obs[0, :, 1] = [-40.0, -20.0]  # sum e over 10 x 4 groups -> -1, -0.5
    obs[0, :, 5] = [18.0, 10.0]    # sum q_l over 10 x 2 pairs -> 0.9, 0.5
    avg = A.thermal_averages(obs, 4)
    np.testing.assert_allclose(avg["e"][0], [-1.0, -0.5])
    np.testing.assert_allclose(avg["ql"][0], [0.9, 0.5])
    S = A.sdy(avg["e"][0], avg["ql"][0], np.array([0.5, 1.0]))
    np.testing.assert_allclose(S, [-1 / 3 + 0.2, -0.5 / 3 + 0.5])


def test_observable_records_and_jsonl(tmp_path):
    import json
    from paper_2605_25872_gb300.analysis import append_jsonl, observable_records
    S, NT, NR = 2, 3, 4
    obs = np.zeros((S, NT, 8))
    obs[..., 0] = 5                               # five measurements
    obs[..., 1] = -1.5 * 5 * NR                   # <e> = -1.5 over 5 x 4 groups
    obs[..., 4] = 0.25 * 5 * (NR // 2)            # <q^2> = 0.25 over 5 x 2 pairs
    pt = np.ones((S, NR, NT), dtype=np.int64)
    cs = np.tile(np.array([3, 40, 10, 20]), (S, NR // 2, NT, 1))
    recs = observable_records(obs, [0.2, 0.9, 1.6], NR, emcs=7, sample_ids=[10, 11], pt_accepted=pt,
                              cluster_stats=cs)
    assert len(recs) == S * NT
    r = recs[4]                                   # sample index 1, k = 1
    assert r["sample"] == 11 and r["k"] == 1 and r["T"] == 0.9 and r["emcs"] == 7 and r["n"] == 5
    assert r["e"] == -1.5 and r["q2"] == 0.25
    assert r["pt_accepted"] == NR and r["clusters"] == 6 and r["largest"] == 80
    path = tmp_path / "obs.jsonl"
    assert append_jsonl(path, recs) == 6 and append_jsonl(path, recs[:1]) == 1
    lines = path.read_text().splitlines()
    assert len(lines) == 7 and json.loads(lines[4]) == r
