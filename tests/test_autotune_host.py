"""Host-side checks of the autotuner's candidate shapes (no GPU needed)."""
from paper_2605_25872_gb300 import BatchConfig
from paper_2605_25872_gb300.autotune import candidates, sweep_lane_threads


def test_sweep_threads_are_whole_lattice_lanes_below_the_default():
    # L = 8: 64 groups per colour -> lanes of 64 threads
    assert sweep_lane_threads(8) == [64, 128, 256]
    # L = 12: 288 groups per colour, one lane is the default block
    assert sweep_lane_threads(12) == []
    # L = 16: 512 groups, no smaller block exists
    assert sweep_lane_threads(16) == []
    # L = 6: 36 groups per colour, the default holds 14 lanes
    assert sweep_lane_threads(6) == [36, 72, 144]
    assert sweep_lane_threads(24) == []


def test_candidates_cover_every_shape_once():
    cfg = BatchConfig(L=8, n_samples=4, n_temps=16, n_res=0, er_on=False)
    shapes = list(candidates(cfg))
    keys = [tuple(sorted(s.items())) for s in shapes]
    assert len(keys) == len(set(keys))
    sweep = [s for s in shapes if "cluster_threads" not in s]
    assert {s.get("sweep_threads", 0) for s in sweep} == {0, 64, 128, 256}
    assert all(s["pt_lattices_per_block"] <= 64 for s in sweep)
    assert any("cluster_threads" in s for s in shapes)
