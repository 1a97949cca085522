"""bench.py's workload descriptions follow the selected workload and spin
layout (no GPU needed): no reservoir or resident-state claims that belong to
another workload."""
import importlib
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture()
def bench():
    sys.path.insert(0, ROOT)
    import bench as B
    B = importlib.reload(B)
    yield B
    importlib.reload(B)


@pytest.mark.parametrize("name", ["c2", "c3", "c4"])
def test_config_follows_the_workload(bench, name):
    import workloads as W
    bench.WL = W.WORKLOADS[name]
    c = bench.config_dict()
    wl = W.WORKLOADS[name]
    assert c["L"] == wl.L and c["n_samples"] == wl.n_samples and c["n_temps"] == wl.n_temps
    assert ("reservoir" in c["workload"]) == bool(wl.er_on)
    assert c["n_res"] == (wl.n_res if wl.er_on else 0)
    assert c["spin_layout"] == "bytes" and c["update_rule"] == "metropolis"
    # resident state from the workload's own sizes
    lat_bytes = 2 * wl.L * wl.L * ((wl.L // 2 + 3) // 4) * 4
    mb = (wl.n_samples * wl.lattices_per_sample * lat_bytes + wl.n_samples * 3 * wl.V * 4) / 1e6
    assert f"{mb:.0f} MB" in c["l2"]


def test_bit_layout_shrinks_the_stated_state(bench):
    import workloads as W
    bench.WL = W.WORKLOADS["c4"]
    full = bench.config_dict()["l2"]
    bench.SPINS = "bits"
    c = bench.config_dict()
    assert c["spin_layout"] == "bits"
    assert c["l2"] != full and "fits in the 129 MB L2" in c["l2"]


def test_batch_config_carries_rule_and_layout(bench):
    import workloads as W
    bench.WL = W.WORKLOADS["c3"]
    bench.RULE, bench.SPINS = "micsa", "bits"
    cfg = bench.batch_config(8)
    assert cfg.L == 12 and cfg.n_samples == 8 and cfg.rule == "micsa" and cfg.spin_layout == "bits"
    assert not cfg.er_on and cfg.n_res == 0
