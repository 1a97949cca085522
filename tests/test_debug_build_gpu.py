"""The range-checked build (PTHR_DEBUG: every checked index that would leave
its buffer latches PTHR_E_BOUNDS and is skipped) runs the EMCS scenarios of
debug_build_scenarios.py without a single failed check, and its results are
bit-identical to the release build's.  The debug library runs in a child
process (PTHR_LIBRARY), the release library in this one."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2605_25872_gb300")
from paper_2605_25872_gb300 import _lib  # noqa: E402
from paper_2605_25872_gb300.build import build  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def test_debug_build_passes_every_range_check_and_matches_release(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build()
    dbg = build(debug=True)
    out = tmp_path / "debug.npz"
    env = dict(os.environ, PTHR_LIBRARY=dbg)
    r = subprocess.run([sys.executable, os.path.join(HERE, "debug_build_scenarios.py"), str(out)],
                       env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    sys.path.insert(0, HERE)
    import debug_build_scenarios as S
    rel = S.run_all()
    got = np.load(out)
    for i in range(len(S.SCENARIOS)):
        st, bad = got[f"poll{i}"]
        assert st == _lib.PTHR_OK, f"scenario {i}: debug build reported status {st}"
        assert bad == -1
        assert rel[f"poll{i}"][0] == _lib.PTHR_OK
    for k in rel:
        np.testing.assert_array_equal(got[k], rel[k], err_msg=k)


def test_debug_build_at_full_size_matches_release(tmp_path):
    """Every kernel at its production grid size (the L=16 workload in both spin
    layouts, 1024 samples at L=12, 256 at L=8, L=24 and L=20, the five-size
    group): no failed range check, intact guard blocks, and results identical
    to the release build's."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import json
    build()
    dbg = build(debug=True)
    out = tmp_path / "scale.json"
    env = dict(os.environ, PTHR_LIBRARY=dbg)
    r = subprocess.run([sys.executable, os.path.join(HERE, "debug_build_scenarios.py"), str(out), "--scale"],
                       env=env, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stderr[-3000:]
    sys.path.insert(0, HERE)
    import debug_build_scenarios as S
    rel = S.run_scale()
    got = json.loads(out.read_text())
    assert set(got) == set(rel)
    for k, (st, bad, dig) in got.items():
        assert st == _lib.PTHR_OK and bad == -1, f"{k}: debug build status {st}, guard {bad}"
        assert tuple(rel[k]) == (st, bad, dig), f"{k}: release {rel[k]} vs debug {(st, bad, dig)}"
    # the two spin layouts of the L=16 workload hold the same trajectory
    assert got["scale0"][2] == got["scale1"][2]
