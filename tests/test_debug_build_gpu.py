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
