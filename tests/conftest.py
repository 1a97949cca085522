import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running statistical check")


def pytest_collection_modifyitems(config, items):
    # test files named test_zz_* run last (pytest sorts by file name already;
    # this keeps it explicit when files are passed in another order)
    items.sort(key=lambda it: (os.path.basename(str(it.fspath)).startswith("test_zz_"),))


@pytest.fixture(autouse=True)
def _guard_blocks_intact(request):
    """After every GPU test: no kernel wrote past the end of a workspace
    sub-buffer of any batch still open (guard blocks, pthr_check_canaries)."""
    yield
    if request.node.get_closest_marker("gpu") is None:
        return
    mod = sys.modules.get("paper_2605_25872_gb300.batch")
    if mod is None:
        return
    for b in list(mod.LIVE):
        if getattr(b, "h", None):
            assert b.check_canaries() == -1, "a guard block after a workspace buffer was overwritten"
