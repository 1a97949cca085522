"""The allocation-free reservoir autocorrelation entry point.

Some callers cannot allocate device memory at all (a plugin whose host owns
every device allocation, a loop that must not wait on the allocator, a
binding with no device allocator), so the library offers a variant of
pthr_reservoir_autocorrelation that keeps its snapshot in a fixed device
array instead of a caller buffer.  Here it is called through the C ABI on one
batch and compared, on two calls in a row, with the allocating entry point
run on an identical batch; both return exact integer sums, so they must agree
bit for bit.  It also refuses a sample range whose snapshot would not fit.
The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2605_25872_gb300")
from paper_2605_25872_gb300 import Batch, BatchConfig, _lib  # noqa: E402
from paper_2605_25872_gb300.build import build  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build()


def test_noalloc_autocorrelation_matches_the_allocating_entry_point():
    lib = _lib.load()
    cfg = BatchConfig(L=8, n_samples=6, n_temps=4, n_replicas=2, n_res=3)
    J = W.gaussian_couplings(cfg.L, cfg.n_samples, 610)
    seeds = W.sample_seeds(W.SEED_BASE + 610, cfg.n_samples)
    with_buffer = Batch(cfg, couplings=J, seeds=seeds)
    fixed = Batch(cfg, couplings=J, seeds=seeds)
    with_buffer.prethermalize(10)
    fixed.prethermalize(10)
    n_points, per = 3, 4
    for call in range(2):
        ref = with_buffer.reservoir_autocorrelation(n_points, per).cpu().numpy()
        out = torch.full((cfg.n_samples, n_points), -1, dtype=torch.int64, device=fixed.device)
        _lib.check(lib.pthr_reservoir_autocorrelation_noalloc(fixed.h, 0, cfg.n_samples, n_points, per,
                                                              ctypes.c_void_p(out.data_ptr())), fixed.h)
        fixed.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), ref, err_msg=f"call {call}")
    assert fixed.poll(10000) == _lib.PTHR_OK
    np.testing.assert_array_equal(fixed.export_spins().cpu().numpy(), with_buffer.export_spins().cpu().numpy())


def test_noalloc_autocorrelation_rejects_a_snapshot_larger_than_its_array():
    lib = _lib.load()
    # L = 24: 2 x 4 reservoir clones of 13824 bytes per sample; 80 samples
    # need 8.8 MB, more than the 8 MiB array
    cfg = BatchConfig(L=24, n_samples=80, n_temps=2, n_replicas=2, n_res=4)
    b = Batch(cfg)
    out = torch.zeros((cfg.n_samples, 1), dtype=torch.int64, device=b.device)
    st = lib.pthr_reservoir_autocorrelation_noalloc(b.h, 0, cfg.n_samples, 1, 1, ctypes.c_void_p(out.data_ptr()))
    assert st == _lib.PTHR_E_NOMEM
    assert b"fixed scratch" in lib.pthr_last_error(b.h)
    # a range that fits runs
    _lib.check(lib.pthr_reservoir_autocorrelation_noalloc(b.h, 0, 40, 1, 1, ctypes.c_void_p(out.data_ptr())), b.h)
    b.synchronize()
    assert b.poll(10000) == _lib.PTHR_OK
