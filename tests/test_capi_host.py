"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, exports every entry point that include/pthr.h declares, and
rejects bad arguments before touching CUDA."""
import ctypes
import os
import re

import pytest

from paper_2605_25872_gb300 import BatchConfig, buffer_info, required_bytes
from paper_2605_25872_gb300 import _lib
from paper_2605_25872_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build()
    return _lib.load()


def declared_entry_points():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"PTHR_API\s+[\w\s\*]+?\b(pthr_\w+)\s*\(", txt)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_entry_points()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_lib.EXPORTS)
    assert lib.pthr_version().startswith(b"pthr-gb300")


def test_required_bytes_and_layout(lib):
    c = BatchConfig(L=16, n_samples=512, n_temps=32)
    total = required_bytes(c)
    prev_end = 0
    for b in range(_lib.NBUF):
        off, n = buffer_info(c, b)
        assert off % 256 == 0 and off >= prev_end
        prev_end = off + n
    assert prev_end <= total
    assert buffer_info(c, _lib.BUF_J)[1] == 512 * 3 * 4096 * 4
    assert buffer_info(c, _lib.BUF_SPINS)[1] == 512 * 144 * 4096
    n = ctypes.c_size_t()
    assert lib.pthr_lattice_bytes(12, ctypes.byref(n)) == 0 and n.value == 2 * 144 * 8


def test_bit_spin_storage_sizes(lib):
    n = ctypes.c_size_t()
    for L in (2, 4, 6, 12, 16, 24):
        lib.pthr_lattice_bytes(L, ctypes.byref(n))
        byte_bytes = n.value
        assert lib.pthr_lattice_storage_bytes(L, _lib.SPINS_BYTES, ctypes.byref(n)) == 0
        assert n.value == byte_bytes
        assert lib.pthr_lattice_storage_bytes(L, _lib.SPINS_BITS, ctypes.byref(n)) == 0
        assert n.value * 8 == byte_bytes and n.value % 4 == 0
    assert lib.pthr_lattice_storage_bytes(12, 2, ctypes.byref(n)) == _lib.PTHR_E_INVAL
    assert lib.pthr_lattice_storage_bytes(13, _lib.SPINS_BITS, ctypes.byref(n)) == _lib.PTHR_E_INVAL
    c = BatchConfig(L=16, n_samples=512, n_temps=32, spin_layout="bits")
    assert buffer_info(c, _lib.BUF_SPINS)[1] == 512 * 144 * 512
    assert required_bytes(c) < required_bytes(BatchConfig(L=16, n_samples=512, n_temps=32)) - 250e6


@pytest.mark.parametrize("field,value", [("L", 3), ("L", 26), ("L", 0), ("n_samples", 0),
                                         ("n_temps", 1), ("n_replicas", 0), ("n_replicas", 3),
                                         ("t_min", 0.0), ("t_max", 0.1), ("acu_interval", 0),
                                         ("n_res", 0), ("rule", "bogus"), ("spin_layout", 2)])
def test_invalid_configs_are_rejected(lib, field, value):
    c = BatchConfig(L=8, n_samples=4, n_temps=8)
    if field == "rule":
        cc = c.to_c()
        cc.update_rule = 7
    elif field == "spin_layout":
        cc = c.to_c()
        cc.spin_layout = 2
    else:
        setattr(c, field, value)
        cc = c.to_c()
    n = ctypes.c_size_t()
    st = lib.pthr_required_bytes(ctypes.byref(cc), ctypes.byref(n))
    assert st == _lib.PTHR_E_INVAL
    assert len(lib.pthr_last_error(None)) > 0


def test_create_rejects_bad_workspace_without_cuda(lib):
    c = BatchConfig(L=8, n_samples=2, n_temps=4).to_c()
    h = ctypes.c_void_p()
    assert lib.pthr_create_batch(ctypes.byref(c), None, 0, None, None, None, ctypes.byref(h)) == _lib.PTHR_E_INVAL
    assert lib.pthr_create_batch(ctypes.byref(c), ctypes.c_void_p(256), 16, None, None, None,
                                 ctypes.byref(h)) == _lib.PTHR_E_NOMEM
    assert lib.pthr_create_batch(ctypes.byref(c), ctypes.c_void_p(100), 1 << 40, None, None, None,
                                 ctypes.byref(h)) == _lib.PTHR_E_INVAL   # misaligned
    assert h.value is None


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.pthr_sweep(None, 1, 1) == _lib.PTHR_E_INVAL
    assert lib.pthr_swap(None, 1) == _lib.PTHR_E_INVAL
    assert lib.pthr_houdayer(None) == _lib.PTHR_E_INVAL
    assert lib.pthr_emcs(None, 1, 0) == _lib.PTHR_E_INVAL
    assert lib.pthr_poll(None, 0) == _lib.PTHR_E_INVAL
    assert lib.pthr_set_update_rule(None, 0) == _lib.PTHR_E_INVAL
    lib.pthr_destroy(None)


def test_measure_peak_rejects_bad_arguments_without_cuda(lib):
    r, t = ctypes.c_double(), ctypes.c_double()
    assert lib.pthr_measure_peak(99, ctypes.c_void_p(256), 1 << 20, None, ctypes.byref(r),
                                 ctypes.byref(t)) == _lib.PTHR_E_INVAL
    assert lib.pthr_measure_peak(_lib.PEAK_SMEM_READ, None, 1 << 20, None, ctypes.byref(r),
                                 ctypes.byref(t)) == _lib.PTHR_E_INVAL
    # the L2 benchmark needs at least 1 MB past the 4 KB of sink words
    assert lib.pthr_measure_peak(_lib.PEAK_L2_READ, ctypes.c_void_p(256), 8192, None, ctypes.byref(r),
                                 ctypes.byref(t)) == _lib.PTHR_E_INVAL


def test_random_configs_are_either_valid_with_a_consistent_layout_or_refused(lib):
    """Random configurations (host-only, no CUDA): every one is either
    accepted, with sub-buffers that are 256-byte aligned, in order, sized by
    the configuration and inside the total, or refused with PTHR_E_INVAL and
    a message, as the documented rules say."""
    import numpy as np
    rng = np.random.default_rng(7)
    accepted = refused = 0
    def pick(good, bad):
        """a valid value mostly, an edge or invalid one 10% of the time"""
        return int(rng.choice(bad)) if rng.random() < 0.1 else int(rng.choice(good))

    for _ in range(600):
        c = _lib.Config(pick([2, 4, 6, 8, 12, 16, 24], [0, 3, 13, 26, -2]), pick([1, 3, 64], [0, -1]),
                        pick([2, 5, 32], [0, 1, 300]), pick([1, 2, 4, 32], [0, 3, 33]), pick([0, 1, 4], [-1, 255]),
                        pick([0, 1, 10], [-1, 1 << 22]), pick([0, 240], [-1, 1 << 22]), pick([1, 8], [0, -3]),
                        pick([0, 1, 2], [3, -1]), pick([0, 1, 2], [3, -1]), pick([0, 1], [0, 1]),
                        pick([0, 1], [2, -1]), float(rng.choice([0.2, 0.5, -0.1, 0.0])),
                        float(rng.choice([1.6, 2.0, 0.1])), 1.0, 5)
        valid = (2 <= c.L <= 24 and c.L % 2 == 0 and c.n_samples >= 1 and c.n_temps >= 2
                 and 1 <= c.n_replicas <= 32 and c.n_res >= 0 and c.n_temps + c.n_res <= 256
                 and not (c.er_on and c.n_res < 1) and 0 <= c.sweeps_per_emcs < (1 << 22)
                 and 0 <= c.res_sweeps_per_emcs < (1 << 22) and c.acu_interval >= 1
                 and c.update_rule in (0, 1, 2)
                 and c.cluster_mode in (0, 1, 2)
                 and not (c.cluster_mode != 0 and (c.n_replicas < 2 or c.n_replicas % 2))
                 and c.t_min > 0 and c.t_max > c.t_min and c.spin_layout in (0, 1))
        n = ctypes.c_size_t()
        st = lib.pthr_required_bytes(ctypes.byref(c), ctypes.byref(n))
        if not valid:
            assert st == _lib.PTHR_E_INVAL and len(lib.pthr_last_error(None)) > 0
            refused += 1
            continue
        assert st == _lib.PTHR_OK
        accepted += 1
        end = 0
        for buf in range(_lib.NBUF):
            off, size = ctypes.c_size_t(), ctypes.c_size_t()
            assert lib.pthr_buffer_info(ctypes.byref(c), buf, ctypes.byref(off), ctypes.byref(size)) == 0
            assert off.value % 256 == 0 and off.value >= end
            end = off.value + size.value
        assert end <= n.value
        off, size = ctypes.c_size_t(), ctypes.c_size_t()
        lib.pthr_buffer_info(ctypes.byref(c), _lib.BUF_SPINS, ctypes.byref(off), ctypes.byref(size))
        lb = ctypes.c_size_t()
        assert lib.pthr_lattice_storage_bytes(c.L, c.spin_layout, ctypes.byref(lb)) == 0
        assert size.value == c.n_samples * c.n_replicas * (c.n_temps + c.n_res) * lb.value
    assert accepted > 20 and refused > 20
