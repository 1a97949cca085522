"""Python handle on a batch of PTHR samples living in one device workspace.

PyTorch provides the device memory (one uint8 tensor holding every
sub-buffer) and the CUDA stream; every operation is a call into libpthr.so.
"""
from __future__ import annotations

import ctypes
import weakref
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib
from ._lib import check

RULES = {"metropolis": _lib.METROPOLIS, "heatbath": _lib.HEATBATH, "micsa": _lib.MICSA}
LIVE = weakref.WeakSet()      # open batches (the tests check their guard blocks)
CLUSTERS = {"off": _lib.CLUSTER_OFF, "acu": _lib.CLUSTER_ACU, "single": _lib.CLUSTER_SINGLE}
# spin storage in the workspace: one byte or one bit per site slot
SPIN_LAYOUTS = {"bytes": _lib.SPINS_BYTES, "bits": _lib.SPINS_BITS}


@dataclass
class BatchConfig:
    L: int
    n_samples: int
    n_temps: int
    t_min: float = 0.2
    t_max: float = 1.6
    n_replicas: int = 4
    n_res: int = 4
    sweeps_per_emcs: int = 10
    res_sweeps_per_emcs: int = 240
    acu_interval: int = 1
    rule: str = "metropolis"
    cluster: str = "acu"
    er_on: bool = True
    acu_t_below: float = 1.0
    seed: int = 0
    spin_layout: str = "bytes"

    def to_c(self) -> _lib.Config:
        return _lib.Config(self.L, self.n_samples, self.n_temps, self.n_replicas, self.n_res,
                           self.sweeps_per_emcs, self.res_sweeps_per_emcs, self.acu_interval,
                           RULES[self.rule], CLUSTERS[self.cluster], int(self.er_on),
                           SPIN_LAYOUTS[self.spin_layout],
                           float(self.t_min), float(self.t_max), float(self.acu_t_below),
                           int(self.seed) & 0xFFFFFFFFFFFFFFFF)

    @property
    def V(self):
        return self.L ** 3

    @property
    def n_slot(self):
        return self.n_temps + self.n_res

    @property
    def n_lat(self):
        return self.n_replicas * self.n_slot


def required_bytes(cfg: BatchConfig) -> int:
    lib = _lib.load()
    n = ctypes.c_size_t(0)
    check(lib.pthr_required_bytes(ctypes.byref(cfg.to_c()), ctypes.byref(n)))
    return n.value


def buffer_info(cfg: BatchConfig, buf: int):
    lib = _lib.load()
    off, n = ctypes.c_size_t(0), ctypes.c_size_t(0)
    check(lib.pthr_buffer_info(ctypes.byref(cfg.to_c()), buf, ctypes.byref(off), ctypes.byref(n)))
    return off.value, n.value


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, torch.Tensor):
        assert x.is_contiguous()
        return ctypes.c_void_p(x.data_ptr())
    assert isinstance(x, np.ndarray) and x.flags["C_CONTIGUOUS"]
    return x.ctypes.data_as(ctypes.c_void_p)


class Batch:
    """S independent disorder samples x N_r replica groups x (N_T + N_res) clones."""

    def __init__(self, cfg: BatchConfig, couplings=None, seeds=None, device="cuda", stream=None,
                 tuning=None):
        self.cfg = cfg
        self.lib = _lib.load()
        self.device = torch.device(device)
        self.nbytes = required_bytes(cfg)
        self.ws = torch.empty(self.nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        if couplings is not None:
            if isinstance(couplings, np.ndarray):
                couplings = np.ascontiguousarray(couplings, dtype=np.float32)
                assert couplings.size == cfg.n_samples * 3 * cfg.V
            else:
                couplings = couplings.contiguous()
        if seeds is not None:
            seeds = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64))
            assert seeds.size == cfg.n_samples
        self._cc = cfg.to_c()
        h = ctypes.c_void_p()
        # the workspace and any device couplings come from torch's current
        # stream; the library works on self.stream
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        self.ws.record_stream(self.stream)
        with torch.cuda.device(self.device):
            check(self.lib.pthr_create_batch(ctypes.byref(self._cc), ctypes.c_void_p(self.ws.data_ptr()),
                                             self.nbytes, _ptr(couplings), _ptr(seeds),
                                             ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self.h = h
        self.stream.synchronize()
        self._views = {}
        LIVE.add(self)
        if tuning:
            self.set_tuning(**tuning)

    # ------------------------------------------------------------------ buffers
    def _view(self, buf, dtype, shape):
        key = (buf, dtype, shape)
        if key not in self._views:
            off, n = buffer_info(self.cfg, buf)
            nel = int(np.prod(shape))
            itemsize = torch.empty((), dtype=dtype).element_size()
            assert nel * itemsize <= n, (buf, nel, itemsize, n)
            self._views[key] = self.ws[off:off + nel * itemsize].view(dtype).view(shape)
        return self._views[key]

    @property
    def J(self):
        c = self.cfg
        return self._view(_lib.BUF_J, torch.float32, (c.n_samples, 3, c.V))

    @property
    def energies(self):
        c = self.cfg
        return self._view(_lib.BUF_ENERGY, torch.float64, (c.n_samples, c.n_lat))

    @property
    def perm(self):
        c = self.cfg
        return self._view(_lib.BUF_PERM, torch.int32, (c.n_samples, c.n_replicas, c.n_slot))

    @property
    def age(self):
        c = self.cfg
        return self._view(_lib.BUF_AGE, torch.int32, (c.n_samples, c.n_replicas, max(c.n_res, 1)))

    @property
    def rt_state(self):
        c = self.cfg
        return self._view(_lib.BUF_RT, torch.uint8, (c.n_samples, c.n_lat))

    @property
    def round_trips(self):
        c = self.cfg
        return self._view(_lib.BUF_TRIPS, torch.int64, (c.n_samples, c.n_replicas))

    @property
    def pt_accepted(self):
        c = self.cfg
        return self._view(_lib.BUF_PTACC, torch.int64, (c.n_samples, c.n_replicas, c.n_temps))

    @property
    def flips(self):
        c = self.cfg
        return self._view(_lib.BUF_FLIPS, torch.int64, (c.n_samples, c.n_lat))

    @property
    def obs(self):
        c = self.cfg
        return self._view(_lib.BUF_OBS, torch.float64, (c.n_samples, c.n_temps, _lib.NOBS))

    @property
    def emcs_counter(self):
        return self._view(_lib.BUF_EMCS, torch.int32, (self.cfg.n_samples,))

    @property
    def active(self):
        return self._view(_lib.BUF_ACTIVE, torch.uint8, (self.cfg.n_samples,))

    @property
    def cluster_stats(self):
        c = self.cfg
        return self._view(_lib.BUF_CSTAT, torch.int64, (c.n_samples, max(c.n_replicas // 2, 1), c.n_temps, 4))

    @property
    def chaos(self):
        c = self.cfg
        return self._view(_lib.BUF_CHAOS, torch.float64, (c.n_samples, c.n_temps, 2))

    # ------------------------------------------------------------------ steps
    def sweep(self, n_pt: int, n_res: int = 0):
        check(self.lib.pthr_sweep(self.h, n_pt, n_res), self.h)

    def houdayer(self):
        check(self.lib.pthr_houdayer(self.h), self.h)

    def swap(self, pt: bool = True, er: bool | None = None):
        if er is None:
            er = self.cfg.er_on
        check(self.lib.pthr_swap(self.h, (_lib.SWAP_PT if pt else 0) | (_lib.SWAP_ER if er else 0)), self.h)

    def measure(self, chaos: bool = False):
        flags = _lib.OBS_MEASURE | (_lib.OBS_CHAOS if chaos else 0)
        check(self.lib.pthr_observables(self.h, flags, None, 0), self.h)

    def read_observables(self, out: np.ndarray | None = None) -> np.ndarray:
        """Copy the accumulators to host memory (synchronises the stream)."""
        c = self.cfg
        if out is None:
            out = np.zeros((c.n_samples, c.n_temps, _lib.NOBS), dtype=np.float64)
        assert out.dtype == np.float64 and out.size == c.n_samples * c.n_temps * _lib.NOBS
        check(self.lib.pthr_observables(self.h, _lib.OBS_READ_HOST, _ptr(out), out.nbytes), self.h)
        return out

    def reset_observables(self):
        check(self.lib.pthr_observables(self.h, _lib.OBS_RESET, None, 0), self.h)

    def emcs(self, n: int = 1, graph: bool = False):
        check(self.lib.pthr_emcs(self.h, n, int(graph)), self.h)

    def prethermalize(self, n_sweeps: int, first: int = 0, count: int | None = None):
        count = self.cfg.n_samples - first if count is None else count
        check(self.lib.pthr_prethermalize_reservoir(self.h, first, count, n_sweeps), self.h)

    def poll(self, timeout_ms: int = -1) -> int:
        return self.lib.pthr_poll(self.h, timeout_ms)

    def _enqueue_with(self, out: torch.Tensor, call):
        """Run `call` on the batch's stream after the work queued so far on
        torch's current stream (which made `out`), and order later work on
        the current stream after it."""
        cur = torch.cuda.current_stream(self.device)
        self.stream.wait_stream(cur)
        call()
        out.record_stream(self.stream)
        cur.wait_stream(self.stream)
        return out

    def export_spins(self) -> torch.Tensor:
        c = self.cfg
        out = torch.empty((c.n_samples, c.n_lat, c.V), dtype=torch.int8, device=self.device)
        return self._enqueue_with(out, lambda: check(
            self.lib.pthr_export_spins(self.h, ctypes.c_void_p(out.data_ptr())), self.h))

    def import_spins(self, spins: torch.Tensor):
        c = self.cfg
        spins = spins.to(device=self.device, dtype=torch.int8).contiguous()
        assert spins.numel() == c.n_samples * c.n_lat * c.V
        self._enqueue_with(spins, lambda: check(
            self.lib.pthr_import_spins(self.h, ctypes.c_void_p(spins.data_ptr())), self.h))
        self.stream.synchronize()

    def cluster_labels(self) -> torch.Tensor:
        c = self.cfg
        out = torch.full((c.n_samples, c.n_replicas // 2, c.n_temps, c.V), -1, dtype=torch.int32,
                         device=self.device)
        return self._enqueue_with(out, lambda: check(
            self.lib.pthr_cluster_labels(self.h, ctypes.c_void_p(out.data_ptr())), self.h))

    def reset_samples(self, first: int, count: int, seeds, couplings=None, pretherm_sweeps: int = 0):
        seeds = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64))
        assert seeds.size == count
        if couplings is not None and isinstance(couplings, np.ndarray):
            couplings = np.ascontiguousarray(couplings, dtype=np.float32)
        check(self.lib.pthr_reset_samples(self.h, first, count, _ptr(couplings), _ptr(seeds),
                                          pretherm_sweeps), self.h)

    def set_active(self, first: int, count: int, active: bool):
        check(self.lib.pthr_set_active(self.h, first, count, int(active)), self.h)

    def set_tuning(self, pt_lattices_per_block=0, res_lattices_per_block=0, sweep_threads=0,
                   cluster_threads=0, cluster_iter_cap=0):
        t = _lib.Tuning(pt_lattices_per_block, res_lattices_per_block, sweep_threads, cluster_threads,
                        cluster_iter_cap)
        check(self.lib.pthr_set_tuning(self.h, ctypes.byref(t)), self.h)

    def set_rule(self, rule: str):
        """Switch the local update rule at an EMCS boundary (the paper's PTHR*:
        Metropolis early, MicSA for the late bins)."""
        import dataclasses
        check(self.lib.pthr_set_update_rule(self.h, RULES[rule]), self.h)
        self.cfg = dataclasses.replace(self.cfg, rule=rule)

    def get_tuning(self) -> dict:
        t = _lib.Tuning()
        check(self.lib.pthr_get_tuning(self.h, ctypes.byref(t)), self.h)
        return {f: getattr(t, f) for f, _ in t._fields_}

    def save(self) -> bytes:
        n = ctypes.c_size_t(0)
        check(self.lib.pthr_save(self.h, None, ctypes.byref(n)), self.h)
        buf = ctypes.create_string_buffer(n.value)
        check(self.lib.pthr_save(self.h, buf, ctypes.byref(n)), self.h)
        return buf.raw

    def load(self, blob: bytes):
        check(self.lib.pthr_load(self.h, ctypes.c_char_p(blob), len(blob)), self.h)

    def reservoir_autocorrelation(self, n_points: int, sweeps_per_point: int, first: int = 0,
                                  count: int | None = None) -> torch.Tensor:
        """Integer sums of s_i(t) s_i(t + tau) over every reservoir clone and
        site of each sample, tau = sweeps_per_point, 2 sweeps_per_point, ...
        (pthr_reservoir_autocorrelation); device int64 [count, n_points]."""
        c = self.cfg
        count = c.n_samples - first if count is None else count
        nbytes = count * c.n_replicas * c.n_res * self.lattice_bytes()
        snap = torch.empty(max(nbytes, 16), dtype=torch.uint8, device=self.device)
        out = torch.zeros((count, n_points), dtype=torch.int64, device=self.device)
        check(self.lib.pthr_reservoir_autocorrelation(self.h, first, count, n_points, sweeps_per_point,
                                                      ctypes.c_void_p(snap.data_ptr()), snap.numel(),
                                                      ctypes.c_void_p(out.data_ptr())), self.h)
        self.stream.synchronize()
        return out

    def lattice_bytes(self) -> int:
        """Workspace bytes of one lattice in this batch's spin layout."""
        n = ctypes.c_size_t(0)
        check(self.lib.pthr_lattice_storage_bytes(self.cfg.L, SPIN_LAYOUTS[self.cfg.spin_layout],
                                                  ctypes.byref(n)))
        return n.value

    def check_canaries(self) -> int:
        """-1 if every guard block after a workspace sub-buffer is intact,
        else the PTHR_BUF_* index of the first overwritten one."""
        bad = ctypes.c_int(-1)
        st = self.lib.pthr_check_canaries(self.h, ctypes.byref(bad))
        if st not in (_lib.PTHR_OK, _lib.PTHR_E_BOUNDS):
            check(st, self.h)
        return bad.value

    def synchronize(self):
        self.stream.synchronize()

    def close(self):
        if getattr(self, "h", None):
            self.lib.pthr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Group:
    """Several batches (e.g. one per lattice size) advanced by one CUDA-graph
    launch per EMCS; each batch runs on its own stream inside the graph."""

    def __init__(self, batches, stream=None):
        import torch
        self.lib = _lib.load()
        self.batches = list(batches)
        self.stream = stream if stream is not None else torch.cuda.Stream(self.batches[0].device)
        arr = (ctypes.c_void_p * len(self.batches))(*[b.h.value for b in self.batches])
        h = ctypes.c_void_p()
        check(self.lib.pthr_group_create(arr, len(self.batches), ctypes.c_void_p(self.stream.cuda_stream),
                                         ctypes.byref(h)))
        self.h = h

    def emcs(self, n: int = 1):
        check(self.lib.pthr_group_emcs(self.h, n))

    @property
    def launches_per_emcs(self) -> int:
        n = ctypes.c_int(0)
        check(self.lib.pthr_group_info(self.h, ctypes.byref(n)))
        return n.value

    def synchronize(self):
        self.stream.synchronize()

    def close(self):
        if getattr(self, "h", None):
            self.lib.pthr_group_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
