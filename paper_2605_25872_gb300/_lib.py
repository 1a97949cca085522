"""ctypes binding of libpthr.so (the C ABI declared in include/pthr.h).

Argument marshalling only: every step of the method runs in the CUDA
kernels of the library.  Importing this module never falls back to another
implementation; if the library is missing it raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libpthr.so")

(PTHR_OK, PTHR_E_INVAL, PTHR_E_NOMEM, PTHR_E_CUDA, PTHR_E_NOCONVERGE, PTHR_E_TIMEOUT, PTHR_E_STATE,
 PTHR_E_BOUNDS) = range(8)
STATUS_NAMES = {0: "PTHR_OK", 1: "PTHR_E_INVAL", 2: "PTHR_E_NOMEM", 3: "PTHR_E_CUDA",
                4: "PTHR_E_NOCONVERGE", 5: "PTHR_E_TIMEOUT", 6: "PTHR_E_STATE", 7: "PTHR_E_BOUNDS"}
METROPOLIS, HEATBATH, MICSA = 0, 1, 2
CLUSTER_OFF, CLUSTER_ACU, CLUSTER_SINGLE = 0, 1, 2
SPINS_BYTES, SPINS_BITS = 0, 1
SWAP_PT, SWAP_ER = 1, 2
OBS_MEASURE, OBS_READ_HOST, OBS_READ_DEVICE, OBS_RESET, OBS_CHAOS = 1, 2, 4, 8, 16
NOBS = 8
MAX_L = 24
(BUF_J, BUF_SPINS, BUF_ENERGY, BUF_PERM, BUF_AGE, BUF_RT, BUF_TRIPS, BUF_PTACC, BUF_FLIPS,
 BUF_OBS, BUF_EMCS, BUF_SEEDS, BUF_ACTIVE, BUF_STATUS, BUF_CSTAT, BUF_CHAOS, BUF_PRETH, BUF_TABLES,
 NBUF) = range(19)

# every exported entry point of include/pthr.h
EXPORTS = ("pthr_required_bytes", "pthr_buffer_info", "pthr_lattice_bytes", "pthr_lattice_storage_bytes",
           "pthr_create_batch", "pthr_set_update_rule",
           "pthr_destroy", "pthr_set_stream", "pthr_set_tuning", "pthr_get_tuning", "pthr_sweep",
           "pthr_houdayer", "pthr_cluster_labels", "pthr_swap", "pthr_observables", "pthr_emcs",
           "pthr_prethermalize_reservoir", "pthr_poll", "pthr_export_spins", "pthr_import_spins",
           "pthr_reset_samples", "pthr_set_active", "pthr_save", "pthr_load", "pthr_last_error",
           "pthr_version", "pthr_group_create", "pthr_group_emcs", "pthr_group_destroy",
           "pthr_measure_peak", "pthr_check_canaries", "pthr_reservoir_autocorrelation",
           "pthr_reservoir_autocorrelation_noalloc", "pthr_group_info")
PEAK_SMEM_READ, PEAK_L2_READ, PEAK_ALU, PEAK_FMA, PEAK_FMA2, PEAK_FP64 = range(6)


class Config(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("n_samples", ctypes.c_int), ("n_temps", ctypes.c_int),
                ("n_replicas", ctypes.c_int), ("n_res", ctypes.c_int),
                ("sweeps_per_emcs", ctypes.c_int), ("res_sweeps_per_emcs", ctypes.c_int),
                ("acu_interval", ctypes.c_int), ("update_rule", ctypes.c_int),
                ("cluster_mode", ctypes.c_int), ("er_on", ctypes.c_int), ("spin_layout", ctypes.c_int),
                ("t_min", ctypes.c_double), ("t_max", ctypes.c_double),
                ("acu_t_below", ctypes.c_double), ("seed", ctypes.c_uint64)]


class Tuning(ctypes.Structure):
    _fields_ = [("pt_lattices_per_block", ctypes.c_int), ("res_lattices_per_block", ctypes.c_int),
                ("sweep_threads", ctypes.c_int), ("cluster_threads", ctypes.c_int),
                ("cluster_iter_cap", ctypes.c_int)]


class PthrError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None


def load(path: str | None = None):
    """Load libpthr.so; raise if it is missing (no fallback path exists).
    PTHR_LIBRARY in the environment names another build of the same library
    (the range-checked debug build)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or os.environ.get("PTHR_LIBRARY") or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"PTHR CUDA library not built: {path} is missing "
                          f"(run paper_2605_25872_gb300.build.build())")
    L = ctypes.CDLL(path)
    vp, i, sz, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_uint64
    P = ctypes.POINTER
    sig = {
        "pthr_required_bytes": [P(Config), P(sz)],
        "pthr_buffer_info": [P(Config), i, P(sz), P(sz)],
        "pthr_lattice_bytes": [i, P(sz)],
        "pthr_lattice_storage_bytes": [i, i, P(sz)],
        "pthr_set_update_rule": [vp, i],
        "pthr_create_batch": [P(Config), vp, sz, vp, vp, vp, P(vp)],
        "pthr_set_stream": [vp, vp],
        "pthr_set_tuning": [vp, P(Tuning)],
        "pthr_get_tuning": [vp, P(Tuning)],
        "pthr_sweep": [vp, i, i],
        "pthr_houdayer": [vp],
        "pthr_cluster_labels": [vp, vp],
        "pthr_swap": [vp, i],
        "pthr_observables": [vp, i, vp, sz],
        "pthr_emcs": [vp, i, i],
        "pthr_prethermalize_reservoir": [vp, i, i, i],
        "pthr_poll": [vp, i],
        "pthr_export_spins": [vp, vp],
        "pthr_import_spins": [vp, vp],
        "pthr_reset_samples": [vp, i, i, vp, vp, i],
        "pthr_set_active": [vp, i, i, i],
        "pthr_save": [vp, vp, P(sz)],
        "pthr_load": [vp, vp, sz],
        "pthr_group_create": [vp, i, vp, P(vp)],
        "pthr_group_emcs": [vp, i],
        "pthr_measure_peak": [i, vp, sz, vp, P(ctypes.c_double), P(ctypes.c_double)],
        "pthr_check_canaries": [vp, P(ctypes.c_int)],
        "pthr_reservoir_autocorrelation": [vp, i, i, i, i, vp, sz, vp],
        "pthr_reservoir_autocorrelation_noalloc": [vp, i, i, i, i, vp],
        "pthr_group_info": [vp, P(i)],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.pthr_destroy.argtypes = [vp]
    L.pthr_destroy.restype = None
    L.pthr_group_destroy.argtypes = [vp]
    L.pthr_group_destroy.restype = None
    L.pthr_last_error.argtypes = [vp]
    L.pthr_last_error.restype = ctypes.c_char_p
    L.pthr_version.argtypes = []
    L.pthr_version.restype = ctypes.c_char_p
    _lib = L
    return L


def check(status: int, handle=None):
    if status != PTHR_OK:
        msg = load().pthr_last_error(handle)
        raise PthrError(status, msg.decode() if msg else "")
    return status
