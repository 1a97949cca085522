"""Python handle on the FP64 CPU oracle (``pthr_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use this module; the product path never imports
it.  It shares no code with the CUDA library.

The C file is compiled on first use (or by ``build()``) with gcc, without
fast-math and without FMA contraction, so that x86 and Arm hosts give the same
FP64 results.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pthr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()

RULE_METROPOLIS, RULE_HEATBATH, RULE_MICSA = 0, 1, 2
ORDER_CHECKERBOARD, ORDER_LEXICOGRAPHIC = 0, 1
CLUSTER_OFF, CLUSTER_ACU, CLUSTER_SINGLE = 0, 1, 2
PRETHERM_EMCS = 0xFFFFFFFF  # EMCS counter word used by reservoir pre-thermalisation

# observable accumulator fields per temperature
OBS_FIELDS = ("n", "e", "e2", "q", "q2", "ql", "S", "q4")


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (idempotent)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Cfg(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("n_temps", ctypes.c_int), ("n_groups", ctypes.c_int),
                ("n_res", ctypes.c_int), ("sweeps_per_emcs", ctypes.c_int),
                ("res_sweeps_per_emcs", ctypes.c_int), ("cluster_mode", ctypes.c_int),
                ("er_on", ctypes.c_int), ("rule", ctypes.c_int), ("order", ctypes.c_int),
                ("acu_t_below", ctypes.c_double), ("tie_eps", ctypes.c_double)]


class _State(ctypes.Structure):
    _fields_ = [("spins", ctypes.c_void_p), ("perm", ctypes.c_void_p), ("E_lat", ctypes.c_void_p),
                ("age", ctypes.c_void_p), ("rt_state", ctypes.c_void_p),
                ("round_trips", ctypes.c_void_p), ("pt_accepted", ctypes.c_void_p),
                ("flips", ctypes.c_void_p), ("n_ties", ctypes.c_void_p), ("obs", ctypes.c_void_p)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # ORACLE_LIB: a prebuilt copy (the mutation tests load deliberately
            # broken copies to show that the pins catch them)
            L = ctypes.CDLL(os.environ.get("ORACLE_LIB") or build())
            vp, i, u32, u64, d = (ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32,
                                  ctypes.c_uint64, ctypes.c_double)
            L.orc_philox4x32_10.argtypes = [vp, vp, vp]
            L.orc_energy.argtypes = [i, vp, vp]
            L.orc_energy.restype = d
            L.orc_couplings_from_seed.argtypes = [i, u64, vp]
            L.orc_init_spins.argtypes = [i, u64, i, vp]
            L.orc_sweep.argtypes = [i, vp, vp, d, u64, i, u32, u32, i, i, d, i, vp, i, vp, vp]
            L.orc_sweep.restype = ctypes.c_long
            L.orc_sweep_micsa.argtypes = [i, vp, vp, d, u64, i, i, u32, u32, d, vp, i, vp, vp, vp]
            L.orc_sweep_micsa.restype = ctypes.c_long
            L.orc_micsa_walker.argtypes = [i, vp, d, d, vp, d, vp]
            L.orc_micsa_walker.restype = d
            L.orc_cc_labels.argtypes = [i, vp, vp, vp]
            L.orc_cc_labels.restype = i
            L.orc_acu.argtypes = [i, vp, vp, u64, u32, u32, vp]
            L.orc_acu.restype = i
            L.orc_houdayer_single.argtypes = [i, vp, vp, u64, u32, u32, vp]
            L.orc_houdayer_single.restype = i
            L.orc_pt_round.argtypes = [i, vp, vp, vp, u64, i, u32, vp, d, vp]
            L.orc_er_step.argtypes = [i, i, vp, vp, vp, vp, vp]
            L.orc_pair_observables.argtypes = [i, vp, vp, vp, d, vp]
            L.orc_enumerate_l2.argtypes = [vp, i, vp, vp, vp]
            L.orc_enumerate_l2.restype = i
            L.orc_temperatures.argtypes = [i, d, d, vp, vp]
            L.orc_measure.argtypes = [ctypes.POINTER(_Cfg), vp, vp, ctypes.POINTER(_State)]
            L.orc_emcs.argtypes = [ctypes.POINTER(_Cfg), vp, vp, vp, u64, u32, ctypes.POINTER(_State)]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


# ----------------------------------------------------------------------------- primitives

def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def couplings_from_seed(L: int, seed: int) -> np.ndarray:
    """J[3, V] (FP64 values on the 2^-18 grid) from the sample seed."""
    J = np.zeros(3 * L ** 3, dtype=np.float64)
    lib().orc_couplings_from_seed(L, seed, _p(J))
    return J.reshape(3, L ** 3)


def init_spins(L: int, seed: int, lat: int) -> np.ndarray:
    s = np.zeros(L ** 3, dtype=np.int8)
    lib().orc_init_spins(L, seed, lat, _p(s))
    return s


def energy(L: int, J: np.ndarray, s: np.ndarray) -> float:
    J = np.ascontiguousarray(J, dtype=np.float64)
    s = np.ascontiguousarray(s, dtype=np.int8)
    return lib().orc_energy(L, _p(J), _p(s))


def sweep(L, J, s, beta, seed, lat, emcs, sweep_idx, order=ORDER_CHECKERBOARD,
          rule=RULE_METROPOLIS, tie_eps=1e-6, field_err_bound=False, max_ties=4096):
    """One sweep in place.  Returns (accepted, tie_sites, dE)."""
    J = np.ascontiguousarray(J, dtype=np.float64)
    assert s.dtype == np.int8 and s.flags["C_CONTIGUOUS"]
    ties = np.zeros(max_ties, dtype=np.int32)
    n_ties = ctypes.c_int(0)
    dE = ctypes.c_double(0.0)
    acc = lib().orc_sweep(L, _p(J), _p(s), float(beta), seed, lat, emcs & 0xFFFFFFFF,
                          sweep_idx, order, rule, tie_eps, int(field_err_bound), _p(ties),
                          max_ties, ctypes.byref(n_ties), ctypes.byref(dE))
    return acc, ties[:min(n_ties.value, max_ties)].copy(), dE.value


def sweep_micsa(L, J, s, beta, seed, e, kind, emcs, sweep_idx, tie_eps=1e-6, max_ties=4096):
    """One MicSA sweep in place (walkers keyed by the lattice's position e
    within its kind).  Returns (accepted, sites a near tie may have changed,
    dE, near-tie decisions)."""
    J = np.ascontiguousarray(J, dtype=np.float64)
    assert s.dtype == np.int8 and s.flags["C_CONTIGUOUS"]
    ties = np.zeros(max_ties, dtype=np.int32)
    n_sites, n_dec = ctypes.c_int(0), ctypes.c_int(0)
    dE = ctypes.c_double(0.0)
    acc = lib().orc_sweep_micsa(L, _p(J), _p(s), float(beta), seed, e, kind, emcs & 0xFFFFFFFF, sweep_idx,
                                tie_eps, _p(ties), max_ties, ctypes.byref(n_sites), ctypes.byref(n_dec),
                                ctypes.byref(dE))
    return acc, ties[:min(n_sites.value, max_ties)].copy(), dE.value, n_dec.value


def micsa_walker(dE, beta, u, tie_eps=1e-6):
    """The walker rule on the sites with energy changes dE (in order):
    returns (flips, energy taken from the walker, near-tie flags)."""
    dE = np.ascontiguousarray(dE, dtype=np.float64)
    flip = np.zeros(len(dE), dtype=np.int32)
    tie = np.zeros(len(dE), dtype=np.int32)
    D = lib().orc_micsa_walker(len(dE), _p(dE), float(beta), float(u), _p(flip), tie_eps, _p(tie))
    return flip, D, tie


def cc_labels(L, sa, sb):
    lab = np.zeros(L ** 3, dtype=np.int32)
    n = lib().orc_cc_labels(L, _p(np.ascontiguousarray(sa, np.int8)),
                            _p(np.ascontiguousarray(sb, np.int8)), _p(lab))
    return lab, n


def acu(L, sa, sb, seed, pair_id, emcs):
    """All-cluster update in place; returns (labels, n_clusters)."""
    lab = np.zeros(L ** 3, dtype=np.int32)
    n = lib().orc_acu(L, _p(sa), _p(sb), seed, pair_id, emcs, _p(lab))
    return lab, n


def houdayer_single(L, sa, sb, seed, pair_id, emcs):
    lab = np.zeros(L ** 3, dtype=np.int32)
    n = lib().orc_houdayer_single(L, _p(sa), _p(sb), seed, pair_id, emcs, _p(lab))
    return lab, n


def pt_round(beta, perm, E, seed, group, emcs, tie_eps=1e-6):
    beta = np.ascontiguousarray(beta, np.float64)
    acc = np.zeros(len(beta), dtype=np.int64)
    ties = ctypes.c_int(0)
    lib().orc_pt_round(len(beta), _p(beta), _p(perm), _p(E), seed, group, emcs, _p(acc),
                       tie_eps, ctypes.byref(ties))
    return acc, ties.value


def er_step(n_temps, n_res, perm, age, rt_state=None, round_trips=None):
    lib().orc_er_step(n_temps, n_res, _p(perm), None, _p(age),
                      None if rt_state is None else _p(rt_state),
                      None if round_trips is None else _p(round_trips))


def pair_observables(L, J, sa, sb, T):
    out = np.zeros(3)
    lib().orc_pair_observables(L, _p(np.ascontiguousarray(J, np.float64)), _p(sa), _p(sb), T, _p(out))
    return out


def enumerate_l2(J, temps, want_probs=False):
    """Exact Boltzmann averages on 2x2x2: rows (<e>, <q^2>, <q_l>, <S>, <e^2>)."""
    J = np.ascontiguousarray(J, np.float64).reshape(-1)
    assert J.size == 24
    T = np.ascontiguousarray(temps, np.float64)
    out = np.zeros((len(T), 5))
    probs = np.zeros((len(T), 256)) if want_probs else None
    lib().orc_enumerate_l2(_p(J), len(T), _p(T), _p(out), None if probs is None else _p(probs))
    return (out, probs) if want_probs else out


def temperatures(n_temps, t_min, t_max):
    T = np.zeros(n_temps)
    b = np.zeros(n_temps)
    lib().orc_temperatures(n_temps, t_min, t_max, _p(T), _p(b))
    return T, b


# ----------------------------------------------------------------------------- one sample

class OracleSample:
    """State of one disorder sample: N_r replica groups, each with N_T PT
    clones and N_res reservoir clones, stepped one EMCS at a time."""

    def __init__(self, L, n_temps, t_min, t_max, seed, J=None, n_groups=4, n_res=4,
                 sweeps_per_emcs=10, res_sweeps_per_emcs=240, cluster_mode=CLUSTER_ACU,
                 er_on=True, rule=RULE_METROPOLIS, order=ORDER_CHECKERBOARD,
                 acu_t_below=1.0, tie_eps=1e-6):
        self.L, self.V = L, L ** 3
        self.seed = int(seed)
        self.cfg = _Cfg(L, n_temps, n_groups, n_res, sweeps_per_emcs, res_sweeps_per_emcs,
                        cluster_mode, int(er_on), rule, order, acu_t_below, tie_eps)
        self.n_temps, self.n_groups, self.n_res = n_temps, n_groups, n_res
        self.nslot = n_temps + n_res
        self.n_lat = n_groups * self.nslot
        self.T, self.beta = temperatures(n_temps, t_min, t_max)
        self.J = (couplings_from_seed(L, self.seed) if J is None
                  else np.ascontiguousarray(np.asarray(J, dtype=np.float64).reshape(3, -1)))
        self.spins = np.zeros((self.n_lat, self.V), dtype=np.int8)
        for lat in range(self.n_lat):
            self.spins[lat] = init_spins(L, self.seed, lat)
        self.perm = np.tile(np.arange(self.nslot, dtype=np.int32), n_groups).copy()
        self.E_lat = np.array([energy(L, self.J, self.spins[l]) for l in range(self.n_lat)])
        # reading: reservoir ages start at 0, 1, ..., n_res-1
        self.age = np.tile(np.arange(n_res, dtype=np.uint32), n_groups).copy()
        self.rt_state = np.zeros(self.n_lat, dtype=np.uint8)
        self.round_trips = np.zeros(n_groups, dtype=np.int64)
        self.pt_accepted = np.zeros(n_groups * n_temps, dtype=np.int64)
        self.flips = np.zeros(self.n_lat, dtype=np.int64)
        self.n_ties = np.zeros(2, dtype=np.int64)
        self.obs = np.zeros((n_temps, len(OBS_FIELDS)))
        self.emcs_done = 0
        self.pretherm_done = 0    # reservoir pre-thermalisation sweeps so far

    def _state(self):
        return _State(*(a.ctypes.data for a in (self.spins, self.perm, self.E_lat, self.age,
                                                self.rt_state, self.round_trips, self.pt_accepted,
                                                self.flips, self.n_ties, self.obs)))

    def prethermalize_reservoir(self, n_sweeps):
        """n_sweeps at T_max of every reservoir clone, EMCS counter word 2^32-1;
        the sweep index continues over successive calls."""
        for g in range(self.n_groups):
            for r in range(self.n_res):
                lat = g * self.nslot + int(self.perm[g * self.nslot + self.n_temps + r])
                for sw in range(n_sweeps):
                    if self.cfg.rule == RULE_MICSA:
                        _, _, _, nt = sweep_micsa(self.L, self.J, self.spins[lat], self.beta[-1], self.seed,
                                                  g * self.n_res + r, 1, PRETHERM_EMCS, self.pretherm_done + sw,
                                                  tie_eps=self.cfg.tie_eps)
                    else:
                        _, ties, _ = sweep(self.L, self.J, self.spins[lat], self.beta[-1], self.seed, lat,
                                           PRETHERM_EMCS, self.pretherm_done + sw, self.cfg.order,
                                           self.cfg.rule, tie_eps=self.cfg.tie_eps)
                        nt = len(ties)
                    self.n_ties[0] += nt
                self.E_lat[lat] = energy(self.L, self.J, self.spins[lat])
        self.pretherm_done += n_sweeps

    def emcs(self, n=1):
        st = self._state()
        for _ in range(n):
            lib().orc_emcs(ctypes.byref(self.cfg), _p(self.J), _p(self.T), _p(self.beta),
                           self.seed, self.emcs_done & 0xFFFFFFFF, ctypes.byref(st))
            self.emcs_done += 1

    def lattice_at(self, g, pos):
        return g * self.nslot + int(self.perm[g * self.nslot + pos])


def run_samples_threaded(samples, n_emcs, threads):
    """Advance independent samples in parallel host threads (the C calls drop
    the GIL).  Returns the number of threads used."""
    threads = max(1, min(threads, len(samples)))
    with ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(lambda s: s.emcs(n_emcs), samples))
    return threads
