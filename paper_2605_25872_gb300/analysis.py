"""Host-side analysis of PTHR runs (NumPy): the quantities of Secs. 2, 4 and 5
of arXiv 2605.25872 computed from the accumulators that the GPU kernels fill.

- log2 time bins (Sec. 4: bin b = [t_max/2^(b+1) + 1, t_max/2^b]);
- thermal averages per (sample, T) and the SDY observable S (Sec. 2, Eq. (5));
- temperature random-walk time tau_TRW = N_r N_T EMCS / round trips (Sec. 5);
- chaotic parameter X_{T1,T2} = <q^2_{T1,T2}> / sqrt(<q^2_{T1,T1}> <q^2_{T2,T2}>)
  (Sec. 5);
- effective dynamic exponent z_eff from two sizes (Sec. 5);
- the T_max spin autocorrelation C(tau) that sets the reservoir residence
  (Sec. 3, ER).
"""
from __future__ import annotations

import numpy as np

# accumulator fields per (sample, T): see include/pthr.h (PTHR_BUF_OBS)
N, SUM_E, SUM_E2, SUM_Q, SUM_Q2, SUM_QL, SUM_S, SUM_Q4 = range(8)


def log2_bins(t_max: int, n_bins: int):
    """Bins b = 0..n_bins-1 as inclusive EMCS ranges [t_max/2^(b+1) + 1,
    t_max/2^b]: bin 0 is the second half of the run, bin 1 the second quarter,
    and so on.  EMCS are counted from 1."""
    out = []
    for b in range(n_bins):
        hi = t_max // (2 ** b)
        lo = t_max // (2 ** (b + 1)) + 1
        if lo > hi:
            break
        out.append((lo, hi))
    return out


def thermal_averages(obs: np.ndarray, n_replicas: int) -> dict:
    """Per (sample, T) averages from accumulators obs[S, N_T, 8]: <e>, <e^2>
    (over measurements and groups), <q>, <q^2>, <q^4>, <q_l>, <S> (over
    measurements and replica pairs)."""
    n = obs[..., N]
    pairs = max(n_replicas // 2, 1)
    ng = n * n_replicas
    npair = n * pairs
    with np.errstate(invalid="ignore", divide="ignore"):
        return {"e": obs[..., SUM_E] / ng, "e2": obs[..., SUM_E2] / ng,
                "q": obs[..., SUM_Q] / npair, "q2": obs[..., SUM_Q2] / npair,
                "q4": obs[..., SUM_Q4] / npair, "ql": obs[..., SUM_QL] / npair,
                "S": obs[..., SUM_S] / npair}


def sdy(e: np.ndarray, ql: np.ndarray, T: np.ndarray) -> np.ndarray:
    """S = H/(3V) + (1 - q_l)/T = e/3 + (1 - q_l)/T (Sec. 2, Eq. (5))."""
    return e / 3.0 + (1.0 - ql) / T


def tau_trw(n_replicas: int, n_temps: int, n_emcs: int, round_trips) -> np.ndarray:
    """tau_TRW = N_r N_T (number of EMCS) / (total number of round trips)."""
    rt = np.asarray(round_trips, dtype=np.float64)
    with np.errstate(divide="ignore"):
        return n_replicas * n_temps * float(n_emcs) / rt


def chaos_parameter(q2_cross, q2_t1, q2_t2):
    """X_{T1,T2} = <q^2_{T1,T2}> / sqrt(<q^2_{T1,T1}> <q^2_{T2,T2}>)."""
    return np.asarray(q2_cross) / np.sqrt(np.asarray(q2_t1) * np.asarray(q2_t2))


def chaos_from_accumulators(chaos: np.ndarray, obs: np.ndarray, n_replicas: int) -> np.ndarray:
    """X_{T_0, T_k} per (sample, k) from the CHAOS buffer [S, N_T, 2] and the
    observable accumulators."""
    avg = thermal_averages(obs, n_replicas)
    with np.errstate(invalid="ignore", divide="ignore"):
        cross = chaos[..., 1] / chaos[..., 0]
    return chaos_parameter(cross, avg["q2"][:, :1], avg["q2"])


def z_eff(tau1: float, tau2: float, L1: float, L2: float) -> float:
    """z_eff(L1, L2) = (log tau(L1) - log tau(L2)) / (log L1 - log L2)."""
    return (np.log(tau1) - np.log(tau2)) / (np.log(L1) - np.log(L2))


def run_binned(batch, t_max: int, n_bins: int, chaos: bool = False):
    """Advance `batch` by t_max EMCS, measuring after every EMCS, and return
    the accumulators of each log2 bin: {b: (obs copy, chaos copy)}.  The
    accumulators are reset at the start of every bin."""
    bins = log2_bins(t_max, n_bins)
    starts = {lo: b for b, (lo, hi) in enumerate(bins)}
    ends = {hi: b for b, (lo, hi) in enumerate(bins)}
    out = {}
    for t in range(1, t_max + 1):
        if t in starts:
            batch.reset_observables()
        batch.sweep(batch.cfg.sweeps_per_emcs, batch.cfg.res_sweeps_per_emcs if batch.cfg.er_on else 0)
        if batch.cfg.cluster != "off":
            batch.houdayer()
        batch.swap(True, batch.cfg.er_on)
        batch.measure(chaos=chaos)
        if t in ends:
            batch.synchronize()          # the batch may run on its own stream
            out[ends[t]] = (batch.obs.cpu().numpy().copy(), batch.chaos.cpu().numpy().copy())
    return out


def spin_autocorrelation(sums, n_replicas: int, n_res: int, V: int):
    """C(tau) = (1/V) sum_i <s_i(t) s_i(t + tau)> (Sec. 3, ER) from the
    integer sums of pthr_reservoir_autocorrelation, out[sample, point]:
    returns (per-sample C [S, n_points], disorder average [n_points], its
    standard error [n_points])."""
    c = np.asarray(sums, dtype=np.float64) / float(n_replicas * n_res * V)
    n = c.shape[0]
    err = c.std(axis=0, ddof=1) / np.sqrt(n) if n > 1 else np.full(c.shape[1], np.nan)
    return c, c.mean(axis=0), err


def observable_records(obs: np.ndarray, T, n_replicas: int, emcs: int, sample_ids=None,
                       pt_accepted=None, cluster_stats=None) -> list:
    """One flat record per (sample, temperature) of the thermal averages of
    `thermal_averages` at EMCS count `emcs`, for logging as JSON lines.
    Optional: PT acceptance counts [S, N_r, N_T] (summed over groups, pair
    (k, k+1) on temperature k) and the last cluster move's statistics
    [S, n_pairs, N_T, 4] (clusters, largest, second largest, flipped sites;
    summed over pairs)."""
    avg = thermal_averages(np.asarray(obs, dtype=np.float64), n_replicas)
    S, NT = obs.shape[:2]
    ids = list(range(S)) if sample_ids is None else [int(x) for x in sample_ids]
    out = []
    for s in range(S):
        for k in range(NT):
            rec = {"emcs": int(emcs), "sample": ids[s], "k": k, "T": float(T[k]),
                   "n": int(obs[s, k, N])}
            rec.update({name: float(v[s, k]) for name, v in avg.items()})
            if pt_accepted is not None:
                rec["pt_accepted"] = int(np.asarray(pt_accepted)[s, :, k].sum())
            if cluster_stats is not None:
                cs = np.asarray(cluster_stats)[s, :, k].sum(axis=0)
                rec.update({"clusters": int(cs[0]), "largest": int(cs[1]), "second": int(cs[2]),
                            "flipped": int(cs[3])})
            out.append(rec)
    return out


def append_jsonl(path, records) -> int:
    """Append records (dicts) to a JSON-lines file; returns the count."""
    import json
    with open(path, "a") as f:
        for r in records:
            f.write(json.dumps(r) + "\n")
    return len(records)
