"""Step-by-step oracle twin of a GPU batch, for the parity tests.

It holds one ``oracle.OracleSample`` per disorder sample and advances it with
the oracle's primitives in the same units as the C ABI (sweep, cluster move,
swap, measure), logging every near tie.  It never reads anything produced by
the CUDA path; the tests only push oracle state into the GPU (resync), never
the other way round.
"""
from __future__ import annotations

import ctypes

import numpy as np

import oracle as O

RULE = {"metropolis": O.RULE_METROPOLIS, "heatbath": O.RULE_HEATBATH, "micsa": O.RULE_MICSA}
CLUSTER = {"off": O.CLUSTER_OFF, "acu": O.CLUSTER_ACU, "single": O.CLUSTER_SINGLE}


class Mirror:
    def __init__(self, cfg, J, seeds, tie_eps=1e-6, field_err_bound=False):
        self.cfg = cfg
        self.L, self.V = cfg.L, cfg.L ** 3
        self.rule = RULE[cfg.rule]
        self.cluster = CLUSTER[cfg.cluster]
        self.tie_eps = tie_eps
        self.field_err_bound = field_err_bound
        self.seeds = [int(x) for x in np.asarray(seeds, dtype=np.uint64)]
        J = np.asarray(J, dtype=np.float32).reshape(cfg.n_samples, 3, self.V)
        self.samples = []
        for s in range(cfg.n_samples):
            smp = O.OracleSample(cfg.L, cfg.n_temps, cfg.t_min, cfg.t_max, self.seeds[s],
                                 J=J[s].astype(np.float64), n_groups=cfg.n_replicas,
                                 n_res=cfg.n_res, sweeps_per_emcs=cfg.sweeps_per_emcs,
                                 res_sweeps_per_emcs=cfg.res_sweeps_per_emcs,
                                 cluster_mode=self.cluster, er_on=cfg.er_on, rule=self.rule,
                                 acu_t_below=cfg.acu_t_below, tie_eps=tie_eps)
            self.samples.append(smp)
        self.T = self.samples[0].T
        self.beta = self.samples[0].beta
        self.n_acu = 0
        if self.cluster != O.CLUSTER_OFF:
            for k in range(cfg.n_temps):
                if self.T[k] < cfg.acu_t_below:
                    self.n_acu = k + 1
        self.pt_off = 0
        self.res_off = 0
        self.decisions = 0    # local accept decisions taken so far
        self.n_ties = 0       # near-tie local decisions among them

    # ---------------------------------------------------------------- sweeps
    def sweep(self, n_pt, n_res, emcs_override=None, samples=None, pretherm=False):
        """Returns {(s, lat): set(tie sites)} for this call.  Pre-thermalisation
        sweeps continue each sample's own pre-thermalisation sweep index."""
        c = self.cfg
        ties = {}
        for s in (range(c.n_samples) if samples is None else samples):
            smp = self.samples[s]
            emcs = O.PRETHERM_EMCS if pretherm else smp.emcs_done
            for g in range(c.n_replicas):
                for pos in range(smp.nslot):
                    in_res = pos >= c.n_temps
                    nsw = n_res if in_res else n_pt
                    if pretherm and not in_res:
                        continue
                    lat = smp.lattice_at(g, pos)
                    b = self.beta[-1] if in_res else self.beta[pos]
                    base = smp.pretherm_done if pretherm else (self.res_off if in_res else self.pt_off)
                    e = g * c.n_res + (pos - c.n_temps) if in_res else g * c.n_temps + pos
                    for sw in range(nsw):
                        if self.rule == O.RULE_MICSA:
                            acc, tl, dE, nt = O.sweep_micsa(self.L, smp.J, smp.spins[lat], b, smp.seed, e,
                                                            int(in_res), emcs & 0xFFFFFFFF, base + sw,
                                                            tie_eps=self.tie_eps)
                        else:
                            acc, tl, dE = O.sweep(self.L, smp.J, smp.spins[lat], b, smp.seed, lat,
                                                  emcs & 0xFFFFFFFF, base + sw, rule=self.rule,
                                                  tie_eps=self.tie_eps,
                                                  field_err_bound=self.field_err_bound)
                            nt = len(tl)
                        smp.flips[lat] += acc
                        self.decisions += self.V
                        self.n_ties += nt
                        if len(tl):
                            ties.setdefault((s, lat), set()).update(int(t) for t in tl)
                    smp.E_lat[lat] = O.energy(self.L, smp.J, smp.spins[lat])
            if pretherm:
                smp.pretherm_done += n_res
        if not pretherm:
            self.pt_off += n_pt
            self.res_off += n_res
        return ties

    # ---------------------------------------------------------------- cluster move
    def houdayer(self, labels_out=None):
        c = self.cfg
        stats = {}
        for s, smp in enumerate(self.samples):
            if smp.emcs_done % c.acu_interval != 0:
                continue
            for p in range(c.n_replicas // 2):
                for k in range(self.n_acu):
                    la = smp.lattice_at(2 * p, k)
                    lb = smp.lattice_at(2 * p + 1, k)
                    pid = p * c.n_temps + k
                    if self.cluster == O.CLUSTER_ACU:
                        lab, n = O.acu(self.L, smp.spins[la], smp.spins[lb], smp.seed, pid,
                                       smp.emcs_done & 0xFFFFFFFF)
                    else:
                        lab, n = O.houdayer_single(self.L, smp.spins[la], smp.spins[lb], smp.seed,
                                                   pid, smp.emcs_done & 0xFFFFFFFF)
                    stats[(s, p, k)] = (lab, n)
                    smp.E_lat[la] = O.energy(self.L, smp.J, smp.spins[la])
                    smp.E_lat[lb] = O.energy(self.L, smp.J, smp.spins[lb])
        return stats

    # ---------------------------------------------------------------- PT / ER
    def swap(self, pt=True, er=None):
        """Returns {sample: near-tie PT decisions} for this call."""
        c = self.cfg
        er = c.er_on if er is None else er
        pt_ties = {}
        for s, smp in enumerate(self.samples):
            for g in range(c.n_replicas):
                perm = smp.perm[g * smp.nslot:(g + 1) * smp.nslot]
                if pt:
                    Ep = np.array([smp.E_lat[g * smp.nslot + perm[q]] for q in range(smp.nslot)])
                    acc, nt = O.pt_round(self.beta, perm, Ep, smp.seed, g,
                                         smp.emcs_done & 0xFFFFFFFF, self.tie_eps)
                    if nt:
                        pt_ties[s] = pt_ties.get(s, 0) + nt
                    smp.pt_accepted[g * c.n_temps:(g + 1) * c.n_temps] += acc
                    rs = smp.rt_state[g * smp.nslot:(g + 1) * smp.nslot]
                    if rs[perm[0]] & 1:
                        rs[perm[0]] |= 2
                if er and c.n_res > 0:
                    O.er_step(c.n_temps, c.n_res, perm, smp.age[g * c.n_res:(g + 1) * c.n_res],
                              smp.rt_state[g * smp.nslot:(g + 1) * smp.nslot],
                              smp.round_trips[g:g + 1])
                # perm is a view into smp.perm: updated in place
            smp.emcs_done += 1
        self.pt_off = 0
        self.res_off = 0
        return pt_ties

    def measure(self):
        for smp in self.samples:
            st = smp._state()
            O.lib().orc_measure(ctypes.byref(smp.cfg), O.oracle._p(smp.J), O.oracle._p(smp.T),
                                ctypes.byref(st))

    def emcs(self):
        c = self.cfg
        ties = self.sweep(c.sweeps_per_emcs, c.res_sweeps_per_emcs if c.er_on else 0)
        if self.cluster != O.CLUSTER_OFF:
            self.houdayer()
        pt_ties = self.swap(True, c.er_on)
        self.measure()
        return ties, pt_ties

    # ---------------------------------------------------------------- state views
    def spins(self):
        return np.stack([smp.spins for smp in self.samples])

    def perms(self):
        c = self.cfg
        return np.stack([smp.perm.reshape(c.n_replicas, -1) for smp in self.samples])

    def energies(self):
        return np.stack([smp.E_lat for smp in self.samples])

    def ages(self):
        c = self.cfg
        return np.stack([smp.age.reshape(c.n_replicas, -1) for smp in self.samples])


def neighbours(L, i):
    x, y, z = i % L, (i // L) % L, i // (L * L)
    out = []
    for dx, dy, dz in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
        out.append(((x + dx) % L) + L * (((y + dy) % L) + L * ((z + dz) % L)))
    return out


def colour(L, i):
    return ((i % L) + (i // L) % L + i // (L * L)) & 1


def explained_by_ties(L, mismatch_sites, tie_sites):
    """Within one checkerboard sweep a near-tie decision at site t can change
    t itself and, if t is of the first colour, its neighbours (second colour,
    updated later in the same sweep).  True iff every mismatch is so explained."""
    allowed = set(tie_sites)
    for t in tie_sites:
        if colour(L, t) == 0:
            allowed.update(neighbours(L, t))
    return set(int(m) for m in mismatch_sites) <= allowed
