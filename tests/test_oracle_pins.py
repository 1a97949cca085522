"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

None of these tests re-types an oracle formula: each checks the oracle against
a published value, a closed form, an invariant, a library routine or an exact
enumeration.  They run on the CPU only.
"""
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy import sparse, stats
from scipy.sparse.csgraph import connected_components

import oracle as O
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------- Philox

def test_philox_known_answers():
    """Philox4x32-10 against the known-answer vectors of its paper (SC'11)."""
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(t, 16) for t in line.split()])
    assert len(rows) == 3
    for r in rows:
        out = O.philox4x32_10(r[0:4], r[4:6])
        assert [int(x) for x in out] == r[6:10]


# ----------------------------------------------------------------------------- couplings / geometry

def test_couplings_from_seed_are_standard_normal_on_grid():
    """Sec. 2: J ~ N(0,1).  Moments and a Kolmogorov-Smirnov test against the
    normal CDF; every value on the 2^-18 grid and within the Box-Muller bound."""
    J = np.concatenate([O.couplings_from_seed(16, 1000 + s).ravel() for s in range(8)])
    n = J.size
    assert abs(J.mean()) < 5.0 / np.sqrt(n)
    assert abs(J.var() - 1.0) < 5.0 * np.sqrt(2.0 / n)
    assert abs(stats.skew(J)) < 5.0 * np.sqrt(6.0 / n)
    assert stats.kstest(J, "norm").pvalue > 1e-4
    assert np.all(np.rint(J * 2 ** 18) == J * 2 ** 18)
    assert np.abs(J).max() <= np.sqrt(-2 * np.log(2.0 ** -24)) + 1e-6
    # the sample seed is the Philox key: different seeds, different couplings
    assert not np.array_equal(O.couplings_from_seed(4, 1), O.couplings_from_seed(4, 2))


def test_init_spins_are_fair_and_distinct_per_lattice():
    s = np.stack([O.init_spins(16, 77, lat) for lat in range(16)]).astype(np.int64)
    n = s.size
    assert set(np.unique(s)) == {-1, 1}
    assert abs(s.mean()) < 5.0 / np.sqrt(n)
    assert not np.array_equal(s[0], s[1])


def _rand_J(L, seed, grid=True):
    return W.gaussian_couplings(L, 1, seed, on_grid=grid)[0].astype(np.float64)


def test_energy_closed_forms_and_symmetries():
    """Eq. (1): ferromagnet H(all up) = -3V; Neel state of the ferromagnet
    +3V; Z2 symmetry H(s) = H(-s) (Sec. 2); gauge invariance
    H_{tau J tau}(tau s) = H_J(s), which fails if any bond is attached to the
    wrong pair of sites."""
    for L in (2, 4, 6):
        V = L ** 3
        J1 = np.ones((3, V))
        up = np.ones(V, np.int8)
        assert O.energy(L, J1, up) == -3.0 * V
        x, y, z = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
        neel = np.where(((x + y + z) % 2).transpose(2, 1, 0).ravel() == 0, 1, -1).astype(np.int8)
        assert O.energy(L, J1, neel) == 3.0 * V
        J = _rand_J(L, 5 + L)
        s = W.random_spins(V, 11 + L)
        H = O.energy(L, J, s)
        assert O.energy(L, J, (-s).astype(np.int8)) == H
        tau = W.random_spins(V, 99 + L).astype(np.float64)
        # gauge-transformed couplings: J'_{mu}(i) = tau_i J_mu(i) tau_{i+mu}
        t3 = tau.reshape(L, L, L)  # [z][y][x]
        shifts = [np.roll(t3, -1, axis=2), np.roll(t3, -1, axis=1), np.roll(t3, -1, axis=0)]
        Jg = np.stack([tau * J[mu] * shifts[mu].ravel() for mu in range(3)])
        sg = (tau * s).astype(np.int8)
        assert O.energy(L, Jg, sg) == pytest.approx(H, abs=1e-12)


def test_sweep_incremental_energy_equals_recomputed():
    """The energy change summed over accepted moves equals the difference of
    energies recomputed from scratch (exact for couplings on the 2^-18 grid)."""
    for L, rule in ((4, O.RULE_METROPOLIS), (6, O.RULE_HEATBATH), (8, O.RULE_METROPOLIS)):
        J = _rand_J(L, 3 * L)
        s = W.random_spins(L ** 3, 7 * L)
        E0 = O.energy(L, J, s)
        tot = 0.0
        for sw in range(20):
            _, _, dE = O.sweep(L, J, s, 1.0 / 0.4, 123, 0, 5, sw, rule=rule)
            tot += dE
        assert E0 + tot == O.energy(L, J, s)


def test_micsa_sweep_incremental_energy_equals_recomputed():
    """MicSA (App. A.1): the energy the walkers hand to the lattice, summed
    over accepted flips, equals the change of the recomputed energy."""
    for L in (4, 6, 8):
        J = _rand_J(L, 5 * L)
        s = W.random_spins(L ** 3, 9 * L)
        E0 = O.energy(L, J, s)
        tot = 0.0
        for sw in range(20):
            _, _, dE, _ = O.sweep_micsa(L, J, s, 1.0 / 0.5, 321, 3, 0, 7, sw)
            tot += dE
        assert E0 + tot == O.energy(L, J, s)


def _walker_kernel(h, beta):
    """Exact transition matrix of one MicSA walker over n non-interacting
    spins with fields h (the sites of one checkerboard group): the walker's
    uniform u is integrated out exactly, the outcome being constant between
    the breakpoints exp(-beta X) of every offset X the walker can reach."""
    n = len(h)
    states = [np.array([1 - 2 * ((st >> k) & 1) for k in range(n)]) for st in range(2 ** n)]
    K = np.zeros((2 ** n, 2 ** n))
    for a, s in enumerate(states):
        dE = 2.0 * s * h
        X = {0.0}
        for k in range(n):
            X = X | {x + dE[k] for x in X}
        cuts = sorted({0.0, 1.0} | {float(np.exp(-beta * x)) for x in X if x > 0})
        for lo, hi in zip(cuts[:-1], cuts[1:]):
            if hi <= lo:
                continue
            u = 0.5 * (lo + hi)
            flip, D, _ = O.micsa_walker(dE, beta, u)
            assert D <= -np.log(u) / beta + 1e-12          # the walker never goes negative
            t = s * np.where(flip == 1, -1, 1)
            b = sum(((1 - t[k]) // 2) << k for k in range(n))
            K[a, b] += hi - lo
    return states, K


def test_micsa_walker_leaves_the_boltzmann_weight_stationary():
    """Detailed balance of the MicSA move (App. A.1) on its own: a walker
    drawn from the canonical exponential at T and debited by every accepted
    Delta E maps the Boltzmann weight of its n independent sites onto itself
    (exactly, with the walker's uniform integrated out)."""
    rng = np.random.default_rng(99)
    for n in (1, 2, 3, 4):
        for rep in range(6):
            h = rng.standard_normal(n) * 2.0
            beta = float(rng.uniform(0.5, 4.0))
            states, K = _walker_kernel(h, beta)
            np.testing.assert_allclose(K.sum(1), 1.0, atol=1e-12)
            pi = np.array([np.exp(beta * float(np.dot(s, h))) for s in states])
            pi /= pi.sum()
            np.testing.assert_allclose(pi @ K, pi, atol=1e-12)


def test_micsa_chain_agrees_with_metropolis_at_L4():
    """At L = 4 a MicSA walker serves two sites, so the 2x2x2 enumeration no
    longer reaches it: the full MicSA PTHR chain is compared with the
    Metropolis chain (pinned against enumeration) on the same sample: <e>
    and <q^2> agree within 5 combined standard errors at every T."""
    L, nT = 4, 4
    J = _rand_J(L, 77)
    est = {}
    for rule in (O.RULE_METROPOLIS, O.RULE_MICSA):
        smp = O.OracleSample(L, nT, 0.5, 1.6, seed=11, J=J, n_groups=4, n_res=2, sweeps_per_emcs=1,
                             res_sweeps_per_emcs=4, rule=rule)
        smp.emcs(300)
        blocks = []
        for b in range(16):
            before = smp.obs.copy()
            smp.emcs(400)
            d = smp.obs - before
            blocks.append(np.stack([d[:, 1] / (d[:, 0] * 4), d[:, 4] / (d[:, 0] * 2)], 1))
        blocks = np.array(blocks)
        est[rule] = (blocks.mean(0), blocks.std(0, ddof=1) / np.sqrt(len(blocks)))
    (m1, e1), (m2, e2) = est[O.RULE_METROPOLIS], est[O.RULE_MICSA]
    z = np.abs(m1 - m2) / np.sqrt(e1 ** 2 + e2 ** 2)
    assert np.all(z < 5.0), z


def test_sweep_is_gauge_covariant():
    """A Metropolis sweep with couplings tau J tau started from tau s, driven
    by the same random numbers, ends in tau times the original end state.  A
    wrong neighbour/bond pairing in the local field breaks this."""
    L = 6
    V = L ** 3
    J = _rand_J(L, 41)
    s = W.random_spins(V, 42)
    tau = W.random_spins(V, 43).astype(np.float64)
    t3 = tau.reshape(L, L, L)
    shifts = [np.roll(t3, -1, axis=2), np.roll(t3, -1, axis=1), np.roll(t3, -1, axis=0)]
    Jg = np.stack([tau * J[mu] * shifts[mu].ravel() for mu in range(3)])
    sg = (tau * s).astype(np.int8)
    for sw in range(10):
        O.sweep(L, J, s, 2.0, 5, 1, 0, sw)
        O.sweep(L, Jg, sg, 2.0, 5, 1, 0, sw)
    assert np.array_equal(sg, (tau * s).astype(np.int8))


def test_checkerboard_counter_layout_is_injective():
    """Every site of one colour gets its own (counter, word) pair."""
    for L in (2, 4, 6, 8, 10, 12, 16):
        Wd = (L // 2 + 3) // 4
        seen = set()
        for z in range(L):
            for y in range(L):
                for x in range(L):
                    c = (x + y + z) & 1
                    r, m = y + L * z, x >> 1
                    key = (c, r * Wd + (m >> 2), m & 3)
                    assert key not in seen
                    seen.add(key)


# ----------------------------------------------------------------------------- exact enumeration

T_GRID = np.array([0.3, 0.6, 0.9, 1.5])


def test_enumeration_closed_forms():
    """2x2x2 enumeration: J = 0 gives e = 0, <q^2> = 1/V, <q_l> = 0,
    <S> = 1/T; the ferromagnet at low T gives e = -3, q^2 = q_l = 1; at high
    T, q^2 -> 1/V."""
    out = O.enumerate_l2(np.zeros(24), T_GRID)
    np.testing.assert_allclose(out[:, 0], 0.0, atol=1e-15)
    np.testing.assert_allclose(out[:, 1], 1.0 / 8.0, rtol=1e-14)
    np.testing.assert_allclose(out[:, 2], 0.0, atol=1e-15)
    np.testing.assert_allclose(out[:, 3], 1.0 / T_GRID, rtol=1e-14)
    low = O.enumerate_l2(np.ones(24), [0.02])
    assert low[0, 0] == pytest.approx(-3.0, abs=1e-12)
    assert low[0, 1] == pytest.approx(1.0, abs=1e-12)
    assert low[0, 2] == pytest.approx(1.0, abs=1e-12)
    hi = O.enumerate_l2(np.ones(24), [1e7])
    assert hi[0, 1] == pytest.approx(1.0 / 8.0, abs=1e-6)


def test_enumeration_fluctuation_dissipation():
    """d<e>/dT = V (<e^2> - <e>^2) / T^2: pins the sign of the Boltzmann
    exponent and the second moment."""
    J = _rand_J(2, 17, grid=False)
    for T in (0.4, 0.9, 1.7):
        h = 1e-5
        ep = O.enumerate_l2(J, [T + h])[0, 0]
        em = O.enumerate_l2(J, [T - h])[0, 0]
        r = O.enumerate_l2(J, [T])[0]
        assert (ep - em) / (2 * h) == pytest.approx(8 * (r[4] - r[0] ** 2) / T ** 2, rel=1e-6)


def test_sdy_identity_disorder_average_is_zero():
    """Sec. 2, Eq. (6): the disorder average of <S> vanishes in equilibrium
    (Gaussian integration by parts).  Pins the coupling convention, the
    link overlap and the enumerator."""
    rng = np.random.Generator(np.random.PCG64(2024))
    vals = []
    for _ in range(3000):
        J = rng.standard_normal(24)
        vals.append(O.enumerate_l2(J, T_GRID)[:, 3])
    vals = np.array(vals)
    mean = vals.mean(0)
    err = vals.std(0, ddof=1) / np.sqrt(len(vals))
    assert np.all(np.abs(mean) < 4.5 * err), (mean, err)
    # a single sample generally has <S> != 0 (Sec. 2)
    assert np.abs(vals).max() > 10 * err.max()


def test_enumeration_gauge_invariance():
    J = _rand_J(2, 23, grid=False)
    tau = W.random_spins(8, 24).astype(np.float64)
    t3 = tau.reshape(2, 2, 2)
    shifts = [np.roll(t3, -1, axis=2), np.roll(t3, -1, axis=1), np.roll(t3, -1, axis=0)]
    Jg = np.stack([tau * J.reshape(3, 8)[mu] * shifts[mu].ravel() for mu in range(3)])
    np.testing.assert_allclose(O.enumerate_l2(Jg, T_GRID), O.enumerate_l2(J, T_GRID), rtol=1e-12)


# ----------------------------------------------------------------------------- clusters and ACU

def _scipy_components(L, sa, sb):
    V = L ** 3
    q = sa.astype(int) * sb.astype(int)
    idx = np.arange(V).reshape(L, L, L)
    rows, cols = [], []
    for ax in range(3):
        nb = np.roll(idx, -1, axis=ax).ravel()
        keep = q == q[nb]
        rows.append(np.arange(V)[keep])
        cols.append(nb[keep])
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    G = sparse.coo_matrix((np.ones(len(r)), (r, c)), shape=(V, V))
    n, comp = connected_components(G, directed=False)
    canon = np.zeros(n, dtype=np.int64) + V
    np.minimum.at(canon, comp, np.arange(V))
    return canon[comp], n


@pytest.mark.parametrize("L", [2, 4, 6, 8])
def test_cc_labels_match_scipy(L):
    """Sec. 3 ACU: clusters = connected components of {i~j: q_i q_j > 0};
    checked against scipy's graph routine, canonical label = min site."""
    V = L ** 3
    for k in range(6):
        sa = W.random_spins(V, 100 * L + k)
        sb = W.random_spins(V, 200 * L + k)
        if k == 4:
            sb = sa.copy()          # every q_i = +1: one cluster
        if k == 5:
            sb = (-sa).astype(np.int8)
        lab, n = O.cc_labels(L, sa, sb)
        ref, nref = _scipy_components(L, sa, sb)
        assert n == nref
        assert np.array_equal(lab, ref)


def test_acu_invariants():
    """Sec. 3: the ACU keeps every q_i (hence the partition), conserves
    H_a + H_b, flips whole clusters with both signs, and applying it twice
    with the same signs restores the pair."""
    L = 8
    V = L ** 3
    J = _rand_J(L, 31)
    flipped_frac = []
    for k in range(20):
        sa = W.random_spins(V, 300 + k)
        sb = W.random_spins(V, 400 + k)
        a0, b0 = sa.copy(), sb.copy()
        H0 = O.energy(L, J, sa) + O.energy(L, J, sb)
        lab0, n0 = O.cc_labels(L, sa, sb)
        lab, n = O.acu(L, sa, sb, 9, k, 3)
        assert np.array_equal(lab, lab0)
        assert np.array_equal(sa * sb, a0 * b0)
        assert np.array_equal(O.cc_labels(L, sa, sb)[0], lab0)
        assert O.energy(L, J, sa) + O.energy(L, J, sb) == H0
        changed = sa != a0
        for c in np.unique(lab0):
            m = lab0 == c
            assert changed[m].all() or not changed[m].any()
        clusters = np.unique(lab0)
        flipped_frac.append(np.mean([changed[lab0 == c][0] for c in clusters]))
        O.acu(L, sa, sb, 9, k, 3)
        assert np.array_equal(sa, a0) and np.array_equal(sb, b0)
    # eta = +-1 with probability 1/2
    assert abs(np.mean(flipped_frac) - 0.5) < 0.08


def test_acu_proposal_is_symmetric_on_2x2x2():
    """Detailed balance of the ACU (Sec. 3): from x, every sign assignment has
    probability 2^-n_c(x); the image y has the same clusters, so the reverse
    move has the same probability.  Checked over all 65536 pair states of
    2x2x2 with one random sign draw each."""
    L, V = 2, 8
    states = np.arange(256)
    spins = np.where((states[:, None] >> np.arange(V)) & 1, -1, 1).astype(np.int8)
    for a in range(0, 256, 3):
        for b in range(0, 256, 5):
            sa, sb = spins[a].copy(), spins[b].copy()
            lab0, n0 = O.cc_labels(L, sa, sb)
            O.acu(L, sa, sb, 1234, a, b)
            lab1, n1 = O.cc_labels(L, sa, sb)
            assert n0 == n1 and np.array_equal(lab0, lab1)


def test_houdayer_single_flips_one_negative_cluster():
    L, V = 6, 216
    counts = np.zeros(V)
    sa = W.random_spins(V, 51)
    sb = W.random_spins(V, 52)
    q = sa * sb
    for emcs in range(4000):
        a, b = sa.copy(), sb.copy()
        lab0, _ = O.cc_labels(L, a, b)
        lab, n = O.houdayer_single(L, a, b, 8, 0, emcs)
        ch = a != sa
        assert n == ch.sum() > 0
        seedsites = np.unique(lab0[ch])
        assert len(seedsites) == 1 and q[lab0 == seedsites[0]][0] == -1
        assert np.array_equal(ch, lab0 == seedsites[0])
        counts[lab0 == seedsites[0]] += 0  # cluster chosen
        counts[seedsites[0]] += 1
    # a cluster is chosen with probability (its size) / (number of q<0 sites)
    lab0, _ = O.cc_labels(L, sa, sb)
    neg = q < 0
    for c in np.unique(lab0[neg])[:5]:
        p = (lab0[neg] == c).mean()
        assert abs(counts[c] / 4000 - p) < 5 * np.sqrt(p * (1 - p) / 4000) + 1e-9
    # no move without negative overlap
    a = sa.copy()
    b = sa.copy()
    _, n = O.houdayer_single(L, a, b, 8, 0, 0)
    assert n == 0 and np.array_equal(a, sa)


# ----------------------------------------------------------------------------- PT and ER

def test_pt_acceptance_is_min_one_exp_delta():
    """Exchange acceptance equals min{1, exp((b_k - b_{k+1})(E_k - E_{k+1}))}:
    the empirical rate over many counters matches it, so forward/backward
    rates stand in the Boltzmann ratio (detailed balance)."""
    beta = np.array([2.0, 1.5])
    # the colder clone holding the lower energy is the favoured order, so
    # exchanging it costs exp((b_k - b_{k+1})(E_k - E_{k+1})) < 1
    for Ek, Ek1, expect in ((-10.0, -9.0, np.exp(-0.5)), (-9.0, -10.0, 1.0),
                            (-13.0, -10.0, np.exp(-1.5))):
        acc = 0
        n = 20000
        for emcs in range(n):
            perm = np.array([0, 1], np.int32)
            E = np.array([Ek, Ek1])
            a, _ = O.pt_round(beta, perm, E, 77, 0, emcs)
            acc += a[0]
            if a[0]:
                assert list(perm) == [1, 0] and list(E) == [Ek1, Ek]
            else:
                assert list(perm) == [0, 1]
        sd = np.sqrt(expect * (1 - expect) / n) + 1e-12
        assert abs(acc / n - expect) < 5 * sd


def test_pt_phases_touch_disjoint_pairs():
    beta = 1.0 / np.linspace(0.2, 1.6, 8)
    perm = np.arange(8, dtype=np.int32)
    E = np.zeros(8)            # delta = 0 -> always accepted
    acc, _ = O.pt_round(beta, perm, E, 1, 0, 0)
    # even phase swaps (0,1)(2,3)(4,5)(6,7), odd phase then swaps (1,2)(3,4)(5,6)
    assert list(acc) == [1, 1, 1, 1, 1, 1, 1, 0]
    assert list(perm) == [1, 3, 0, 5, 2, 7, 4, 6]


def test_er_fifo_and_round_trips():
    """Sec. 3 ER: the clone at T_max is exchanged with the oldest reservoir
    clone, so each clone spends exactly n_res EMCS (n_res * 240 = 960
    sweeps) in the reservoir; round trips count T_max -> T_min -> T_max."""
    nT, nres = 3, 4
    perm = np.arange(nT + nres, dtype=np.int32)
    age = np.arange(nres, dtype=np.uint32)
    rt = np.zeros(nT + nres, np.uint8)
    trips = np.zeros(1, np.int64)
    entered = {}
    for t in range(40):
        out_clone = int(perm[nT - 1])
        O.er_step(nT, nres, perm, age, rt, trips)
        entered[out_clone] = t
        inj = int(perm[nT - 1])
        if inj in entered and t >= 8:
            assert t - entered[inj] == nres
    assert sorted(age) == list(range(nres))
    # scripted round trip: inject, visit T_min, come back
    perm = np.arange(nT + nres, dtype=np.int32)
    age = np.arange(nres, dtype=np.uint32)
    rt = np.zeros(nT + nres, np.uint8)
    trips = np.zeros(1, np.int64)
    O.er_step(nT, nres, perm, age, rt, trips)
    c = int(perm[nT - 1])
    assert rt[c] == 1
    rt[c] |= 2                  # as the PT bookkeeping does at T_min
    O.er_step(nT, nres, perm, age, rt, trips)
    assert trips[0] == 1 and rt[c] == 0


def test_pair_observables_closed_forms():
    L, V = 4, 64
    J = _rand_J(L, 61)
    sa = W.random_spins(V, 62)
    q, ql, S = O.pair_observables(L, J, sa, sa.copy(), 0.5)
    assert q == 1.0 and ql == 1.0
    assert S == pytest.approx(O.energy(L, J, sa) / (3 * V))
    q, ql, S = O.pair_observables(L, J, sa, (-sa).astype(np.int8), 0.5)
    assert q == -1.0 and ql == 1.0


# ----------------------------------------------------------------------------- temperature grid

@pytest.mark.parametrize("n_temps,t_min,t_max", [(12, 0.2, 1.6), (16, 0.2, 1.6), (24, 0.2, 1.6),
                                                 (32, 0.2, 1.6), (24, 0.42, 1.8), (60, 0.2, 2.0),
                                                 (7, 0.35, 2.0), (2, 0.5, 1.5)])
def test_temperature_grid_is_uniform_with_both_ends(n_temps, t_min, t_max):
    """App. A.2: N_T temperatures uniformly spaced between T_min and T_max,
    both included.  Checked against exact rational arithmetic on the two
    binary64 end points: T_0 is T_min exactly, every T_k lies within the
    rounding error of four IEEE operations (3 ulps of T_max) of
    T_min + k (T_max - T_min)/(N_T - 1), so T_{N_T-1} is T_max and the
    spacing is uniform to that precision; 1/T_k is the correctly rounded
    reciprocal."""
    T, beta = O.temperatures(n_temps, t_min, t_max)
    a, b = Fraction(t_min), Fraction(t_max)
    assert T[0] == t_min
    for k in range(n_temps):
        exact = a + k * (b - a) / (n_temps - 1)
        assert abs(Fraction(float(T[k])) - exact) <= 3 * Fraction(np.spacing(t_max))
        assert Fraction(float(beta[k])) == Fraction(float(1 / Fraction(float(T[k]))))
    assert abs(T[-1] - t_max) <= 3 * np.spacing(t_max)
    step = (t_max - t_min) / (n_temps - 1)
    np.testing.assert_allclose(np.diff(T), step, rtol=0, atol=8 * np.spacing(t_max))


# ----------------------------------------------------------------------------- the chain vs exact enumeration

_SPINS_2x2x2 = np.where((np.arange(256)[:, None] >> np.arange(8)) & 1, -1, 1).astype(np.float64)


def exact_pair_moments(J, T):
    """<q^2> and <q^4> of two independent replicas on 2x2x2 (Eqs. (2)-(3)):
    q(a, b) = (1/V) sum_i s^a_i s^b_i summed over all 65536 pair states with
    the product of the two Boltzmann weights from the enumeration."""
    _, P = O.enumerate_l2(J, T, want_probs=True)
    Q = _SPINS_2x2x2 @ _SPINS_2x2x2.T / 8.0
    q2 = np.array([p @ (Q ** 2) @ p for p in P])
    q4 = np.array([p @ (Q ** 4) @ p for p in P])
    return q2, q4


def test_pair_moments_enumeration_agrees_with_the_enumerator():
    """The pair-state sum for <q^2> equals the enumerator's
    (1/V^2) sum_ij <s_i s_j>^2: two different routes to the same number."""
    J = _rand_J(2, 19, grid=False)
    q2, q4 = exact_pair_moments(J, T_GRID)
    np.testing.assert_allclose(q2, O.enumerate_l2(J, T_GRID)[:, 1], rtol=1e-12)
    assert np.all(q4 <= q2 + 1e-15) and np.all(q4 >= q2 ** 2 - 1e-15)   # q^2 <= 1; Jensen


# accumulator columns of the chain (per temperature): (name, obs column,
# divisor per measurement: 4 groups or 2 pairs)
_CHAIN_COLS = (("e", 1, 4), ("e2", 2, 4), ("q", 3, 2), ("q2", 4, 2), ("ql", 5, 2), ("S", 6, 2),
               ("q4", 7, 2))


def _chain_vs_exact(rule, order, cluster, er_on, n_blocks=20, block=800, seed=5):
    L = 2
    J = _rand_J(2, seed, grid=True)
    T, _ = O.temperatures(4, 0.4, 1.6)
    smp = O.OracleSample(L, 4, 0.4, 1.6, seed=seed, J=J, n_groups=4, n_res=4,
                         sweeps_per_emcs=1, res_sweeps_per_emcs=3, cluster_mode=cluster,
                         er_on=er_on, rule=rule, order=order)
    smp.emcs(200)
    smp.obs[:] = 0
    means = []
    for b in range(n_blocks):
        before = smp.obs.copy()
        smp.emcs(block)
        d = smp.obs - before
        n = d[:, 0]
        means.append(np.stack([d[:, col] / (n * div) for _, col, div in _CHAIN_COLS], 1))
    means = np.array(means)
    est = means.mean(0)
    err = means.std(0, ddof=1) / np.sqrt(n_blocks)
    ex = O.enumerate_l2(J, T)
    q2, q4 = exact_pair_moments(J, T)
    # Z2 symmetry (Sec. 2): <q> = 0 for every sample
    exact = np.stack([ex[:, 0], ex[:, 4], np.zeros(len(T)), q2, ex[:, 2], ex[:, 3], q4], 1)
    z = np.abs(est - exact) / np.maximum(err, 1e-9)
    return z, smp


@pytest.mark.parametrize("rule,order,cluster,er_on", [
    (O.RULE_METROPOLIS, O.ORDER_CHECKERBOARD, O.CLUSTER_ACU, True),
    (O.RULE_HEATBATH, O.ORDER_CHECKERBOARD, O.CLUSTER_ACU, True),
    (O.RULE_METROPOLIS, O.ORDER_LEXICOGRAPHIC, O.CLUSTER_OFF, False),
    (O.RULE_METROPOLIS, O.ORDER_CHECKERBOARD, O.CLUSTER_SINGLE, True),
    (O.RULE_MICSA, O.ORDER_CHECKERBOARD, O.CLUSTER_ACU, True),
])
def test_pthr_chain_reproduces_exact_averages_on_2x2x2(rule, order, cluster, er_on):
    """The full EMCS (sweeps, cluster move, PT, ER) samples the Boltzmann
    weight at every temperature: every accumulator -- <e>, <e^2>, <q>,
    <q^2>, <q_l>, <S>, <q^4> -- agrees with exact enumeration (<q> = 0 by
    symmetry) within 5 standard errors (20 blocks)."""
    z, smp = _chain_vs_exact(rule, order, cluster, er_on)
    assert np.all(z < 5.0), dict(zip([c[0] for c in _CHAIN_COLS], z.T))
    assert smp.pt_accepted.sum() > 0
    if er_on:
        assert smp.round_trips.sum() > 0
