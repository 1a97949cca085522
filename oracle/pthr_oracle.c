/*
 * pthr_oracle.c -- plain FP64 CPU oracle for PTHR (Parallel Tempering with
 * all-cluster Houdayer moves and an entropic Reservoir) on the 3D
 * Edwards-Anderson Ising spin glass with Gaussian couplings.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the tests, the smoke check and the CPU baseline leg of
 * the benchmark use it.  It shares no code, header, table or constant
 * generator with the CUDA library; the only thing both sides agree on is the
 * written specification (Philox4x32-10 counter layout, lattice geometry,
 * update rules), and each side implements it independently.
 *
 * Everything here is written for clarity, not speed: one Philox call per
 * random number, natural site order, FP64 arithmetic throughout (the
 * couplings are FP32 values promoted to FP64).
 *
 * Passages followed (arXiv 2605.25872):
 *   Sec. 2, Eq. (1)      Hamiltonian H = -sum_<ij> J_ij s_i s_j, periodic
 *                        simple-cubic lattice, V = L^3, J ~ N(0,1).
 *   Sec. 2, Eqs. (2)-(4) site overlap q_i, overlap q, link overlap q_l.
 *   Sec. 2, Eq. (5)      SDY observable S = H/(3V) + (1 - q_l)/T.
 *   Sec. 3, items i-iv   one EMCS = local sweeps, ACU, PT step, ER step.
 *   Sec. 3 (ACU)         clusters = connected components of {i~j : q_i q_j>0},
 *                        one random sign per cluster applied to both replicas,
 *                        restricted to T < 1.
 *   Sec. 3 (PT)          neighbouring temperatures exchange with a rule that
 *                        satisfies detailed balance.
 *   Sec. 3 (ER)          reservoir clones at T_max, 960/4 sweeps per EMCS, the
 *                        oldest reservoir clone is exchanged with the clone at
 *                        T_max.
 *   Sec. 5 (round trips) T_max -> T_min -> T_max excursions of a clone.
 *   App. A.1             Delta E = 2 s_i sum_j J_ij s_j, Metropolis
 *                        acceptance min{1, exp(-Delta E / T)}; MicSA: a spin
 *                        flips when its walker holds at least Delta E, which
 *                        is then taken from the walker.
 * Readings where the paper is silent are stated at the point of use below.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, written from Salmon, Moraes, Dror and Shaw, "Parallel     */
/* random numbers: as easy as 1, 2, 3" (SC'11): ten rounds of two 32x32->64 */
/* multiplications with the Weyl key schedule.                              */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Stream tags (fourth counter word, low byte). */
enum { TAG_INIT = 0, TAG_SWEEP = 1, TAG_ACU = 2, TAG_PT = 3, TAG_SINGLE = 4,
       TAG_COUPLING = 5, TAG_SWEEP_LEX = 6, TAG_MICSA = 7 };

/* One 32-bit Philox word: key = the sample seed, counter (c0, c1, c2, c3). */
static uint32_t rng_word(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                         uint32_t c3, int word)
{
    uint32_t ctr[4] = { c0, c1, c2, c3 };
    uint32_t key[2] = { (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32) };
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[word];
}

/* Uniform in [0,1) on 24 bits; exact in both FP32 and FP64. */
static double uniform24(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }

/* ------------------------------------------------------------------------ */
/* Lattice geometry (Sec. 2): site i = x + L*(y + L*z), periodic.           */
/* Couplings J[mu*V + i] belong to the bond (i, i + e_mu), mu = x, y, z.    */
/* ------------------------------------------------------------------------ */
static int site_of(int L, int x, int y, int z)
{
    x = (x % L + L) % L; y = (y % L + L) % L; z = (z % L + L) % L;
    return x + L * (y + L * z);
}

/* The six neighbours of site i in the order +x, -x, +y, -y, +z, -z, and the
 * coupling index of the bond to each of them. */
static void neighbours(int L, int i, int nb[6], int bond[6])
{
    int V = L * L * L;
    int x = i % L, y = (i / L) % L, z = i / (L * L);
    nb[0] = site_of(L, x + 1, y, z); bond[0] = 0 * V + i;
    nb[1] = site_of(L, x - 1, y, z); bond[1] = 0 * V + nb[1];
    nb[2] = site_of(L, x, y + 1, z); bond[2] = 1 * V + i;
    nb[3] = site_of(L, x, y - 1, z); bond[3] = 1 * V + nb[3];
    nb[4] = site_of(L, x, y, z + 1); bond[4] = 2 * V + i;
    nb[5] = site_of(L, x, y, z - 1); bond[5] = 2 * V + nb[5];
}

/* Local field h_i = sum_{j in nbrs(i)} J_ij s_j (App. A.1, Delta E = 2 s_i h_i). */
static double local_field(int L, const double *J, const int8_t *s, int i)
{
    int nb[6], bond[6];
    neighbours(L, i, nb, bond);
    double h = 0.0;
    for (int k = 0; k < 6; k++) h += J[bond[k]] * (double)s[nb[k]];
    return h;
}

/* Eq. (1): H = -sum over the 3V forward bonds of J_b s_i s_j. */
double orc_energy(int L, const double *J, const int8_t *s)
{
    int V = L * L * L;
    double H = 0.0;
    for (int i = 0; i < V; i++) {
        int nb[6], bond[6];
        neighbours(L, i, nb, bond);
        H -= J[bond[0]] * s[i] * s[nb[0]];
        H -= J[bond[2]] * s[i] * s[nb[2]];
        H -= J[bond[4]] * s[i] * s[nb[4]];
    }
    return H;
}

/* ------------------------------------------------------------------------ */
/* a1: couplings and initial spins.                                          */
/* ------------------------------------------------------------------------ */

/* Gaussian couplings from the sample seed (Sec. 2: J ~ N(0,1), quenched).
 * Reading: Box-Muller on two 24-bit uniforms, u1 in (0,1], u2 in [0,1); bond
 * b uses Philox call b>>2, words (0,1) for b&3 in {0,1} and (2,3) for
 * {2,3}; even b takes r cos(theta), odd b takes r sin(theta).  The normal
 * is rounded to the nearest multiple of 2^-18 (|J| <= 5.77 because
 * u1 >= 2^-24), so J is exact in FP32 and every partial sum of six
 * couplings is exact in FP32 as well. */
void orc_couplings_from_seed(int L, uint64_t seed, double *J)
{
    const double two_pi = 6.283185307179586476925286766559;
    int V = L * L * L;
    for (int b = 0; b < 3 * V; b++) {
        int pair = (b & 3) >> 1;           /* 0 -> words 0,1 ; 1 -> words 2,3 */
        uint32_t w1 = rng_word(seed, (uint32_t)(b >> 2), 0, 0, TAG_COUPLING, 2 * pair);
        uint32_t w2 = rng_word(seed, (uint32_t)(b >> 2), 0, 0, TAG_COUPLING, 2 * pair + 1);
        double u1 = (double)((w1 >> 8) + 1u) * (1.0 / 16777216.0);
        double u2 = (double)(w2 >> 8) * (1.0 / 16777216.0);
        double r = sqrt(-2.0 * log(u1));
        double z = (b & 1) ? r * sin(two_pi * u2) : r * cos(two_pi * u2);
        J[b] = nearbyint(z * 262144.0) / 262144.0;
    }
}

/* Random initial spins (hot start): site i of local lattice `lat` takes
 * word i&3 of the call (i>>2, lat, 0, TAG_INIT); top bit set -> -1. */
void orc_init_spins(int L, uint64_t seed, int lat, int8_t *s)
{
    int V = L * L * L;
    for (int i = 0; i < V; i++) {
        uint32_t w = rng_word(seed, (uint32_t)(i >> 2), (uint32_t)lat, 0, TAG_INIT, i & 3);
        s[i] = (w >> 31) ? -1 : 1;
    }
}

/* ------------------------------------------------------------------------ */
/* a2/a3: one full-lattice sweep at inverse temperature beta.               */
/* ------------------------------------------------------------------------ */
enum { ORDER_CHECKERBOARD = 0, ORDER_LEXICOGRAPHIC = 1 };
enum { RULE_METROPOLIS = 0, RULE_HEATBATH = 1, RULE_MICSA = 2 };

/* The random word that the checkerboard sweep uses at site i.
 * Sites of colour c = (x+y+z)&1 in row r = y + L z sit at x = 2m + p; the
 * word is (r*W + (m>>2), lat, emcs, TAG_SWEEP | c<<8 | sweep<<9)[m & 3] with
 * W = ceil((L/2)/4).  The lexicographic sweep (the paper's order) uses
 * (i>>2, lat, emcs, TAG_SWEEP_LEX | sweep<<9)[i & 3]. */
static uint32_t sweep_word(int L, uint64_t seed, int lat, uint32_t emcs,
                           uint32_t sweep, int order, int i)
{
    if (order == ORDER_LEXICOGRAPHIC)
        return rng_word(seed, (uint32_t)(i >> 2), (uint32_t)lat, emcs,
                        TAG_SWEEP_LEX | (sweep << 9), i & 3);
    int x = i % L, y = (i / L) % L, z = i / (L * L);
    int c = (x + y + z) & 1;
    int r = y + L * z;
    int m = x >> 1;
    int W = (L / 2 + 3) / 4;
    return rng_word(seed, (uint32_t)(r * W + (m >> 2)), (uint32_t)lat, emcs,
                    TAG_SWEEP | ((uint32_t)c << 8) | (sweep << 9), m & 3);
}

/*
 * One sweep of lattice s (Sec. 3 item i).  Checkerboard order updates all
 * even sites, then all odd sites; with even L no two sites of one colour are
 * neighbours, so both orders leave the Boltzmann weight stationary.
 *
 * Metropolis (App. A.1): Delta E = 2 s_i h_i; flip if Delta E <= 0, else flip
 * iff u < exp(-beta Delta E).  Heat bath: s_i = +1 iff
 * u < 1 / (1 + exp(-2 beta h_i)).
 *
 * Near ties: a decision is logged when |u - p| < tie_eps, or when
 * |beta Delta E| < tie_eps (Metropolis).  With field_err_bound = 1 the
 * margin also includes a bound on the error of an FP32 evaluation of the
 * field in the order +x,-x,+y,-y,+z,-z, of beta rounded to FP32 and of an
 * FP32 exponential (used for couplings off the 2^-18 grid).
 * Returns the number of spins that changed; *dE accumulates the energy
 * change of every accepted move.
 */
long orc_sweep(int L, const double *J, int8_t *s, double beta, uint64_t seed,
               int lat, uint32_t emcs, uint32_t sweep, int order, int rule,
               double tie_eps, int field_err_bound, int32_t *tie_sites,
               int max_ties, int *n_ties, double *dE)
{
    int V = L * L * L;
    long accepted = 0;
    const double u32 = 5.9604644775390625e-08;   /* 2^-24 */
    for (int pass = 0; pass < (order == ORDER_CHECKERBOARD ? 2 : 1); pass++) {
        for (int i = 0; i < V; i++) {
            if (order == ORDER_CHECKERBOARD) {
                int x = i % L, y = (i / L) % L, z = i / (L * L);
                if (((x + y + z) & 1) != pass) continue;
            }
            double h = local_field(L, J, s, i);
            double u = uniform24(sweep_word(L, seed, lat, emcs, sweep, order, i));
            double p, margin_extra = 0.0;
            int flip;
            int tie = 0;
            if (field_err_bound) {
                int nb[6], bond[6];
                neighbours(L, i, nb, bond);
                double part = 0.0, err = 0.0;
                for (int k = 0; k < 6; k++) {
                    part += J[bond[k]] * s[nb[k]];
                    if (k > 0) err += fabs(part) * u32;
                }
                margin_extra = 2.0 * beta * 2.0 * err + 8.0 * u32 * (1.0 + fabs(2.0 * beta * h));
            }
            if (rule == RULE_METROPOLIS) {
                double dEi = 2.0 * s[i] * h;
                if (fabs(beta * dEi) < tie_eps + margin_extra) tie = 1;
                if (dEi <= 0.0) {
                    flip = 1;
                } else {
                    p = exp(-beta * dEi);
                    flip = (u < p);
                    if (fabs(u - p) < tie_eps + p * margin_extra) tie = 1;
                }
            } else {
                p = 1.0 / (1.0 + exp(-2.0 * beta * h));
                int snew = (u < p) ? 1 : -1;
                flip = (snew != s[i]);
                if (fabs(u - p) < tie_eps + p * (1.0 - p) * margin_extra) tie = 1;
            }
            if (tie && n_ties) {
                if (*n_ties < max_ties && tie_sites) tie_sites[*n_ties] = i;
                (*n_ties)++;
            }
            if (flip) {
                if (dE) *dE += 2.0 * s[i] * h;
                s[i] = (int8_t)(-s[i]);
                accepted++;
            }
        }
    }
    return accepted;
}

/* ------------------------------------------------------------------------ */
/* a2 variant: microcanonical simulated annealing (MicSA; Sec. 3 item i,     */
/* App. A.1: a walker holds an energy; a spin flips when the walker has at   */
/* least Delta E, which is then taken from the walker).                      */
/* ------------------------------------------------------------------------ */

/*
 * One walker serving n sites in order.  Reading of the walker's initial
 * energy and refresh (the paper defers them to its MicSA reference): the
 * walker is drawn afresh from the canonical distribution of a non-negative
 * energy at temperature T, E_w = -T ln u, each time it starts its sites, so
 * that (spins, walker) keep the weight exp(-(H + E_w)/T).  Site k flips iff
 * Delta E_k < E_w - D, D = sum of the Delta E already taken by earlier
 * flips of this walker, i.e. iff X_k = D + Delta E_k <= 0 or
 * u < exp(-beta X_k); a flip adds Delta E_k to D.  u is the walker's
 * uniform.  tie[k] (if not NULL) is set for a near-tie decision:
 * |u - exp(-beta X)| < tie_eps, 0 < |beta X| < tie_eps, or an offset X
 * that FP32 cannot hold exactly (X = 0 is exact and flips on both sides).
 * flip[k] receives 0/1; returns D.
 */
double orc_micsa_walker(int n, const double *dE, double beta, double u, int *flip,
                        double tie_eps, int *tie)
{
    double D = 0.0;
    for (int k = 0; k < n; k++) {
        double X = D + dE[k];
        int f;
        int t = (X != 0.0 && fabs(beta * X) < tie_eps) || (double)(float)X != X;
        if (X <= 0.0) {
            f = 1;
        } else {
            double p = exp(-beta * X);
            f = (u < p);
            if (fabs(u - p) < tie_eps) t = 1;
        }
        if (tie) tie[k] = t;
        flip[k] = f;
        if (f) D += dE[k];
    }
    return D;
}

/*
 * One MicSA sweep of lattice s in checkerboard order.  Sites of colour c in
 * row r = y + L z sit at x = 2m + p; the walker of group (r, j) serves the
 * sites m = 4j .. 4j+3 (those that exist) in ascending m, and a new walker
 * starts at every group of every colour pass.  Its uniform is word e & 3 of
 * the call (r W + j, (e >> 2) | kind << 24, emcs, TAG_MICSA | c << 8 |
 * sweep << 9), where e is the lattice's position within its kind (PT
 * clones: group * N_T + temperature index; reservoir: group * N_res + slot)
 * and kind = 1 for reservoir clones.  Within a group the sites are not
 * neighbours, so every Delta E of the group is taken before any of its
 * flips.  Returns the number of flips; *dE accumulates the energy change;
 * *n_tie_decisions counts near-tie decisions and tie_sites receives every
 * site a near tie may have changed (*n_tie_sites of them).
 */
long orc_sweep_micsa(int L, const double *J, int8_t *s, double beta, uint64_t seed, int e, int kind,
                     uint32_t emcs, uint32_t sweep, double tie_eps, int32_t *tie_sites, int max_ties,
                     int *n_tie_sites, int *n_tie_decisions, double *dE_total)
{
    int W = (L / 2 + 3) / 4, Lh = L / 2;
    long accepted = 0;
    for (int c = 0; c < 2; c++) {
        for (int r = 0; r < L * L; r++) {
            int y = r % L, z = r / L, p = (c + y + z) & 1;
            for (int j = 0; j < W; j++) {
                int sites[4], n = 0;
                double dE[4];
                int flip[4], tie[4];
                for (int k = 0; k < 4; k++) {
                    int m = 4 * j + k;
                    if (m >= Lh) break;
                    int i = (2 * m + p) + L * r;
                    sites[n] = i;
                    dE[n] = 2.0 * s[i] * local_field(L, J, s, i);
                    n++;
                }
                uint32_t w = rng_word(seed, (uint32_t)(r * W + j), ((uint32_t)e >> 2) | ((uint32_t)kind << 24),
                                      emcs, TAG_MICSA | ((uint32_t)c << 8) | (sweep << 9), e & 3);
                orc_micsa_walker(n, dE, beta, uniform24(w), flip, tie_eps, tie);
                /* a near tie at site k may change k and, through the walker,
                 * every later site of the group: all of them are logged */
                int tied = 0;
                for (int k = 0; k < n; k++) {
                    if (tie[k] && n_tie_decisions) (*n_tie_decisions)++;
                    tied |= tie[k];
                    if (tied && n_tie_sites) {
                        if (*n_tie_sites < max_ties && tie_sites) tie_sites[*n_tie_sites] = sites[k];
                        (*n_tie_sites)++;
                    }
                    if (flip[k]) {
                        if (dE_total) *dE_total += dE[k];
                        s[sites[k]] = (int8_t)(-s[sites[k]]);
                        accepted++;
                    }
                }
            }
        }
    }
    return accepted;
}

/* ------------------------------------------------------------------------ */
/* a5: overlap and connected components (Sec. 3, ACU step 1 and 2).          */
/* ------------------------------------------------------------------------ */

/* Clusters: i ~ j iff i, j are nearest neighbours and q_i q_j > 0, with
 * q_i = s^a_i s^b_i (Eq. (2)).  Breadth-first search from every unlabelled
 * site in ascending order, so each cluster's label is its smallest site
 * index.  Returns the number of clusters. */
int orc_cc_labels(int L, const int8_t *sa, const int8_t *sb, int32_t *lab)
{
    int V = L * L * L;
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)V);
    int nclus = 0;
    for (int i = 0; i < V; i++) lab[i] = -1;
    for (int i = 0; i < V; i++) {
        if (lab[i] >= 0) continue;
        nclus++;
        int head = 0, tail = 0;
        lab[i] = i;
        queue[tail++] = i;
        while (head < tail) {
            int v = queue[head++];
            int qv = sa[v] * sb[v];
            int nb[6], bond[6];
            neighbours(L, v, nb, bond);
            for (int k = 0; k < 6; k++) {
                int w = nb[k];
                if (lab[w] < 0 && sa[w] * sb[w] == qv) {
                    lab[w] = i;
                    queue[tail++] = w;
                }
            }
        }
    }
    free(queue);
    return nclus;
}

/* a6: the all-cluster update (Sec. 3, ACU step 3).  Every cluster c draws
 * eta_c = +-1 with probability 1/2 -- reading: word 0 of the call
 * (label, pair_id, emcs, TAG_ACU), eta = -1 iff its top bit is set -- and
 * both replicas' spins in c are multiplied by eta_c.  Returns the number of
 * clusters; lab (if not NULL) receives the labels. */
int orc_acu(int L, int8_t *sa, int8_t *sb, uint64_t seed, uint32_t pair_id,
            uint32_t emcs, int32_t *lab_out)
{
    int V = L * L * L;
    int32_t *lab = (int32_t *)malloc(sizeof(int32_t) * (size_t)V);
    int nclus = orc_cc_labels(L, sa, sb, lab);
    for (int i = 0; i < V; i++) {
        uint32_t w = rng_word(seed, (uint32_t)lab[i], pair_id, emcs, TAG_ACU, 0);
        int eta = (w >> 31) ? -1 : 1;
        sa[i] = (int8_t)(sa[i] * eta);
        sb[i] = (int8_t)(sb[i] * eta);
    }
    if (lab_out) memcpy(lab_out, lab, sizeof(int32_t) * (size_t)V);
    free(lab);
    return nclus;
}

/* Original single-cluster Houdayer move (Sec. 3, the second difference from
 * Houdayer's proposal): one cluster of negative overlap is traced from a seed
 * and flipped with probability one.  Reading: u from word 0 of
 * (0, pair_id, emcs, TAG_SINGLE); the seed is the floor(u * n)-th site with
 * q_i = -1 in ascending site order, n = number of such sites; no move when
 * n = 0.  Returns the size of the flipped cluster. */
int orc_houdayer_single(int L, int8_t *sa, int8_t *sb, uint64_t seed,
                        uint32_t pair_id, uint32_t emcs, int32_t *lab_out)
{
    int V = L * L * L;
    int32_t *lab = (int32_t *)malloc(sizeof(int32_t) * (size_t)V);
    orc_cc_labels(L, sa, sb, lab);
    int n = 0;
    for (int i = 0; i < V; i++) n += (sa[i] * sb[i] < 0);
    int flipped = 0;
    if (n > 0) {
        double u = uniform24(rng_word(seed, 0, pair_id, emcs, TAG_SINGLE, 0));
        int target = (int)floor(u * (double)n);
        int seed_site = -1, seen = 0;
        for (int i = 0; i < V; i++) {
            if (sa[i] * sb[i] < 0) {
                if (seen == target) { seed_site = i; break; }
                seen++;
            }
        }
        int c = lab[seed_site];
        for (int i = 0; i < V; i++) {
            if (lab[i] == c) { sa[i] = (int8_t)-sa[i]; sb[i] = (int8_t)-sb[i]; flipped++; }
        }
    }
    if (lab_out) memcpy(lab_out, lab, sizeof(int32_t) * (size_t)V);
    free(lab);
    return flipped;
}

/* ------------------------------------------------------------------------ */
/* a7: one PT round for one replica group (Sec. 3, PT step).                 */
/* ------------------------------------------------------------------------ */

/* perm[k] = storage slot of the clone at temperature k, E[k] its energy.
 * Reading: the exchange of the clones at T_k < T_{k+1} is accepted with
 * probability min{1, exp((beta_k - beta_{k+1})(E_k - E_{k+1}))} (the
 * Metropolis rule of the Hukushima-Nemoto exchange, which the paper cites
 * but does not print); an even phase (k even) then an odd phase (k odd);
 * pair (k, k+1) of phase ph in group g uses word 0 of
 * (k, 2g + ph, emcs, TAG_PT).  Temperatures are exchanged, spins are not.
 * accepted[k] counts accepted exchanges of the pair (k, k+1). */
void orc_pt_round(int n_temps, const double *beta, int32_t *perm, double *E,
                  uint64_t seed, int group, uint32_t emcs, int64_t *accepted,
                  double tie_eps, int *n_ties)
{
    for (int ph = 0; ph < 2; ph++) {
        for (int k = ph; k + 1 < n_temps; k += 2) {
            double delta = (beta[k] - beta[k + 1]) * (E[k] - E[k + 1]);
            double u = uniform24(rng_word(seed, (uint32_t)k, (uint32_t)(2 * group + ph),
                                          emcs, TAG_PT, 0));
            int acc;
            if (delta >= 0.0) {
                acc = 1;
                if (n_ties && fabs(delta) < tie_eps) (*n_ties)++;
            } else {
                double p = exp(delta);
                acc = (u < p);
                if (n_ties && fabs(u - p) < tie_eps) (*n_ties)++;
            }
            if (acc) {
                int32_t t = perm[k]; perm[k] = perm[k + 1]; perm[k + 1] = t;
                double e = E[k]; E[k] = E[k + 1]; E[k + 1] = e;
                if (accepted) accepted[k]++;
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* a8: one entropic-reservoir step for one replica group (Sec. 3, ER step).  */
/* ------------------------------------------------------------------------ */

/* perm[0 .. n_temps-1] are the PT positions, perm[n_temps .. n_temps+n_res-1]
 * the reservoir slots, age[r] the EMCS that reservoir slot r has spent in the
 * reservoir.  The clone at T_max (position n_temps-1) is exchanged with the
 * reservoir clone that has been there longest (reading: ties -> lowest slot);
 * the exchange needs no acceptance test because both sit at T_max.  The slot
 * that receives the outgoing clone restarts at age 0, every other slot ages
 * by one.  Round trips (Sec. 5): a clone is armed when it is injected from
 * the reservoir, marked when it reaches T_min, and counts one round trip
 * when, armed and marked, it leaves T_max for the reservoir.
 * rt_state[slot] bit0 = armed, bit1 = has visited T_min. */
void orc_er_step(int n_temps, int n_res, int32_t *perm, double *E_pos,
                 uint32_t *age, uint8_t *rt_state, int64_t *round_trips)
{
    int best = 0;
    for (int r = 1; r < n_res; r++) if (age[r] > age[best]) best = r;
    int pos_hot = n_temps - 1, pos_res = n_temps + best;
    int out_clone = perm[pos_hot], in_clone = perm[pos_res];
    if (rt_state) {
        if ((rt_state[out_clone] & 3u) == 3u && round_trips) (*round_trips)++;
        rt_state[out_clone] = 0;
        rt_state[in_clone] = 1;
    }
    perm[pos_hot] = in_clone;
    perm[pos_res] = out_clone;
    if (E_pos) { double e = E_pos[pos_hot]; E_pos[pos_hot] = E_pos[pos_res]; E_pos[pos_res] = e; }
    for (int r = 0; r < n_res; r++) age[r] = (r == best) ? 0u : age[r] + 1u;
}

/* ------------------------------------------------------------------------ */
/* a9: observables of one replica pair at one temperature (Eqs. (2)-(5)).    */
/* ------------------------------------------------------------------------ */

/* out[0] = q, out[1] = q_l, out[2] = S computed with H_a. */
void orc_pair_observables(int L, const double *J, const int8_t *sa, const int8_t *sb,
                          double T, double *out)
{
    int V = L * L * L;
    double q = 0.0, ql = 0.0;
    for (int i = 0; i < V; i++) {
        int nb[6], bond[6];
        neighbours(L, i, nb, bond);
        double qi = (double)(sa[i] * sb[i]);
        q += qi;
        ql += qi * (double)(sa[nb[0]] * sb[nb[0]]);
        ql += qi * (double)(sa[nb[2]] * sb[nb[2]]);
        ql += qi * (double)(sa[nb[4]] * sb[nb[4]]);
    }
    q /= (double)V;
    ql /= 3.0 * (double)V;
    double Ha = orc_energy(L, J, sa);
    out[0] = q;
    out[1] = ql;
    out[2] = Ha / (3.0 * V) + (1.0 - ql) / T;
}

/* ------------------------------------------------------------------------ */
/* Exact enumeration on 2x2x2 (V = 8, 256 states) for the pins.              */
/* ------------------------------------------------------------------------ */

/* For each temperature T[t]: out[t*5 + 0..4] = <e>, <q^2>, <q_l>, <S>, <e^2>
 * with e = H/V, <q^2> = (1/V^2) sum_ij <s_i s_j>^2,
 * <q_l> = (1/3V) sum_bonds <s_i s_j>^2 (two independent replicas), and
 * <S> = <H>/(3V) + (1 - <q_l>)/T.  probs (if not NULL) receives the
 * Boltzmann probability of every state (bit k of the state index set means
 * s_k = -1), n_temps x 256. */
int orc_enumerate_l2(const double *J, int n_temps, const double *T, double *out,
                     double *probs)
{
    const int L = 2, V = 8, NS = 256;
    double H[256];
    int8_t s[8];
    for (int st = 0; st < NS; st++) {
        for (int k = 0; k < V; k++) s[k] = ((st >> k) & 1) ? -1 : 1;
        H[st] = orc_energy(L, J, s);
    }
    double Hmin = H[0];
    for (int st = 1; st < NS; st++) if (H[st] < Hmin) Hmin = H[st];
    for (int t = 0; t < n_temps; t++) {
        double beta = 1.0 / T[t];
        double Z = 0.0, eH = 0.0, eH2 = 0.0, C[8][8];
        memset(C, 0, sizeof(C));
        for (int st = 0; st < NS; st++) {
            double w = exp(-beta * (H[st] - Hmin));
            Z += w;
            eH += w * H[st];
            eH2 += w * H[st] * H[st];
            for (int a = 0; a < V; a++)
                for (int b = 0; b < V; b++) {
                    int sa = ((st >> a) & 1) ? -1 : 1, sb = ((st >> b) & 1) ? -1 : 1;
                    C[a][b] += w * sa * sb;
                }
        }
        eH /= Z; eH2 /= Z;
        double q2 = 0.0;
        for (int a = 0; a < V; a++)
            for (int b = 0; b < V; b++) { C[a][b] /= Z; }
        for (int a = 0; a < V; a++)
            for (int b = 0; b < V; b++) q2 += C[a][b] * C[a][b];
        q2 /= (double)(V * V);
        double ql = 0.0;
        for (int i = 0; i < V; i++) {
            int nb[6], bond[6];
            neighbours(L, i, nb, bond);
            ql += C[i][nb[0]] * C[i][nb[0]] + C[i][nb[2]] * C[i][nb[2]] + C[i][nb[4]] * C[i][nb[4]];
        }
        ql /= 3.0 * V;
        out[t * 5 + 0] = eH / V;
        out[t * 5 + 1] = q2;
        out[t * 5 + 2] = ql;
        out[t * 5 + 3] = eH / (3.0 * V) + (1.0 - ql) / T[t];
        out[t * 5 + 4] = eH2 / ((double)V * V);
        if (probs)
            for (int st = 0; st < NS; st++) probs[t * NS + st] = exp(-beta * (H[st] - Hmin)) / Z;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* One EMCS of one sample (Sec. 3): sweeps, ACU, PT, ER, measurement.        */
/* ------------------------------------------------------------------------ */

typedef struct {
    int L, n_temps, n_groups, n_res;
    int sweeps_per_emcs;      /* local sweeps of the PT clones (paper: 10)   */
    int res_sweeps_per_emcs;  /* sweeps of each reservoir clone (paper: 240) */
    int cluster_mode;         /* 0 off, 1 ACU, 2 single-cluster Houdayer     */
    int er_on;                /* entropic reservoir on/off                   */
    int rule;                 /* RULE_METROPOLIS / RULE_HEATBATH             */
    int order;                /* ORDER_CHECKERBOARD / ORDER_LEXICOGRAPHIC    */
    double acu_t_below;       /* cluster moves only for T_k < this (1.0)     */
    double tie_eps;
} orc_cfg;

/* State of one sample.  Storage lattice `lat` = g*(n_temps+n_res) + slot
 * holds spins[lat*V ..]; perm[g*(n_temps+n_res) + pos] is the slot at
 * position pos (pos < n_temps: temperature index, else reservoir slot);
 * E_lat[lat] its energy; age[g*n_res + r]; rt_state[lat]; counters. */
typedef struct {
    int8_t *spins;
    int32_t *perm;
    double *E_lat;
    uint32_t *age;
    uint8_t *rt_state;
    int64_t *round_trips;     /* [n_groups]                      */
    int64_t *pt_accepted;     /* [n_groups * n_temps]            */
    int64_t *flips;           /* [n_lat] accepted local moves    */
    int64_t *n_ties;          /* [2] near ties: local, PT        */
    double *obs;              /* [n_temps * 8] accumulators      */
} orc_state;

/* beta_k = 1 / T_k with T_k = t_min + k (t_max - t_min) / (n_temps - 1)
 * (App. A.2: uniformly spaced, both ends included). */
void orc_temperatures(int n_temps, double t_min, double t_max, double *T, double *beta)
{
    for (int k = 0; k < n_temps; k++) {
        double t = (n_temps == 1) ? t_min
                                  : t_min + (double)k * (t_max - t_min) / (double)(n_temps - 1);
        T[k] = t;
        beta[k] = 1.0 / t;
    }
}

/* Observable accumulator layout per temperature (8 doubles):
 * [0] measurements, [1] sum e over groups, [2] sum e^2 over groups,
 * [3] sum q over pairs, [4] sum q^2, [5] sum q_l, [6] sum S, [7] sum q^4. */
void orc_measure(const orc_cfg *cfg, const double *J, const double *T, orc_state *st)
{
    int L = cfg->L, V = L * L * L;
    int nslot = cfg->n_temps + cfg->n_res;
    for (int k = 0; k < cfg->n_temps; k++) {
        double *o = st->obs + 8 * k;
        o[0] += 1.0;
        for (int g = 0; g < cfg->n_groups; g++) {
            int lat = g * nslot + st->perm[g * nslot + k];
            double e = st->E_lat[lat] / V;
            o[1] += e;
            o[2] += e * e;
        }
        for (int p = 0; p + 1 < cfg->n_groups; p += 2) {
            int la = p * nslot + st->perm[p * nslot + k];
            int lb = (p + 1) * nslot + st->perm[(p + 1) * nslot + k];
            double r[3];
            orc_pair_observables(L, J, st->spins + (size_t)la * V, st->spins + (size_t)lb * V,
                                 T[k], r);
            o[3] += r[0];
            o[4] += r[0] * r[0];
            o[5] += r[1];
            o[6] += r[2];
            o[7] += r[0] * r[0] * r[0] * r[0];
        }
    }
}

/* One EMCS (Sec. 3 items i-iv, in the paper's order).  The sweep counter
 * word of every lattice restarts at 0 in each EMCS; the EMCS index is the
 * third counter word. */
void orc_emcs(const orc_cfg *cfg, const double *J, const double *T, const double *beta,
              uint64_t seed, uint32_t emcs, orc_state *st)
{
    int L = cfg->L, V = L * L * L;
    int nslot = cfg->n_temps + cfg->n_res;
    double beta_max = beta[cfg->n_temps - 1];
    int ties_local = 0, ties_pt = 0;

    /* (i) local sweeps of every PT clone at its temperature, and of every
     * reservoir clone at T_max (Sec. 3: the reservoir evolves while the PT
     * clones perform their EMCS). */
    for (int g = 0; g < cfg->n_groups; g++) {
        for (int pos = 0; pos < nslot; pos++) {
            int in_res = pos >= cfg->n_temps;
            if (in_res && !cfg->er_on) continue;
            int lat = g * nslot + st->perm[g * nslot + pos];
            double b = in_res ? beta_max : beta[pos];
            int nsw = in_res ? cfg->res_sweeps_per_emcs : cfg->sweeps_per_emcs;
            int e = in_res ? g * cfg->n_res + (pos - cfg->n_temps) : g * cfg->n_temps + pos;
            for (int sw = 0; sw < nsw; sw++) {
                double dE = 0.0;
                if (cfg->rule == RULE_MICSA)
                    st->flips[lat] += orc_sweep_micsa(L, J, st->spins + (size_t)lat * V, b, seed, e, in_res,
                                                      emcs, (uint32_t)sw, cfg->tie_eps, NULL, 0, NULL,
                                                      &ties_local, &dE);
                else
                    st->flips[lat] += orc_sweep(L, J, st->spins + (size_t)lat * V, b, seed, lat,
                                                emcs, (uint32_t)sw, cfg->order, cfg->rule,
                                                cfg->tie_eps, 0, NULL, 0, &ties_local, &dE);
            }
        }
    }

    /* (ii) cluster move on the pairs (0,1), (2,3), ... at every T_k < 1. */
    if (cfg->cluster_mode != 0) {
        for (int p = 0; p + 1 < cfg->n_groups; p += 2) {
            for (int k = 0; k < cfg->n_temps; k++) {
                if (!(T[k] < cfg->acu_t_below)) continue;
                int la = p * nslot + st->perm[p * nslot + k];
                int lb = (p + 1) * nslot + st->perm[(p + 1) * nslot + k];
                uint32_t pair_id = (uint32_t)((p / 2) * cfg->n_temps + k);
                if (cfg->cluster_mode == 1)
                    orc_acu(L, st->spins + (size_t)la * V, st->spins + (size_t)lb * V, seed,
                            pair_id, emcs, NULL);
                else
                    orc_houdayer_single(L, st->spins + (size_t)la * V,
                                        st->spins + (size_t)lb * V, seed, pair_id, emcs, NULL);
            }
        }
    }

    /* Energies of every clone, recomputed from scratch in FP64 (Eq. (1)). */
    int nlat = cfg->n_groups * nslot;
    for (int lat = 0; lat < nlat; lat++)
        st->E_lat[lat] = orc_energy(L, J, st->spins + (size_t)lat * V);

    /* (iii) PT step, independently for each replica group. */
    double *Epos = (double *)malloc(sizeof(double) * (size_t)nslot);
    for (int g = 0; g < cfg->n_groups; g++) {
        int32_t *perm = st->perm + g * nslot;
        for (int pos = 0; pos < nslot; pos++) Epos[pos] = st->E_lat[g * nslot + perm[pos]];
        orc_pt_round(cfg->n_temps, beta, perm, Epos, seed, g, emcs,
                     st->pt_accepted + (size_t)g * cfg->n_temps, cfg->tie_eps, &ties_pt);
        /* Round-trip bookkeeping: the clone now at T_min is marked. */
        if (st->rt_state) {
            uint8_t *rs = st->rt_state + g * nslot;
            if (rs[perm[0]] & 1u) rs[perm[0]] |= 2u;
        }
        /* (iv) ER step. */
        if (cfg->er_on)
            orc_er_step(cfg->n_temps, cfg->n_res, perm, NULL, st->age + g * cfg->n_res,
                        st->rt_state + g * nslot, st->round_trips + g);
    }
    free(Epos);
    if (st->n_ties) { st->n_ties[0] += ties_local; st->n_ties[1] += ties_pt; }

    /* Measurement after the ER step. */
    orc_measure(cfg, J, T, st);
}
