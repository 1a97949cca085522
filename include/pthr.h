/*
 * pthr.h -- C ABI of the GB300 (sm_103a) PTHR hot path.
 *
 * PTHR (arXiv 2605.25872) is Parallel Tempering with all-cluster Houdayer
 * moves and an entropic Reservoir, applied to the 3D Edwards-Anderson Ising
 * spin glass with Gaussian couplings and periodic boundaries (Sec. 2,
 * Eq. (1)).  One elementary Monte Carlo step (EMCS, Sec. 3) is
 *   (i)   local sweeps of every clone at its temperature,     pthr_sweep
 *   (ii)  the all-cluster update (ACU) of replica pairs, T<1, pthr_houdayer
 *   (iii) the parallel-tempering (PT) exchange,               pthr_swap
 *   (iv)  the entropic-reservoir (ER) exchange,               pthr_swap
 * followed by a measurement,                                  pthr_observables.
 *
 * Conventions shared by every entry point:
 *  - Plain pointers and sizes only.  "device" pointers are CUDA device (or
 *    managed) memory of the current device; "host" pointers are CPU memory.
 *  - The library allocates no device memory of its own: the caller allocates
 *    one device workspace of pthr_required_bytes() bytes and keeps it alive
 *    until pthr_destroy().  The library never frees it.  Each sub-buffer is
 *    followed by a 256-byte guard block (pthr_check_canaries).
 *  - Every call is asynchronous on the CUDA stream given at creation (or by
 *    pthr_set_stream) and returns as soon as its kernels are enqueued.
 *    Errors found on the host (bad arguments) return PTHR_E_INVAL at once;
 *    CUDA launch errors return PTHR_E_CUDA; errors found on the device (a
 *    bounded loop that hit its cap) are latched in a device status word and
 *    returned by the next pthr_poll().
 *  - Calls on one handle are not thread-safe; different handles are
 *    independent.  pthr_last_error() describes the last failure.
 *  - Every call that enqueues GPU work opens an NVTX range named after
 *    itself (no cost unless a profiler is attached).
 *
 * Geometry: site i = x + L*(y + L*z), 0 <= x,y,z < L, L even.  Couplings
 * J[s][mu][i] (mu = 0,1,2 for x,y,z) belong to the bond (i, i + e_mu) of
 * sample s.  Spins are +1/-1.  Temperatures T_k = t_min + k (t_max - t_min)
 * / (n_temps - 1), k = 0..n_temps-1 (App. A.2).  Replica groups g =
 * 0..n_replicas-1; the Houdayer pairs are (0,1), (2,3), ...  Each group owns
 * n_temps + n_res storage lattices ("clones"); a permutation maps positions
 * (temperature indices 0..n_temps-1, then reservoir slots) to clones.
 * The local lattice index of clone c of group g is g*(n_temps+n_res) + c.
 */
#ifndef PTHR_H
#define PTHR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define PTHR_API __attribute__((visibility("default")))
#else
#define PTHR_API
#endif

#define PTHR_MAX_L 24        /* largest supported linear size (shared-memory bound) */
#define PTHR_NOBS 8          /* observable accumulators per (sample, temperature)   */

typedef struct pthr_batch pthr_batch;   /* opaque handle; owns no device memory */

typedef enum {
    PTHR_OK = 0,
    PTHR_E_INVAL = 1,        /* invalid argument or configuration                  */
    PTHR_E_NOMEM = 2,        /* workspace smaller than pthr_required_bytes()       */
    PTHR_E_CUDA = 3,         /* a CUDA runtime call or launch failed               */
    PTHR_E_NOCONVERGE = 4,   /* a bounded device loop hit its iteration cap        */
    PTHR_E_TIMEOUT = 5,      /* pthr_poll() timed out before the stream drained    */
    PTHR_E_STATE = 6,        /* call not valid now (e.g. during stream capture)    */
    PTHR_E_BOUNDS = 7        /* a device-side range check failed (the work it
                                guarded was skipped, nothing was written)          */
} pthr_status;

/* Local update rules (Sec. 3 item i).  PTHR_MICSA: microcanonical
 * simulated annealing (App. A.1), one walker per (clone, 4-site group of the
 * checkerboard, colour pass), drawn from the canonical distribution of a
 * non-negative energy at the clone's temperature (E_w = -T ln u) when the
 * pass reaches its group; a spin flips when the walker holds more than its
 * Delta E, which is then taken from the walker. */
enum { PTHR_METROPOLIS = 0, PTHR_HEATBATH = 1, PTHR_MICSA = 2 };
enum { PTHR_CLUSTER_OFF = 0, PTHR_CLUSTER_ACU = 1, PTHR_CLUSTER_SINGLE = 2 };
enum { PTHR_SWAP_PT = 1, PTHR_SWAP_ER = 2 };
/* Spin storage in the workspace (the paper keeps spins as exact +-1; either
 * form is exact).  BYTES: one byte per site slot, the form the kernels work
 * on in shared memory.  BITS: one bit per site slot, 8x less device memory
 * (more resident samples per GB); the sweep and cluster kernels expand a
 * lattice to bytes when they stage it and pack it again on write-back.
 * Results are identical in both layouts. */
enum { PTHR_SPINS_BYTES = 0, PTHR_SPINS_BITS = 1 };
enum { PTHR_OBS_MEASURE = 1, PTHR_OBS_READ_HOST = 2, PTHR_OBS_READ_DEVICE = 4, PTHR_OBS_RESET = 8,
       PTHR_OBS_CHAOS = 16 };

/* Workspace sub-buffers (pthr_buffer_info).  Layouts:
 *  J      float    [S][3][V]        couplings, natural site order
 *  SPINS  uint8    [S][n_lat][lat_bytes] internal packed layout (use
 *                                   pthr_export_spins / pthr_import_spins);
 *                                   lat_bytes = pthr_lattice_storage_bytes(L,
 *                                   spin_layout): one byte per site slot
 *                                   (PTHR_SPINS_BYTES) or one bit
 *                                   (PTHR_SPINS_BITS, 8x smaller)
 *  ENERGY double   [S][n_lat]       energy of every clone (Eq. (1)), FP64
 *  PERM   int32    [S][n_replicas][n_temps+n_res] position -> clone
 *  AGE    uint32   [S][n_replicas][max(n_res,1)] EMCS spent in the reservoir
 *  RT     uint8    [S][n_lat]       round-trip state (bit0 armed, bit1 saw T_min)
 *  TRIPS  int64    [S][n_replicas]  completed round trips T_max->T_min->T_max
 *  PTACC  int64    [S][n_replicas][n_temps] accepted exchanges of pair (k,k+1)
 *  FLIPS  uint64   [S][n_lat]       accepted local moves
 *  OBS    double   [S][n_temps][PTHR_NOBS] accumulators: count, sum e, sum e^2
 *                                   (over groups), sum q, sum q^2, sum q_l,
 *                                   sum S, sum q^4 (over pairs)
 *  EMCS   uint32   [S]              EMCS counter of each sample
 *  SEEDS  uint64   [S]              Philox key of each sample
 *  ACTIVE uint8    [S]              0 = slot idle (skipped by every kernel)
 *  STATUS uint32   [4]              device status word (error bits)
 *  CSTAT  int64    [S][n_pairs][n_temps][4] cluster statistics of the last
 *                                   cluster move: clusters, largest, second
 *                                   largest, sites flipped
 *  PRETH  uint32   [S]              reservoir pre-thermalisation sweeps done since
 *                                   the sample was created or reset (the sweep
 *                                   index of the next pre-thermalisation sweep)
 *  CHAOS  double   [S][n_temps][2]  temperature-chaos accumulators: count and
 *                                   sum over pairs of q^2 between the clone of
 *                                   group 2p at T_0 and the clone of group 2p+1
 *                                   at T_k (Sec. 5, chaotic parameter)
 *  TABLES                           read-only, written at creation: double
 *                                   T_k [n_temps], 1/T_k [n_temps],
 *                                   (V-2n)/V [V+1], (3V-2n)/(3V) [3V+1], then
 *                                   float -2 log2(e)/T_k [n_temps]; each value
 *                                   one IEEE-rounded division
 */
enum {
    PTHR_BUF_J = 0, PTHR_BUF_SPINS, PTHR_BUF_ENERGY, PTHR_BUF_PERM, PTHR_BUF_AGE,
    PTHR_BUF_RT, PTHR_BUF_TRIPS, PTHR_BUF_PTACC, PTHR_BUF_FLIPS, PTHR_BUF_OBS,
    PTHR_BUF_EMCS, PTHR_BUF_SEEDS, PTHR_BUF_ACTIVE, PTHR_BUF_STATUS, PTHR_BUF_CSTAT,
    PTHR_BUF_CHAOS, PTHR_BUF_PRETH, PTHR_BUF_TABLES, PTHR_NBUF
};

typedef struct {
    int L;                    /* linear size: even, 2 <= L <= PTHR_MAX_L            */
    int n_samples;            /* S >= 1 independent disorder samples                 */
    int n_temps;              /* N_T >= 2 PT temperatures                            */
    int n_replicas;           /* N_r >= 1 replica groups (even for cluster moves)    */
    int n_res;                /* reservoir clones per group (paper: 4; 0 = none)     */
    int sweeps_per_emcs;      /* local sweeps of PT clones per EMCS (paper: 10)      */
    int res_sweeps_per_emcs;  /* sweeps of each reservoir clone per EMCS (960/4)     */
    int acu_interval;         /* cluster move every acu_interval EMCS (>= 1)         */
    int update_rule;          /* PTHR_METROPOLIS, PTHR_HEATBATH or PTHR_MICSA        */
    int cluster_mode;         /* PTHR_CLUSTER_OFF / _ACU / _SINGLE                   */
    int er_on;                /* 1: entropic reservoir step on                       */
    int spin_layout;          /* PTHR_SPINS_BYTES (0) or PTHR_SPINS_BITS             */
    double t_min, t_max;      /* temperature grid ends (t_max > t_min > 0)           */
    double acu_t_below;       /* cluster moves only at T_k < acu_t_below (paper: 1)  */
    uint64_t seed;            /* sample s uses Philox key seed + s unless seeds given */
} pthr_config;

/* Kernel shape knobs (autotuner).  0 = library default. */
typedef struct {
    int pt_lattices_per_block;    /* lattices of one sample per sweep block, PT      */
    int res_lattices_per_block;   /* same for reservoir clones                       */
    int sweep_threads;            /* threads per sweep block (multiple of the work)  */
    int cluster_threads;          /* threads per cluster-move block (<= 512)         */
    int cluster_iter_cap;         /* 0: automatic bound 4V+64 on every union-find
                                     loop; a small value exercises the bounded-loop
                                     error path (PTHR_E_NOCONVERGE, spins unchanged) */
} pthr_tuning;

/* Total workspace bytes for cfg (every sub-buffer 256-byte aligned).
 * Returns PTHR_E_INVAL for an invalid cfg.  Host-only; no CUDA call. */
PTHR_API pthr_status pthr_required_bytes(const pthr_config *cfg, size_t *bytes);

/* Offset and size in bytes of workspace sub-buffer `buffer` (PTHR_BUF_*).
 * Host-only; no CUDA call. */
PTHR_API pthr_status pthr_buffer_info(const pthr_config *cfg, int buffer, size_t *offset,
                                      size_t *bytes);

/* Bytes of one lattice in the byte spin layout (PTHR_SPINS_BYTES), the
 * form the kernels keep in shared memory. */
PTHR_API pthr_status pthr_lattice_bytes(int L, size_t *bytes);

/* Bytes of one lattice in the workspace for spin_layout (PTHR_SPINS_*):
 * pthr_lattice_bytes(L) for bytes, an eighth of it for bits.  PTHR_E_INVAL
 * for an invalid L or layout.  Host-only; no CUDA call. */
PTHR_API pthr_status pthr_lattice_storage_bytes(int L, int spin_layout, size_t *bytes);

/* Create a batch of cfg->n_samples samples in the caller-owned device
 * workspace (>= pthr_required_bytes bytes, 256-byte aligned).
 * couplings: host or device float [S][3][V] (copied), or NULL to draw them
 *            on the device from each sample's seed (Sec. 2: J ~ N(0,1);
 *            Box-Muller on Philox, rounded to multiples of 2^-18).
 * seeds:     host uint64 [S] Philox keys, or NULL for cfg->seed + s.
 * stream:    cudaStream_t (NULL = legacy default stream).
 * Initialises hot-start spins (Sec. 3: random), identity permutations,
 * reservoir ages 0..n_res-1, zero counters and every clone's energy.
 * On success *out receives the handle.  Asynchronous. */
PTHR_API pthr_status pthr_create_batch(const pthr_config *cfg, void *device_workspace,
                                       size_t workspace_bytes, const float *couplings,
                                       const uint64_t *seeds, void *stream, pthr_batch **out);

/* Release the handle (not the workspace).  Safe on NULL. */
PTHR_API void pthr_destroy(pthr_batch *b);

/* Change the stream used by later calls. */
PTHR_API pthr_status pthr_set_stream(pthr_batch *b, void *stream);

/* Set kernel shape knobs (NULL restores defaults).  Results do not depend on
 * them: every random number is keyed by (sample, lattice, site, step). */
PTHR_API pthr_status pthr_set_tuning(pthr_batch *b, const pthr_tuning *t);
PTHR_API pthr_status pthr_get_tuning(const pthr_batch *b, pthr_tuning *t);

/* Switch the local update rule (PTHR_METROPOLIS, PTHR_HEATBATH, PTHR_MICSA)
 * from the next sweep on.  The paper's PTHR* runs Metropolis for the early
 * bins and the MicSA walker (App. A.1) for the late ones.  Only at an EMCS
 * boundary (else PTHR_E_STATE); PTHR_E_INVAL for an unknown rule.  The sweep
 * draws of each rule follow their own counter streams from then on; the
 * batch's captured EMCS graph is rebuilt on the next graph replay.  A group
 * created earlier keeps the rule it was created with (create it again).
 * Host-only; no CUDA call besides releasing the old graph. */
PTHR_API pthr_status pthr_set_update_rule(pthr_batch *b, int rule);

/* Step (i) of the EMCS (Sec. 3; App. A.1): n_pt_sweeps full-lattice
 * checkerboard sweeps of every PT clone at its temperature and, at the same
 * time, n_res_sweeps sweeps of every reservoir clone at T_max, with the
 * configured update rule (Metropolis: flip iff Delta E <= 0 or
 * u < exp(-Delta E / T); heat bath: s = +1 iff u < 1/(1 + exp(-2 h / T))),
 * FP32 local fields, then every swept clone's energy in FP64.  Sweep
 * indices continue within the current EMCS.  n_* >= 0; (0, 0) only
 * recomputes energies. */
PTHR_API pthr_status pthr_sweep(pthr_batch *b, int n_pt_sweeps, int n_res_sweeps);

/* Step (ii) (Sec. 3, ACU): for each pair (2p, 2p+1) and each T_k <
 * acu_t_below, the two clones at T_k: site overlaps q_i, clusters =
 * connected components of {i ~ j : neighbours, q_i q_j > 0}, one random sign
 * per cluster applied to both clones (PTHR_CLUSTER_ACU), or one q = -1
 * cluster flipped (PTHR_CLUSTER_SINGLE), then both energies in FP64.  Runs
 * only on EMCS whose index is a multiple of acu_interval. */
PTHR_API pthr_status pthr_houdayer(pthr_batch *b);

/* Canonical cluster labels (step (ii) without the flip) of every replica pair
 * at every temperature: out_device int32 [S][n_replicas/2][n_temps][V]
 * receives, for each site, the smallest site index of its cluster (the
 * connected component of {i ~ j : neighbours, q_i q_j > 0}, Sec. 3).
 * Diagnostic entry point; the spins are not changed. */
PTHR_API pthr_status pthr_cluster_labels(pthr_batch *b, int32_t *out_device);

/* Steps (iii) and (iv), then the end of the EMCS: PTHR_SWAP_PT runs one PT
 * round per group (even pairs, then odd pairs; accept with
 * min{1, exp((1/T_k - 1/T_{k+1})(E_k - E_{k+1}))}); PTHR_SWAP_ER exchanges
 * the clone at T_max with the oldest reservoir clone (Sec. 3, ER).  Every
 * call increments the EMCS counter of each active sample, whatever flags. */
PTHR_API pthr_status pthr_swap(pthr_batch *b, int flags);

/* Observables (Sec. 2, Eqs. (2)-(5)).  PTHR_OBS_MEASURE adds the current
 * e = H/V, q, q^2, q_l, S = H/(3V) + (1 - q_l)/T and q^4 of every (sample,
 * temperature) to the OBS accumulators; PTHR_OBS_READ_HOST (host out) or
 * PTHR_OBS_READ_DEVICE (device out) copies the accumulators, double
 * [S][n_temps][PTHR_NOBS], into out (bytes must be >= that size; a host
 * read synchronises the stream); PTHR_OBS_RESET zeroes them afterwards.
 * PTHR_OBS_CHAOS (with MEASURE) also adds, for every T_k, q^2 between the
 * T_0 clone of group 2p and the T_k clone of group 2p+1 to the CHAOS buffer
 * (reset with the other accumulators). */
PTHR_API pthr_status pthr_observables(pthr_batch *b, int flags, void *out, size_t bytes);

/* n full EMCS: pthr_sweep(sweeps_per_emcs, er_on ? res_sweeps_per_emcs : 0),
 * pthr_houdayer (if a cluster mode is set), pthr_swap(PT | ER if er_on),
 * pthr_observables(MEASURE).  With use_graph = 1 one EMCS is captured into a
 * CUDA graph on first use and replayed. */
PTHR_API pthr_status pthr_emcs(pthr_batch *b, int n, int use_graph);

/* n_sweeps sweeps at T_max of every reservoir clone before EMCS 0 (Sec. 3:
 * the reservoir refreshes clones for 960 sweeps); uses EMCS counter word
 * 0xFFFFFFFF.  Only the samples in [first, first+count).  The sweep index
 * continues from the sample's PRETH counter, so two calls of n sweeps equal
 * one call of 2n (fresh random numbers, never a replay); the counter restarts
 * at creation and at pthr_reset_samples.  A sample whose counter would pass
 * 2^23 is skipped and pthr_poll() then returns PTHR_E_BOUNDS. */
PTHR_API pthr_status pthr_prethermalize_reservoir(pthr_batch *b, int first, int count,
                                                  int n_sweeps);

/* Wait up to timeout_ms (< 0: forever) for the stream to drain, then return
 * the latched device status (PTHR_E_NOCONVERGE if a device loop hit its cap,
 * PTHR_E_BOUNDS if a device range check failed), or PTHR_E_TIMEOUT if the
 * stream is still busy (the status word is then left for a later poll).
 * Clears the status word after reading it. */
PTHR_API pthr_status pthr_poll(pthr_batch *b, int timeout_ms);

/* Spins of every clone in natural order, int8 +1/-1, [S][n_lat][V], device
 * memory (out / in).  Import also recomputes every energy. */
PTHR_API pthr_status pthr_export_spins(pthr_batch *b, int8_t *out_device);
PTHR_API pthr_status pthr_import_spins(pthr_batch *b, const int8_t *in_device);

/* Serving: reinitialise samples [first, first+count) as new disorder
 * samples (couplings host/device [count][3][V] or NULL = from seeds; seeds
 * host [count], not NULL), EMCS counter 0, fresh spins, permutations, ages,
 * counters and accumulators, optional reservoir pre-thermalisation, and mark
 * them active.  Other samples are untouched (a request's result does not
 * depend on its slot or neighbours). */
PTHR_API pthr_status pthr_reset_samples(pthr_batch *b, int first, int count,
                                        const float *couplings, const uint64_t *seeds,
                                        int pretherm_sweeps);

/* Mark samples [first, first+count) active (1) or idle (0). */
PTHR_API pthr_status pthr_set_active(pthr_batch *b, int first, int count, int active);

/* Groups: several batches (for instance one per lattice size) advanced
 * together by one CUDA graph per EMCS (Sec. 3: the same EMCS for every
 * sample, whatever its size).  When the batches share an update rule, have
 * L in {4, 6, 8, 10, 12, 14, 16}, number at most 8 and set no
 * cluster_iter_cap, the graph holds four launches in all -- the sweep, the
 * cluster move, the swap and the measurement of every batch, each step one
 * kernel over the blocks of all batches; otherwise it holds each batch's own
 * EMCS on its own stream, forked from and joined to `stream`.
 * pthr_group_emcs replays the graph n times on `stream`, after the work
 * already queued on every member's own stream and before the work queued on
 * them later (events), so per-batch calls and group EMCS may be mixed.
 * Inside the caller's own capture of `stream` the four-launch form enqueues
 * its kernels (captured in order, no events); the per-batch-graph form then
 * returns PTHR_E_STATE without touching the capture.  The
 * batches must be at an EMCS boundary, must not be destroyed before the
 * group, and their idle slots cost no work.  Kernel shapes are fixed at
 * creation.  Results are those of stepping every batch alone. */
typedef struct pthr_group pthr_group;
PTHR_API pthr_status pthr_group_create(pthr_batch *const *batches, int n, void *stream,
                                       pthr_group **out);
PTHR_API pthr_status pthr_group_emcs(pthr_group *g, int n);
PTHR_API void pthr_group_destroy(pthr_group *g);
/* Kernel launches per EMCS in the group's graph (4 for the one-launch-per-
 * step form). */
PTHR_API pthr_status pthr_group_info(const pthr_group *g, int *launches_per_emcs);

/* Checkpoint: the workspace holds the whole state (counter-based random
 * numbers make resume exact), so a blob is the workspace plus a header.
 * pthr_save with blob == NULL returns the size in *bytes; otherwise blob
 * (host) receives it and the stream is synchronised.  pthr_load restores a
 * blob saved from a batch with the same configuration. */
PTHR_API pthr_status pthr_save(pthr_batch *b, void *blob, size_t *bytes);
PTHR_API pthr_status pthr_load(pthr_batch *b, const void *blob, size_t bytes);

/* Spin autocorrelation of the reservoir clones at T_max (Sec. 3, ER: the
 * residence of 960 sweeps is set by C(960) < 1e-3, with
 * C(tau) = (1/V) sum_i <s_i(t) s_i(t + tau)> from an equilibrium start at
 * T_max).  For the samples [first, first+count): the current configuration
 * of every reservoir clone is copied to the snapshot, then n_points times
 * sweeps_per_point reservoir sweeps at T_max are run (the
 * pre-thermalisation sweeps of pthr_prethermalize_reservoir, which continue
 * the sample's PRETH sweep index) and after the p-th block
 * out_device[s - first][p] (int64, device) receives
 *   sum over the sample's n_replicas * n_res reservoir clones and V sites of
 *   s_i(snapshot) s_i(now),
 * an exact integer: C(tau = (p+1) sweeps_per_point) = out / (n_replicas *
 * n_res * V) for that sample.  The reservoir clones keep the extra sweeps
 * (a stationary evolution at T_max).  snapshot_device: caller-owned device
 * scratch, 16-byte aligned, at least count * n_replicas * n_res *
 * pthr_lattice_storage_bytes(L, spin_layout) bytes (else PTHR_E_NOMEM); its contents are not
 * needed afterwards.  Needs n_res >= 1 and an EMCS boundary (PTHR_E_STATE).
 * Asynchronous. */
PTHR_API pthr_status pthr_reservoir_autocorrelation(pthr_batch *b, int first, int count, int n_points,
                                                    int sweeps_per_point, void *snapshot_device,
                                                    size_t snapshot_bytes, int64_t *out_device);

/* The same measurement as pthr_reservoir_autocorrelation, for callers that
 * cannot allocate device memory: a plugin inside a host program that owns
 * every device allocation through its own pool, a control loop that must
 * not wait on (or risk a failure of) the allocator part-way through a run,
 * or a language binding with no way to obtain device memory.  The paper has
 * no counterpart; this is an interface convenience only.
 * Instead of a caller-provided snapshot it uses a fixed 8 MiB device array
 * inside the library, which every GPU that loads the library keeps until
 * the process exits; it allocates nothing (no cudaMalloc or cudaFree, no
 * allocating library call).  The snapshot must fit in it: count *
 * n_replicas * n_res * pthr_lattice_storage_bytes(L, spin_layout) <= 8 MiB
 * (128 samples of the L = 16, 4 x 4 reservoir in the byte layout, 1024 in
 * the bit layout), else PTHR_E_NOMEM and nothing runs; split
 * larger batches into sample ranges.  The first call on a device looks up
 * the array's address on that device (the batch's device must be current,
 * else PTHR_E_INVAL); make that first call before any stream capture.
 * Every call reuses the same array: each call writes every snapshot word it
 * later reads, so nothing needs clearing between calls, but calls that
 * overlap on the GPU (other streams, other batches, other threads) race on
 * it and must be serialised by the caller.  Arguments, results and
 * asynchrony are those of pthr_reservoir_autocorrelation. */
PTHR_API pthr_status pthr_reservoir_autocorrelation_noalloc(pthr_batch *b, int first, int count, int n_points,
                                                            int sweeps_per_point, int64_t *out_device);

/* Guard check: every workspace sub-buffer is followed by a 256-byte guard
 * block written with a fixed pattern at creation (included in
 * pthr_required_bytes).  Synchronises the stream and compares every guard
 * block; returns PTHR_OK if all are intact, else PTHR_E_BOUNDS with
 * *bad_buffer (if not NULL) set to the PTHR_BUF_* index of the first
 * sub-buffer whose guard was overwritten (-1 when all are intact).  A
 * debugging aid for out-of-range writes; pthr_load restores the guards
 * from the blob. */
PTHR_API pthr_status pthr_check_canaries(pthr_batch *b, int *bad_buffer);

/* Description of the last error on this handle (never NULL). */
PTHR_API const char *pthr_last_error(const pthr_batch *b);

/* Library version string. */
PTHR_API const char *pthr_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PTHR_H */
