// capi.cu -- the extern "C" boundary declared in include/pthr.h: configuration
// checks, workspace layout, launch shapes, EMCS schedule, CUDA-graph replay,
// device-status polling and checkpoints.  Every entry point that enqueues
// GPU work opens an NVTX range named after itself (a no-op unless a
// profiler is attached), so traces show the C-ABI calls around the kernels.
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>
#include <thread>

#include <nvtx3/nvToolsExt.h>

#include "kernels.cuh"

using namespace pthr;

namespace {
// NVTX range for the lifetime of one C-ABI call
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
}  // namespace
#define PTHR_TRACE(name) const NvtxRange pthr_nvtx_range_(name)

struct pthr_batch {
    pthr_config cfg;
    Batch dev;
    cudaStream_t stream;
    pthr_tuning tuning;
    void *ws;
    size_t ws_bytes;
    int pt_sweep_off, res_sweep_off;   // sweep index within the current EMCS
    cudaGraph_t graph;
    cudaGraphExec_t graph_exec;
    int graph_ok;
    char err[512];
};

namespace {

thread_local char g_err[512] = "";

pthr_status fail(pthr_batch *b, pthr_status st, const char *fmt, ...) {
    char *dst = b ? b->err : g_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 512, fmt, ap);
    va_end(ap);
    return st;
}

pthr_status cuda_fail(pthr_batch *b, cudaError_t e, const char *what) {
    return fail(b, PTHR_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CUDA_TRY(b, call, what)                         \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail((b), e_, (what)); \
    } while (0)

int n_pairs(const pthr_config *c) { return c->n_replicas / 2; }
int n_slot(const pthr_config *c) { return c->n_temps + c->n_res; }
int n_lat(const pthr_config *c) { return c->n_replicas * n_slot(c); }

double host_temperature(const pthr_config *c, int k) {
    Batch t{};
    t.NT = c->n_temps;
    t.t_min = c->t_min;
    t.t_max = c->t_max;
    return temperature(t, k);
}

int count_acu(const pthr_config *c) {
    if (c->cluster_mode == PTHR_CLUSTER_OFF || c->n_replicas < 2) return 0;
    int n = 0;
    for (int k = 0; k < c->n_temps; ++k)
        if (host_temperature(c, k) < c->acu_t_below) n = k + 1;
    return n;
}

pthr_status check_config(const pthr_config *c) {
    if (!c) return fail(nullptr, PTHR_E_INVAL, "config is NULL");
    if (c->L < 2 || c->L > PTHR_MAX_L || (c->L & 1))
        return fail(nullptr, PTHR_E_INVAL, "L must be even, 2 <= L <= %d (got %d)", PTHR_MAX_L, c->L);
    if (c->n_samples < 1) return fail(nullptr, PTHR_E_INVAL, "n_samples must be >= 1");
    if (c->n_temps < 2) return fail(nullptr, PTHR_E_INVAL, "n_temps must be >= 2");
    if (c->n_replicas < 1 || c->n_replicas > 32)
        return fail(nullptr, PTHR_E_INVAL, "n_replicas must be in [1, 32]");
    if (c->n_res < 0) return fail(nullptr, PTHR_E_INVAL, "n_res must be >= 0");
    if (n_slot(c) > 256) return fail(nullptr, PTHR_E_INVAL, "n_temps + n_res must be <= 256");
    if (c->er_on && c->n_res < 1) return fail(nullptr, PTHR_E_INVAL, "er_on needs n_res >= 1");
    if (c->sweeps_per_emcs < 0 || c->sweeps_per_emcs >= (1 << 22) || c->res_sweeps_per_emcs < 0 ||
        c->res_sweeps_per_emcs >= (1 << 22))
        return fail(nullptr, PTHR_E_INVAL, "sweeps per EMCS must be in [0, 2^22)");
    if (c->acu_interval < 1) return fail(nullptr, PTHR_E_INVAL, "acu_interval must be >= 1");
    if (c->update_rule != PTHR_METROPOLIS && c->update_rule != PTHR_HEATBATH && c->update_rule != PTHR_MICSA)
        return fail(nullptr, PTHR_E_INVAL, "unknown update_rule %d", c->update_rule);
    if (c->cluster_mode < PTHR_CLUSTER_OFF || c->cluster_mode > PTHR_CLUSTER_SINGLE)
        return fail(nullptr, PTHR_E_INVAL, "unknown cluster_mode %d", c->cluster_mode);
    if (c->cluster_mode != PTHR_CLUSTER_OFF && (c->n_replicas < 2 || (c->n_replicas & 1)))
        return fail(nullptr, PTHR_E_INVAL, "cluster moves need an even n_replicas >= 2");
    if (!(c->t_min > 0.0) || !(c->t_max > c->t_min))
        return fail(nullptr, PTHR_E_INVAL, "need 0 < t_min < t_max");
    if (c->spin_layout != PTHR_SPINS_BYTES && c->spin_layout != PTHR_SPINS_BITS)
        return fail(nullptr, PTHR_E_INVAL, "unknown spin_layout %d", c->spin_layout);
    return PTHR_OK;
}

// Every sub-buffer starts on a 256-byte boundary and is followed by a
// 256-byte guard block filled with CANARY at creation; pthr_check_canaries
// finds any write that ran past the end of a sub-buffer.
constexpr size_t GUARD_BYTES = 256;
constexpr unsigned char CANARY = 0xC5;

struct Layout {
    size_t off[PTHR_NBUF];
    size_t len[PTHR_NBUF];
    size_t guard[PTHR_NBUF];   // offset of the guard block after each sub-buffer
    size_t total;
};

Layout make_layout(const pthr_config *c) {
    const size_t S = (size_t)c->n_samples, V = (size_t)c->L * c->L * c->L;
    const size_t NL = (size_t)n_lat(c), NR = (size_t)c->n_replicas, NT = (size_t)c->n_temps;
    const size_t NRES = (size_t)(c->n_res > 0 ? c->n_res : 1);
    const size_t NP = (size_t)(n_pairs(c) > 0 ? n_pairs(c) : 1);
    Layout l{};
    l.len[PTHR_BUF_J] = S * 3 * V * sizeof(float);
    l.len[PTHR_BUF_SPINS] = S * NL * (size_t)storage_words(c->L, c->spin_layout) * 4;
    l.len[PTHR_BUF_ENERGY] = S * NL * sizeof(double);
    l.len[PTHR_BUF_PERM] = S * NR * (size_t)n_slot(c) * sizeof(int32_t);
    l.len[PTHR_BUF_AGE] = S * NR * NRES * sizeof(uint32_t);
    l.len[PTHR_BUF_RT] = S * NL;
    l.len[PTHR_BUF_TRIPS] = S * NR * sizeof(long long);
    l.len[PTHR_BUF_PTACC] = S * NR * NT * sizeof(long long);
    l.len[PTHR_BUF_FLIPS] = S * NL * sizeof(unsigned long long);
    l.len[PTHR_BUF_OBS] = S * NT * PTHR_NOBS * sizeof(double);
    l.len[PTHR_BUF_EMCS] = S * sizeof(uint32_t);
    l.len[PTHR_BUF_SEEDS] = S * sizeof(unsigned long long);
    l.len[PTHR_BUF_ACTIVE] = S;
    l.len[PTHR_BUF_STATUS] = 4 * sizeof(uint32_t);
    l.len[PTHR_BUF_CSTAT] = S * NP * NT * 4 * sizeof(long long);
    l.len[PTHR_BUF_CHAOS] = S * NT * 2 * sizeof(double);
    l.len[PTHR_BUF_PRETH] = S * sizeof(uint32_t);
    l.len[PTHR_BUF_TABLES] = (2 * NT + 4 * V + 2) * sizeof(double) + NT * sizeof(float);
    size_t o = 0;
    for (int i = 0; i < PTHR_NBUF; ++i) {
        l.off[i] = o;
        o += (l.len[i] + 255) & ~(size_t)255;
        l.guard[i] = o;
        o += GUARD_BYTES;
    }
    l.total = o;
    return l;
}

// Kernel shapes.  Sweep: lattices per block K (PT / reservoir); Gt 4-site
// groups per lattice lane (divides G, <= 512); P lattice lanes of KT
// lattices each (KT one of the compiled variants); threads = P * Gt.
struct SweepShape { int K_pt, K_res, Gt, P, KT, threads, pt_tasks, res_tasks; };

int default_k(const pthr_config *c, int total_entries) {
    const size_t lb = (size_t)lattice_words(c->L) * 4;
    const size_t budget = 220 * 1024;
    long k = (long)((budget - 12 * lb) / lb);
    if (c->L >= 12 && k > 16) k = 16;   // from L = 12 up; two blocks per SM at L = 12
    if (k > sweep_max_k()) k = sweep_max_k();
    if (k < 1) k = 1;
    if (k > total_entries) k = total_entries;
    return (int)k;
}

// forced_kt > 0: lattices per thread fixed (the mixed-L group sweep compiles
// one value per lattice size); the lattices per block then follow from it.
SweepShape sweep_shape(const pthr_batch *b, int forced_kt = 0) {
    const pthr_config *c = &b->cfg;
    SweepShape sh{};
    const int npt = c->n_replicas * c->n_temps;
    const int nres = c->n_replicas * (c->n_res > 0 ? c->n_res : 1);
    sh.K_pt = b->tuning.pt_lattices_per_block > 0 ? b->tuning.pt_lattices_per_block : default_k(c, npt);
    sh.K_res = b->tuning.res_lattices_per_block > 0 ? b->tuning.res_lattices_per_block : default_k(c, nres);
    if (sh.K_pt > npt) sh.K_pt = npt;
    if (sh.K_res > nres) sh.K_res = nres;
    const int G = sweep_groups_for(c->L);
    int Gt = G;
    if (G > 512) {
        for (int d = 2; d <= G; ++d)
            if (G % d == 0 && G / d <= 512) { Gt = G / d; break; }
    }
    sh.Gt = Gt;
    int P0 = 512 / Gt;
    if (b->tuning.sweep_threads > 0) P0 = b->tuning.sweep_threads / Gt;
    if (P0 < 1) P0 = 1;
    int opts[16];
    const int nopt = sweep_kt_options(c->L, c->update_rule, opts);
    int Kmax = sh.K_pt > sh.K_res ? sh.K_pt : sh.K_res;
    if (P0 > Kmax) P0 = Kmax;
    const int need = (Kmax + P0 - 1) / P0;
    int KT = opts[nopt - 1];
    for (int i = 0; i < nopt; ++i)
        if (opts[i] >= need) { KT = opts[i]; break; }
    if (forced_kt > 0) KT = forced_kt;
    if (P0 * KT < Kmax) {            // largest variant too small: fewer lattices per block
        if (sh.K_pt > P0 * KT) sh.K_pt = P0 * KT;
        if (sh.K_res > P0 * KT) sh.K_res = P0 * KT;
        Kmax = sh.K_pt > sh.K_res ? sh.K_pt : sh.K_res;
    }
    sh.KT = KT;
    sh.P = (Kmax + KT - 1) / KT;
    sh.threads = sh.P * Gt;
    sh.pt_tasks = (npt + sh.K_pt - 1) / sh.K_pt;
    sh.res_tasks = (nres + sh.K_res - 1) / sh.K_res;
    return sh;
}

struct SweepLaunch { SweepArgs a; int blocks, threads, KT; size_t smem; };

// Arguments and shape of one sweep launch (blocks == 0: nothing to do).
pthr_status sweep_launch(pthr_batch *b, int n_pt, int n_res, int first, int count, int pretherm,
                         int forced_kt, SweepLaunch *out) {
    const pthr_config *c = &b->cfg;
    SweepShape sh = sweep_shape(b, forced_kt);
    SweepArgs a{};
    a.b = b->dev;
    a.n_pt_sweeps = n_pt;
    a.n_res_sweeps = n_res;
    a.pt_sweep_base = pretherm ? 0 : b->pt_sweep_off;
    a.res_sweep_base = pretherm ? 0 : b->res_sweep_off;
    a.K_pt = sh.K_pt;
    a.K_res = sh.K_res;
    a.pt_tasks = sh.pt_tasks;
    a.res_tasks = sh.res_tasks;
    a.do_pt = pretherm ? 0 : ((n_pt > 0 || n_res == 0) ? 1 : 0);
    a.do_res = (c->n_res > 0 && (n_res > 0 || n_pt == 0)) ? 1 : 0;
    a.sample_first = first;
    a.sample_count = count;
    a.emcs_override = pretherm;
    a.Gt = sh.Gt;
    out->a = a;
    out->blocks = count * ((a.do_res ? sh.res_tasks : 0) + (a.do_pt ? sh.pt_tasks : 0));
    out->threads = sh.threads;
    out->KT = sh.KT;
    out->smem = sweep_smem_bytes_for(c->L, sh.K_pt > sh.K_res ? sh.K_pt : sh.K_res);
    if (out->smem > 220 * 1024)
        return fail(b, PTHR_E_INVAL, "sweep block needs %zu bytes of shared memory; lower the lattices per block",
                    out->smem);
    return PTHR_OK;
}

pthr_status do_sweep(pthr_batch *b, int n_pt, int n_res, int first, int count, int pretherm) {
    SweepLaunch sl{};
    pthr_status st = sweep_launch(b, n_pt, n_res, first, count, pretherm, 0, &sl);
    if (st != PTHR_OK) return st;
    if (sl.blocks == 0) return PTHR_OK;
    CUDA_TRY(b, launch_sweep(sl.a, sl.blocks, sl.threads, sl.KT, b->stream), "sweep launch");
    if (pretherm)   // the next pre-thermalisation sweeps continue the index
        CUDA_TRY(b, launch_advance_pretherm(b->dev, first, count, n_res, b->stream), "pretherm counter");
    return PTHR_OK;
}

// Threads per cluster-move block: about eight sites per thread, 128..512.
int default_cluster_threads(int L) {
    const int V = L * L * L;
    int t = ((V / 8 + 31) / 32) * 32;
    return t < 128 ? 128 : (t > 512 ? 512 : t);
}

int cluster_threads_of(const pthr_batch *b) {
    int threads = b->tuning.cluster_threads > 0 ? b->tuning.cluster_threads : default_cluster_threads(b->cfg.L);
    const int V = b->cfg.L * b->cfg.L * b->cfg.L;
    if (threads > ((V + 31) / 32) * 32) threads = ((V + 31) / 32) * 32;
    if (threads < 32) threads = 32;
    return (threads / 32) * 32;
}

pthr_status do_cluster(pthr_batch *b, int label_only, int32_t *labels) {
    if (b->dev.n_acu == 0 && !label_only) return PTHR_OK;
    ClusterArgs a{};
    a.b = b->dev;
    if (label_only) {   // label every temperature
        a.b.n_acu = b->cfg.n_temps;
        if (b->dev.NPAIR == 0) return fail(b, PTHR_E_INVAL, "no replica pairs");
    }
    a.sample_first = 0;
    a.sample_count = b->cfg.n_samples;
    a.label_only = label_only;
    a.labels_out = labels;
    a.iter_cap = b->tuning.cluster_iter_cap;
    int threads = b->tuning.cluster_threads > 0 ? b->tuning.cluster_threads : default_cluster_threads(b->cfg.L);
    const int V = b->cfg.L * b->cfg.L * b->cfg.L;
    if (threads > ((V + 31) / 32) * 32) threads = ((V + 31) / 32) * 32;
    if (threads < 32) threads = 32;
    threads = (threads / 32) * 32;
    if (cluster_smem_bytes_for(b->cfg.L) > 200 * 1024)
        return fail(b, PTHR_E_INVAL, "cluster block does not fit in shared memory");
    CUDA_TRY(b, launch_cluster(a, threads, b->stream), "cluster launch");
    return PTHR_OK;
}

pthr_status one_emcs(pthr_batch *b) {
    const pthr_config *c = &b->cfg;
    pthr_status st = do_sweep(b, c->sweeps_per_emcs, c->er_on ? c->res_sweeps_per_emcs : 0, 0,
                              c->n_samples, 0);
    if (st != PTHR_OK) return st;
    if (c->cluster_mode != PTHR_CLUSTER_OFF) {
        st = do_cluster(b, 0, nullptr);
        if (st != PTHR_OK) return st;
    }
    CUDA_TRY(b, launch_swap(b->dev, PTHR_SWAP_PT | (c->er_on ? PTHR_SWAP_ER : 0), 0, c->n_samples,
                            b->stream), "swap launch");
    CUDA_TRY(b, launch_measure(b->dev, 0, c->n_samples, 0, b->stream), "measure launch");
    return PTHR_OK;
}

bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return false;
    return cs != cudaStreamCaptureStatusNone;
}

}  // namespace

extern "C" {

PTHR_API const char *pthr_version(void) { return "pthr-gb300 0.1 (sm_103a)"; }

PTHR_API pthr_status pthr_required_bytes(const pthr_config *cfg, size_t *bytes) {
    pthr_status st = check_config(cfg);
    if (st != PTHR_OK) return st;
    if (!bytes) return fail(nullptr, PTHR_E_INVAL, "bytes is NULL");
    *bytes = make_layout(cfg).total;
    return PTHR_OK;
}

PTHR_API pthr_status pthr_buffer_info(const pthr_config *cfg, int buffer, size_t *offset, size_t *bytes) {
    pthr_status st = check_config(cfg);
    if (st != PTHR_OK) return st;
    if (buffer < 0 || buffer >= PTHR_NBUF || !offset || !bytes)
        return fail(nullptr, PTHR_E_INVAL, "bad buffer id or NULL output");
    Layout l = make_layout(cfg);
    *offset = l.off[buffer];
    *bytes = l.len[buffer];
    return PTHR_OK;
}

PTHR_API pthr_status pthr_lattice_bytes(int L, size_t *bytes) {
    if (L < 2 || L > PTHR_MAX_L || (L & 1) || !bytes) return fail(nullptr, PTHR_E_INVAL, "bad L");
    *bytes = (size_t)lattice_words(L) * 4;
    return PTHR_OK;
}

PTHR_API pthr_status pthr_lattice_storage_bytes(int L, int spin_layout, size_t *bytes) {
    if (L < 2 || L > PTHR_MAX_L || (L & 1) || !bytes) return fail(nullptr, PTHR_E_INVAL, "bad L");
    if (spin_layout != PTHR_SPINS_BYTES && spin_layout != PTHR_SPINS_BITS)
        return fail(nullptr, PTHR_E_INVAL, "unknown spin_layout %d", spin_layout);
    *bytes = (size_t)storage_words(L, spin_layout) * 4;
    return PTHR_OK;
}

PTHR_API pthr_status pthr_create_batch(const pthr_config *cfg, void *device_workspace, size_t workspace_bytes,
                                       const float *couplings, const uint64_t *seeds, void *stream,
                                       pthr_batch **out) {
    PTHR_TRACE("pthr_create_batch");
    pthr_status st = check_config(cfg);
    if (st != PTHR_OK) return st;
    if (!out) return fail(nullptr, PTHR_E_INVAL, "out is NULL");
    *out = nullptr;
    if (!device_workspace) return fail(nullptr, PTHR_E_INVAL, "workspace is NULL");
    if (((uintptr_t)device_workspace) & 255) return fail(nullptr, PTHR_E_INVAL, "workspace must be 256-byte aligned");
    Layout l = make_layout(cfg);
    if (workspace_bytes < l.total)
        return fail(nullptr, PTHR_E_NOMEM, "workspace has %zu bytes, needs %zu", workspace_bytes, l.total);
    pthr_batch *b = new pthr_batch();
    memset(b->err, 0, sizeof(b->err));
    b->cfg = *cfg;
    b->stream = (cudaStream_t)stream;
    b->ws = device_workspace;
    b->ws_bytes = workspace_bytes;
    unsigned char *base = (unsigned char *)device_workspace;
    Batch &d = b->dev;
    d.J = (float *)(base + l.off[PTHR_BUF_J]);
    d.spins = (uint32_t *)(base + l.off[PTHR_BUF_SPINS]);
    d.E = (double *)(base + l.off[PTHR_BUF_ENERGY]);
    d.perm = (int32_t *)(base + l.off[PTHR_BUF_PERM]);
    d.age = (uint32_t *)(base + l.off[PTHR_BUF_AGE]);
    d.rt = (uint8_t *)(base + l.off[PTHR_BUF_RT]);
    d.trips = (long long *)(base + l.off[PTHR_BUF_TRIPS]);
    d.ptacc = (long long *)(base + l.off[PTHR_BUF_PTACC]);
    d.flips = (unsigned long long *)(base + l.off[PTHR_BUF_FLIPS]);
    d.obs = (double *)(base + l.off[PTHR_BUF_OBS]);
    d.emcs = (uint32_t *)(base + l.off[PTHR_BUF_EMCS]);
    d.seeds = (unsigned long long *)(base + l.off[PTHR_BUF_SEEDS]);
    d.active = (uint8_t *)(base + l.off[PTHR_BUF_ACTIVE]);
    d.status = (uint32_t *)(base + l.off[PTHR_BUF_STATUS]);
    d.cstat = (long long *)(base + l.off[PTHR_BUF_CSTAT]);
    d.chaos = (double *)(base + l.off[PTHR_BUF_CHAOS]);
    d.preth = (uint32_t *)(base + l.off[PTHR_BUF_PRETH]);
    double *tab = (double *)(base + l.off[PTHR_BUF_TABLES]);
    const int NTt = cfg->n_temps, Vt = cfg->L * cfg->L * cfg->L;
    d.tabT = tab;
    d.tabBeta = tab + NTt;
    d.tabQ = tab + 2 * NTt;
    d.tabQl = tab + 2 * NTt + Vt + 1;
    d.tabTb = (const float *)(tab + 2 * NTt + 4 * Vt + 2);
    d.S = cfg->n_samples;
    d.L = cfg->L;
    d.NT = cfg->n_temps;
    d.NR = cfg->n_replicas;
    d.NRES = cfg->n_res;
    d.NSLOT = n_slot(cfg);
    d.NLAT = n_lat(cfg);
    d.NPAIR = n_pairs(cfg);
    d.lat_words = storage_words(cfg->L, cfg->spin_layout);
    d.bits = cfg->spin_layout == PTHR_SPINS_BITS ? 1 : 0;
    d.rule = cfg->update_rule;
    d.cluster_mode = cfg->cluster_mode;
    d.acu_interval = cfg->acu_interval;
    d.n_acu = count_acu(cfg);
    d.t_min = cfg->t_min;
    d.t_max = cfg->t_max;

    // seeds (host), status word
    unsigned long long *hs = new unsigned long long[cfg->n_samples];
    for (int s = 0; s < cfg->n_samples; ++s) hs[s] = seeds ? seeds[s] : cfg->seed + (unsigned long long)s;
    cudaError_t e = cudaMemcpyAsync(d.seeds, hs, sizeof(unsigned long long) * cfg->n_samples,
                                    cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);   // hs is pageable and freed below
    delete[] hs;
    if (e == cudaSuccess) e = cudaMemsetAsync(d.status, 0, 16, b->stream);
    for (int i = 0; i < PTHR_NBUF && e == cudaSuccess; ++i)
        e = cudaMemsetAsync(base + l.guard[i], CANARY, GUARD_BYTES, b->stream);
    if (e == cudaSuccess) {
        // tables: one IEEE-rounded division each, the same bits as the
        // per-use divisions they replace
        std::vector<unsigned char> ht(l.len[PTHR_BUF_TABLES]);
        double *T = (double *)ht.data();
        double *beta = T + NTt, *q = T + 2 * NTt, *ql = q + Vt + 1;
        float *tb = (float *)(ql + 3 * Vt + 1);
        for (int k = 0; k < NTt; ++k) {
            T[k] = host_temperature(cfg, k);
            volatile double one = 1.0, m2l2e = -2.0 * 1.4426950408889634073599;
            beta[k] = one / T[k];
            tb[k] = (float)(m2l2e / T[k]);
        }
        for (int n = 0; n <= Vt; ++n) { volatile double num = (double)(Vt - 2 * n); q[n] = num / (double)Vt; }
        for (int n = 0; n <= 3 * Vt; ++n) {
            volatile double num = (double)(3 * Vt - 2 * n), den = 3.0 * (double)Vt;
            ql[n] = num / den;
        }
        e = cudaMemcpyAsync(tab, ht.data(), ht.size(), cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);   // ht is freed below
    }
    if (e != cudaSuccess) { pthr_status r = cuda_fail(nullptr, e, "create"); delete b; return r; }
    if (couplings) {
        e = cudaMemcpyAsync(d.J, couplings, l.len[PTHR_BUF_J], cudaMemcpyDefault, b->stream);
    } else {
        e = launch_couplings_from_seed(d, 0, cfg->n_samples, b->stream);
    }
    if (e == cudaSuccess) e = launch_init_state(d, 0, cfg->n_samples, b->stream);
    if (e != cudaSuccess) { pthr_status r = cuda_fail(nullptr, e, "create/init"); delete b; return r; }
    st = do_sweep(b, 0, 0, 0, cfg->n_samples, 0);   // energies of every clone
    if (st != PTHR_OK) { fail(nullptr, st, "%s", b->err); delete b; return st; }
    *out = b;
    return PTHR_OK;
}

PTHR_API void pthr_destroy(pthr_batch *b) {
    if (!b) return;
    if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    delete b;
}

PTHR_API pthr_status pthr_set_stream(pthr_batch *b, void *stream) {
    if (!b) return fail(nullptr, PTHR_E_INVAL, "NULL handle");
    b->stream = (cudaStream_t)stream;
    return PTHR_OK;
}

PTHR_API pthr_status pthr_set_tuning(pthr_batch *b, const pthr_tuning *t) {
    if (!b) return fail(nullptr, PTHR_E_INVAL, "NULL handle");
    pthr_tuning nt{};
    if (t) nt = *t;
    if (nt.pt_lattices_per_block < 0 || nt.pt_lattices_per_block > sweep_max_k() ||
        nt.res_lattices_per_block < 0 || nt.res_lattices_per_block > sweep_max_k() ||
        nt.sweep_threads < 0 || nt.sweep_threads > 512 || nt.cluster_threads < 0 || nt.cluster_threads > 512 ||
        nt.cluster_iter_cap < 0)
        return fail(b, PTHR_E_INVAL, "tuning out of range");
    pthr_tuning old = b->tuning;
    b->tuning = nt;
    SweepShape sh = sweep_shape(b);
    const size_t smem = sweep_smem_bytes_for(b->cfg.L, sh.K_pt > sh.K_res ? sh.K_pt : sh.K_res);
    if (smem > 220 * 1024) {
        b->tuning = old;
        return fail(b, PTHR_E_INVAL, "tuning needs %zu bytes of shared memory per block", smem);
    }
    if (b->graph_exec) { cudaGraphExecDestroy(b->graph_exec); b->graph_exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    b->graph_ok = 0;
    return PTHR_OK;
}

PTHR_API pthr_status pthr_set_update_rule(pthr_batch *b, int rule) {
    if (!b) return fail(nullptr, PTHR_E_INVAL, "NULL handle");
    if (rule != PTHR_METROPOLIS && rule != PTHR_HEATBATH && rule != PTHR_MICSA)
        return fail(b, PTHR_E_INVAL, "unknown update_rule %d", rule);
    if (b->pt_sweep_off || b->res_sweep_off)
        return fail(b, PTHR_E_STATE, "the update rule changes only at an EMCS boundary (call pthr_swap first)");
    b->cfg.update_rule = rule;
    b->dev.rule = rule;
    // the captured EMCS graph holds the old rule's kernels
    if (b->graph_exec) { cudaGraphExecDestroy(b->graph_exec); b->graph_exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    b->graph_ok = 0;
    return PTHR_OK;
}

PTHR_API pthr_status pthr_get_tuning(const pthr_batch *b, pthr_tuning *t) {
    if (!b || !t) return fail(nullptr, PTHR_E_INVAL, "NULL argument");
    SweepShape sh = sweep_shape(b);
    t->pt_lattices_per_block = sh.K_pt;
    t->res_lattices_per_block = sh.K_res;
    t->sweep_threads = sh.threads;
    t->cluster_threads = b->tuning.cluster_threads > 0 ? b->tuning.cluster_threads : default_cluster_threads(b->cfg.L);
    t->cluster_iter_cap = b->tuning.cluster_iter_cap;
    return PTHR_OK;
}

PTHR_API pthr_status pthr_sweep(pthr_batch *b, int n_pt_sweeps, int n_res_sweeps) {
    PTHR_TRACE("pthr_sweep");
    if (!b) return fail(nullptr, PTHR_E_INVAL, "NULL handle");
    if (n_pt_sweeps < 0 || n_res_sweeps < 0) return fail(b, PTHR_E_INVAL, "negative sweep count");
    if ((long)b->pt_sweep_off + n_pt_sweeps >= (1L << 23) || (long)b->res_sweep_off + n_res_sweeps >= (1L << 23))
        return fail(b, PTHR_E_INVAL, "more than 2^23 sweeps in one EMCS");
    if (n_res_sweeps > 0 && b->cfg.n_res == 0) n_res_sweeps = 0;
    pthr_status st = do_sweep(b, n_pt_sweeps, n_res_sweeps, 0, b->cfg.n_samples, 0);
    if (st != PTHR_OK) return st;
    b->pt_sweep_off += n_pt_sweeps;
    b->res_sweep_off += n_res_sweeps;
    return PTHR_OK;
}

PTHR_API pthr_status pthr_houdayer(pthr_batch *b) {
    PTHR_TRACE("pthr_houdayer");
    if (!b) return fail(nullptr, PTHR_E_INVAL, "NULL handle");
    if (b->cfg.cluster_mode == PTHR_CLUSTER_OFF) return PTHR_OK;
    return do_cluster(b, 0, nullptr);
}

PTHR_API pthr_status pthr_cluster_labels(pthr_batch *b, int32_t *out_device) {
    PTHR_TRACE("pthr_cluster_labels");
    if (!b || !out_device) return fail(b, PTHR_E_INVAL, "NULL argument");
    return do_cluster(b, 1, out_device);
}

PTHR_API pthr_status pthr_swap(pthr_batch *b, int flags) {
    PTHR_TRACE("pthr_swap");
    if (!b) return fail(nullptr, PTHR_E_INVAL, "NULL handle");
    if (flags & ~(PTHR_SWAP_PT | PTHR_SWAP_ER)) return fail(b, PTHR_E_INVAL, "unknown swap flags");
    if ((flags & PTHR_SWAP_ER) && b->cfg.n_res < 1) return fail(b, PTHR_E_INVAL, "ER needs n_res >= 1");
    CUDA_TRY(b, launch_swap(b->dev, flags, 0, b->cfg.n_samples, b->stream), "swap launch");
    b->pt_sweep_off = 0;
    b->res_sweep_off = 0;
    return PTHR_OK;
}

PTHR_API pthr_status pthr_observables(pthr_batch *b, int flags, void *out, size_t bytes) {
    PTHR_TRACE("pthr_observables");
    if (!b) return fail(nullptr, PTHR_E_INVAL, "NULL handle");
    const size_t need = (size_t)b->cfg.n_samples * b->cfg.n_temps * PTHR_NOBS * sizeof(double);
    if ((flags & (PTHR_OBS_READ_HOST | PTHR_OBS_READ_DEVICE)) && (!out || bytes < need))
        return fail(b, PTHR_E_INVAL, "output buffer needs %zu bytes", need);
    if (flags & PTHR_OBS_MEASURE)
        CUDA_TRY(b, launch_measure(b->dev, 0, b->cfg.n_samples, (flags & PTHR_OBS_CHAOS) ? 1 : 0,
                                   b->stream), "measure launch");
    if (flags & PTHR_OBS_READ_DEVICE)
        CUDA_TRY(b, cudaMemcpyAsync(out, b->dev.obs, need, cudaMemcpyDeviceToDevice, b->stream), "obs copy");
    if (flags & PTHR_OBS_READ_HOST) {
        CUDA_TRY(b, cudaMemcpyAsync(out, b->dev.obs, need, cudaMemcpyDeviceToHost, b->stream), "obs copy");
        CUDA_TRY(b, cudaStreamSynchronize(b->stream), "obs sync");
    }
    if (flags & PTHR_OBS_RESET) {
        CUDA_TRY(b, cudaMemsetAsync(b->dev.obs, 0, need, b->stream), "obs reset");
        CUDA_TRY(b, cudaMemsetAsync(b->dev.chaos, 0, (size_t)b->cfg.n_samples * b->cfg.n_temps * 2 * sizeof(double),
                                    b->stream), "chaos reset");
    }
    return PTHR_OK;
}

PTHR_API pthr_status pthr_emcs(pthr_batch *b, int n, int use_graph) {
    PTHR_TRACE("pthr_emcs");
    if (!b) return fail(nullptr, PTHR_E_INVAL, "NULL handle");
    if (n < 0) return fail(b, PTHR_E_INVAL, "negative EMCS count");
    if (b->pt_sweep_off || b->res_sweep_off)
        return fail(b, PTHR_E_STATE, "pthr_emcs must start at an EMCS boundary (call pthr_swap first)");
    if (use_graph && b->stream != nullptr && !capturing(b->stream)) {
        if (!b->graph_ok) {
            CUDA_TRY(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
            pthr_status st = one_emcs(b);
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamEndCapture(b->stream, &g);
            if (st != PTHR_OK) { if (g) cudaGraphDestroy(g); return st; }
            if (e != cudaSuccess) return cuda_fail(b, e, "end capture");
            cudaGraphExec_t ge = nullptr;
            e = cudaGraphInstantiate(&ge, g, 0);
            if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_fail(b, e, "graph instantiate"); }
            b->graph = g;
            b->graph_exec = ge;
            b->graph_ok = 1;
        }
        for (int i = 0; i < n; ++i) CUDA_TRY(b, cudaGraphLaunch(b->graph_exec, b->stream), "graph launch");
        return PTHR_OK;
    }
    for (int i = 0; i < n; ++i) {
        pthr_status st = one_emcs(b);
        if (st != PTHR_OK) return st;
    }
    return PTHR_OK;
}

PTHR_API pthr_status pthr_prethermalize_reservoir(pthr_batch *b, int first, int count, int n_sweeps) {
    PTHR_TRACE("pthr_prethermalize_reservoir");
    if (!b) return fail(nullptr, PTHR_E_INVAL, "NULL handle");
    if (first < 0 || count < 0 || first + count > b->cfg.n_samples || n_sweeps < 0 || n_sweeps >= (1 << 23))
        return fail(b, PTHR_E_INVAL, "bad sample range or sweep count");
    if (b->cfg.n_res == 0 || n_sweeps == 0 || count == 0) return PTHR_OK;
    return do_sweep(b, 0, n_sweeps, first, count, 1);
}

PTHR_API pthr_status pthr_poll(pthr_batch *b, int timeout_ms) {
    if (!b) return fail(nullptr, PTHR_E_INVAL, "NULL handle");
    cudaEvent_t ev;
    CUDA_TRY(b, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event create");
    cudaError_t e = cudaEventRecord(ev, b->stream);
    if (e != cudaSuccess) { cudaEventDestroy(ev); return cuda_fail(b, e, "event record"); }
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        e = cudaEventQuery(ev);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) { cudaEventDestroy(ev); return cuda_fail(b, e, "stream"); }
        if (timeout_ms >= 0) {
            auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count();
            if (ms > timeout_ms) { cudaEventDestroy(ev); return fail(b, PTHR_E_TIMEOUT, "stream still busy after %d ms", timeout_ms); }
        }
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
    cudaEventDestroy(ev);
    uint32_t st[4] = {0, 0, 0, 0};
    CUDA_TRY(b, cudaMemcpy(st, b->dev.status, sizeof(st), cudaMemcpyDeviceToHost), "status read");
    CUDA_TRY(b, cudaMemset(b->dev.status, 0, sizeof(st)), "status clear");
    if (st[0] & STATUS_NOCONVERGE) return fail(b, PTHR_E_NOCONVERGE, "a cluster labelling loop hit its iteration cap");
    if (st[0] & STATUS_BOUNDS) return fail(b, PTHR_E_BOUNDS, "a device range check failed (the guarded work was skipped)");
    return PTHR_OK;
}

PTHR_API pthr_status pthr_export_spins(pthr_batch *b, int8_t *out_device) {
    PTHR_TRACE("pthr_export_spins");
    if (!b || !out_device) return fail(b, PTHR_E_INVAL, "NULL argument");
    CUDA_TRY(b, launch_export_spins(b->dev, out_device, b->stream), "export launch");
    return PTHR_OK;
}

PTHR_API pthr_status pthr_import_spins(pthr_batch *b, const int8_t *in_device) {
    PTHR_TRACE("pthr_import_spins");
    if (!b || !in_device) return fail(b, PTHR_E_INVAL, "NULL argument");
    CUDA_TRY(b, launch_import_spins(b->dev, in_device, b->stream), "import launch");
    return do_sweep(b, 0, 0, 0, b->cfg.n_samples, 0);
}

PTHR_API pthr_status pthr_reset_samples(pthr_batch *b, int first, int count, const float *couplings,
                                        const uint64_t *seeds, int pretherm_sweeps) {
    PTHR_TRACE("pthr_reset_samples");
    if (!b) return fail(nullptr, PTHR_E_INVAL, "NULL handle");
    if (first < 0 || count < 1 || first + count > b->cfg.n_samples || !seeds || pretherm_sweeps < 0)
        return fail(b, PTHR_E_INVAL, "bad sample range, seeds or pre-thermalisation");
    if (b->pt_sweep_off || b->res_sweep_off)
        return fail(b, PTHR_E_STATE, "samples can only be reset at an EMCS boundary");
    const Batch &d = b->dev;
    const size_t V = (size_t)d.L * d.L * d.L;
    CUDA_TRY(b, cudaMemcpyAsync(d.seeds + first, seeds, sizeof(unsigned long long) * count,
                                cudaMemcpyDefault, b->stream), "seed copy");
    // seeds may be pageable host memory: make the copy complete before returning
    CUDA_TRY(b, cudaStreamSynchronize(b->stream), "seed copy sync");
    if (couplings)
        CUDA_TRY(b, cudaMemcpyAsync(d.J + (size_t)first * 3 * V, couplings, sizeof(float) * 3 * V * count,
                                    cudaMemcpyDefault, b->stream), "coupling copy");
    else
        CUDA_TRY(b, launch_couplings_from_seed(d, first, count, b->stream), "couplings");
    CUDA_TRY(b, launch_init_state(d, first, count, b->stream), "init");
    pthr_status st = do_sweep(b, 0, 0, first, count, 0);
    if (st != PTHR_OK) return st;
    if (pretherm_sweeps > 0 && b->cfg.n_res > 0) {
        st = do_sweep(b, 0, pretherm_sweeps, first, count, 1);
        if (st != PTHR_OK) return st;
    }
    return PTHR_OK;
}

PTHR_API pthr_status pthr_set_active(pthr_batch *b, int first, int count, int active) {
    if (!b) return fail(nullptr, PTHR_E_INVAL, "NULL handle");
    if (first < 0 || count < 0 || first + count > b->cfg.n_samples) return fail(b, PTHR_E_INVAL, "bad sample range");
    if (count == 0) return PTHR_OK;
    CUDA_TRY(b, cudaMemsetAsync(b->dev.active + first, active ? 1 : 0, count, b->stream), "set active");
    return PTHR_OK;
}

struct BlobHeader {
    char magic[8];
    uint32_t version;
    uint32_t pad;
    pthr_config cfg;
    int32_t pt_sweep_off, res_sweep_off;
    uint64_t ws_bytes;
};

PTHR_API pthr_status pthr_save(pthr_batch *b, void *blob, size_t *bytes) {
    PTHR_TRACE("pthr_save");
    if (!b || !bytes) return fail(b, PTHR_E_INVAL, "NULL argument");
    const size_t total = make_layout(&b->cfg).total;
    const size_t need = sizeof(BlobHeader) + total;
    if (!blob) { *bytes = need; return PTHR_OK; }
    if (*bytes < need) return fail(b, PTHR_E_INVAL, "blob needs %zu bytes", need);
    BlobHeader h{};
    memcpy(h.magic, "PTHRBLOB", 8);
    h.version = 1;
    h.cfg = b->cfg;
    h.pt_sweep_off = b->pt_sweep_off;
    h.res_sweep_off = b->res_sweep_off;
    h.ws_bytes = total;
    memcpy(blob, &h, sizeof(h));
    CUDA_TRY(b, cudaMemcpyAsync((unsigned char *)blob + sizeof(h), b->ws, total, cudaMemcpyDeviceToHost, b->stream), "save copy");
    CUDA_TRY(b, cudaStreamSynchronize(b->stream), "save sync");
    *bytes = need;
    return PTHR_OK;
}

PTHR_API pthr_status pthr_load(pthr_batch *b, const void *blob, size_t bytes) {
    PTHR_TRACE("pthr_load");
    if (!b || !blob) return fail(b, PTHR_E_INVAL, "NULL argument");
    BlobHeader h;
    if (bytes < sizeof(h)) return fail(b, PTHR_E_INVAL, "blob too small");
    memcpy(&h, blob, sizeof(h));
    const size_t total = make_layout(&b->cfg).total;
    if (memcmp(h.magic, "PTHRBLOB", 8) != 0 || h.version != 1) return fail(b, PTHR_E_INVAL, "not a pthr blob");
    if (memcmp(&h.cfg, &b->cfg, sizeof(pthr_config)) != 0 || h.ws_bytes != total || bytes < sizeof(h) + total)
        return fail(b, PTHR_E_INVAL, "blob was saved from a different configuration");
    CUDA_TRY(b, cudaMemcpyAsync(b->ws, (const unsigned char *)blob + sizeof(h), total, cudaMemcpyHostToDevice, b->stream), "load copy");
    CUDA_TRY(b, cudaStreamSynchronize(b->stream), "load sync");
    b->pt_sweep_off = h.pt_sweep_off;
    b->res_sweep_off = h.res_sweep_off;
    return PTHR_OK;
}

struct pthr_group {
    cudaStream_t stream;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    int n;
    int launches;   // kernel launches per EMCS in the graph
    int fused;      // 1: the four-launch form (group kernels), 0: per-batch graphs
    pthr_batch **batches;   // [n] members, for ordering against their own streams
    cudaEvent_t *ev_in;     // [n] work queued on each member's stream
    cudaEvent_t ev_out;     // the group's EMCS, for the members' later work
};

namespace {

// A new group handle with its ordering events; nullptr if an event could not
// be created (then nothing is left allocated).
pthr_group *new_group(pthr_batch *const *batches, int n, cudaStream_t st, cudaGraph_t g, cudaGraphExec_t exec,
                      int launches, int fused) {
    pthr_group *grp = new pthr_group();
    grp->stream = st;
    grp->graph = g;
    grp->exec = exec;
    grp->n = n;
    grp->launches = launches;
    grp->fused = fused;
    grp->batches = new pthr_batch *[n];
    grp->ev_in = new cudaEvent_t[n]();
    grp->ev_out = nullptr;
    bool ok = cudaEventCreateWithFlags(&grp->ev_out, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; i < n; ++i) {
        grp->batches[i] = batches[i];
        ok = ok && cudaEventCreateWithFlags(&grp->ev_in[i], cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) {
        for (int i = 0; i < n; ++i) if (grp->ev_in[i]) cudaEventDestroy(grp->ev_in[i]);
        if (grp->ev_out) cudaEventDestroy(grp->ev_out);
        delete[] grp->ev_in;
        delete[] grp->batches;
        delete grp;
        return nullptr;
    }
    return grp;
}

}  // namespace

namespace {

// One EMCS of every batch as four launches in total (sweep, cluster move,
// swap, measurement), each over the blocks of all batches; possible when
// the batches share an update rule, their sizes are compiled into the group
// kernels and no error-path knob is set.  Returns PTHR_E_STATE (nothing
// enqueued) when the group does not qualify.
pthr_status group_fused_emcs(pthr_batch *const *batches, int n, cudaStream_t st, int *launches) {
    if (n > GROUP_MAX) return PTHR_E_STATE;
    const int rule = batches[0]->cfg.update_rule;
    for (int i = 0; i < n; ++i) {
        const pthr_batch *b = batches[i];
        if (b->cfg.update_rule != rule || !group_supports_L(b->cfg.L) || b->tuning.cluster_iter_cap > 0 ||
            b->cfg.n_replicas > 32)
            return PTHR_E_STATE;
    }
    // heaviest batches first
    int order[GROUP_MAX];
    for (int i = 0; i < n; ++i) order[i] = i;
    for (int i = 1; i < n; ++i)
        for (int j = i; j > 0 && batches[order[j]]->cfg.L > batches[order[j - 1]]->cfg.L; --j) {
            const int t = order[j]; order[j] = order[j - 1]; order[j - 1] = t;
        }
    GroupSweepArgs gs{};
    GroupClusterArgs gc{};
    GroupBatchArgs gw{}, gm{};
    int sw_threads = 32, cl_threads = 32, sw_blocks = 0, cl_blocks = 0, w_blocks = 0, m_blocks = 0, w_threads = 32;
    size_t sw_smem = 0, cl_smem = 0, w_smem = 0, m_smem = 0;
    for (int ii = 0; ii < n; ++ii) {
        pthr_batch *b = batches[order[ii]];
        const pthr_config *c = &b->cfg;
        SweepLaunch sl{};
        if (sweep_launch(b, c->sweeps_per_emcs, c->er_on ? c->res_sweeps_per_emcs : 0, 0, c->n_samples, 0,
                         group_sweep_kt(c->L), &sl) != PTHR_OK)
            return PTHR_E_STATE;
        gs.a[gs.n] = sl.a;
        gs.off[gs.n] = sw_blocks;
        ++gs.n;
        sw_blocks += sl.blocks;
        if (sl.threads > sw_threads) sw_threads = sl.threads;
        if (sl.smem > sw_smem) sw_smem = sl.smem;
        if (c->cluster_mode != PTHR_CLUSTER_OFF && b->dev.n_acu > 0) {
            ClusterArgs a{};
            a.b = b->dev;
            a.sample_first = 0;
            a.sample_count = c->n_samples;
            a.iter_cap = 0;
            gc.a[gc.n] = a;
            gc.off[gc.n] = cl_blocks;
            ++gc.n;
            cl_blocks += c->n_samples * b->dev.NPAIR * b->dev.n_acu;
            const int t = cluster_threads_of(b);
            if (t > cl_threads) cl_threads = t;
            if (cluster_smem_bytes_for(c->L) > cl_smem) cl_smem = cluster_smem_bytes_for(c->L);
        }
        gw.b[gw.n] = b->dev;
        gw.flags[gw.n] = PTHR_SWAP_PT | (c->er_on ? PTHR_SWAP_ER : 0);
        gw.off[gw.n] = w_blocks;
        ++gw.n;
        w_blocks += c->n_samples;
        if (32 * c->n_replicas > w_threads) w_threads = 32 * c->n_replicas;
        const size_t ws = (size_t)b->dev.NR * b->dev.NSLOT * (sizeof(double) + sizeof(int));
        if (ws > w_smem) w_smem = ws;
        gm.b[gm.n] = b->dev;
        gm.off[gm.n] = m_blocks;
        ++gm.n;
        m_blocks += (c->n_samples * c->n_temps + 7) / 8;
        if (measure_smem_bytes_for(c->L) > m_smem) m_smem = measure_smem_bytes_for(c->L);
    }
    gs.off[gs.n] = sw_blocks;
    gc.off[gc.n] = cl_blocks;
    gw.off[gw.n] = w_blocks;
    gm.off[gm.n] = m_blocks;
    if (sw_smem > 200 * 1024 || cl_smem > 200 * 1024) return PTHR_E_STATE;
    if (launch_group_sweep(gs, rule, sw_blocks, sw_threads, sw_smem, st) != cudaSuccess) return PTHR_E_CUDA;
    if (launch_group_cluster(gc, cl_blocks, cl_threads, cl_smem, st) != cudaSuccess) return PTHR_E_CUDA;
    if (launch_group_swap(gw, w_blocks, w_threads, w_smem, st) != cudaSuccess) return PTHR_E_CUDA;
    if (launch_group_measure(gm, m_blocks, m_smem, st) != cudaSuccess) return PTHR_E_CUDA;
    *launches = (sw_blocks > 0) + (cl_blocks > 0) + (w_blocks > 0) + (m_blocks > 0);
    return PTHR_OK;
}

}  // namespace

PTHR_API pthr_status pthr_group_create(pthr_batch *const *batches, int n, void *stream, pthr_group **out) {
    PTHR_TRACE("pthr_group_create");
    if (!batches || n < 1 || !out || !stream)
        return fail(nullptr, PTHR_E_INVAL, "group needs batches, n >= 1, a non-default stream and out");
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        if (!batches[i]) return fail(nullptr, PTHR_E_INVAL, "NULL batch in group");
        if (batches[i]->pt_sweep_off || batches[i]->res_sweep_off)
            return fail(nullptr, PTHR_E_STATE, "group batches must be at an EMCS boundary");
        if (batches[i]->stream == nullptr || batches[i]->stream == (cudaStream_t)stream)
            return fail(nullptr, PTHR_E_INVAL, "each batch needs its own non-default stream");
    }
    cudaStream_t master = (cudaStream_t)stream;
    if (capturing(master)) return fail(nullptr, PTHR_E_STATE, "stream is already capturing");
    // kernel attributes are set outside the capture (first launch of a kind)
    {
        cudaError_t e = cudaStreamBeginCapture(master, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "begin capture");
        int launches = 0;
        pthr_status st = group_fused_emcs(batches, n, master, &launches);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(master, &g);
        if (st == PTHR_OK && e == cudaSuccess) {
            cudaGraphExec_t exec = nullptr;
            e = cudaGraphInstantiate(&exec, g, 0);
            if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_fail(nullptr, e, "group graph instantiate"); }
            pthr_group *grp = new_group(batches, n, master, g, exec, launches, 1);
            if (!grp) {
                cudaGraphExecDestroy(exec);
                cudaGraphDestroy(g);
                return fail(nullptr, PTHR_E_CUDA, "group event create");
            }
            *out = grp;
            return PTHR_OK;
        }
        if (g) cudaGraphDestroy(g);
        if (st == PTHR_E_CUDA) return fail(nullptr, st, "group kernel launch failed during capture");
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "group capture");
        cudaGetLastError();
    }
    // otherwise one EMCS of every batch, each on its own stream, in one graph
    cudaEvent_t fork = nullptr;
    cudaEvent_t *join = new cudaEvent_t[n]();
    cudaError_t e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    for (int i = 0; i < n && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming);
    pthr_status st = PTHR_OK;
    int failed = -1;   // batch whose EMCS could not be captured
    cudaGraph_t g = nullptr;
    if (e == cudaSuccess) e = cudaStreamBeginCapture(master, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        e = cudaEventRecord(fork, master);
        for (int i = 0; i < n && e == cudaSuccess && st == PTHR_OK; ++i) {
            e = cudaStreamWaitEvent(batches[i]->stream, fork, 0);
            if (e == cudaSuccess) st = one_emcs(batches[i]);
            if (st != PTHR_OK) failed = i;
            if (e == cudaSuccess && st == PTHR_OK) e = cudaEventRecord(join[i], batches[i]->stream);
            if (e == cudaSuccess && st == PTHR_OK) e = cudaStreamWaitEvent(master, join[i], 0);
        }
        cudaError_t e2 = cudaStreamEndCapture(master, &g);
        if (e == cudaSuccess) e = e2;
    }
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess && st == PTHR_OK) e = cudaGraphInstantiate(&exec, g, 0);
    if (fork) cudaEventDestroy(fork);
    for (int i = 0; i < n; ++i) if (join[i]) cudaEventDestroy(join[i]);
    delete[] join;
    if (st != PTHR_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        if (st != PTHR_OK) return fail(nullptr, st, "batch %d: %s", failed, batches[failed]->err);
        return cuda_fail(nullptr, e, "group capture");
    }
    int launches = 0;
    for (int i = 0; i < n; ++i)
        launches += 2 + (batches[i]->cfg.cluster_mode != PTHR_CLUSTER_OFF && batches[i]->dev.n_acu > 0) + 1;
    pthr_group *grp = new_group(batches, n, master, g, exec, launches, 0);
    if (!grp) {
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(g);
        return fail(nullptr, PTHR_E_CUDA, "group event create");
    }
    *out = grp;
    return PTHR_OK;
}

PTHR_API pthr_status pthr_group_info(const pthr_group *g, int *launches_per_emcs) {
    if (!g || !launches_per_emcs) return fail(nullptr, PTHR_E_INVAL, "NULL group or output");
    *launches_per_emcs = g->launches;
    return PTHR_OK;
}

PTHR_API pthr_status pthr_group_emcs(pthr_group *g, int n) {
    PTHR_TRACE("pthr_group_emcs");
    if (!g || n < 0) return fail(nullptr, PTHR_E_INVAL, "bad group or count");
    if (n == 0) return PTHR_OK;
    if (capturing(g->stream)) {
        // inside the caller's capture a graph cannot be launched: the
        // four-launch form enqueues its kernels instead (the capture orders
        // them); the per-batch-graph form cannot be captured
        if (!g->fused)
            return fail(nullptr, PTHR_E_STATE, "this group runs per-batch graphs and cannot be captured");
        for (int i = 0; i < n; ++i) {
            int launches = 0;
            const pthr_status st = group_fused_emcs(g->batches, g->n, g->stream, &launches);
            if (st != PTHR_OK) return fail(nullptr, st, "group kernels could not be enqueued in the capture");
        }
        return PTHR_OK;
    }
    // after the work already queued on every member's stream ...
    for (int i = 0; i < g->n; ++i) {
        cudaError_t e = cudaEventRecord(g->ev_in[i], g->batches[i]->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(g->stream, g->ev_in[i], 0);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "group ordering");
    }
    for (int i = 0; i < n; ++i) {
        cudaError_t e = cudaGraphLaunch(g->exec, g->stream);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "group graph launch");
    }
    // ... and before the work queued on them later
    cudaError_t e = cudaEventRecord(g->ev_out, g->stream);
    for (int i = 0; i < g->n && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(g->batches[i]->stream, g->ev_out, 0);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "group ordering");
    return PTHR_OK;
}

PTHR_API void pthr_group_destroy(pthr_group *g) {
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    for (int i = 0; i < g->n; ++i) if (g->ev_in[i]) cudaEventDestroy(g->ev_in[i]);
    if (g->ev_out) cudaEventDestroy(g->ev_out);
    delete[] g->ev_in;
    delete[] g->batches;
    delete g;
}

PTHR_API const char *pthr_last_error(const pthr_batch *b) { return b ? b->err : g_err; }

PTHR_API pthr_status pthr_reservoir_autocorrelation(pthr_batch *b, int first, int count, int n_points,
                                                    int sweeps_per_point, void *snapshot_device,
                                                    size_t snapshot_bytes, int64_t *out_device) {
    PTHR_TRACE("pthr_reservoir_autocorrelation");
    if (!b) return fail(nullptr, PTHR_E_INVAL, "NULL handle");
    if (b->cfg.n_res < 1) return fail(b, PTHR_E_INVAL, "the batch has no reservoir clones");
    if (first < 0 || count < 1 || first + count > b->cfg.n_samples || n_points < 1 || sweeps_per_point < 1 ||
        (long long)n_points * sweeps_per_point >= (1LL << 23) || !snapshot_device || !out_device)
        return fail(b, PTHR_E_INVAL, "bad sample range, point count, sweeps or NULL buffer");
    if (((uintptr_t)snapshot_device) & 15) return fail(b, PTHR_E_INVAL, "snapshot must be 16-byte aligned");
    const size_t need = (size_t)count * b->cfg.n_replicas * b->cfg.n_res * (size_t)b->dev.lat_words * 4;
    if (snapshot_bytes < need)
        return fail(b, PTHR_E_NOMEM, "snapshot needs %zu bytes, got %zu", need, snapshot_bytes);
    if (b->pt_sweep_off || b->res_sweep_off)
        return fail(b, PTHR_E_STATE, "call at an EMCS boundary");
    uint32_t *snap = (uint32_t *)snapshot_device;
    CUDA_TRY(b, launch_snapshot_reservoir(b->dev, first, count, snap, b->stream), "snapshot");
    for (int p = 0; p < n_points; ++p) {
        pthr_status st = do_sweep(b, 0, sweeps_per_point, first, count, 1);
        if (st != PTHR_OK) return st;
        CUDA_TRY(b, launch_reservoir_overlap(b->dev, first, count, snap, (long long *)out_device, n_points, p,
                                             b->stream), "overlap");
    }
    return PTHR_OK;
}

PTHR_API pthr_status pthr_reservoir_autocorrelation_noalloc(pthr_batch *b, int first, int count, int n_points,
                                                            int sweeps_per_point, int64_t *out_device) {
    PTHR_TRACE("pthr_reservoir_autocorrelation_noalloc");
    if (!b) return fail(nullptr, PTHR_E_INVAL, "NULL handle");
    if (b->cfg.n_res < 1) return fail(b, PTHR_E_INVAL, "the batch has no reservoir clones");
    if (first < 0 || count < 1 || first + count > b->cfg.n_samples || n_points < 1 || sweeps_per_point < 1 ||
        !out_device)
        return fail(b, PTHR_E_INVAL, "bad sample range, point count, sweeps or NULL output");
    const size_t need = (size_t)count * b->cfg.n_replicas * b->cfg.n_res * (size_t)b->dev.lat_words * 4;
    cudaPointerAttributes pa{};
    int dev = 0;
    CUDA_TRY(b, cudaPointerGetAttributes(&pa, b->ws), "workspace attributes");
    CUDA_TRY(b, cudaGetDevice(&dev), "current device");
    if (pa.type == cudaMemoryTypeDevice && pa.device != dev)
        return fail(b, PTHR_E_INVAL, "make the batch's device (%d) current first (current: %d)", pa.device, dev);
    void *snap = nullptr;
    size_t cap = 0;
    CUDA_TRY(b, noalloc_snapshot(&snap, &cap), "fixed snapshot address");
    if (need > cap)
        return fail(b, PTHR_E_NOMEM,
                    "the reservoir snapshot of %d samples needs %zu bytes; the fixed scratch holds %zu "
                    "(call it on fewer samples at a time)", count, need, cap);
    return pthr_reservoir_autocorrelation(b, first, count, n_points, sweeps_per_point, snap, cap, out_device);
}

PTHR_API pthr_status pthr_check_canaries(pthr_batch *b, int *bad_buffer) {
    if (!b) return fail(nullptr, PTHR_E_INVAL, "NULL handle");
    const Layout l = make_layout(&b->cfg);
    std::vector<unsigned char> h(GUARD_BYTES * PTHR_NBUF);
    const unsigned char *base = (const unsigned char *)b->ws;
    for (int i = 0; i < PTHR_NBUF; ++i)
        CUDA_TRY(b, cudaMemcpyAsync(h.data() + i * GUARD_BYTES, base + l.guard[i], GUARD_BYTES,
                                    cudaMemcpyDeviceToHost, b->stream), "guard copy");
    CUDA_TRY(b, cudaStreamSynchronize(b->stream), "guard sync");
    if (bad_buffer) *bad_buffer = -1;
    for (int i = 0; i < PTHR_NBUF; ++i)
        for (size_t k = 0; k < GUARD_BYTES; ++k)
            if (h[i * GUARD_BYTES + k] != CANARY) {
                if (bad_buffer) *bad_buffer = i;
                return fail(b, PTHR_E_BOUNDS, "guard block after workspace buffer %d was overwritten", i);
            }
    return PTHR_OK;
}

PTHR_API pthr_status pthr_measure_peak(int kind, void *scratch_device, size_t scratch_bytes, void *stream,
                                       double *rate, double *seconds) {
    if (kind < 0 || kind >= PTHR_NPEAK || !rate || !seconds)
        return fail(nullptr, PTHR_E_INVAL, "bad peak kind or NULL output");
    if (!scratch_device || scratch_bytes < (size_t)PEAK_SINK_BYTES ||
        (kind == PTHR_PEAK_L2_READ && scratch_bytes < (size_t)PEAK_SINK_BYTES + (1u << 20)))
        return fail(nullptr, PTHR_E_INVAL, "scratch buffer too small (%zu bytes)", scratch_bytes);
    double work = 0.0;
    float ms = 0.f;
    cudaError_t e = run_peak(kind, scratch_device, scratch_bytes, (cudaStream_t)stream, &work, &ms);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "peak microbenchmark");
    *seconds = ms * 1e-3;
    *rate = ms > 0.f ? work / (ms * 1e-3) : 0.0;
    return PTHR_OK;
}

}  // extern "C"
