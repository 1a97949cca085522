// cluster.cu -- step (ii) of the EMCS (Sec. 3): the all-cluster Houdayer
// update (ACU) and the original single-cluster Houdayer move, one block per
// replica pair at one temperature.
//
// The block copies the two clones into shared memory, computes the site
// overlaps q_i = s^a_i s^b_i (Eq. (2)), labels the connected components of
// {i ~ j : neighbours, q_i = q_j} with a lock-free union-find in shared memory
// (larger root always hooked under the smaller one, so every root is the
// smallest site index of its cluster: the canonical label), draws one sign per
// root from Philox keyed by that label, flips both clones, recomputes both
// energies (FP64) and writes the pair back.  Every loop is bounded; hitting a
// bound sets STATUS_NOCONVERGE instead of spinning.
#include "kernels.cuh"

namespace pthr {

namespace {

__device__ __forceinline__ int find_root(volatile int *parent, int x, int cap, bool &ok) {
    for (int it = 0; it < cap; ++it) {
        const int p = parent[x];
        if (p == x) return x;
        const int gp = parent[p];
        if (gp != p) parent[x] = gp;   // path halving: gp is an ancestor of x
        x = gp;
    }
    ok = false;
    return x;
}

__device__ __forceinline__ void unite(volatile int *parent, int a, int b, int cap, bool &ok) {
    for (int it = 0; it < cap; ++it) {
        a = find_root(parent, a, cap, ok);
        b = find_root(parent, b, cap, ok);
        if (!ok || a == b) return;
        if (a < b) { const int t = a; a = b; b = t; }   // hook the larger root a under b
        const int old = atomicCAS(const_cast<int *>(&parent[a]), a, b);
        if (old == a) return;
    }
    ok = false;
}

template <int L>
__device__ __forceinline__ int neighbour(int i, int mu) {
    const int x = i % L, y = (i / L) % L, z = i / (L * L);
    if (mu == 0) return ((x + 1) % L) + L * (y + L * z);
    if (mu == 1) return x + L * (((y + 1) % L) + L * z);
    return x + L * (y + L * ((z + 1) % L));
}

template <int L>
__device__ __forceinline__ unsigned char spin_byte(const unsigned char *S, int i) {
    int w, by;
    site_slot<L>(i, w, by);
    return S[4 * w + by];
}

// CAPPED = false: every loop bound is the compile-time constant 4V+64 (the
// production path; a runtime bound makes the labelling loops markedly
// slower).  CAPPED = true: the bound comes from the tuning knob, used only to
// exercise the error path.
template <int L, bool CAPPED>
__global__ void __launch_bounds__(1024) cluster_kernel(ClusterArgs a) {
    using Gm = Geom<L>;
    constexpr int V = Gm::V, LW = Gm::LAT_WORDS;
    extern __shared__ __align__(16) unsigned char smem[];
    int *parent = reinterpret_cast<int *>(smem);                       // [V]
    int *cnt = parent + V;                                             // [V]
    uint32_t *sa = reinterpret_cast<uint32_t *>(cnt + V);              // [LW]
    uint32_t *sb = sa + LW;                                            // [LW]
    unsigned char *flag = reinterpret_cast<unsigned char *>(sb + LW);  // [V]
    __shared__ int s_ok;
    __shared__ int s_nneg, s_root, s_nclus, s_nflip;
    __shared__ int s_top[2][32];
    __shared__ double s_E[2];
    __shared__ int s_scan[1024];

    const Batch &b = a.b;
    const int n_acu = b.n_acu;
    int t = blockIdx.x;
    const int k = t % n_acu; t /= n_acu;
    const int P = t % b.NPAIR; t /= b.NPAIR;
    const int s = a.sample_first + t;
    if (!b.active[s]) return;
    const uint32_t emcs = b.emcs[s];
    if (!a.label_only && (emcs % (uint32_t)b.acu_interval) != 0u) return;
    const unsigned long long seed = b.seeds[s];
    const int tid = threadIdx.x, T = blockDim.x;
    const int ga = 2 * P, gb = 2 * P + 1;
    const int la = ga * b.NSLOT + b.perm[((size_t)s * b.NR + ga) * b.NSLOT + k];
    const int lb = gb * b.NSLOT + b.perm[((size_t)s * b.NR + gb) * b.NSLOT + k];
    const uint32_t pair_id = (uint32_t)(P * b.NT + k);
    uint32_t *ga_ptr = b.spins + ((size_t)s * b.NLAT + la) * LW;
    uint32_t *gb_ptr = b.spins + ((size_t)s * b.NLAT + lb) * LW;

    if (tid == 0) { s_ok = 1; s_nneg = 0; s_root = -1; s_nclus = 0; s_nflip = 0; }
    if (tid < 2) s_E[tid] = 0.0;
    for (int i = tid; i < LW / 4; i += T) {
        reinterpret_cast<uint4 *>(sa)[i] = reinterpret_cast<const uint4 *>(ga_ptr)[i];
        reinterpret_cast<uint4 *>(sb)[i] = reinterpret_cast<const uint4 *>(gb_ptr)[i];
    }
    __syncthreads();
    const unsigned char *A = reinterpret_cast<const unsigned char *>(sa);
    const unsigned char *B = reinterpret_cast<const unsigned char *>(sb);
    // q_i < 0 <=> the two bytes differ (0x3F vs 0xBF)
    for (int i = tid; i < V; i += T) {
        flag[i] = (spin_byte<L>(A, i) ^ spin_byte<L>(B, i)) >> 7;
        parent[i] = i;
        cnt[i] = 0;
    }
    __syncthreads();
    bool ok = true;
    const int cap = CAPPED ? a.iter_cap : 4 * V + 64;
    volatile int *vp = parent;
    for (int i = tid; i < V; i += T) {
        const unsigned char qi = flag[i];
#pragma unroll
        for (int mu = 0; mu < 3; ++mu) {
            const int j = neighbour<L>(i, mu);
            if (flag[j] == qi) unite(vp, i, j, cap, ok);
        }
    }
    __syncthreads();
    for (int i = tid; i < V; i += T) {
        const int r = find_root(vp, i, cap, ok);
        parent[i] = r;
    }
    if (!ok) s_ok = 0;
    __syncthreads();
    if (!s_ok) {
        if (tid == 0) set_status(b.status, STATUS_NOCONVERGE);
        return;
    }
    if (a.labels_out) {
        int32_t *out = a.labels_out + ((size_t)(s * b.NPAIR + P) * b.NT + k) * V;
        for (int i = tid; i < V; i += T) out[i] = parent[i];
    }
    // cluster sizes (statistics)
    for (int i = tid; i < V; i += T) atomicAdd(&cnt[parent[i]], 1);
    __syncthreads();
    if (a.label_only) return;

    if (b.cluster_mode == PTHR_CLUSTER_ACU) {
        // one sign per cluster: eta = -1 iff top bit of word 0 of
        // (label, pair_id, emcs, TAG_ACU); the root's flag byte receives it
        for (int i = tid; i < V; i += T) {
            if (parent[i] == i) {
                const uint32_t w = philox_word0(seed, (uint32_t)i, pair_id, emcs, TAG_ACU);
                flag[i] = (unsigned char)(w >> 31);
            }
        }
        __syncthreads();
    } else {
        // single cluster: seed = the floor(u*n)-th q = -1 site, n = #(q = -1)
        const int chunk = (V + T - 1) / T;
        const int lo = tid * chunk, hi = min(V, lo + chunk);
        int my = 0;
        for (int i = lo; i < hi; ++i) my += flag[i];
        s_scan[tid] = my;
        __syncthreads();
        if (tid == 0) {
            int acc = 0;
            for (int u = 0; u < T; ++u) { const int v = s_scan[u]; s_scan[u] = acc; acc += v; }
            s_nneg = acc;
        }
        __syncthreads();
        const int n = s_nneg;
        if (n > 0) {
            const uint32_t w = philox_word0(seed, 0u, pair_id, emcs, TAG_SINGLE);
            const int target = (int)(((unsigned long long)(w >> 8) * (unsigned long long)n) >> 24);
            int seen = s_scan[tid];
            if (target >= seen && target < seen + my) {
                for (int i = lo; i < hi; ++i) {
                    if (flag[i]) {
                        if (seen == target) { s_root = parent[i]; break; }
                        ++seen;
                    }
                }
            }
        }
        __syncthreads();
        const int root = s_root;
        for (int i = tid; i < V; i += T)
            if (parent[i] == i) flag[i] = (unsigned char)(i == root);
        __syncthreads();
    }
    // flip both clones on the selected clusters
    unsigned char *Aw = reinterpret_cast<unsigned char *>(sa);
    unsigned char *Bw = reinterpret_cast<unsigned char *>(sb);
    int nflip = 0;
    for (int i = tid; i < V; i += T) {
        if (flag[parent[i]]) {
            int w, by;
            site_slot<L>(i, w, by);
            Aw[4 * w + by] ^= 0x80u;
            Bw[4 * w + by] ^= 0x80u;
            ++nflip;
        }
    }
    // statistics: number of clusters, two largest sizes
    int nroots = 0, t1 = 0, t2 = 0;
    for (int i = tid; i < V; i += T) {
        if (parent[i] == i) {
            ++nroots;
            const int c = cnt[i];
            if (c > t1) { t2 = t1; t1 = c; } else if (c > t2) { t2 = c; }
        }
    }
    atomicAdd(&s_nclus, nroots);
    atomicAdd(&s_nflip, nflip);
    // warp top-2 then block top-2
    for (int o = 16; o > 0; o >>= 1) {
        const int u1 = __shfl_xor_sync(0xffffffffu, t1, o), u2 = __shfl_xor_sync(0xffffffffu, t2, o);
        int n1, n2;
        if (u1 > t1) { n1 = u1; n2 = max(t1, u2); } else { n1 = t1; n2 = max(t2, u1); }
        t1 = n1; t2 = n2;
    }
    if ((tid & 31) == 0) { s_top[0][tid >> 5] = t1; s_top[1][tid >> 5] = t2; }
    __syncthreads();
    // energies of both clones (Eq. (1)), exact FP32 pairs then FP64
    const float *J = b.J + (size_t)s * 3 * V;
    float ha = 0.f, la_ = 0.f, hb = 0.f, lb_ = 0.f;
    for (int i = tid; i < V; i += T) {
        const float ai = spin_byte<L>(Aw, i) == SPIN_DN ? -1.f : 1.f;
        const float bi = spin_byte<L>(Bw, i) == SPIN_DN ? -1.f : 1.f;
#pragma unroll
        for (int mu = 0; mu < 3; ++mu) {
            const int j = neighbour<L>(i, mu);
            const float Jm = J[mu * V + i];
            const float aj = spin_byte<L>(Aw, j) == SPIN_DN ? -1.f : 1.f;
            const float bj = spin_byte<L>(Bw, j) == SPIN_DN ? -1.f : 1.f;
            two_sum_acc(ha, la_, ai * (Jm * aj));
            two_sum_acc(hb, lb_, bi * (Jm * bj));
        }
    }
    double ea = (double)ha + (double)la_, eb = (double)hb + (double)lb_;
    for (int o = 16; o > 0; o >>= 1) {
        ea += __shfl_xor_sync(0xffffffffu, ea, o);
        eb += __shfl_xor_sync(0xffffffffu, eb, o);
    }
    if ((tid & 31) == 0) { atomicAdd(&s_E[0], ea); atomicAdd(&s_E[1], eb); }
    __syncthreads();
    for (int i = tid; i < LW / 4; i += T) {
        reinterpret_cast<uint4 *>(ga_ptr)[i] = reinterpret_cast<const uint4 *>(sa)[i];
        reinterpret_cast<uint4 *>(gb_ptr)[i] = reinterpret_cast<const uint4 *>(sb)[i];
    }
    if (tid == 0) {
        b.E[(size_t)s * b.NLAT + la] = -s_E[0];
        b.E[(size_t)s * b.NLAT + lb] = -s_E[1];
        int a1 = 0, a2 = 0;
        for (int w = 0; w < (T + 31) / 32; ++w) {
            const int u1 = s_top[0][w], u2 = s_top[1][w];
            if (u1 > a1) { a2 = max(a1, u2); a1 = u1; } else { a2 = max(a2, u1); }
        }
        long long *cs = b.cstat + (((size_t)s * b.NPAIR + P) * b.NT + k) * 4;
        cs[0] = s_nclus;
        cs[1] = a1;
        cs[2] = a2;
        cs[3] = s_nflip;
    }
}

template <int L>
size_t cluster_smem(void) {
    using Gm = Geom<L>;
    return (size_t)8 * Gm::V + (size_t)8 * Gm::LAT_WORDS + (size_t)Gm::V + 16;
}

template <int L>
cudaError_t launch_cluster_L(const ClusterArgs &a, int threads, cudaStream_t st) {
    static bool configured = false;
    if (!configured) {
        cudaError_t e = allow_max_dynamic_smem(cluster_kernel<L, false>);
        if (e == cudaSuccess) e = allow_max_dynamic_smem(cluster_kernel<L, true>);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const int blocks = a.sample_count * a.b.NPAIR * a.b.n_acu;
    if (blocks <= 0) return cudaSuccess;
    if (a.iter_cap > 0)
        cluster_kernel<L, true><<<blocks, threads, cluster_smem<L>(), st>>>(a);
    else
        cluster_kernel<L, false><<<blocks, threads, cluster_smem<L>(), st>>>(a);
    return cudaGetLastError();
}

}  // namespace

size_t cluster_smem_bytes_for(int L) {
#define X(LL) if (L == LL) return cluster_smem<LL>();
    PTHR_FOR_EACH_L(X)
#undef X
    return 0;
}

cudaError_t launch_cluster(const ClusterArgs &a, int threads, cudaStream_t st) {
#define X(LL) if (a.b.L == LL) return launch_cluster_L<LL>(a, threads, st);
    PTHR_FOR_EACH_L(X)
#undef X
    return cudaErrorInvalidValue;
}

}  // namespace pthr
