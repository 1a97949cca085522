// cluster.cu -- step (ii) of the EMCS (Sec. 3): the all-cluster Houdayer
// update (ACU) and the original single-cluster Houdayer move, one block per
// replica pair at one temperature.
//
// The block copies the two clones into shared memory and computes the site
// overlaps q_i = s^a_i s^b_i (Eq. (2)) with one XOR per 4-site word.  It then
// labels the connected components of {i ~ j : neighbours, q_i = q_j}:
//  1. runs of equal q along each x row (with the periodic wrap) become stars
//     rooted at their smallest site;
//  2. a lock-free union-find in shared memory joins runs across y and z
//     edges, always hooking the larger root under the smaller one, so every
//     root is the smallest site index of its cluster (the canonical label).
//     An edge whose left neighbours in both rows are in the same two runs is
//     implied by that neighbouring edge and skipped; x = 0 never skips.
// The q values of a row are one bit mask, so runs and the edges to join come
// from a few bit operations per row.  One sign per root is drawn from Philox
// keyed by the label; both clones flip word by word, the energies are updated
// (on the coupling grid H_a is recomputed and H_b follows from the conserved
// H_a + H_b) and the pair is written back.  Every loop is bounded; hitting a bound sets STATUS_NOCONVERGE
// instead of spinning.
#include "kernels.cuh"
#include "bitrows.cuh"

namespace pthr {

namespace {

__device__ __forceinline__ int find_root(volatile int *parent, int x, int cap, bool &ok,
                                         uint32_t *status = nullptr, int V = 0) {
    for (int it = 0; it < cap; ++it) {
        const int p = parent[x];
        if (p == x) return x;
#ifdef PTHR_DEBUG
        if (!PTHR_DCHECK(status, p >= 0 && p < V && parent[p] >= 0 && parent[p] < V)) { ok = false; return x; }
#endif
        const int gp = parent[p];
        if (gp != p) parent[x] = gp;   // path halving: gp is an ancestor of x
        x = gp;
    }
    ok = false;
    return x;
}

// The root of x without writing anything.  For flattening after every join
// is done: the forest no longer changes, but other threads are writing the
// final roots, and a path-halving store could replace a final root with an
// intermediate ancestor after its owner wrote it.
__device__ __forceinline__ int find_root_readonly(volatile int *parent, int x, int cap, bool &ok,
                                                  uint32_t *status = nullptr, int V = 0) {
    for (int it = 0; it < cap; ++it) {
        const int p = parent[x];
        if (p == x) return x;
#ifdef PTHR_DEBUG
        if (!PTHR_DCHECK(status, p >= 0 && p < V)) { ok = false; return x; }
#endif
        x = p;
    }
    ok = false;
    return x;
}

__device__ __forceinline__ void unite(volatile int *parent, int a, int b, int cap, bool &ok,
                                      uint32_t *status = nullptr, int V = 0) {
    for (int it = 0; it < cap; ++it) {
        a = find_root(parent, a, cap, ok, status, V);
        b = find_root(parent, b, cap, ok, status, V);
        if (!ok || a == b) return;
        if (a < b) { const int t = a; a = b; b = t; }   // hook the larger root a under b
        const int old = atomicCAS(const_cast<int *>(&parent[a]), a, b);
        if (old == a) return;
    }
    ok = false;
}

// compact_bits, spread_bits and rot_next: bitrows.cuh; sign_nibble: pthr_internal.cuh

// natural site index of byte kk of packed word w
template <int L>
__device__ __forceinline__ int site_of_word(int w, int kk) {
    using Gm = Geom<L>;
    constexpr int W = Gm::W, ROWS = Gm::ROWS;
    const int c = w / (ROWS * W);
    const int g = w - c * ROWS * W;
    const int r = g / W, j = g - (g / W) * W;
    const int y = r % L, z = r / L;
    const int x = 2 * (4 * j + kk) + ((c + y + z) & 1);
    return x + L * r;
}

// FP32 TwoSum pair (h, l) of this thread's share of sum_i sum_mu J_{i,mu}
// s_i s_{i+mu} over the forward bonds of clone S (packed layout).  Every term
// +-J is exact; h + l is the exact sum while l does not round.
// With S2 set, the same for a second clone into (*h2, *l2) in the same pass.
template <int L>
__device__ __forceinline__ void clone_energy_pairs(const uint32_t *S, const float *J, int tid, int T,
                                                   float &h, float &l, const uint32_t *S2 = nullptr,
                                                   float *h2 = nullptr, float *l2 = nullptr) {
    using Gm = Geom<L>;
    constexpr int V = Gm::V, LW = Gm::LAT_WORDS, W = Gm::W, Lh = Gm::Lh;
    for (int w = tid; w < LW; w += T) {
        const int c = w / (Gm::ROWS * W);
        const int g = w - c * Gm::ROWS * W;
        const GroupGeo q = group_geo<L>(g, c);
        const int j = g % W;
        const uint32_t X = 0x3F3F3F3Fu;
        const uint32_t o = S[q.own];
        const uint32_t x = q.par ? __byte_perm(S[q.wA], S[q.wB], q.selx) : S[q.xa];
        // bytes 0x3F where s_i s_{i+mu} = +1, 0xBF where -1
        const uint32_t px = o ^ x ^ X, py = o ^ S[q.yp] ^ X, pz = o ^ S[q.zp] ^ X;
        uint32_t px2 = 0, py2 = 0, pz2 = 0;
        if (S2) {
            const uint32_t o2 = S2[q.own];
            const uint32_t x2 = q.par ? __byte_perm(S2[q.wA], S2[q.wB], q.selx) : S2[q.xa];
            px2 = o2 ^ x2 ^ X;
            py2 = o2 ^ S2[q.yp] ^ X;
            pz2 = o2 ^ S2[q.zp] ^ X;
        }
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            if (!Gm::FULL && 4 * j + kk >= Lh) continue;
            const int i = site_of_word<L>(w, kk);
            const float Jx = J[i], Jy = J[V + i], Jz = J[2 * V + i];
            two_sum_acc(h, l, Jx * spinf(px, kk));
            two_sum_acc(h, l, Jy * spinf(py, kk));
            two_sum_acc(h, l, Jz * spinf(pz, kk));
            if (S2) {
                two_sum_acc(*h2, *l2, Jx * spinf(px2, kk));
                two_sum_acc(*h2, *l2, Jy * spinf(py2, kk));
                two_sum_acc(*h2, *l2, Jz * spinf(pz2, kk));
            }
        }
    }
}

// CAPPED = false: every loop bound is the compile-time constant 4V+64 (the
// production path; a runtime bound makes the labelling loops markedly
// slower).  CAPPED = true: the bound comes from the tuning knob, used only to
// exercise the error path.
template <int L, bool CAPPED>
__device__ __forceinline__ void cluster_block(const ClusterArgs &a, int bid, unsigned char *smem) {
    using Gm = Geom<L>;
    constexpr int V = Gm::V, LW = Gm::LAT_WORDS, W = Gm::W, Lh = Gm::Lh;
    int *parent = reinterpret_cast<int *>(smem);                       // [V]
    int *cnt = parent + V;                                             // [V]
    uint32_t *sa = reinterpret_cast<uint32_t *>(cnt + V);              // [LW]
    uint32_t *sb = sa + LW;                                            // [LW]
    unsigned char *flag = reinterpret_cast<unsigned char *>(sb + LW);  // [V] sign of each root
    uint32_t *qrow = reinterpret_cast<uint32_t *>(flag + ((V + 3) & ~3));  // [L*L] q bits per x row,
                                                                           // later the flip bits
    uint32_t *arow = qrow + L * L;                                     // [L*L] clone a: 1 = spin -1
    int *s_scan = reinterpret_cast<int *>(arow + L * L);               // [blockDim.x] row-count scan
    __shared__ int s_ok;
    __shared__ int s_nneg, s_root, s_nclus, s_nflip;
    __shared__ int s_top[2][32];
    __shared__ double s_E[2];
    __shared__ unsigned long long s_Ei[1];

    const Batch &b = a.b;
    const int n_acu = b.n_acu;
    int t = bid;
    const int k = t % n_acu; t /= n_acu;
    const int P = t % b.NPAIR; t /= b.NPAIR;
    const int s = a.sample_first + t;
    if (!PTHR_DCHECK(b.status, s >= 0 && s < b.S && k < b.NT && P < b.NPAIR)) return;
    if (!b.active[s]) return;
    const uint32_t emcs = b.emcs[s];
    if (!a.label_only && (emcs % (uint32_t)b.acu_interval) != 0u) return;
    const unsigned long long seed = b.seeds[s];
    const int tid = threadIdx.x, T = blockDim.x;
    const int ga = 2 * P, gb = 2 * P + 1;
    const int la = ga * b.NSLOT + b.perm[((size_t)s * b.NR + ga) * b.NSLOT + k];
    const int lb = gb * b.NSLOT + b.perm[((size_t)s * b.NR + gb) * b.NSLOT + k];
    if (!PTHR_DCHECK(b.status, la >= ga * b.NSLOT && la < (ga + 1) * b.NSLOT &&
                                lb >= gb * b.NSLOT && lb < (gb + 1) * b.NSLOT && gb < b.NR)) return;
    const uint32_t pair_id = (uint32_t)(P * b.NT + k);
    uint32_t *ga_ptr = b.spins + ((size_t)s * b.NLAT + la) * b.lat_words;
    uint32_t *gb_ptr = b.spins + ((size_t)s * b.NLAT + lb) * b.lat_words;
    constexpr int LB8 = LW / 8;     // bit words per lattice (bit storage)

    if (tid == 0) { s_ok = 1; s_nneg = 0; s_root = -1; s_nclus = 0; s_nflip = 0; }
    if (tid < 2) s_E[tid] = 0.0;
    if (tid == 0) s_Ei[0] = 0ull;
    if (b.bits) {
        for (int i = tid; i < 2 * LB8; i += T) {
            const int u = i < LB8 ? i : i - LB8;
            uint4 lo, hi;
            expand_bits(i < LB8 ? ga_ptr[u] : gb_ptr[u], lo, hi);
            uint4 *d = reinterpret_cast<uint4 *>((i < LB8 ? sa : sb) + 8 * u);
            d[0] = lo;
            d[1] = hi;
        }
    } else {
        for (int i = tid; i < LW / 4; i += T) {
            reinterpret_cast<uint4 *>(sa)[i] = reinterpret_cast<const uint4 *>(ga_ptr)[i];
            reinterpret_cast<uint4 *>(sb)[i] = reinterpret_cast<const uint4 *>(gb_ptr)[i];
        }
    }
    __syncthreads();
    // q bits of every natural x row r = y + L z: bit x of qrow[r] is 1 iff
    // q_i = -1 at i = x + L r.  The two clones' bytes differ exactly there
    // (0x3F vs 0xBF): one XOR per 4 sites, a multiply gathers the four sign
    // bits, and the two colour rows interleave (colour c holds x = 2m + p_c).
    constexpr uint32_t M = L == 32 ? 0xffffffffu : ((1u << L) - 1u);
    for (int r = tid; r < L * L; r += T) {
        const int y = r % L, z = r / L;
        uint32_t bits[2], abits[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            uint32_t acc = 0, aacc = 0;
#pragma unroll
            for (int j = 0; j < W; ++j) {
                const int w = (c * Gm::ROWS + r) * W + j;
                acc |= sign_nibble(sa[w] ^ sb[w]) << (4 * j);
                aacc |= sign_nibble(sa[w]) << (4 * j);
            }
            bits[c] = acc & ((1u << Lh) - 1u);
            abits[c] = aacc & ((1u << Lh) - 1u);
        }
        const int p0 = (y + z) & 1;
        qrow[r] = (spread_bits(bits[0]) << p0) | (spread_bits(bits[1]) << (p0 ^ 1));
        arow[r] = (spread_bits(abits[0]) << p0) | (spread_bits(abits[1]) << (p0 ^ 1));
    }
    for (int i = tid; i < V; i += T) cnt[i] = 0;
    __syncthreads();
    // 1. runs of equal q along each periodic x row, rooted at their first
    //    site; the last run is rooted at x = 0 when it wraps onto the first
    for (int r = tid; r < L * L; r += T) {
        const int i0 = L * r;
        const uint32_t q = qrow[r];
        const uint32_t st = (q ^ (q << 1)) & M & ~1u;       // bit x >= 1: q[x] != q[x-1]
        const bool wrap = ((q ^ (q >> (L - 1))) & 1u) == 0u;  // q[0] == q[L-1]
        const int last = st ? 31 - __clz(st) : L;            // start of the last run
        int root = i0;
        for (int x = 0; x < L; ++x) {
            if ((st >> x) & 1u) root = i0 + x;
            parent[i0 + x] = (wrap && x >= last) ? i0 : root;
        }
    }
    __syncthreads();
    // 2. join runs across y and z edges, one thread per (row, direction).
    //    Edges join equal q; an edge at x != 0 where no run starts in either
    //    row is implied by the edge at x - 1 and skipped.
    bool ok = true;
    const int cap = CAPPED ? a.iter_cap : 4 * V + 64;
    volatile int *vp = parent;
    for (int tsk = tid; tsk < 2 * L * L; tsk += T) {
        const int r = tsk >> 1;
        const int y = r % L, z = r / L;
        const int r2 = (tsk & 1) ? y + L * ((z + 1) % L) : ((y + 1) % L) + L * z;
        const uint32_t q1 = qrow[r], q2 = qrow[r2];
        uint32_t C = ~(q1 ^ q2) & M & ((q1 ^ (q1 << 1)) | (q2 ^ (q2 << 1)) | 1u);
        while (C) {
            const int x = __ffs(C) - 1;
            C &= C - 1u;
            unite(vp, L * r + x, L * r2 + x, cap, ok, b.status, V);
        }
    }
    __syncthreads();
    // every site points straight at its root; only final roots are written
    // here (no path halving), so after the barrier parent[i] is the root
    for (int i = tid; i < V; i += T) {
        const int r = find_root_readonly(vp, i, cap, ok, b.status, V);
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
    // cluster sizes (statistics): one atomic per distinct root per warp
    for (int i0 = 0; i0 < V; i0 += T) {
        const int i = i0 + tid;
        const int root = i < V ? parent[i] : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, root);
        if (i < V && (tid & 31) == __ffs(peers) - 1) atomicAdd(&cnt[root], __popc(peers));
    }
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
        // single cluster: seed = the floor(u*n)-th q = -1 site (natural
        // order), n = #(q = -1); each thread counts a contiguous range of rows
        const int chunk = (L * L + T - 1) / T;
        const int lo = min(L * L, tid * chunk), hi = min(L * L, lo + chunk);
        int my = 0;
        for (int r = lo; r < hi; ++r) my += __popc(qrow[r]);
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
                for (int r = lo; r < hi; ++r) {
                    uint32_t v = qrow[r];
                    const int c = __popc(v);
                    if (target < seen + c) {
                        for (int m = target - seen; m > 0; --m) v &= v - 1u;
                        s_root = parent[L * r + __ffs(v) - 1];
                        break;
                    }
                    seen += c;
                }
            }
        }
        __syncthreads();
        const int root = s_root;
        for (int i = tid; i < V; i += T)
            if (parent[i] == i) flag[i] = (unsigned char)(i == root);
        __syncthreads();
    }
    // flip bits of every natural x row (bit x set iff the cluster of site
    // x + L r is flipped); the q rows are no longer needed
    uint32_t *frow = qrow;
    int nflip = 0;
    for (int r = tid; r < L * L; r += T) {
        uint32_t f = 0u;
#pragma unroll
        for (int x = 0; x < L; ++x) f |= (uint32_t)flag[parent[L * r + x]] << x;
        frow[r] = f;
        nflip += __popc(f);
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
    for (int o = 16; o > 0; o >>= 1) {
        const int u1 = __shfl_xor_sync(0xffffffffu, t1, o), u2 = __shfl_xor_sync(0xffffffffu, t2, o);
        int n1, n2;
        if (u1 > t1) { n1 = u1; n2 = max(t1, u2); } else { n1 = t1; n2 = max(t2, u1); }
        t1 = n1; t2 = n2;
    }
    if ((tid & 31) == 0) { s_top[0][tid >> 5] = t1; s_top[1][tid >> 5] = t2; }
    __syncthreads();
    // flip both clones word by word: the colour-c bits of the row mask,
    // compacted, give the word's four flip bits
    for (int w = tid; w < LW; w += T) {
        const int c = w / (Gm::ROWS * W);
        const int g = w - c * Gm::ROWS * W;
        const int r = g / W, j = g - r * W;
        const int y = r % L, z = r / L;
        const uint32_t nib = (compact_bits(frow[r] >> ((c + y + z) & 1)) >> (4 * j)) & 0xFu;
        const uint32_t m = ((nib * 0x00204081u) & 0x01010101u) << 7;
        sa[w] ^= m;
        sb[w] ^= m;
    }
    // energies (Eq. (1)).  Only bonds with exactly one flipped end change:
    // for them s'_i s'_j = -s_i s_j, so Delta H_a = sum of 2 J s_i s_j (old
    // spins of clone a).  Such a bond joins sites of opposite q, where the two
    // clones' terms cancel, so H_a + H_b is conserved and Delta H_b =
    // -Delta H_a.  On the coupling grid (every thread's FP32 pair sum a
    // multiple of 2^-18) Delta H_a is summed exactly in integers and both
    // energies are updated exactly in FP64; the energies before are those of
    // the resident spins (every entry point that changes spins recomputes
    // them).  Off the grid both energies are recomputed and reduced in FP64.
    const float *J = b.J + (size_t)s * 3 * V;
    float ha = 0.f, la_ = 0.f;
    for (int r = tid; r < L * L; r += T) {
        const int y = r % L, z = r / L;
        const int ry = ((y + 1) % L) + L * z, rz = y + L * ((z + 1) % L);
        const uint32_t f = frow[r], av = arow[r];
        const uint32_t cut[3] = {f ^ rot_next<L>(f), f ^ frow[ry], f ^ frow[rz]};
        const uint32_t neg[3] = {av ^ rot_next<L>(av), av ^ arow[ry], av ^ arow[rz]};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            uint32_t cb = cut[d];
            while (cb) {
                const int x = __ffs(cb) - 1;
                cb &= cb - 1u;
                const float t = 2.f * J[d * V + L * r + x];
                two_sum_acc(ha, la_, ((neg[d] >> x) & 1u) ? -t : t);
            }
        }
    }
    const float xa = ha * 262144.f, xla = la_ * 262144.f;
    const bool ig = xa == rintf(xa) && xla == rintf(xla) && fabsf(xa) < 536870912.f && fabsf(xla) < 65536.f;
    const bool exact_E = __syncthreads_and(ig) != 0;
    if (exact_E) {
        const int va = __float2int_rn(xa) + __float2int_rn(xla);
        // split so that the 32-lane sums cannot overflow
        const int ah = __reduce_add_sync(0xffffffffu, va >> 12);
        const unsigned al = __reduce_add_sync(0xffffffffu, (unsigned)(va & 0xFFF));
        if ((tid & 31) == 0) atomicAdd(&s_Ei[0], (unsigned long long)((long long)ah * 4096 + (long long)al));
    } else {
        float hb = 0.f, lb_ = 0.f;
        ha = 0.f;
        la_ = 0.f;
        clone_energy_pairs<L>(sa, J, tid, T, ha, la_, sb, &hb, &lb_);
        double ea = (double)ha + (double)la_, eb = (double)hb + (double)lb_;
        for (int o = 16; o > 0; o >>= 1) {
            ea += __shfl_xor_sync(0xffffffffu, ea, o);
            eb += __shfl_xor_sync(0xffffffffu, eb, o);
        }
        if ((tid & 31) == 0) { atomicAdd(&s_E[0], ea); atomicAdd(&s_E[1], eb); }
    }
    __syncthreads();
    if (b.bits) {
        for (int i = tid; i < 2 * LB8; i += T) {
            const int u = i < LB8 ? i : i - LB8;
            const uint4 *w = reinterpret_cast<const uint4 *>((i < LB8 ? sa : sb) + 8 * u);
            (i < LB8 ? ga_ptr : gb_ptr)[u] = pack_bits(w[0], w[1]);
        }
    } else {
        for (int i = tid; i < LW / 4; i += T) {
            reinterpret_cast<uint4 *>(ga_ptr)[i] = reinterpret_cast<const uint4 *>(sa)[i];
            reinterpret_cast<uint4 *>(gb_ptr)[i] = reinterpret_cast<const uint4 *>(sb)[i];
        }
    }
    if (tid == 0) {
        double *E = b.E + (size_t)s * b.NLAT;
        if (exact_E) {
            const double dH = (double)(long long)s_Ei[0] * (1.0 / 262144.0);
            E[la] = E[la] + dH;
            E[lb] = E[lb] - dH;
        } else {
            E[la] = -s_E[0];
            E[lb] = -s_E[1];
        }
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

template <int L, bool CAPPED>
__global__ void __launch_bounds__(512, 4) cluster_kernel(ClusterArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    cluster_block<L, CAPPED>(a, blockIdx.x, smem);
}

// parent, cnt [V] int; both clones [LW]; root flags [V] bytes; q and clone-a
// rows [L*L]; the row-count scan of the single-cluster move [<= 1024] int
template <int L>
size_t cluster_smem(void) {
    using Gm = Geom<L>;
    return (size_t)8 * Gm::V + (size_t)8 * Gm::LAT_WORDS + (size_t)((Gm::V + 3) & ~3) +
           (size_t)8 * L * L + (size_t)4 * 1024 + 16;
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

// The cluster step of a mixed-L group (see kernels.cuh): the blocks of every
// batch's cluster launch, dispatching on its lattice size; block size = the
// largest of the group (every loop strides by the block size).
__global__ void __launch_bounds__(512, 2) group_cluster_kernel(GroupClusterArgs g) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ClusterArgs ca;
    const int i = group_member(g.off, g.n, (int)blockIdx.x);
    if (threadIdx.x == 0) {
        switch (i) {
#define PICK(J) case J: ca = g.a[J]; break;
            PICK(0) PICK(1) PICK(2) PICK(3) PICK(4) PICK(5) PICK(6) PICK(7)
#undef PICK
        }
    }
    __syncthreads();
    const int bid = (int)blockIdx.x - g.off[i];
    switch (ca.b.L) {
#define X(LL) case LL: cluster_block<LL, false>(ca, bid, smem); break;
        X(4) X(6) X(8) X(10) X(12) X(14) X(16)
#undef X
    }
}

}  // namespace

cudaError_t launch_group_cluster(const GroupClusterArgs &g, int blocks, int threads, size_t smem, cudaStream_t st) {
    if (blocks <= 0) return cudaSuccess;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = allow_max_dynamic_smem(group_cluster_kernel);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    group_cluster_kernel<<<blocks, threads, smem, st>>>(g);
    return cudaGetLastError();
}

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
