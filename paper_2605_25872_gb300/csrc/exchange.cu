// exchange.cu -- steps (iii) and (iv) of the EMCS (Sec. 3: PT and ER) and the
// measurement of the observables (Sec. 2, Eqs. (2)-(5)).
//
// swap_kernel: one block per sample, one warp per replica group.  The warp
// holds its group's permutation and energies in shared memory, runs the even
// then the odd phase of the PT round (disjoint pairs, one lane each), marks
// the clone that reached T_min, exchanges the clone at T_max with the oldest
// reservoir clone, and finally the block advances the sample's EMCS counter.
#include "kernels.cuh"
#include "bitrows.cuh"

namespace pthr {

namespace {

constexpr int MAX_SLOT = 256;

// One block of the swap launch (block bid = sample first + bid); warps past
// the batch's groups only take part in the barrier.
__device__ __forceinline__ void swap_block(const Batch &b, int flags, int first, int bid, unsigned char *smem) {
    const int s = first + bid;
    if (!b.active[s]) return;
    const int g = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *s_E = reinterpret_cast<double *>(smem);                    // [NR][NSLOT]
    int *s_perm = reinterpret_cast<int *>(s_E + b.NR * b.NSLOT);       // [NR][NSLOT]
    const uint32_t emcs = b.emcs[s];
    const unsigned long long seed = b.seeds[s];
    if (g < b.NR) {
        int *perm = s_perm + g * b.NSLOT;
        double *Ep = s_E + g * b.NSLOT;
        int32_t *gperm = b.perm + ((size_t)s * b.NR + g) * b.NSLOT;
        for (int i = lane; i < b.NSLOT; i += 32) {
            int v = gperm[i];
            if (!PTHR_DCHECK(b.status, v >= 0 && v < b.NSLOT)) v = i;
            perm[i] = v;
        }
        __syncwarp();
        for (int i = lane; i < b.NT; i += 32) Ep[i] = b.E[(size_t)s * b.NLAT + g * b.NSLOT + perm[i]];
        __syncwarp();
        if (flags & PTHR_SWAP_PT) {
            long long *acc = b.ptacc + ((size_t)s * b.NR + g) * b.NT;
            for (int ph = 0; ph < 2; ++ph) {
                for (int k = ph + 2 * lane; k + 1 < b.NT; k += 64) {
                    const double bk = b.tabBeta[k], bk1 = b.tabBeta[k + 1];
                    const double delta = __dmul_rn(__dsub_rn(bk, bk1), __dsub_rn(Ep[k], Ep[k + 1]));
                    bool accept = delta >= 0.0;
                    if (!accept) {
                        const double u = uniform24d(philox_word0(seed, (uint32_t)k,
                                                                 (uint32_t)(2 * g + ph), emcs, TAG_PT));
                        accept = u < exp(delta);
                    }
                    if (accept) {
                        const int tp = perm[k]; perm[k] = perm[k + 1]; perm[k + 1] = tp;
                        const double te = Ep[k]; Ep[k] = Ep[k + 1]; Ep[k + 1] = te;
                        acc[k] += 1;
                    }
                }
                __syncwarp();
            }
            if (lane == 0) {
                uint8_t *rt = b.rt + (size_t)s * b.NLAT + g * b.NSLOT;
                if (rt[perm[0]] & 1u) rt[perm[0]] |= 2u;
            }
        }
        if ((flags & PTHR_SWAP_ER) && b.NRES > 0 && lane == 0) {
            uint32_t *age = b.age + ((size_t)s * b.NR + g) * b.NRES;
            int best = 0;
            for (int r = 1; r < b.NRES; ++r) if (age[r] > age[best]) best = r;
            const int hot = b.NT - 1, res = b.NT + best;
            const int out = perm[hot], in = perm[res];
            uint8_t *rt = b.rt + (size_t)s * b.NLAT + g * b.NSLOT;
            if ((rt[out] & 3u) == 3u) b.trips[(size_t)s * b.NR + g] += 1;
            rt[out] = 0;
            rt[in] = 1;
            perm[hot] = in;
            perm[res] = out;
            for (int r = 0; r < b.NRES; ++r) age[r] = (r == best) ? 0u : age[r] + 1u;
        }
        __syncwarp();
        for (int i = lane; i < b.NSLOT; i += 32) gperm[i] = perm[i];
    }
    __syncthreads();
    if (threadIdx.x == 0) b.emcs[s] = emcs + 1u;
}

__global__ void swap_kernel(Batch b, int flags, int first) {
    extern __shared__ __align__(16) unsigned char smem[];
    swap_block(b, flags, first, blockIdx.x, smem);
}

constexpr int MEASURE_WARPS = 8;   // (sample, temperature) items per measurement block

// One warp per (sample, temperature index k), eight per block.  Accumulator
// layout per (s, k): [0] measurements, [1] sum e, [2] sum e^2 (over groups),
// [3] sum q, [4] sum q^2, [5] sum q_l, [6] sum S, [7] sum q^4 (over pairs).
//
// For every replica pair the warp builds the q rows of the two clones (one
// L-bit mask per natural x row, bit x set where q_i = -1; each packed word is
// read once, row by row, so a warp's loads are consecutive words) into its
// shared-memory slot, then counts the sites with q_i = -1 and the forward
// links (i, i + mu) with q_i != q_{i+mu} by popcounts of each row against
// its rotation (x), its y + 1 row and its z + 1 row.  Lane P keeps pair P's
// counts.  Then the FP64 quantities of the groups and pairs are evaluated on
// separate lanes, and lane 0 adds them to the accumulators in the fixed
// order (groups, then pairs) with one IEEE rounding per operation.
template <int L>
__device__ __forceinline__ void measure_block(const Batch &b, int first, int count, int chaos, int bid,
                                              unsigned char *smem) {
    using Gm = Geom<L>;
    constexpr int V = Gm::V, ROWS = Gm::ROWS;
    uint32_t *s_q = reinterpret_cast<uint32_t *>(smem);   // [MEASURE_WARPS][ROWS]
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int item = bid * MEASURE_WARPS + wid;
    if (item >= count * b.NT) return;                 // warp-uniform
    const int s = first + item / b.NT, k = item % b.NT;
    if (!PTHR_DCHECK(b.status, s >= 0 && s < b.S)) return;
    if (!b.active[s]) return;
    const int32_t *perm = b.perm + (size_t)s * b.NR * b.NSLOT;
    const int lw = b.lat_words;                       // storage words per lattice
    const uint32_t *spins = b.spins + (size_t)s * b.NLAT * lw;
    uint32_t *qr = s_q + wid * ROWS;
    int tn = 0, td = 0, tc = 0;                       // pair `lane`'s counts
    for (int P = 0; P < b.NPAIR; ++P) {
        const int la = 2 * P * b.NSLOT + perm[2 * P * b.NSLOT + k];
        const int lb = (2 * P + 1) * b.NSLOT + perm[(2 * P + 1) * b.NSLOT + k];
        if (!PTHR_DCHECK(b.status, la >= 2 * P * b.NSLOT && la < (2 * P + 1) * b.NSLOT &&
                                    lb >= (2 * P + 1) * b.NSLOT && lb < (2 * P + 2) * b.NSLOT)) return;
        const uint32_t *A = spins + (size_t)la * lw, *B = spins + (size_t)lb * lw;
        int nneg = 0, ndiff = 0, cneg = 0;
        for (int r = lane; r < ROWS; r += 32) {
            const uint32_t q = b.bits ? diff_row<L, true>(A, B, r) : diff_row<L>(A, B, r);
            qr[r] = q;
            nneg += __popc(q);
        }
        __syncwarp();
        for (int r = lane; r < ROWS; r += 32) {
            const int y = r % L, z = r / L;
            const uint32_t q = qr[r];
            const uint32_t qy = qr[((y + 1) % L) + L * z], qz = qr[y + L * ((z + 1) % L)];
            ndiff += __popc(q ^ rot_next<L>(q)) + __popc(q ^ qy) + __popc(q ^ qz);
        }
        if (chaos) {
            // temperature chaos: clone of group 2P at T_0 against group 2P+1 at T_k
            const uint32_t *A0 = spins + (size_t)(2 * P * b.NSLOT + perm[2 * P * b.NSLOT]) * lw;
            for (int r = lane; r < ROWS; r += 32)
                cneg += __popc(b.bits ? diff_row<L, true>(A0, B, r) : diff_row<L>(A0, B, r));
        }
        __syncwarp();                                 // qr is reused by the next pair
        nneg = __reduce_add_sync(0xffffffffu, nneg);
        ndiff = __reduce_add_sync(0xffffffffu, ndiff);
        cneg = __reduce_add_sync(0xffffffffu, cneg);
        if (lane == P) { tn = nneg; td = ndiff; tc = cneg; }
    }
    // per-group energy density on lane g, per-pair overlaps on lane P
    double e = 0.0, q = 0.0, ql = 0.0, S = 0.0, qc = 0.0;
    // e = H / V (exact scaling when V is a power of two); q, q_l and T_k
    // come from the creation-time tables of the same divisions
    if (lane < b.NR) {
        const int lat = lane * b.NSLOT + perm[lane * b.NSLOT + k];
        const double H = b.E[(size_t)s * b.NLAT + lat];
        e = ((V & (V - 1)) == 0) ? __dmul_rn(H, 1.0 / (double)V) : __ddiv_rn(H, (double)V);
    }
    if (lane < b.NPAIR) {
        const double Tk = b.tabT[k];
        const int la = 2 * lane * b.NSLOT + perm[2 * lane * b.NSLOT + k];
        if (!PTHR_DCHECK(b.status, tn >= 0 && tn <= V && td >= 0 && td <= 3 * V && tc >= 0 && tc <= V)) {
            tn = 0; td = 0; tc = 0;
        }
        q = b.tabQ[tn];
        ql = b.tabQl[td];
        const double Ha = b.E[(size_t)s * b.NLAT + la];
        S = __dadd_rn(__ddiv_rn(Ha, 3.0 * (double)V), __ddiv_rn(__dsub_rn(1.0, ql), Tk));
        qc = b.tabQ[tc];
    }
    double *o = b.obs + ((size_t)s * b.NT + k) * PTHR_NOBS;
    double se = 0.0, se2 = 0.0;
    if (lane == 0) { se = o[1]; se2 = o[2]; }
    for (int g = 0; g < b.NR; ++g) {
        const double eg = __shfl_sync(0xffffffffu, e, g);
        if (lane == 0) {
            se = __dadd_rn(se, eg);
            se2 = __dadd_rn(se2, __dmul_rn(eg, eg));
        }
    }
    if (lane == 0) {
        o[0] = __dadd_rn(o[0], 1.0);
        o[1] = se;
        o[2] = se2;
    }
    double *c = b.chaos + ((size_t)s * b.NT + k) * 2;
    for (int P = 0; P < b.NPAIR; ++P) {
        const double qP = __shfl_sync(0xffffffffu, q, P), qlP = __shfl_sync(0xffffffffu, ql, P);
        const double SP = __shfl_sync(0xffffffffu, S, P), qcP = __shfl_sync(0xffffffffu, qc, P);
        if (lane == 0) {
            const double q2 = __dmul_rn(qP, qP);
            o[3] = __dadd_rn(o[3], qP);
            o[4] = __dadd_rn(o[4], q2);
            o[5] = __dadd_rn(o[5], qlP);
            o[6] = __dadd_rn(o[6], SP);
            o[7] = __dadd_rn(o[7], __dmul_rn(__dmul_rn(q2, qP), qP));
            if (chaos) {
                c[0] = __dadd_rn(c[0], 1.0);
                c[1] = __dadd_rn(c[1], __dmul_rn(qcP, qcP));
            }
        }
    }
}

template <int L>
__global__ void __launch_bounds__(32 * MEASURE_WARPS) measure_kernel(Batch b, int first, int count,
                                                                     int chaos) {
    extern __shared__ __align__(16) unsigned char smem[];
    measure_block<L>(b, first, count, chaos, blockIdx.x, smem);
}

// Swap and measurement steps of a mixed-L group (see kernels.cuh).
__global__ void group_swap_kernel(GroupBatchArgs g) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Batch bb;
    __shared__ int fl;
    const int i = group_member(g.off, g.n, (int)blockIdx.x);
    if (threadIdx.x == 0) {
        switch (i) {
#define PICK(J) case J: bb = g.b[J]; fl = g.flags[J]; break;
            PICK(0) PICK(1) PICK(2) PICK(3) PICK(4) PICK(5) PICK(6) PICK(7)
#undef PICK
        }
    }
    __syncthreads();
    swap_block(bb, fl, 0, (int)blockIdx.x - g.off[i], smem);
}

__global__ void __launch_bounds__(32 * MEASURE_WARPS) group_measure_kernel(GroupBatchArgs g) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Batch bb;
    const int i = group_member(g.off, g.n, (int)blockIdx.x);
    if (threadIdx.x == 0) {
        switch (i) {
#define PICK(J) case J: bb = g.b[J]; break;
            PICK(0) PICK(1) PICK(2) PICK(3) PICK(4) PICK(5) PICK(6) PICK(7)
#undef PICK
        }
    }
    __syncthreads();
    const int bid = (int)blockIdx.x - g.off[i];
    switch (bb.L) {
#define X(LL) case LL: measure_block<LL>(bb, 0, bb.S, 0, bid, smem); break;
        X(4) X(6) X(8) X(10) X(12) X(14) X(16)
#undef X
    }
}

}  // namespace

cudaError_t launch_group_swap(const GroupBatchArgs &g, int blocks, int threads, size_t smem, cudaStream_t st) {
    if (blocks <= 0) return cudaSuccess;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = allow_max_dynamic_smem(group_swap_kernel);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    group_swap_kernel<<<blocks, threads, smem, st>>>(g);
    return cudaGetLastError();
}

cudaError_t launch_group_measure(const GroupBatchArgs &g, int blocks, size_t smem, cudaStream_t st) {
    if (blocks <= 0) return cudaSuccess;
    group_measure_kernel<<<blocks, 32 * MEASURE_WARPS, smem, st>>>(g);
    return cudaGetLastError();
}

size_t measure_smem_bytes_for(int L) { return (size_t)MEASURE_WARPS * L * L * 4; }

cudaError_t launch_swap(const Batch &b, int flags, int first, int count, cudaStream_t st) {
    if (b.NR > 32 || b.NSLOT > MAX_SLOT) return cudaErrorInvalidValue;
    const size_t sm = (size_t)b.NR * b.NSLOT * (sizeof(double) + sizeof(int));
    static bool configured = false;
    if (!configured) {
        cudaError_t e = allow_max_dynamic_smem(swap_kernel);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    swap_kernel<<<count, 32 * b.NR, sm, st>>>(b, flags, first);
    return cudaGetLastError();
}

cudaError_t launch_measure(const Batch &b, int first, int count, int chaos, cudaStream_t st) {
    if (b.NR > 32) return cudaErrorInvalidValue;
    const long items = (long)count * b.NT;
    if (items <= 0) return cudaSuccess;
    const int blocks = (int)((items + MEASURE_WARPS - 1) / MEASURE_WARPS);
#define X(LL) if (b.L == LL) { \
        measure_kernel<LL><<<blocks, 32 * MEASURE_WARPS, measure_smem_bytes_for(LL), st>>>(b, first, count, chaos); \
        return cudaGetLastError(); }
    PTHR_FOR_EACH_L(X)
#undef X
    return cudaErrorInvalidValue;
}

}  // namespace pthr
