// sweep.cu -- step (i) of the EMCS (Sec. 3; App. A.1): checkerboard
// Metropolis / heat-bath sweeps of many lattices of one sample per block,
// with the couplings and the spins held in shared memory, followed by every
// swept lattice's FP64 energy (Eq. (1)).
//
// Block = (sample, up to K lattices of one kind: PT clones or reservoir
// clones).  The block loads the sample's couplings (FP32) into shared memory
// in the packed colour-row layout and its lattices' spins (one byte each),
// runs all its sweeps without touching global memory, then writes the spins
// back.  A thread owns one 4-site group (4 consecutive same-colour sites of a
// row = one Philox call) and loops over its lattices, so the group's 24
// couplings stay in registers across lattices.
#include "pthr_internal.cuh"
#include "kernels.cuh"

namespace pthr {

namespace {

constexpr int MAXK = 64;   // lattices per block (shared-memory bound below)

struct GroupGeo {
    int own, xa, yp, ym, zp, zm;   // word offsets in a lattice
    int wA, wB;                    // words of the shifted x neighbour
    uint32_t selx;                 // byte_perm selector of the shifted x word
    int par;                       // x parity of this row/colour
};

// Geometry of 4-site group g of colour c (see pthr_internal.cuh for layout).
template <int L>
__device__ __forceinline__ GroupGeo group_geo(int g, int c) {
    using Gm = Geom<L>;
    constexpr int W = Gm::W, ROWS = Gm::ROWS, Lh = Gm::Lh;
    GroupGeo q;
    const int r = g / W, j = g - (g / W) * W;
    const int y = r % L, z = r / L;
    const int cc = c ^ 1;
    q.par = (c + y + z) & 1;
    const int ryp = ((y + 1) % L) + L * z, rym = ((y + L - 1) % L) + L * z;
    const int rzp = y + L * ((z + 1) % L), rzm = y + L * ((z + L - 1) % L);
    q.own = (c * ROWS + r) * W + j;
    const int rowcc = (cc * ROWS + r) * W;
    q.xa = rowcc + j;
    q.yp = (cc * ROWS + ryp) * W + j;
    q.ym = (cc * ROWS + rym) * W + j;
    q.zp = (cc * ROWS + rzp) * W + j;
    q.zm = (cc * ROWS + rzm) * W + j;
    // Shifted x neighbour: m' = m - 1 (par 0, the -x neighbour) or m + 1
    // (par 1, the +x neighbour), cyclic in [0, Lh).
    const int d = q.par ? 1 : Lh - 1;
    int wa = -1, wb = -1;
    uint32_t sel = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int m = 4 * j + k;
        if (m >= Lh) m = Lh - 1;              // padding byte: any valid source
        const int mp = (m + d) % Lh;
        const int w = mp >> 2, by = mp & 3;
        int src;
        if (wa < 0 || wa == w) { wa = w; src = by; }
        else { wb = w; src = 4 + by; }
        sel |= (uint32_t)src << (4 * k);
    }
    if (wb < 0) wb = wa;
    q.wA = rowcc + wa;
    q.wB = rowcc + wb;
    q.selx = sel;
    return q;
}

template <int L, int RULE>
__global__ void __launch_bounds__(512) sweep_kernel(SweepArgs a) {
    using Gm = Geom<L>;
    constexpr int W = Gm::W, ROWS = Gm::ROWS, Lh = Gm::Lh, G = Gm::G;
    constexpr int LW = Gm::LAT_WORDS, LB = Gm::LAT_BYTES;
    extern __shared__ __align__(16) unsigned char smem[];
    float *Js = reinterpret_cast<float *>(smem);                       // [3][LB]
    uint32_t *Ss = reinterpret_cast<uint32_t *>(smem + 12 * LB);       // [K][LW]
    __shared__ int s_lat[MAXK];
    __shared__ float s_tb[MAXK];
    __shared__ unsigned int s_flips[MAXK];
    __shared__ double s_E[MAXK];

    const Batch &b = a.b;
    // ---- decode the task
    int t = blockIdx.x;
    const int nres_tasks = a.do_res ? a.res_tasks : 0;
    const int nall_res = a.sample_count * nres_tasks;
    int s, kind, chunk;
    if (t < nall_res) { s = a.sample_first + t / nres_tasks; chunk = t % nres_tasks; kind = 1; }
    else {
        t -= nall_res;
        if (!a.do_pt) return;
        s = a.sample_first + t / a.pt_tasks; chunk = t % a.pt_tasks; kind = 0;
    }
    if (!b.active[s]) return;
    const int per = kind ? b.NRES : b.NT;
    const int total = b.NR * per;
    const int Kmax = kind ? a.K_res : a.K_pt;
    const int e0 = chunk * Kmax;
    const int K = min(Kmax, total - e0);
    if (K <= 0) return;
    const int nsw = kind ? a.n_res_sweeps : a.n_pt_sweeps;
    const int sweep_base = kind ? a.res_sweep_base : a.pt_sweep_base;
    const uint32_t emcs = a.emcs_override ? PRETHERM_EMCS : b.emcs[s];
    const unsigned long long seed = b.seeds[s];
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const int tid = threadIdx.x, T = blockDim.x;

    if (tid < K) {
        const int e = e0 + tid;
        const int g = e / per, pos = kind ? b.NT + (e % per) : (e % per);
        const int clone = b.perm[((size_t)s * b.NR + g) * b.NSLOT + pos];
        s_lat[tid] = g * b.NSLOT + clone;
        const double T_k = temperature(b, kind ? b.NT - 1 : pos);
        // -2 beta log2(e): exp(-beta dE) = 2^(s_i * tb * h) with dE = 2 s_i h
        s_tb[tid] = (float)(-2.0 * 1.4426950408889634073599 / T_k);
        s_flips[tid] = 0u;
        s_E[tid] = 0.0;
    }
    // ---- couplings -> shared memory, packed colour-row layout
    const float *Jg = b.J + (size_t)s * 3 * Gm::V;
    if (!Gm::FULL) {
        for (int i = tid; i < 3 * LB; i += T) Js[i] = 0.f;
        __syncthreads();
    }
    for (int i = tid; i < Gm::V; i += T) {
        int w, by;
        site_slot<L>(i, w, by);
        const int slot = 4 * w + by;
        Js[slot] = Jg[i];
        Js[LB + slot] = Jg[Gm::V + i];
        Js[2 * LB + slot] = Jg[2 * Gm::V + i];
    }
    __syncthreads();
    // ---- spins -> shared memory
    for (int k = 0; k < K; ++k) {
        const uint4 *src = reinterpret_cast<const uint4 *>(
            b.spins + ((size_t)s * b.NLAT + s_lat[k]) * LW);
        uint4 *dst = reinterpret_cast<uint4 *>(Ss + k * LW);
        for (int i = tid; i < LW / 4; i += T) dst[i] = src[i];
    }
    __syncthreads();

    const int Gt = a.Gt;                 // groups handled per "lane" pass
    const int P = T / Gt;                // lattice lanes
    const int lane_p = tid / Gt, g0 = tid - lane_p * Gt;
    const int GP = G / Gt;
    const bool warp_uniform = (Gt % 32) == 0;

    for (int sw = 0; sw < nsw; ++sw) {
        const uint32_t c3base = TAG_SWEEP | ((uint32_t)(sweep_base + sw) << 9);
        for (int c = 0; c < 2; ++c) {
            for (int gi = 0; gi < GP; ++gi) {
                const int g = g0 + gi * Gt;
                const GroupGeo q = group_geo<L>(g, c);
                const int j = g % W;
                // couplings of the group's 4 sites: +x,-x,+y,-y,+z,-z
                float Jc[4][6];
                const int cc = c ^ 1;
                const int r = g / W;
                const int y = r % L, z = r / L;
                const int rym = ((y + L - 1) % L) + L * z, rzm = y + L * ((z + L - 1) % L);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    int m = 4 * j + kk;
                    if (m >= Lh) m = Lh - 1;
                    const int so = 4 * q.own + kk;
                    const int mxm = q.par ? m : (m + Lh - 1) % Lh;
                    Jc[kk][0] = Js[so];
                    Jc[kk][1] = Js[4 * ((cc * ROWS + r) * W) + mxm];
                    Jc[kk][2] = Js[LB + so];
                    Jc[kk][3] = Js[LB + 4 * ((cc * ROWS + rym) * W) + m];
                    Jc[kk][4] = Js[2 * LB + so];
                    Jc[kk][5] = Js[2 * LB + 4 * ((cc * ROWS + rzm) * W) + m];
                }
                const uint32_t c3 = c3base | ((uint32_t)c << 8);
                for (int k = lane_p; k < K; k += P) {
                    uint32_t *S = Ss + k * LW;
                    const uint32_t own = S[q.own];
                    const uint32_t xa = S[q.xa];
                    const uint32_t xs = __byte_perm(S[q.wA], S[q.wB], q.selx);
                    const uint32_t wxp = q.par ? xs : xa, wxm = q.par ? xa : xs;
                    const uint32_t wyp = S[q.yp], wym = S[q.ym], wzp = S[q.zp], wzm = S[q.zm];
                    const u4 rnd = philox10((uint32_t)g, (uint32_t)s_lat[k], emcs, c3, k0, k1);
                    const uint32_t rw[4] = {rnd.x, rnd.y, rnd.z, rnd.w};
                    const float tb = s_tb[k];
                    uint32_t fm = 0;
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        if (!Gm::FULL && 4 * j + kk >= Lh) continue;
                        const float si = spinf(own, kk);
                        float h = Jc[kk][0] * spinf(wxp, kk);
                        h = fmaf(Jc[kk][1], spinf(wxm, kk), h);
                        h = fmaf(Jc[kk][2], spinf(wyp, kk), h);
                        h = fmaf(Jc[kk][3], spinf(wym, kk), h);
                        h = fmaf(Jc[kk][4], spinf(wzp, kk), h);
                        h = fmaf(Jc[kk][5], spinf(wzm, kk), h);
                        const float u = uniform24f(rw[kk]);
                        bool flip;
                        if (RULE == PTHR_METROPOLIS) {
                            const float yv = (si * tb) * h;      // -beta dE log2(e)
                            flip = (yv >= 0.f) || (u < fast_exp2(yv));
                        } else {
                            const float p_up = __frcp_rn(1.f + fast_exp2(tb * h));
                            flip = (u < p_up) != (si > 0.f);
                        }
                        fm |= flip ? (0x80u << (8 * kk)) : 0u;
                    }
                    S[q.own] = own ^ fm;
                    const unsigned nf = __popc(fm);
                    if (warp_uniform) {
                        const unsigned tot = __reduce_add_sync(0xffffffffu, nf);
                        if ((tid & 31) == 0 && tot) atomicAdd(&s_flips[k], tot);
                    } else if (nf) {
                        atomicAdd(&s_flips[k], nf);
                    }
                }
            }
            __syncthreads();
        }
    }

    // ---- energies (Eq. (1)) of the swept lattices: each thread sums the
    // forward bonds of its sites exactly in FP32 pairs, then FP64 reduction.
    for (int k = lane_p; k < K; k += P) {
        const uint32_t *S = Ss + k * LW;
        float hi = 0.f, lo = 0.f;
        for (int gi = 0; gi < GP; ++gi) {
            const int g = g0 + gi * Gt;
            const int j = g % W;
            for (int c = 0; c < 2; ++c) {
                const GroupGeo q = group_geo<L>(g, c);
                const uint32_t own = S[q.own];
                const uint32_t xa = S[q.xa];
                const uint32_t xs = __byte_perm(S[q.wA], S[q.wB], q.selx);
                const uint32_t wxp = q.par ? xs : xa;
                const uint32_t wyp = S[q.yp], wzp = S[q.zp];
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    if (!Gm::FULL && 4 * j + kk >= Lh) continue;
                    const int so = 4 * q.own + kk;
                    const float si = spinf(own, kk);
                    two_sum_acc(hi, lo, si * (Js[so] * spinf(wxp, kk)));
                    two_sum_acc(hi, lo, si * (Js[LB + so] * spinf(wyp, kk)));
                    two_sum_acc(hi, lo, si * (Js[2 * LB + so] * spinf(wzp, kk)));
                }
            }
        }
        double v = (double)hi + (double)lo;
        if (warp_uniform) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if ((tid & 31) == 0) atomicAdd(&s_E[k], v);
        } else {
            atomicAdd(&s_E[k], v);
        }
    }
    __syncthreads();
    // ---- write back
    for (int k = 0; k < K; ++k) {
        uint4 *dst = reinterpret_cast<uint4 *>(b.spins + ((size_t)s * b.NLAT + s_lat[k]) * LW);
        const uint4 *src = reinterpret_cast<const uint4 *>(Ss + k * LW);
        for (int i = tid; i < LW / 4; i += T) dst[i] = src[i];
    }
    if (tid < K) {
        const size_t li = (size_t)s * b.NLAT + s_lat[tid];
        b.E[li] = -s_E[tid];
        if (s_flips[tid]) atomicAdd(&b.flips[li], (unsigned long long)s_flips[tid]);
    }
}

template <int L>
size_t sweep_smem_bytes(int K) {
    return (size_t)12 * Geom<L>::LAT_BYTES + (size_t)K * Geom<L>::LAT_BYTES;
}

template <int L>
int groups_per_colour() { return Geom<L>::G; }

template <int L, int RULE>
cudaError_t launch_sweep_L(const SweepArgs &a, int blocks, int threads, cudaStream_t st) {
    const int K = a.K_pt > a.K_res ? a.K_pt : a.K_res;
    const size_t sm = sweep_smem_bytes<L>(K);
    static bool configured = false;
    if (!configured) {
        cudaError_t e = allow_max_dynamic_smem(sweep_kernel<L, RULE>);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    sweep_kernel<L, RULE><<<blocks, threads, sm, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

size_t sweep_smem_bytes_for(int L, int K) {
#define X(LL) if (L == LL) return sweep_smem_bytes<LL>(K);
    PTHR_FOR_EACH_L(X)
#undef X
    return 0;
}

int sweep_groups_for(int L) {
#define X(LL) if (L == LL) return groups_per_colour<LL>();
    PTHR_FOR_EACH_L(X)
#undef X
    return 0;
}

int sweep_max_k() { return MAXK; }

cudaError_t launch_sweep(const SweepArgs &a, int blocks, int threads, cudaStream_t st) {
    const int L = a.b.L;
#define X(LL)                                                                      \
    if (L == LL) return a.b.rule == PTHR_HEATBATH                                  \
                            ? launch_sweep_L<LL, PTHR_HEATBATH>(a, blocks, threads, st) \
                            : launch_sweep_L<LL, PTHR_METROPOLIS>(a, blocks, threads, st);
    PTHR_FOR_EACH_L(X)
#undef X
    return cudaErrorInvalidValue;
}

}  // namespace pthr
