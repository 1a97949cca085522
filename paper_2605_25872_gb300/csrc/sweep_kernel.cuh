// sweep_kernel.cuh -- step (i) of the EMCS (Sec. 3; App. A.1): checkerboard
// Metropolis / heat-bath sweeps of many lattices of one sample per block,
// with the couplings and the spins held in shared memory, followed by every
// swept lattice's FP64 energy (Eq. (1)).
//
// Block = (sample, up to K lattices of one kind: PT clones or reservoir
// clones).  The block loads the sample's couplings (FP32) into shared memory
// in the packed colour-row layout and its lattices' spins (one byte each),
// runs all its sweeps without touching global memory, then writes the spins
// back.  Thread = (lattice lane p, 4-site group g): it owns one 4-site group
// (4 consecutive same-colour sites of a row = one Philox call) of KT
// consecutive lattices, so the group's 24 couplings stay in registers while
// it walks its lattices, and the lattice loop unrolls with immediate
// shared-memory offsets.
//
// Metropolis (App. A.1): with t_i = sum_j J_ij s_i s_j (the six products
// s_i s_j come from one 3-input XOR of the site word with each neighbour
// word), Delta E = 2 t_i and the move is accepted iff u < 2^(tb t_i) with
// tb = -2 log2(e) / T, i.e. iff the FP32 difference u - p is negative; the
// four sign bits of one group become the byte flip mask with three byte
// permutes.  Heat bath: s_i = +1 iff u < 1 / (1 + 2^(tb h_i)).  MicSA
// (App. A.1): a walker per (lattice, 4-site group, colour pass) starts with
// energy -T ln u and pays for the group's flips in order.
#pragma once

#include "kernels.cuh"
#include "geometry.cuh"

namespace pthr {
namespace sweep_detail {

constexpr int MAXK = 64;   // lattices per block

// 32x32 -> 64-bit product as one wide multiply.
__device__ __forceinline__ void mul_wide(uint32_t a, uint32_t b, uint32_t &hi, uint32_t &lo) {
    unsigned long long p;
    asm("mul.wide.u32 %0, %1, %2;" : "=l"(p) : "r"(a), "r"(b));
    lo = (uint32_t)p;
    hi = (uint32_t)(p >> 32);
}

// Philox4x32-10 (Salmon et al., SC'11) of the sweep counter (g, lat, emcs,
// c3), keyed by the sample seed with the ten round keys rk0/rk1 precomputed,
// split by what each part depends on.  A round maps (c0, c1, c2, c3) to
// (hi(M1 c2) ^ c1 ^ rk0[r], lo(M1 c2), hi(M0 c0) ^ c3 ^ rk1[r], lo(M0 c0)).
// In rounds 0-2 some products do not depend on the lattice: M1 * emcs is
// fixed for the block, M0 * g for the group, and with the colour/sweep word
// c3 the round-0 output word 2, then M1 times it and M0 times the round-1
// output word 0, are fixed for a (group, colour, sweep); M0 times the
// round-0 word 0 is fixed for a lattice.  SweepRng holds the group parts
// already combined with their round keys, so a draw costs 15 wide
// multiplies and 17 XORs instead of 20 and 20.
struct SweepRng {
    uint32_t y2;    // lo(M0 * g) ^ rk1[1]
    uint32_t z3;    // lo(M1 * w2) ^ rk0[2], w2 = round-0 output word 2
    uint32_t w3;    // hi(M0 * v0) ^ rk1[2], v0 = round-1 output word 0
    uint32_t clo;   // lo(M0 * v0)
};

// Parts fixed for a (group, colour, sweep): ahi, alo = M0 * g; elo =
// lo(M1 * emcs); c3 = the counter's colour/sweep word.  (Round-0 word 0 is
// hi(M1 * emcs) ^ rk0[0] ^ lat; the block prologue multiplies it per lattice.)
__device__ __forceinline__ SweepRng sweep_rng(uint32_t ahi, uint32_t alo, uint32_t elo,
                                              uint32_t c3, const uint32_t (&rk0)[10],
                                              const uint32_t (&rk1)[10]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t w2 = ahi ^ c3 ^ rk1[0];
    uint32_t bhi, blo, chi, clo;
    mul_wide(M1, w2, bhi, blo);
    const uint32_t v0 = bhi ^ elo ^ rk0[1];
    mul_wide(M0, v0, chi, clo);
    return SweepRng{alo ^ rk1[1], blo ^ rk0[2], chi ^ rk1[2], clo};
}

// Philox4x32-10 of (g, lat, emcs, c3) from the precomputed parts; (ph, pl)
// = M0 * (hi(M1 * emcs) ^ rk0[0] ^ lat), fixed per lattice for a launch.
// Round 2 needs one wide multiply, rounds 3-9 are computed in full.
__device__ __forceinline__ u4 philox10_sweep(uint32_t ph, uint32_t pl, const SweepRng &p,
                                             const uint32_t (&rk0)[10], const uint32_t (&rk1)[10]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    uint32_t hi, lo;
    const uint32_t a2 = ph ^ p.y2, a3 = pl;      // round 1
    mul_wide(M1, a2, hi, lo);                   // round 2, lattice-dependent half
    uint32_t c0 = hi ^ p.z3, c1 = lo, c2 = a3 ^ p.w3, c3 = p.clo;
#pragma unroll
    for (int r = 3; r < 10; ++r) {
        uint32_t hi0, lo0, hi1, lo1;
        mul_wide(M0, c0, hi0, lo0);
        mul_wide(M1, c2, hi1, lo1);
        const uint32_t n0 = hi1 ^ c1 ^ rk0[r];
        const uint32_t n2 = hi0 ^ c3 ^ rk1[r];
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    return u4{c0, c1, c2, c3};
}

// Packed FP32 pairs (Blackwell f32x2 arithmetic): two independent IEEE
// round-to-nearest operations per instruction.
typedef unsigned long long f2;
__device__ __forceinline__ f2 pack2(float a, float b) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void unpack2(f2 v, float &a, float &b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
// Knuth's TwoSum on both halves: hi + lo stays the exact running sum while
// lo does not round.
__device__ __forceinline__ void two_sum2(f2 &hi, f2 &lo, f2 t) {
    const f2 s = add2(hi, t);
    const f2 bb = sub2(s, hi);
    lo = add2(lo, add2(sub2(hi, sub2(s, bb)), sub2(t, bb)));
    hi = s;
}
// spins of sites 2h and 2h+1 of a product word as a packed pair
__device__ __forceinline__ f2 spin_pair(uint32_t w, int h) {
    return pack2(spinf(w, 2 * h), spinf(w, 2 * h + 1));
}

// A coupling on the 2^-18 grid with |J| <= 8: then every partial sum of at
// most six terms +-J is a multiple of 2^-18 below 64 in magnitude, which
// FP32 holds exactly, and so is every local field.
__device__ __forceinline__ bool on_coupling_grid(float j) {
    const float y = j * 262144.f;
    return fabsf(j) <= 8.f && y == rintf(y);
}

// Couplings of the four sites of group g, colour c, in the order +x, -x, +y,
// -y, +z, -z, times `scale`, as packed pairs (sites 0,1 and 2,3); row padding
// sites get zero couplings.
template <int L>
__device__ __forceinline__ void group_couplings(const float *Js, const GroupGeo &q, int g, int c,
                                                float scale, f2 (&Jp)[2][6]) {
    using Gm = Geom<L>;
    constexpr int W = Gm::W, ROWS = Gm::ROWS, Lh = Gm::Lh, LB = Gm::LAT_BYTES;
    const int j = g % W, r = g / W;
    const int y = r % L, z = r / L, cc = c ^ 1;
    const int rym = ((y + L - 1) % L) + L * z, rzm = y + L * ((z + L - 1) % L);
    float Jc[4][6];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        int m = 4 * j + kk;
        const bool pad = !Gm::FULL && m >= Lh;
        if (pad) m = Lh - 1;
        const int so = 4 * q.own + kk;
        const int mxm = q.par ? m : (m + Lh - 1) % Lh;
        const float f = pad ? 0.f : scale;
        Jc[kk][0] = f * Js[so];
        Jc[kk][1] = f * Js[4 * ((cc * ROWS + r) * W) + mxm];
        Jc[kk][2] = f * Js[LB + so];
        Jc[kk][3] = f * Js[LB + 4 * ((cc * ROWS + rym) * W) + m];
        Jc[kk][4] = f * Js[2 * LB + so];
        Jc[kk][5] = f * Js[2 * LB + 4 * ((cc * ROWS + rzm) * W) + m];
    }
#pragma unroll
    for (int n = 0; n < 6; ++n) {
        Jp[0][n] = pack2(Jc[0][n], Jc[1][n]);
        Jp[1][n] = pack2(Jc[2][n], Jc[3][n]);
    }
}

// t_i = sum_j J_ij s_i s_j of the four sites of group q of lattice S, as two
// packed pairs, in the fixed order +x, -x, +y, -y, +z, -z.
__device__ __forceinline__ void group_fields(const uint32_t *S, const GroupGeo &q,
                                             const f2 (&Jp)[2][6], f2 (&tt)[2]) {
    const uint32_t own = S[q.own];
    const uint32_t xa = S[q.xa];
    const uint32_t xs = __byte_perm(S[q.wA], S[q.wB], q.selx);
    const uint32_t wxp = q.par ? xs : xa, wxm = q.par ? xa : xs;
    const uint32_t X = 0x3F3F3F3Fu;
    const uint32_t pxp = own ^ wxp ^ X, pxm = own ^ wxm ^ X;
    const uint32_t pyp = own ^ S[q.yp] ^ X, pym = own ^ S[q.ym] ^ X;
    const uint32_t pzp = own ^ S[q.zp] ^ X, pzm = own ^ S[q.zm] ^ X;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        f2 t = mul2(Jp[h][0], spin_pair(pxp, h));
        t = fma2(Jp[h][1], spin_pair(pxm, h), t);
        t = fma2(Jp[h][2], spin_pair(pyp, h), t);
        t = fma2(Jp[h][3], spin_pair(pym, h), t);
        t = fma2(Jp[h][4], spin_pair(pzp, h), t);
        tt[h] = fma2(Jp[h][5], spin_pair(pzm, h), t);
    }
}

// Sums w and f over the lanes of this warp that share this thread's lattice
// lane (a contiguous run of lanes: group index g0 within a lane of Gt
// groups); the run's first lane (lane 0 or g0 == 0) holds the result.  nl =
// lanes present in the warp, wmask = their mask.
__device__ __forceinline__ void segment_sum(long long &w, unsigned &f, int lane, int nl, int g0,
                                            int Gt, unsigned wmask) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long wu = __shfl_down_sync(wmask, w, o);
        const unsigned fu = __shfl_down_sync(wmask, f, o);
        if (lane + o < nl && g0 + o < Gt) {
            w += wu;
            f += fu;
        }
    }
}

// Groups per lattice lane for size L: all G groups of a colour when G <= 512,
// else the largest proper divisor of G that is at most 512 (the host's block
// shape follows the same rule).
constexpr int groups_per_lane(int G) {
    if (G <= 512) return G;
    for (int d = 2; d <= G; ++d)
        if (G % d == 0 && G / d <= 512) return G / d;
    return 1;
}
// Largest block of size L (whole lattice lanes, at most 512 threads), and the
// blocks per SM to keep registers for: for the Metropolis rule two when two
// such blocks fit at 112 registers a thread (L = 12: 288 threads).
template <int L, int RULE>
struct SweepBounds {
    static constexpr int Gt = groups_per_lane(Geom<L>::G);
    static constexpr int threads = Gt * (512 / Gt);
    static constexpr int min_blocks =
        (RULE == PTHR_METROPOLIS && 65536 / (threads * 112) >= 2) ? 2 : 1;
};

// One block of the sweep launch: block `bid` of the launch described by a,
// dynamic shared memory at smem.  Threads past the block's lattice lanes
// (a launch shared with larger shapes) take part in the barriers only.
template <int L, int RULE, int KT>
__device__ __forceinline__ void sweep_block(const SweepArgs &a, int bid, unsigned char *smem) {
    using Gm = Geom<L>;
    constexpr int W = Gm::W, ROWS = Gm::ROWS, Lh = Gm::Lh, G = Gm::G;
    constexpr int LW = Gm::LAT_WORDS, LB = Gm::LAT_BYTES;
    float *Js = reinterpret_cast<float *>(smem);                       // [3][LB]
    uint32_t *Ss = reinterpret_cast<uint32_t *>(smem + 12 * LB);       // [K][LW]
    __shared__ int s_lat[MAXK];
    __shared__ unsigned int s_flips[MAXK];
    __shared__ double s_E[MAXK];
    __shared__ unsigned long long s_Ei[MAXK];
    // per lattice: M0 * (round-0 word 0) of its draws (hi, lo) and the
    // exponent factor tb, read together with one 16-byte load
    __shared__ uint4 s_lr[MAXK];

    const Batch &b = a.b;
    // ---- decode the task
    int t = bid;
    const int nres_tasks = a.do_res ? a.res_tasks : 0;
    const int nall_res = a.sample_count * nres_tasks;
    int s, kind, chunk;
    if (t < nall_res) { s = a.sample_first + t / nres_tasks; chunk = t % nres_tasks; kind = 1; }
    else {
        t -= nall_res;
        if (!a.do_pt) return;
        s = a.sample_first + t / a.pt_tasks; chunk = t % a.pt_tasks; kind = 0;
    }
    if (!PTHR_DCHECK(b.status, s >= 0 && s < b.S)) return;
    if (!b.active[s]) return;
    const int per = kind ? b.NRES : b.NT;
    const int total = b.NR * per;
    const int Kmax = kind ? a.K_res : a.K_pt;
    const int e0 = chunk * Kmax;
    const int K = min(Kmax, total - e0);
    if (K <= 0) return;
    if (!PTHR_DCHECK(b.status, K <= MAXK)) return;
    const int nsw = kind ? a.n_res_sweeps : a.n_pt_sweeps;
    int sweep_base = kind ? a.res_sweep_base : a.pt_sweep_base;
    if (a.emcs_override) {
        // pre-thermalisation continues the sample's own sweep index; an index
        // past the counter's 23 bits would repeat random numbers: skip
        const uint32_t p = b.preth[s];
        if ((unsigned long long)p + (unsigned long long)nsw >= (1ull << 23)) {
            if (threadIdx.x == 0) set_status(b.status, STATUS_BOUNDS);
            return;
        }
        sweep_base = (int)p;
    }
    const uint32_t emcs = a.emcs_override ? PRETHERM_EMCS : b.emcs[s];
    const unsigned long long seed = b.seeds[s];
    const int tid = threadIdx.x, T = blockDim.x;

    uint32_t rk0[10], rk1[10];
    {
        uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
        for (int r = 0; r < 10; ++r) { rk0[r] = k0; rk1[r] = k1; k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    }
    uint32_t rng_x1, rng_elo;        // parts of every sweep draw fixed for the block
    {
        uint32_t ehi;
        mul_wide(0xCD9E8D57u, emcs, ehi, rng_elo);
        rng_x1 = ehi ^ rk0[0];
    }

    if (tid < K) {
        const int e = e0 + tid;
        const int g = e / per, pos = kind ? b.NT + (e % per) : (e % per);
        int clone = b.perm[((size_t)s * b.NR + g) * b.NSLOT + pos];
        if (!PTHR_DCHECK(b.status, g < b.NR && clone >= 0 && clone < b.NSLOT)) clone = 0;
        s_lat[tid] = g * b.NSLOT + clone;
        // round 1 of every sweep draw of this lattice starts from M0 times
        // its round-0 word 0, which depends on the lattice and the block only
        // (MicSA: the walker draws are keyed by the position e within the
        // kind, four positions per Philox call, instead of by the lattice)
        const uint32_t c1 = RULE == PTHR_MICSA ? ((uint32_t)(e >> 2) | ((uint32_t)kind << 24))
                                                : (uint32_t)(g * b.NSLOT + clone);
        uint32_t ph, pl;
        mul_wide(0xD2511F53u, rng_x1 ^ c1, ph, pl);
        // -2 beta log2(e): exp(-beta dE) = 2^(tb t) with dE = 2 t
        s_lr[tid] = make_uint4(ph, pl, __float_as_uint(b.tabTb[kind ? b.NT - 1 : pos]), 0u);
        s_flips[tid] = 0u;
        s_E[tid] = 0.0;
        s_Ei[tid] = 0ull;
    }
    // ---- couplings -> shared memory, packed colour-row layout; several
    // loads in flight per thread.  Note whether all of them lie on the 2^-18
    // grid with |J| <= 8 (then the energies are summed exactly in integers).
    const float *Jg = b.J + (size_t)s * 3 * Gm::V;
    if (!Gm::FULL)
        for (int i = tid; i < 3 * LB; i += T) Js[i] = 0.f;
    __syncthreads();     // lattice ids and zeroed row padding visible
    bool on_grid = true;
    if (L % 4 == 0) {
        // four consecutive sites x0..x0+3 (x0 a multiple of 4) of one x row
        // per 16-byte load: they alternate colours, and sites x0, x0+2 (and
        // x0+1, x0+3) are adjacent bytes m0, m0+1 of one packed word
        constexpr int JQ = 2;
        for (int t0 = tid; t0 < Gm::V / 4; t0 += JQ * T) {
            float4 jv[JQ][3];
#pragma unroll
            for (int u = 0; u < JQ; ++u) {
                const int t = t0 + u * T;
                if (t < Gm::V / 4) {
#pragma unroll
                    for (int d = 0; d < 3; ++d)
                        jv[u][d] = __ldg(reinterpret_cast<const float4 *>(Jg + d * Gm::V) + t);
                }
            }
#pragma unroll
            for (int u = 0; u < JQ; ++u) {
                const int t = t0 + u * T;
                if (t < Gm::V / 4) {
                    const int i = 4 * t;
                    const int x0 = i % L, r = i / L;
                    const int c0 = (x0 + r % L + r / L) & 1;
                    const int m0 = x0 >> 1;
                    const int s0 = 4 * ((c0 * ROWS + r) * W + (m0 >> 2)) + (m0 & 3);
                    const int s1 = 4 * (((c0 ^ 1) * ROWS + r) * W + (m0 >> 2)) + (m0 & 3);
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        const float4 v = jv[u][d];
                        *reinterpret_cast<float2 *>(Js + d * LB + s0) = make_float2(v.x, v.z);
                        *reinterpret_cast<float2 *>(Js + d * LB + s1) = make_float2(v.y, v.w);
                        on_grid = on_grid && on_coupling_grid(v.x) && on_coupling_grid(v.y) &&
                                  on_coupling_grid(v.z) && on_coupling_grid(v.w);
                    }
                }
            }
        }
    } else {
        constexpr int JU = 4;
        for (int i0 = tid; i0 < Gm::V; i0 += JU * T) {
            float jv[JU][3];
#pragma unroll
            for (int u = 0; u < JU; ++u) {
                const int i = i0 + u * T;
                if (i < Gm::V) {
                    jv[u][0] = __ldg(Jg + i);
                    jv[u][1] = __ldg(Jg + Gm::V + i);
                    jv[u][2] = __ldg(Jg + 2 * Gm::V + i);
                }
            }
#pragma unroll
            for (int u = 0; u < JU; ++u) {
                const int i = i0 + u * T;
                if (i < Gm::V) {
                    int w, by;
                    site_slot<L>(i, w, by);
                    const int slot = 4 * w + by;
                    Js[slot] = jv[u][0];
                    Js[LB + slot] = jv[u][1];
                    Js[2 * LB + slot] = jv[u][2];
                    on_grid = on_grid && on_coupling_grid(jv[u][0]) && on_coupling_grid(jv[u][1]) &&
                              on_coupling_grid(jv[u][2]);
                }
            }
        }
    }
    // ---- spins -> shared memory: all K lattices in one flat loop (bit
    // storage: one bit word expands to eight packed words)
    if (b.bits) {
        constexpr int LB8 = LW / 8;
        const int nq = K * LB8;
        for (int i = tid; i < nq; i += T) {
            const int k = i / LB8;
            uint4 lo, hi;
            expand_bits(b.spins[((size_t)s * b.NLAT + s_lat[k]) * LB8 + (i - k * LB8)], lo, hi);
            uint4 *d = reinterpret_cast<uint4 *>(Ss + k * LW + 8 * (i - k * LB8));
            d[0] = lo;
            d[1] = hi;
        }
    } else {
        constexpr int LQ = LW / 4;
        const int nq = K * LQ;
        constexpr int SU = 4;
        for (int i0 = tid; i0 < nq; i0 += SU * T) {
            uint4 v[SU];
#pragma unroll
            for (int u = 0; u < SU; ++u) {
                const int i = i0 + u * T;
                if (i < nq) {
                    const int k = i / LQ;
                    v[u] = reinterpret_cast<const uint4 *>(
                        b.spins + ((size_t)s * b.NLAT + s_lat[k]) * LW)[i - k * LQ];
                }
            }
#pragma unroll
            for (int u = 0; u < SU; ++u) {
                const int i = i0 + u * T;
                if (i < nq) {
                    const int k = i / LQ;
                    reinterpret_cast<uint4 *>(Ss + k * LW)[i - k * LQ] = v[u];
                }
            }
        }
    }
    const bool exact_E = __syncthreads_and(on_grid) != 0;

    const int Gt = a.Gt;                 // groups per lattice lane pass (divides G)
    const int lane_p = tid / Gt, g0 = tid - lane_p * Gt;
    const int GP = G / Gt;
    const int kbase = lane_p * KT;       // this thread's lattices: kbase .. kbase+KT-1
    const bool warp_uniform = (Gt % 32) == 0;
    uint32_t *Sb = Ss + kbase * LW;
    unsigned nfl[KT];
#pragma unroll
    for (int jj = 0; jj < KT; ++jj) nfl[jj] = 0u;

    // one group per colour (G <= 512): its geometry in both colours, once
    // (not where two blocks share an SM: there the registers are short)
    constexpr bool ONE_G = G <= 512 && SweepBounds<L, RULE>::min_blocks == 1;
    GroupGeo qc0{}, qc1{};
    if (ONE_G) {
        qc0 = group_geo<L>(g0, 0);
        qc1 = group_geo<L>(g0, 1);
    }
    for (int sw = 0; sw < nsw; ++sw) {
        const uint32_t c3base = (RULE == PTHR_MICSA ? TAG_MICSA : TAG_SWEEP) | ((uint32_t)(sweep_base + sw) << 9);
        for (int c = 0; c < 2; ++c) {
            const uint32_t c3 = c3base | ((uint32_t)c << 8);
            for (int gi = 0; gi < GP; ++gi) {
                const int g = g0 + gi * Gt;
                const GroupGeo q = ONE_G ? (c ? qc1 : qc0) : group_geo<L>(g, c);
#ifdef PTHR_DEBUG
                {
                    const int cm = ((c ^ 1) * ROWS + ROWS - 1) * W + W - 1;
                    const bool in = g < G && q.own >= 0 && q.own < LW && q.xa >= 0 && q.xa < LW &&
                                    q.wA >= 0 && q.wA < LW && q.wB >= 0 && q.wB < LW && q.yp >= 0 &&
                                    q.yp < LW && q.ym >= 0 && q.ym < LW && q.zp >= 0 && q.zp < LW &&
                                    q.zm >= 0 && q.zm < LW && 4 * q.own + 3 < LB && 4 * cm + 3 < LB &&
                                    (kbase >= K || kbase + min(KT, K - kbase) <= MAXK);
                    if (!PTHR_DCHECK(b.status, in)) continue;
                }
#endif
                uint32_t ahi, alo;
                mul_wide(0xD2511F53u, (uint32_t)g, ahi, alo);
                const SweepRng rng = sweep_rng(ahi, alo, rng_elo, c3, rk0, rk1);
                const int j = g % W;
                const int cc = c ^ 1;
                const int r = g / W;
                const int y = r % L, z = r / L;
                const int rym = ((y + L - 1) % L) + L * z, rzm = y + L * ((z + L - 1) % L);
                // couplings of the group's 4 sites: +x,-x,+y,-y,+z,-z
                float Jc[4][6];
                if (Gm::FULL) {
                    // no row padding: the four sites' couplings of every
                    // direction but -x are one aligned 16-byte load
                    const float4 px = *reinterpret_cast<const float4 *>(Js + 4 * q.own);
                    const float4 py = *reinterpret_cast<const float4 *>(Js + LB + 4 * q.own);
                    const float4 pz = *reinterpret_cast<const float4 *>(Js + 2 * LB + 4 * q.own);
                    const float4 my = *reinterpret_cast<const float4 *>(
                        Js + LB + 4 * ((cc * ROWS + rym) * W) + 4 * j);
                    const float4 mz = *reinterpret_cast<const float4 *>(
                        Js + 2 * LB + 4 * ((cc * ROWS + rzm) * W) + 4 * j);
                    const float vpx[4] = {px.x, px.y, px.z, px.w}, vpy[4] = {py.x, py.y, py.z, py.w};
                    const float vpz[4] = {pz.x, pz.y, pz.z, pz.w}, vmy[4] = {my.x, my.y, my.z, my.w};
                    const float vmz[4] = {mz.x, mz.y, mz.z, mz.w};
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const int m = 4 * j + kk;
                        const int mxm = q.par ? m : (m + Lh - 1) % Lh;
                        Jc[kk][0] = vpx[kk];
                        Jc[kk][1] = Js[4 * ((cc * ROWS + r) * W) + mxm];
                        Jc[kk][2] = vpy[kk];
                        Jc[kk][3] = vmy[kk];
                        Jc[kk][4] = vpz[kk];
                        Jc[kk][5] = vmz[kk];
                    }
                } else {
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
                }
                // the same couplings as packed pairs (sites 0,1 and 2,3); the x
                // pair is ordered as (aligned word xa, shifted word xs), so the
                // lattice loop needs no select on the row parity
                f2 Jp[2][6];
#pragma unroll
                for (int n = 0; n < 6; ++n) {
                    Jp[0][n] = pack2(Jc[0][n], Jc[1][n]);
                    Jp[1][n] = pack2(Jc[2][n], Jc[3][n]);
                }
                if (q.par) {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const f2 t = Jp[h][0];
                        Jp[h][0] = Jp[h][1];
                        Jp[h][1] = t;
                    }
                }
                // flip-mask bits of the real sites of this group
                uint32_t vmask = 0x80808080u;
                if (!Gm::FULL) {
                    const int nv = Lh - 4 * j;
                    vmask = nv >= 4 ? 0x80808080u : (0x80808080u >> (8 * (4 - nv)));
                }
                u4 walker_rnd{};       // MicSA: one Philox call serves four positions
#pragma unroll
                for (int jj = 0; jj < KT; ++jj) {
                    const int k = kbase + jj;
                    if (k >= K) break;
                    uint32_t *S = Sb + jj * LW;
                    const uint32_t own = S[q.own];
                    const uint32_t xa = S[q.xa];
                    const uint32_t xs = __byte_perm(S[q.wA], S[q.wB], q.selx);
                    const uint32_t wyp = S[q.yp], wym = S[q.ym], wzp = S[q.zp], wzm = S[q.zm];
                    const uint4 lr = s_lr[k];
                    u4 rnd;
                    if (RULE == PTHR_MICSA) {
                        if (jj == 0 || ((e0 + k) & 3) == 0)
                            walker_rnd = philox10_sweep(lr.x, lr.y, rng, rk0, rk1);
                        rnd = walker_rnd;
                    } else {
                        rnd = philox10_sweep(lr.x, lr.y, rng, rk0, rk1);
                    }
                    const uint32_t rw[4] = {rnd.x, rnd.y, rnd.z, rnd.w};
                    const float tb = __uint_as_float(lr.z);
                    uint32_t fm;
                    if (RULE == PTHR_MICSA) {
                        // one walker per (lattice, group, colour pass) with
                        // energy -T ln u; site kk flips iff u < 2^(tb y), y =
                        // D + t_kk, D the share already taken by this pass's
                        // flips (in units of t = Delta E / 2), then D = y
                        const uint32_t X = 0x3F3F3F3Fu;
                        const uint32_t pxa = own ^ xa ^ X, pxs = own ^ xs ^ X;
                        const uint32_t pyp = own ^ wyp ^ X, pym = own ^ wym ^ X;
                        const uint32_t pzp = own ^ wzp ^ X, pzm = own ^ wzm ^ X;
                        float tv[4];
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            f2 tt = mul2(Jp[h][0], spin_pair(pxa, h));
                            tt = fma2(Jp[h][1], spin_pair(pxs, h), tt);
                            tt = fma2(Jp[h][2], spin_pair(pyp, h), tt);
                            tt = fma2(Jp[h][3], spin_pair(pym, h), tt);
                            tt = fma2(Jp[h][4], spin_pair(pzp, h), tt);
                            tt = fma2(Jp[h][5], spin_pair(pzm, h), tt);
                            unpack2(tt, tv[2 * h], tv[2 * h + 1]);
                        }
                        const int sel = (e0 + k) & 3;
                        const uint32_t wsel = sel == 0 ? rw[0] : (sel == 1 ? rw[1] : (sel == 2 ? rw[2] : rw[3]));
                        const float uw = uniform24f(wsel);
                        float D = 0.f;
                        fm = 0u;
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const float y = D + tv[kk];
                            const bool flip = uw < fast_exp2(tb * y);
                            if (flip) {
                                D = y;
                                fm |= 0x80u << (8 * kk);
                            }
                        }
                        fm &= vmask;
                    } else if (RULE == PTHR_METROPOLIS) {
                        // bytes 0x3F where s_i s_j = +1, 0xBF where -1
                        const uint32_t X = 0x3F3F3F3Fu;
                        const uint32_t pxa = own ^ xa ^ X, pxs = own ^ xs ^ X;
                        const uint32_t pyp = own ^ wyp ^ X, pym = own ^ wym ^ X;
                        const uint32_t pzp = own ^ wzp ^ X, pzm = own ^ wzm ^ X;
                        float dv[4];
                        const f2 tb2 = pack2(tb, tb);
                        const f2 sc2 = pack2(5.9604644775390625e-08f, 5.9604644775390625e-08f);
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            // t = sum_j J_ij s_i s_j for sites 2h, 2h+1 (packed)
                            f2 tt = mul2(Jp[h][0], spin_pair(pxa, h));
                            tt = fma2(Jp[h][1], spin_pair(pxs, h), tt);
                            tt = fma2(Jp[h][2], spin_pair(pyp, h), tt);
                            tt = fma2(Jp[h][3], spin_pair(pym, h), tt);
                            tt = fma2(Jp[h][4], spin_pair(pzp, h), tt);
                            tt = fma2(Jp[h][5], spin_pair(pzm, h), tt);
                            float y0, y1;
                            unpack2(mul2(tb2, tt), y0, y1);
                            const f2 negp = pack2(-fast_exp2(y0), -fast_exp2(y1));
                            // u - p < 0  <=>  accept (u = (x >> 8) 2^-24, exact)
                            const f2 u2 = pack2(__uint2float_rz(rw[2 * h] >> 8),
                                                __uint2float_rz(rw[2 * h + 1] >> 8));
                            unpack2(fma2(u2, sc2, negp), dv[2 * h], dv[2 * h + 1]);
                        }
                        // sign byte of each difference -> byte kk of the mask
                        const uint32_t lo = __byte_perm(__float_as_uint(dv[0]), __float_as_uint(dv[1]), 0x0073u);
                        const uint32_t hi = __byte_perm(__float_as_uint(dv[2]), __float_as_uint(dv[3]), 0x7300u);
                        fm = __byte_perm(lo, hi, 0x7610u) & vmask;
                    } else {
                        fm = 0u;
                        const uint32_t wxp = q.par ? xs : xa, wxm = q.par ? xa : xs;
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const float si = spinf(own, kk);
                            float h = Jc[kk][0] * spinf(wxp, kk);
                            h = fmaf(Jc[kk][1], spinf(wxm, kk), h);
                            h = fmaf(Jc[kk][2], spinf(wyp, kk), h);
                            h = fmaf(Jc[kk][3], spinf(wym, kk), h);
                            h = fmaf(Jc[kk][4], spinf(wzp, kk), h);
                            h = fmaf(Jc[kk][5], spinf(wzm, kk), h);
                            const float u = uniform24f(rw[kk]);
                            const float p_up = __frcp_rn(1.f + fast_exp2(tb * h));
                            const bool flip = (u < p_up) != (si > 0.f);
                            fm |= flip ? (0x80u << (8 * kk)) : 0u;
                        }
                        fm &= vmask;
                    }
                    S[q.own] = own ^ fm;
                    nfl[jj] += __popc(fm);
                }
            }
            __syncthreads();
        }
    }

    // ---- energies (Eq. (1)) of the swept lattices and their flip counts
    const int lane = tid & 31;
    const int nl = min(32, T - (tid & ~31));                  // lanes of this warp
    const unsigned wmask = nl == 32 ? 0xffffffffu : ((1u << nl) - 1u);
    if (exact_E) {
        // Every bond joins the two colours, so H = -(sum of t_i over the
        // colour-0 sites).  With the couplings scaled by 2^18 every t_i is an
        // integer below 2^24 in FP32, the packed TwoSum keeps each thread's
        // sum exact, and the sum over threads runs in integers.
        constexpr bool ONE = G <= 512;   // then Gt = G: one group per thread
        GroupGeo q1{};
        f2 J1[2][6];
        if (ONE) {
            q1 = group_geo<L>(g0, 0);
            group_couplings<L>(Js, q1, g0, 0, 262144.f, J1);
        }
#pragma unroll
        for (int jj = 0; jj < KT; ++jj) {
            const int k = kbase + jj;
            const bool mine = k < K;
            int v = 0;
            if (mine) {
                const uint32_t *S = Sb + jj * LW;
                f2 hi = 0ull, lo = 0ull, tt[2];
                if (ONE) {
                    group_fields(S, q1, J1, tt);
                    hi = tt[0];
                    two_sum2(hi, lo, tt[1]);
                } else {
                    for (int gi = 0; gi < GP; ++gi) {
                        const int g = g0 + gi * Gt;
                        const GroupGeo q = group_geo<L>(g, 0);
                        f2 Jq[2][6];
                        group_couplings<L>(Js, q, g, 0, 262144.f, Jq);
                        group_fields(S, q, Jq, tt);
                        two_sum2(hi, lo, tt[0]);
                        two_sum2(hi, lo, tt[1]);
                    }
                }
                float h0, h1, l0, l1;
                unpack2(hi, h0, h1);
                unpack2(lo, l0, l1);
                v = __float2int_rn(h0) + __float2int_rn(h1) + __float2int_rn(l0) + __float2int_rn(l1);
            }
            unsigned nf = nfl[jj];
            if (warp_uniform) {
                // every lane of a warp has the same lattice lane, hence the same
                // k; split v so that the 32-lane sums cannot overflow
                const int shi = __reduce_add_sync(0xffffffffu, v >> 12);
                const unsigned slo = __reduce_add_sync(0xffffffffu, (unsigned)(v & 0xFFF));
                nf = __reduce_add_sync(0xffffffffu, nf);
                if (lane == 0 && mine) {
                    atomicAdd(&s_Ei[k], (unsigned long long)((long long)shi * 4096 + (long long)slo));
                    atomicAdd(&s_flips[k], nf);
                }
            } else {
                long long w = v;
                segment_sum(w, nf, lane, nl, g0, Gt, wmask);
                if ((lane == 0 || g0 == 0) && mine) {
                    atomicAdd(&s_Ei[k], (unsigned long long)w);
                    atomicAdd(&s_flips[k], nf);
                }
            }
        }
    } else {
        // couplings off the grid: each thread sums the forward bonds of its
        // sites in FP32 TwoSum pairs, then FP64 reduction
#pragma unroll
        for (int jj = 0; jj < KT; ++jj) {
            const int k = kbase + jj;
            const bool mine = k < K;
            float hi = 0.f, lo = 0.f;
            if (mine) {
                const uint32_t *S = Sb + jj * LW;
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
            }
            double v = (double)hi + (double)lo;
            unsigned nf = nfl[jj];
            if (warp_uniform) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                nf = __reduce_add_sync(0xffffffffu, nf);
                if (lane == 0 && mine) {
                    atomicAdd(&s_E[k], v);
                    atomicAdd(&s_flips[k], nf);
                }
            } else if (mine) {
                atomicAdd(&s_E[k], v);
                atomicAdd(&s_flips[k], nf);
            }
        }
    }
    __syncthreads();
    // ---- write back: one flat loop over all K lattices
    if (b.bits) {
        constexpr int LB8 = LW / 8;
        const int nq = K * LB8;
        for (int i = tid; i < nq; i += T) {
            const int k = i / LB8;
            const uint4 *w = reinterpret_cast<const uint4 *>(Ss + k * LW + 8 * (i - k * LB8));
            b.spins[((size_t)s * b.NLAT + s_lat[k]) * LB8 + (i - k * LB8)] = pack_bits(w[0], w[1]);
        }
    } else {
        constexpr int LQ = LW / 4;
        const int nq = K * LQ;
        for (int i = tid; i < nq; i += T) {
            const int k = i / LQ;
            reinterpret_cast<uint4 *>(b.spins + ((size_t)s * b.NLAT + s_lat[k]) * LW)[i - k * LQ] =
                reinterpret_cast<const uint4 *>(Ss + k * LW)[i - k * LQ];
        }
    }
    if (tid < K) {
        const size_t li = (size_t)s * b.NLAT + s_lat[tid];
        b.E[li] = exact_E ? (double)(long long)s_Ei[tid] * (-1.0 / 262144.0) : -s_E[tid];
        if (s_flips[tid]) atomicAdd(&b.flips[li], (unsigned long long)s_flips[tid]);
    }
}

template <int L, int RULE, int KT>
__global__ void __launch_bounds__(SweepBounds<L, RULE>::threads, SweepBounds<L, RULE>::min_blocks)
sweep_kernel(SweepArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    sweep_block<L, RULE, KT>(a, blockIdx.x, smem);
}

template <int L, int RULE, int KT>
cudaError_t launch_sweep_tpl(const SweepArgs &a, int blocks, int threads, size_t smem,
                             cudaStream_t st) {
    static bool configured = false;
    if (!configured) {
        cudaError_t e = allow_max_dynamic_smem(sweep_kernel<L, RULE, KT>);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    sweep_kernel<L, RULE, KT><<<blocks, threads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace sweep_detail
}  // namespace pthr
