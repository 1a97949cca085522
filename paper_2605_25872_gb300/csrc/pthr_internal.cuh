// pthr_internal.cuh -- shared device helpers of the PTHR CUDA library (sm_103a).
//
// Internal spin layout ("packed colour rows").  A lattice is split by the
// checkerboard colour c = (x+y+z)&1.  Row r = y + L*z of colour c holds the
// L/2 sites x = 2m + p, p = (c + y + z)&1, m = 0..L/2-1, one byte each, padded
// to W = ceil((L/2)/4) 32-bit words.  Byte value 0x3F is spin +1, 0xBF spin -1:
// byte_perm(word, 0x80, 0x?455) then yields the FP32 value +-1.0f directly.
// Word index: (c * L*L + r) * W + (m >> 2), byte m & 3.
//
// Spin storage in HBM (pthr_config.spin_layout): either that byte layout, or
// one sign bit per byte slot -- bit 4w + k of a lattice's 32-bit bit words
// (word (4w + k) >> 5, bit (4w + k) & 31) is bit 7 of byte k of packed word w,
// 1 = spin -1, so one bit word holds eight packed words and row padding is
// 0.  Kernels that keep lattices in shared memory expand the bits to the byte
// layout when they stage them and pack them again on write-back.
//
// Random numbers: Philox4x32-10 (Salmon et al., SC'11) keyed by the sample's
// 64-bit seed; counter words (c0, c1, c2, c3) per stream:
//   init spins  (i>>2, lattice, 0, TAG_INIT)              word i & 3
//   sweep       (r*W + (m>>2), lattice, emcs, TAG_SWEEP | c<<8 | sweep<<9)
//                                                        word m & 3
//   MicSA walker (r*W + j, (e>>2) | kind<<24, emcs, TAG_MICSA | c<<8 | sweep<<9)
//                                   word e & 3, e = position within the kind
//   ACU sign    (label, pair*n_temps + k, emcs, TAG_ACU)  word 0, top bit
//   PT          (k, 2*group + phase, emcs, TAG_PT)        word 0
//   single seed (0, pair*n_temps + k, emcs, TAG_SINGLE)   word 0
//   couplings   (bond>>2, 0, 0, TAG_COUPLING)             Box-Muller pair
// Uniform u = (word >> 8) * 2^-24.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pthr.h"

namespace pthr {

constexpr uint32_t TAG_INIT = 0, TAG_SWEEP = 1, TAG_ACU = 2, TAG_PT = 3, TAG_SINGLE = 4,
                   TAG_COUPLING = 5, TAG_MICSA = 7;
constexpr uint32_t PRETHERM_EMCS = 0xFFFFFFFFu;
constexpr uint32_t STATUS_NOCONVERGE = 1u;
constexpr uint32_t STATUS_BOUNDS = 2u;

constexpr unsigned char SPIN_UP = 0x3F, SPIN_DN = 0xBF;

template <int L>
struct Geom {
    static constexpr int Lh = L / 2;
    static constexpr int W = (Lh + 3) / 4;           // words per colour row
    static constexpr int ROWS = L * L;               // rows per colour
    static constexpr int G = ROWS * W;               // 4-site groups per colour
    static constexpr int LAT_WORDS = 2 * ROWS * W;   // 32-bit words per lattice
    static constexpr int LAT_BYTES = 4 * LAT_WORDS;
    static constexpr int V = L * L * L;
    static constexpr bool FULL = (Lh % 4) == 0;      // every group holds 4 sites
};

__host__ __device__ inline int lattice_words(int L) {
    int W = (L / 2 + 3) / 4;
    return 2 * L * L * W;
}

// 32-bit words per lattice in HBM: the byte layout's words, or an eighth of
// them in the bit layout (L even makes lattice_words(L) a multiple of 8)
__host__ __device__ inline int storage_words(int L, int bits) {
    return bits ? lattice_words(L) / 8 : lattice_words(L);
}

// bit 7 of the four bytes of w (the sign of a packed spin, or where two
// packed words differ) as the low four bits; a multiply gathers them
__device__ __forceinline__ uint32_t sign_nibble(uint32_t w) {
    return ((w & 0x80808080u) * 0x00204081u) >> 28;
}

// the inverse: four sign bits as the packed word of their 0x3F / 0xBF bytes
// (the multiply places bit k at bit 8k; the shifted copies fall elsewhere)
__device__ __forceinline__ uint32_t expand_nibble(uint32_t n) {
    return 0x3F3F3F3Fu | (((n * 0x00204081u) & 0x01010101u) << 7);
}

// Packed words 8u .. 8u+7 of a lattice from its bit word u, and back.
__device__ __forceinline__ void expand_bits(uint32_t bw, uint4 &lo, uint4 &hi) {
    lo = make_uint4(expand_nibble(bw & 0xFu), expand_nibble((bw >> 4) & 0xFu),
                    expand_nibble((bw >> 8) & 0xFu), expand_nibble((bw >> 12) & 0xFu));
    hi = make_uint4(expand_nibble((bw >> 16) & 0xFu), expand_nibble((bw >> 20) & 0xFu),
                    expand_nibble((bw >> 24) & 0xFu), expand_nibble(bw >> 28));
}
__device__ __forceinline__ uint32_t pack_bits(const uint4 &lo, const uint4 &hi) {
    return sign_nibble(lo.x) | (sign_nibble(lo.y) << 4) | (sign_nibble(lo.z) << 8) |
           (sign_nibble(lo.w) << 12) | (sign_nibble(hi.x) << 16) | (sign_nibble(hi.y) << 20) |
           (sign_nibble(hi.z) << 24) | (sign_nibble(hi.w) << 28);
}

// Everything a kernel needs about the batch; passed by value.
struct Batch {
    float *J;                 // [S][3][V]
    uint32_t *spins;          // [S][n_lat][lat_words]
    double *E;                // [S][n_lat]
    int32_t *perm;            // [S][NR][NSLOT]
    uint32_t *age;            // [S][NR][max(NRES,1)]
    uint8_t *rt;              // [S][n_lat]
    long long *trips;         // [S][NR]
    long long *ptacc;         // [S][NR][NT]
    unsigned long long *flips;// [S][n_lat]
    double *obs;              // [S][NT][PTHR_NOBS]
    uint32_t *emcs;           // [S]
    unsigned long long *seeds;// [S]
    uint8_t *active;          // [S]
    uint32_t *status;         // [4]
    long long *cstat;         // [S][NPAIR][NT][4]
    double *chaos;            // [S][NT][2]
    uint32_t *preth;          // [S]     reservoir pre-thermalisation sweeps done
    const double *tabT;       // [NT]    T_k
    const double *tabBeta;    // [NT]    1 / T_k
    const double *tabQ;       // [V+1]   (V - 2n) / V
    const double *tabQl;      // [3V+1]  (3V - 2n) / (3V)
    const float *tabTb;       // [NT]    (float)(-2 log2(e) / T_k)
    int S, L, NT, NR, NRES, NSLOT, NLAT, NPAIR, lat_words;   // lat_words: storage words
    int bits;                 // spin storage: 0 bytes, 1 bits (PTHR_SPINS_*)
    int rule, cluster_mode, acu_interval, n_acu;
    double t_min, t_max;
};

// T_k = t_min + k (t_max - t_min) / (n_temps - 1) (App. A.2), evaluated with
// one IEEE rounding per operation in this order (no contraction), so that
// host and device get the same bits.
__host__ __device__ inline double temperature(const Batch &b, int k) {
    if (b.NT == 1) return b.t_min;
#ifdef __CUDA_ARCH__
    return __dadd_rn(b.t_min, __ddiv_rn(__dmul_rn((double)k, __dsub_rn(b.t_max, b.t_min)),
                                        (double)(b.NT - 1)));
#else
    volatile double d = (double)k * (b.t_max - b.t_min);
    volatile double q = d / (double)(b.NT - 1);
    return b.t_min + q;
#endif
}

// ---------------------------------------------------------------- Philox4x32-10
struct u4 { uint32_t x, y, z, w; };

__device__ __forceinline__ u4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                       uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(M0, c0), lo0 = M0 * c0;
        const uint32_t hi1 = __umulhi(M1, c2), lo1 = M1 * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += W0; k1 += W1;
    }
    return u4{c0, c1, c2, c3};
}

__device__ __forceinline__ uint32_t philox_word0(unsigned long long seed, uint32_t c0,
                                                 uint32_t c1, uint32_t c2, uint32_t c3) {
    return philox10(c0, c1, c2, c3, (uint32_t)seed, (uint32_t)(seed >> 32)).x;
}

// 24-bit uniform in [0,1), exact in FP32.
__device__ __forceinline__ float uniform24f(uint32_t x) {
    return __uint2float_rz(x >> 8) * 5.9604644775390625e-08f;
}
__device__ __forceinline__ double uniform24d(uint32_t x) {
    return (double)(x >> 8) * (1.0 / 16777216.0);
}

// byte k of w (0x3F / 0xBF) as the FP32 spin +-1.0f
__device__ __forceinline__ float spinf(uint32_t w, int k) {
    return __uint_as_float(__byte_perm(w, 0x80u, 0x0455u | ((uint32_t)k << 12)));
}

__device__ __forceinline__ float fast_exp2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Error-free FP32 accumulation (hi + lo holds the exact running sum as long as
// lo stays exact): Knuth's TwoSum.
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float t) {
    const float s = hi + t;
    const float bb = s - hi;
    const float e = (hi - (s - bb)) + (t - bb);
    hi = s;
    lo += e;
}

// natural site -> (word index, byte) in the packed colour-row layout
template <int L>
__host__ __device__ __forceinline__ void site_slot(int i, int &word, int &byte) {
    using Gm = Geom<L>;
    const int x = i % L, y = (i / L) % L, z = i / (L * L);
    const int c = (x + y + z) & 1;
    const int r = y + L * z;
    const int m = x >> 1;
    word = (c * Gm::ROWS + r) * Gm::W + (m >> 2);
    byte = m & 3;
}

// Raise a kernel's dynamic shared-memory limit to what the device allows on
// top of the kernel's static shared memory (once per kernel).
template <typename F>
inline cudaError_t allow_max_dynamic_smem(F *kernel) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - (int)fa.sharedSizeBytes);
}

__device__ __forceinline__ void set_status(uint32_t *status, uint32_t bit) {
    atomicOr(status, bit);
}

// Range checks of the debug build (PTHR_DEBUG, the stand-in for a memory
// sanitizer): a failed check latches STATUS_BOUNDS and evaluates to false,
// and the caller then skips or clamps the access, so nothing outside a
// buffer is read or written.  Release builds compile every check away.
#ifdef PTHR_DEBUG
#define PTHR_DCHECK(status, cond) ((cond) ? true : (::pthr::set_status((status), ::pthr::STATUS_BOUNDS), false))
#else
#define PTHR_DCHECK(status, cond) true
#endif

// Supported linear sizes (template instantiations).
#define PTHR_FOR_EACH_L(X) X(2) X(4) X(6) X(8) X(10) X(12) X(14) X(16) X(18) X(20) X(22) X(24)

}  // namespace pthr
