// init.cu -- step a1 (couplings and hot-start state) and the natural-order
// spin import/export used by checkpoints and tests.
#include "kernels.cuh"

namespace pthr {

namespace {

__device__ __forceinline__ void slot_rt(int L, int i, int &word, int &byte) {
    const int W = (L / 2 + 3) / 4;
    const int x = i % L, y = (i / L) % L, z = i / (L * L);
    const int c = (x + y + z) & 1;
    const int r = y + L * z;
    const int m = x >> 1;
    word = (c * L * L + r) * W + (m >> 2);
    byte = m & 3;
}

// Sec. 2: J ~ N(0,1), quenched.  Box-Muller on two 24-bit uniforms
// (u1 in (0,1], u2 in [0,1)), FP64, rounded to the nearest multiple of 2^-18.
// Thread = one Philox call = bonds 4q .. 4q+3 of one sample.
__global__ void couplings_kernel(Batch b, int first, int count) {
    const int V = b.L * b.L * b.L;
    const int nq = (3 * V + 3) / 4;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)count * nq) return;
    const int s = first + (int)(idx / nq);
    const int q = (int)(idx % nq);
    const unsigned long long seed = b.seeds[s];
    const u4 w = philox10((uint32_t)q, 0u, 0u, TAG_COUPLING, (uint32_t)seed, (uint32_t)(seed >> 32));
    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
    const double two_pi = 6.283185307179586476925286766559;
    float *J = b.J + (size_t)s * 3 * V;
#pragma unroll
    for (int pair = 0; pair < 2; ++pair) {
        const double u1 = (double)((ws[2 * pair] >> 8) + 1u) * (1.0 / 16777216.0);
        const double u2 = (double)(ws[2 * pair + 1] >> 8) * (1.0 / 16777216.0);
        const double r = sqrt(-2.0 * log(u1));
        const double th = two_pi * u2;
        const double zc = r * cos(th), zs = r * sin(th);
        const int b0 = 4 * q + 2 * pair;
        if (b0 < 3 * V) J[b0] = (float)(rint(zc * 262144.0) / 262144.0);
        if (b0 + 1 < 3 * V) J[b0 + 1] = (float)(rint(zs * 262144.0) / 262144.0);
    }
}

// Hot start (random spins): site i of lattice lat takes word i&3 of
// (i>>2, lat, 0, TAG_INIT); top bit set -> -1.  Thread = 4 sites.
__global__ void init_spins_kernel(Batch b, int first, int count) {
    const int V = b.L * b.L * b.L;
    const int nq = (V + 3) / 4;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long per_sample = (long long)b.NLAT * nq;
    if (idx >= (long long)count * per_sample) return;
    const int s = first + (int)(idx / per_sample);
    const int rem = (int)(idx % per_sample);
    const int lat = rem / nq, q = rem % nq;
    const unsigned long long seed = b.seeds[s];
    const u4 w = philox10((uint32_t)q, (uint32_t)lat, 0u, TAG_INIT, (uint32_t)seed, (uint32_t)(seed >> 32));
    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
    uint32_t *Sw = b.spins + ((size_t)s * b.NLAT + lat) * b.lat_words;
    unsigned char *S = reinterpret_cast<unsigned char *>(Sw);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int i = 4 * q + k;
        if (i >= V) break;
        int word, byte;
        slot_rt(b.L, i, word, byte);
        if (!b.bits)
            S[4 * word + byte] = (ws[k] >> 31) ? SPIN_DN : SPIN_UP;
        else if (ws[k] >> 31)   // bit storage, cleared before: set the -1 spins
            atomicOr(&Sw[(4 * word + byte) >> 5], 1u << ((4 * word + byte) & 31));
    }
}

// Identity permutations, reservoir ages 0..n_res-1, zero counters.
__global__ void init_meta_kernel(Batch b, int first, int count) {
    const int s = first + blockIdx.x;
    if (s >= first + count) return;
    for (int i = threadIdx.x; i < b.NR * b.NSLOT; i += blockDim.x)
        b.perm[(size_t)s * b.NR * b.NSLOT + i] = i % b.NSLOT;
    const int nres = b.NRES > 0 ? b.NRES : 1;
    for (int i = threadIdx.x; i < b.NR * nres; i += blockDim.x)
        b.age[(size_t)s * b.NR * nres + i] = (uint32_t)(i % nres);
    for (int i = threadIdx.x; i < b.NLAT; i += blockDim.x) {
        b.rt[(size_t)s * b.NLAT + i] = 0;
        b.flips[(size_t)s * b.NLAT + i] = 0ull;
        b.E[(size_t)s * b.NLAT + i] = 0.0;
    }
    for (int i = threadIdx.x; i < b.NR; i += blockDim.x) b.trips[(size_t)s * b.NR + i] = 0;
    for (int i = threadIdx.x; i < b.NR * b.NT; i += blockDim.x) b.ptacc[(size_t)s * b.NR * b.NT + i] = 0;
    for (int i = threadIdx.x; i < b.NT * PTHR_NOBS; i += blockDim.x) b.obs[(size_t)s * b.NT * PTHR_NOBS + i] = 0.0;
    for (int i = threadIdx.x; i < b.NT * 2; i += blockDim.x) b.chaos[(size_t)s * b.NT * 2 + i] = 0.0;
    const int ncs = (b.NPAIR > 0 ? b.NPAIR : 1) * b.NT * 4;
    for (int i = threadIdx.x; i < ncs; i += blockDim.x) b.cstat[(size_t)s * ncs + i] = 0;
    if (threadIdx.x == 0) {
        b.emcs[s] = 0u;
        b.preth[s] = 0u;
        b.active[s] = 1;
    }
}

// After a pre-thermalisation launch of n sweeps: the next one continues the
// sweep index (the launch itself skipped a sample whose index would pass 2^23).
__global__ void advance_pretherm_kernel(Batch b, int first, int count, int n) {
    const int s = first + blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= first + count || !b.active[s]) return;
    const uint32_t p = b.preth[s];
    if ((unsigned long long)p + (unsigned long long)n < (1ull << 23)) b.preth[s] = p + (uint32_t)n;
}

__global__ void export_kernel(Batch b, int8_t *out) {
    const int V = b.L * b.L * b.L;
    const long long n = (long long)b.S * b.NLAT * V;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long lat = idx / V;
        const int i = (int)(idx % V);
        int word, byte;
        slot_rt(b.L, i, word, byte);
        const uint32_t *Sw = b.spins + lat * b.lat_words;
        const bool down = b.bits ? ((Sw[(4 * word + byte) >> 5] >> ((4 * word + byte) & 31)) & 1u) != 0u
                                 : reinterpret_cast<const unsigned char *>(Sw)[4 * word + byte] == SPIN_DN;
        out[idx] = down ? (int8_t)-1 : (int8_t)1;
    }
}

__global__ void import_kernel(Batch b, const int8_t *in) {
    const int V = b.L * b.L * b.L;
    const long long n = (long long)b.S * b.NLAT * V;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long lat = idx / V;
        const int i = (int)(idx % V);
        int word, byte;
        slot_rt(b.L, i, word, byte);
        uint32_t *Sw = b.spins + lat * b.lat_words;
        if (b.bits) {   // other threads set other bits of the same word
            const uint32_t m = 1u << ((4 * word + byte) & 31);
            if (in[idx] < 0) atomicOr(&Sw[(4 * word + byte) >> 5], m);
            else atomicAnd(&Sw[(4 * word + byte) >> 5], ~m);
        } else {
            reinterpret_cast<unsigned char *>(Sw)[4 * word + byte] = (in[idx] < 0) ? SPIN_DN : SPIN_UP;
        }
    }
}

inline int grid_for(long long n, int threads) {
    long long g = (n + threads - 1) / threads;
    return (int)(g < 1 ? 1 : (g > 2147483647LL ? 2147483647LL : g));
}

}  // namespace

cudaError_t launch_couplings_from_seed(const Batch &b, int first, int count, cudaStream_t st) {
    const int V = b.L * b.L * b.L;
    const long long n = (long long)count * ((3 * V + 3) / 4);
    couplings_kernel<<<grid_for(n, 256), 256, 0, st>>>(b, first, count);
    return cudaGetLastError();
}

cudaError_t launch_init_state(const Batch &b, int first, int count, cudaStream_t st) {
    const size_t lat_bytes = (size_t)b.lat_words * 4;
    // every slot +1 first (row padding included): 0x3F bytes, or clear bits
    cudaError_t e = cudaMemsetAsync(reinterpret_cast<unsigned char *>(b.spins) + (size_t)first * b.NLAT * lat_bytes,
                                    b.bits ? 0 : SPIN_UP, (size_t)count * b.NLAT * lat_bytes, st);
    if (e != cudaSuccess) return e;
    const int V = b.L * b.L * b.L;
    const long long n = (long long)count * b.NLAT * ((V + 3) / 4);
    init_spins_kernel<<<grid_for(n, 256), 256, 0, st>>>(b, first, count);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    init_meta_kernel<<<count, 256, 0, st>>>(b, first, count);
    return cudaGetLastError();
}

cudaError_t launch_advance_pretherm(const Batch &b, int first, int count, int n_sweeps, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    advance_pretherm_kernel<<<(count + 255) / 256, 256, 0, st>>>(b, first, count, n_sweeps);
    return cudaGetLastError();
}

cudaError_t launch_export_spins(const Batch &b, int8_t *out, cudaStream_t st) {
    const long long n = (long long)b.S * b.NLAT * b.L * b.L * b.L;
    const int g = grid_for(n, 256);
    export_kernel<<<g > 65535 * 16 ? 65535 * 16 : g, 256, 0, st>>>(b, out);
    return cudaGetLastError();
}

cudaError_t launch_import_spins(const Batch &b, const int8_t *in, cudaStream_t st) {
    const long long n = (long long)b.S * b.NLAT * b.L * b.L * b.L;
    const int g = grid_for(n, 256);
    import_kernel<<<g > 65535 * 16 ? 65535 * 16 : g, 256, 0, st>>>(b, in);
    return cudaGetLastError();
}

}  // namespace pthr
