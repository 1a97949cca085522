// autocorr.cu -- the spin autocorrelation of the reservoir clones at T_max
// (Sec. 3, ER): C(tau) = (1/V) sum_i <s_i(t) s_i(t + tau)>, where s(t) is a
// configuration in equilibrium at T_max and s(t + tau) follows from tau
// full-lattice sweeps at T_max.  The paper calibrates the reservoir
// residence with it (C(960) < 1e-3).
//
// snapshot_kernel copies every reservoir clone of a sample into a scratch
// buffer; overlap_kernel then counts, after each block of sweeps, the sum
// over the clone's sites of s_i(t) s_i(t + tau) in integers (V minus twice
// the sites that differ), summed over the sample's reservoir clones.  The
// sweeps in between are ordinary reservoir pre-thermalisation sweeps.
#include <mutex>

#include "kernels.cuh"

namespace pthr {

// Snapshot storage for pthr_reservoir_autocorrelation_noalloc: a fixed
// device array that every GPU which loads the library holds until the
// process exits.  Host code must not use the name as an address (it is a
// host-side stand-in); noalloc_snapshot() looks the device address up.
constexpr size_t NOALLOC_SNAPSHOT_BYTES = size_t(8) << 20;
static __device__ __align__(256) uint32_t g_noalloc_snapshot[NOALLOC_SNAPSHOT_BYTES / 4];

namespace {

// one block per (sample, reservoir clone): the clone's packed words
__global__ void snapshot_kernel(Batch b, int first, int count, uint32_t *snap) {
    const int t = blockIdx.x;
    const int nres = b.NR * b.NRES;
    const int s = first + t / nres, e = t % nres;
    if (s >= first + count) return;
    const int g = e / b.NRES, r = e % b.NRES;
    int clone = b.perm[((size_t)s * b.NR + g) * b.NSLOT + b.NT + r];
    if (!PTHR_DCHECK(b.status, clone >= 0 && clone < b.NSLOT)) clone = b.NT + r;
    const uint32_t *src = b.spins + ((size_t)s * b.NLAT + g * b.NSLOT + clone) * b.lat_words;
    uint32_t *dst = snap + ((size_t)(s - first) * nres + e) * b.lat_words;
    for (int w = threadIdx.x; w < b.lat_words; w += blockDim.x) dst[w] = src[w];
}

// one block per sample: sum over its reservoir clones and sites of
// s_i(t) s_i(t + tau) = V - 2 #(differing sites), into out[s - first][point]
__global__ void overlap_kernel(Batch b, int first, int count, const uint32_t *snap, long long *out,
                               int n_points, int point) {
    const int s = first + blockIdx.x;
    if (s >= first + count) return;
    const int nres = b.NR * b.NRES;
    const int W = (b.L / 2 + 3) / 4, Lh = b.L / 2;
    int ndiff = 0;
    for (int e = 0; e < nres; ++e) {
        const int g = e / b.NRES, r = e % b.NRES;
        int clone = b.perm[((size_t)s * b.NR + g) * b.NSLOT + b.NT + r];
        if (!PTHR_DCHECK(b.status, clone >= 0 && clone < b.NSLOT)) clone = b.NT + r;
        const uint32_t *cur = b.spins + ((size_t)s * b.NLAT + g * b.NSLOT + clone) * b.lat_words;
        const uint32_t *old = snap + ((size_t)(s - first) * nres + e) * b.lat_words;
        if (b.bits) {                    // one bit per slot; row padding is always 0
            for (int w = threadIdx.x; w < b.lat_words; w += blockDim.x) ndiff += __popc(cur[w] ^ old[w]);
        } else {
            for (int w = threadIdx.x; w < b.lat_words; w += blockDim.x) {
                const int j = w % W;
                const int nv = Lh - 4 * j;   // real sites in this word (the rest is row padding)
                const uint32_t vm = nv >= 4 ? 0x80808080u : (0x80808080u >> (8 * (4 - nv)));
                ndiff += __popc((cur[w] ^ old[w]) & vm);
            }
        }
    }
    __shared__ int s_sum[32];
    ndiff = __reduce_add_sync(0xffffffffu, ndiff);
    if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = ndiff;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long d = 0;
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) d += s_sum[w];
        const long long V = (long long)b.L * b.L * b.L;
        out[(size_t)(s - first) * n_points + point] = (long long)nres * V - 2 * d;
    }
}

}  // namespace

// Device address of g_noalloc_snapshot on the current device: looked up with
// cudaGetSymbolAddress the first time a device asks (with that device
// current), then cached per device.
cudaError_t noalloc_snapshot(void **ptr, size_t *bytes) {
    static std::mutex mu;
    static void *addr[256] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_snapshot);
        if (e != cudaSuccess) return e;
        addr[dev] = p;
    }
    *ptr = addr[dev];
    *bytes = NOALLOC_SNAPSHOT_BYTES;
    return cudaSuccess;
}

cudaError_t launch_snapshot_reservoir(const Batch &b, int first, int count, uint32_t *snap, cudaStream_t st) {
    const int blocks = count * b.NR * b.NRES;
    if (blocks <= 0) return cudaSuccess;
    snapshot_kernel<<<blocks, 256, 0, st>>>(b, first, count, snap);
    return cudaGetLastError();
}

cudaError_t launch_reservoir_overlap(const Batch &b, int first, int count, const uint32_t *snap,
                                     long long *out, int n_points, int point, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    overlap_kernel<<<count, 256, 0, st>>>(b, first, count, snap, out, n_points, point);
    return cudaGetLastError();
}

}  // namespace pthr
