// peaks.cu -- microbenchmarks of the on-chip rates that bound the PTHR
// kernels: shared-memory and L2 load bandwidth, and the issue rates of the
// integer-logic (ALU), FP32 FMA, packed f32x2 FMA and FP64 FMA pipes.  The
// sweep kernel is bound by these, not by HBM, so its roofline needs them
// measured on the device it runs on rather than taken from a data sheet.
//
// Every kernel does a known amount of work in loops the compiler cannot
// remove (inline PTX marked volatile, results folded into one word that is
// stored), launched over every SM, and is timed with CUDA events on the
// caller's stream after one warm-up launch.
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace pthr {
namespace {

constexpr int PEAK_THREADS = 512;
constexpr int SMEM_WORDS = 4096;          // uint4 words: 64 KB of shared memory per block

// Shared-memory loads: each thread reads 16 bytes per load; a warp's 32
// loads cover 512 consecutive bytes (four wavefronts, no bank conflict).
// The eight addresses of a loop trip are fixed, so no index arithmetic
// competes with the loads; the loads are volatile, so the compiler cannot
// hoist them out of the loop.
__global__ void __launch_bounds__(PEAK_THREADS) peak_smem_kernel(uint32_t *sink, int iters) {
    extern __shared__ __align__(16) uint4 buf[];
    const int tid = threadIdx.x;
    for (int i = tid; i < SMEM_WORDS; i += blockDim.x) buf[i] = make_uint4(i, i * 3u, i * 5u, i * 7u);
    __syncthreads();
    uint32_t a0 = 0, a1 = 0;
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(buf) + 16u * (uint32_t)tid;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            uint32_t x, y, z, w;
            asm volatile("ld.volatile.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(x), "=r"(y), "=r"(z), "=r"(w) : "r"(base + 16u * 512u * (uint32_t)u));
            a0 ^= x ^ y;
            a1 ^= z ^ w;
        }
    }
    const uint32_t r = a0 ^ a1;
    if (r == 0x9E3779B9u) sink[blockIdx.x] = r;   // practically never; keeps the loads live
}

// L2 loads that bypass L1 (.cg): 16 bytes per thread and load, grid-stride
// over a buffer small enough to stay resident in L2 (n16 a multiple of the
// grid's thread count, so every thread loads the same number of words).
// The pass loop is not unrolled, so each pass issues its loads again.
__global__ void __launch_bounds__(PEAK_THREADS) peak_l2_kernel(const uint4 *buf, size_t n16, uint32_t *sink,
                                                              int passes) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    uint32_t a0 = 0, a1 = 0;
#pragma unroll 1
    for (int p = 0; p < passes; ++p) {
#pragma unroll 4
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) {
            uint32_t x, y, z, w;
            asm volatile("ld.global.cg.v4.u32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(x), "=r"(y), "=r"(z), "=r"(w) : "l"(buf + i));
            a0 ^= x ^ y;
            a1 ^= z ^ w;
        }
    }
    const uint32_t r = a0 ^ a1;
    if (r == 0x9E3779B9u) sink[blockIdx.x] = r;
}

// Eight independent dependency chains per thread, eight instructions per
// chain per iteration: 64 instructions of one kind per loop trip.
__global__ void __launch_bounds__(PEAK_THREADS) peak_alu_kernel(uint32_t *sink, int iters) {
    uint32_t c[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) c[k] = threadIdx.x * (k + 1);
    const uint32_t m1 = blockIdx.x | 1u, m2 = threadIdx.x ^ 0x5bd1e995u;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
#pragma unroll
            for (int k = 0; k < 8; ++k)
                asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(c[k]) : "r"(m1), "r"(m2));
        }
    }
    uint32_t r = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) r ^= c[k];
    if (r == 0x9E3779B9u) sink[blockIdx.x] = r;
}

__global__ void __launch_bounds__(PEAK_THREADS) peak_fma_kernel(uint32_t *sink, int iters) {
    float c[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) c[k] = (float)(threadIdx.x + k);
    const float m = 0.999f, a = 1e-3f * (float)(blockIdx.x & 7);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
#pragma unroll
            for (int k = 0; k < 8; ++k) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(c[k]) : "f"(m), "f"(a));
        }
    }
    float r = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) r += c[k];
    if (r == 1234.5f) sink[blockIdx.x] = 1u;
}

__global__ void __launch_bounds__(PEAK_THREADS) peak_fma2_kernel(uint32_t *sink, int iters) {
    unsigned long long c[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float x = (float)(threadIdx.x + k), y = (float)k;
        asm("mov.b64 %0, {%1, %2};" : "=l"(c[k]) : "f"(x), "f"(y));
    }
    unsigned long long m, a;
    {
        const float mv = 0.999f, av = 1e-3f * (float)(blockIdx.x & 7);
        asm("mov.b64 %0, {%1, %1};" : "=l"(m) : "f"(mv));
        asm("mov.b64 %0, {%1, %1};" : "=l"(a) : "f"(av));
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
#pragma unroll
            for (int k = 0; k < 8; ++k)
                asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(c[k]) : "l"(m), "l"(a));
        }
    }
    unsigned long long r = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) r ^= c[k];
    if (r == 0x9E3779B97F4A7C15ull) sink[blockIdx.x] = 1u;
}

__global__ void __launch_bounds__(PEAK_THREADS) peak_fp64_kernel(uint32_t *sink, int iters) {
    double c[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) c[k] = (double)(threadIdx.x + k);
    const double m = 0.999, a = 1e-3 * (double)(blockIdx.x & 7);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
#pragma unroll
            for (int k = 0; k < 8; ++k) asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(c[k]) : "d"(m), "d"(a));
        }
    }
    double r = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) r += c[k];
    if (r == 1234.5) sink[blockIdx.x] = 1u;
}

}  // namespace

// One timed launch (after one warm-up launch) of microbenchmark `kind`;
// *work receives the bytes moved or instructions executed (thread level),
// *ms the CUDA-event time of the timed launch.
cudaError_t run_peak(int kind, void *scratch, size_t scratch_bytes, cudaStream_t st, double *work, float *ms) {
    if (!scratch || scratch_bytes < PEAK_SINK_BYTES) return cudaErrorInvalidValue;
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    uint32_t *sink = reinterpret_cast<uint32_t *>(scratch);
    const int blocks_per_sm = 2;
    const int grid = nsm * blocks_per_sm;
    if (grid * (int)sizeof(uint32_t) > PEAK_SINK_BYTES) return cudaErrorInvalidValue;
    const double threads = (double)grid * PEAK_THREADS;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    if (e != cudaSuccess) { if (t0) cudaEventDestroy(t0); return e; }
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
        if (rep == 1) e = cudaEventRecord(t0, st);
        if (e != cudaSuccess) break;
        switch (kind) {
        case PTHR_PEAK_SMEM_READ: {
            const int iters = 4096;
            const size_t smem = (size_t)SMEM_WORDS * 16;
            e = cudaFuncSetAttribute(peak_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) break;
            peak_smem_kernel<<<grid, PEAK_THREADS, smem, st>>>(sink, iters);
            *work = threads * iters * 8.0 * 16.0;
            break;
        }
        case PTHR_PEAK_L2_READ: {
            // the buffer past the sink words, at most 16 MB (resident in L2),
            // a whole number of grid-wide rows
            size_t n16 = (scratch_bytes - PEAK_SINK_BYTES) / 16;
            if (n16 > (16u << 20) / 16) n16 = (16u << 20) / 16;
            const size_t row = (size_t)grid * PEAK_THREADS;
            n16 = (n16 / row) * row;
            if (n16 == 0) { e = cudaErrorInvalidValue; break; }
            const int passes = 32;
            const uint4 *buf = reinterpret_cast<const uint4 *>(reinterpret_cast<char *>(scratch) + PEAK_SINK_BYTES);
            peak_l2_kernel<<<grid, PEAK_THREADS, 0, st>>>(buf, n16, sink, passes);
            *work = (double)passes * (double)n16 * 16.0;
            break;
        }
        case PTHR_PEAK_ALU:
            peak_alu_kernel<<<grid, PEAK_THREADS, 0, st>>>(sink, 2048);
            *work = threads * 2048.0 * 64.0;
            break;
        case PTHR_PEAK_FMA:
            peak_fma_kernel<<<grid, PEAK_THREADS, 0, st>>>(sink, 2048);
            *work = threads * 2048.0 * 64.0;
            break;
        case PTHR_PEAK_FMA2:
            peak_fma2_kernel<<<grid, PEAK_THREADS, 0, st>>>(sink, 2048);
            *work = threads * 2048.0 * 64.0;
            break;
        case PTHR_PEAK_FP64:
            peak_fp64_kernel<<<grid, PEAK_THREADS, 0, st>>>(sink, 64);
            *work = threads * 64.0 * 64.0;
            break;
        default:
            e = cudaErrorInvalidValue;
        }
        if (e == cudaSuccess) e = cudaGetLastError();
        if (rep == 1 && e == cudaSuccess) e = cudaEventRecord(t1, st);
    }
    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, t0, t1);
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    return e;
}

}  // namespace pthr
