// sweep_table.h -- compiled (L, lattices per thread) variants of the sweep kernel.
// Lattices per thread KT times lattice lanes P is the lattices per block K;
// the largest KT per L follows the shared-memory bound on K (L = 12 stops at
// 16, the largest that fits two blocks per SM without spilling).
#pragma once

#include <cuda_runtime.h>

#define PTHR_SWEEP_METRO_A_TABLE(X) \
    X(2, 1) X(4, 1) X(4, 2) X(6, 1) X(6, 2) X(6, 4) X(6, 8) X(8, 1) X(8, 2) X(8, 4) X(8, 8) \
    X(10, 1) X(10, 2) X(10, 4) X(10, 8) X(10, 16) X(10, 32) \
    X(12, 1) X(12, 2) X(12, 4) X(12, 8) X(12, 16)
#define PTHR_SWEEP_METRO_B_TABLE(X) \
    X(14, 1) X(14, 2) X(14, 4) X(14, 8) X(14, 16) X(14, 32) \
    X(16, 1) X(16, 2) X(16, 4) X(16, 8) X(16, 16) X(16, 32) \
    X(18, 1) X(18, 2) X(18, 4) X(18, 8) X(18, 16) \
    X(20, 1) X(20, 2) X(20, 4) X(20, 8) X(22, 1) X(22, 2) X(22, 4) X(24, 1) X(24, 2) X(24, 4)
#define PTHR_SWEEP_HB_TABLE(X) \
    X(2, 1) X(4, 2) X(6, 8) X(8, 8) X(10, 32) X(12, 32) X(14, 32) X(16, 32) X(18, 16) X(20, 8) \
    X(22, 4) X(24, 4)
#define PTHR_SWEEP_MICSA_TABLE(X) \
    X(2, 1) X(4, 2) X(6, 8) X(8, 8) X(10, 16) X(12, 16) X(14, 16) X(16, 16) X(18, 16) X(20, 8) \
    X(22, 4) X(24, 4)

namespace pthr {
struct SweepArgs;
bool launch_sweep_metro_a(const SweepArgs &a, int blocks, int threads, int KT, size_t smem,
                          cudaStream_t st, cudaError_t *err);
bool launch_sweep_metro_b(const SweepArgs &a, int blocks, int threads, int KT, size_t smem,
                          cudaStream_t st, cudaError_t *err);
bool launch_sweep_hb(const SweepArgs &a, int blocks, int threads, int KT, size_t smem,
                     cudaStream_t st, cudaError_t *err);
bool launch_sweep_micsa(const SweepArgs &a, int blocks, int threads, int KT, size_t smem,
                        cudaStream_t st, cudaError_t *err);
}  // namespace pthr
