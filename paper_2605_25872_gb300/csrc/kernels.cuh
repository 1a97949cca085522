// kernels.cuh -- launch interfaces of the PTHR kernels (internal to the library).
#pragma once

#include "pthr_internal.cuh"
#include "pthr_peaks.h"

namespace pthr {

struct SweepArgs {
    Batch b;
    int n_pt_sweeps, n_res_sweeps;       // sweeps per kind in this launch
    int pt_sweep_base, res_sweep_base;   // sweep index of the first sweep in this EMCS
    int K_pt, K_res;                     // lattices per block
    int pt_tasks, res_tasks;             // blocks per sample per kind
    int do_pt, do_res;                   // launch PT / reservoir blocks (0/1)
    int sample_first, sample_count;
    int emcs_override;                   // 1: counter word PRETHERM_EMCS, sweep index
                                         //    from the sample's PRETH counter
    int Gt;                              // groups per lattice lane (divides G and threads)
};

cudaError_t launch_sweep(const SweepArgs &a, int blocks, int threads, int KT, cudaStream_t st);
size_t sweep_smem_bytes_for(int L, int K);
int sweep_groups_for(int L);
int sweep_max_k();
int sweep_kt_options(int L, int rule, int *out);   // compiled lattices-per-thread values

// cluster.cu
struct ClusterArgs {
    Batch b;
    int sample_first, sample_count;
    int label_only;          // 1: only write labels (no flip, no energies)
    int32_t *labels_out;     // optional [S][NPAIR][NT][V] canonical labels
    int iter_cap;            // bound on every union-find loop (> 0)
};
cudaError_t launch_cluster(const ClusterArgs &a, int threads, cudaStream_t st);
size_t cluster_smem_bytes_for(int L);

// exchange.cu
cudaError_t launch_swap(const Batch &b, int flags, int first, int count, cudaStream_t st);
cudaError_t launch_measure(const Batch &b, int first, int count, int chaos, cudaStream_t st);

// init.cu
cudaError_t launch_couplings_from_seed(const Batch &b, int first, int count, cudaStream_t st);
cudaError_t launch_init_state(const Batch &b, int first, int count, cudaStream_t st);
cudaError_t launch_advance_pretherm(const Batch &b, int first, int count, int n_sweeps, cudaStream_t st);
cudaError_t launch_export_spins(const Batch &b, int8_t *out, cudaStream_t st);
cudaError_t launch_import_spins(const Batch &b, const int8_t *in, cudaStream_t st);

// Mixed-L groups: one launch per EMCS step over the blocks of up to
// GROUP_MAX batches (group_sweep.cuh, cluster.cu, exchange.cu).  Block b of
// the launch belongs to batch i with off[i] <= b < off[i+1], as its block
// b - off[i].
constexpr int GROUP_MAX = 8;
struct GroupSweepArgs { int n; int off[GROUP_MAX + 1]; SweepArgs a[GROUP_MAX]; };
struct GroupClusterArgs { int n; int off[GROUP_MAX + 1]; ClusterArgs a[GROUP_MAX]; };
struct GroupBatchArgs { int n; int off[GROUP_MAX + 1]; int flags[GROUP_MAX]; Batch b[GROUP_MAX]; };
bool group_supports_L(int L);
int group_sweep_kt(int L);                 // lattices per thread of the group sweep
cudaError_t launch_group_sweep(const GroupSweepArgs &g, int rule, int blocks, int threads, size_t smem,
                               cudaStream_t st);
cudaError_t launch_group_cluster(const GroupClusterArgs &g, int blocks, int threads, size_t smem, cudaStream_t st);
cudaError_t launch_group_swap(const GroupBatchArgs &g, int blocks, int threads, size_t smem, cudaStream_t st);
cudaError_t launch_group_measure(const GroupBatchArgs &g, int blocks, size_t smem, cudaStream_t st);
size_t measure_smem_bytes_for(int L);

// Block index of a group launch -> batch index (static indices only).
__device__ __forceinline__ int group_member(const int (&off)[GROUP_MAX + 1], int n, int blk) {
    int i = 0;
#pragma unroll
    for (int j = 1; j < GROUP_MAX; ++j)
        if (j < n && blk >= off[j]) i = j;
    return i;
}

// autocorr.cu
cudaError_t launch_snapshot_reservoir(const Batch &b, int first, int count, uint32_t *snap, cudaStream_t st);
cudaError_t launch_reservoir_overlap(const Batch &b, int first, int count, const uint32_t *snap,
                                     long long *out, int n_points, int point, cudaStream_t st);
cudaError_t noalloc_snapshot(void **ptr, size_t *bytes);   // fixed device scratch, per device

// peaks.cu
constexpr int PEAK_SINK_BYTES = 4096;   // scratch words the microbenchmarks may store to
cudaError_t run_peak(int kind, void *scratch, size_t scratch_bytes, cudaStream_t st, double *work, float *ms);

}  // namespace pthr
