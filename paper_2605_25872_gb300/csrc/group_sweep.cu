// group_sweep.cu -- instantiations and dispatch of the mixed-L group sweep.
#include "group_sweep.cuh"  // PTHR_GROUP_L, group_kt_of

namespace pthr {

bool group_supports_L(int L) {
#define X(LL) if (L == LL) return true;
    PTHR_GROUP_L(X)
#undef X
    return false;
}

int group_sweep_kt(int L) { return group_kt_of(L); }

// the three update rules are instantiated in group_sweep_rules.cu (one
// translation unit per rule, compiled in parallel)
cudaError_t launch_group_sweep_metropolis(const GroupSweepArgs &g, int blocks, int threads, size_t smem, cudaStream_t st);
cudaError_t launch_group_sweep_heatbath(const GroupSweepArgs &g, int blocks, int threads, size_t smem, cudaStream_t st);
cudaError_t launch_group_sweep_micsa(const GroupSweepArgs &g, int blocks, int threads, size_t smem, cudaStream_t st);

cudaError_t launch_group_sweep(const GroupSweepArgs &g, int rule, int blocks, int threads, size_t smem,
                               cudaStream_t st) {
    if (blocks <= 0) return cudaSuccess;
    if (rule == PTHR_METROPOLIS) return launch_group_sweep_metropolis(g, blocks, threads, smem, st);
    if (rule == PTHR_HEATBATH) return launch_group_sweep_heatbath(g, blocks, threads, smem, st);
    if (rule == PTHR_MICSA) return launch_group_sweep_micsa(g, blocks, threads, smem, st);
    return cudaErrorInvalidValue;
}

}  // namespace pthr
