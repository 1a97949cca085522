// group_sweep_heatbath.cu -- the mixed-L group sweep for the heatbath rule.
#include "group_sweep.cuh"

namespace pthr {

cudaError_t launch_group_sweep_heatbath(const GroupSweepArgs &g, int blocks, int threads, size_t smem,
                                       cudaStream_t st) {
    return launch_group_sweep_rule<PTHR_HEATBATH>(g, blocks, threads, smem, st);
}

}  // namespace pthr
