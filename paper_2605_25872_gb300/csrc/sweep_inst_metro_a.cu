// sweep_inst_metro_a.cu -- instantiations of the sweep kernel (PTHR_SWEEP_METRO_A_TABLE).
#include "sweep_kernel.cuh"
#include "sweep_table.h"

namespace pthr {

bool launch_sweep_metro_a(const SweepArgs &a, int blocks, int threads, int KT, size_t smem,
                          cudaStream_t st, cudaError_t *err) {
#define X(LL, KK)                                                                          \
    if (a.b.L == LL && KT == KK) {                                                         \
        *err = sweep_detail::launch_sweep_tpl<LL, PTHR_METROPOLIS, KK>(a, blocks, threads, smem, st); \
        return true;                                                                       \
    }
    PTHR_SWEEP_METRO_A_TABLE(X)
#undef X
    return false;
}

}  // namespace pthr
