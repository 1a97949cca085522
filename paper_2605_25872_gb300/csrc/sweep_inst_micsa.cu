// sweep_inst_micsa.cu -- instantiations of the sweep kernel (PTHR_SWEEP_MICSA_TABLE).
#include "sweep_kernel.cuh"
#include "sweep_table.h"

namespace pthr {

bool launch_sweep_micsa(const SweepArgs &a, int blocks, int threads, int KT, size_t smem,
                          cudaStream_t st, cudaError_t *err) {
#define X(LL, KK)                                                                          \
    if (a.b.L == LL && KT == KK) {                                                         \
        *err = sweep_detail::launch_sweep_tpl<LL, PTHR_MICSA, KK>(a, blocks, threads, smem, st); \
        return true;                                                                       \
    }
    PTHR_SWEEP_MICSA_TABLE(X)
#undef X
    return false;
}

}  // namespace pthr
