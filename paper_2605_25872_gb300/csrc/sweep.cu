// sweep.cu -- host side of step (i): shapes and dispatch of the templated
// sweep kernel (sweep_kernel.cuh) over (L, update rule, lattices per thread).
// The instantiations live in sweep_inst_*.cu so that they compile in parallel.
#include "sweep_kernel.cuh"
#include "sweep_table.h"

namespace pthr {

size_t sweep_smem_bytes_for(int L, int K) {
    const size_t lb = (size_t)lattice_words(L) * 4;
    return 12 * lb + (size_t)K * lb;
}

int sweep_groups_for(int L) {
    const int W = (L / 2 + 3) / 4;
    return L * L * W;
}

int sweep_max_k() { return sweep_detail::MAXK; }

// Lattices-per-thread values compiled for (L, rule), ascending.
int sweep_kt_options(int L, int rule, int *out) {
    int n = 0;
#define X(LL, KK) if (L == LL) out[n++] = KK;
    if (rule == PTHR_HEATBATH) { PTHR_SWEEP_HB_TABLE(X) }
    else if (rule == PTHR_MICSA) { PTHR_SWEEP_MICSA_TABLE(X) }
    else { PTHR_SWEEP_METRO_A_TABLE(X) PTHR_SWEEP_METRO_B_TABLE(X) }
#undef X
    return n;
}

cudaError_t launch_sweep(const SweepArgs &a, int blocks, int threads, int KT, cudaStream_t st) {
    const int K = a.K_pt > a.K_res ? a.K_pt : a.K_res;
    const size_t smem = sweep_smem_bytes_for(a.b.L, K);
    cudaError_t e = cudaErrorInvalidValue;
    if (a.b.rule == PTHR_HEATBATH) {
        if (launch_sweep_hb(a, blocks, threads, KT, smem, st, &e)) return e;
    } else if (a.b.rule == PTHR_MICSA) {
        if (launch_sweep_micsa(a, blocks, threads, KT, smem, st, &e)) return e;
    } else {
        if (launch_sweep_metro_a(a, blocks, threads, KT, smem, st, &e)) return e;
        if (launch_sweep_metro_b(a, blocks, threads, KT, smem, st, &e)) return e;
    }
    return cudaErrorInvalidValue;
}

}  // namespace pthr
