// group_sweep.cuh -- the sweep step of a mixed-L group: one launch runs the
// sweep blocks of every batch of the group (each batch's blocks are those
// of its own sweep launch), dispatching on the batch's lattice size.  Each
// size is compiled with one lattices-per-thread value (group_sweep_kt), and
// the block size is the largest of the group, so a batch's block may have
// threads past its own lattice lanes; they take part in the barriers only.
#pragma once

#include "sweep_kernel.cuh"

namespace pthr {

// lattice sizes compiled into the group kernels
#define PTHR_GROUP_L(X) X(4) X(6) X(8) X(10) X(12) X(14) X(16)

__host__ __device__ constexpr int group_kt_of(int L) { return L <= 4 ? 2 : (L <= 8 ? 8 : 16); }

template <int RULE>
__global__ void __launch_bounds__(512, 1) group_sweep_kernel(GroupSweepArgs g) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ SweepArgs sa;
    const int i = group_member(g.off, g.n, (int)blockIdx.x);
    if (threadIdx.x == 0) {
        switch (i) {
#define PICK(J) case J: sa = g.a[J]; break;
            PICK(0) PICK(1) PICK(2) PICK(3) PICK(4) PICK(5) PICK(6) PICK(7)
#undef PICK
        }
    }
    __syncthreads();
    const int bid = (int)blockIdx.x - g.off[i];
    switch (sa.b.L) {
#define X(LL) case LL: sweep_detail::sweep_block<LL, RULE, group_kt_of(LL)>(sa, bid, smem); break;
        PTHR_GROUP_L(X)
#undef X
    }
}

template <int RULE>
cudaError_t launch_group_sweep_rule(const GroupSweepArgs &g, int blocks, int threads, size_t smem,
                                    cudaStream_t st) {
    static bool configured = false;
    if (!configured) {
        cudaError_t e = allow_max_dynamic_smem(group_sweep_kernel<RULE>);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    group_sweep_kernel<RULE><<<blocks, threads, smem, st>>>(g);
    return cudaGetLastError();
}

}  // namespace pthr
