// bitrows.cuh -- the q (or spin) values of one natural x row as an L-bit
// mask, built from the two colour rows of the packed layout (shared by the
// cluster and measurement kernels).
#pragma once

#include "geometry.cuh"

namespace pthr {

// bit m of v -> bit 2m (m < 16)
__device__ __forceinline__ uint32_t spread_bits(uint32_t v) {
    v = (v | (v << 8)) & 0x00FF00FFu;
    v = (v | (v << 4)) & 0x0F0F0F0Fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}

// bit 2m of v -> bit m
__device__ __forceinline__ uint32_t compact_bits(uint32_t v) {
    v &= 0x55555555u;
    v = (v | (v >> 1)) & 0x33333333u;
    v = (v | (v >> 2)) & 0x0F0F0F0Fu;
    v = (v | (v >> 4)) & 0x00FF00FFu;
    v = (v | (v >> 8)) & 0x0000FFFFu;
    return v;
}

// L-bit row rotated so that bit x holds bit (x + 1) mod L
template <int L>
__device__ __forceinline__ uint32_t rot_next(uint32_t v) {
    return (v >> 1) | ((v & 1u) << (L - 1));
}

// Row r = y + L z of the bit mask where lattices A and B differ (q_i = -1):
// bit x set iff the spins at x + L r differ.  A and B in the storage layout
// (BITS: the bit layout, else the byte layout).
template <int L, bool BITS = false>
__device__ __forceinline__ uint32_t diff_row(const uint32_t *A, const uint32_t *B, int r) {
    using Gm = Geom<L>;
    constexpr int W = Gm::W, ROWS = Gm::ROWS, Lh = Gm::Lh;
    uint32_t bits[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        uint32_t acc = 0;
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const int w = (c * ROWS + r) * W + j;
            if (BITS)
                acc |= (((A[w >> 3] ^ B[w >> 3]) >> (4 * (w & 7))) & 0xFu) << (4 * j);
            else
                acc |= sign_nibble(A[w] ^ B[w]) << (4 * j);
        }
        bits[c] = acc & ((1u << Lh) - 1u);
    }
    const int p0 = ((r % L) + (r / L)) & 1;     // x parity of colour 0 in this row
    return (spread_bits(bits[0]) << p0) | (spread_bits(bits[1]) << (p0 ^ 1));
}

}  // namespace pthr
