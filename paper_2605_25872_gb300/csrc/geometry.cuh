// geometry.cuh -- 4-site groups of the packed colour-row layout: where a
// group's own word and its six neighbour words are (shared by the sweep and
// measurement kernels).
#pragma once

#include "pthr_internal.cuh"

namespace pthr {

struct GroupGeo {
    int own, xa, yp, ym, zp, zm;   // word offsets in a lattice
    int wA, wB;                    // words of the shifted x neighbour
    uint32_t selx;                 // byte_perm selector of the shifted x word
    int par;                       // x parity of this row/colour
};

// Geometry of 4-site group g of colour c (see pthr_internal.cuh for layout).
template <int L>
__device__ __forceinline__ GroupGeo group_geo(int g, int c) {
    using Gm = Geom<L>;
    constexpr int W = Gm::W, ROWS = Gm::ROWS, Lh = Gm::Lh;
    GroupGeo q;
    const int r = g / W, j = g - (g / W) * W;
    const int y = r % L, z = r / L;
    const int cc = c ^ 1;
    q.par = (c + y + z) & 1;
    const int ryp = ((y + 1) % L) + L * z, rym = ((y + L - 1) % L) + L * z;
    const int rzp = y + L * ((z + 1) % L), rzm = y + L * ((z + L - 1) % L);
    q.own = (c * ROWS + r) * W + j;
    const int rowcc = (cc * ROWS + r) * W;
    q.xa = rowcc + j;
    q.yp = (cc * ROWS + ryp) * W + j;
    q.ym = (cc * ROWS + rym) * W + j;
    q.zp = (cc * ROWS + rzp) * W + j;
    q.zm = (cc * ROWS + rzm) * W + j;
    // Shifted x neighbour: m' = m - 1 (par 0, the -x neighbour) or m + 1
    // (par 1, the +x neighbour), cyclic in [0, Lh).  At most two words.
    const int d = q.par ? 1 : Lh - 1;
    int wa = -1, wb = -1;
    uint32_t sel = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int m = 4 * j + k;
        if (m >= Lh) m = Lh - 1;              // padding byte: any valid source
        const int mp = (m + d) % Lh;
        const int w = mp >> 2, by = mp & 3;
        int src;
        if (wa < 0 || wa == w) { wa = w; src = by; }
        else { wb = w; src = 4 + by; }
        sel |= (uint32_t)src << (4 * k);
    }
    if (wb < 0) wb = wa;
    q.wA = rowcc + wa;
    q.wB = rowcc + wb;
    q.selx = sel;
    return q;
}


// Bit 7 of the bytes of group word j that hold real sites (not row padding).
template <int L>
__device__ __forceinline__ uint32_t valid_mask(int j) {
    constexpr int Lh = L / 2;
    if ((Lh % 4) == 0) return 0x80808080u;
    const int nv = Lh - 4 * j;
    return nv >= 4 ? 0x80808080u : (0x80808080u >> (8 * (4 - nv)));
}

}  // namespace pthr
