// cells.cuh -- cell lists and surface columns of a walker (device helpers
// shared by the sweep and the molecular-dynamics kernels).
//
// Cells are at least rc on a side, so every partner within rc of a point lies
// in the 27 cells around the point's cell (with periodic images).  A cell
// holds up to cap particle indices (uint16); a particle's packed float4 w
// carries its cell (high 16 bits) and slot (low 16 bits).
#pragma once

#include "regc_internal.cuh"

namespace regc {

__device__ __forceinline__ unsigned lanemask_le(int lane) { return 0xffffffffu >> (31 - lane); }
__device__ __forceinline__ unsigned lanemask_lt(int lane) { return (1u << lane) - 1u; }

struct Cell3 {
    int x, y, z;
};

__device__ __forceinline__ Cell3 cell3_of(const SweepParams& P, float x, float y, float z) {
    Cell3 c;
    c.x = min(P.cg.ncx - 1, (int)(x * P.cg.icx));
    c.y = min(P.cg.ncy - 1, (int)(y * P.cg.icy));
    const float zz = P.g.periodic_z ? z : (z - P.g.z_lo);
    c.z = min(P.cg.ncz - 1, max(0, (int)(zz * P.cg.icz)));
    return c;
}

__device__ __forceinline__ int cell_index(const SweepParams& P, Cell3 c) {
    return (c.z * P.cg.ncy + c.y) * P.cg.ncx + c.x;
}

__device__ __forceinline__ int cell_of(const SweepParams& P, float x, float y, float z) {
    return cell_index(P, cell3_of(P, x, y, z));
}

// Surface column of a point (x, y), and whether a point at height z can reach
// any surface atom.
__device__ __forceinline__ int surface_col(const SweepParams& P, float x, float y) {
    const int sx = min(P.st.nsx - 1, (int)(x * P.st.isx));
    const int sy = min(P.st.nsy - 1, (int)(y * P.st.isy));
    return sy * P.st.nsx + sx;
}

__device__ __forceinline__ bool near_surface(const SweepParams& P, float z) {
    return P.st.n_all > 0 && (P.g.periodic_z || z < P.st.z_reach);
}

__device__ __forceinline__ float4 packed(float x, float y, float z, int cell, int slot) {
    return make_float4(x, y, z, __uint_as_float(((unsigned)cell << 16) | (unsigned)slot));
}
__device__ __forceinline__ int cell_bits(float w) { return (int)(__float_as_uint(w) >> 16); }
__device__ __forceinline__ int slot_bits(float w) { return (int)(__float_as_uint(w) & 0xffffu); }

// Deterministic cell build by one warp: particles in index order, ties inside
// a batch of 32 resolved by lane order; every particle's w gets its cell and
// slot.  A full cell sets ERR_CAPACITY and leaves the particle out.
__device__ __forceinline__ void build_cell_list(const SweepParams& P, float4* pos, int N, uint16_t* cnt,
                                                uint16_t* slots, int lane) {
    for (int c = lane; c < P.cg.ncell; c += 32) cnt[c] = 0;
    __syncwarp();
    for (int base = 0; base < N; base += 32) {
        const int j = base + lane;
        const bool act = j < N;
        int c = -1;
        float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
        if (act) {
            p = pos[j];
            c = cell_of(P, p.x, p.y, p.z);
        }
        const unsigned grp = __match_any_sync(0xffffffffu, c);
        int before = 0;
        if (act) {
            before = cnt[c];
            const int slot = before + __popc(grp & lanemask_lt(lane));
            if (slot < P.cg.cap) {
                slots[c * P.cg.cap + slot] = (uint16_t)j;
                pos[j] = packed(p.x, p.y, p.z, c, slot);
            } else {
                atomicOr(P.error, ERR_CAPACITY);
            }
        }
        __syncwarp();
        if (act && lane == __ffs(grp) - 1) cnt[c] = (uint16_t)min(P.cg.cap, before + __popc(grp));
        __syncwarp();
    }
}

}  // namespace regc
