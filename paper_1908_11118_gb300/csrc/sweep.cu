// sweep.cu -- the grand-canonical Monte Carlo sweep of every replica (sm_103a).
//
// One warp owns one walker (replica configuration) for a whole launch:
//   1. its positions are staged from HBM into shared memory by a bulk TMA
//      copy (cp.async.bulk, completion on an mbarrier with a bounded wait);
//   2. a cell list (cells >= rc on a side, fixed capacity per cell) is built
//      in shared memory, in particle order, so that it is deterministic;
//   3. every trial move (Sec. II.A.1 insertion / removal, Sec. II.A.3
//      displacement) evaluates the truncated-LJ energy of the moved particle
//      against the frozen surface and the other mobile particles; the 32
//      lanes split the candidate partners of the 27-cell stencil, and the
//      partial sums are reduced with warp shuffles;
//   4. the Metropolis / grand-canonical acceptance test is taken in FP64
//      (a binary32 pre-test decides all but near-ties);
//   5. after each sweep the walker is observed into its state's histograms;
//   6. positions, N and the running energy go back to HBM.
// Energies are 64-bit fixed-point sums of binary32 pair terms, so the
// running total never drifts from the from-scratch energy.
#include "launch.h"

namespace regc {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr long long kWaitCycles = 2000000000LL;  // ~1 s at 2 GHz

// A non-empty cell of the stencil of the moved particle: its first index in
// the flattened candidate list and the periodic shifts of its image.  The
// displacement to a partner p in this cell is (q - oA) - (p - oB) per axis;
// oA, oB are 0 or the period, and each shifted operand is exact (Sterbenz),
// so the displacement is rounded once.
struct StEntry {
    int cell, excl;
    float oAx, oBx, oAy, oBy, oAz, oBz;
};

struct WalkerSmem {
    float4* pos;        // [nmax]  x, y, z, (cell << 16 | slot) as bits
    uint64_t* bar;      // mbarrier of the position copy
    StEntry* stencil;   // [32]
    uint16_t* cnt;      // [ncell]
    uint16_t* slots;    // [ncell][cap] particle indices
};

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

__device__ inline WalkerSmem carve(char* base, const SweepParams& P) {
    WalkerSmem w;
    size_t off = 0;
    w.pos = reinterpret_cast<float4*>(base + off);
    off += align16(size_t(P.nmax) * 16);
    w.bar = reinterpret_cast<uint64_t*>(base + off);
    off += 16;
    w.stencil = reinterpret_cast<StEntry*>(base + off);
    off += 32 * sizeof(StEntry);
    w.cnt = reinterpret_cast<uint16_t*>(base + off);
    off += align16(size_t(P.cg.ncell) * 2);
    w.slots = reinterpret_cast<uint16_t*>(base + off);
    return w;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned lanemask_le(int lane) { return FULL >> (31 - lane); }
__device__ __forceinline__ unsigned lanemask_lt(int lane) { return (1u << lane) - 1u; }

// ---------------------------------------------------- bulk copy + mbarrier

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Wait for phase 0 of bar with a cycle budget.  Returns false on timeout.
__device__ bool mbar_wait_bounded(uint64_t* bar) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, 0)) {
        if (clock64() - t0 > kWaitCycles) return false;
    }
    return true;
}

// --------------------------------------------------------------- cells

__device__ __forceinline__ int cell_of(const SweepParams& P, float x, float y, float z) {
    const int cx = min(P.cg.ncx - 1, (int)(x * P.cg.icx));
    const int cy = min(P.cg.ncy - 1, (int)(y * P.cg.icy));
    const float zz = P.g.periodic_z ? z : (z - P.g.z_lo);
    const int cz = min(P.cg.ncz - 1, max(0, (int)(zz * P.cg.icz)));
    return (cz * P.cg.ncy + cy) * P.cg.ncx + cx;
}

__device__ __forceinline__ int wrap_idx(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Stencil entry handled by this lane for the cell `cell` of the moved
// particle (cell = -1 if the lane has none) and the stencil size.  Periodic
// axes always contribute three images (-1, 0, +1); with fewer than three
// cells along an axis the same cell appears with different shifts, which
// evaluates every periodic image of its particles (at most one of them can be
// within rc, because every period is at least 2 rc).
__device__ __forceinline__ StEntry stencil_entry(const SweepParams& P, int cell, int lane, int& nst) {
    const int ncx = P.cg.ncx, ncy = P.cg.ncy, ncz = P.cg.ncz;
    const int cx = cell % ncx, cy = (cell / ncx) % ncy, cz = cell / (ncx * ncy);
    int zfirst = 0, nzs = 3;
    if (!P.g.periodic_z) {
        zfirst = max(0, cz - 1);
        nzs = min(ncz - 1, cz + 1) - zfirst + 1;
    }
    nst = 9 * nzs;
    StEntry e{-1, 0, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (lane >= nst) return e;
    const int lx = lane % 3, ly = (lane / 3) % 3, lz = lane / 9;
    int ix = cx - 1 + lx, iy = cy - 1 + ly, iz;
    if (ix < 0) { ix += ncx; e.oBx = P.g.Lx; }
    else if (ix >= ncx) { ix -= ncx; e.oAx = P.g.Lx; }
    if (iy < 0) { iy += ncy; e.oBy = P.g.Ly; }
    else if (iy >= ncy) { iy -= ncy; e.oAy = P.g.Ly; }
    if (P.g.periodic_z) {
        iz = cz - 1 + lz;
        if (iz < 0) { iz += ncz; e.oBz = P.g.Lz; }
        else if (iz >= ncz) { iz -= ncz; e.oAz = P.g.Lz; }
    } else {
        iz = zfirst + lz;
    }
    e.cell = (iz * ncy + iy) * ncx + ix;
    return e;
}

// Energy of NQ positions (sharing one stencil cell) against the mobile
// particles of the stencil, skipping particle `skip`.  The candidate list is
// the concatenation of the non-empty stencil entries; lane j of a batch takes
// flat index base + j and finds its entry from the OR-reduced mask of entry
// starts inside the batch.
template <int NQ>
__device__ __forceinline__ void mobile_energy(const SweepParams& P, const WalkerSmem& W, int cell,
                                              const float (&qx)[NQ], const float (&qy)[NQ],
                                              const float (&qz)[NQ], int skip, long long (&acc)[NQ],
                                              int& n_in, int& n_cand, int& overlap, int lane) {
    int nst;
    StEntry se = stencil_entry(P, cell, lane, nst);
    const int c = se.cell >= 0 ? (int)W.cnt[se.cell] : 0;
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += t;
    }
    const int excl = incl - c;
    const int total = __shfl_sync(FULL, incl, 31);
    const unsigned nonempty = __ballot_sync(FULL, c > 0);
    if (c > 0) {
        se.excl = excl;
        W.stencil[__popc(nonempty & lanemask_lt(lane))] = se;
    }
    __syncwarp();
    int started = 0;
    for (int base = 0; base < total; base += 32) {
        const unsigned bit =
            (c > 0 && excl >= base && excl < base + 32) ? (1u << (excl - base)) : 0u;
        const unsigned starts = __reduce_or_sync(FULL, bit);
        const int j = base + lane;
        if (j < total) {
            const int r = started + __popc(starts & lanemask_le(lane)) - 1;
            const StEntry& e = W.stencil[r];
            const int pj = W.slots[e.cell * P.cg.cap + (j - e.excl)];
            if (pj != skip) {
                const float4 p = W.pos[pj];
                const float bx = __fsub_rn(p.x, e.oBx), by = __fsub_rn(p.y, e.oBy);
                const float bz = __fsub_rn(p.z, e.oBz);
                n_cand += NQ;
#pragma unroll
                for (int k = 0; k < NQ; ++k) {
                    const float dx = __fsub_rn(__fsub_rn(qx[k], e.oAx), bx);
                    const float dy = __fsub_rn(__fsub_rn(qy[k], e.oAy), by);
                    const float dz = __fsub_rn(__fsub_rn(qz[k], e.oAz), bz);
                    acc[k] += pair_fix_d(dx, dy, dz, P.g, P.gg, n_in, overlap);
                }
            }
        }
        started += __popc(starts);
    }
    __syncwarp();
}

// Energy of NQ positions (sharing one surface column) against the images of
// frozen surface atoms listed for that column.  Each listed image carries the
// exact shifts of its displacement: the stored coordinate is already shifted
// by -L where that is exact, and the flag bits ask for the query to be
// shifted by -L instead.
template <int NQ>
__device__ __forceinline__ void surface_energy(const SweepParams& P, int col, const float (&qx)[NQ],
                                               const float (&qy)[NQ], const float (&qz)[NQ],
                                               long long (&acc)[NQ], int& n_in, int& n_cand,
                                               int& overlap, int lane) {
    const int beg = P.st.col_off[col], end = P.st.col_off[col + 1];
    for (int j = beg + lane; j < end; j += 32) {
        const float4 a = __ldg(&P.st.atoms[j]);
        const unsigned bits = __float_as_uint(a.w);
        const PairTab& t = surf_tab(P, (int)(bits & 3u));
        const float sx = (bits & 4u) ? P.g.Lx : 0.f, sy = (bits & 8u) ? P.g.Ly : 0.f;
        const float sz = (bits & 16u) ? P.g.Lz : 0.f;
        n_cand += NQ;
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
            const float dx = __fsub_rn(__fsub_rn(qx[k], sx), a.x);
            const float dy = __fsub_rn(__fsub_rn(qy[k], sy), a.y);
            const float dz = __fsub_rn(__fsub_rn(qz[k], sz), a.z);
            acc[k] += pair_fix_d(dx, dy, dz, P.g, t, n_in, overlap);
        }
    }
}

__device__ __forceinline__ int surface_col(const SweepParams& P, float x, float y) {
    const int sx = min(P.st.nsx - 1, (int)(x * P.st.isx));
    const int sy = min(P.st.nsy - 1, (int)(y * P.st.isy));
    return sy * P.st.nsx + sx;
}

__device__ __forceinline__ bool near_surface(const SweepParams& P, float z) {
    return P.g.periodic_z || z < P.st.z_reach;
}

// Interaction energy (fixed point, summed over the warp) of one position.
__device__ long long energy_one(const SweepParams& P, const WalkerSmem& W, float x, float y, float z,
                                int skip, int& n_in, int& n_cand, int& overlap, int lane) {
    const float qx[1] = {x}, qy[1] = {y}, qz[1] = {z};
    long long acc[1] = {0};
    mobile_energy<1>(P, W, cell_of(P, x, y, z), qx, qy, qz, skip, acc, n_in, n_cand, overlap, lane);
    if (near_surface(P, z)) surface_energy<1>(P, surface_col(P, x, y), qx, qy, qz, acc, n_in, n_cand, overlap, lane);
    return acc[0];
}

// New-minus-old energy of a displacement of particle i from o to n.
__device__ long long energy_diff(const SweepParams& P, const WalkerSmem& W, float4 o, float nx, float ny,
                                 float nz, int i, int& n_in, int& n_cand, int& overlap, int lane) {
    const int c_old = cell_of(P, o.x, o.y, o.z), c_new = cell_of(P, nx, ny, nz);
    long long d = 0;
    int ov_new = 0, ov_old = 0;
    if (c_old == c_new) {
        const float qx[2] = {nx, o.x}, qy[2] = {ny, o.y}, qz[2] = {nz, o.z};
        long long acc[2] = {0, 0};
        int dummy = 0;
        mobile_energy<2>(P, W, c_new, qx, qy, qz, i, acc, n_in, n_cand, dummy, lane);
        ov_new |= dummy;  // the old position never overlaps (invariant of the state)
        d += acc[0] - acc[1];
    } else {
        const float ax[1] = {nx}, ay[1] = {ny}, az[1] = {nz};
        const float bx[1] = {o.x}, by[1] = {o.y}, bz[1] = {o.z};
        long long a1[1] = {0}, b1[1] = {0};
        mobile_energy<1>(P, W, c_new, ax, ay, az, i, a1, n_in, n_cand, ov_new, lane);
        mobile_energy<1>(P, W, c_old, bx, by, bz, i, b1, n_in, n_cand, ov_old, lane);
        d += a1[0] - b1[0];
    }
    const bool sn = near_surface(P, nz), so = near_surface(P, o.z);
    const int col_n = surface_col(P, nx, ny), col_o = surface_col(P, o.x, o.y);
    if (sn && so && col_n == col_o) {
        const float qx[2] = {nx, o.x}, qy[2] = {ny, o.y}, qz[2] = {nz, o.z};
        long long acc[2] = {0, 0};
        surface_energy<2>(P, col_n, qx, qy, qz, acc, n_in, n_cand, ov_new, lane);
        d += acc[0] - acc[1];
    } else {
        if (sn) {
            const float qx[1] = {nx}, qy[1] = {ny}, qz[1] = {nz};
            long long acc[1] = {0};
            surface_energy<1>(P, col_n, qx, qy, qz, acc, n_in, n_cand, ov_new, lane);
            d += acc[0];
        }
        if (so) {
            const float qx[1] = {o.x}, qy[1] = {o.y}, qz[1] = {o.z};
            long long acc[1] = {0};
            surface_energy<1>(P, col_o, qx, qy, qz, acc, n_in, n_cand, ov_old, lane);
            d -= acc[0];
        }
    }
    overlap |= ov_new;
    return d;
}

__device__ __forceinline__ float4 packed(float x, float y, float z, int cell, int slot) {
    return make_float4(x, y, z, __uint_as_float(((unsigned)cell << 16) | (unsigned)slot));
}
__device__ __forceinline__ int cell_bits(float w) { return (int)(__float_as_uint(w) >> 16); }
__device__ __forceinline__ int slot_bits(float w) { return (int)(__float_as_uint(w) & 0xffffu); }

// Remove particle i (whose packed w gives its cell and slot) from its cell.
__device__ __forceinline__ void cell_remove(const SweepParams& P, const WalkerSmem& W, float wbits) {
    const int c = cell_bits(wbits), s = slot_bits(wbits);
    if (c >= P.cg.ncell || s >= P.cg.cap || s >= (int)W.cnt[c]) {
        // only reachable after a capacity overflow left a particle out of the list
        atomicOr(P.error, ERR_CAPACITY);
        return;
    }
    const int last = W.cnt[c] - 1;
    const int moved = W.slots[c * P.cg.cap + last];
    W.slots[c * P.cg.cap + s] = (uint16_t)moved;
    W.pos[moved].w = __uint_as_float(((unsigned)c << 16) | (unsigned)s);
    W.cnt[c] = (uint16_t)last;
}

// Deterministic cell build: particles in index order, ties inside a batch of
// 32 resolved by lane order.
__device__ void build_cells(const SweepParams& P, const WalkerSmem& W, int N, int lane) {
    for (int c = lane; c < P.cg.ncell; c += 32) W.cnt[c] = 0;
    __syncwarp();
    for (int base = 0; base < N; base += 32) {
        const int j = base + lane;
        const bool act = j < N;
        int c = -1;
        float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
        if (act) {
            p = W.pos[j];
            c = cell_of(P, p.x, p.y, p.z);
        }
        const unsigned grp = __match_any_sync(FULL, c);
        int before = 0;
        if (act) {
            before = W.cnt[c];
            const int slot = before + __popc(grp & lanemask_lt(lane));
            if (slot < P.cg.cap) {
                W.slots[c * P.cg.cap + slot] = (uint16_t)j;
                W.pos[j] = packed(p.x, p.y, p.z, c, slot);
            } else {
                atomicOr(P.error, ERR_CAPACITY);
            }
        }
        __syncwarp();
        if (act && lane == __ffs(grp) - 1) W.cnt[c] = (uint16_t)min(P.cg.cap, before + __popc(grp));
        __syncwarp();
    }
}

template <bool TRACE>
__global__ void __launch_bounds__(256) sweep_kernel(const __grid_constant__ SweepParams P) {
    extern __shared__ __align__(16) char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int w = blockIdx.x * (blockDim.x >> 5) + warp;
    if (w >= P.S) return;
    const WalkerSmem W = carve(smem + size_t(warp) * P.smem_per_walker, P);

    int N = P.n[w];
    long long E = P.efix[w];
    const int s = P.state_of_walker[w];
    const double beta = P.beta[s], c_ins = P.c_ins[s], c_del = P.c_del[s];
    float4* gpos = P.pos + size_t(w) * P.nmax;

    // 1. stage positions with a bulk copy
    if (N > 0) {
        if (lane == 0) {
            mbar_init(W.bar);
            bulk_load(W.pos, gpos, uint32_t(N) * 16u, W.bar);
        }
        __syncwarp();
        bool ok = mbar_wait_bounded(W.bar);
        ok = __all_sync(FULL, ok);
        if (!ok) {
            if (lane == 0) atomicOr(P.error, ERR_TIMEOUT);
            mbar_wait_bounded(W.bar);  // give the copy in flight one more bounded chance
            return;
        }
    }
    // 2. cell list
    build_cells(P, W, N, lane);

    long long tr0 = 0, tr1 = 0, tr2 = 0, ac0 = 0, ac1 = 0, ac2 = 0;
    int n_in = 0, n_cand = 0;
    unsigned long long om = 0, eo = 0;
    double m0 = 0, m1 = 0, m2 = 0, m3 = 0;
    const int cap = P.cg.cap;

    for (int ts = 0; ts < P.n_sweeps; ++ts) {
        const uint32_t t = P.t0 + uint32_t(ts);
        for (int kb = 0; kb < P.mps; kb += 32) {
            const int k_lane = kb + lane;
            U4 A{0, 0, 0, 0}, B{0, 0, 0, 0};
            if (k_lane < P.mps) {
                A = philox(uint32_t(k_lane), t, uint32_t(w), 0u, P.key0, P.key1);
                B = philox(uint32_t(k_lane), t, uint32_t(w), 1u, P.key0, P.key1);
            }
            const int kn = min(32, P.mps - kb);
            for (int kk = 0; kk < kn; ++kk) {
                const uint32_t a0 = __shfl_sync(FULL, A.x, kk), a1 = __shfl_sync(FULL, A.y, kk);
                const uint32_t a2 = __shfl_sync(FULL, A.z, kk), a3 = __shfl_sync(FULL, A.w, kk);
                const uint32_t b0 = __shfl_sync(FULL, B.x, kk), b1 = __shfl_sync(FULL, B.y, kk);
                const uint32_t b2 = __shfl_sync(FULL, B.z, kk);
                const int type = (unsigned long long)a0 < P.th_disp ? 0 : ((b2 >> 31) == 0u ? 2 : 1);
                int status = 0, idx = -1, overlap = 0, n_in0 = n_in;
                long long dfix = 0;
                float nx = 0.f, ny = 0.f, nz = 0.f;
                float4 old = make_float4(0.f, 0.f, 0.f, 0.f);
                double la = 0.0;
                if (type == 0) {
                    if (N == 0) {
                        status = 1;
                    } else {
                        idx = (int)(((unsigned long long)b0 * (unsigned)N) >> 32);
                        old = W.pos[idx];
                        const float dx = __fmul_rn(P.max_disp, __fsub_rn(__fmul_rn(2.0f, u24(a1)), 1.0f));
                        const float dy = __fmul_rn(P.max_disp, __fsub_rn(__fmul_rn(2.0f, u24(a2)), 1.0f));
                        const float dz = __fmul_rn(P.max_disp, __fsub_rn(__fmul_rn(2.0f, u24(a3)), 1.0f));
                        nx = __fadd_rn(old.x, dx);
                        ny = __fadd_rn(old.y, dy);
                        nz = __fadd_rn(old.z, dz);
                        if (nx < 0.f) nx = __fadd_rn(nx, P.g.Lx);
                        if (nx >= P.g.Lx) nx = __fsub_rn(nx, P.g.Lx);
                        if (ny < 0.f) ny = __fadd_rn(ny, P.g.Ly);
                        if (ny >= P.g.Ly) ny = __fsub_rn(ny, P.g.Ly);
                        if (P.g.periodic_z) {
                            if (nz < 0.f) nz = __fadd_rn(nz, P.g.Lz);
                            if (nz >= P.g.Lz) nz = __fsub_rn(nz, P.g.Lz);
                        } else if (nz < P.g.z_lo || nz > P.g.z_hi) {
                            status = 2;
                        }
                        if (status == 0) {
                            dfix = energy_diff(P, W, old, nx, ny, nz, idx, n_in, n_cand, overlap, lane);
                            dfix = warp_sum_ll(dfix);
                            la = -beta * ((double)dfix * kFixUnit);
                        }
                    }
                } else if (type == 1) {
                    if (N == P.nmax) {
                        status = 1;
                    } else {
                        idx = N;
                        nx = __fmul_rn(P.g.Lx, u24(a1));
                        ny = __fmul_rn(P.g.Ly, u24(a2));
                        nz = __fadd_rn(P.g.z_lo, __fmul_rn(P.g.height, u24(a3)));
                        if (nx >= P.g.Lx) nx = __fsub_rn(nx, P.g.Lx);
                        if (ny >= P.g.Ly) ny = __fsub_rn(ny, P.g.Ly);
                        if (P.g.periodic_z && nz >= P.g.Lz) nz = __fsub_rn(nz, P.g.Lz);
                        dfix = warp_sum_ll(energy_one(P, W, nx, ny, nz, -1, n_in, n_cand, overlap, lane));
                        la = c_ins - P.ln_tab[N + 1] - beta * ((double)dfix * kFixUnit);
                    }
                } else {
                    if (N == 0) {
                        status = 1;
                    } else {
                        idx = (int)(((unsigned long long)b0 * (unsigned)N) >> 32);
                        old = W.pos[idx];
                        int ov = 0;
                        dfix = -warp_sum_ll(energy_one(P, W, old.x, old.y, old.z, idx, n_in, n_cand, ov, lane));
                        la = c_del + P.ln_tab[N] - beta * ((double)dfix * kFixUnit);
                    }
                }
                overlap = __any_sync(FULL, overlap);
                // capacity of the destination cell
                int c_new = -1;
                if (status == 0 && type != 2) {
                    c_new = cell_of(P, nx, ny, nz);
                    const bool same = type == 0 && c_new == cell_bits(old.w);
                    if (!same && W.cnt[c_new] >= cap) {
                        status = 3;
                        if (lane == 0) atomicOr(P.error, ERR_CAPACITY);
                    }
                }
                // acceptance: ln u < la, binary32 pre-test outside a 1e-4 band
                int accepted = 0;
                double ln_u = 0.0;
                if (status == 0 && !overlap) {
                    if (la >= 0.0) {
                        accepted = 1;
                    } else {
                        const float lf = __logf(((float)b1 + 0.5f) * 2.3283064365386963e-10f);
                        if ((double)lf < la - 1e-4) accepted = 1;
                        else if ((double)lf > la + 1e-4) accepted = 0;
                        else accepted = log(((double)b1 + 0.5) * 2.3283064365386963e-10) < la;
                    }
                }
                if (TRACE) ln_u = log(((double)b1 + 0.5) * 2.3283064365386963e-10);
                if (accepted) {
                    if (lane == 0) {
                        if (type == 0) {
                            const int c_old = cell_bits(old.w);
                            if (c_new == c_old) {
                                W.pos[idx] = make_float4(nx, ny, nz, old.w);
                            } else {
                                cell_remove(P, W, old.w);
                                const int sl = W.cnt[c_new];
                                W.slots[c_new * cap + sl] = (uint16_t)idx;
                                W.cnt[c_new] = (uint16_t)(sl + 1);
                                W.pos[idx] = packed(nx, ny, nz, c_new, sl);
                            }
                        } else if (type == 1) {
                            const int sl = W.cnt[c_new];
                            W.slots[c_new * cap + sl] = (uint16_t)N;
                            W.cnt[c_new] = (uint16_t)(sl + 1);
                            W.pos[N] = packed(nx, ny, nz, c_new, sl);
                        } else {
                            cell_remove(P, W, old.w);
                            const int last = N - 1;
                            if (idx != last) {
                                const float4 pl = W.pos[last];
                                W.pos[idx] = pl;
                                W.slots[cell_bits(pl.w) * cap + slot_bits(pl.w)] = (uint16_t)idx;
                            }
                        }
                    }
                    __syncwarp();
                    E += dfix;
                    N += (type == 1) - (type == 2);
                }
                tr0 += type == 0;
                tr1 += type == 1;
                tr2 += type == 2;
                ac0 += accepted && type == 0;
                ac1 += accepted && type == 1;
                ac2 += accepted && type == 2;
                if (TRACE) {
                    const int np = warp_sum_i(n_in - n_in0);
                    if (lane == 0) {
                        regc_move_record r;
                        r.type = type;
                        r.index = status == 1 ? 0 : idx;
                        r.accepted = accepted;
                        r.status = status == 3 ? 0 : status;
                        r.dE = status == 0 || status == 3 ? (double)dfix * kFixUnit : 0.0;
                        r.log_alpha = overlap ? -INFINITY : la;
                        r.ln_u = ln_u;
                        r.sum_abs = 0.0;
                        r.band = 0.0;
                        r.n_pairs = np;
                        r.pad = 0;
                        P.trace[(size_t(w) * P.n_sweeps + ts) * P.mps + kb + kk] = r;
                    }
                }
            }
        }
        // 5. observe once per sweep into the current state's histograms
        if (lane == 0) {
            const double e = (double)E * kFixUnit;
            P.hN[size_t(s) * (P.nmax + 1) + N] += 1ull;
            om += 1;
            m0 += (double)N;
            m1 += (double)N * (double)N;
            m2 += e;
            m3 += e * e;
            const double kb = floor((e - P.e_lo) / P.e_bin);
            if (kb >= 0.0 && kb < (double)P.n_e_bins) {
                atomicAdd(&P.hNE[size_t(N) * P.n_e_bins + (size_t)kb], 1ull);
            } else {
                eo += 1;
            }
        }
    }

    // 6. write back
    __syncwarp();
    for (int j = lane; j < N; j += 32) gpos[j] = W.pos[j];
    const int sum_in = warp_sum_i(n_in), sum_cand = warp_sum_i(n_cand);
    if (lane == 0) {
        P.n[w] = N;
        P.efix[w] = E;
        P.omega[s] += om;
        P.e_out[s] += eo;
        double* m = P.moments + size_t(s) * 4;
        m[0] += m0;
        m[1] += m1;
        m[2] += m2;
        m[3] += m3;
        long long* mc = P.move_counts + size_t(w) * 6;
        mc[0] += tr0;
        mc[1] += ac0;
        mc[2] += tr1;
        mc[3] += ac1;
        mc[4] += tr2;
        mc[5] += ac2;
        atomicAdd(&P.pair_counts[0], (unsigned long long)sum_in);
        atomicAdd(&P.pair_counts[1], (unsigned long long)sum_cand);
    }
}

// Displacement q - p with the exact minimum image on periodic axes.
__device__ __forceinline__ void disp_exact(const Geometry& g, float4 q, float4 p, float& dx, float& dy, float& dz) {
    dx = min_image_exact(q.x, p.x, g.Lx, g.hLx);
    dy = min_image_exact(q.y, p.y, g.Ly, g.hLy);
    dz = g.periodic_z ? min_image_exact(q.z, p.z, g.Lz, g.hLz) : __fsub_rn(q.z, p.z);
}

// From-scratch energy of every walker: all pairs i < j and all particle-surface
// pairs, with the nearest periodic image.  Every pair within rc gets the same
// rounded displacement, hence the same fixed-point term, as in the sweep.
__global__ void __launch_bounds__(256) energy_kernel(const __grid_constant__ SweepParams P, long long* out,
                                                     int check_overlap) {
    const int lane = threadIdx.x & 31;
    const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w >= P.S) return;
    const int N = P.n[w];
    const float4* pos = P.pos + size_t(w) * P.nmax;
    long long acc = 0;
    int n_in = 0, overlap = 0;
    float dx, dy, dz;
    for (int i = 0; i < N; ++i) {
        const float4 pi = pos[i];
        for (int j = i + 1 + lane; j < N; j += 32) {
            disp_exact(P.g, pi, pos[j], dx, dy, dz);
            acc += pair_fix_d(dx, dy, dz, P.g, P.gg, n_in, overlap);
        }
        for (int a = lane; a < P.st.n_all; a += 32) {
            const float4 at = P.st.all[a];
            disp_exact(P.g, pi, at, dx, dy, dz);
            acc += pair_fix_d(dx, dy, dz, P.g, surf_tab(P, (int)at.w), n_in, overlap);
        }
    }
    acc = warp_sum_ll(acc);
    overlap = __any_sync(FULL, overlap);
    if (lane == 0) {
        out[w] = acc;
        if (overlap && check_overlap) atomicOr(P.error, ERR_OVERLAP);
    }
}

}  // namespace

size_t sweep_smem_per_walker(int nmax, int ncell, int cap) {
    return align16(size_t(nmax) * 16) + 16 + 32 * sizeof(StEntry) + align16(size_t(ncell) * 2) +
           align16(size_t(ncell) * cap * 2);
}

cudaError_t launch_sweep(const SweepParams& P, int wpc, cudaStream_t s) {
    if (P.n_sweeps <= 0) return cudaSuccess;
    const size_t smem = size_t(wpc) * P.smem_per_walker;
    const int grid = (P.S + wpc - 1) / wpc;
    cudaError_t err;
    if (P.trace) {
        err = cudaFuncSetAttribute(sweep_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
        sweep_kernel<true><<<grid, 32 * wpc, smem, s>>>(P);
    } else {
        err = cudaFuncSetAttribute(sweep_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
        sweep_kernel<false><<<grid, 32 * wpc, smem, s>>>(P);
    }
    return cudaGetLastError();
}

cudaError_t launch_energy(const SweepParams& P, long long* out, int check_overlap, cudaStream_t s) {
    const int wpc = 4;
    energy_kernel<<<(P.S + wpc - 1) / wpc, 32 * wpc, 0, s>>>(P, out, check_overlap);
    return cudaGetLastError();
}

}  // namespace regc
