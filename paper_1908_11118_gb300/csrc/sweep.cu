// sweep.cu -- the grand-canonical Monte Carlo sweep of every replica (sm_103a).
//
// One CTA of K warps (K = 1, 2 or 4) owns one walker (replica configuration)
// for a whole launch:
//   1. its positions are staged from HBM into shared memory by a bulk TMA
//      copy (cp.async.bulk, completion on an mbarrier with a bounded wait);
//   2. a cell list (cells >= rc on a side, fixed capacity per cell) is built
//      in shared memory, in particle order, so that it is deterministic;
//   3. the trial moves (Sec. II.A.1 insertion / removal, Sec. II.A.3
//      displacement) are processed in rounds: warp j evaluates move m0 + j of
//      the walker's sequence against the current configuration -- the
//      truncated-LJ energy change of the moved particle against the other
//      mobile particles of its 27-cell stencil and the frozen surface atoms
//      listed for its column, each pair term added in exact fixed point and
//      reduced with redux.sync;
//   4. thread 0 then commits the round's moves in order.  Move m0 + j keeps
//      its evaluated energy change if no earlier move of the round that was
//      accepted changed anything it depends on (N, for a move that picks a
//      particle by index; any position within rc of its query points);
//      otherwise the round stops there and the move is evaluated again in the
//      next round.  Fixed-point sums do not depend on the order of the pairs,
//      so a kept energy change is bit-identical to the one a strictly
//      sequential evaluation would compute, and the chain is exactly the
//      sequential Markov chain.  The acceptance test ln u < ln alpha is
//      decided in binary32 when the two sides differ by more than 1e-3, and in
//      FP64 otherwise, which gives the FP64 decision in every case;
//   5. after each sweep the walker is observed into its state's histograms;
//   6. positions, N and the running energy go back to HBM.
#include "cells.cuh"
#include "launch.h"
#include "surrogate.cuh"

namespace regc {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr long long kWaitCycles = 2000000000LL;  // ~1 s at 2 GHz
constexpr double kLn2m32 = -22.18070977791825;   // ln 2^-32
constexpr int kRing = 64;                         // Philox blocks of moves kept ahead

// A non-empty cell of a stencil: its first index in the flattened candidate
// list and the periodic shifts of its image.  The displacement from query k to
// a partner p of the cell is a_k - (p - ob) per axis, where a_k is the query
// shifted by 0 or minus the period and ob is 0 or the period; every shifted
// operand is exact (Sterbenz), so the displacement is rounded once.
struct StEntry {
    int cell, excl;
    float ax0, ay0, az0, ax1, ay1, az1;
    float obx, oby, obz;
    int pad;
};

// The evaluation of one trial move, handed from its warp to the committer.
struct MoveRes {
    int type;      // 0 displacement, 1 insertion, 2 removal
    int status;    // 0 evaluated, 1 at the N boundary, 2 displacement left the region
    int idx;       // particle picked (insertion: unused)
    int n_eval;    // N the move was evaluated with
    int big, hi, lo;   // fixed-point energy change
    int flags;     // bit 0 overlap, bits 1.. pairs within rc
    float q0x, q0y, q0z;   // new position (removal: the old one)
    float q1x, q1y, q1z;   // old position of a displacement
    int dec;       // decision with N = n_eval: 0 reject, 1 accept, 2 near tie (FP64 needed)
    int stage1;    // delayed acceptance: 1 if the surrogate stage accepted
    float dE_sur;  // delayed acceptance: surrogate energy change
    int gy;        // two mobile species: 0 if the moved (inserted, removed) particle is
                   // of the first (index < split), 1 of the second
};

// Pair tables of the moving particle's species against a cluster partner (tA)
// and a grand-canonical partner (tB); mA: the moving particle is a cluster atom.
// Binary32 pair energy without branches: 0 unless `use` and r < rc.  An
// in-range term is computed with the same operations as pair_phi, hence is
// bit-identical to it; the branch-free form lets the candidate loop be one
// basic block, so independent loads and arithmetic overlap.
__device__ __forceinline__ float pair_phi_sel(float dx, float dy, float dz, float rc2, const PairTab& t, bool use,
                                              int& n_in, int& overlap) {
    const float r2 = r2_of(dx, dy, dz);
    const bool in = use && r2 < rc2;
    const float rr = in ? r2 : 1.0f;
    const float s2 = __fdividef(t.sig2, rr);
    const float s6 = __fmul_rn(__fmul_rn(s2, s2), s2);
    const float phi = __fmul_rn(t.eps4, __fmaf_rn(s6, s6, -s6));
    n_in += in;
    overlap |= in && (r2 < t.rhc2);
    return in ? phi : 0.0f;
}

struct MoveTabs {
    PairTab tA, tB;
    bool mA;
};

// Constants of the walker's state for the binary32 pre-test of the acceptance.
struct StateF {
    float beta, c_ins, c_del;
    float c_ins2, c_del2;   // a second grand-canonical species
};

// Binary32 pre-test of ln u < ln alpha with N particles before the move:
// 0 reject, 1 accept, 2 the two sides are within 1e-3 and FP64 must decide.
__device__ __forceinline__ int pretest(const StateF& sf, int type, int N, int big, int hi, int lo, uint32_t b1) {
    const float de_f = __fmaf_rn((float)lo, 9.313225746154785e-10f,
                                 __fmaf_rn((float)hi, 0.00390625f, (float)big * 8192.0f));
    float c_f = 0.f;
    if (type == 1) c_f = sf.c_ins - __logf((float)(N + 1));
    else if (type == 2) c_f = sf.c_del + __logf((float)N);
    const float la_f = c_f - sf.beta * de_f;
    const float lu_f = __logf(((float)b1 + 0.5f) * 2.3283064365386963e-10f);
    if (la_f >= 0.f || lu_f < la_f - 1e-3f) return 1;
    if (lu_f > la_f + 1e-3f) return 0;
    return 2;
}

// Per-launch statistics of the walker, kept by thread 0.
struct WalkerStats {
    long long mN, mN2, mE;
    double mE2;
    unsigned long long om, eo;
    unsigned long long pairs;   // pairs within rc of the committed moves
    unsigned long long rounds, evals;
    unsigned long long screened, passed;   // delayed acceptance: stage-1 screens and passes
    int tr[3], ac[3];
    long long mC, mC2;                      // second grand-canonical species: sum N_C, N_C^2
};

// Round state broadcast by the committer.
struct RoundHdr {
    int N;
    int committed;
    long long E;
    int split;   // two mobile species: the current boundary
    int pad;
};

struct WalkerSmem {
    float4* pos;        // [nmax]  x, y, z, (cell << 16 | slot) as bits
    uint64_t* bar;      // mbarrier of the position copy
    WalkerStats* stats;
    RoundHdr* hdr;
    uint4* rng;         // [kRing][2] Philox blocks A, B of upcoming moves
    MoveRes* res;       // [K]
    StEntry* stencil;   // [K][32]
    float* scratch;     // [K][64] surrogate activations
    uint16_t* cnt;      // [ncell]
    uint16_t* slots;    // [ncell][cap] particle indices
};

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

__host__ __device__ inline size_t smem_bytes(int nmax, int ncell, int cap, int K) {
    return align16(size_t(nmax) * 16) + 16 + align16(sizeof(WalkerStats)) + align16(sizeof(RoundHdr)) +
           size_t(kRing) * 2 * sizeof(uint4) + align16(size_t(K) * sizeof(MoveRes)) +
           size_t(K) * 32 * sizeof(StEntry) + size_t(K) * 64 * sizeof(float) + align16(size_t(ncell) * 2) +
           align16(size_t(ncell) * cap * 2);
}

template <int K>
__device__ inline WalkerSmem carve(char* base, const SweepParams& P) {
    WalkerSmem w;
    size_t off = 0;
    w.pos = reinterpret_cast<float4*>(base + off);
    off += align16(size_t(P.nmax) * 16);
    w.bar = reinterpret_cast<uint64_t*>(base + off);
    off += 16;
    w.stats = reinterpret_cast<WalkerStats*>(base + off);
    off += align16(sizeof(WalkerStats));
    w.hdr = reinterpret_cast<RoundHdr*>(base + off);
    off += align16(sizeof(RoundHdr));
    w.rng = reinterpret_cast<uint4*>(base + off);
    off += size_t(kRing) * 2 * sizeof(uint4);
    w.res = reinterpret_cast<MoveRes*>(base + off);
    off += align16(size_t(K) * sizeof(MoveRes));
    w.stencil = reinterpret_cast<StEntry*>(base + off);
    off += size_t(K) * 32 * sizeof(StEntry);
    w.scratch = reinterpret_cast<float*>(base + off);
    off += size_t(K) * 64 * sizeof(float);
    w.cnt = reinterpret_cast<uint16_t*>(base + off);
    off += align16(size_t(P.cg.ncell) * 2);
    w.slots = reinterpret_cast<uint16_t*>(base + off);
    return w;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}


// ---------------------------------------------------- bulk copy + mbarrier

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
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

// Synchronise the K warps of a walker group: a warp barrier for one warp,
// else named barrier bar over the group's 32 K threads (bar 0 with the whole
// CTA in the one-walker-per-CTA kernel, where it is __syncthreads()).
template <int K>
__device__ __forceinline__ void group_sync(int bar) {
    if (K == 1) __syncwarp();
    else asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(32 * K) : "memory");
}

// True in every thread of the group iff p holds in all of them (a barrier).
template <int K>
__device__ __forceinline__ bool group_all(int bar, bool p) {
    if (K == 1) return __all_sync(0xffffffffu, p) != 0;
    unsigned r;
    asm volatile(
        "{\n\t.reg .pred q, a;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.and.pred a, %2, %3, q;\n\t"
        "selp.u32 %0, 1, 0, a;\n\t}"
        : "=r"(r)
        : "r"((unsigned)p), "r"(bar), "r"(32 * K)
        : "memory");
    return r != 0;
}

// Stencil entry handled by this lane (cell = -1 if none), for queries q0, q1
// in cell c.  Periodic axes always contribute three images (-1, 0, +1); with
// fewer than three cells along an axis the same cell appears with different
// shifts, which evaluates every periodic image of its particles (at most one
// of them can be within rc, because every period is at least 2 rc).
__device__ __forceinline__ StEntry stencil_entry(const SweepParams& P, Cell3 c, int lane, float q0x, float q0y,
                                                 float q0z, float q1x, float q1y, float q1z) {
    int zfirst = 0, nzs = 3;
    if (!P.g.periodic_z) {
        zfirst = max(0, c.z - 1);
        nzs = min(P.cg.ncz - 1, c.z + 1) - zfirst + 1;
    }
    StEntry e;
    e.cell = -1;
    e.excl = 0;
    if (lane >= 9 * nzs) return e;
    const int lx = lane % 3, ly = (lane / 3) % 3, lz = lane / 9;
    int ix = c.x - 1 + lx, iy = c.y - 1 + ly, iz;
    float oax = 0.f, oay = 0.f, oaz = 0.f;
    e.obx = e.oby = e.obz = 0.f;
    if (ix < 0) { ix += P.cg.ncx; e.obx = P.g.Lx; }
    else if (ix >= P.cg.ncx) { ix -= P.cg.ncx; oax = P.g.Lx; }
    if (iy < 0) { iy += P.cg.ncy; e.oby = P.g.Ly; }
    else if (iy >= P.cg.ncy) { iy -= P.cg.ncy; oay = P.g.Ly; }
    if (P.g.periodic_z) {
        iz = c.z - 1 + lz;
        if (iz < 0) { iz += P.cg.ncz; e.obz = P.g.Lz; }
        else if (iz >= P.cg.ncz) { iz -= P.cg.ncz; oaz = P.g.Lz; }
    } else {
        iz = zfirst + lz;
    }
    e.cell = (iz * P.cg.ncy + iy) * P.cg.ncx + ix;
    e.ax0 = __fsub_rn(q0x, oax);
    e.ay0 = __fsub_rn(q0y, oay);
    e.az0 = __fsub_rn(q0z, oaz);
    e.ax1 = __fsub_rn(q1x, oax);
    e.ay1 = __fsub_rn(q1y, oay);
    e.az1 = __fsub_rn(q1z, oaz);
    return e;
}

// Fixed-point energy of NQ queries (sharing the stencil of cell c) against the
// mobile particles of the stencil except `skip`: query 0 enters with sign
// sgn0, query 1 with -1.  The candidate list is the concatenation of the
// non-empty stencil entries; lane j of a batch of 32 finds its entry from the
// OR-reduced mask of entry starts in the batch.
template <int NQ, bool CL>
__device__ __forceinline__ void mobile_pass(const SweepParams& P, const WalkerSmem& S, Cell3 c, float q0x,
                                            float q0y, float q0z, float q1x, float q1y, float q1z, int skip,
                                            int sgn0, Fix3& acc, int& n_in, int& n_cand, int& overlap, int lane,
                                            int warp, int split, const MoveTabs& mt) {
    StEntry* st = S.stencil + warp * 32;
    StEntry se = stencil_entry(P, c, lane, q0x, q0y, q0z, q1x, q1y, q1z);
    const int cnt = se.cell >= 0 ? (int)S.cnt[se.cell] : 0;
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += t;
    }
    const int excl = incl - cnt;
    const int total = __shfl_sync(FULL, incl, 31);
    const unsigned nonempty = __ballot_sync(FULL, cnt > 0);
    if (cnt > 0) {
        se.excl = excl;
        st[__popc(nonempty & lanemask_lt(lane))] = se;
    }
    __syncwarp();
    int ov = 0, started = 0;
#pragma unroll 2   // two batches' independent chains may overlap
    for (int base = 0; base < total; base += 32) {
        const unsigned bit = (cnt > 0 && excl >= base && excl < base + 32) ? (1u << (excl - base)) : 0u;
        const unsigned starts = __reduce_or_sync(FULL, bit);
        const int j = base + lane;
        const bool act = j < total;
        // every lane finds a valid entry (some entry starts at or below it);
        // lanes past the end read particle 0 and discard the term
        const int r = started + __popc(starts & lanemask_le(lane)) - 1;
        const StEntry& e = st[r];
        int pj = -1;
        if (act) pj = S.slots[e.cell * P.cg.cap + (j - e.excl)];
        const bool use = act && pj != skip;
        const float4 p = S.pos[use ? pj : 0];
        const float bx = __fsub_rn(p.x, e.obx), by = __fsub_rn(p.y, e.oby), bz = __fsub_rn(p.z, e.obz);
        n_cand += use ? NQ : 0;
        const PairTab& tp = CL ? (pj < split ? mt.tA : mt.tB) : P.gg;
        const float dy0 = __fsub_rn(e.ay0, by);
        const float phi0 = pair_phi_sel(cart_dx(P.g, __fsub_rn(e.ax0, bx), dy0), dy0, __fsub_rn(e.az0, bz),
                                        P.g.rc2, tp, use, n_in, ov);
        fix_add(acc, phi0, sgn0);
        if (NQ == 2) {
            int ov1 = 0;
            const float dy1 = __fsub_rn(e.ay1, by);
            const float phi1 = pair_phi_sel(cart_dx(P.g, __fsub_rn(e.ax1, bx), dy1), dy1, __fsub_rn(e.az1, bz),
                                            P.g.rc2, tp, use, n_in, ov1);
            fix_add(acc, phi1, -1);
        }
        started += __popc(starts);
    }
    overlap |= ov;
    __syncwarp();
}

// Fixed-point energy of NQ queries (sharing one surface column) against the
// images of frozen surface atoms listed for that column.  Each listed image
// holds its coordinate already shifted by minus the period where that is
// exact; flag bits ask for the query to be shifted by minus the period instead.
template <int NQ, bool CL>
__device__ __forceinline__ void surface_pass(const SweepParams& P, int col, float q0x, float q0y, float q0z,
                                             float q1x, float q1y, float q1z, int sgn0, Fix3& acc, int& n_in,
                                             int& n_cand, int& overlap, int lane, bool mA) {
    const int beg = col * P.st.stride, end = beg + P.st.stride;
    int ov = 0;
    for (int j = beg + lane; j < end; j += 32) {
        const float4 a = __ldg(&P.st.atoms[j]);
        const unsigned bits = __float_as_uint(a.w);
        const PairTab& t = (CL && mA) ? P.gsA[bits & 3u] : surf_tab(P, (int)(bits & 3u));
        const float sx = (bits & 4u) ? P.g.Lx : 0.f, sy = (bits & 8u) ? P.g.Ly : 0.f;
        const float sz = (bits & 16u) ? P.g.Lz : 0.f;
        if (!(bits & 32u)) n_cand += NQ;   // padding slots are not candidates
        const float dy0 = __fsub_rn(__fsub_rn(q0y, sy), a.y);
        const float phi0 = pair_phi_sel(cart_dx(P.g, __fsub_rn(__fsub_rn(q0x, sx), a.x), dy0), dy0,
                                        __fsub_rn(__fsub_rn(q0z, sz), a.z), P.g.rc2, t, true, n_in, ov);
        fix_add(acc, phi0, sgn0);
        if (NQ == 2) {
            int ov1 = 0;
            const float dy1 = __fsub_rn(__fsub_rn(q1y, sy), a.y);
            const float phi1 = pair_phi_sel(cart_dx(P.g, __fsub_rn(__fsub_rn(q1x, sx), a.x), dy1), dy1,
                                            __fsub_rn(__fsub_rn(q1z, sz), a.z), P.g.rc2, t, true, n_in, ov1);
            fix_add(acc, phi1, -1);
        }
    }
    overlap |= ov;
}

// Surrogate features of NQ queries (sharing the stencil of cell c) from the
// mobile particles of the stencil except `skip`, accumulated per lane.
template <int NQ, bool CL>
__device__ __forceinline__ void feature_mobile(const SweepParams& P, const WalkerSmem& S, Cell3 c, float q0x,
                                               float q0y, float q0z, float q1x, float q1y, float q1z, int skip,
                                               float (&F0)[kNF], float (&F1)[kNF], int lane, int warp,
                                               int split, const MoveTabs& mt) {
    StEntry* st = S.stencil + warp * 32;
    StEntry se = stencil_entry(P, c, lane, q0x, q0y, q0z, q1x, q1y, q1z);
    const int cnt = se.cell >= 0 ? (int)S.cnt[se.cell] : 0;
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += t;
    }
    const int excl = incl - cnt;
    const int total = __shfl_sync(FULL, incl, 31);
    const unsigned nonempty = __ballot_sync(FULL, cnt > 0);
    if (cnt > 0) {
        se.excl = excl;
        st[__popc(nonempty & lanemask_lt(lane))] = se;
    }
    __syncwarp();
    int started = 0;
    for (int base = 0; base < total; base += 32) {
        const unsigned bit = (cnt > 0 && excl >= base && excl < base + 32) ? (1u << (excl - base)) : 0u;
        const unsigned starts = __reduce_or_sync(FULL, bit);
        const int j = base + lane;
        if (j < total) {
            const int r = started + __popc(starts & lanemask_le(lane)) - 1;
            const StEntry& e = st[r];
            const int pj = S.slots[e.cell * P.cg.cap + (j - e.excl)];
            if (pj != skip) {
                const float4 p = S.pos[pj];
                const float bx = __fsub_rn(p.x, e.obx), by = __fsub_rn(p.y, e.oby), bz = __fsub_rn(p.z, e.obz);
                const float dy0 = __fsub_rn(e.ay0, by);
                const float r20 = r2_of(cart_dx(P.g, __fsub_rn(e.ax0, bx), dy0), dy0, __fsub_rn(e.az0, bz));
                const float wp = CL ? (pj < split ? mt.tA.eps : mt.tB.eps) : P.gg.eps;
                if (r20 < P.g.rc2) add_features(F0, r20, wp, P.g.rc);
                if (NQ == 2) {
                    const float dy1 = __fsub_rn(e.ay1, by);
                    const float r21 = r2_of(cart_dx(P.g, __fsub_rn(e.ax1, bx), dy1), dy1, __fsub_rn(e.az1, bz));
                    if (r21 < P.g.rc2) add_features(F1, r21, wp, P.g.rc);
                }
            }
        }
        started += __popc(starts);
    }
    __syncwarp();
}

// Surrogate features of NQ queries (sharing one surface column) from the
// images of frozen surface atoms listed for that column.
template <int NQ, bool CL>
__device__ __forceinline__ void feature_surface(const SweepParams& P, int col, float q0x, float q0y, float q0z,
                                                float q1x, float q1y, float q1z, float (&F0)[kNF],
                                                float (&F1)[kNF], int lane, bool mA) {
    const int beg = col * P.st.stride, end = beg + P.st.stride;
    for (int j = beg + lane; j < end; j += 32) {
        const float4 a = __ldg(&P.st.atoms[j]);
        const unsigned bits = __float_as_uint(a.w);
        const PairTab& t = (CL && mA) ? P.gsA[bits & 3u] : surf_tab(P, (int)(bits & 3u));
        const float sx = (bits & 4u) ? P.g.Lx : 0.f, sy = (bits & 8u) ? P.g.Ly : 0.f;
        const float sz = (bits & 16u) ? P.g.Lz : 0.f;
        const float dy0 = __fsub_rn(__fsub_rn(q0y, sy), a.y);
        const float r20 = r2_of(cart_dx(P.g, __fsub_rn(__fsub_rn(q0x, sx), a.x), dy0), dy0,
                                __fsub_rn(__fsub_rn(q0z, sz), a.z));
        if (r20 < P.g.rc2) add_features(F0, r20, t.eps, P.g.rc);
        if (NQ == 2) {
            const float dy1 = __fsub_rn(__fsub_rn(q1y, sy), a.y);
            const float r21 = r2_of(cart_dx(P.g, __fsub_rn(__fsub_rn(q1x, sx), a.x), dy1), dy1,
                                    __fsub_rn(__fsub_rn(q1z, sz), a.z));
            if (r21 < P.g.rc2) add_features(F1, r21, t.eps, P.g.rc);
        }
    }
}

// Remove a particle (whose packed w gives its cell and slot) from its cell.
__device__ __forceinline__ void cell_remove(const SweepParams& P, const WalkerSmem& S, float wbits) {
    const int c = cell_bits(wbits), s = slot_bits(wbits);
    if (c >= P.cg.ncell || s >= P.cg.cap || s >= (int)S.cnt[c]) {
        // only reachable after a capacity overflow left a particle out of the list
        atomicOr(P.error, ERR_CAPACITY);
        return;
    }
    const int last = S.cnt[c] - 1;
    const int moved = S.slots[c * P.cg.cap + last];
    S.slots[c * P.cg.cap + s] = (uint16_t)moved;
    S.pos[moved].w = __uint_as_float(((unsigned)c << 16) | (unsigned)s);
    S.cnt[c] = (uint16_t)last;
}

// Deterministic cell build of the walker's staged positions by warp 0.
__device__ __forceinline__ void build_cells(const SweepParams& P, const WalkerSmem& S, int N, int lane) {
    build_cell_list(P, S.pos, N, S.cnt, S.slots, lane);
}

// Evaluate trial move m of the launch (sweep m / mps, move m % mps) with one
// warp against the current configuration with N particles; lane 0 stores the
// result in *out.
template <bool DA, bool CL>
__device__ void evaluate_move(const SweepParams& P, const WalkerSmem& S, const StateF& sf, int s, int m, int N,
                              int slot, int split_in, int& n_in, int& n_cand, int lane, int warp, const NetFrag* nf,
                              MoveRes* out) {
    // Two mobile species (CL): particles [0, split) are of the first, the
    // rest of the second -- a cluster (split = n_cluster, moved only by
    // displacement; insertion and removal act on the gas after it) or two
    // grand-canonical species B and C (split = N_B, gc2).
    const int split = CL ? split_in : 0;
    const uint4 A = S.rng[2 * (m % kRing)], B = S.rng[2 * (m % kRing) + 1];
    // the species of a grand-canonical move: the second (the gas after a
    // cluster), or with two grand-canonical species the one bit 30 of B2 picks
    const int gy = (CL && P.gc2) ? (int)((B.z >> 30) & 1u) : 1;
    const int gcnt = gy ? N - split : split;          // its count before the move
    const bool use2 = CL && P.gc2 && gy == 1;         // species C's constants
    const float cins_f = use2 ? sf.c_ins2 : sf.c_ins, cdel_f = use2 ? sf.c_del2 : sf.c_del;
    // the kind of move: drawn from A0 in a sweep (slot -1), fixed by its place
    // in a REGC cycle step (slot 1: the particle exchange, 0: a displacement)
    const int gc_type = (B.z >> 31) == 0u ? 2 : 1;
    const int type = slot < 0 ? ((unsigned long long)A.x < P.th_disp ? 0 : gc_type) : (slot ? gc_type : 0);
    int status = 0, idx = -1, overlap = 0;
    const int n_in0 = n_in;
    float q0x = 0.f, q0y = 0.f, q0z = 0.f, q1x = 0.f, q1y = 0.f, q1z = 0.f;
    int sgn0 = 1, nq = 1;
    if (type == 0) {
        if (N == 0) {
            status = 1;
        } else {
            idx = (int)(((unsigned long long)B.x * (unsigned)N) >> 32);
            const float4 old = S.pos[idx];
            const float dx = __fmul_rn(P.max_disp, __fsub_rn(__fmul_rn(2.0f, u24(A.y)), 1.0f));
            const float dy = __fmul_rn(P.max_disp, __fsub_rn(__fmul_rn(2.0f, u24(A.z)), 1.0f));
            const float dz = __fmul_rn(P.max_disp, __fsub_rn(__fmul_rn(2.0f, u24(A.w)), 1.0f));
            float nx = __fadd_rn(old.x, dx), ny = __fadd_rn(old.y, dy), nz = __fadd_rn(old.z, dz);
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
            q0x = nx; q0y = ny; q0z = nz;
            q1x = old.x; q1y = old.y; q1z = old.z;
            nq = 2;
        }
    } else if (type == 1) {
        if (N == P.nmax) {
            status = 1;
        } else {
            float nx = __fmul_rn(P.g.Lx, u24(A.y));
            float ny = __fmul_rn(P.g.Ly, u24(A.z));
            float nz = __fadd_rn(P.g.z_lo, __fmul_rn(P.g.height, u24(A.w)));
            if (nx >= P.g.Lx) nx = __fsub_rn(nx, P.g.Lx);
            if (ny >= P.g.Ly) ny = __fsub_rn(ny, P.g.Ly);
            if (P.g.periodic_z && nz >= P.g.Lz) nz = __fsub_rn(nz, P.g.Lz);
            q0x = q1x = nx; q0y = q1y = ny; q0z = q1z = nz;
        }
    } else {
        if (gcnt == 0) {
            status = 1;
        } else {
            idx = (gy ? split : 0) + (int)(((unsigned long long)B.x * (unsigned)gcnt) >> 32);
            const float4 old = S.pos[idx];
            q0x = q1x = old.x; q0y = q1y = old.y; q0z = q1z = old.z;
            sgn0 = -1;
        }
    }
    // pair tables of the moving species
    MoveTabs mt;
    mt.mA = CL && ((type != 1 && idx >= 0 && idx < split) || (type == 1 && gy == 0));
    if (CL) {
        mt.tA = mt.mA ? P.gA : P.gAB;
        mt.tB = mt.mA ? P.gAB : P.gg;
    }

    // delayed acceptance, stage 1: the surrogate energy change dE~
    int stage1 = 1;
    float dEs = 0.f;
    if (DA && status == 0) {
        float F0[kNF], F1[kNF];
#pragma unroll
        for (int k = 0; k < kNF; ++k) F0[k] = F1[k] = 0.f;
        const int skip = type == 1 ? -1 : idx;
        const Cell3 c0 = cell3_of(P, q0x, q0y, q0z);
        const Cell3 c1 = nq == 2 ? cell3_of(P, q1x, q1y, q1z) : c0;
        if (nq == 2 && c0.x == c1.x && c0.y == c1.y && c0.z == c1.z) {
            feature_mobile<2, CL>(P, S, c0, q0x, q0y, q0z, q1x, q1y, q1z, skip, F0, F1, lane, warp, split, mt);
        } else {
            feature_mobile<1, CL>(P, S, c0, q0x, q0y, q0z, q0x, q0y, q0z, skip, F0, F1, lane, warp, split, mt);
            if (nq == 2)
                feature_mobile<1, CL>(P, S, c1, q1x, q1y, q1z, q1x, q1y, q1z, skip, F1, F0, lane, warp, split, mt);
        }
        const bool s0 = near_surface(P, q0z), s1 = nq == 2 && near_surface(P, q1z);
        const int col0 = surface_col(P, q0x, q0y), col1 = nq == 2 ? surface_col(P, q1x, q1y) : col0;
        if (s0 && s1 && col0 == col1) {
            feature_surface<2, CL>(P, col0, q0x, q0y, q0z, q1x, q1y, q1z, F0, F1, lane, mt.mA);
        } else {
            if (s0) feature_surface<1, CL>(P, col0, q0x, q0y, q0z, q0x, q0y, q0z, F0, F1, lane, mt.mA);
            if (s1) feature_surface<1, CL>(P, col1, q1x, q1y, q1z, q1x, q1y, q1z, F1, F0, lane, mt.mA);
        }
        // both positions through the network at once: rows 0 and 1 of the tiles
        const float r0 = warp_reduce16(F0, lane);
        const float r1 = nq == 2 ? warp_reduce16(F1, lane) : 0.f;
        uint32_t a[4];
        features_to_frag(r0, r1, lane, a);
        float e1 = 0.f;
        const float e0 = net_mma(*nf, a, &e1);
        dEs = type == 1 ? e0 : (type == 2 ? -e0 : e0 - e1);
        // ln u1 < ln alpha with dE~ in place of dE (u1 from B3)
        float c_f = 0.f;
        if (type == 1) c_f = cins_f - __logf((float)(gcnt + 1));
        else if (type == 2) c_f = cdel_f + __logf((float)gcnt);
        const float la1 = c_f - sf.beta * dEs;
        const float lu1 = __logf(((float)B.w + 0.5f) * 2.3283064365386963e-10f);
        if (la1 >= 0.f || lu1 < la1 - 1e-3f) stage1 = 1;
        else if (lu1 > la1 + 1e-3f) stage1 = 0;
        else {
            double c = 0.0;
            if (type == 1) c = (use2 ? P.c_ins2[s] : P.c_ins[s]) - P.ln_tab[gcnt + 1];
            else if (type == 2) c = (use2 ? P.c_del2[s] : P.c_del[s]) + P.ln_tab[gcnt];
            stage1 = (log((double)B.w + 0.5) + kLn2m32) < c - P.beta[s] * (double)dEs;
        }
    }

    Fix3 acc{0, 0, 0};
    if (status == 0 && stage1) {
        const int skip = type == 1 ? -1 : idx;
        const Cell3 c0 = cell3_of(P, q0x, q0y, q0z);
        const Cell3 c1 = nq == 2 ? cell3_of(P, q1x, q1y, q1z) : c0;
        const bool same = c0.x == c1.x && c0.y == c1.y && c0.z == c1.z;
        if (nq == 2 && same) {
            mobile_pass<2, CL>(P, S, c0, q0x, q0y, q0z, q1x, q1y, q1z, skip, 1, acc, n_in, n_cand, overlap, lane, warp,
                               split, mt);
        } else {
            // one pass per query: query 0 with its sign, then (a displacement
            // across cells) the old position with -1
            for (int pass = 0; pass < nq; ++pass) {
                const float px = pass ? q1x : q0x, py = pass ? q1y : q0y, pz = pass ? q1z : q0z;
                int ovp = 0;
                mobile_pass<1, CL>(P, S, pass ? c1 : c0, px, py, pz, px, py, pz, skip, pass ? -1 : sgn0, acc, n_in,
                                   n_cand, ovp, lane, warp, split, mt);
                if (pass == 0) overlap |= ovp;
            }
        }
        const bool s0 = near_surface(P, q0z);
        const bool s1 = nq == 2 && near_surface(P, q1z);
        const int col0 = surface_col(P, q0x, q0y);
        const int col1 = nq == 2 ? surface_col(P, q1x, q1y) : col0;
        if (s0 && s1 && col0 == col1) {
            surface_pass<2, CL>(P, col0, q0x, q0y, q0z, q1x, q1y, q1z, 1, acc, n_in, n_cand, overlap, lane, mt.mA);
        } else {
            for (int pass = 0; pass < nq; ++pass) {
                if (!(pass ? s1 : s0)) continue;
                const float px = pass ? q1x : q0x, py = pass ? q1y : q0y, pz = pass ? q1z : q0z;
                int ovp = 0;
                surface_pass<1, CL>(P, pass ? col1 : col0, px, py, pz, px, py, pz, pass ? -1 : sgn0, acc, n_in, n_cand,
                                ovp, lane, mt.mA);
                if (pass == 0) overlap |= ovp;
            }
        }
        if (type == 2) overlap = 0;   // the old position of a particle never overlaps
    }
    const int big = (int)__reduce_add_sync(FULL, (unsigned)acc.big);
    const int hi = (int)__reduce_add_sync(FULL, (unsigned)acc.hi);
    const int lo = (int)__reduce_add_sync(FULL, (unsigned)acc.lo);
    const int ovl = __any_sync(FULL, overlap) ? 1 : 0;
    const int npairs = (int)__reduce_add_sync(FULL, (unsigned)(n_in - n_in0));
    if (lane == 0) {
        MoveRes r;
        r.type = type;
        r.status = status;
        r.idx = idx;
        r.n_eval = N;
        r.big = big;
        r.hi = hi;
        r.lo = lo;
        r.flags = ovl | (npairs << 1);
        r.q0x = q0x; r.q0y = q0y; r.q0z = q0z;
        r.q1x = q1x; r.q1y = q1y; r.q1z = q1z;
        r.stage1 = stage1;
        r.dE_sur = dEs;
        r.gy = gy;
        if (!DA) {
            r.dec = (status == 0 && !ovl) ? pretest(StateF{sf.beta, cins_f, cdel_f, 0.f, 0.f}, type, gcnt, big, hi,
                                                    lo, B.y)
                                          : 0;
        } else if (status != 0 || ovl || !stage1) {
            r.dec = 0;
        } else {
            // stage 2: ln u2 < -beta (dE - dE~) (u2 from B1)
            const float de_f = __fmaf_rn((float)lo, 9.313225746154785e-10f,
                                         __fmaf_rn((float)hi, 0.00390625f, (float)big * 8192.0f));
            const float la2 = -sf.beta * (de_f - dEs);
            const float lu2 = __logf(((float)B.y + 0.5f) * 2.3283064365386963e-10f);
            if (la2 >= 0.f || lu2 < la2 - 1e-3f) r.dec = 1;
            else if (lu2 > la2 + 1e-3f) r.dec = 0;
            else
                r.dec = (log((double)B.y + 0.5) + kLn2m32) <
                        -P.beta[s] * ((double)fix_value(big, hi, lo) * kFixUnit - (double)dEs);
        }
        *out = r;
    }
}

// floor(d / bin) for d >= 0 and bin >= 1 from the FP64 quotient (inv = 1 / bin
// in FP64): within one of it while the quotient is below 2^52, so one
// correction settles it; the integer division remains for anything beyond.
__device__ __forceinline__ long long floor_div_fp64(long long d, long long bin, double inv) {
    long long q = (long long)((double)d * inv);
    if (q * bin > d) --q;
    else if ((q + 1) * bin <= d) ++q;
    if (q < 0 || q * bin > d || (q + 1) * bin <= d) q = d / bin;
    return q;
}

// One observation of energy E (2^-30 units) into state s's own histogram:
// bin 0 below the window, k + 1 for window bin k, hE_bins + 1 at or beyond its end.
__device__ __forceinline__ void observe_state_energy(const SweepParams& P, int s, long long E, double inv_bin) {
    const long long d = E - P.hE_lo_fix[s];
    const long long kb = d >= 0 ? floor_div_fp64(d, P.hE_bin_fix, inv_bin) : -1;
    const int idx = kb < 0 ? 0 : (kb >= P.hE_bins ? P.hE_bins + 1 : (int)kb + 1);
    atomicAdd(&P.hE[size_t(s) * (P.hE_bins + 2) + idx], 1ull);
}

// Squared minimum-image distance in binary32 (periodic axes per geometry).
__device__ __forceinline__ float dist2(const SweepParams& P, float ax, float ay, float az, float bx, float by,
                                       float bz) {
    const float dy = min_image_exact(ay, by, P.g.Ly, P.g.hLy);
    const float dx = cart_dx(P.g, min_image_exact(ax, bx, P.g.Lx, P.g.hLx), dy);
    const float dz = P.g.periodic_z ? min_image_exact(az, bz, P.g.Lz, P.g.hLz) : __fsub_rn(az, bz);
    return r2_of(dx, dy, dz);
}

// n_sweeps sweeps of walker w by a group of K warps (tid: thread index in the
// group, smem: the group's shared-memory region, bar: the group's named
// barrier when K > 1).
template <int K, bool TRACE, bool DA, bool CL>
__device__ __forceinline__ void walker_sweep(const SweepParams& P, int w, char* smem, int tid, int bar) {
    const int lane = tid & 31, warp = tid >> 5;
    const WalkerSmem S = carve<K>(smem, P);

    int N = P.n[w];
    long long E = P.efix[w];
    const int s = P.state_of_walker[w];
    const bool two = CL && P.gc2;
    // two mobile species: particles [0, split) are the cluster, or species B
    // of two grand-canonical species (then split = N_B changes with the moves)
    int split = CL ? (two ? P.nb[w] : P.n_cluster) : 0;
    const StateF sf{P.beta_f[s], P.c_ins_f[s], P.c_del_f[s], two ? P.c_ins2_f[s] : 0.f,
                    two ? P.c_del2_f[s] : 0.f};
    float4* gpos = P.pos + size_t(w) * P.nmax;

    // 1. stage positions with a bulk copy
    if (N > 0) {
        if (tid == 0) {
            mbar_init(S.bar);
            // the region may have been read and written by ordinary accesses
            // (a previous walker): order those before the asynchronous copy
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            if (!P.expire_waits) bulk_load(S.pos, gpos, uint32_t(N) * 16u, S.bar);
        }
        group_sync<K>(bar);
        const bool ok = mbar_wait_bounded(S.bar);
        const bool all_ok = group_all<K>(bar, ok);
        if (!all_ok) {
            if (tid == 0) atomicOr(P.error, ERR_TIMEOUT);
            mbar_wait_bounded(S.bar);  // one more bounded chance for the copy in flight
            return;
        }
        group_sync<K>(bar);
        if (tid == 0) mbar_inval(S.bar);   // the barrier's memory is reused by the next walker
    }
    // 2. cell list
    if (warp == 0) build_cells(P, S, N, lane);
    if (tid == 0)
        *S.stats = WalkerStats{0, 0, 0, 0.0, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull, {0, 0, 0}, {0, 0, 0}, 0, 0};
    group_sync<K>(bar);

    int n_in = 0, n_cand = 0;
    NetFrag nf;                       // the surrogate's weights in this lane's fragments
    if (DA) load_net(P.net, lane, nf);
    const int total_moves = P.n_sweeps * P.mps;
    const float rc_guard = P.g.rc2 * 1.0004f + 1e-6f;   // a little beyond rc, conservatively
    int filled = 0;   // moves whose Philox blocks are in the ring
    int m0 = P.m_first;   // first move of the round
    // the committer's statistics and move place, in its registers
    WalkerStats sr = WalkerStats{0, 0, 0, 0.0, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull, {0, 0, 0}, {0, 0, 0}, 0, 0};
    int kcur = P.m_first % P.mps;
    // energy bins of the observations without a 64-bit integer division
    const double inv_ebin = 1.0 / (double)P.e_bin_fix;
    const double inv_hebin = P.hE ? 1.0 / (double)P.hE_bin_fix : 0.0;

    while (m0 < total_moves) {
        // 3a. Philox blocks of the next 32 moves, drawn by all lanes at once
        if (m0 + K > filled) {
            for (int q = tid; q < 64; q += 32 * K) {
                const int m = filled + (q >> 1);
                if (m < total_moves) {
                    const int ts = m / P.mps;
                    const U4 v = philox(uint32_t(m - ts * P.mps), P.t0 + uint32_t(ts), uint32_t(w), uint32_t(q & 1),
                                        P.key0, P.key1);
                    S.rng[2 * (m % kRing) + (q & 1)] = make_uint4(v.x, v.y, v.z, v.w);
                }
            }
            filled += 32;
            group_sync<K>(bar);
        }
        // 3b. evaluate moves m0 .. m0 + K - 1 in parallel, one warp each
        const int mj = m0 + warp;
        if (mj < total_moves) {
            int slot = -1;
            if (P.cycle) slot = (mj % P.mps) == 0;
            evaluate_move<DA, CL>(P, S, sf, s, mj, N, slot, split, n_in, n_cand, lane, warp, &nf, S.res + warp);
        }
        group_sync<K>(bar);

        // 4. commit in order (thread 0)
        int committed = 0;
        if (tid == 0) {
            bool any_acc = false, n_changed = false;
            float chx[2 * K], chy[2 * K], chz[2 * K];   // positions changed by accepted moves
            int nch = 0;
            // not unrolled: one copy of the commit keeps the speculative kernels'
            // code small enough for the instruction caches (K = 4: 153 -> 86 KB)
#pragma unroll 1
            for (int j = 0; j < K && m0 + j < total_moves; ++j) {
                const MoveRes r = S.res[j];
                const int m = m0 + j;
                // is the evaluation still the one the sequential chain would make?
                if (any_acc) {
                    bool valid = true;
                    if (n_changed && r.type != 1) valid = false;                    // index of N picked
                    if (r.type == 1 && r.status == 1 && N != P.nmax) valid = false;  // no longer full
                    // a changed position within rc of a query point: the energy
                    // change would differ; the old position of a displacement is
                    // checked whatever its status, since its particle may have moved
                    if (valid && (r.status == 0 || (r.type == 0 && r.status == 2))) {
#pragma unroll 1   // rolled for the same reason as the commit loop
                        for (int c = 0; c < nch; ++c) {
                            if (r.status == 0 && dist2(P, chx[c], chy[c], chz[c], r.q0x, r.q0y, r.q0z) < rc_guard)
                                valid = false;
                            if (r.type == 0 && dist2(P, chx[c], chy[c], chz[c], r.q1x, r.q1y, r.q1z) < rc_guard)
                                valid = false;
                        }
                    }
                    if (!valid) break;
                }
                const uint4 B = S.rng[2 * (m % kRing) + 1];
                int status = r.status;
                if (r.type == 1 && N == P.nmax) status = 1;    // became full in this round
                const long long dfix = fix_value(r.big, r.hi, r.lo);
                // capacity of the destination cell
                int c_new = -1;
                float4 old = make_float4(0.f, 0.f, 0.f, 0.f);
                if (r.type != 1 && status != 1) old = S.pos[r.idx];
                if (status == 0 && r.type != 2) {
                    c_new = cell_of(P, r.q0x, r.q0y, r.q0z);
                    const bool stay = r.type == 0 && c_new == cell_bits(old.w);
                    if (!stay && S.cnt[c_new] >= P.cg.cap) {
                        status = 3;
                        atomicOr(P.error, ERR_CAPACITY);
                    }
                }
                // 5. acceptance: ln u < ln alpha (pre-tested in the evaluating warp
                // when N is still the one it saw)
                int accepted = 0;
                double la = 0.0;
                const bool ovl = (r.flags & 1) != 0;
                // the grand-canonical species of the move: its count and constants
                const int gcnt = (CL && r.gy == 0) ? split : N - split;
                const bool use2 = two && r.gy == 1;
                const double* cins = use2 ? P.c_ins2 : P.c_ins;
                const double* cdel = use2 ? P.c_del2 : P.c_del;
                if (DA && status == 0) {
                    // both stages were decided by the evaluating warp (one warp per walker)
                    accepted = !ovl && r.dec == 1;
                    sr.screened += 1;
                    sr.passed += r.stage1;
                    if (TRACE) {
                        double c = 0.0;
                        if (r.type == 1) c = cins[s] - P.ln_tab[gcnt + 1];
                        else if (r.type == 2) c = cdel[s] + P.ln_tab[gcnt];
                        la = r.stage1 ? c - P.beta[s] * ((double)dfix * kFixUnit) : (double)NAN;
                    }
                } else if (status == 0 && !ovl) {
                    const int dec = N == r.n_eval ? r.dec
                                                  : pretest(StateF{sf.beta, use2 ? sf.c_ins2 : sf.c_ins,
                                                                   use2 ? sf.c_del2 : sf.c_del, 0.f, 0.f},
                                                            r.type, gcnt, r.big, r.hi, r.lo, B.y);
                    accepted = dec == 1;
                    if (dec == 2 || TRACE) {
                        double c = 0.0;
                        if (r.type == 1) c = cins[s] - P.ln_tab[gcnt + 1];
                        else if (r.type == 2) c = cdel[s] + P.ln_tab[gcnt];
                        la = c - P.beta[s] * ((double)dfix * kFixUnit);
                        if (dec == 2) accepted = (log((double)B.y + 0.5) + kLn2m32) < la;
                    }
                }
                const int n_before = N, split_before = split;
                if (accepted) {
                    const int cap = P.cg.cap;
                    if (r.type == 0) {
                        const int c_old = cell_bits(old.w);
                        if (c_new == c_old) {
                            S.pos[r.idx] = make_float4(r.q0x, r.q0y, r.q0z, old.w);
                        } else {
                            cell_remove(P, S, old.w);
                            const int sl = S.cnt[c_new];
                            S.slots[c_new * cap + sl] = (uint16_t)r.idx;
                            S.cnt[c_new] = (uint16_t)(sl + 1);
                            S.pos[r.idx] = packed(r.q0x, r.q0y, r.q0z, c_new, sl);
                        }
                        chx[nch] = r.q0x; chy[nch] = r.q0y; chz[nch] = r.q0z; ++nch;
                        chx[nch] = r.q1x; chy[nch] = r.q1y; chz[nch] = r.q1z; ++nch;
                    } else if (r.type == 1) {
                        // a new particle goes to the end, or (species B of two
                        // grand-canonical species) to index split, whose C moves to the end
                        int at = N;
                        if (two && r.gy == 0) {
                            at = split;
                            if (split < N) {
                                const float4 pc = S.pos[split];
                                S.pos[N] = pc;
                                S.slots[cell_bits(pc.w) * cap + slot_bits(pc.w)] = (uint16_t)N;
                            }
                            split += 1;
                        }
                        const int sl = S.cnt[c_new];
                        S.slots[c_new * cap + sl] = (uint16_t)at;
                        S.cnt[c_new] = (uint16_t)(sl + 1);
                        S.pos[at] = packed(r.q0x, r.q0y, r.q0z, c_new, sl);
                        chx[nch] = r.q0x; chy[nch] = r.q0y; chz[nch] = r.q0z; ++nch;
                        n_changed = true;
                    } else {
                        cell_remove(P, S, old.w);
                        const int last = N - 1;
                        // the gap is filled from the end of the particle's block; a
                        // removed B's block end is then filled by the last C
                        const int fill = (two && r.gy == 0) ? split - 1 : last;
                        if (r.idx != fill) {
                            const float4 pl = S.pos[fill];
                            S.pos[r.idx] = pl;
                            S.slots[cell_bits(pl.w) * cap + slot_bits(pl.w)] = (uint16_t)r.idx;
                        }
                        if (fill != last) {
                            const float4 pc = S.pos[last];
                            S.pos[fill] = pc;
                            S.slots[cell_bits(pc.w) * cap + slot_bits(pc.w)] = (uint16_t)fill;
                        }
                        if (two && r.gy == 0) split -= 1;
                        chx[nch] = r.q0x; chy[nch] = r.q0y; chz[nch] = r.q0z; ++nch;
                        n_changed = true;
                    }
                    any_acc = true;
                    E += dfix;
                    N += (r.type == 1) - (r.type == 2);
                }
                WalkerStats& st = sr;
                st.tr[0] += r.type == 0;
                st.tr[1] += r.type == 1;
                st.tr[2] += r.type == 2;
                st.ac[0] += accepted && r.type == 0;
                st.ac[1] += accepted && r.type == 1;
                st.ac[2] += accepted && r.type == 2;
                // pairs that entered dE (a move that became impossible in this
                // round, status 1, has none, whatever its evaluation counted)
                if (status != 1) st.pairs += (unsigned)(r.flags >> 1);
                const int k = kcur;
                kcur = kcur + 1 == P.mps ? 0 : kcur + 1;
                if (TRACE) {
                    const int ts = m / P.mps;
                    regc_move_record t;
                    t.type = r.type;
                    t.index = status == 1 ? 0 : (r.type == 1 ? ((two && r.gy == 0) ? split_before : n_before) : r.idx);
                    t.accepted = accepted;
                    t.status = status == 3 ? 0 : status;
                    t.dE = (status == 0 || status == 3) ? (double)dfix * kFixUnit : 0.0;
                    if (DA && status == 0 && !r.stage1) t.dE = (double)NAN;
                    t.log_alpha = (status == 0 || status == 3) ? (ovl ? -INFINITY : la) : 0.0;
                    t.ln_u = log((double)B.y + 0.5) + kLn2m32;
                    t.sum_abs = 0.0;
                    t.band = 0.0;
                    t.n_pairs = r.flags >> 1;
                    t.stage1 = DA ? r.stage1 : 1;
                    t.dE_sur = DA ? (double)r.dE_sur : 0.0;
                    t.ln_u1 = log((double)B.w + 0.5) + kLn2m32;
                    P.trace[(size_t(w) * P.trace_steps + ts) * P.mps + k] = t;
                }
                // 6. observe once per sweep into the current state's histograms
                if (k == P.mps - 1) {
                    // N_B: the grand-canonical count (with two species, species B's)
                    const int NB = two ? split : N - split;
                    const int NC = two ? N - split : 0;
                    atomicAdd(&P.hN[size_t(s) * (P.nmax + 1) + NB], 1ull);   // fire-and-forget reduction
                    if (two) {
                        atomicAdd(&P.hN2[size_t(s) * (P.nmax + 1) + NC], 1ull);
                        st.mC += NC;
                        st.mC2 += (long long)NC * NC;
                    }
                    st.om += 1;
                    st.mN += NB;
                    st.mN2 += (long long)NB * NB;
                    st.mE += E;
                    const double e = (double)E * kFixUnit;
                    st.mE2 = fma(e, e, st.mE2);
                    const long long d = E - P.e_lo_fix;
                    const long long kb = d >= 0 ? floor_div_fp64(d, P.e_bin_fix, inv_ebin) : -1;
                    const size_t row = two ? size_t(NB) * (P.nmax + 1) + NC : size_t(NB);
                    if (kb >= 0 && kb < P.n_e_bins) atomicAdd(&P.hNE[row * P.n_e_bins + (size_t)kb], 1ull);
                    else st.eo += 1;
                    if (P.hE) observe_state_energy(P, s, E, inv_hebin);
                }
                ++committed;
            }
            if (K > 1) {
                S.hdr->N = N;
                S.hdr->E = E;
                S.hdr->split = split;
                S.hdr->committed = committed;
            }
            sr.rounds += 1;
            sr.evals += min(K, total_moves - m0);
        }
        group_sync<K>(bar);
        if (K == 1) {
            // the committer is lane 0 of the walker's one warp
            N = __shfl_sync(FULL, N, 0);
            E = __shfl_sync(FULL, E, 0);
            split = __shfl_sync(FULL, split, 0);
            m0 += __shfl_sync(FULL, committed, 0);
        } else {
            N = S.hdr->N;
            E = S.hdr->E;
            split = S.hdr->split;
            m0 += S.hdr->committed;
            group_sync<K>(bar);   // the header and results are rewritten by the next round
        }
    }

    if (tid == 0) *S.stats = sr;
    group_sync<K>(bar);
    // 7. write back
    for (int j = tid; j < N; j += 32 * K) gpos[j] = S.pos[j];
    // candidate distances evaluated (all evaluations, kept or not)
    const unsigned sum_cand = __reduce_add_sync(FULL, (unsigned)n_cand);
    if (lane == 0) atomicAdd(&P.pair_counts[1], (unsigned long long)sum_cand);
    if (tid == 0) {
        const WalkerStats& st = *S.stats;
        atomicAdd(&P.pair_counts[0], st.pairs);
        atomicAdd(&P.pair_counts[2], st.rounds);
        atomicAdd(&P.pair_counts[3], st.evals);
        atomicAdd(&P.pair_counts[4], st.screened);
        atomicAdd(&P.pair_counts[5], st.passed);
        P.n[w] = N;
        if (two) {
            P.nb[w] = split;
            P.moments2[size_t(s) * 2] += (double)st.mC;
            P.moments2[size_t(s) * 2 + 1] += (double)st.mC2;
        }
        P.efix[w] = E;
        P.omega[s] += st.om;
        P.e_out[s] += st.eo;
        double* mm = P.moments + size_t(s) * 4;
        mm[0] += (double)st.mN;
        mm[1] += (double)st.mN2;
        mm[2] += (double)st.mE * kFixUnit;
        mm[3] += st.mE2;
        long long* mc = P.move_counts + size_t(w) * 6;
        for (int k = 0; k < 3; ++k) {
            mc[2 * k] += st.tr[k];
            mc[2 * k + 1] += st.ac[k];
        }
    }
}


template <int K, bool TRACE, bool DA, bool CL>
__global__ void __launch_bounds__(32 * K, K == 4 ? 7 : 1) sweep_kernel(const __grid_constant__ SweepParams P) {
    extern __shared__ __align__(16) char smem[];
    const int w = P.w_begin + (int)blockIdx.x;
    if (w >= P.w_end) return;
    walker_sweep<K, TRACE, DA, CL>(P, w, smem, threadIdx.x, 0);
}

// Displacement q - p with the exact minimum image on periodic axes (cell
// frame), x made Cartesian.
__device__ __forceinline__ void disp_exact(const Geometry& g, float4 q, float4 p, float& dx, float& dy, float& dz) {
    dy = min_image_exact(q.y, p.y, g.Ly, g.hLy);
    dx = cart_dx(g, min_image_exact(q.x, p.x, g.Lx, g.hLx), dy);
    dz = g.periodic_z ? min_image_exact(q.z, p.z, g.Lz, g.hLz) : __fsub_rn(q.z, p.z);
}

// From-scratch energy of every walker: every unordered pair of particles and
// every particle-surface pair, with the nearest periodic image.  A walker gets
// kEnergySplit CTAs of kEnergyThreads threads; its positions are staged in
// shared memory.  Two enumerations of the mobile pairs:
//
// * cells (the cell grid of the sweep has at least three cells along every
//   periodic axis, so the 27 cells around a cell are distinct): every CTA
//   builds the walker's cell list (shared-memory atomics; the order inside a
//   cell does not matter) and takes items (i, o) -- particle i against the
//   o-th cell of the forward half of its stencil (o = 0: its own cell, partners
//   j > i; o = 1..13: the 13 offsets after (0, 0, 0) in (z, y, x) order) --
//   which lists every pair within rc once;
// * all pairs (small periodic boxes, or a cell over capacity): the circulant
//   order (i, i + d mod N), d = 1 .. floor(N / 2) (for even N the offset N / 2
//   only from i < N / 2), which lists each unordered pair once and gives every
//   particle the same number of partners.
//
// Consecutive threads take consecutive items.  The displacement is
// antisymmetric under exchange of the pair (min_image_exact and cart_dx round
// -x to -fl(x)), so r^2, hence every pair term, is the one the sweep computes
// for that pair.  The surface partners of a particle come from its column of
// the surface table, one warp per particle, exactly as in the sweep.  Partial
// sums are folded to 64 bits before the int32 parts of a Fix3 can overflow and
// added to the walker's total with a 64-bit integer atomic: fixed-point sums do
// not depend on the order, so the result is deterministic and equals the
// sweep's running total exactly.
constexpr int kEnergyThreads = 256;
constexpr int kEnergySplit = 4;
constexpr int kEnergyTeam = kEnergySplit * kEnergyThreads;
constexpr int kFoldEvery = 256;   // pair terms per thread between folds (|lo| < 2^21 per term)

struct EnergyAcc {
    Fix3 acc;
    long long total;
    int folds, n_in, overlap;
    __device__ __forceinline__ void add(float phi) {
        fix_add(acc, phi, 1);
        if (++folds == kFoldEvery) fold();
    }
    __device__ __forceinline__ void fold() {
        total += fix_value(acc.big, acc.hi, acc.lo);
        acc = Fix3{0, 0, 0};
        folds = 0;
    }
};

template <bool CL>
__device__ __forceinline__ void energy_pair(const SweepParams& P, const float4* sp, int i, int j, int split,
                                            EnergyAcc& a) {
    const bool iA = CL && i < split, jA = CL && j < split;
    const PairTab& tp = iA ? (jA ? P.gA : P.gAB) : (jA ? P.gAB : P.gg);
    float dx, dy, dz;
    disp_exact(P.g, sp[i], sp[j], dx, dy, dz);
    a.add(pair_phi(dx, dy, dz, P.g.rc2, tp, a.n_in, a.overlap));
}

template <bool CL>
__global__ void __launch_bounds__(kEnergyThreads) energy_kernel(const __grid_constant__ SweepParams P,
                                                                unsigned long long* out, int check_overlap,
                                                                int use_cells) {
    extern __shared__ float4 sp[];   // [nmax] positions (w: packed cell), then cnt [ncell], slots [ncell][cap]
    int* cnt = reinterpret_cast<int*>(sp + P.nmax);
    uint16_t* slots = reinterpret_cast<uint16_t*>(cnt + ((P.cg.ncell + 3) & ~3));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int w = blockIdx.x / kEnergySplit, c = blockIdx.x % kEnergySplit;
    const int N = P.n[w];
    const int split = CL ? (P.gc2 ? P.nb[w] : P.n_cluster) : 0;   // two mobile species: the boundary
    const int t = c * kEnergyThreads + threadIdx.x;
    const float4* pos = P.pos + size_t(w) * P.nmax;
    if (use_cells)
        for (int k = threadIdx.x; k < P.cg.ncell; k += kEnergyThreads) cnt[k] = 0;
    for (int i = threadIdx.x; i < N; i += kEnergyThreads) {
        float4 q = pos[i];
        if (use_cells) {
            const Cell3 cc = cell3_of(P, q.x, q.y, q.z);
            q.w = __uint_as_float((unsigned)cc.x | ((unsigned)cc.y << 10) | ((unsigned)cc.z << 20));
        }
        sp[i] = q;
    }
    __syncthreads();
    bool cells = false;
    if (use_cells) {
        int full = 0;
        for (int i = threadIdx.x; i < N; i += kEnergyThreads) {
            const unsigned b = __float_as_uint(sp[i].w);
            const int cell = (int)(((b >> 20) * P.cg.ncy + ((b >> 10) & 1023u)) * P.cg.ncx + (b & 1023u));
            const int k = atomicAdd(cnt + cell, 1);
            if (k < P.cg.cap) slots[cell * P.cg.cap + k] = (uint16_t)i;
            else full = 1;
        }
        cells = !__syncthreads_or(full);   // identical in every CTA of the walker (counts are)
    }
    EnergyAcc a{{0, 0, 0}, 0, 0, 0, 0};
    if (cells) {
        // item k = 14 i + o; this thread takes k = t, t + T, ... (one division)
        int i = t / 14, o = t % 14;
        constexpr int qT = kEnergyTeam / 14, rT = kEnergyTeam % 14;
        while (i < N) {
            const unsigned b = __float_as_uint(sp[i].w);
            const int idx = 13 + o;   // offset (ox, oy, oz) = (idx % 3, idx / 3 % 3, idx / 9) - 1
            int nx = (int)(b & 1023u) + idx % 3 - 1;
            int ny = (int)((b >> 10) & 1023u) + (idx / 3) % 3 - 1;
            int nz = (int)(b >> 20) + idx / 9 - 1;
            if (nx < 0) nx += P.cg.ncx;
            else if (nx >= P.cg.ncx) nx -= P.cg.ncx;
            if (ny < 0) ny += P.cg.ncy;
            else if (ny >= P.cg.ncy) ny -= P.cg.ncy;
            bool ok = true;
            if (nz >= P.cg.ncz) {
                if (P.g.periodic_z) nz -= P.cg.ncz;
                else ok = false;
            }
            if (ok) {
                const int cell = (nz * P.cg.ncy + ny) * P.cg.ncx + nx;
                const int n_c = cnt[cell];
                const uint16_t* sl = slots + cell * P.cg.cap;
                for (int m = 0; m < n_c; ++m) {
                    const int j = sl[m];
                    if (o == 0 && j <= i) continue;
                    energy_pair<CL>(P, sp, i, j, split, a);
                }
            }
            o += rT;
            i += qT;
            if (o >= 14) {
                o -= 14;
                i += 1;
            }
        }
    } else if (N >= 2) {
        // item k = (d - 1) N + i, d = 1 .. D
        const int D = N >> 1;
        int i = t % N, d = t / N + 1;
        const int qT = kEnergyTeam / N, rT = kEnergyTeam % N;
        const bool even = (N & 1) == 0;
        while (d <= D) {
            if (!(even && d == D && i >= D)) {
                int j = i + d;
                if (j >= N) j -= N;
                energy_pair<CL>(P, sp, i, j, split, a);
            }
            i += rT;
            d += qT;
            if (i >= N) {
                i -= N;
                d += 1;
            }
        }
    }
    a.fold();
    // surface partners: one warp per particle
    for (int i = c * (kEnergyThreads / 32) + warp; i < N; i += kEnergyTeam / 32) {
        const float4 pi = sp[i];
        if (near_surface(P, pi.z)) {
            int n_cand = 0;
            surface_pass<1, CL>(P, surface_col(P, pi.x, pi.y), pi.x, pi.y, pi.z, pi.x, pi.y, pi.z, 1, a.acc,
                                a.n_in, n_cand, a.overlap, lane, CL && i < split);
            a.fold();
        }
    }
    // each warp adds its share (two's complement: exact, in any order) and
    // leaves; no barrier after the items, so a warp that finished early exits
    const long long total = warp_sum_ll(a.total);
    const int overlap = __any_sync(FULL, a.overlap);
    if (lane == 0) {
        if (total != 0) atomicAdd(out + w, (unsigned long long)total);
        if (overlap && check_overlap) atomicOr(P.error, check_overlap == 2 ? ERR_NUMERIC : ERR_OVERLAP);
    }
}

template <int K, bool DA, bool CL>
cudaError_t launch_k(const SweepParams& P, cudaStream_t s) {
    const size_t smem = smem_bytes(P.nmax, P.cg.ncell, P.cg.cap, K);
    const int n_walkers = P.w_end - P.w_begin;   // one CTA per walker of the shard
    if (n_walkers <= 0) return cudaSuccess;
    cudaError_t err;
    if (P.trace) {
        err = cudaFuncSetAttribute(sweep_kernel<K, true, DA, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem);
        if (err != cudaSuccess) return err;
        sweep_kernel<K, true, DA, CL><<<n_walkers, 32 * K, smem, s>>>(P);
    } else {
        err = cudaFuncSetAttribute(sweep_kernel<K, false, DA, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem);
        if (err != cudaSuccess) return err;
        sweep_kernel<K, false, DA, CL><<<n_walkers, 32 * K, smem, s>>>(P);
    }
    return cudaGetLastError();
}

// Persistent sweep of a batch of walkers from several systems.  Every group
// of K warps of the CTA is one walker at a time: its first thread takes the
// next (system, walker) item from the queue, the group copies that system's
// parameters into its slot of shared memory and runs the walker's sweeps in
// its own shared-memory region of `region` bytes (K > 1: the speculative
// walker, synchronised by the group's named barrier 1 + group); items are
// listed largest first, so the queue balances the uneven costs.  DA: the
// systems of the launch sample with delayed acceptance (their networks'
// fragments take ~240 registers per thread, so at most kBatchMaxWarpsDA
// walkers per CTA); CL: every system of the launch carries a cluster species.
constexpr int kBatchMaxWarps = 16;
constexpr int kBatchMaxWarpsDA = 4;

template <bool DA, bool CL, int K>
__global__ void __launch_bounds__(32 * (DA ? kBatchMaxWarpsDA : kBatchMaxWarps))
    batch_sweep_kernel(const SweepParams* __restrict__ sys, const int2* __restrict__ items, int n_items,
                       int* counter, int region) {
    constexpr int kGroups = (DA ? kBatchMaxWarpsDA : kBatchMaxWarps) / K;
    extern __shared__ __align__(16) char smem[];
    __shared__ SweepParams Psh[kGroups];
    __shared__ int item_sh[kGroups];
    const int tid = threadIdx.x % (32 * K), grp = threadIdx.x / (32 * K);
    const int bar = K == 1 ? 0 : 1 + grp;
    char* mine = smem + (size_t)grp * region;
    for (;;) {
        int item = 0;
        if (K == 1) {
            if (tid == 0) item = atomicAdd(counter, 1);
            item = __shfl_sync(FULL, item, 0);
        } else {
            if (tid == 0) item_sh[grp] = atomicAdd(counter, 1);
            group_sync<K>(bar);
            item = item_sh[grp];
        }
        if (item >= n_items) break;
        const int2 mw = items[item];
        const int* src = reinterpret_cast<const int*>(sys + mw.x);
        int* dst = reinterpret_cast<int*>(&Psh[grp]);
        for (int k = tid; k < (int)(sizeof(SweepParams) / sizeof(int)); k += 32 * K) dst[k] = src[k];
        group_sync<K>(bar);
        walker_sweep<K, false, DA, CL>(Psh[grp], mw.y, mine, tid, bar);
        group_sync<K>(bar);   // the slot and the item are rewritten for the next walker
    }
}

}  // namespace

size_t batch_static_smem(bool da) {
    return (sizeof(SweepParams) + sizeof(int)) * (da ? kBatchMaxWarpsDA : kBatchMaxWarps);
}

int batch_max_warps(bool da) { return da ? kBatchMaxWarpsDA : kBatchMaxWarps; }

namespace {

template <bool DA, bool CL, int K>
cudaError_t launch_batch_k(const SweepParams* sys, const int2* items, int n_items, int* counter,
                           int walkers_per_cta, int grid, int region, cudaStream_t s) {
    const size_t smem = (size_t)walkers_per_cta * region;
    batch_sweep_kernel<DA, CL, K><<<grid, 32 * K * walkers_per_cta, smem, s>>>(sys, items, n_items, counter, region);
    return cudaGetLastError();
}

template <bool DA, bool CL, int K>
cudaError_t prepare_k(int max_smem) {
    return cudaFuncSetAttribute(batch_sweep_kernel<DA, CL, K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                max_smem - (int)batch_static_smem(DA));
}

template <bool DA, bool CL, int K>
int occupancy_k(int walkers_per_cta, size_t smem) {
    int n = 0;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_sweep_kernel<DA, CL, K>, 32 * K * walkers_per_cta,
                                                         smem) == cudaSuccess
               ? n
               : 0;
}

}  // namespace

cudaError_t launch_batch_sweep(const SweepParams* sys, const int2* items, int n_items, int* counter,
                               int walkers_per_cta, int warps_per_walker, int grid, int region, bool da, bool cl,
                               cudaStream_t s) {
    if (n_items <= 0) return cudaSuccess;
    const int K = warps_per_walker;
    if (walkers_per_cta < 1 || K * walkers_per_cta > batch_max_warps(da) || grid < 1) return cudaErrorInvalidValue;
    if (K != 1 && (da || cl)) return cudaErrorInvalidValue;   // speculation: plain one-species walkers only
    if (da) {
        return cl ? launch_batch_k<true, true, 1>(sys, items, n_items, counter, walkers_per_cta, grid, region, s)
                  : launch_batch_k<true, false, 1>(sys, items, n_items, counter, walkers_per_cta, grid, region, s);
    }
    if (cl) return launch_batch_k<false, true, 1>(sys, items, n_items, counter, walkers_per_cta, grid, region, s);
    switch (K) {
        case 1: return launch_batch_k<false, false, 1>(sys, items, n_items, counter, walkers_per_cta, grid, region, s);
        case 2: return launch_batch_k<false, false, 2>(sys, items, n_items, counter, walkers_per_cta, grid, region, s);
        case 4: return launch_batch_k<false, false, 4>(sys, items, n_items, counter, walkers_per_cta, grid, region, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t batch_prepare(int max_smem) {
    cudaError_t e = prepare_k<false, false, 1>(max_smem);
    if (e == cudaSuccess) e = prepare_k<false, false, 2>(max_smem);
    if (e == cudaSuccess) e = prepare_k<false, false, 4>(max_smem);
    if (e == cudaSuccess) e = prepare_k<false, true, 1>(max_smem);
    if (e == cudaSuccess) e = prepare_k<true, false, 1>(max_smem);
    if (e == cudaSuccess) e = prepare_k<true, true, 1>(max_smem);
    return e;
}

int batch_occupancy(int walkers_per_cta, int warps_per_walker, int region, bool da, bool cl) {
    const size_t smem = (size_t)walkers_per_cta * region;   // within the limit batch_prepare set
    if (da) return cl ? occupancy_k<true, true, 1>(walkers_per_cta, smem) : occupancy_k<true, false, 1>(walkers_per_cta, smem);
    if (cl) return occupancy_k<false, true, 1>(walkers_per_cta, smem);
    switch (warps_per_walker) {
        case 1: return occupancy_k<false, false, 1>(walkers_per_cta, smem);
        case 2: return occupancy_k<false, false, 2>(walkers_per_cta, smem);
        case 4: return occupancy_k<false, false, 4>(walkers_per_cta, smem);
    }
    return 0;
}

size_t sweep_smem_per_walker(int nmax, int ncell, int cap, int warps_per_walker) {
    return smem_bytes(nmax, ncell, cap, warps_per_walker);
}

cudaError_t launch_sweep(const SweepParams& P, cudaStream_t s) {
    if (P.n_sweeps <= 0) return cudaSuccess;
    // delayed acceptance and the cluster species: one warp per walker
    if (P.n_cluster > 0 || P.gc2) return P.delayed ? launch_k<1, true, true>(P, s) : launch_k<1, false, true>(P, s);
    if (P.delayed) return launch_k<1, true, false>(P, s);
    switch (P.warps_per_walker) {
        case 1: return launch_k<1, false, false>(P, s);
        case 2: return launch_k<2, false, false>(P, s);
        case 4: return launch_k<4, false, false>(P, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_energy(const SweepParams& P, long long* out, int check_overlap, cudaStream_t s) {
    constexpr size_t kMaxSmem = 232448;   // 227 KB per block
    const size_t base = size_t(P.nmax) * sizeof(float4);
    const size_t with_cells = base + size_t((P.cg.ncell + 3) & ~3) * 4 + size_t(P.cg.ncell) * P.cg.cap * 2;
    // cells: 27 distinct stencil cells, cell coordinates packed in 10 bits each
    const int use_cells = P.cg.ncx >= 3 && P.cg.ncy >= 3 && (!P.g.periodic_z || P.cg.ncz >= 3) &&
                          P.cg.ncx < 1024 && P.cg.ncy < 1024 && P.cg.ncz < 1024 && with_cells + 1024 <= kMaxSmem;
    const size_t smem = use_cells ? with_cells : base;
    // the pair tables of a second species only where the walkers hold a cluster
    auto kernel = (P.n_cluster > 0 || P.gc2) ? energy_kernel<true> : energy_kernel<false>;
    cudaError_t e = cudaSuccess;
    if (smem > 48 * 1024) e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaMemsetAsync(out, 0, size_t(P.S) * sizeof(long long), s);
    if (e != cudaSuccess) return e;
    kernel<<<P.S * kEnergySplit, kEnergyThreads, smem, s>>>(P, reinterpret_cast<unsigned long long*>(out),
                                                            check_overlap, use_cells);
    return cudaGetLastError();
}

}  // namespace regc
