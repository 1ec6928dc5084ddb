// regc_internal.cuh -- device-side building blocks of the REGC library (sm_103a).
//
// Shared by the kernels of this library only.  Nothing here is visible through
// the C ABI.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/regc.h"

namespace regc {

// Error bits of the per-handle device error word.
enum : int {
    ERR_CAPACITY = 1,   // a cell of a walker's cell list was full
    ERR_OVERLAP = 2,    // two particles closer than the hard-core guard radius
    ERR_TIMEOUT = 4,    // a bounded wait on an mbarrier gave up
    ERR_NUMERIC = 8,    // a non-finite energy
    ERR_INPUT = 16,     // a caller-supplied coordinate outside the region
};

// Energies are accumulated as 64-bit fixed-point integers in units of 2^-30
// eps.  Every pair term is a binary32 value phi rounded once to that grid, so a
// sum does not depend on the order in which pairs are visited and a running
// total built from move energies equals the from-scratch sum exactly.
constexpr double kFixUnit = 1.0 / 1073741824.0;     // 2^-30
constexpr double kFixPerUnit = 1073741824.0;        // 2^30

// ------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of two
// 32x32->64-bit products (multipliers 0xD2511F53, 0xCD9E8D57) with the key
// bumped by the Weyl constants 0x9E3779B9, 0xBB67AE85 between rounds.
struct U4 {
    uint32_t x, y, z, w;
};

__host__ __device__ __forceinline__ U4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                              uint32_t k0, uint32_t k1) {
#ifdef __CUDA_ARCH__
#pragma unroll
#endif
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
#ifdef __CUDA_ARCH__
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
#else
        const uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
        const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
#endif
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return U4{c0, c1, c2, c3};
}

// 24-bit uniform in [0, 1), exact in binary32.
__device__ __forceinline__ float u24(uint32_t a) { return (float)(a >> 8) * (1.0f / 16777216.0f); }

// ------------------------------------------------------------ parameters

struct PairTab {
    float eps4;   // 4 eps_ij
    float sig2;   // sigma_ij^2
    float rhc2;   // hard-core guard radius^2 (0 when eps_ij = 0)
    float eps;    // eps_ij (the surrogate's neighbour weight)
};

// The surrogate network's BF16 inference copy (unit-major weights, FP32
// biases); see surrogate.cuh.
struct SurrogateDev {
    const __nv_bfloat16* w1;   // [64][16]: unit u's 16 input weights
    const float* b1;           // [64]
    const __nv_bfloat16* w2;   // [64][64]: unit v's 64 input weights
    const float* b2;           // [64]
    const __nv_bfloat16* w3;   // [64]
    const float* b3;           // [1]
};

struct Geometry {
    float Lx, Ly, Lz;      // periods
    float hLx, hLy, hLz;   // half periods
    int periodic_z;
    float z_lo, z_hi;
    float height;          // binary32(z_hi - z_lo)
    float rc2;
    float rc;
    float shear;           // the cell's second lattice vector is (shear Ly, Ly): x = u + shear v
};

struct CellGrid {
    int ncx, ncy, ncz, ncell, cap;
    float icx, icy, icz;   // cells per unit length
};

struct SurfaceTab {
    int nsx, nsy;          // surface column grid
    float isx, isy;        // columns per unit length
    float z_reach;         // surface atoms are out of reach at z >= z_reach
    int stride;            // slots per column, a multiple of 32
    const float4* atoms;   // [nsx*nsy][stride] images listed per column: x, y, z
                           // of the image (shifted by -L where exact), w = bits:
                           // type (0-1), query shifted by -Lx (2), -Ly (3),
                           // -Lz (4), padding slot (5; z = 1e30, out of reach)
    const float4* all;     // every surface atom, w = type (energy recompute)
    int n_all;
};

struct SweepParams {
    Geometry g;
    CellGrid cg;
    SurfaceTab st;
    PairTab gg;            // mobile-mobile (grand-canonical species)
    PairTab gs[4];         // mobile-surface by surface type
    int n_cluster;         // particles 0..n_cluster-1 are the cluster species (0: none)
    PairTab gA, gAB;       // cluster-cluster, cluster-grand-canonical
    PairTab gsA[4];        // cluster-surface by surface type
    // A second grand-canonical species (gc2 = 1): walker w's particles
    // [0, nb[w]) are species B and [nb[w], N) species C; the two-species
    // tables above then hold B-B (gA), B-C (gAB), C-C (gg), B-surface (gsA)
    // and C-surface (gs), so the cluster's code paths serve with the split
    // taken per walker.  A grand-canonical move picks its species by bit 30
    // of Philox word B2 (0: B, 1: C).
    int gc2;
    // failure-detection test hook: the walkers issue no bulk copy of their
    // positions, so their bounded waits on it expire (ERR_TIMEOUT)
    int expire_waits;
    int* nb;               // [S] species-B count of each walker
    const double* c_ins2;  // [S] ln V - 3 ln Lambda_C,s + beta_s mu2_s
    const double* c_del2;  // [S] 3 ln Lambda_C,s - ln V - beta_s mu2_s
    const float* c_ins2_f;
    const float* c_del2_f;
    unsigned long long* hN2;      // [S][nmax+1] observations of N_C
    double* moments2;             // [S][2] sum N_C, sum N_C^2
    float max_disp;
    unsigned long long th_disp;   // displacement if A0 < th_disp (0 .. 2^32)
    int S, nmax, mps;
    int w_begin, w_end;    // the walkers a sweep steps: [w_begin, w_end) (a shard; 0, S by default)
    uint32_t key0, key1;
    const double* beta;    // [S] per state
    const double* c_ins;   // [S] ln V - 3 ln Lambda_s + beta_s mu_s
    const double* c_del;   // [S] 3 ln Lambda_s - ln V - beta_s mu_s
    const double* ln_tab;  // [nmax + 2] ln k
    const float* beta_f;   // binary32 copies for the pre-test of the acceptance rule
    const float* c_ins_f;
    const float* c_del_f;
    const float* ln_tab_f;
    float4* pos;           // [S][nmax]
    int* n;                // [S]
    long long* efix;       // [S]
    const int* state_of_walker;
    unsigned long long* hN;       // [S][nmax+1]
    unsigned long long* omega;    // [S]
    double* moments;              // [S][4]
    unsigned long long* hNE;      // [nmax+1][n_e_bins]
    unsigned long long* e_out;    // [S]
    double e_lo, e_bin;
    long long e_lo_fix, e_bin_fix;  // E-histogram origin and bin width in units of 2^-30
    int n_e_bins;
    unsigned long long* hE;       // [S][hE_bins + 2] per-state energy histograms, or null: bin 0
                                  //     below the state's window, k + 1 window bin k, hE_bins + 1 beyond
    const long long* hE_lo_fix;   // [S] window origins in units of 2^-30
    long long hE_bin_fix;         // window bin width in units of 2^-30
    int hE_bins;
    long long* move_counts;       // [S][6]
    unsigned long long* pair_counts;  // [6] pairs in rc, candidates, rounds, evaluations,
                                      //     surrogate-screened moves, stage-1 passes
    int* error;
    regc_move_record* trace;      // device [S][trace_steps][mps] or null, at this launch's first sweep
    int trace_steps;              // sweeps (steps) per walker in the trace buffer
    uint32_t t0;
    int n_sweeps;
    int cycle;                    // 1: REGC cycle steps -- move 0 of a step is a particle exchange
                                  //    (insertion or removal), moves 1 .. mps-1 are displacements
    int m_first;                  // first move of the launch (1: its first step began with a
                                  //    replica exchange, so its particle exchange is not attempted)
    int smem_per_walker;          // bytes
    int warps_per_walker;         // 1, 2 or 4
    int delayed;                  // 1: two-stage delayed acceptance with the surrogate
    SurrogateDev net;             // the surrogate (delayed acceptance)
};

struct ExchangeParams {
    int L, M;
    uint32_t key0, key1;
    const double* beta;    // [S]
    const double* bmu;     // [S] beta_s mu_s
    const double* lnbeta;  // [S]
    const int* n;
    const long long* efix;
    int* state_of_walker;
    int* walker_of_state;
    long long* ex_counts;  // [S][2 x directions]
    int K;                 // a third grid axis (mu2 of a second species; 1: none)
    const int* nb;         // [S] walkers' species-B counts, or null (one species)
    const double* bmu2;    // [S] beta_s mu2_s (with nb)
};

// ----------------------------------------------------------- pair energy
// A pair energy phi (|phi| < 2^35) split exactly into integer counts of
// 2^13, 2^-8 and 2^-30 eps: phi = big 2^13 + hi 2^-8 + lo 2^-30 after one
// round-to-nearest-even onto the 2^-30 grid.  Adding 1.5 2^(23+u) to a float
// below 2^(22+u) in magnitude rounds it to a multiple of 2^u and leaves that
// multiple in the low bits of the sum, so each level costs two FADDs and an
// IADD, on the FP32 and integer pipes.  The parts are accumulated in int32.
struct Fix3 {
    int big, hi, lo;
};

constexpr float kM2 = 103079215104.0f;   // 1.5 * 2^36: unit 2^13
constexpr float kM1 = 49152.0f;          // 1.5 * 2^15: unit 2^-8
constexpr float kM0 = 0.01171875f;       // 1.5 * 2^-7: unit 2^-30

__device__ __forceinline__ void fix_add(Fix3& a, float phi, int sign) {
    const float t2 = __fadd_rn(phi, kM2);
    const float r1 = __fsub_rn(phi, __fsub_rn(t2, kM2));
    const float t1 = __fadd_rn(r1, kM1);
    const float r0 = __fsub_rn(r1, __fsub_rn(t1, kM1));
    const float t0 = __fadd_rn(r0, kM0);
    a.big += sign * (__float_as_int(t2) - __float_as_int(kM2));
    a.hi += sign * (__float_as_int(t1) - __float_as_int(kM1));
    a.lo += sign * (__float_as_int(t0) - __float_as_int(kM0));
}

// The 64-bit fixed-point value (units of 2^-30) of a Fix3 sum.
__device__ __forceinline__ long long fix_value(int big, int hi, int lo) {
    return ((long long)big << 43) + ((long long)hi << 22) + (long long)lo;
}

// Binary32 pair energy phi(r) from r^2 (r < rc).  Explicit round-to-nearest
// intrinsics keep the value identical wherever it is inlined.
__device__ __forceinline__ float phi_of_r2(float r2, const PairTab& t) {
    const float s2 = __fdividef(t.sig2, r2);
    const float s6 = __fmul_rn(__fmul_rn(s2, s2), s2);
    return __fmul_rn(t.eps4, __fmaf_rn(s6, s6, -s6));
}

// Cartesian x component of a displacement (du, dv) in the cell frame.
__device__ __forceinline__ float cart_dx(const Geometry& g, float du, float dv) {
    return __fadd_rn(du, __fmul_rn(g.shear, dv));
}

__device__ __forceinline__ float r2_of(float dx, float dy, float dz) {
    return __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmul_rn(dz, dz)));
}

// Binary32 pair energy of one pair from its displacement, 0 beyond rc.  It
// depends on (dx, dy, dz) only through r^2, so it is the same for both orders
// of the pair.
__device__ __forceinline__ float pair_phi(float dx, float dy, float dz, float rc2, const PairTab& t,
                                          int& n_in, int& overlap) {
    const float r2 = r2_of(dx, dy, dz);
    float phi = 0.0f;
    if (r2 < rc2) {
        phi = phi_of_r2(r2, t);
        n_in += 1;
        overlap |= (r2 < t.rhc2);
    }
    return phi;
}

// Minimum-image displacement q - p along a periodic axis of period L, rounded
// once: when the nearest image lies across the boundary, the shifted operand
// (q - L when q > L/2, p - L when p > L/2) is exact (Sterbenz), so only the
// final subtraction rounds.
__device__ __forceinline__ float min_image_exact(float q, float p, float L, float hL) {
    const float e = __fsub_rn(q, p);
    if (e > hL) return __fsub_rn(__fsub_rn(q, L), p);
    if (e < -hL) return __fsub_rn(q, __fsub_rn(p, L));
    return e;
}

__device__ __forceinline__ const PairTab& surf_tab(const SweepParams& P, int type) {
    return P.gs[type & 3];
}

// Warp-wide sum of a 64-bit integer.
__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int warp_sum_i(int v) {
    return __reduce_add_sync(0xffffffffu, (unsigned)v);
}

}  // namespace regc
