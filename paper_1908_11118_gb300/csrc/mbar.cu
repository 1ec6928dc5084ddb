// mbar.cu -- FP64 MBAR reweighting on the device (Sec. II.B), sm_103a.
//
// The self-consistent equations of Eq. normlizationconstant, pooled over the
// occupied (N, E) bins b with counts H_b, in log form:
//   D_b = ln sum_k Omega_k exp(f_k - u_k(b))        (one thread per bin)
//   f_s = -ln sum_b H_b exp(-u_s(b) - D_b)           (one block per state)
// with f_0 = 0 after each iteration, accelerated by Anderson mixing on the
// host (mbar_solve_dev).  Two forms of the map:
// * on a kernel matrix K_sb (every state sampled, the matrix within its
//   memory bound): each map is two FP64 matrix-vector products, the matrix
//   rebuilt when the iterate has moved far from the point it was built at;
// * log-sum-exp in FP64 over the terms within 50 of the largest (the others
//   weigh less than the FP64 rounding of the sum), found by a binary32
//   screening pass, so that with well separated states a bin costs a few FP64
//   terms rather than one per state (the allocation-free solve, and the final
//   D_b of either form).
// The query keeps an online maximum over all terms.
// Query states reuse the D_b: the weight of bin b at state q is
// H_b exp(-u_q(b) - D_b + f_q), giving <N> and p_N (Eq. textbook with the
// phase indicator chi_i = [N = i]).
#include <math.h>

#include <cmath>

#include <cooperative_groups.h>

#include <algorithm>
#include <vector>

#include "mbar.h"

namespace cg = cooperative_groups;

namespace regc {
namespace {

constexpr double kSkip = 50.0;

struct Lse {
    double m, s;
};

__device__ __forceinline__ void lse_add(Lse& L, double x) {
    if (x > L.m) {
        L.s = L.s * exp(L.m - x) + 1.0;
        L.m = x;
    } else if (x > L.m - kSkip) {
        L.s += exp(x - L.m);
    }
}

__device__ __forceinline__ Lse lse_merge(Lse a, Lse b) {
    if (b.m == -INFINITY) return a;
    if (a.m == -INFINITY) return b;
    const double m = fmax(a.m, b.m);
    return Lse{m, a.s * exp(a.m - m) + b.s * exp(b.m - m)};
}

__device__ __forceinline__ Lse warp_merge(Lse L) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Lse other{__shfl_xor_sync(0xffffffffu, L.m, o), __shfl_xor_sync(0xffffffffu, L.s, o)};
        L = lse_merge(L, other);
    }
    return L;
}

// Merge across a block (blockDim a multiple of 32, <= 1024); result valid in all threads.
__device__ Lse block_merge(Lse L) {
    __shared__ double sm[32], ss[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    L = warp_merge(L);
    __syncthreads();
    if (lane == 0) {
        sm[warp] = L.m;
        ss[warp] = L.s;
    }
    __syncthreads();
    Lse r{-INFINITY, 0.0};
    if (lane < nw) r = Lse{sm[lane], ss[lane]};
    r = warp_merge(r);
    return r;
}

__device__ double block_sum(double v) {
    __shared__ double sh[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double r = lane < nw ? sh[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    return r;
}

__device__ double block_max(double v) {
    __shared__ double sh[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double r = lane < nw ? sh[lane] : -INFINITY;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
    return r;
}

// Every sum is screened in binary32 first: the largest term of the sum
// computed from binary32 copies (absolute error far below kMargin for terms
// of magnitude up to 1e5), then only the terms within kSkip + kMargin of that
// maximum are evaluated in FP64, summed by an online log-sum-exp.  The FP64
// pipe of this GPU is narrow; with well separated states a bin or a state
// has only a few such terms.
constexpr float kMargin = 1.0f;
constexpr int kDTile = 512;

__global__ void en32_kernel(int B, const double* E_b, const int* N_b, float2* EN32, const int* N2_b, float* N2f) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) {
        EN32[b] = make_float2((float)E_b[b], (float)N_b[b]);
        if (N2_b) N2f[b] = (float)N2_b[b];
    }
}

// The reduced potential of state (a, c, c2) at bin (E, N, N2): a E + c N,
// plus c2 N2 with a second species (TWO); the same in binary32 for the
// screening.
template <bool TWO>
__device__ __forceinline__ double u_of(double a, double c, double c2, double E, double N, double N2) {
    return TWO ? fma(a, E, fma(c2, N2, c * N)) : fma(a, E, c * N);
}
template <bool TWO>
__device__ __forceinline__ float u32_of(float a, float c, float c2, float E, float N, float N2) {
    return TWO ? fmaf(a, E, fmaf(c2, N2, c * N)) : fmaf(a, E, c * N);
}

// D_b = ln sum_k exp(lnom_k + f_k - u_k(b))
template <bool TWO>
__global__ void __launch_bounds__(256) d_kernel(const __grid_constant__ MbarDev m, int always) {
    if (!always && m.state[0]) return;
    __shared__ double sa[kDTile], sc[kDTile], sg[kDTile], sc2[TWO ? kDTile : 1];
    __shared__ float fa[kDTile], fc[kDTile], fg[kDTile], fc2[TWO ? kDTile : 1];
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = b < m.B;
    const double E = act ? m.E_b[b] : 0.0;
    const double N = act ? (double)m.N_b[b] : 0.0;
    const double N2 = (TWO && act) ? (double)m.N2_b[b] : 0.0;
    const float2 en = act ? m.EN32[b] : make_float2(0.f, 0.f);
    const float n2f = (TWO && act) ? m.N2f[b] : 0.f;
    const bool one_tile = m.S <= kDTile;
    float mx32 = -INFINITY;
    Lse L{-INFINITY, 0.0};
    for (int pass = 0; pass < 2; ++pass) {
        for (int k0 = 0; k0 < m.S; k0 += kDTile) {
            const int nk = min(kDTile, m.S - k0);
            if (pass == 0 || !one_tile) {
                __syncthreads();
                for (int k = threadIdx.x; k < nk; k += blockDim.x) {
                    const double g = m.lnom[k0 + k] + m.f[k0 + k];
                    sa[k] = m.a[k0 + k];
                    sc[k] = m.c[k0 + k];
                    sg[k] = g;
                    fa[k] = (float)sa[k];
                    fc[k] = (float)sc[k];
                    fg[k] = (float)g;
                    if (TWO) {
                        sc2[k] = m.c2[k0 + k];
                        fc2[k] = (float)sc2[k];
                    }
                }
                __syncthreads();
            }
            if (!act) continue;
            if (pass == 0) {
                for (int k = 0; k < nk; ++k)
                    mx32 = fmaxf(mx32, fg[k] - u32_of<TWO>(fa[k], fc[k], fc2[TWO ? k : 0], en.x, en.y, n2f));
            } else {
                const float th = mx32 - (float)kSkip - kMargin;
                for (int k = 0; k < nk; ++k)
                    if (fg[k] - u32_of<TWO>(fa[k], fc[k], fc2[TWO ? k : 0], en.x, en.y, n2f) > th)
                        lse_add(L, sg[k] - u_of<TWO>(sa[k], sc[k], sc2[TWO ? k : 0], E, N, N2));
            }
        }
    }
    if (act) {
        const double D = L.m + log(L.s);
        m.D[b] = D;
        m.DH32[b] = (float)(D - m.lnH[b]);
    }
}

// f_new_s = -ln sum_b exp(lnH_b - a_s E_b - c_s N_b - D_b).  A cluster of
// kFSplit CTAs per state, each over a contiguous quarter of the bins (its own
// binary32 screening: a term more than kSkip below the largest of its
// quarter is also that far below the largest of all); the quarters' partial
// sums meet in CTA rank 0 through distributed shared memory and are merged
// in rank order (deterministic).
constexpr int kFThreads = 256;
constexpr int kFSplit = 4;
template <bool TWO>
__global__ void __cluster_dims__(kFSplit, 1, 1) __launch_bounds__(kFThreads)
    f_kernel(const __grid_constant__ MbarDev m) {
    __shared__ double part[2];
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int s = blockIdx.x / kFSplit;
    const bool live = !m.state[0];
    Lse L{-INFINITY, 0.0};
    if (live) {
        const int per = (m.B + kFSplit - 1) / kFSplit;
        const int b0 = rank * per, b1 = min(m.B, b0 + per);
        const double a = m.a[s], c = m.c[s], c2 = TWO ? m.c2[s] : 0.0;
        const float a32 = (float)a, c32 = (float)c, c232 = (float)c2;
        float mx32 = -INFINITY;
        for (int b = b0 + threadIdx.x; b < b1; b += kFThreads) {
            const float2 en = m.EN32[b];
            mx32 = fmaxf(mx32, -u32_of<TWO>(a32, c32, c232, en.x, en.y, TWO ? m.N2f[b] : 0.f) - m.DH32[b]);
        }
        mx32 = (float)block_max((double)mx32);
        const float th = mx32 - (float)kSkip - kMargin;
        for (int b = b0 + threadIdx.x; b < b1; b += kFThreads) {
            const float2 en = m.EN32[b];
            if (-u32_of<TWO>(a32, c32, c232, en.x, en.y, TWO ? m.N2f[b] : 0.f) - m.DH32[b] > th)
                lse_add(L, m.lnH[b] - u_of<TWO>(a, c, c2, m.E_b[b], (double)m.N_b[b],
                                                 TWO ? (double)m.N2_b[b] : 0.0) - m.D[b]);
        }
        L = block_merge(L);
    }
    if (threadIdx.x == 0) {
        part[0] = L.m;
        part[1] = L.s;
    }
    cluster.sync();
    if (live && rank == 0 && threadIdx.x == 0) {
        Lse T{-INFINITY, 0.0};
        for (int r = 0; r < kFSplit; ++r) {
            const double* pr = cluster.map_shared_rank(part, r);
            T = lse_merge(T, Lse{pr[0], pr[1]});
        }
        m.f_new[s] = -(T.m + log(T.s));
    }
    cluster.sync();   // the partial sums stay readable until rank 0 has merged them
}

__global__ void __launch_bounds__(256) query_kernel(const __grid_constant__ MbarDev m, const double* a_q,
                                                    const double* c_q, int nmax, double* n_mean,
                                                    double* pN, double* f_q) {
    extern __shared__ double hist[];   // [nmax + 1]
    const int q = blockIdx.x;
    const double a = a_q[q], c = c_q[q];
    for (int n = threadIdx.x; n <= nmax; n += blockDim.x) hist[n] = 0.0;
    Lse L{-INFINITY, 0.0};
    for (int b = threadIdx.x; b < m.B; b += blockDim.x)
        lse_add(L, m.lnH[b] - fma(a, m.E_b[b], c * (double)m.N_b[b]) - m.D[b]);
    L = block_merge(L);
    const double fq = -(L.m + log(L.s));
    double nsum = 0.0;
    __syncthreads();
    for (int b = threadIdx.x; b < m.B; b += blockDim.x) {
        const double x = m.lnH[b] - fma(a, m.E_b[b], c * (double)m.N_b[b]) - m.D[b] + fq;
        if (x > -745.0) {
            const double w = exp(x);
            const int n = m.N_b[b];
            nsum += w * (double)n;
            if (pN && n <= nmax) atomicAdd(&hist[n], w);
        }
    }
    nsum = block_sum(nsum);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (n_mean) n_mean[q] = nsum;
        if (f_q) f_q[q] = fq;
    }
    if (pN)
        for (int n = threadIdx.x; n <= nmax; n += blockDim.x) pN[size_t(q) * (nmax + 1) + n] = hist[n];
}

// ------------------------------------------------------------- compaction

constexpr int kChunk = 1024;  // elements per block, 256 threads x 4

__global__ void __launch_bounds__(256) count_kernel(const unsigned long long* h, long long n, int* counts) {
    const long long base = (long long)blockIdx.x * kChunk;
    int c = 0;
    for (int k = 0; k < 4; ++k) {
        const long long i = base + threadIdx.x * 4 + k;
        c += (i < n && h[i] != 0ull);
    }
    c = __reduce_add_sync(0xffffffffu, (unsigned)c);
    __shared__ int sh[8];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < 8; ++w) t += sh[w];
        counts[blockIdx.x] = t;
    }
}

// exclusive scan of counts[nblk] in place, total -> *total (one block)
__global__ void __launch_bounds__(1024) scan_kernel(int* counts, int nblk, int* total) {
    __shared__ int carry;
    __shared__ int wsum[32];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nblk; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const int v = i < nblk ? counts[i] : 0;
        int x = v;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += t;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int y = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, y, o);
                if (lane >= o) y += t;
            }
            wsum[lane] = y;
        }
        __syncthreads();
        const int incl = x + (warp > 0 ? wsum[warp - 1] : 0);
        if (i < nblk) counts[i] = carry + incl - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(256) write_kernel(const unsigned long long* h, long long n, int nbins,
                                                    double e_lo, double e_bin, const int* offsets,
                                                    int* N_b, double* E_b, double* lnH, int rows2, int* N2_b) {
    const long long base = (long long)blockIdx.x * kChunk;
    int c = 0;
    for (int k = 0; k < 4; ++k) {
        const long long i = base + threadIdx.x * 4 + k;
        c += (i < n && h[i] != 0ull);
    }
    // block exclusive scan of c
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
    }
    __shared__ int wsum[8];
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    int before = 0;
    for (int w = 0; w < warp; ++w) before += wsum[w];
    int out = offsets[blockIdx.x] + before + x - c;
    for (int k = 0; k < 4; ++k) {
        const long long i = base + threadIdx.x * 4 + k;
        if (i < n && h[i] != 0ull) {
            const long long nn = i / nbins, kb = i - nn * nbins;
            if (N2_b) {
                // two species: the row is N (rows2) + N2
                N_b[out] = (int)(nn / rows2);
                N2_b[out] = (int)(nn % rows2);
            } else {
                N_b[out] = (int)nn;
            }
            E_b[out] = __dadd_rn(e_lo, __dmul_rn((double)kb + 0.5, e_bin));   // as written: no contraction
            lnH[out] = log((double)h[i]);
            ++out;
        }
    }
}

// a = beta, c = 3 ln Lambda - beta mu, lnom = ln Omega (-inf when Omega = 0);
// Omega from omega_d (double) or omega_u (uint64), either may be null.
__global__ void prep_states_kernel(int S, const double* kT, const double* mu, double lambda0,
                                   const double* omega_d, const unsigned long long* omega_u, double* a,
                                   double* c, double* lnom) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const double b = 1.0 / kT[s];
    a[s] = b;
    c[s] = 3.0 * (log(lambda0) - 0.5 * log(kT[s])) - b * mu[s];
    if (lnom) {
        const double om = omega_d ? omega_d[s] : (omega_u ? (double)omega_u[s] : 0.0);
        lnom[s] = om > 0.0 ? log(om) : -INFINITY;
    }
}

// c2 = 3 ln Lambda_C - beta mu2 of a second species.
__global__ void prep_states2_kernel(int S, const double* kT, const double* mu2, double lambda0_2, double* c2) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    c2[s] = 3.0 * (log(lambda0_2) - 0.5 * log(kT[s])) - mu2[s] / kT[s];
}

// Two species: the query of query_kernel with u = a E + c N + c2 N2, and the
// distributions of both counts.
__global__ void __launch_bounds__(256) query2_kernel(const __grid_constant__ MbarDev m, const double* a_q,
                                                     const double* c_q, const double* c2_q, int nmax,
                                                     double* n_mean, double* n2_mean, double* pN, double* pN2,
                                                     double* f_q) {
    extern __shared__ double hist2[];   // [2][nmax + 1]
    const int q = blockIdx.x;
    const double a = a_q[q], c = c_q[q], c2 = c2_q[q];
    for (int n = threadIdx.x; n < 2 * (nmax + 1); n += blockDim.x) hist2[n] = 0.0;
    Lse L{-INFINITY, 0.0};
    for (int b = threadIdx.x; b < m.B; b += blockDim.x)
        lse_add(L, m.lnH[b] - u_of<true>(a, c, c2, m.E_b[b], (double)m.N_b[b], (double)m.N2_b[b]) - m.D[b]);
    L = block_merge(L);
    const double fq = -(L.m + log(L.s));
    double nsum = 0.0, n2sum = 0.0;
    __syncthreads();
    for (int b = threadIdx.x; b < m.B; b += blockDim.x) {
        const double x =
            m.lnH[b] - u_of<true>(a, c, c2, m.E_b[b], (double)m.N_b[b], (double)m.N2_b[b]) - m.D[b] + fq;
        if (x > -745.0) {
            const double w = exp(x);
            const int n = m.N_b[b], n2 = m.N2_b[b];
            nsum += w * (double)n;
            n2sum += w * (double)n2;
            if (n <= nmax) atomicAdd(&hist2[n], w);
            if (n2 <= nmax) atomicAdd(&hist2[nmax + 1 + n2], w);
        }
    }
    nsum = block_sum(nsum);
    __syncthreads();
    n2sum = block_sum(n2sum);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (n_mean) n_mean[q] = nsum;
        if (n2_mean) n2_mean[q] = n2sum;
        if (f_q) f_q[q] = fq;
    }
    for (int n = threadIdx.x; n <= nmax; n += blockDim.x) {
        if (pN) pN[size_t(q) * (nmax + 1) + n] = hist2[n];
        if (pN2) pN2[size_t(q) * (nmax + 1) + n] = hist2[nmax + 1 + n];
    }
}

__global__ void prep_bins_kernel(int B, const double* H, double* lnH) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) lnH[b] = log(H[b]);
}

// ---- iterations on the kernel matrix
// With every state sampled, the map can be iterated in linear space: for a
// reference point f_ref (the iterate at the last build),
//   K_sb = exp(t_sb - M_b),  t_sb = ln Omega_s + f_ref,s - u_s(b),  M_b = max_s t_sb,
// so that with w_s = exp(f_s - f_ref,s)
//   D_b = M_b + ln d_b,  d_b = sum_s K_sb w_s,
//   f_new,s = ln Omega_s + f_ref,s - ln sum_b (H_b / d_b) K_sb.
// Each map is then two FP64 matrix-vector products over a matrix built once
// per reference point (one exponential per entry), instead of S B
// exponentials.  The reference moves with the iterate: once some
// |f_s - f_ref,s| exceeds kRebuild the matrix is rebuilt, so w stays within
// e^(+-kRebuild) and d_b >= e^-kRebuild (the largest entry of a column is 1),
// far from the FP64 range limits (e^-708 .. e^709); a sum of positive terms
// keeps its relative accuracy whatever their spread.  Entries below e^-708
// (subnormal or zero) weigh less than e^(-708 + 2 kRebuild) = e^-108 against
// the sums they enter.  The build (one FP64 exponential per entry) costs
// about ten maps, so the bound is set wide.
constexpr double kRebuild = 300.0;
constexpr size_t kMatBytes = size_t(2) << 30;

struct MatDev {
    double* K;      // [S][B]
    double* M;      // [B]
    double* V;      // [B] H_b / d_b of the last map
    double* fref;   // [S]
    double* w;      // [S] exp(f_s - f_ref,s) of the current iterate (from the host)
};

// One thread per bin: t_sb over the states (tiled through shared memory),
// M_b, then the column of K.  Block 0 records f_ref = f.
template <bool TWO>
__global__ void __launch_bounds__(256) mat_build_kernel(const __grid_constant__ MbarDev m, MatDev k) {
    __shared__ double sa[kDTile], sc[kDTile], sg[kDTile], sc2[TWO ? kDTile : 1];
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = b < m.B;
    if (blockIdx.x == 0)
        for (int q = threadIdx.x; q < m.S; q += blockDim.x) k.fref[q] = m.f[q];
    const double E = act ? m.E_b[b] : 0.0;
    const double N = act ? (double)m.N_b[b] : 0.0;
    const double N2 = (TWO && act) ? (double)m.N2_b[b] : 0.0;
    double M = -INFINITY;
    for (int pass = 0; pass < 2; ++pass) {
        for (int k0 = 0; k0 < m.S; k0 += kDTile) {
            const int nk = min(kDTile, m.S - k0);
            __syncthreads();
            for (int q = threadIdx.x; q < nk; q += blockDim.x) {
                sa[q] = m.a[k0 + q];
                sc[q] = m.c[k0 + q];
                sg[q] = m.lnom[k0 + q] + m.f[k0 + q];
                if (TWO) sc2[q] = m.c2[k0 + q];
            }
            __syncthreads();
            if (!act) continue;
            if (pass == 0) {
                for (int q = 0; q < nk; ++q) M = fmax(M, sg[q] - u_of<TWO>(sa[q], sc[q], sc2[TWO ? q : 0], E, N, N2));
            } else {
                for (int q = 0; q < nk; ++q)
                    k.K[size_t(k0 + q) * m.B + b] = exp(sg[q] - u_of<TWO>(sa[q], sc[q], sc2[TWO ? q : 0], E, N, N2) - M);
            }
        }
    }
    if (act) k.M[b] = M;
}

// d_b = sum_s K_sb w_s, V_b = H_b / d_b.  A block takes 32 bins; its
// kDGroups warps take every kDGroups-th state (two independent FMA chains
// each), and the partial sums of a bin are added in a fixed order.  Rows of
// K are read 32 consecutive bins (256 bytes) at a time.
constexpr int kDGroups = 4;
__global__ void __launch_bounds__(32 * kDGroups) mat_d_kernel(const __grid_constant__ MbarDev m, MatDev k) {
    __shared__ double sw[kDTile];
    __shared__ double part[kDGroups][32];
    const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
    const int b = blockIdx.x * 32 + lane;
    const bool act = b < m.B;
    double d0 = 0.0, d1 = 0.0;
    for (int k0 = 0; k0 < m.S; k0 += kDTile) {
        const int nk = min(kDTile, m.S - k0);
        __syncthreads();
        for (int q = threadIdx.x; q < nk; q += blockDim.x) sw[q] = k.w[k0 + q];
        __syncthreads();
        if (!act) continue;
        const double* col = k.K + size_t(k0) * m.B + b;
        int q = grp;
        for (; q + kDGroups < nk; q += 2 * kDGroups) {
            d0 = fma(col[size_t(q) * m.B], sw[q], d0);
            d1 = fma(col[size_t(q + kDGroups) * m.B], sw[q + kDGroups], d1);
        }
        if (q < nk) d0 = fma(col[size_t(q) * m.B], sw[q], d0);
    }
    part[grp][lane] = d0 + d1;
    __syncthreads();
    if (grp == 0 && act) {
        const double d = (part[0][lane] + part[1][lane]) + (part[2][lane] + part[3][lane]);
        k.V[b] = exp(m.lnH[b]) / d;
    }
}

// f_new,s = ln Omega_s + f_ref,s - ln sum_b V_b K_sb: a cluster of kFSplit
// CTAs per state, each over a contiguous quarter of the row; the quarters'
// sums meet in CTA rank 0 through distributed shared memory, added in rank
// order (deterministic).
__global__ void __cluster_dims__(kFSplit, 1, 1) __launch_bounds__(kFThreads)
    mat_f_kernel(const __grid_constant__ MbarDev m, MatDev k) {
    __shared__ double part;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int s = blockIdx.x / kFSplit;
    const int per = (m.B + kFSplit - 1) / kFSplit;
    const int b0 = rank * per, b1 = min(m.B, b0 + per);
    const double* row = k.K + size_t(s) * m.B;
    double acc = 0.0;
    for (int b = b0 + threadIdx.x; b < b1; b += kFThreads) acc = fma(k.V[b], row[b], acc);
    acc = block_sum(acc);
    if (threadIdx.x == 0) part = acc;
    cluster.sync();
    if (rank == 0 && threadIdx.x == 0) {
        double t = 0.0;
        for (int r = 0; r < kFSplit; ++r) t += *cluster.map_shared_rank(&part, r);
        m.f_new[s] = m.lnom[s] + k.fref[s] - log(t);
    }
    cluster.sync();   // the partial sums stay readable until rank 0 has added them
}

}  // namespace

// The self-consistent map G(f) = gauge(f_new(D(f))) is iterated with
// Anderson acceleration (Walker & Ni, SIAM J. Numer. Anal. 49, 1715 (2011),
// "type II" with differences): with the residuals r_i = G(x_i) - x_i of the
// last kDepth iterates, gamma minimises |r_k - sum_j gamma_j (r_{j+1} - r_j)|
// and x_{k+1} = G(x_k) - sum_j gamma_j (G(x_{j+1}) - G(x_j)).  The fixed point
// is the one of the plain iteration (x = G(x)); only the path to it is
// shorter.  An iterate whose residual grows past 100 times the best one so far
// restarts the history from the best image.  Converged when max |r| < tol.
cudaError_t mbar_solve_dev(const MbarDev& m, double tol, int max_iter, int* iters_out, cudaStream_t s,
                           bool allow_matrix) {
    constexpr int kDepth = 16;
    const int S = m.S;
    cudaError_t err = cudaMemsetAsync(m.state, 0, 2 * sizeof(int), s);
    if (err != cudaSuccess) return err;
    err = cudaMemsetAsync(m.f, 0, size_t(S) * sizeof(double), s);
    if (err != cudaSuccess) return err;
    const int dgrid = (m.B + 255) / 256;
    const int dgrid128 = (m.B + 127) / 128;   // a bin per thread, small blocks to spread over every SM
    en32_kernel<<<dgrid, 256, 0, s>>>(m.B, m.E_b, m.N_b, m.EN32, m.N2_b, m.N2f);
    const bool two = m.N2_b != nullptr;
    // the kernel matrix, when every state is sampled and it fits
    MatDev mat{};
    void* mat_block = nullptr;
    const size_t mat_doubles = size_t(S) * m.B + 2 * size_t(m.B) + 2 * size_t(S);
    if (allow_matrix && mat_doubles * sizeof(double) <= kMatBytes) {
        std::vector<double> lnom_h(S);
        err = cudaMemcpyAsync(lnom_h.data(), m.lnom, size_t(S) * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (err == cudaSuccess) err = cudaStreamSynchronize(s);
        if (err != cudaSuccess) return err;
        bool all_sampled = true;
        for (int k = 0; k < S; ++k) all_sampled = all_sampled && std::isfinite(lnom_h[k]);
        if (all_sampled) {
            if (cudaMallocAsync(&mat_block, mat_doubles * sizeof(double), s) == cudaSuccess) {
                double* p = static_cast<double*>(mat_block);
                double* q = p + size_t(S) * m.B;
                mat = MatDev{p, q, q + m.B, q + 2 * size_t(m.B), q + 2 * size_t(m.B) + S};
            } else {
                mat_block = nullptr;
                (void)cudaGetLastError();   // out of memory is not sticky: iterate on log-sum-exps
            }
        }
    }
    struct FreeOnExit {
        void* p;
        cudaStream_t s;
        ~FreeOnExit() {
            if (p) cudaFreeAsync(p, s);
        }
    } free_mat{mat_block, s};
    std::vector<double> fref_h(S, 0.0), w_h(S);
    bool build = true;
    std::vector<double> x(S, 0.0), g(S), r(S), best_g(S, 0.0), rhs(kDepth), A(kDepth * kDepth), gam(kDepth);
    std::vector<std::vector<double>> dR, dG;       // differences of residuals and images, oldest first
    std::vector<double> r_prev, g_prev;
    double best = INFINITY;
    int it = 0;
    while (it < max_iter) {
        if (it > 0) {
            err = cudaMemcpyAsync(m.f, x.data(), size_t(S) * sizeof(double), cudaMemcpyHostToDevice, s);
            if (err != cudaSuccess) return err;
        }
        if (mat.K) {
            double drift = 0.0;
            for (int k = 0; k < S; ++k) drift = fmax(drift, fabs(x[k] - fref_h[k]));
            if (build || !(drift <= kRebuild)) {
                if (two) mat_build_kernel<true><<<dgrid, 256, 0, s>>>(m, mat);
                else mat_build_kernel<false><<<dgrid, 256, 0, s>>>(m, mat);
                fref_h = x;
                build = false;
            }
            for (int k = 0; k < S; ++k) w_h[k] = exp(x[k] - fref_h[k]);
            err = cudaMemcpyAsync(mat.w, w_h.data(), size_t(S) * sizeof(double), cudaMemcpyHostToDevice, s);
            if (err != cudaSuccess) return err;
            mat_d_kernel<<<(m.B + 31) / 32, 32 * kDGroups, 0, s>>>(m, mat);
            mat_f_kernel<<<S * kFSplit, kFThreads, 0, s>>>(m, mat);
        } else {
            if (two) {
                d_kernel<true><<<dgrid128, 128, 0, s>>>(m, 1);
                f_kernel<true><<<S * kFSplit, kFThreads, 0, s>>>(m);
            } else {
                d_kernel<false><<<dgrid128, 128, 0, s>>>(m, 1);
                f_kernel<false><<<S * kFSplit, kFThreads, 0, s>>>(m);
            }
        }
        err = cudaGetLastError();
        if (err != cudaSuccess) return err;
        err = cudaMemcpyAsync(g.data(), m.f_new, size_t(S) * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (err == cudaSuccess) err = cudaStreamSynchronize(s);
        if (err != cudaSuccess) return err;
        ++it;
        const double g0 = g[0];
        double delta = 0.0;
        for (int k = 0; k < S; ++k) {
            g[k] -= g0;
            r[k] = g[k] - x[k];
            delta = fmax(delta, fabs(r[k]));
        }
        if (!(delta == delta)) return cudaErrorInvalidValue;   // NaN: no fixed point to approach
        if (delta < tol) {
            x = g;
            break;
        }
        if (delta < best) {
            best = delta;
            best_g = g;
        } else if (delta > 100.0 * best) {
            dR.clear();
            dG.clear();
            r_prev.clear();
            x = best_g;
            continue;
        }
        if (!r_prev.empty()) {
            std::vector<double> a(S), b(S);
            for (int k = 0; k < S; ++k) {
                a[k] = r[k] - r_prev[k];
                b[k] = g[k] - g_prev[k];
            }
            dR.push_back(a);
            dG.push_back(b);
            if ((int)dR.size() > kDepth) {
                dR.erase(dR.begin());
                dG.erase(dG.begin());
            }
        }
        r_prev = r;
        g_prev = g;
        const int mh = (int)dR.size();
        x = g;
        if (mh > 0) {
            // normal equations (dR^T dR + eps I) gamma = dR^T r, by Gaussian elimination
            for (int i = 0; i < mh; ++i) {
                rhs[i] = 0.0;
                for (int k = 0; k < S; ++k) rhs[i] += dR[i][k] * r[k];
                for (int j = 0; j < mh; ++j) {
                    double v = 0.0;
                    for (int k = 0; k < S; ++k) v += dR[i][k] * dR[j][k];
                    A[i * kDepth + j] = v;
                }
            }
            double diag = 0.0;
            for (int i = 0; i < mh; ++i) diag = fmax(diag, A[i * kDepth + i]);
            for (int i = 0; i < mh; ++i) A[i * kDepth + i] += 1e-12 * diag + 1e-300;
            bool ok = true;
            for (int c = 0; c < mh && ok; ++c) {
                int piv = c;
                for (int i = c + 1; i < mh; ++i)
                    if (fabs(A[i * kDepth + c]) > fabs(A[piv * kDepth + c])) piv = i;
                if (!(fabs(A[piv * kDepth + c]) > 0.0)) {
                    ok = false;
                    break;
                }
                if (piv != c) {
                    for (int j = 0; j < mh; ++j) std::swap(A[c * kDepth + j], A[piv * kDepth + j]);
                    std::swap(rhs[c], rhs[piv]);
                }
                for (int i = c + 1; i < mh; ++i) {
                    const double f = A[i * kDepth + c] / A[c * kDepth + c];
                    for (int j = c; j < mh; ++j) A[i * kDepth + j] -= f * A[c * kDepth + j];
                    rhs[i] -= f * rhs[c];
                }
            }
            if (ok) {
                for (int i = mh - 1; i >= 0; --i) {
                    double v = rhs[i];
                    for (int j = i + 1; j < mh; ++j) v -= A[i * kDepth + j] * gam[j];
                    gam[i] = v / A[i * kDepth + i];
                }
                for (int j = 0; j < mh; ++j)
                    for (int k = 0; k < S; ++k) x[k] -= gam[j] * dG[j][k];
            }
        }
    }
    err = cudaMemcpyAsync(m.f, x.data(), size_t(S) * sizeof(double), cudaMemcpyHostToDevice, s);
    if (err != cudaSuccess) return err;
    if (two) d_kernel<true><<<dgrid128, 128, 0, s>>>(m, 1);  // D_b of the final f
    else d_kernel<false><<<dgrid128, 128, 0, s>>>(m, 1);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    // the host vectors go out of scope: wait for the copy that reads x
    err = cudaStreamSynchronize(s);
    if (err != cudaSuccess) return err;
    if (iters_out) *iters_out = it;
    return cudaSuccess;
}

cudaError_t mbar_query_dev(const MbarDev& m, int Q, const double* a_q, const double* c_q, int nmax,
                           double* n_mean, double* pN, double* f_q, cudaStream_t s) {
    if (Q <= 0) return cudaSuccess;
    const size_t smem = size_t(nmax + 1) * sizeof(double);
    cudaError_t err = cudaFuncSetAttribute(query_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    query_kernel<<<Q, 256, smem, s>>>(m, a_q, c_q, nmax, n_mean, pN, f_q);
    return cudaGetLastError();
}

size_t compact_scratch_ints(long long n) { return size_t((n + kChunk - 1) / kChunk) + 1; }

cudaError_t compact_count_dev(const unsigned long long* hist, long long n, int* scratch, int* count_out,
                              cudaStream_t s) {
    const int nblk = (int)((n + kChunk - 1) / kChunk);
    if (nblk == 0) return cudaMemsetAsync(count_out, 0, sizeof(int), s);
    count_kernel<<<nblk, 256, 0, s>>>(hist, n, scratch);
    scan_kernel<<<1, 1024, 0, s>>>(scratch, nblk, count_out);
    return cudaGetLastError();
}

cudaError_t compact_write_dev(const unsigned long long* hist, long long n, int nbins, double e_lo, double e_bin,
                              const int* scratch, int* N_b, double* E_b, double* lnH, cudaStream_t s) {
    const int nblk = (int)((n + kChunk - 1) / kChunk);
    if (nblk == 0) return cudaSuccess;
    write_kernel<<<nblk, 256, 0, s>>>(hist, n, nbins, e_lo, e_bin, scratch, N_b, E_b, lnH, 1, nullptr);
    return cudaGetLastError();
}

cudaError_t compact_write2_dev(const unsigned long long* hist, long long n, int nbins, int rows2, double e_lo,
                               double e_bin, const int* scratch, int* N_b, int* N2_b, double* E_b, double* lnH,
                               cudaStream_t s) {
    const int nblk = (int)((n + kChunk - 1) / kChunk);
    if (nblk == 0) return cudaSuccess;
    write_kernel<<<nblk, 256, 0, s>>>(hist, n, nbins, e_lo, e_bin, scratch, N_b, E_b, lnH, rows2, N2_b);
    return cudaGetLastError();
}

cudaError_t mbar_prep_states2(int S, const double* kT, const double* mu2, double lambda0_2, double* c2,
                              cudaStream_t s) {
    if (S <= 0) return cudaSuccess;
    prep_states2_kernel<<<(S + 255) / 256, 256, 0, s>>>(S, kT, mu2, lambda0_2, c2);
    return cudaGetLastError();
}

cudaError_t mbar_query2_dev(const MbarDev& m, int Q, const double* a_q, const double* c_q, const double* c2_q,
                            int nmax, double* n_mean, double* n2_mean, double* pN, double* pN2, double* f_q,
                            cudaStream_t s) {
    if (Q <= 0) return cudaSuccess;
    const size_t smem = 2 * size_t(nmax + 1) * sizeof(double);
    cudaError_t err = cudaFuncSetAttribute(query2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    query2_kernel<<<Q, 256, smem, s>>>(m, a_q, c_q, c2_q, nmax, n_mean, n2_mean, pN, pN2, f_q);
    return cudaGetLastError();
}

cudaError_t mbar_prep_states(int S, const double* kT, const double* mu, double lambda0, const double* omega_d,
                             const unsigned long long* omega_u, double* a, double* c, double* lnom, cudaStream_t s) {
    if (S <= 0) return cudaSuccess;
    prep_states_kernel<<<(S + 255) / 256, 256, 0, s>>>(S, kT, mu, lambda0, omega_d, omega_u, a, c, lnom);
    return cudaGetLastError();
}

cudaError_t mbar_prep_bins(int B, const double* H, double* lnH, cudaStream_t s) {
    if (B <= 0) return cudaSuccess;
    prep_bins_kernel<<<(B + 255) / 256, 256, 0, s>>>(B, H, lnH);
    return cudaGetLastError();
}

}  // namespace regc
