// mbar.cu -- FP64 MBAR reweighting on the device (Sec. II.B), sm_103a.
//
// The self-consistent equations of Eq. normlizationconstant, pooled over the
// occupied (N, E) bins b with counts H_b, in log form:
//   D_b = ln sum_k Omega_k exp(f_k - u_k(b))        (one thread per bin)
//   f_s = -ln sum_b H_b exp(-u_s(b) - D_b)           (one block per state)
// with f_0 = 0 after each iteration, accelerated by Anderson mixing on the
// host (mbar_solve_dev).  Two forms of the map:
// * on the kept entries of a kernel matrix K_sb (every state sampled, the
//   entries within their memory bound): each map is two FP64 sparse
//   matrix-vector products, the matrix rebuilt when the iterate has moved
//   far from the point it was built at;
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

// Reweighting to query state q = (a, c, c2): bin b weighs
// H_b exp(-u_q(b) - D_b + f_q), f_q = -ln sum_b H_b exp(-u_q(b) - D_b), giving
// <N>, p_N (Eq. textbook with the phase indicator chi_i = [N = i]) and, with
// a second species (TWO), <N2> and p_N2.  Screened as the maps are, but per
// phase: a binary32 pass finds the largest term of every N (and every N2),
// and only the terms within kSkip + kMargin of the largest of their N (or of
// their N2) are taken in FP64.  Each dropped term weighs below e^-50 of the
// largest term of its own phase, so every p_N keeps its relative accuracy,
// however small it is (the per-phase averages of the structure divide by
// it).
constexpr int kQThreads = 256;

// atomic maximum of a binary32 value in shared memory (any sign, -inf start)
__device__ __forceinline__ void atomic_max_f32(float* addr, float v) {
    if (v >= 0.f) atomicMax(reinterpret_cast<int*>(addr), __float_as_int(v));
    else atomicMin(reinterpret_cast<unsigned int*>(addr), __float_as_uint(v));
}

template <bool TWO>
__global__ void __launch_bounds__(kQThreads)
    query_kernel(const __grid_constant__ MbarDev m, const double* a_q, const double* c_q, const double* c2_q,
                 int nmax, double* n_mean, double* n2_mean, double* pN, double* pN2, double* f_q) {
    // [nmax + 1] doubles of p_N (then of p_N2), [nmax + 1] floats of the
    // largest screen value per N (then per N2)
    extern __shared__ double hist[];
    const int rows = nmax + 1, nh = (TWO ? 2 : 1) * rows;
    float* rmax = reinterpret_cast<float*>(hist + nh);
    const int q = blockIdx.x;
    const double a = a_q[q], c = c_q[q], c2 = TWO ? c2_q[q] : 0.0;
    const float a32 = (float)a, c32 = (float)c, c232 = (float)c2;
    for (int n = threadIdx.x; n < nh; n += blockDim.x) {
        hist[n] = 0.0;
        rmax[n] = -INFINITY;
    }
    __syncthreads();
    auto screen = [&](int b) {
        const float2 en = m.EN32[b];
        return -u32_of<TWO>(a32, c32, c232, en.x, en.y, TWO ? m.N2f[b] : 0.f) - m.DH32[b];
    };
    auto term = [&](int b) {
        return m.lnH[b] - u_of<TWO>(a, c, c2, m.E_b[b], (double)m.N_b[b], TWO ? (double)m.N2_b[b] : 0.0) - m.D[b];
    };
    // a count beyond nmax (a caller's bins) shares the last row's threshold slot
    auto row = [&](int n) { return min(max(n, 0), nmax); };
    for (int b = threadIdx.x; b < m.B; b += blockDim.x) {
        const float x = screen(b);
        atomic_max_f32(&rmax[row(m.N_b[b])], x);
        if (TWO) atomic_max_f32(&rmax[rows + row(m.N2_b[b])], x);
    }
    __syncthreads();
    constexpr float kCut = (float)kSkip + kMargin;
    auto keep = [&](int b) {
        const float x = screen(b);
        return x > rmax[row(m.N_b[b])] - kCut || (TWO && x > rmax[rows + row(m.N2_b[b])] - kCut);
    };
    Lse L{-INFINITY, 0.0};
    for (int b = threadIdx.x; b < m.B; b += blockDim.x)
        if (keep(b)) lse_add(L, term(b));
    L = block_merge(L);
    const double fq = -(L.m + log(L.s));
    double nsum = 0.0, n2sum = 0.0;
    __syncthreads();
    for (int b = threadIdx.x; b < m.B; b += blockDim.x) {
        if (!keep(b)) continue;
        const double w = exp(term(b) + fq);
        const int n = m.N_b[b];
        nsum = fma(w, (double)n, nsum);
        if (pN && n <= nmax) atomicAdd(&hist[n], w);
        if (TWO) {
            const int n2 = m.N2_b[b];
            n2sum = fma(w, (double)n2, n2sum);
            if (pN2 && n2 <= nmax) atomicAdd(&hist[rows + n2], w);
        }
    }
    nsum = block_sum(nsum);
    __syncthreads();
    if (TWO) n2sum = block_sum(n2sum);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (n_mean) n_mean[q] = nsum;
        if (TWO && n2_mean) n2_mean[q] = n2sum;
        if (f_q) f_q[q] = fq;
    }
    for (int n = threadIdx.x; n <= nmax; n += blockDim.x) {
        if (pN) pN[size_t(q) * rows + n] = hist[n];
        if (TWO && pN2) pN2[size_t(q) * rows + n] = hist[rows + n];
    }
}

// The query over runs of bins with equal (N, N2) in the bin order (the
// handle's compacted histogram is row-major, so a run is a whole row).  A
// binary32 pass over all bins finds the query's largest screen value M_q;
// then a warp takes whole runs: the run's largest screen value, and the sum
// of exp(t_b - M_q) in FP64 over the run's terms within kSkip + kMargin of
// that largest one (one exponential per kept term), added to the warp's own
// sums per N (and per N2), N- and N2-weighted and in total.  The warps' sums
// are added in warp order at the end, so the query is deterministic:
//   f_q = -(M_q + ln total),  p_N = sum_N / total,  <N> = sum_{N-weighted} / total.
// Each dropped term weighs below e^-50 of the largest term of its own run,
// so every run sum -- hence every p_N -- keeps its relative accuracy down to
// the FP64 range (a phase below e^-708 of the largest term is 0, as the
// oracle's weights are).
constexpr int kRunWarps = 8;

template <bool TWO>
__global__ void __launch_bounds__(32 * kRunWarps)
    query_runs_kernel(const __grid_constant__ MbarDev m, const double* a_q, const double* c_q, const double* c2_q,
                      int nmax, const int* run_start, int n_runs, int warps, double* n_mean, double* n2_mean,
                      double* pN, double* pN2, double* f_q) {
    // per warp: [nmax + 1] sums per N (then per N2), then total, N-, N2-weighted
    extern __shared__ double acc[];
    const int rows = nmax + 1, per_warp = (TWO ? 2 : 1) * rows + 3;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double* mine = acc + (size_t)warp * per_warp;   // used only by the first `warps` warps
    if (warp < warps)
        for (int i = lane; i < per_warp; i += 32) mine[i] = 0.0;
    const int q = blockIdx.x;
    const double a = a_q[q], c = c_q[q], c2 = TWO ? c2_q[q] : 0.0;
    const float a32 = (float)a, c32 = (float)c, c232 = (float)c2;
    auto screen = [&](int b, float n32, float n232) {
        return -u32_of<TWO>(a32, c32, c232, m.EN32[b].x, n32, n232) - m.DH32[b];
    };
    float mall = -INFINITY;
    for (int b = threadIdx.x; b < m.B; b += blockDim.x)
        mall = fmaxf(mall, screen(b, m.EN32[b].y, TWO ? m.N2f[b] : 0.f));
    const double Mq = block_max((double)mall);
    __syncthreads();
    double* tot = mine + (TWO ? 2 : 1) * rows;
    if (warp < warps) {
        for (int r = warp; r < n_runs; r += warps) {
            const int b0 = run_start[r], b1 = run_start[r + 1];
            const float n32 = m.EN32[b0].y, n232 = TWO ? m.N2f[b0] : 0.f;
            float mx = -INFINITY;
            for (int b = b0 + lane; b < b1; b += 32) mx = fmaxf(mx, screen(b, n32, n232));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            const float th = mx - (float)kSkip - kMargin;
            const double nd = (double)m.N_b[b0], n2d = TWO ? (double)m.N2_b[b0] : 0.0;
            double sum = 0.0;
            for (int b = b0 + lane; b < b1; b += 32)
                if (screen(b, n32, n232) > th)
                    sum += exp(m.lnH[b] - u_of<TWO>(a, c, c2, m.E_b[b], nd, n2d) - m.D[b] - Mq);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
            if (lane == 0 && sum > 0.0) {
                const int n = m.N_b[b0];
                if (n >= 0 && n <= nmax) mine[n] += sum;
                tot[0] += sum;
                tot[1] = fma(nd, sum, tot[1]);
                if (TWO) {
                    const int n2 = m.N2_b[b0];
                    if (n2 >= 0 && n2 <= nmax) mine[rows + n2] += sum;
                    tot[2] = fma(n2d, sum, tot[2]);
                }
            }
        }
    }
    __syncthreads();
    // add the warps' sums in warp order into warp 0's
    for (int i = threadIdx.x; i < per_warp; i += blockDim.x) {
        double x = acc[i];
        for (int w = 1; w < warps; ++w) x += acc[(size_t)w * per_warp + i];
        acc[i] = x;
    }
    __syncthreads();
    const double total = acc[(TWO ? 2 : 1) * rows];
    if (threadIdx.x == 0) {
        if (n_mean) n_mean[q] = acc[(TWO ? 2 : 1) * rows + 1] / total;
        if (TWO && n2_mean) n2_mean[q] = acc[(TWO ? 2 : 1) * rows + 2] / total;
        if (f_q) f_q[q] = -(Mq + log(total));
    }
    for (int n = threadIdx.x; n < rows; n += blockDim.x) {
        if (pN) pN[size_t(q) * rows + n] = acc[n] / total;
        if (TWO && pN2) pN2[size_t(q) * rows + n] = acc[rows + n] / total;
    }
}

// Runs of equal (N, N2): cnt[b + 1] = 1 where a run starts, then (after the
// inclusive scan) run_start[cnt[b + 1] - 1] = b, and run_start[n_runs] = B.
__global__ void run_flag_kernel(int B, const int* N_b, const int* N2_b, long long* cnt) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    cnt[b + 1] = (b == 0 || N_b[b] != N_b[b - 1] || (N2_b && N2_b[b] != N2_b[b - 1])) ? 1 : 0;
}

__global__ void run_start_kernel(int B, const int* N_b, const int* N2_b, const long long* cnt, int* run_start) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b == 0) run_start[cnt[B]] = B;
    if (b >= B) return;
    if (b == 0 || N_b[b] != N_b[b - 1] || (N2_b && N2_b[b] != N2_b[b - 1])) run_start[cnt[b + 1] - 1] = b;
}

// binary32 copies of the bins for the screening: (E, N), N2, D - lnH
__global__ void prep32_kernel(int B, const double* E_b, const int* N_b, const int* N2_b, const double* D,
                              const double* lnH, float2* EN32, float* N2f, float* DH32) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    EN32[b] = make_float2((float)E_b[b], (float)N_b[b]);
    if (N2_b) N2f[b] = (float)N2_b[b];
    DH32[b] = (float)(D[b] - lnH[b]);
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

__global__ void prep_bins_kernel(int B, const double* H, double* lnH) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) lnH[b] = log(H[b]);
}

// ---- iterations on a sparse kernel matrix
// With every state sampled, the map can be iterated in linear space: for a
// reference point f_ref (the iterate at the last build),
//   K_sb = exp(t_sb - M_b),  t_sb = ln Omega_s + f_ref,s - u_s(b),  M_b = max_s t_sb,
// so that with w_s = exp(f_s - f_ref,s)
//   D_b = M_b + ln d_b,  d_b = sum_s K_sb w_s,
//   f_new,s = ln Omega_s + f_ref,s - ln sum_b (H_b / d_b) K_sb,
// two FP64 sparse matrix-vector products per map and no exponentials.  Of
// the S B entries only those whose binary32 screen value (t_sb in binary32)
// is within kKeep + kMargin of the largest of their bin are kept: with
// hundreds of states most of a bin's terms lie far below its largest.  The
// matrix holds to e^-50 while the spread of the drift, max_s (f_s - f_ref,s)
// - min_s (f_s - f_ref,s), is at most kSpreadAcc: a dropped entry then weighs
// at most e^(-kKeep + kSpreadAcc) = e^-50 of the largest term of its bin (a
// uniform shift of f changes nothing), so the (at most 65536) dropped terms
// of d_b stay below 1e-17 of it, and those of a state's sum below 1e-17 of
// it too while its observations Omega_s are not below N_obs / S e^-13.  Far
// from the fixed point the iteration runs on the matrix until the spread
// exceeds kSpreadMax (its map then errs by at most e^-10 relative, which
// changes the path, not the end point); convergence is accepted only on a
// map evaluated within kSpreadAcc, else the matrix is rebuilt there.
// Each bin keeps its largest entry (K = 1), so d_b > 0; a state whose sum has
// no kept entry (possible far from the fixed point) makes that map fall back
// to the log-sum-exp form.
// The entries are held twice: by bin (CSR, states ascending) for d_b and by
// state (in kFSplit bin quarters, bins ascending) for f_new; both are summed
// in a fixed order, so the iteration is deterministic.
constexpr long long kWarmMinBins = 65536;   // smaller problems solve from f = 0
constexpr double kKeep = 70.0;
constexpr double kSpreadAcc = 20.0;
constexpr double kSpreadMax = 60.0;

struct SpDev {
    long long* rp;   // [B + 1] entries of bin b: rp[b] .. rp[b + 1] - 1
    int* ci;         // [nnz] their states, ascending within a bin
    double* cv;      // [nnz] K_sb
    long long* cp;   // [kFSplit S + 1] entries of state s in bin quarter r: cp[kFSplit s + r] ..
    int* bi;         // [nnz] their bins, ascending within a segment
    double* bv;      // [nnz] K_sb
    float* thr;      // [B] the bin's binary32 screening threshold
    double* M;       // [B] M_b
    double* H;       // [B] H_b
    double* V;       // [B] H_b / d_b of the last map
    double* fref;    // [S]
    double* w;       // [S] exp(f_s - f_ref,s) of the current iterate (from the host)
    int* flag;       // [2] entries of the state segments missing from their bin's row; empty state sums
    // the by-state sums in pieces (sp_fp_kernel, sp_fs_kernel)
    long long* pc_begin;   // [n_pieces + 1] first entry of each piece
    int* pc_first;         // [S + 1] first piece of each state
    double* pc_sum;        // [n_pieces]
};

// The binary32 screen value of state (g, a, c, c2) at bin (en, n2).  The row
// and the state passes evaluate this same expression on the same binary32
// operands, so they keep the same entries.
template <bool TWO>
__device__ __forceinline__ float screen32(float g, float a, float c, float c2, float2 en, float n2) {
    return g - u32_of<TWO>(a, c, c2, en.x, en.y, n2);
}

template <bool TWO>
__device__ __forceinline__ void state32(const MbarDev& m, const double* fref, int k, float& g, float& a, float& c,
                                        float& c2) {
    g = (float)(m.lnom[k] + fref[k]);
    a = (float)m.a[k];
    c = (float)m.c[k];
    c2 = TWO ? (float)m.c2[k] : 0.f;
}

// One thread per bin: the largest screen value over the states (tiled
// through shared memory), the threshold, and the number of kept entries
// (-> rp[b + 1], scanned afterwards).
template <bool TWO>
__global__ void __launch_bounds__(256) sp_screen_kernel(const __grid_constant__ MbarDev m, SpDev p) {
    __shared__ float fa[kDTile], fc[kDTile], fg[kDTile], fc2[TWO ? kDTile : 1];
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = b < m.B;
    const float2 en = act ? m.EN32[b] : make_float2(0.f, 0.f);
    const float n2f = (TWO && act) ? m.N2f[b] : 0.f;
    const bool one_tile = m.S <= kDTile;
    float mx = -INFINITY, th = -INFINITY;
    long long cnt = 0;
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) th = mx - (float)kKeep - kMargin;
        for (int k0 = 0; k0 < m.S; k0 += kDTile) {
            const int nk = min(kDTile, m.S - k0);
            if (pass == 0 || !one_tile) {
                __syncthreads();
                for (int q = threadIdx.x; q < nk; q += blockDim.x) {
                    float c2;
                    state32<TWO>(m, p.fref, k0 + q, fg[q], fa[q], fc[q], c2);
                    if (TWO) fc2[q] = c2;
                }
                __syncthreads();
            }
            if (!act) continue;
            if (pass == 0) {
                for (int q = 0; q < nk; ++q)
                    mx = fmaxf(mx, screen32<TWO>(fg[q], fa[q], fc[q], fc2[TWO ? q : 0], en, n2f));
            } else {
                for (int q = 0; q < nk; ++q)
                    cnt += screen32<TWO>(fg[q], fa[q], fc[q], fc2[TWO ? q : 0], en, n2f) > th;
            }
        }
    }
    if (act) {
        p.thr[b] = th;
        p.rp[b + 1] = cnt;
    }
}

// One thread per bin: M_b over the kept states in FP64, then the row
// (states ascending, K_sb = exp(t_sb - M_b)).
template <bool TWO>
__global__ void __launch_bounds__(256) sp_rows_kernel(const __grid_constant__ MbarDev m, SpDev p) {
    __shared__ double sa[kDTile], sc[kDTile], sg[kDTile], sc2[TWO ? kDTile : 1];
    __shared__ float fa[kDTile], fc[kDTile], fg[kDTile], fc2[TWO ? kDTile : 1];
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = b < m.B;
    const double E = act ? m.E_b[b] : 0.0;
    const double N = act ? (double)m.N_b[b] : 0.0;
    const double N2 = (TWO && act) ? (double)m.N2_b[b] : 0.0;
    const float2 en = act ? m.EN32[b] : make_float2(0.f, 0.f);
    const float n2f = (TWO && act) ? m.N2f[b] : 0.f;
    const float th = act ? p.thr[b] : 0.f;
    const bool one_tile = m.S <= kDTile;
    double M = -INFINITY;
    long long e = act ? p.rp[b] : 0;
    for (int pass = 0; pass < 2; ++pass) {
        for (int k0 = 0; k0 < m.S; k0 += kDTile) {
            const int nk = min(kDTile, m.S - k0);
            if (pass == 0 || !one_tile) {
                __syncthreads();
                for (int q = threadIdx.x; q < nk; q += blockDim.x) {
                    float c2;
                    state32<TWO>(m, p.fref, k0 + q, fg[q], fa[q], fc[q], c2);
                    sa[q] = m.a[k0 + q];
                    sc[q] = m.c[k0 + q];
                    sg[q] = m.lnom[k0 + q] + p.fref[k0 + q];
                    if (TWO) {
                        fc2[q] = c2;
                        sc2[q] = m.c2[k0 + q];
                    }
                }
                __syncthreads();
            }
            if (!act) continue;
            for (int q = 0; q < nk; ++q) {
                if (!(screen32<TWO>(fg[q], fa[q], fc[q], fc2[TWO ? q : 0], en, n2f) > th)) continue;
                const double t = sg[q] - u_of<TWO>(sa[q], sc[q], sc2[TWO ? q : 0], E, N, N2);
                if (pass == 0) {
                    M = fmax(M, t);
                } else {
                    p.ci[e] = k0 + q;
                    p.cv[e] = exp(t - M);
                    ++e;
                }
            }
        }
    }
    if (act) {
        p.M[b] = M;
        p.H[b] = exp(m.lnH[b]);
    }
}

// The entries by state: kFSplit CTAs per state, CTA r over bin quarter r.
// COUNT: the number of kept entries -> cp[kFSplit s + r + 1] (scanned
// afterwards).  Otherwise the segment is written in bin order (a block-wide
// ordered compaction), each value taken from the bin's row (binary search
// over its ascending states).
template <bool TWO, bool COUNT>
__global__ void __launch_bounds__(kFThreads) sp_cols_kernel(const __grid_constant__ MbarDev m, SpDev p) {
    constexpr int kWarps = kFThreads / 32;
    __shared__ int wcnt[kWarps];
    const int s = blockIdx.x / kFSplit, r = blockIdx.x % kFSplit;
    const int per = (m.B + kFSplit - 1) / kFSplit;
    const int b0 = r * per, b1 = min(m.B, b0 + per);
    float g, a, c, c2;
    state32<TWO>(m, p.fref, s, g, a, c, c2);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (COUNT) {
        long long cnt = 0;
        for (int b = b0 + threadIdx.x; b < b1; b += kFThreads)
            cnt += screen32<TWO>(g, a, c, c2, m.EN32[b], TWO ? m.N2f[b] : 0.f) > p.thr[b];
        const double tot = block_sum((double)cnt);   // exact: counts below 2^53
        if (threadIdx.x == 0) p.cp[blockIdx.x + 1] = (long long)tot;
        return;
    }
    long long base = p.cp[blockIdx.x];
    for (int bb = b0; bb < b1; bb += kFThreads) {
        const int b = bb + threadIdx.x;
        const bool keep = b < b1 && screen32<TWO>(g, a, c, c2, m.EN32[b], TWO ? m.N2f[b] : 0.f) > p.thr[b];
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) wcnt[warp] = __popc(bal);
        __syncthreads();
        int off = 0, tot = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            off += w < warp ? wcnt[w] : 0;
            tot += wcnt[w];
        }
        if (keep) {
            const long long e = base + off + __popc(bal & ((1u << lane) - 1u));
            long long lo = p.rp[b], hi = p.rp[b + 1];
            while (lo < hi) {
                const long long mid = (lo + hi) >> 1;
                if (p.ci[mid] < s) lo = mid + 1;
                else hi = mid;
            }
            p.bi[e] = b;
            if (lo < p.rp[b + 1] && p.ci[lo] == s) {
                p.bv[e] = p.cv[lo];
            } else {
                p.bv[e] = 0.0;
                atomicAdd(&p.flag[0], 1);
            }
        }
        base += tot;
        __syncthreads();   // wcnt is rewritten by the next round
    }
}

// d_b = sum_s K_sb w_s over the bin's row, then V_b = H_b / d_b; FINAL:
// D_b = M_b + ln d_b instead.  kDLanes lanes per bin (8 bins per warp): a
// warp-wide FP64 instruction costs the narrow FP64 pipe the same whatever its
// active lanes, so the reduction and the division are shared by 8 bins, while
// a lane group still reads 32 consecutive bytes of its row per step.  Two
// FMA chains per lane, combined in a fixed order (deterministic).
constexpr int kDLanes = 4;
template <bool FINAL>
__global__ void __launch_bounds__(256) sp_d_kernel(const __grid_constant__ MbarDev m, SpDev p) {
    const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long b = gt / kDLanes;
    const int sub = (int)(gt % kDLanes);
    const bool act = b < m.B;
    double d0 = 0.0, d1 = 0.0;
    if (act) {
        const long long e1 = p.rp[b + 1];
        long long e = p.rp[b] + sub;
        for (; e + kDLanes < e1; e += 2 * kDLanes) {
            d0 = fma(p.cv[e], __ldg(p.w + p.ci[e]), d0);
            d1 = fma(p.cv[e + kDLanes], __ldg(p.w + p.ci[e + kDLanes]), d1);
        }
        if (e < e1) d0 = fma(p.cv[e], __ldg(p.w + p.ci[e]), d0);
    }
    double d = d0 + d1;
#pragma unroll
    for (int o = 1; o < kDLanes; o <<= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    if (act && sub == 0) {
        if (FINAL) {
            const double D = p.M[b] + log(d);
            m.D[b] = D;
            m.DH32[b] = (float)(D - m.lnH[b]);
        } else {
            p.V[b] = p.H[b] / d;
        }
    }
}

// The by-state sums in balanced pieces: a state's entries (its kFSplit
// segments, contiguous) are cut into pieces of at most kPiece entries (fewer
// for a small matrix), one
// CTA per piece, so that a state with many entries does not hold back the
// map; sp_fs_kernel then adds each state's piece sums in piece order
// (deterministic) into f_new,s = ln Omega_s + f_ref,s - ln sum_b V_b K_sb.
constexpr long long kPiece = 32768;
__global__ void __launch_bounds__(kFThreads) sp_fp_kernel(const __grid_constant__ SpDev p) {
    const long long e0 = p.pc_begin[blockIdx.x], e1 = p.pc_begin[blockIdx.x + 1];
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    long long e = e0 + threadIdx.x;
    for (; e + 3 * kFThreads < e1; e += 4 * kFThreads) {
        const int b0 = p.bi[e], b1 = p.bi[e + kFThreads], b2 = p.bi[e + 2 * kFThreads], b3 = p.bi[e + 3 * kFThreads];
        const double k0 = p.bv[e], k1 = p.bv[e + kFThreads], k2 = p.bv[e + 2 * kFThreads], k3 = p.bv[e + 3 * kFThreads];
        a0 = fma(k0, p.V[b0], a0);
        a1 = fma(k1, p.V[b1], a1);
        a2 = fma(k2, p.V[b2], a2);
        a3 = fma(k3, p.V[b3], a3);
    }
    for (; e < e1; e += kFThreads) a0 = fma(p.bv[e], p.V[p.bi[e]], a0);
    const double acc = block_sum((a0 + a1) + (a2 + a3));
    if (threadIdx.x == 0) p.pc_sum[blockIdx.x] = acc;
}

// One thread per state: its pieces are pc_first[s] .. pc_first[s + 1] - 1.
// An empty sum raises flag[1].
__global__ void __launch_bounds__(256) sp_fs_kernel(const __grid_constant__ MbarDev m, SpDev p) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= m.S) return;
    double t = 0.0;
    for (int q = p.pc_first[s]; q < p.pc_first[s + 1]; ++q) t += p.pc_sum[q];
    if (t > 0.0) {
        m.f_new[s] = m.lnom[s] + p.fref[s] - log(t);
    } else {
        m.f_new[s] = 0.0;
        atomicAdd(&p.flag[1], 1);
    }
}

// ---- warm start: the problem coarsened in energy.  Bins adjacent in the
// bin order with equal N (and N2) and equal floor(E / width) are merged: the
// counts added, the energy their count-weighted mean.
__device__ __forceinline__ bool same_coarse(const MbarDev& m, long long b, long long c, double width) {
    return m.N_b[b] == m.N_b[c] && (m.N2_b == nullptr || m.N2_b[b] == m.N2_b[c]) &&
           floor(m.E_b[b] / width) == floor(m.E_b[c] / width);
}

__global__ void __launch_bounds__(256) coarse_flag_kernel(const __grid_constant__ MbarDev m, double width,
                                                          long long* cnt) {
    const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= m.B) return;
    cnt[b + 1] = (b == 0 || !same_coarse(m, b, b - 1, width)) ? 1 : 0;
}

// after the inclusive scan of cnt[1 .. B]: the run starting at b is coarse bin cnt[b + 1] - 1
__global__ void __launch_bounds__(256) coarse_fill_kernel(const __grid_constant__ MbarDev m, double width,
                                                          const long long* cnt, int* Nc, int* N2c, double* Ec,
                                                          double* lnHc) {
    const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= m.B || !(b == 0 || !same_coarse(m, b, b - 1, width))) return;
    double h = 0.0, he = 0.0;
    for (long long c = b; c < m.B && same_coarse(m, c, b, width); ++c) {
        const double hc = exp(m.lnH[c]);
        h += hc;
        he = fma(hc, m.E_b[c], he);
    }
    const long long o = cnt[b + 1] - 1;
    Nc[o] = m.N_b[b];
    if (N2c) N2c[o] = m.N2_b[b];
    Ec[o] = he / h;
    lnHc[o] = log(h);
}

// ---- inclusive scan of long long x[n] in place: chunk totals, one block
// over the totals (exclusive), then every chunk with its offset.
constexpr int kScanChunk = 1024;   // 256 threads x 4

__device__ __forceinline__ long long block_scan_incl(long long v, long long* wsum, long long* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) wsum[warp] = v;
    __syncthreads();
    if (warp == 0) {
        long long y = lane < nw ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long t = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += t;
        }
        wsum[lane] = y;
    }
    __syncthreads();
    const long long r = v + (warp > 0 ? wsum[warp - 1] : 0);
    if (total) *total = wsum[nw - 1];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(256) lchunk_sum_kernel(const long long* x, long long n, long long* tot) {
    const long long base = (long long)blockIdx.x * kScanChunk;
    long long v = 0;
    for (int k = 0; k < 4; ++k) {
        const long long i = base + threadIdx.x * 4 + k;
        if (i < n) v += x[i];
    }
    const double t = block_sum((double)v);   // exact: totals below 2^53
    if (threadIdx.x == 0) tot[blockIdx.x] = (long long)t;
}

__global__ void __launch_bounds__(1024) ltot_scan_kernel(long long* tot, long long nblk) {
    __shared__ long long wsum[32];
    __shared__ long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (long long b0 = 0; b0 < nblk; b0 += blockDim.x) {
        const long long i = b0 + threadIdx.x;
        const long long v = i < nblk ? tot[i] : 0;
        long long all;
        const long long incl = block_scan_incl(v, wsum, &all);
        if (i < nblk) tot[i] = carry + incl - v;
        __syncthreads();
        if (threadIdx.x == 0) carry += all;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) lchunk_scan_kernel(long long* x, long long n, const long long* tot) {
    __shared__ long long wsum[32];
    const long long i0 = (long long)blockIdx.x * kScanChunk + threadIdx.x * 4;
    long long v[4], run = 0;
    for (int k = 0; k < 4; ++k) {
        v[k] = i0 + k < n ? x[i0 + k] : 0;
        run += v[k];
        v[k] = run;
    }
    const long long excl = block_scan_incl(run, wsum, nullptr) - run + tot[blockIdx.x];
    for (int k = 0; k < 4; ++k)
        if (i0 + k < n) x[i0 + k] = v[k] + excl;
}

}  // namespace

namespace {

double spread_of(const std::vector<double>& x, const std::vector<double>& ref) {
    double lo = INFINITY, hi = -INFINITY;
    for (size_t k = 0; k < x.size(); ++k) {
        lo = fmin(lo, x[k] - ref[k]);
        hi = fmax(hi, x[k] - ref[k]);
    }
    return x.empty() ? 0.0 : hi - lo;
}

cudaError_t lscan(long long* x, long long n, long long* tmp, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const long long nblk = (n + kScanChunk - 1) / kScanChunk;
    lchunk_sum_kernel<<<(unsigned)nblk, 256, 0, s>>>(x, n, tmp);
    ltot_scan_kernel<<<1, 1024, 0, s>>>(tmp, nblk);
    lchunk_scan_kernel<<<(unsigned)nblk, 256, 0, s>>>(x, n, tmp);
    return cudaGetLastError();
}

// The sparse kernel matrix on the device (allocated on the stream, freed
// with it) and its build at the iterate held in m.f.
struct SparseMat {
    cudaStream_t s = nullptr;
    void* fixed = nullptr;     // the bin- and state-sized arrays
    void* entries = nullptr;   // cap entries: cv, bv (double), ci, bi (int)
    void* pieces = nullptr;    // pc_begin, pc_sum, pc_first for up to pc_cap pieces
    long long cap = 0, nnz = 0, pc_cap = 0, n_pieces = 0;
    long long* tmp = nullptr;  // scan scratch
    SpDev p{};

    ~SparseMat() {
        if (pieces) cudaFreeAsync(pieces, s);
        if (entries) cudaFreeAsync(entries, s);
        if (fixed) cudaFreeAsync(fixed, s);
    }

    cudaError_t init(const MbarDev& m) {
        const size_t B = size_t(m.B), S = size_t(m.S), SF = size_t(kFSplit) * S;
        const size_t nt = std::max((B + kScanChunk - 1) / kScanChunk, (SF + kScanChunk - 1) / kScanChunk) + 1;
        const size_t n8 = (B + 1) + (SF + 1) + 3 * B + 2 * S + nt;
        cudaError_t e = cudaMallocAsync(&fixed, n8 * 8 + B * 4 + 16, s);
        if (e != cudaSuccess) {
            fixed = nullptr;
            return e;
        }
        long long* q = static_cast<long long*>(fixed);
        p.rp = q;
        p.cp = p.rp + (B + 1);
        double* d = reinterpret_cast<double*>(p.cp + (SF + 1));
        p.M = d;
        p.H = d + B;
        p.V = d + 2 * B;
        p.fref = d + 3 * B;
        p.w = p.fref + S;
        tmp = reinterpret_cast<long long*>(p.w + S);
        p.thr = reinterpret_cast<float*>(tmp + nt);
        p.flag = reinterpret_cast<int*>(p.thr + B);
        e = cudaMemsetAsync(p.rp, 0, sizeof(long long), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(p.cp, 0, sizeof(long long), s);
        return e;
    }

    // *ok is false when the entries do not fit (half the free device memory)
    // or the two orders disagree; the caller then iterates on log-sum-exps.
    template <bool TWO>
    cudaError_t build(const MbarDev& m, bool* ok) {
        *ok = false;
        const int S = m.S, B = m.B;
        cudaError_t e = cudaMemcpyAsync(p.fref, m.f, size_t(S) * sizeof(double), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
        sp_screen_kernel<TWO><<<(B + 255) / 256, 256, 0, s>>>(m, p);
        e = lscan(p.rp + 1, B, tmp, s);
        long long n_h = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&n_h, p.rp + B, sizeof(long long), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return e;
        if (n_h > cap) {
            if (entries) cudaFreeAsync(entries, s);
            entries = nullptr;
            cap = 0;
            size_t fr = 0, tot = 0;
            e = cudaMemGetInfo(&fr, &tot);
            if (e != cudaSuccess) return e;
            const size_t need = size_t(n_h) * 24;
            if (need > fr / 2) return cudaSuccess;
            if (cudaMallocAsync(&entries, need, s) != cudaSuccess) {
                entries = nullptr;
                (void)cudaGetLastError();   // out of memory is not sticky
                return cudaSuccess;
            }
            cap = n_h;
            p.cv = static_cast<double*>(entries);
            p.bv = p.cv + cap;
            p.ci = reinterpret_cast<int*>(p.bv + cap);
            p.bi = p.ci + cap;
        }
        nnz = n_h;
        sp_rows_kernel<TWO><<<(B + 255) / 256, 256, 0, s>>>(m, p);
        sp_cols_kernel<TWO, true><<<S * kFSplit, kFThreads, 0, s>>>(m, p);
        e = lscan(p.cp + 1, (long long)S * kFSplit, tmp, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(p.flag, 0, 2 * sizeof(int), s);
        if (e != cudaSuccess) return e;
        sp_cols_kernel<TWO, false><<<S * kFSplit, kFThreads, 0, s>>>(m, p);
        int flag_h = 0;
        std::vector<long long> cp_h(size_t(S) * kFSplit + 1);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&flag_h, p.flag, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(cp_h.data(), p.cp, cp_h.size() * sizeof(long long), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return e;
        if (flag_h != 0 || cp_h.back() != nnz) return cudaSuccess;
        // pieces of at most kPiece entries (fewer for a small matrix, so that
        // there are about eight per SM), at least one per state
        int sms = 152;
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            (void)cudaGetLastError();
            sms = 152;
        }
        const long long piece = std::max(2048LL, std::min(kPiece, nnz / (8LL * sms) + 1));
        std::vector<long long> begin;
        std::vector<int> first(size_t(S) + 1);
        for (int k = 0; k < S; ++k) {
            first[k] = (int)begin.size();
            const long long a = cp_h[size_t(k) * kFSplit], b = cp_h[size_t(k + 1) * kFSplit];
            const long long np = std::max(1LL, (b - a + piece - 1) / piece);
            for (long long q = 0; q < np; ++q) begin.push_back(a + (b - a) * q / np);
        }
        first[S] = (int)begin.size();
        n_pieces = (long long)begin.size();
        begin.push_back(nnz);
        if (n_pieces > pc_cap) {
            if (pieces) cudaFreeAsync(pieces, s);
            pieces = nullptr;
            pc_cap = 0;
            const long long want = n_pieces + n_pieces / 4 + 16;
            e = cudaMallocAsync(&pieces, size_t(want + 1) * 16 + size_t(S + 1) * 4, s);
            if (e != cudaSuccess) {
                pieces = nullptr;
                (void)cudaGetLastError();   // out of memory is not sticky
                return cudaSuccess;
            }
            pc_cap = want;
            p.pc_begin = static_cast<long long*>(pieces);
            p.pc_sum = reinterpret_cast<double*>(p.pc_begin + (want + 1));
            p.pc_first = reinterpret_cast<int*>(p.pc_sum + want);
        }
        e = cudaMemcpyAsync(p.pc_begin, begin.data(), begin.size() * sizeof(long long), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(p.pc_first, first.data(), first.size() * sizeof(int), cudaMemcpyHostToDevice, s);
        // the host vectors go out of scope: wait for the copies
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return e;
        *ok = true;
        return cudaSuccess;
    }
};

}  // namespace

// The self-consistent map G(f) = gauge(f_new(D(f))) is iterated with
// Anderson acceleration (Walker & Ni, SIAM J. Numer. Anal. 49, 1715 (2011),
// "type II" with differences): with the residuals r_i = G(x_i) - x_i of the
// last kDepth iterates, gamma minimises |r_k - sum_j gamma_j (r_{j+1} - r_j)|
// and x_{k+1} = G(x_k) - sum_j gamma_j (G(x_{j+1}) - G(x_j)).  The fixed point
// is the one of the plain iteration (x = G(x)); only the path to it is
// shorter.  An iterate whose residual grows past 100 times the best one so far
// restarts the history from the best image.  Converged when max |r| < tol.
namespace {
thread_local MbarInfo g_last_info{};
}

MbarInfo mbar_last_info() { return g_last_info; }

cudaError_t mbar_solve_dev(const MbarDev& m, double tol, int max_iter, int* iters_out, cudaStream_t s,
                           bool allow_matrix, const double* x0) {
    constexpr int kDepth = 16;
    const int S = m.S;
    MbarInfo& info = g_last_info;
    info = MbarInfo{0, 0, 0, 0, 0, S, m.B, 0.0, 0.0, 0, 0, 0, 0, 0};
    // device time of the builds and of the maps on the matrix
    struct Timer {
        cudaEvent_t a = nullptr, b = nullptr;
        Timer() {
            if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
                (void)cudaGetLastError();
                a = b = nullptr;
            }
        }
        ~Timer() {
            if (a) cudaEventDestroy(a);
            if (b) cudaEventDestroy(b);
        }
        void start(cudaStream_t s) {
            if (a) cudaEventRecord(a, s);
        }
        void stop(cudaStream_t s) {
            if (b) cudaEventRecord(b, s);
        }
        // once the stream has been synchronised past the stop event
        double ms() const {
            float t = 0.f;
            return (a && b && cudaEventElapsedTime(&t, a, b) == cudaSuccess) ? (double)t : 0.0;
        }
    } tb, tm;
    cudaError_t err = cudaMemsetAsync(m.state, 0, 2 * sizeof(int), s);
    if (err != cudaSuccess) return err;
    std::vector<double> x(S, 0.0);
    if (x0)
        for (int k = 0; k < S; ++k) x[k] = x0[k] - x0[0];
    err = cudaMemcpyAsync(m.f, x.data(), size_t(S) * sizeof(double), cudaMemcpyHostToDevice, s);
    if (err != cudaSuccess) return err;
    const int dgrid = (m.B + 255) / 256;
    const int dgrid128 = (m.B + 127) / 128;   // a bin per thread, small blocks to spread over every SM
    en32_kernel<<<dgrid, 256, 0, s>>>(m.B, m.E_b, m.N_b, m.EN32, m.N2_b, m.N2f);
    const bool two = m.N2_b != nullptr;
    // the sparse kernel matrix, when every state is sampled and it fits
    SparseMat sp;
    sp.s = s;
    bool use_sp = false;
    if (allow_matrix) {
        std::vector<double> lnom_h(S);
        err = cudaMemcpyAsync(lnom_h.data(), m.lnom, size_t(S) * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (err == cudaSuccess) err = cudaStreamSynchronize(s);
        if (err != cudaSuccess) return err;
        bool all_sampled = true;
        for (int k = 0; k < S; ++k) all_sampled = all_sampled && std::isfinite(lnom_h[k]);
        if (all_sampled) {
            use_sp = sp.init(m) == cudaSuccess;
            if (!use_sp) (void)cudaGetLastError();   // out of memory is not sticky: iterate on log-sum-exps
        }
    }
    std::vector<double> fref_h(x), w_h(S);
    bool build = true;
    std::vector<double> g(S), r(S), best_g(x), rhs(kDepth), A(kDepth * kDepth), gam(kDepth);
    std::vector<std::vector<double>> dR, dG;       // differences of residuals and images, oldest first
    std::vector<double> r_prev, g_prev;
    double best = INFINITY;
    int it = 0;
    while (it < max_iter) {
        if (it > 0) {
            err = cudaMemcpyAsync(m.f, x.data(), size_t(S) * sizeof(double), cudaMemcpyHostToDevice, s);
            if (err != cudaSuccess) return err;
        }
        double spread = 0.0;
        if (use_sp) {
            spread = spread_of(x, fref_h);
            if (build || !(spread <= kSpreadMax)) {
                bool ok = false;
                tb.start(s);
                err = two ? sp.build<true>(m, &ok) : sp.build<false>(m, &ok);
                if (err != cudaSuccess) return err;
                tb.stop(s);
                err = cudaStreamSynchronize(s);
                if (err != cudaSuccess) return err;
                info.ms_build += tb.ms();
                use_sp = ok;   // too large or inconsistent: log-sum-exps from here on
                info.path = ok ? 1 : 0;
                info.builds += ok ? 1 : 0;
                info.nnz = ok ? sp.nnz : 0;
                fref_h = x;
                spread = 0.0;
                build = false;
                // the map has changed: the Anderson history starts again
                dR.clear();
                dG.clear();
                r_prev.clear();
                best = INFINITY;
            }
        }
        bool mapped = false;
        if (use_sp) {
            for (int k = 0; k < S; ++k) w_h[k] = exp(x[k] - fref_h[k]);
            int empty = 0;
            err = cudaMemcpyAsync(sp.p.w, w_h.data(), size_t(S) * sizeof(double), cudaMemcpyHostToDevice, s);
            if (err == cudaSuccess) err = cudaMemsetAsync(sp.p.flag + 1, 0, sizeof(int), s);
            if (err != cudaSuccess) return err;
            tm.start(s);
            sp_d_kernel<false><<<(unsigned)((m.B * (long long)kDLanes + 255) / 256), 256, 0, s>>>(m, sp.p);
            sp_fp_kernel<<<(unsigned)sp.n_pieces, kFThreads, 0, s>>>(sp.p);
            sp_fs_kernel<<<(S + 255) / 256, 256, 0, s>>>(m, sp.p);
            tm.stop(s);
            err = cudaGetLastError();
            if (err == cudaSuccess)
                err = cudaMemcpyAsync(g.data(), m.f_new, size_t(S) * sizeof(double), cudaMemcpyDeviceToHost, s);
            if (err == cudaSuccess) err = cudaMemcpyAsync(&empty, sp.p.flag + 1, sizeof(int), cudaMemcpyDeviceToHost, s);
            if (err == cudaSuccess) err = cudaStreamSynchronize(s);
            if (err != cudaSuccess) return err;
            info.ms_maps += tm.ms();
            ++info.sparse_maps;
            mapped = empty == 0;   // else a state had no kept entry: this map on log-sum-exps
        }
        if (!mapped) {
            ++info.lse_maps;
            if (two) {
                d_kernel<true><<<dgrid128, 128, 0, s>>>(m, 1);
                f_kernel<true><<<S * kFSplit, kFThreads, 0, s>>>(m);
            } else {
                d_kernel<false><<<dgrid128, 128, 0, s>>>(m, 1);
                f_kernel<false><<<S * kFSplit, kFThreads, 0, s>>>(m);
            }
            err = cudaGetLastError();
            if (err != cudaSuccess) return err;
            err = cudaMemcpyAsync(g.data(), m.f_new, size_t(S) * sizeof(double), cudaMemcpyDeviceToHost, s);
            if (err == cudaSuccess) err = cudaStreamSynchronize(s);
            if (err != cudaSuccess) return err;
        }
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
            // converged on a matrix that no longer holds to e^-50 at x: rebuild
            // there and go on
            if (mapped && !(spread <= kSpreadAcc)) {
                build = true;
                continue;
            }
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
    // D_b of the final f: on the matrix while it holds for f, else log-sum-exps
    if (use_sp && spread_of(x, fref_h) <= kSpreadAcc) {
        for (int k = 0; k < S; ++k) w_h[k] = exp(x[k] - fref_h[k]);
        err = cudaMemcpyAsync(sp.p.w, w_h.data(), size_t(S) * sizeof(double), cudaMemcpyHostToDevice, s);
        if (err != cudaSuccess) return err;
        sp_d_kernel<true><<<(unsigned)((m.B * (long long)kDLanes + 255) / 256), 256, 0, s>>>(m, sp.p);
    } else if (two) {
        d_kernel<true><<<dgrid128, 128, 0, s>>>(m, 1);
    } else {
        d_kernel<false><<<dgrid128, 128, 0, s>>>(m, 1);
    }
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    // the host vectors go out of scope: wait for the copy that reads x
    err = cudaStreamSynchronize(s);
    if (err != cudaSuccess) return err;
    if (iters_out) *iters_out = it;
    info.iterations = it;
    return cudaSuccess;
}

cudaError_t mbar_solve_warm_dev(const MbarDev& m, double width, double tol, int max_iter, int* iters_out,
                                cudaStream_t s) {
    std::vector<double> x0;
    long long Bc = 0;
    int it_c = 0;
    if (width > 0.0 && m.B >= kWarmMinBins) {
        std::vector<void*> blocks;
        struct Free {
            std::vector<void*>& v;
            cudaStream_t s;
            ~Free() {
                for (void* q : v) cudaFreeAsync(q, s);
            }
        } free_all{blocks, s};
        auto get = [&](size_t bytes) -> void* {
            void* q = nullptr;
            if (cudaMallocAsync(&q, std::max<size_t>(bytes, 16), s) != cudaSuccess) {
                (void)cudaGetLastError();
                return nullptr;
            }
            blocks.push_back(q);
            return q;
        };
        const long long B = m.B;
        long long* cnt = static_cast<long long*>(get(size_t(B + 1) * 8));
        long long* tmp = static_cast<long long*>(get(size_t((B + kScanChunk - 1) / kScanChunk + 1) * 8));
        bool ok = cnt && tmp;
        cudaError_t e = cudaSuccess;
        if (ok) {
            e = cudaMemsetAsync(cnt, 0, 8, s);
            if (e == cudaSuccess) {
                coarse_flag_kernel<<<(unsigned)((B + 255) / 256), 256, 0, s>>>(m, width, cnt);
                e = lscan(cnt + 1, B, tmp, s);
            }
            if (e == cudaSuccess) e = cudaMemcpyAsync(&Bc, cnt + B, 8, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return e;
        }
        // worth it only when the merge shrinks the problem well
        if (ok && Bc > 0 && Bc * 4 <= B) {
            MbarDev c = m;
            const size_t Sz = size_t(m.S);
            c.B = (int)Bc;
            int* Nc = static_cast<int*>(get(size_t(Bc) * 4));
            int* N2c = m.N2_b ? static_cast<int*>(get(size_t(Bc) * 4)) : nullptr;
            double* Ec = static_cast<double*>(get(size_t(Bc) * 8));
            double* lnHc = static_cast<double*>(get(size_t(Bc) * 8));
            c.f = static_cast<double*>(get(Sz * 8));
            c.f_new = static_cast<double*>(get(Sz * 8));
            c.D = static_cast<double*>(get(size_t(Bc) * 8));
            c.EN32 = static_cast<float2*>(get(size_t(Bc) * 8));
            c.DH32 = static_cast<float*>(get(size_t(Bc) * 4));
            c.N2f = m.N2_b ? static_cast<float*>(get(size_t(Bc) * 4)) : nullptr;
            c.delta = static_cast<double*>(get(8));
            c.state = static_cast<int*>(get(8));
            ok = Nc && Ec && lnHc && c.f && c.f_new && c.D && c.EN32 && c.DH32 && c.delta && c.state &&
                 (!m.N2_b || (N2c && c.N2f));
            if (ok) {
                coarse_fill_kernel<<<(unsigned)((B + 255) / 256), 256, 0, s>>>(m, width, cnt, Nc, N2c, Ec, lnHc);
                e = cudaGetLastError();
                if (e != cudaSuccess) return e;
                c.N_b = Nc;
                c.N2_b = N2c;
                c.E_b = Ec;
                c.lnH = lnHc;
                // a loose solve: it only has to land near the fine fixed point
                e = mbar_solve_dev(c, std::max(tol, 1e-6), max_iter, &it_c, s, true, nullptr);
                if (e != cudaSuccess) return e;
                x0.resize(Sz);
                e = cudaMemcpyAsync(x0.data(), c.f, Sz * 8, cudaMemcpyDeviceToHost, s);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                if (e != cudaSuccess) return e;
            }
        }
    }
    const MbarInfo coarse = g_last_info;
    cudaError_t e = mbar_solve_dev(m, tol, max_iter, iters_out, s, true, x0.empty() ? nullptr : x0.data());
    if (!x0.empty()) {
        g_last_info.coarse_B = Bc;
        g_last_info.coarse_iterations = it_c;
        g_last_info.ms_build += coarse.ms_build;
        g_last_info.ms_maps += coarse.ms_maps;
        g_last_info.coarse_builds = coarse.builds;
        g_last_info.coarse_maps = coarse.sparse_maps;
    }
    return e;
}

size_t mbar_runs_scratch(int B) {
    return size_t(B) + 1 + size_t((B + kScanChunk - 1) / kScanChunk) + 1;
}

cudaError_t mbar_runs_dev(const MbarDev& m, long long* scratch, int* run_start, int* n_runs, cudaStream_t s) {
    const int B = m.B;
    long long* cnt = scratch;
    long long* tmp = scratch + B + 1;
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(long long), s);
    if (e != cudaSuccess) return e;
    run_flag_kernel<<<(B + 255) / 256, 256, 0, s>>>(B, m.N_b, m.N2_b, cnt);
    e = lscan(cnt + 1, B, tmp, s);
    if (e == cudaSuccess) {
        run_start_kernel<<<(B + 255) / 256, 256, 0, s>>>(B, m.N_b, m.N2_b, cnt, run_start);
        e = cudaGetLastError();
    }
    long long n = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&n, cnt + B, sizeof(long long), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) *n_runs = (int)n;
    return e;
}

namespace {

// The query over runs when the per-warp accumulators fit in shared memory.
template <bool TWO>
bool query_runs(const MbarDev& m, int Q, const double* a_q, const double* c_q, const double* c2_q, int nmax,
                double* n_mean, double* n2_mean, double* pN, double* pN2, double* f_q, cudaStream_t s,
                cudaError_t* err) {
    if (!m.run_start || m.n_runs <= 0) return false;
    const size_t per_warp = ((TWO ? 2 : 1) * size_t(nmax + 1) + 3) * sizeof(double);
    const int warps = (int)std::min<size_t>(kRunWarps, size_t(200 * 1024) / per_warp);
    if (warps < 1) return false;
    const size_t smem = per_warp * warps;
    *err = cudaFuncSetAttribute(query_runs_kernel<TWO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (*err == cudaSuccess) {
        query_runs_kernel<TWO><<<Q, 32 * kRunWarps, smem, s>>>(m, a_q, c_q, c2_q, nmax, m.run_start, m.n_runs, warps,
                                                               n_mean, n2_mean, pN, pN2, f_q);
        *err = cudaGetLastError();
    }
    return true;
}

}  // namespace

cudaError_t mbar_query_dev(const MbarDev& m, int Q, const double* a_q, const double* c_q, int nmax,
                           double* n_mean, double* pN, double* f_q, cudaStream_t s) {
    if (Q <= 0) return cudaSuccess;
    cudaError_t rerr = cudaSuccess;
    if (query_runs<false>(m, Q, a_q, c_q, nullptr, nmax, n_mean, nullptr, pN, nullptr, f_q, s, &rerr)) return rerr;
    const size_t smem = size_t(nmax + 1) * (sizeof(double) + sizeof(float));
    cudaError_t err = cudaFuncSetAttribute(query_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    query_kernel<false><<<Q, kQThreads, smem, s>>>(m, a_q, c_q, nullptr, nmax, n_mean, nullptr, pN, nullptr, f_q);
    return cudaGetLastError();
}

cudaError_t mbar_prep32_dev(const MbarDev& m, cudaStream_t s) {
    if (m.B <= 0) return cudaSuccess;
    prep32_kernel<<<(m.B + 255) / 256, 256, 0, s>>>(m.B, m.E_b, m.N_b, m.N2_b, m.D, m.lnH, m.EN32, m.N2f, m.DH32);
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
    cudaError_t rerr = cudaSuccess;
    if (query_runs<true>(m, Q, a_q, c_q, c2_q, nmax, n_mean, n2_mean, pN, pN2, f_q, s, &rerr)) return rerr;
    const size_t smem = 2 * size_t(nmax + 1) * (sizeof(double) + sizeof(float));
    cudaError_t err = cudaFuncSetAttribute(query_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    query_kernel<true><<<Q, kQThreads, smem, s>>>(m, a_q, c_q, c2_q, nmax, n_mean, n2_mean, pN, pN2, f_q);
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
