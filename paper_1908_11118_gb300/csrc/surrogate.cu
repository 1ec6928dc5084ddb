// surrogate.cu -- the learned surrogate of the delayed-acceptance sweep (sm_103a).
//
// The paper has no surrogate.  This file holds:
//   * pack_kernel: FP32 master parameters -> the BF16 inference layout;
//   * eval_kernel: the surrogate energy (and features) of arbitrary positions
//     in one walker, one warp per position, over every partner (no cells);
//   * harvest_kernel: training rows (features, clipped exact interaction
//     energy) of particles of every walker and of random probe positions;
//   * grad_kernel / reduce_adam_kernel: one step of mini-batch training -- the
//     forward and backward passes of 128 rows per CTA in shared memory, the
//     per-CTA gradients summed in a fixed order, and Adam on the FP32 masters.
#include "launch.h"
#include "surrogate.cuh"

namespace regc {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kRows = 128;           // rows per training CTA (one per thread)
constexpr int kLd = kNH + 1;         // padded row stride of the activation tiles
constexpr int kLdX = kNF + 1;        // padded row stride of the feature tile

__global__ void pack_kernel(const float* theta, __nv_bfloat16* w1, float* b1, __nv_bfloat16* w2, float* b2,
                            __nv_bfloat16* w3, float* b3) {
    const float* W1 = theta;
    const float* B1 = W1 + kNF * kNH;
    const float* W2 = B1 + kNH;
    const float* B2 = W2 + kNH * kNH;
    const float* W3 = B2 + kNH;
    const float* B3 = W3 + kNH;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kNH * kNH; i += gridDim.x * blockDim.x) {
        const int v = i / kNH, u = i % kNH;          // unit v, input u
        w2[i] = __float2bfloat16_rn(W2[u * kNH + v]);
        if (i < kNH * kNF) {
            const int uu = i / kNF, k = i % kNF;     // unit uu, input k
            w1[i] = __float2bfloat16_rn(W1[k * kNH + uu]);
        }
        if (i < kNH) {
            b1[i] = B1[i];
            b2[i] = B2[i];
            w3[i] = __float2bfloat16_rn(W3[i]);
        }
        if (i == 0) b3[0] = B3[0];
    }
}

// Displacement q - p with the exact minimum image on periodic axes.
__device__ __forceinline__ float r2_exact(const Geometry& g, float qx, float qy, float qz, float4 p) {
    const float dy = min_image_exact(qy, p.y, g.Ly, g.hLy);
    const float dx = cart_dx(g, min_image_exact(qx, p.x, g.Lx, g.hLx), dy);
    const float dz = g.periodic_z ? min_image_exact(qz, p.z, g.Lz, g.hLz) : __fsub_rn(qz, p.z);
    return r2_of(dx, dy, dz);
}

// Features (per lane, before the warp sum) and exact binary32 interaction
// energy (warp sum) of a grand-canonical particle at q against every partner
// of walker w (cluster partners with the cluster pair table).
__device__ float features_all(const SweepParams& P, int w, int N, float qx, float qy, float qz, int skip,
                              float (&F)[kNF], int lane) {
    const float4* pos = P.pos + size_t(w) * P.nmax;
    float e = 0.f;
    for (int j = lane; j < N; j += 32) {
        if (j == skip) continue;
        const PairTab& t = j < P.n_cluster ? P.gAB : P.gg;
        const float r2 = r2_exact(P.g, qx, qy, qz, pos[j]);
        if (r2 < P.g.rc2) {
            add_features(F, r2, t.eps, P.g.rc);
            e += phi_of_r2(r2, t);
        }
    }
    for (int a = lane; a < P.st.n_all; a += 32) {
        const float4 at = P.st.all[a];
        const PairTab& t = surf_tab(P, (int)at.w);
        const float r2 = r2_exact(P.g, qx, qy, qz, at);
        if (r2 < P.g.rc2) {
            add_features(F, r2, t.eps, P.g.rc);
            e += phi_of_r2(r2, t);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(FULL, e, o);
    return e;
}

// One warp per pair of positions (2i, 2i + 1): features of each, then both
// through the network as rows 0 and 1 of its tensor-core tiles -- the sweep's
// code path.
__global__ void __launch_bounds__(128) eval_kernel(const __grid_constant__ SweepParams P, int w, int Q,
                                                   const float4* q, float* e_out, float* f_out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = 2 * (blockIdx.x * 4 + warp);
    if (i >= Q) return;
    const bool two = i + 1 < Q;
    float r[2];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const float4 x = q[two ? i + p : i];
        float F[kNF];
#pragma unroll
        for (int k = 0; k < kNF; ++k) F[k] = 0.f;
        features_all(P, w, P.n[w], x.x, x.y, x.z, -1, F, lane);
        r[p] = warp_reduce16(F, lane);
    }
    NetFrag nf;
    load_net(P.net, lane, nf);
    uint32_t a[4];
    features_to_frag(r[0], r[1], lane, a);
    float e1 = 0.f;
    const float e0 = net_mma(nf, a, &e1);
    if ((lane & 1) == 0) {
        f_out[size_t(i) * kNF + (lane >> 1)] = r[0];
        if (two) f_out[size_t(i + 1) * kNF + (lane >> 1)] = r[1];
    }
    if (lane == 0) {
        e_out[i] = e0;
        if (two) e_out[i + 1] = e1;
    }
}

// Row r of a harvest: walker r / per_w, slot r % per_w; the first `parts`
// slots are particles of the walker (evenly spaced indices), the rest (and
// every slot of an empty walker) random probe positions of the gas region
// (Philox stream 5).  Rows go to a ring of `cap` rows starting at `base`.
__global__ void __launch_bounds__(128) harvest_kernel(const __grid_constant__ SweepParams P, int parts, int probes,
                                                      float clip, uint32_t round, float* X, float* y, int base,
                                                      int cap) {
    const int lane = threadIdx.x & 31;
    const int per_w = parts + probes;
    const long long r = (long long)blockIdx.x * 4 + (threadIdx.x >> 5);
    if (r >= (long long)P.S * per_w) return;
    const int w = (int)(r / per_w), slot = (int)(r % per_w);
    const long long out = (base + r) % cap;
    const int N = P.n[w];
    float qx, qy, qz;
    int skip = -1;
    const int nB = N - P.n_cluster;   // rows are grand-canonical particles
    if (slot < parts && nB > 0) {
        skip = P.n_cluster + (int)(((long long)slot * nB) / parts);
        const float4 p = P.pos[size_t(w) * P.nmax + skip];
        qx = p.x; qy = p.y; qz = p.z;
    } else {
        const U4 u = philox(uint32_t(slot), uint32_t(w), round, 5u, P.key0, P.key1);
        qx = __fmul_rn(P.g.Lx, u24(u.x));
        qy = __fmul_rn(P.g.Ly, u24(u.y));
        qz = __fadd_rn(P.g.z_lo, __fmul_rn(P.g.height, u24(u.z)));
        if (qx >= P.g.Lx) qx = 0.f;
        if (qy >= P.g.Ly) qy = 0.f;
        if (P.g.periodic_z && qz >= P.g.Lz) qz = 0.f;
    }
    float F[kNF];
#pragma unroll
    for (int k = 0; k < kNF; ++k) F[k] = 0.f;
    const float e = features_all(P, w, N, qx, qy, qz, skip, F, lane);
    const float g = warp_reduce16(F, lane);
    if ((lane & 1) == 0) X[out * kNF + (lane >> 1)] = g;
    if (lane == 0) y[out] = fminf(e, clip);
}

__device__ __forceinline__ float dsilu_f(float x) {
    const float s = 1.0f / (1.0f + expf(-x));
    return s * (1.0f + x * (1.0f - s));
}

// Forward and backward pass of up to kRows rows (row t = idx[t] or base + t)
// with FP32 parameters theta; writes this CTA's gradient of
// sum_t (e_t - y_t)^2 * scale into partial[blockIdx.x][5313] and its sum of
// squared residuals into partial_loss[blockIdx.x].
__global__ void __launch_bounds__(kRows) grad_kernel(const float* theta, const float* X, const float* yv,
                                                     const int* idx, int n, float scale, float* partial,
                                                     float* partial_loss) {
    extern __shared__ __align__(16) float sm[];
    float* Wsh = sm;                                  // [5313] parameters
    float* Xs = Wsh + ((kNParams + 3) & ~3);          // [kRows][kLdX]
    float* Z1 = Xs + kRows * kLdX;                    // [kRows][kLd] z1, later dz1
    float* H1 = Z1 + kRows * kLd;                     // [kRows][kLd] h1
    float* Z2 = H1 + kRows * kLd;                     // [kRows][kLd] z2, later dz2
    float* gsh = Z2 + kRows * kLd;                    // [kRows] d loss / d e
    const int t = threadIdx.x;
    const int row0 = blockIdx.x * kRows;
    for (int i = t; i < kNParams; i += kRows) Wsh[i] = theta[i];
    const int row = row0 + t;
    const bool act = row < n;
    const int src = act ? (idx ? idx[row] : row) : 0;
    for (int k = 0; k < kNF; ++k) Xs[t * kLdX + k] = act ? X[size_t(src) * kNF + k] : 0.f;
    __syncthreads();
    const float* W1 = Wsh;
    const float* b1 = W1 + kNF * kNH;
    const float* W2 = b1 + kNH;
    const float* b2 = W2 + kNH * kNH;
    const float* W3 = b2 + kNH;
    const float b3 = W3[kNH];
    // forward, one row per thread
    for (int u = 0; u < kNH; ++u) {
        float z = b1[u];
        for (int k = 0; k < kNF; ++k) z = fmaf(W1[k * kNH + u], Xs[t * kLdX + k], z);
        Z1[t * kLd + u] = z;
        H1[t * kLd + u] = z / (1.0f + expf(-z));
    }
    float out = b3;
    for (int v = 0; v < kNH; ++v) {
        float z = b2[v];
        for (int u = 0; u < kNH; ++u) z = fmaf(W2[u * kNH + v], H1[t * kLd + u], z);
        Z2[t * kLd + v] = z;
        out = fmaf(W3[v], z / (1.0f + expf(-z)), out);
    }
    const float res = act ? out - yv[src] : 0.f;
    gsh[t] = 2.0f * res * scale;
    float* G = partial + size_t(blockIdx.x) * kNParams;
    float* gW1 = G;
    float* gb1 = gW1 + kNF * kNH;
    float* gW2 = gb1 + kNH;
    float* gb2 = gW2 + kNH * kNH;
    float* gW3 = gb2 + kNH;
    __syncthreads();
    // d loss / d W3, b3 (threads 0..63 own one unit each)
    if (t < kNH) {
        float acc = 0.f;
        for (int r = 0; r < kRows; ++r) {
            const float z = Z2[r * kLd + t];
            acc = fmaf(gsh[r], z / (1.0f + expf(-z)), acc);
        }
        gW3[t] = acc;
    } else if (t == kNH) {
        float acc = 0.f;
        for (int r = 0; r < kRows; ++r) acc += gsh[r];
        gW3[kNH] = acc;   // b3
    }
    __syncthreads();
    // dz2 = g W3 silu'(z2), in place
    for (int v = 0; v < kNH; ++v) {
        const float z = Z2[t * kLd + v];
        Z2[t * kLd + v] = gsh[t] * W3[v] * dsilu_f(z);
    }
    __syncthreads();
    // d W2 [u][v] = sum_r h1[r][u] dz2[r][v]; d b2
    for (int i = t; i < kNH * kNH; i += kRows) {
        const int u = i / kNH, v = i % kNH;
        float acc = 0.f;
        for (int r = 0; r < kRows; ++r) acc = fmaf(H1[r * kLd + u], Z2[r * kLd + v], acc);
        gW2[i] = acc;
    }
    if (t < kNH) {
        float acc = 0.f;
        for (int r = 0; r < kRows; ++r) acc += Z2[r * kLd + t];
        gb2[t] = acc;
    }
    __syncthreads();
    // dz1 = (W2 dz2) silu'(z1), in place of z1
    for (int u = 0; u < kNH; ++u) {
        float acc = 0.f;
        for (int v = 0; v < kNH; ++v) acc = fmaf(W2[u * kNH + v], Z2[t * kLd + v], acc);
        Z1[t * kLd + u] = acc * dsilu_f(Z1[t * kLd + u]);
    }
    __syncthreads();
    // d W1 [k][u] = sum_r x[r][k] dz1[r][u]; d b1
    for (int i = t; i < kNF * kNH; i += kRows) {
        const int k = i / kNH, u = i % kNH;
        float acc = 0.f;
        for (int r = 0; r < kRows; ++r) acc = fmaf(Xs[r * kLdX + k], Z1[r * kLd + u], acc);
        gW1[i] = acc;
    }
    if (t < kNH) {
        float acc = 0.f;
        for (int r = 0; r < kRows; ++r) acc += Z1[r * kLd + t];
        gb1[t] = acc;
    }
    // sum of squared residuals
    float sq = res * res;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(FULL, sq, o);
    __shared__ float wsum[kRows / 32];
    if ((t & 31) == 0) wsum[t >> 5] = sq;
    __syncthreads();
    if (t == 0) {
        float tot = 0.f;
        for (int k = 0; k < kRows / 32; ++k) tot += wsum[k];
        partial_loss[blockIdx.x] = tot;
    }
}

// Sum the per-CTA gradients in a fixed order; optionally take an Adam step.
// ------------------------------------------------ training on tensor cores
//
// The same gradient as grad_kernel with every matrix product on BF16
// mma.sync.m16n8k16 tiles (FP32 accumulation) and the element-wise work in
// FP32, 128 rows per CTA of four warps (two 16-row tiles each):
//   forward   z1 = bf(X) bf(W1) + b1,  h1 = silu(z1),
//             z2 = bf(h1) bf(W2) + b2, h2 = silu(z2),  e = h2 . W3 + b3   (FP32),
//   backward  g = 2 (e - y) scale,  dW3 = sum g h2,  db3 = sum g,
//             dz2 = g W3 silu'(z2),  db2 = sum dz2,  dW2 = bf(h1)^T bf(dz2),
//             dz1 = (bf(dz2) bf(W2)^T) silu'(z1), db1 = sum dz1, dW1 = bf(X)^T bf(dz1),
// with bf the rounding to bfloat16 (nearest, ties to even) and FP32 master
// parameters.  The per-row tiles of the forward and backward passes stay in
// registers (a C tile of one layer is the A fragment of the next, as in the
// sampler's network); the weight gradients contract over the CTA's rows, so
// bf(X), bf(h1), bf(dz2), bf(dz1) also go to shared memory transposed
// (unit-major), where each A and B fragment pair is one 32-bit word.
constexpr int kTcWarps = 4;
constexpr int kTcRows = 32 * kTcWarps;
constexpr int kTcLd = kTcRows + 8;   // row stride (bf16) of the transposed tiles

struct TcSmem {
    __nv_bfloat16 w1u[kNH][kNF];       // W1 unit-major: [u][k]
    __nv_bfloat16 w2u[kNH][kNH];       // W2 unit-major: [v][u] (forward B)
    __nv_bfloat16 w2r[kNH][kNH];       // W2 as stored: [u][v] (backward B)
    float w3[kNH], b1[kNH], b2[kNH];
    float b3, pad[3];
    __nv_bfloat16 xt[kNF][kTcLd];      // bf(X)^T
    __nv_bfloat16 h1t[kNH][kTcLd];     // bf(h1)^T
    __nv_bfloat16 d2t[kNH][kTcLd];     // bf(dz2)^T
    __nv_bfloat16 d1t[kNH][kTcLd];     // bf(dz1)^T
    float red[kTcWarps][3][kNH];       // per-warp sums over rows: dW3, db2, db1
    float red_s[kTcWarps][2];          // per-warp db3, squared residuals
};

__device__ __forceinline__ uint32_t lds_u32(const __nv_bfloat16* p) {
    return *reinterpret_cast<const uint32_t*>(p);
}

// Sum over the 8 lane groups (g) of a warp: every lane ends with the total of
// its t.
__device__ __forceinline__ float sum_over_g(float v) {
    v += __shfl_xor_sync(FULL, v, 4);
    v += __shfl_xor_sync(FULL, v, 8);
    v += __shfl_xor_sync(FULL, v, 16);
    return v;
}

__global__ void __launch_bounds__(kTcRows) grad_tc_kernel(const float* theta, const float* X, const float* yv,
                                                          const int* idx, int n, float scale, float* partial,
                                                          float* partial_loss) {
    extern __shared__ __align__(16) unsigned char tc_raw[];
    TcSmem& sm = *reinterpret_cast<TcSmem*>(tc_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    const float* W1 = theta;
    const float* B1 = W1 + kNF * kNH;
    const float* W2 = B1 + kNH;
    const float* B2 = W2 + kNH * kNH;
    const float* W3 = B2 + kNH;
    for (int i = tid; i < kNH * kNH; i += kTcRows) {
        const int u = i / kNH, v = i % kNH;   // W2[u][v]
        const __nv_bfloat16 w = __float2bfloat16_rn(W2[i]);
        sm.w2r[u][v] = w;
        sm.w2u[v][u] = w;
        if (i < kNF * kNH) {
            const int k = i / kNH, uu = i % kNH;   // W1[k][uu]
            sm.w1u[uu][k] = __float2bfloat16_rn(W1[i]);
        }
        if (i < kNH) {
            sm.w3[i] = W3[i];
            sm.b1[i] = B1[i];
            sm.b2[i] = B2[i];
        }
    }
    if (tid == 0) sm.b3 = W3[kNH];
    // layer-1 A fragments: this warp's rows 32 warp + 16 mt + (g, g + 8)
    const int row0 = blockIdx.x * kTcRows + warp * 32;
    uint32_t ax[2][4];
    int src[2][2];
    bool act[2][2];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int row = row0 + 16 * mt + g + 8 * h;
            act[mt][h] = row < n;
            src[mt][h] = act[mt][h] ? (idx ? idx[row] : row) : 0;
            float2 lo = make_float2(0.f, 0.f), hi = make_float2(0.f, 0.f);
            if (act[mt][h]) {
                const float* xr = X + size_t(src[mt][h]) * kNF;
                lo = make_float2(xr[2 * t], xr[2 * t + 1]);
                hi = make_float2(xr[2 * t + 8], xr[2 * t + 9]);
            }
            ax[mt][h] = pack_bf16(lo.x, lo.y);        // A regs 0 (row g) and 1 (row g + 8)
            ax[mt][2 + h] = pack_bf16(hi.x, hi.y);    // A regs 2 and 3
            const int r = warp * 32 + 16 * mt + g + 8 * h;   // row within the CTA
            const __nv_bfloat162 l2 = *reinterpret_cast<const __nv_bfloat162*>(&ax[mt][h]);
            const __nv_bfloat162 h2 = *reinterpret_cast<const __nv_bfloat162*>(&ax[mt][2 + h]);
            sm.xt[2 * t][r] = l2.x;
            sm.xt[2 * t + 1][r] = l2.y;
            sm.xt[2 * t + 8][r] = h2.x;
            sm.xt[2 * t + 9][r] = h2.y;
        }
    }
    __syncthreads();   // the weights in shared memory
    // forward, layer 1: z1 (kept for silu'), bf(h1) as layer-2 A fragments and transposed
    float z1[2][8][4];
    uint32_t ah[2][4][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int u = 8 * j + 2 * t;
            z1[mt][j][0] = z1[mt][j][2] = sm.b1[u];
            z1[mt][j][1] = z1[mt][j][3] = sm.b1[u + 1];
            const uint32_t b[2] = {lds_u32(&sm.w1u[8 * j + g][2 * t]), lds_u32(&sm.w1u[8 * j + g][2 * t + 8])};
            mma_bf16(z1[mt][j], ax[mt], b);
        }
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
            for (int q = 0; q < 2; ++q) {            // tiles 2kk (A regs 0, 1) and 2kk + 1 (A regs 2, 3)
                const float* c = z1[mt][2 * kk + q];
                ah[mt][kk][2 * q] = pack_bf16(silu_f(c[0]), silu_f(c[1]));
                ah[mt][kk][2 * q + 1] = pack_bf16(silu_f(c[2]), silu_f(c[3]));
            }
        }
        // A regs are (row g, k lo), (row g + 8, k lo), (row g, k hi), (row g + 8, k hi)
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const int rg = warp * 32 + 16 * mt + g;
            const int u = 16 * kk + 2 * t;
            const __nv_bfloat162 a0 = *reinterpret_cast<const __nv_bfloat162*>(&ah[mt][kk][0]);
            const __nv_bfloat162 a1 = *reinterpret_cast<const __nv_bfloat162*>(&ah[mt][kk][1]);
            const __nv_bfloat162 a2 = *reinterpret_cast<const __nv_bfloat162*>(&ah[mt][kk][2]);
            const __nv_bfloat162 a3 = *reinterpret_cast<const __nv_bfloat162*>(&ah[mt][kk][3]);
            sm.h1t[u][rg] = a0.x;     sm.h1t[u + 1][rg] = a0.y;
            sm.h1t[u][rg + 8] = a1.x; sm.h1t[u + 1][rg + 8] = a1.y;
            sm.h1t[u + 8][rg] = a2.x; sm.h1t[u + 9][rg] = a2.y;
            sm.h1t[u + 8][rg + 8] = a3.x; sm.h1t[u + 9][rg + 8] = a3.y;
        }
    }
    // forward, layer 2 and the output
    float z2[2][8][4];
    float e[2][2];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        float o0 = 0.f, o1 = 0.f;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int v = 8 * j + 2 * t;
            z2[mt][j][0] = z2[mt][j][2] = sm.b2[v];
            z2[mt][j][1] = z2[mt][j][3] = sm.b2[v + 1];
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const uint32_t b[2] = {lds_u32(&sm.w2u[8 * j + g][16 * kk + 2 * t]),
                                       lds_u32(&sm.w2u[8 * j + g][16 * kk + 2 * t + 8])};
                mma_bf16(z2[mt][j], ah[mt][kk], b);
            }
            o0 = fmaf(silu_f(z2[mt][j][0]), sm.w3[v], fmaf(silu_f(z2[mt][j][1]), sm.w3[v + 1], o0));
            o1 = fmaf(silu_f(z2[mt][j][2]), sm.w3[v], fmaf(silu_f(z2[mt][j][3]), sm.w3[v + 1], o1));
        }
        // the four lanes of a group hold the row's partial dot products
        o0 += __shfl_xor_sync(FULL, o0, 1);
        o0 += __shfl_xor_sync(FULL, o0, 2);
        o1 += __shfl_xor_sync(FULL, o1, 1);
        o1 += __shfl_xor_sync(FULL, o1, 2);
        e[mt][0] = o0 + sm.b3;
        e[mt][1] = o1 + sm.b3;
    }
    // residuals and d loss / d e
    float ge[2][2], sq = 0.f, gsum = 0.f;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float res = act[mt][h] ? e[mt][h] - yv[src[mt][h]] : 0.f;
            ge[mt][h] = 2.0f * res * scale;
            if (t == 0) {
                sq = fmaf(res, res, sq);
                gsum += ge[mt][h];
            }
        }
    // dW3, db2 partials and dz2 (in place of z2), bf(dz2) as A fragments and transposed
    uint32_t ad[2][4][4];
    float dw3[8][2], db2[8][2];
#pragma unroll
    for (int j = 0; j < 8; ++j) dw3[j][0] = dw3[j][1] = db2[j][0] = db2[j][1] = 0.f;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int v = 8 * j + 2 * t;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float zz = z2[mt][j][c];
                const float gr = ge[mt][c >> 1];
                dw3[j][c & 1] = fmaf(gr, silu_f(zz), dw3[j][c & 1]);
                const float d = gr * sm.w3[v + (c & 1)] * dsilu_f(zz);
                z2[mt][j][c] = d;
                db2[j][c & 1] += d;
            }
        }
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const float* c = z2[mt][2 * kk + q];
                ad[mt][kk][2 * q] = pack_bf16(c[0], c[1]);
                ad[mt][kk][2 * q + 1] = pack_bf16(c[2], c[3]);
            }
            const int rg = warp * 32 + 16 * mt + g;
            const int v = 16 * kk + 2 * t;
            const __nv_bfloat162 a0 = *reinterpret_cast<const __nv_bfloat162*>(&ad[mt][kk][0]);
            const __nv_bfloat162 a1 = *reinterpret_cast<const __nv_bfloat162*>(&ad[mt][kk][1]);
            const __nv_bfloat162 a2 = *reinterpret_cast<const __nv_bfloat162*>(&ad[mt][kk][2]);
            const __nv_bfloat162 a3 = *reinterpret_cast<const __nv_bfloat162*>(&ad[mt][kk][3]);
            sm.d2t[v][rg] = a0.x;     sm.d2t[v + 1][rg] = a0.y;
            sm.d2t[v][rg + 8] = a1.x; sm.d2t[v + 1][rg + 8] = a1.y;
            sm.d2t[v + 8][rg] = a2.x; sm.d2t[v + 9][rg] = a2.y;
            sm.d2t[v + 8][rg + 8] = a3.x; sm.d2t[v + 9][rg + 8] = a3.y;
        }
    }
    // backward through layer 2: dh1 = bf(dz2) bf(W2)^T, dz1 = dh1 silu'(z1)
    float db1[8][2];
#pragma unroll
    for (int j = 0; j < 8; ++j) db1[j][0] = db1[j][1] = 0.f;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const uint32_t b[2] = {lds_u32(&sm.w2r[8 * j + g][16 * kk + 2 * t]),
                                       lds_u32(&sm.w2r[8 * j + g][16 * kk + 2 * t + 8])};
                mma_bf16(c, ad[mt][kk], b);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float d = c[q] * dsilu_f(z1[mt][j][q]);
                z1[mt][j][q] = d;
                db1[j][q & 1] += d;
            }
        }
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            uint32_t r[4];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const float* c = z1[mt][2 * kk + q];
                r[2 * q] = pack_bf16(c[0], c[1]);
                r[2 * q + 1] = pack_bf16(c[2], c[3]);
            }
            const int rg = warp * 32 + 16 * mt + g;
            const int u = 16 * kk + 2 * t;
            const __nv_bfloat162 a0 = *reinterpret_cast<const __nv_bfloat162*>(&r[0]);
            const __nv_bfloat162 a1 = *reinterpret_cast<const __nv_bfloat162*>(&r[1]);
            const __nv_bfloat162 a2 = *reinterpret_cast<const __nv_bfloat162*>(&r[2]);
            const __nv_bfloat162 a3 = *reinterpret_cast<const __nv_bfloat162*>(&r[3]);
            sm.d1t[u][rg] = a0.x;     sm.d1t[u + 1][rg] = a0.y;
            sm.d1t[u][rg + 8] = a1.x; sm.d1t[u + 1][rg + 8] = a1.y;
            sm.d1t[u + 8][rg] = a2.x; sm.d1t[u + 9][rg] = a2.y;
            sm.d1t[u + 8][rg + 8] = a3.x; sm.d1t[u + 9][rg + 8] = a3.y;
        }
    }
    // per-warp sums over rows of dW3, db2, db1, db3 and the squared residuals
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const float a = sum_over_g(dw3[j][q]), b = sum_over_g(db2[j][q]), c = sum_over_g(db1[j][q]);
            if (g == 0) {
                sm.red[warp][0][8 * j + 2 * t + q] = a;
                sm.red[warp][1][8 * j + 2 * t + q] = b;
                sm.red[warp][2][8 * j + 2 * t + q] = c;
            }
        }
    sq += __shfl_xor_sync(FULL, sq, 4);
    sq += __shfl_xor_sync(FULL, sq, 8);
    sq += __shfl_xor_sync(FULL, sq, 16);
    gsum += __shfl_xor_sync(FULL, gsum, 4);
    gsum += __shfl_xor_sync(FULL, gsum, 8);
    gsum += __shfl_xor_sync(FULL, gsum, 16);
    if (lane == 0) {
        sm.red_s[warp][0] = gsum;
        sm.red_s[warp][1] = sq;
    }
    __syncthreads();   // every warp's transposed tiles and partial sums
    float* G = partial + size_t(blockIdx.x) * kNParams;
    float* gW1 = G;
    float* gb1 = gW1 + kNF * kNH;
    float* gW2 = gb1 + kNH;
    float* gb2 = gW2 + kNH * kNH;
    float* gW3 = gb2 + kNH;
    // dW2 = bf(h1)^T bf(dz2) over the CTA's rows: 4 x 8 tiles of 16 x 8, two per warp and pass
#pragma unroll 1
    for (int tile = warp; tile < 32; tile += kTcWarps) {
        const int u0 = 16 * (tile >> 3), v0 = 8 * (tile & 7);
        float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kk = 0; kk < kTcRows / 16; ++kk) {
            const int r = 16 * kk + 2 * t;
            const uint32_t a[4] = {lds_u32(&sm.h1t[u0 + g][r]), lds_u32(&sm.h1t[u0 + g + 8][r]),
                                   lds_u32(&sm.h1t[u0 + g][r + 8]), lds_u32(&sm.h1t[u0 + g + 8][r + 8])};
            const uint32_t b[2] = {lds_u32(&sm.d2t[v0 + g][r]), lds_u32(&sm.d2t[v0 + g][r + 8])};
            mma_bf16(c, a, b);
        }
        gW2[(u0 + g) * kNH + v0 + 2 * t] = c[0];
        gW2[(u0 + g) * kNH + v0 + 2 * t + 1] = c[1];
        gW2[(u0 + g + 8) * kNH + v0 + 2 * t] = c[2];
        gW2[(u0 + g + 8) * kNH + v0 + 2 * t + 1] = c[3];
    }
    // dW1 = bf(X)^T bf(dz1): 1 x 8 tiles
#pragma unroll 1
    for (int tile = warp; tile < 8; tile += kTcWarps) {
        const int u0 = 8 * tile;
        float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kk = 0; kk < kTcRows / 16; ++kk) {
            const int r = 16 * kk + 2 * t;
            const uint32_t a[4] = {lds_u32(&sm.xt[g][r]), lds_u32(&sm.xt[g + 8][r]), lds_u32(&sm.xt[g][r + 8]),
                                   lds_u32(&sm.xt[g + 8][r + 8])};
            const uint32_t b[2] = {lds_u32(&sm.d1t[u0 + g][r]), lds_u32(&sm.d1t[u0 + g][r + 8])};
            mma_bf16(c, a, b);
        }
        gW1[g * kNH + u0 + 2 * t] = c[0];
        gW1[g * kNH + u0 + 2 * t + 1] = c[1];
        gW1[(g + 8) * kNH + u0 + 2 * t] = c[2];
        gW1[(g + 8) * kNH + u0 + 2 * t + 1] = c[3];
    }
    // the row sums, added over the warps in a fixed order
    if (tid < kNH) {
        float a = 0.f, b = 0.f, c = 0.f;
        for (int w = 0; w < kTcWarps; ++w) {
            a += sm.red[w][0][tid];
            b += sm.red[w][1][tid];
            c += sm.red[w][2][tid];
        }
        gW3[tid] = a;
        gb2[tid] = b;
        gb1[tid] = c;
    } else if (tid == kNH) {
        float a = 0.f, b = 0.f;
        for (int w = 0; w < kTcWarps; ++w) {
            a += sm.red_s[w][0];
            b += sm.red_s[w][1];
        }
        gW3[kNH] = a;                 // db3
        partial_loss[blockIdx.x] = b;
    }
}

__global__ void reduce_adam_kernel(const float* partial, const float* partial_loss, int nblk, float* grad,
                                   float* loss, float* theta, float* m, float* v, int adam_t, float lr) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        float tot = 0.f;
        for (int b = 0; b < nblk; ++b) tot += partial_loss[b];
        *loss = tot;
    }
    if (i >= kNParams) return;
    float g = 0.f;
    for (int b = 0; b < nblk; ++b) g += partial[size_t(b) * kNParams + i];
    if (grad) grad[i] = g;
    if (adam_t > 0) {
        const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
        const float mi = b1 * m[i] + (1.f - b1) * g;
        const float vi = b2 * v[i] + (1.f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        const float mh = mi / (1.f - powf(b1, (float)adam_t));
        const float vh = vi / (1.f - powf(b2, (float)adam_t));
        theta[i] -= lr * mh / (sqrtf(vh) + eps);
    }
}

// Seeded initial parameters: every weight normal with standard deviation
// scale / sqrt(fan-in) (Box-Muller on Philox stream 7, counter (i, 0, 0, 7)),
// every bias zero.
__global__ void init_kernel(float* theta, float scale, uint32_t k0, uint32_t k1) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kNParams) return;
    const int o1 = kNF * kNH, o2 = o1 + kNH, o3 = o2 + kNH * kNH, o4 = o3 + kNH, o5 = o4 + kNH;
    float fan = 0.f;
    if (i < o1) fan = (float)kNF;
    else if (i >= o2 && i < o3) fan = (float)kNH;
    else if (i >= o4 && i < o5) fan = (float)kNH;
    if (fan == 0.f) {
        theta[i] = 0.f;
        return;
    }
    const U4 u = philox(uint32_t(i), 0u, 0u, 7u, k0, k1);
    const float u1 = ((float)(u.x >> 8) + 0.5f) * (1.0f / 16777216.0f);
    const float u2 = (float)(u.y >> 8) * (1.0f / 16777216.0f);
    const float z = sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
    theta[i] = z * scale * rsqrtf(fan);
}

// Random row indices of a training step (Philox stream 6).
__global__ void batch_index_kernel(int* idx, int batch, int count, uint32_t step, uint32_t k0, uint32_t k1) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= batch) return;
    const U4 u = philox(uint32_t(i), step, 0u, 6u, k0, k1);
    idx[i] = (int)(((unsigned long long)u.x * (unsigned)count) >> 32);
}

size_t grad_smem() {
    return (size_t(((kNParams + 3) & ~3)) + kRows * kLdX + 3 * kRows * kLd + kRows) * sizeof(float);
}

}  // namespace

cudaError_t surrogate_pack(const float* theta, const SurrogateStore& st, cudaStream_t s) {
    pack_kernel<<<16, 256, 0, s>>>(theta, st.w1, st.b1, st.w2, st.b2, st.w3, st.b3);
    return cudaGetLastError();
}

cudaError_t surrogate_eval(const SweepParams& P, int w, int Q, const float4* q, float* e_out, float* f_out,
                           cudaStream_t s) {
    if (Q <= 0) return cudaSuccess;
    eval_kernel<<<(Q + 7) / 8, 128, 0, s>>>(P, w, Q, q, e_out, f_out);
    return cudaGetLastError();
}

cudaError_t surrogate_harvest(const SweepParams& P, int parts, int probes, float clip, uint32_t round, float* X,
                              float* y, int base, int cap, cudaStream_t s) {
    const long long rows = (long long)P.S * (parts + probes);
    if (rows <= 0 || cap <= 0) return cudaSuccess;
    harvest_kernel<<<(unsigned)((rows + 3) / 4), 128, 0, s>>>(P, parts, probes, clip, round, X, y, base, cap);
    return cudaGetLastError();
}

size_t surrogate_partial_floats(int n) { return size_t((n + kRows - 1) / kRows) * (kNParams + 1); }

cudaError_t surrogate_step(const float* theta_in, const float* X, const float* y, const int* idx, int n,
                           float* partial, float* grad, float* loss, float* theta, float* m, float* v, int adam_t,
                           float lr, bool tensor_cores, cudaStream_t s) {
    static_assert(kTcRows == kRows, "both gradient kernels take 128 rows per CTA");
    const int nblk = (n + kRows - 1) / kRows;
    float* partial_loss = partial + size_t(nblk) * kNParams;
    cudaError_t err;
    if (tensor_cores) {
        const size_t smem = sizeof(TcSmem);
        err = cudaFuncSetAttribute(grad_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
        grad_tc_kernel<<<nblk, kTcRows, smem, s>>>(theta_in, X, y, idx, n, 1.0f / (float)n, partial, partial_loss);
    } else {
        const size_t smem = grad_smem();
        err = cudaFuncSetAttribute(grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
        grad_kernel<<<nblk, kRows, smem, s>>>(theta_in, X, y, idx, n, 1.0f / (float)n, partial, partial_loss);
    }
    reduce_adam_kernel<<<(kNParams + 255) / 256, 256, 0, s>>>(partial, partial_loss, nblk, grad, loss, theta, m, v,
                                                              adam_t, lr);
    return cudaGetLastError();
}

cudaError_t surrogate_init(float* theta, float scale, uint32_t k0, uint32_t k1, cudaStream_t s) {
    init_kernel<<<(kNParams + 255) / 256, 256, 0, s>>>(theta, scale, k0, k1);
    return cudaGetLastError();
}

cudaError_t surrogate_batch_index(int* idx, int batch, int count, uint32_t step, uint32_t k0, uint32_t k1,
                                  cudaStream_t s) {
    batch_index_kernel<<<(batch + 255) / 256, 256, 0, s>>>(idx, batch, count, step, k0, k1);
    return cudaGetLastError();
}

}  // namespace regc
