// surrogate.cuh -- device pieces of the learned surrogate (delayed acceptance).
//
// The paper has no surrogate.  The network predicts the interaction energy
// e~(r) of a mobile particle at r from 16 Gaussian radial features of its
// neighbours within rc:
//   G_k = sum_j eps_0j exp(-eta (r_j - c_k)^2) (cos(pi r_j / rc) + 1) / 2,
//   c_k = 0.8 + 1.7 k / 15 (k = 0..15), eta = 1 / (2 (1.7/15)^2),
// followed by 16 -> 64 -> 64 -> 1 with SiLU hidden layers.
//
// Parameters: FP32 master vector of 5313 values (W1 [16][64], b1 [64],
// W2 [64][64], b2 [64], W3 [64], b3), and a BF16 inference copy packed so that
// every hidden unit's weights are contiguous (unit-major).  Inference runs the
// layers on tensor cores: every layer's inputs (the features, then the hidden
// activations) and weights are BF16, accumulation and biases FP32.
#pragma once

#include <cuda_bf16.h>

#include "regc_internal.cuh"

namespace regc {

constexpr int kNF = 16, kNH = 64;
constexpr int kNParams = kNF * kNH + kNH + kNH * kNH + kNH + kNH + 1;   // 5313
constexpr float kFeatC0 = 0.8f, kFeatDc = 1.7f / 15.0f;
// exp(-eta (r - c)^2) = exp2(-eta log2(e) (r - c)^2)
constexpr float kFeatEta2 = 1.4426950408889634f / (2.0f * (1.7f / 15.0f) * (1.7f / 15.0f));

// The 16 Gaussians of one neighbour from six exponentials.  With eta = 1 /
// (2 dc^2) and u = (r - c_a) / dc at an anchor centre a, the Gaussian there is
// exp(-u^2 / 2) and neighbouring centres follow by ratios:
//   g_{k+1} = g_k exp(u_k - 1/2),   g_{k-1} = g_k exp(-u_k - 1/2),
// with u_{k+1} = u_k - 1, so each ratio is the previous one times e^-1.
// Anchors 4 and 11 keep every chain within four products; a Gaussian that is
// reached through many products or from a tiny anchor value is itself tiny
// (far from r), so its error stays far below the feature tolerance.
constexpr float kLog2E = 1.4426950408889634f;
constexpr float kInvE = 0.36787944117144233f;   // e^-1

template <int A, int K0, int K1>
__device__ __forceinline__ void gaussians_from(float (&g)[kNF], float r) {
    const float u = (r - (kFeatC0 + kFeatDc * A)) * (1.0f / kFeatDc);
    g[A] = exp2f(-0.5f * kLog2E * u * u);
    float up = exp2f(kLog2E * (u - 0.5f)), dn = exp2f(-kLog2E * (u + 0.5f));
#pragma unroll
    for (int k = A + 1; k <= K1; ++k) {
        g[k] = g[k - 1] * up;
        up *= kInvE;
    }
#pragma unroll
    for (int k = A - 1; k >= K0; --k) {
        g[k] = g[k + 1] * dn;
        dn *= kInvE;
    }
}

// Add one neighbour at squared distance r2 < rc^2 with weight w to F.
__device__ __forceinline__ void add_features(float (&F)[kNF], float r2, float w, float rc) {
    const float r = sqrtf(r2);
    const float fc = 0.5f * (__cosf(3.14159265358979f * r / rc) + 1.0f) * w;
    float g[kNF];
    gaussians_from<4, 0, 7>(g, r);
    gaussians_from<11, 8, 15>(g, r);
#pragma unroll
    for (int k = 0; k < kNF; ++k) F[k] = fmaf(fc, g[k], F[k]);
}

// Warp sum of 16 values per lane by recursive halving; afterwards lane l holds
// the sum of value (l >> 1) & 15 (lanes l and l ^ 1 hold the same one).
__device__ __forceinline__ float warp_reduce16(float (&F)[kNF], int lane) {
#pragma unroll
    for (int half = 8, off = 16; half >= 1; half >>= 1, off >>= 1) {
        const bool upper = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const float send = upper ? F[i] : F[i + half];
            const float keep = upper ? F[i + half] : F[i];
            F[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
    return F[0] + __shfl_xor_sync(0xffffffffu, F[0], 1);
}

__device__ __forceinline__ float silu_f(float x) { return __fdividef(x, 1.0f + __expf(-x)); }

// ------------------------------------------------ the network on tensor cores
//
// Every layer is BF16 x BF16 with FP32 accumulation on mma.sync.m16n8k16
// tiles: A (16 x 16, row-major) holds layer inputs, one row per trial
// position; B (16 x 8) holds 16 inputs x 8 units of the layer's weights; C
// (16 x 8, FP32) the pre-activations.  Only rows 0 and 1 of A are positions
// (a move's new and old position); the other rows stay zero.  In the PTX
// fragment layouts lane l, with g = l / 4 and t = l % 4, holds
//   A: rows g and g + 8, columns 2t, 2t + 1, 2t + 8, 2t + 9,
//   B: column (unit) g, rows (inputs) 2t, 2t + 1, 2t + 8, 2t + 9,
//   C: rows g and g + 8, columns 2t, 2t + 1,
// so a layer's C tiles for units 16 kk .. 16 kk + 15 are, after the bias,
// SiLU and rounding to BF16, the next layer's A fragment for inputs
// 16 kk .. 16 kk + 15 without leaving the registers.  The unit-major BF16
// inference copy puts each B fragment pair in one 32-bit word.

// This lane's B fragments of the three layers and the biases of its columns,
// loaded once per launch.
struct NetFrag {
    uint32_t w1[8][2];       // layer 1, units 8j .. 8j + 7
    uint32_t w2[8][4][2];    // layer 2, units 8j .. 8j + 7, inputs 16kk .. 16kk + 15
    uint32_t w3[4][2];       // output unit (column 0 of the tile), inputs 16kk ..
    const float2* b1;        // biases, read where used (L1-resident; registers are scarce)
    const float2* b2;
    const float* b3;
};

__device__ __forceinline__ uint32_t ld_bf16x2(const __nv_bfloat16* p) {
    return __ldg(reinterpret_cast<const unsigned int*>(p));
}

__device__ __forceinline__ void load_net(const SurrogateDev& net, int lane, NetFrag& F) {
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int u = 8 * j + g;
        F.w1[j][0] = ld_bf16x2(net.w1 + u * kNF + 2 * t);
        F.w1[j][1] = ld_bf16x2(net.w1 + u * kNF + 2 * t + 8);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            F.w2[j][kk][0] = ld_bf16x2(net.w2 + u * kNH + 16 * kk + 2 * t);
            F.w2[j][kk][1] = ld_bf16x2(net.w2 + u * kNH + 16 * kk + 2 * t + 8);
        }
    }
    F.b1 = reinterpret_cast<const float2*>(net.b1) + t;   // + 4 j: units 8j + 2t, 8j + 2t + 1
    F.b2 = reinterpret_cast<const float2*>(net.b2) + t;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        F.w3[kk][0] = g == 0 ? ld_bf16x2(net.w3 + 16 * kk + 2 * t) : 0u;
        F.w3[kk][1] = g == 0 ? ld_bf16x2(net.w3 + 16 * kk + 2 * t + 8) : 0u;
    }
    F.b3 = net.b3;
}

// Two binary32 values rounded to BF16 (nearest, ties to even), lo in the low half.
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

// c += A B on one m16n8k16 tile, BF16 operands, FP32 accumulation.
__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Layer-1 A fragment from the features of two positions held as warp_reduce16
// leaves them (feature k of position p in lanes 2k and 2k + 1 of r_p): lanes
// 0..3 take position 0's, lanes 4..7 position 1's, the rest zero.
__device__ __forceinline__ void features_to_frag(float r0, float r1, int lane, uint32_t (&a)[4]) {
    const int g = lane >> 2, t = lane & 3;
    const float x0 = __shfl_sync(0xffffffffu, r0, 4 * t), x1 = __shfl_sync(0xffffffffu, r0, 4 * t + 2);
    const float x2 = __shfl_sync(0xffffffffu, r0, 4 * t + 16), x3 = __shfl_sync(0xffffffffu, r0, 4 * t + 18);
    const float y0 = __shfl_sync(0xffffffffu, r1, 4 * t), y1 = __shfl_sync(0xffffffffu, r1, 4 * t + 2);
    const float y2 = __shfl_sync(0xffffffffu, r1, 4 * t + 16), y3 = __shfl_sync(0xffffffffu, r1, 4 * t + 18);
    a[0] = g == 0 ? pack_bf16(x0, x1) : (g == 1 ? pack_bf16(y0, y1) : 0u);
    a[2] = g == 0 ? pack_bf16(x2, x3) : (g == 1 ? pack_bf16(y2, y3) : 0u);
    a[1] = a[3] = 0u;   // rows 8..15
}

// A fragment for inputs 16kk .. 16kk + 15 of the next layer from the C tiles
// 2kk, 2kk + 1 of this one: bias, SiLU, BF16 (rows 8..15 stay zero).
__device__ __forceinline__ void silu_to_frag(const float (&c0)[4], const float (&c1)[4], uint32_t (&a)[4]) {
    a[0] = pack_bf16(silu_f(c0[0]), silu_f(c0[1]));
    a[2] = pack_bf16(silu_f(c1[0]), silu_f(c1[1]));
    a[1] = a[3] = 0u;
}

// e~ of the positions in rows 0 and 1 of the layer-1 fragment a: returns
// row 0's in every lane and stores row 1's in *e1.
__device__ __forceinline__ float net_mma(const NetFrag& W, const uint32_t (&a)[4], float* e1) {
    float c[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float2 b = __ldg(W.b1 + 4 * j);
        c[j][0] = b.x;
        c[j][1] = b.y;
        c[j][2] = c[j][3] = 0.f;
        mma_bf16(c[j], a, W.w1[j]);
    }
    uint32_t h[4][4];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) silu_to_frag(c[2 * kk], c[2 * kk + 1], h[kk]);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float2 b = __ldg(W.b2 + 4 * j);
        c[j][0] = b.x;
        c[j][1] = b.y;
        c[j][2] = c[j][3] = 0.f;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) mma_bf16(c[j], h[kk], W.w2[j][kk]);
    }
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) silu_to_frag(c[2 * kk], c[2 * kk + 1], h[kk]);
    float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) mma_bf16(o, h[kk], W.w3[kk]);
    // column 0 of row g sits in lane 4 g (t = 0)
    const float b3 = __ldg(W.b3);
    *e1 = __shfl_sync(0xffffffffu, o[0], 4) + b3;
    return __shfl_sync(0xffffffffu, o[0], 0) + b3;
}

}  // namespace regc
