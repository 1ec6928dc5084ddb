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
// every hidden unit's weights are contiguous (unit-major).
#pragma once

#include <cuda_bf16.h>

#include "regc_internal.cuh"

namespace regc {

constexpr int kNF = 16, kNH = 64;
constexpr int kNParams = kNF * kNH + kNH + kNH * kNH + kNH + kNH + 1;   // 5313
constexpr float kFeatC0 = 0.8f, kFeatDc = 1.7f / 15.0f;
// exp(-eta (r - c)^2) = exp2(-eta log2(e) (r - c)^2)
constexpr float kFeatEta2 = 1.4426950408889634f / (2.0f * (1.7f / 15.0f) * (1.7f / 15.0f));

// Add one neighbour at squared distance r2 < rc^2 with weight w to F.
__device__ __forceinline__ void add_features(float (&F)[kNF], float r2, float w, float rc) {
    const float r = sqrtf(r2);
    const float fc = 0.5f * (__cosf(3.14159265358979f * r / rc) + 1.0f) * w;
#pragma unroll
    for (int k = 0; k < kNF; ++k) {
        const float d = r - (kFeatC0 + kFeatDc * k);
        F[k] = fmaf(fc, exp2f(-kFeatEta2 * d * d), F[k]);
    }
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

// Network output for the features held as in warp_reduce16 (lane l holds
// G[(l >> 1) & 15]).  scratch: 64 floats of shared memory for this warp.
__device__ __forceinline__ float mlp_forward(const SurrogateDev& net, float g_lane, float* scratch, int lane) {
    if ((lane & 1) == 0) scratch[lane >> 1] = g_lane;
    __syncwarp();
    float G[kNF];
#pragma unroll
    for (int k = 0; k < kNF; k += 4) {
        const float4 v = *reinterpret_cast<const float4*>(scratch + k);
        G[k] = v.x; G[k + 1] = v.y; G[k + 2] = v.z; G[k + 3] = v.w;
    }
    __syncwarp();
    float h[2];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const int u = lane + 32 * t;
        const __nv_bfloat162* wr = reinterpret_cast<const __nv_bfloat162*>(net.w1 + u * kNF);
        float z = net.b1[u];
#pragma unroll
        for (int k = 0; k < kNF; k += 2) {
            const float2 wf = __bfloat1622float2(wr[k / 2]);
            z = fmaf(wf.x, G[k], z);
            z = fmaf(wf.y, G[k + 1], z);
        }
        h[t] = silu_f(z);
    }
    scratch[lane] = h[0];
    scratch[lane + 32] = h[1];
    __syncwarp();
    float o = 0.0f;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const int v = lane + 32 * t;
        const __nv_bfloat162* wr = reinterpret_cast<const __nv_bfloat162*>(net.w2 + v * kNH);
        float z = net.b2[v];
#pragma unroll 8
        for (int u = 0; u < kNH; u += 4) {
            const float4 hv = *reinterpret_cast<const float4*>(scratch + u);
            const float2 a = __bfloat1622float2(wr[u / 2]);
            const float2 b = __bfloat1622float2(wr[u / 2 + 1]);
            z = fmaf(a.x, hv.x, z);
            z = fmaf(a.y, hv.y, z);
            z = fmaf(b.x, hv.z, z);
            z = fmaf(b.y, hv.w, z);
        }
        o = fmaf(__bfloat162float(net.w3[v]), silu_f(z), o);
    }
    __syncwarp();
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) o += __shfl_xor_sync(0xffffffffu, o, off);
    return o + __ldg(net.b3);
}

}  // namespace regc
