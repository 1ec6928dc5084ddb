// md.cu -- molecular-dynamics segments of every walker (REGCMD), sm_103a.
//
// Sec. II.A.3: the canonical sampling between grand-canonical and exchange
// moves may be done by MD instead of Metropolis displacements; Appendix:
// velocity Verlet with the stochastic velocity rescaling thermostat.  One CTA
// of kMdWarps warps per walker; thread t owns particles t, t + 128, ...
// Per segment:
//   - velocities drawn from the Maxwell-Boltzmann distribution at the
//     walker's kT (particle i: Philox counter (i, seg, w, 8), Box-Muller);
//   - every step: the thermostat of Bussi, Donadio & Parrinello (2007) with
//     time constant tau over all 3N degrees of freedom (normals from counters
//     (k, seg * n_steps + step, w, 9)), then velocity Verlet
//     (v += f dt/2, r += v dt, cells rebuilt, f = F(r), v += f dt/2);
//   - forces from the distinct neighbour cells (nearest image) and the
//     particle's surface column, FP32; per-particle sums in a fixed order, so
//     a segment is reproducible;
//   - x, y periodic (z too in a periodic box), else walls at z_lo and z_hi
//     reflect;
//   - positions and (optionally) kinetic energies back to HBM; the caller
//     recomputes the exact energies.
#include "cells.cuh"
#include "launch.h"

namespace regc {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kMdWarps = 4;
constexpr int kMdThreads = 32 * kMdWarps;

__host__ __device__ inline size_t md_align16(size_t v) { return (v + 15) & ~size_t(15); }

__host__ __device__ inline size_t md_smem_bytes(int nmax, int ncell, int cap) {
    return 3 * md_align16(size_t(nmax) * 16) + md_align16(size_t(ncell) * 2) + md_align16(size_t(ncell) * cap * 2);
}

// Four standard normals from one Philox block (Box-Muller on words 0-1, 2-3;
// uniforms from the top 24 bits, offset by half a step so that none is 0).
__device__ __forceinline__ void normals4(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                         uint32_t k1, float g[4]) {
    const U4 u = philox(c0, c1, c2, c3, k0, k1);
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const float u1 = ((float)(w[2 * h] >> 8) + 0.5f) * (1.0f / 16777216.0f);
        const float u2 = ((float)(w[2 * h + 1] >> 8) + 0.5f) * (1.0f / 16777216.0f);
        const float r = sqrtf(-2.0f * logf(u1));
        g[2 * h] = r * cospif(2.0f * u2);
        g[2 * h + 1] = r * sinpif(2.0f * u2);
    }
}

// Sum of one float per thread over the CTA in a fixed order; every thread
// receives the sum.
__device__ __forceinline__ float cta_sum(float v, float* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    const int warp = threadIdx.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[warp] = v;
    __syncthreads();
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kMdWarps; ++k) s += red[k];
    return s;
}

// The range of distinct cell offsets along one axis of n cells: periodic
// -1..1 while those are distinct cells (0..1 for two cells, 0 for one),
// otherwise the offsets that stay inside the grid.  With nearest-image
// displacements a cell visited twice would count its pairs twice.
__device__ __forceinline__ void axis_range(int c, int n, bool periodic, int& lo, int& hi) {
    if (periodic) {
        lo = n >= 3 ? -1 : 0;
        hi = n >= 2 ? 1 : 0;
    } else {
        lo = c > 0 ? -1 : 0;
        hi = c < n - 1 ? 1 : 0;
    }
}

__device__ __forceinline__ void lj_force_add(const PairTab& t, float r2, float dx, float dy, float dz, float& fx,
                                             float& fy, float& fz) {
    const float inv = __fdividef(1.0f, r2);
    const float s2 = t.sig2 * inv;
    const float s6 = s2 * s2 * s2;
    const float g = 6.0f * t.eps4 * (2.0f * s6 * s6 - s6) * inv;   // 24 eps (2 s^12 - s^6) / r^2
    fx = fmaf(g, dx, fx);
    fy = fmaf(g, dy, fy);
    fz = fmaf(g, dz, fz);
}

// Force on particle i at p.
template <bool CL>
__device__ __forceinline__ float3 md_force(const SweepParams& P, const float4* pos, const uint16_t* cnt,
                                           const uint16_t* slots, int i, float4 p) {
    float fx = 0.f, fy = 0.f, fz = 0.f;
    const bool iA = CL && i < P.n_cluster;
    const Cell3 c = cell3_of(P, p.x, p.y, p.z);
    int xlo, xhi, ylo, yhi, zlo, zhi;
    axis_range(c.x, P.cg.ncx, true, xlo, xhi);
    axis_range(c.y, P.cg.ncy, true, ylo, yhi);
    axis_range(c.z, P.cg.ncz, P.g.periodic_z != 0, zlo, zhi);
    for (int a = zlo; a <= zhi; ++a)
        for (int b = ylo; b <= yhi; ++b)
            for (int d = xlo; d <= xhi; ++d) {
                int cz = c.z + a, cy = c.y + b, cx = c.x + d;   // wrapped into the grid
                if (cz < 0) cz += P.cg.ncz;
                if (cz >= P.cg.ncz) cz -= P.cg.ncz;
                if (cy < 0) cy += P.cg.ncy;
                if (cy >= P.cg.ncy) cy -= P.cg.ncy;
                if (cx < 0) cx += P.cg.ncx;
                if (cx >= P.cg.ncx) cx -= P.cg.ncx;
                const int cell = (cz * P.cg.ncy + cy) * P.cg.ncx + cx;
                const int m = cnt[cell];
                for (int s = 0; s < m; ++s) {
                    const int j = slots[cell * P.cg.cap + s];
                    if (j == i) continue;
                    const float4 q = pos[j];
                    const float dy = min_image_exact(p.y, q.y, P.g.Ly, P.g.hLy);
                    const float dx = cart_dx(P.g, min_image_exact(p.x, q.x, P.g.Lx, P.g.hLx), dy);
                    const float dz = P.g.periodic_z ? min_image_exact(p.z, q.z, P.g.Lz, P.g.hLz) : p.z - q.z;
                    const float r2 = r2_of(dx, dy, dz);
                    if (r2 < P.g.rc2) {
                        const bool jA = CL && j < P.n_cluster;
                        const PairTab& t = CL ? (iA ? (jA ? P.gA : P.gAB) : (jA ? P.gAB : P.gg)) : P.gg;
                        lj_force_add(t, r2, dx, dy, dz, fx, fy, fz);
                    }
                }
            }
    if (near_surface(P, p.z)) {
        const int beg = surface_col(P, p.x, p.y) * P.st.stride;
        for (int k = beg; k < beg + P.st.stride; ++k) {
            const float4 at = __ldg(&P.st.atoms[k]);
            const unsigned bits = __float_as_uint(at.w);
            if (bits & 32u) break;   // padding: the column's images are listed first
            const PairTab& t = (CL && iA) ? P.gsA[bits & 3u] : P.gs[bits & 3u];
            const float sx = (bits & 4u) ? P.g.Lx : 0.f, sy = (bits & 8u) ? P.g.Ly : 0.f;
            const float sz = (bits & 16u) ? P.g.Lz : 0.f;
            const float dy = (p.y - sy) - at.y, dz = (p.z - sz) - at.z;
            const float dx = cart_dx(P.g, (p.x - sx) - at.x, dy);
            const float r2 = r2_of(dx, dy, dz);
            if (r2 < P.g.rc2) lj_force_add(t, r2, dx, dy, dz, fx, fy, fz);
        }
    }
    return make_float3(fx, fy, fz);
}

template <bool CL>
__device__ __forceinline__ void forces_all(const SweepParams& P, const float4* pos, const uint16_t* cnt,
                                           const uint16_t* slots, float4* frc, float4* vel, int N, float half_dt,
                                           bool kick) {
    for (int i = threadIdx.x; i < N; i += kMdThreads) {
        const float3 f = md_force<CL>(P, pos, cnt, slots, i, pos[i]);
        frc[i] = make_float4(f.x, f.y, f.z, 0.f);
        if (kick) {
            float4 v = vel[i];
            v.x = fmaf(half_dt, f.x, v.x);
            v.y = fmaf(half_dt, f.y, v.y);
            v.z = fmaf(half_dt, f.z, v.z);
            vel[i] = v;
        }
    }
}

template <bool CL>
__global__ void __launch_bounds__(kMdThreads) md_kernel(const __grid_constant__ SweepParams P, int n_steps, float dt,
                                                        double c_tau, uint32_t seg, float* kin_out) {
    extern __shared__ __align__(16) char smem[];
    __shared__ float red[kMdWarps];
    __shared__ float alpha_sh;
    const int w = blockIdx.x;
    if (w >= P.S) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float4* pos = reinterpret_cast<float4*>(smem);
    float4* vel = reinterpret_cast<float4*>(smem + md_align16(size_t(P.nmax) * 16));
    float4* frc = reinterpret_cast<float4*>(smem + 2 * md_align16(size_t(P.nmax) * 16));
    uint16_t* cnt = reinterpret_cast<uint16_t*>(smem + 3 * md_align16(size_t(P.nmax) * 16));
    uint16_t* slots = cnt + md_align16(size_t(P.cg.ncell) * 2) / 2;
    const int N = P.n[w];
    const int s = P.state_of_walker[w];
    const float kT = (float)(1.0 / P.beta[s]);
    float4* gpos = P.pos + size_t(w) * P.nmax;

    for (int i = tid; i < N; i += kMdThreads) {
        pos[i] = gpos[i];
        float g[4];
        normals4((uint32_t)i, seg, (uint32_t)w, 8u, P.key0, P.key1, g);
        const float sk = sqrtf(kT);
        vel[i] = make_float4(sk * g[0], sk * g[1], sk * g[2], 0.f);
    }
    __syncthreads();
    if (warp == 0) build_cell_list(P, pos, N, cnt, slots, lane);
    __syncthreads();
    forces_all<CL>(P, pos, cnt, slots, frc, vel, N, 0.5f * dt, false);
    __syncthreads();

    const int nf = 3 * N;
    const double Kt = 0.5 * nf * (double)kT;
    for (int step = 0; step < n_steps && N > 0; ++step) {
        // thermostat: kinetic energy and the normals of this step
        float kp = 0.f, chi = 0.f, r1 = 0.f;
        for (int i = tid; i < N; i += kMdThreads) {
            const float4 v = vel[i];
            kp += 0.5f * (v.x * v.x + v.y * v.y + v.z * v.z);
        }
        const uint32_t gstep = seg * (uint32_t)n_steps + (uint32_t)step;
        for (int k = tid; 4 * k < nf; k += kMdThreads) {
            float g[4];
            normals4((uint32_t)k, gstep, (uint32_t)w, 9u, P.key0, P.key1, g);
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int idx = 4 * k + h;
                if (idx == 0) r1 = g[h];
                else if (idx < nf) chi += g[h] * g[h];
            }
        }
        const float K = cta_sum(kp, red);
        const float CHI = cta_sum(chi, red);
        const float R1 = cta_sum(r1, red);   // only thread 0 contributes
        if (tid == 0) {
            double a = 1.0;
            if (K > 0.f) {
                const double k_new = c_tau * K + (1.0 - c_tau) * Kt * ((double)R1 * R1 + CHI) / nf +
                                     2.0 * R1 * sqrt(c_tau * (1.0 - c_tau) * K * Kt / nf);
                a = sqrt(fmax(k_new, 0.0) / K);
                if (R1 + sqrt(c_tau * nf * K / ((1.0 - c_tau) * Kt)) < 0.0) a = -a;
            }
            alpha_sh = (float)a;
        }
        __syncthreads();
        const float alpha = alpha_sh;
        // half kick, drift, walls
        for (int i = tid; i < N; i += kMdThreads) {
            float4 v = vel[i];
            const float4 f = frc[i];
            v.x = fmaf(0.5f * dt, f.x, alpha * v.x);
            v.y = fmaf(0.5f * dt, f.y, alpha * v.y);
            v.z = fmaf(0.5f * dt, f.z, alpha * v.z);
            float4 p = pos[i];
            p.x = fmaf(dt, fmaf(-P.g.shear, v.y, v.x), p.x);   // u = x - shear y
            p.y = fmaf(dt, v.y, p.y);
            p.z = fmaf(dt, v.z, p.z);
            if (p.x < 0.f) p.x += P.g.Lx;
            if (p.x >= P.g.Lx) p.x -= P.g.Lx;
            if (p.y < 0.f) p.y += P.g.Ly;
            if (p.y >= P.g.Ly) p.y -= P.g.Ly;
            if (P.g.periodic_z) {
                if (p.z < 0.f) p.z += P.g.Lz;
                if (p.z >= P.g.Lz) p.z -= P.g.Lz;
            } else {
                if (p.z < P.g.z_lo) { p.z = 2.0f * P.g.z_lo - p.z; v.z = -v.z; }
                if (p.z > P.g.z_hi) { p.z = 2.0f * P.g.z_hi - p.z; v.z = -v.z; }
                p.z = fminf(fmaxf(p.z, P.g.z_lo), P.g.z_hi);
            }
            if (!(p.x >= 0.f && p.x < P.g.Lx)) p.x = 0.f;   // rounding at the boundary
            if (!(p.y >= 0.f && p.y < P.g.Ly)) p.y = 0.f;
            if (P.g.periodic_z && !(p.z >= 0.f && p.z < P.g.Lz)) p.z = 0.f;
            pos[i] = p;
            vel[i] = v;
        }
        __syncthreads();
        if (warp == 0) build_cell_list(P, pos, N, cnt, slots, lane);
        __syncthreads();
        forces_all<CL>(P, pos, cnt, slots, frc, vel, N, 0.5f * dt, true);
        __syncthreads();
    }
    float kp = 0.f;
    for (int i = tid; i < N; i += kMdThreads) {
        const float4 v = vel[i];
        kp += 0.5f * (v.x * v.x + v.y * v.y + v.z * v.z);
        const float4 p = pos[i];
        gpos[i] = make_float4(p.x, p.y, p.z, 0.f);
    }
    const float K = cta_sum(kp, red);
    if (tid == 0 && kin_out) kin_out[w] = K;
}

}  // namespace

size_t md_smem(int nmax, int ncell, int cap) { return md_smem_bytes(nmax, ncell, cap); }

cudaError_t launch_md(const SweepParams& P, int n_steps, float dt, float tau, uint32_t seg, float* kin_out,
                      cudaStream_t s) {
    const size_t smem = md_smem_bytes(P.nmax, P.cg.ncell, P.cg.cap);
    const double c_tau = exp(-(double)dt / (double)tau);   // thermostat decay per step
    cudaError_t err;
    if (P.n_cluster > 0) {
        err = cudaFuncSetAttribute(md_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
        md_kernel<true><<<P.S, kMdThreads, smem, s>>>(P, n_steps, dt, c_tau, seg, kin_out);
    } else {
        err = cudaFuncSetAttribute(md_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
        md_kernel<false><<<P.S, kMdThreads, smem, s>>>(P, n_steps, dt, c_tau, seg, kin_out);
    }
    return cudaGetLastError();
}

}  // namespace regc
