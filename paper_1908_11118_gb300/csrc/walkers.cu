// walkers.cu -- walker state in and out of the device (sm_103a).
//
// The caller's positions are [S][nmax][3] binary32; the device keeps
// float4 [S][nmax].  These kernels convert between the two on the device, so a
// state upload or download is one contiguous copy of the caller's buffer and
// one launch, with the coordinate checks of regc_set_walkers done on the GPU.
#include "launch.h"

namespace regc {
namespace {

__global__ void pack_walkers_kernel(const float* xyz, const int* n, int S, int nmax, Geometry g, float4* pos,
                                    int* error) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long long)S * nmax) return;
    const int w = (int)(k / nmax), i = (int)(k % nmax);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i < n[w]) {
        const float x = xyz[3 * k], y = xyz[3 * k + 1], z = xyz[3 * k + 2];
        const bool okx = x >= 0.0f && x < g.Lx, oky = y >= 0.0f && y < g.Ly;
        const bool okz = g.periodic_z ? (z >= 0.0f && z < g.Lz) : (z >= g.z_lo && z <= g.z_hi);
        if (okx && oky && okz) v = make_float4(x, y, z, 0.0f);
        else atomicOr(error, ERR_INPUT);
    }
    pos[k] = v;
}

__global__ void unpack_walkers_kernel(const float4* pos, long long count, int nmax, const int* n, float* xyz) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    if (n && (int)(k % nmax) >= n[k / nmax]) return;   // beyond N: left as it was
    const float4 v = pos[k];
    xyz[3 * k] = v.x;
    xyz[3 * k + 1] = v.y;
    xyz[3 * k + 2] = v.z;
}

}  // namespace

cudaError_t pack_walkers(const float* xyz, const int* n, int S, int nmax, const Geometry& g, float4* pos, int* error,
                         cudaStream_t s) {
    const long long count = (long long)S * nmax;
    if (count == 0) return cudaSuccess;
    pack_walkers_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(xyz, n, S, nmax, g, pos, error);
    return cudaGetLastError();
}

cudaError_t unpack_walkers(const float4* pos, long long count, int nmax, const int* n, float* xyz, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    unpack_walkers_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(pos, count, nmax, n, xyz);
    return cudaGetLastError();
}

}  // namespace regc
