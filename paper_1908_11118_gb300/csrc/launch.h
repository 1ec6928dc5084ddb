// launch.h -- host-side launchers of the REGC kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>

#include "regc_internal.cuh"

namespace regc {

// Shared-memory bytes of the sweep kernel's CTA (one walker, W warps).
size_t sweep_smem_per_walker(int nmax, int ncell, int cap, int warps_per_walker);

// P.n_sweeps sweeps of every walker with P.warps_per_walker warps per walker;
// P.trace may be null.
cudaError_t launch_sweep(const SweepParams& P, cudaStream_t s);

// From-scratch fixed-point energy of every walker into out[S]; a pair inside
// the hard-core guard sets ERR_OVERLAP (check_overlap 1) or ERR_NUMERIC
// (check_overlap 2) in P.error.
cudaError_t launch_energy(const SweepParams& P, long long* out, int check_overlap,
                          cudaStream_t s);

// Caller positions xyz [S][nmax][3] -> pos [S][nmax] (zeros beyond n[w]);
// coordinates outside the region set ERR_INPUT in *error.
cudaError_t pack_walkers(const float* xyz, const int* n, int S, int nmax, const Geometry& g, float4* pos, int* error,
                         cudaStream_t s);

// pos [count] -> xyz [count][3] (count = S nmax); with n [S], only the first
// n[w] entries of each walker are written.
cudaError_t unpack_walkers(const float4* pos, long long count, int nmax, const int* n, float* xyz, cudaStream_t s);

// ---------------------------------------------------------------- batch
// Static shared memory of the batch sweep kernel and its warp limit per CTA
// (da: the delayed-acceptance instantiation).
size_t batch_static_smem(bool da);
int batch_max_warps(bool da);

// Persistent sweep of items (system, walker) of the systems sys[] (device
// table; every system's n_sweeps and t0 are read from it), taken in order from
// the queue *counter (zero before the launch); walkers_per_cta walkers of
// warps_per_walker warps each per CTA (1, 2 or 4; more than one for plain
// one-species systems only), each with `region` bytes of dynamic shared
// memory.  da: every system of the items samples with delayed acceptance; cl:
// every system carries a cluster species.
cudaError_t launch_batch_sweep(const SweepParams* sys, const int2* items, int n_items, int* counter,
                               int walkers_per_cta, int warps_per_walker, int grid, int region, bool da, bool cl,
                               cudaStream_t s);

// Allow every batch sweep kernel up to max_smem bytes of shared memory in all
// (before any launch or capture that needs more than 48 KB).
cudaError_t batch_prepare(int max_smem);

// Resident CTAs per SM of the batch sweep kernel for this shape (0 if none fit).
int batch_occupancy(int walkers_per_cta, int warps_per_walker, int region, bool da, bool cl);

// One exchange attempt of every system's grid (attempt numbers e_ctr[]), then
// e_ctr[m] += 1 and sys[m].t0 += n_sweeps on the device.
cudaError_t launch_batch_exchange(const ExchangeParams* xs, uint32_t* e_ctr, SweepParams* sys, int n_systems,
                                  int n_sweeps, cudaStream_t s);

// One MD segment of every walker (md.cu): n_steps velocity-Verlet steps of
// length dt with the stochastic velocity rescaling thermostat (time constant
// tau) from Maxwell-Boltzmann velocities (segment number seg); kinetic
// energies after the last step into kin_out[S] if not null.  Positions are
// written back; energies are not recomputed.
cudaError_t launch_md(const SweepParams& P, int n_steps, float dt, float tau, uint32_t seg, float* kin_out,
                      cudaStream_t s);
size_t md_smem(int nmax, int ncell, int cap);

// One collective exchange attempt number e.
cudaError_t launch_exchange(const ExchangeParams& X, uint32_t e, cudaStream_t s);

// ------------------------------------------------------------ surrogate
// Device buffers of the surrogate's BF16 inference copy.
struct SurrogateStore {
    __nv_bfloat16* w1;   // [64][16]
    float* b1;           // [64]
    __nv_bfloat16* w2;   // [64][64]
    float* b2;           // [64]
    __nv_bfloat16* w3;   // [64]
    float* b3;           // [1]
};

// FP32 master parameters theta[5313] -> the inference copy.
cudaError_t surrogate_pack(const float* theta, const SurrogateStore& st, cudaStream_t s);

// Surrogate energies e_out[Q] and features f_out[Q][16] of Q positions q
// (x, y, z) against every particle of walker w and the surface.
cudaError_t surrogate_eval(const SweepParams& P, int w, int Q, const float4* q, float* e_out, float* f_out,
                           cudaStream_t s);

// S * (parts + probes) training rows (features X[.][16], targets y = min(e, clip))
// written to the ring of cap rows starting at row base.
cudaError_t surrogate_harvest(const SweepParams& P, int parts, int probes, float clip, uint32_t round, float* X,
                              float* y, int base, int cap, cudaStream_t s);

// Floats of the per-CTA gradient scratch of surrogate_step for n rows.
size_t surrogate_partial_floats(int n);

// Gradient of the mean squared error of n rows (idx[t] or t) at theta_in into
// grad (may be null) and the sum of squared residuals into *loss; then, when
// adam_t > 0, Adam step number adam_t with learning rate lr on theta, m, v.
// tensor_cores: the matrix products in BF16 on mma.sync tiles (FP32
// accumulation); else everything in binary32 on the FP32 pipe.
cudaError_t surrogate_step(const float* theta_in, const float* X, const float* y, const int* idx, int n,
                           float* partial, float* grad, float* loss, float* theta, float* m, float* v, int adam_t,
                           float lr, bool tensor_cores, cudaStream_t s);

// Seeded initial parameters (normal weights of standard deviation
// scale / sqrt(fan-in), zero biases) into theta[5313].
cudaError_t surrogate_init(float* theta, float scale, uint32_t k0, uint32_t k1, cudaStream_t s);

// batch uniform row indices in [0, count) for training step `step`.
cudaError_t surrogate_batch_index(int* idx, int batch, int count, uint32_t step, uint32_t k0, uint32_t k1,
                                  cudaStream_t s);

}  // namespace regc
