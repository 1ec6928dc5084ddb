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

// From-scratch fixed-point energy of every walker into out[S]; overlap flags
// go to P.error (ERR_OVERLAP) when check_overlap is set.
cudaError_t launch_energy(const SweepParams& P, long long* out, int check_overlap,
                          cudaStream_t s);

// One collective exchange attempt number e.
cudaError_t launch_exchange(const ExchangeParams& X, uint32_t e, cudaStream_t s);

}  // namespace regc
