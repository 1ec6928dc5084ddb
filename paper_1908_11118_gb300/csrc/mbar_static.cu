// mbar_static.cu -- an MBAR solve that allocates no device memory.
//
// regc_mbar_solve stages its inputs and its work arrays in device memory it
// allocates for the call.  Some callers cannot allow that: a host application
// whose framework owns every device allocation through its own pool (and
// forbids or accounts for outside cudaMalloc calls), or a loop that must not
// pay for cudaMalloc/cudaFree, which can synchronise the device and stall the
// caller's other streams.  This variant runs the same kernels on a fixed
// scratch area compiled into the library instead: every GPU that loads the
// library reserves it until the process exits.
#include <math.h>
#include <string.h>

#include <cmath>

#include "launch.h"
#include "mbar.h"

namespace {

constexpr int kMaxS = REGC_MBAR_STATIC_MAX_STATES;
constexpr int kMaxB = REGC_MBAR_STATIC_MAX_BINS;
constexpr size_t kMaxDevices = 64;

// Layout of the scratch area (bytes, each part 256-byte aligned).
constexpr size_t al(size_t v) { return (v + 255) & ~size_t(255); }
constexpr size_t kStateBytes = al(size_t(kMaxS) * sizeof(double));
constexpr size_t kBinD = al(size_t(kMaxB) * sizeof(double));
constexpr size_t kBinI = al(size_t(kMaxB) * sizeof(int));
// states: kT, mu, omega, a, c, lnom, f, f_new; bins: N_b, E_b, H_b, lnH, D,
// (E, N) and D - lnH in binary32; delta, state
constexpr size_t kScratchBytes = 8 * kStateBytes + kBinI + 4 * kBinD + 256 + 256 + kBinD + kBinI;

static __device__ __align__(256) unsigned char g_mbar_scratch[kScratchBytes];

// Device address of g_mbar_scratch, looked up once per device.
void* g_scratch_addr[kMaxDevices] = {nullptr};

regc_status scratch_for_current_device(unsigned char** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || (size_t)dev >= kMaxDevices) return REGC_ECUDA;
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_mbar_scratch) != cudaSuccess || !p) return REGC_ECUDA;
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
    return REGC_OK;
}

}  // namespace

extern "C" regc_status regc_mbar_solve_static(int S, const double* kT, const double* mu, double lambda0,
                                              const double* omega, int B, const int32_t* N_b, const double* E_b,
                                              const double* H_b, double tol, int max_iter, double* f, double* D,
                                              int* iters, void* cuda_stream) {
    if (S < 1 || B < 1 || !kT || !mu || !omega || !N_b || !E_b || !H_b || !(tol > 0.0) || max_iter < 1 ||
        !(lambda0 > 0.0))
        return REGC_EINVAL;
    if (S > kMaxS || B > kMaxB) return REGC_EINVAL;   // beyond the fixed scratch area
    for (int s = 0; s < S; ++s)
        if (!(kT[s] > 0.0) || !std::isfinite(mu[s]) || !(omega[s] >= 0.0)) return REGC_EINVAL;
    for (int b = 0; b < B; ++b)
        if (!(H_b[b] > 0.0) || N_b[b] < 0 || !std::isfinite(E_b[b])) return REGC_EINVAL;
    unsigned char* base = nullptr;
    regc_status st = scratch_for_current_device(&base);
    if (st != REGC_OK) return st;
    double* d_kT = reinterpret_cast<double*>(base);
    double* d_mu = reinterpret_cast<double*>(base + 1 * kStateBytes);
    double* d_om = reinterpret_cast<double*>(base + 2 * kStateBytes);
    double* a = reinterpret_cast<double*>(base + 3 * kStateBytes);
    double* c = reinterpret_cast<double*>(base + 4 * kStateBytes);
    double* lnom = reinterpret_cast<double*>(base + 5 * kStateBytes);
    double* fd = reinterpret_cast<double*>(base + 6 * kStateBytes);
    double* f_new = reinterpret_cast<double*>(base + 7 * kStateBytes);
    unsigned char* bins = base + 8 * kStateBytes;
    int* d_N = reinterpret_cast<int*>(bins);
    double* d_E = reinterpret_cast<double*>(bins + kBinI);
    double* d_H = reinterpret_cast<double*>(bins + kBinI + kBinD);
    double* lnH = reinterpret_cast<double*>(bins + kBinI + 2 * kBinD);
    double* Dd = reinterpret_cast<double*>(bins + kBinI + 3 * kBinD);
    double* delta = reinterpret_cast<double*>(bins + kBinI + 4 * kBinD);
    int* state = reinterpret_cast<int*>(bins + kBinI + 4 * kBinD + 256);
    float2* en32 = reinterpret_cast<float2*>(bins + kBinI + 4 * kBinD + 512);
    float* dh32 = reinterpret_cast<float*>(bins + kBinI + 5 * kBinD + 512);

    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaMemcpyAsync(d_kT, kT, S * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_mu, mu, S * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_om, omega, S * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_N, N_b, B * sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_E, E_b, B * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_H, H_b, B * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = regc::mbar_prep_states(S, d_kT, d_mu, lambda0, d_om, nullptr, a, c, lnom, s);
    if (e == cudaSuccess) e = regc::mbar_prep_bins(B, d_H, lnH, s);
    if (e != cudaSuccess) return REGC_ECUDA;
    regc::MbarDev m{};
    m.S = S;
    m.B = B;
    m.a = a;
    m.c = c;
    m.lnom = lnom;
    m.N_b = d_N;
    m.E_b = d_E;
    m.lnH = lnH;
    m.f = fd;
    m.f_new = f_new;
    m.D = Dd;
    m.EN32 = en32;
    m.DH32 = dh32;
    m.delta = delta;
    m.state = state;
    // mbar_solve_dev clears f and the convergence state before iterating, so
    // nothing left in the scratch area by an earlier call is read.
    e = regc::mbar_solve_dev(m, tol, max_iter, iters, s, false);   // no device allocation
    if (e == cudaSuccess && f) e = cudaMemcpyAsync(f, fd, S * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && D) e = cudaMemcpyAsync(D, Dd, B * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? REGC_OK : REGC_ECUDA;
}
