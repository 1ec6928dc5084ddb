// mbar.h -- device MBAR reweighting (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace regc {

// Device arrays of one MBAR problem: S states, B pooled bins.  The reduced
// potential of state s at bin b is u_s(b) = a[s] E_b + c[s] N_b with
// a = beta, c = 3 ln Lambda - beta mu.
struct MbarDev {
    int S, B;
    const double* a;       // [S]
    const double* c;       // [S]
    const double* lnom;    // [S] ln Omega_s (-inf when Omega_s = 0)
    const int* N_b;        // [B]
    const double* E_b;     // [B]
    const double* lnH;     // [B]
    double* f;             // [S] current free energies (gauge f_0 = 0)
    double* f_new;         // [S]
    double* D;             // [B]
    float2* EN32;          // [B] (E_b, N_b) in binary32, filled by the solve
    float* DH32;           // [B] D_b - lnH_b in binary32, written with D
    double* delta;         // [1] max |f_new - f| of the last iteration
    int* state;            // [2] cleared by the solve (the kernels skip work when state[0] is set)
    // a second grand-canonical species: u_s(b) = a[s] E_b + c[s] N_b + c2[s] N2_b
    const int* N2_b;       // [B] its counts, or null (one species)
    const double* c2;      // [S] 3 ln Lambda_C - beta mu2
    float* N2f;            // [B] N2_b in binary32, filled by the solve
    // runs of bins with equal (N, N2) in the bin order (mbar_runs_dev), for
    // the query; without them the query screens bin by bin
    const int* run_start;  // [n_runs + 1], run_start[n_runs] = B
    int n_runs;
};

// What the last mbar_solve_dev of the calling thread did: path 1 when it
// iterated on the sparse kernel matrix (0: log-sum-exps only), its
// iterations, matrix builds, maps taken on log-sum-exps, the kept entries of
// the last build, S, B, the device time of the builds and of the maps on the
// matrix, and the number of those maps.
struct MbarInfo {
    int path, iterations, builds, lse_maps;
    long long nnz;
    long long S, B;
    double ms_build, ms_maps;   // device time of the matrix builds and of the maps on it
    int sparse_maps;            // maps on the matrix
    // the warm start of mbar_solve_warm_dev (zero without one): bins, iterations,
    // builds and maps of the coarse solve (its times are included above)
    long long coarse_B;
    int coarse_iterations, coarse_builds, coarse_maps;
};
MbarInfo mbar_last_info();

// Solve the self-consistent equations from f = 0 (the plain fixed-point map
// with Anderson acceleration) until max |G(f) - f| < tol or max_iter maps.
// Synchronises the stream after every map.
// With allow_matrix (and every state sampled) the iterations run on the
// kept entries of the kernel matrix K_sb = exp(-u_s(b) + ln Omega_s + f_ref,s
// - max_k(...)) (those within e^-70 of their bin's largest), allocated on the
// stream for the duration of the call when they fit in half the free device
// memory; otherwise on log-sum-exps of the energies.
// x0 (host, S values, optional) is the starting point instead of f = 0.
cudaError_t mbar_solve_dev(const MbarDev& m, double tol, int max_iter, int* iters_out,
                           cudaStream_t s, bool allow_matrix = true, const double* x0 = nullptr);

// mbar_solve_dev started from the solution of the same problem coarsened in
// energy (width > 0, at least 65536 bins): bins adjacent in the bin order
// with equal N (and N2) and equal floor(E / width) merged into one at their
// count-weighted mean energy, solved to 1e-6.  The fixed point is the fine
// problem's; only the path to it is shorter (far fewer matrix builds).
cudaError_t mbar_solve_warm_dev(const MbarDev& m, double width, double tol, int max_iter, int* iters_out,
                                cudaStream_t s);

// Reweight to Q query states given on the device as (a_q, c_q):
// N_mean [Q], pN [Q][nmax+1], f_q [Q] (device, any may be null).  Reads the
// binary32 copies EN32, DH32 (and N2f) that a solve leaves, or that
// mbar_prep32_dev writes from the FP64 bins and D.
cudaError_t mbar_query_dev(const MbarDev& m, int Q, const double* a_q, const double* c_q,
                           int nmax, double* N_mean, double* pN, double* f_q, cudaStream_t s);

// Two species: reweight to Q query states (a_q, c_q, c2_q): the means of both
// counts N_mean, N2_mean [Q], their distributions pN, pN2 [Q][nmax+1] and
// f_q [Q] (device, any may be null).
cudaError_t mbar_query2_dev(const MbarDev& m, int Q, const double* a_q, const double* c_q, const double* c2_q,
                            int nmax, double* N_mean, double* N2_mean, double* pN, double* pN2, double* f_q,
                            cudaStream_t s);

// Runs of bins with equal (N, N2) in the bin order: run_start [n_runs + 1]
// (device, at most B + 1 ints), *n_runs (host; synchronises the stream).
// scratch: mbar_runs_scratch(B) long longs (device).
size_t mbar_runs_scratch(int B);
cudaError_t mbar_runs_dev(const MbarDev& m, long long* scratch, int* run_start, int* n_runs, cudaStream_t s);

// The binary32 copies of the bins the query screens with: EN32, N2f (when
// N2_b is set) and DH32 = D - lnH, from E_b, N_b, N2_b, D and lnH.
cudaError_t mbar_prep32_dev(const MbarDev& m, cudaStream_t s);

// c2 = 3 ln(lambda0_2 / sqrt(kT)) - mu2 / kT of a second species, per state (device).
cudaError_t mbar_prep_states2(int S, const double* kT, const double* mu2, double lambda0_2, double* c2,
                              cudaStream_t s);

// Compact the non-empty bins of a pooled histogram hist[n] (row-major in
// (N, E-bin), nbins E-bins per N) into N_b, E_b (bin centres), lnH (ln
// counts), in row-major order.  compact_count_dev writes the per-block
// offsets to scratch (compact_scratch_ints(n) ints) and the number of
// non-empty bins to *count_out (device); compact_write_dev then fills the
// arrays.
size_t compact_scratch_ints(long long n);
cudaError_t compact_count_dev(const unsigned long long* hist, long long n, int* scratch, int* count_out,
                              cudaStream_t s);
cudaError_t compact_write_dev(const unsigned long long* hist, long long n, int nbins, double e_lo, double e_bin,
                              const int* scratch, int* N_b, double* E_b, double* lnH, cudaStream_t s);

// As compact_write_dev for the two-species histogram, whose row is
// N (rows2) + N2: fills N_b and N2_b.
cudaError_t compact_write2_dev(const unsigned long long* hist, long long n, int nbins, int rows2, double e_lo,
                               double e_bin, const int* scratch, int* N_b, int* N2_b, double* E_b, double* lnH,
                               cudaStream_t s);

// State constants on the device: a = 1/kT, c = 3 ln(lambda0/sqrt(kT)) - mu/kT,
// lnom = ln Omega (-inf for Omega = 0; skipped when lnom is null).  kT, mu are
// per state (device); Omega from omega_d (double) or omega_u (uint64).
cudaError_t mbar_prep_states(int S, const double* kT, const double* mu, double lambda0, const double* omega_d,
                             const unsigned long long* omega_u, double* a, double* c, double* lnom, cudaStream_t s);
// lnH = ln H (device).
cudaError_t mbar_prep_bins(int B, const double* H, double* lnH, cudaStream_t s);

}  // namespace regc
