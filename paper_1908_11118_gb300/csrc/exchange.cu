// exchange.cu -- collective replica exchange on the (T, mu) grid (sm_103a).
//
// Sec. II.A.2: one of four neighbour directions (T, mu, diagonal,
// anti-diagonal) is drawn with probability 1/4 together with a parity bit.
// Every state (l, m) whose row (column, for the mu direction) has that parity
// is paired with (l + dl, m + dm); pairs are disjoint, so one thread per pair
// decides and swaps without races.  The swap rule is Eq. Pacc in log form,
// evaluated in FP64; a swap exchanges the two walkers' state labels.
#include "launch.h"

namespace regc {
namespace {

// One exchange attempt e of one (T, mu) grid, by the threads of one CTA.
// With a second species on a third axis (K > 1) a fifth direction, along
// mu2, joins the four: type = (C0 * 5) >> 32, pairing (l, m, k) with
// (l, m, k + 1) for k of the drawn parity; the other directions act within
// every k-slice.  With two species the swap rule takes both: the Lambda
// factor the total N (both wavelengths scale as beta^(1/2)), the mu terms
// each species' count.
__device__ __forceinline__ void exchange_grid(const ExchangeParams& X, uint32_t e, int first, int stride) {
    const int K = X.K;
    const int n_dir = K > 1 ? 5 : 4;
    const U4 C = philox(e, 0u, 0u, 2u, X.key0, X.key1);
    const int type = (int)(((unsigned long long)C.x * (unsigned long long)n_dir) >> 32);
    const int parity = (int)(C.y >> 31);
    const int dk = type == 4 ? 1 : 0;
    const int dl = (type == 1 || type == 4) ? 0 : 1;
    const int dm = (type == 0 || type == 4) ? 0 : (type == 3 ? -1 : 1);
    const int S = X.L * X.M * K;
    for (int a = first; a < S; a += stride) {
        const int lm = a / K, k = a - lm * K;
        const int l = lm / X.M, m = lm - l * X.M;
        const int key = dk ? k : (dl ? l : m);
        if ((key & 1) != parity) continue;
        const int l2 = l + dl, m2 = m + dm, k2 = k + dk;
        if (l2 >= X.L || m2 < 0 || m2 >= X.M || k2 >= K) continue;
        const int b = (l2 * X.M + m2) * K + k2;
        const int wa = X.walker_of_state[a], wb = X.walker_of_state[b];
        const double dn = (double)(X.n[wa] - X.n[wb]);
        const double ea = (double)X.efix[wa] * kFixUnit, eb = (double)X.efix[wb] * kFixUnit;
        double la;
        if (X.nb) {
            const double dnb = (double)(X.nb[wa] - X.nb[wb]);
            const double dnc = dn - dnb;
            la = 1.5 * dn * (X.lnbeta[a] - X.lnbeta[b]) - (X.beta[a] - X.beta[b]) * (eb - ea) -
                 (X.bmu[a] - X.bmu[b]) * dnb - (X.bmu2[a] - X.bmu2[b]) * dnc;
        } else {
            la = 1.5 * dn * (X.lnbeta[a] - X.lnbeta[b]) - (X.beta[a] - X.beta[b]) * (eb - ea) -
                 (X.bmu[a] - X.bmu[b]) * dn;
        }
        const U4 D = philox(e, (uint32_t)a, 0u, 3u, X.key0, X.key1);
        // ln u < ln alpha, decided in binary32 when the two sides are more than
        // 1e-3 apart (ln u to about 1e-6, and ln alpha's rounding matters only
        // where it is within a few units of ln u >= -22.2), else in FP64: the
        // FP64 decision in every case, without an FP64 logarithm per pair on
        // this part's narrow FP64 pipe
        const float lu_f = __logf(((float)D.x + 0.5f) * 2.3283064365386963e-10f);
        const float la_f = (float)la;
        bool acc;
        if (lu_f < la_f - 1e-3f) acc = true;
        else if (lu_f > la_f + 1e-3f) acc = false;
        else acc = log(((double)D.x + 0.5) * 2.3283064365386963e-10) < la;
        X.ex_counts[2 * n_dir * a + 2 * type] += 1;
        X.ex_counts[2 * n_dir * a + 2 * type + 1] += acc;
        if (acc) {
            X.walker_of_state[a] = wb;
            X.walker_of_state[b] = wa;
            X.state_of_walker[wa] = b;
            X.state_of_walker[wb] = a;
        }
    }
}

// The pairs of one attempt are disjoint (every state of the drawn parity with
// its neighbour in the drawn direction), so they are spread over CTAs.
constexpr int kExThreads = 128;

__global__ void __launch_bounds__(kExThreads) exchange_kernel(const __grid_constant__ ExchangeParams X, uint32_t e) {
    exchange_grid(X, e, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// One exchange attempt of every grid of a batch (CTA m: grid m, attempt
// number e_ctr[m]); afterwards each grid's exchange counter advances by one
// and its sweep counter t0 by the sweeps just run, on the device, so that a
// captured step can be replayed.
__global__ void __launch_bounds__(256) batch_exchange_kernel(const ExchangeParams* xs, uint32_t* e_ctr,
                                                             SweepParams* sys, int n_sweeps) {
    const int m = blockIdx.x;
    const ExchangeParams X = xs[m];
    const uint32_t e = e_ctr[m];
    exchange_grid(X, e, threadIdx.x, blockDim.x);
    __syncthreads();
    if (threadIdx.x == 0) {
        e_ctr[m] = e + 1u;
        sys[m].t0 += (uint32_t)n_sweeps;
    }
}

}  // namespace

cudaError_t launch_batch_exchange(const ExchangeParams* xs, uint32_t* e_ctr, SweepParams* sys, int n_systems,
                                  int n_sweeps, cudaStream_t s) {
    if (n_systems <= 0) return cudaSuccess;
    batch_exchange_kernel<<<n_systems, 256, 0, s>>>(xs, e_ctr, sys, n_sweeps);
    return cudaGetLastError();
}

cudaError_t launch_exchange(const ExchangeParams& X, uint32_t e, cudaStream_t s) {
    const int S = X.L * X.M * X.K;
    exchange_kernel<<<(S + kExThreads - 1) / kExThreads, kExThreads, 0, s>>>(X, e);
    return cudaGetLastError();
}

}  // namespace regc
