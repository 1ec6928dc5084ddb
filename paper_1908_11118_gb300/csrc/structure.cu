// structure.cu -- structural observables of the sampled configurations and
// their MBAR averages per phase (Sec. III.A "Structural properties": the
// axial distribution rho(z) in slabs parallel to the surface and the lateral
// radial distribution g_xy(r) of an adsorbate layer; Sec. II.B, Eq. avegr).
//
// sample:   one CTA per walker counts its grand-canonical particles per slab
//           and, per layer, its unordered pairs per lateral distance bin, in
//           shared memory, and appends one row per walker to the store.
// reweight: MBAR over the samples (every sample its own bin, the device solve
//           of mbar.cu), the weight of every sample at each query state, then
//           per phase the weighted column sums of the rows -- a streaming
//           pass over the store, bound by HBM bandwidth.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "handle.h"
#include "mbar.h"

using namespace regc;

namespace {

constexpr size_t kMaxSmemStructure = 232448;  // 227 KB per block on sm_103a
constexpr int kSampleThreads = 256;
constexpr int kAccThreads = 128;
constexpr int kQB = 8;                          // query states per pass of the accumulation
constexpr double kPi = 3.14159265358979323846;
// aiAT keys: energy (2^-30 units) << 16 | walker; energies beyond +-2^46
// units (65536 energy units) are not tracked.  An empty slot holds the byte
// pattern 0x7f.. (larger than every key).
constexpr long long kKeyEmpty = 0x7f7f7f7f7f7f7f7fLL;
constexpr long long kKeyEnergyLimit = 1LL << 46;

struct SampleParams {
    const float4* pos;
    const int* n;
    const long long* efix;
    const int* sow;
    int nmax, n_cluster;
    float Lx, Ly, hLx, hLy, z_lo, shear;
    int n_z;
    float inv_dz;
    int n_layers;
    float layer_lo[4], layer_hi[4];
    int n_r;
    float inv_dr;
    int rho_stride, pair_stride;
    long long base;
    int32_t* state;
    int32_t* nb;
    double* energy;
    int32_t* pop;
    uint16_t* rho;
    uint32_t* pairs;
    long long* best_key;
};

size_t sample_smem(int nmax, int n_z, int n_layers, int n_r) {
    size_t b = (size_t)nmax * 12;                            // x, y, z
    b += (size_t)n_z * 4 + (size_t)n_layers * n_r * 4;       // counts
    b += (size_t)n_layers * nmax * 2;                        // layer member lists
    b += 20;                                                 // layer populations (+ alignment)
    return (b + 15) & ~(size_t)15;
}

__global__ void __launch_bounds__(kSampleThreads) structure_sample_kernel(const __grid_constant__ SampleParams P) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int w = blockIdx.x, tid = threadIdx.x;
    const int nA = P.n_cluster;
    const int N = P.n[w];
    const int m = max(0, N - nA);
    float* xs = reinterpret_cast<float*>(smem);
    float* ys = xs + P.nmax;
    float* zs = ys + P.nmax;
    uint32_t* hz = reinterpret_cast<uint32_t*>(zs + P.nmax);
    uint32_t* hp = hz + P.n_z;
    uint16_t* lists = reinterpret_cast<uint16_t*>(hp + P.n_layers * P.n_r);
    int* cnt = reinterpret_cast<int*>(lists + P.n_layers * P.nmax);
    // the lists may end on a 2-byte boundary: cnt is placed at the next 4-byte one
    cnt = reinterpret_cast<int*>((reinterpret_cast<uintptr_t>(cnt) + 3) & ~uintptr_t(3));

    for (int k = tid; k < P.n_z; k += kSampleThreads) hz[k] = 0u;
    for (int k = tid; k < P.n_layers * P.n_r; k += kSampleThreads) hp[k] = 0u;
    if (tid < 4) cnt[tid] = 0;
    const float4* gp = P.pos + (size_t)w * P.nmax;
    for (int i = tid; i < m; i += kSampleThreads) {
        const float4 q = gp[nA + i];
        xs[i] = q.x;
        ys[i] = q.y;
        zs[i] = q.z;
    }
    __syncthreads();
    // slabs and layer membership
    for (int i = tid; i < m; i += kSampleThreads) {
        const float z = zs[i];
        const float k = floorf(__fmul_rn(__fsub_rn(z, P.z_lo), P.inv_dz));
        if (k >= 0.0f && k < (float)P.n_z) atomicAdd(&hz[(int)k], 1u);
        for (int l = 0; l < P.n_layers; ++l)
            if (P.layer_lo[l] <= z && z < P.layer_hi[l]) lists[l * P.nmax + atomicAdd(&cnt[l], 1)] = (uint16_t)i;
    }
    __syncthreads();
    // unordered pairs of each layer: warps take rows, lanes columns
    const int lane = tid & 31, warp = tid >> 5;
    for (int l = 0; l < P.n_layers; ++l) {
        const int ml = cnt[l];
        const uint16_t* li = lists + l * P.nmax;
        uint32_t* hl = hp + l * P.n_r;
        for (int a = warp; a < ml; a += kSampleThreads / 32) {
            const int ia = li[a];
            const float xa = xs[ia], ya = ys[ia];
            for (int b = a + 1 + lane; b < ml; b += 32) {
                const int ib = li[b];
                const float dy = min_image_exact(ya, ys[ib], P.Ly, P.hLy);
                const float dx = __fadd_rn(min_image_exact(xa, xs[ib], P.Lx, P.hLx), __fmul_rn(P.shear, dy));
                const float r = __fsqrt_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)));
                const float k = floorf(__fmul_rn(r, P.inv_dr));
                if (k < (float)P.n_r) atomicAdd(&hl[(int)k], 1u);
            }
        }
    }
    __syncthreads();
    const long long row = P.base + w;
    uint16_t* rr = P.rho + row * P.rho_stride;
    for (int k = tid; k < P.rho_stride; k += kSampleThreads) rr[k] = k < P.n_z ? (uint16_t)hz[k] : (uint16_t)0;
    uint32_t* pr = P.pairs + row * (long long)P.pair_stride;
    for (int k = tid; k < P.pair_stride; k += kSampleThreads) pr[k] = k < P.n_layers * P.n_r ? hp[k] : 0u;
    if (tid < 4) P.pop[row * 4 + tid] = tid < P.n_layers ? cnt[tid] : 0;
    if (tid == 0) {
        const long long E = P.efix[w];
        P.state[row] = P.sow[w];
        P.nb[row] = m;
        P.energy[row] = (double)E * kFixUnit;
        if (E > -kKeyEnergyLimit && E < kKeyEnergyLimit)
            atomicMin(&P.best_key[m], (long long)(((unsigned long long)E << 16) | (unsigned long long)w));
    }
}

// The walker whose key is the lowest of its N_B copies its configuration
// (keys are unique: one walker at most matches).
__global__ void best_config_kernel(const float4* pos, const int* n, const long long* efix, int nmax, int n_cluster,
                                   const long long* best_key, float* best_xyz, int32_t* best_n) {
    const int w = blockIdx.x;
    const int N = n[w], m = max(0, N - n_cluster);
    const long long E = efix[w];
    if (!(E > -kKeyEnergyLimit && E < kKeyEnergyLimit)) return;
    const long long key = (long long)(((unsigned long long)E << 16) | (unsigned long long)w);
    if (best_key[m] != key) return;
    const float4* gp = pos + (size_t)w * nmax;
    float* out = best_xyz + (size_t)m * nmax * 3;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const float4 q = gp[j];
        out[3 * j] = q.x;
        out[3 * j + 1] = q.y;
        out[3 * j + 2] = q.z;
    }
    if (threadIdx.x == 0) best_n[m] = N;
}

// omega[s] = number of samples of state s (exact in double).
__global__ void count_states_kernel(const int32_t* state, long long count, double* omega) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x)
        atomicAdd(&omega[state[i]], 1.0);
}

// W[q][n] = exp(-(a_q E_n + c_q N_n) - D_bin(n) + f_q).
__global__ void weights_kernel(const int32_t* nb, const double* energy, const int32_t* bin_of, const double* D,
                               long long count, int nq, const double* a_q, const double* c_q, const double* f_q,
                               double* W) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count * nq;
         i += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(i / count);
        const long long n = i - (long long)q * count;
        W[i] = exp(-fma(a_q[q], energy[n], c_q[q] * (double)nb[n]) - D[bin_of[n]] + f_q[q]);
    }
}

constexpr int kChunk = 256;                     // samples of one phase per CTA of the accumulation

struct AccParams {
    const int32_t* order;     // sample indices grouped by phase, in sample order within a phase
    const int4* chunks;       // [n_chunks] (phase, first entry of order, samples, 0)
    const uint16_t* rho;      // [count][rho_stride]
    const uint32_t* pairs;    // [count][pair_stride]
    const int32_t* pop;
    const double* W;          // [nq][count]
    long long count;
    int rho_stride, pair_stride, n_r, nq;
    double area;
    double* Jp;               // [n_chunks][nq][rho_stride + pair_stride] partial sums per chunk
};

// Weighted column sums of one chunk of a phase's samples.  The chunk's sample
// indices, weights and layer normalisations are staged in shared memory; each
// query state's weights are divided by their largest value in the chunk, so
// that the products and the sum over the chunk (at most kChunk terms, all
// non-negative) run on the binary32 pipe, relative error below kChunk 2^-24
// (1.6e-5); the chunk's sum is scaled back in FP64.  Each thread takes two
// adjacent columns (slabs, or a layer's distance bins; the row strides are
// multiples of 16 bytes, so a pair never straddles the two parts) with one
// vector load per row, eight rows in flight, for kQB query states.
__global__ void __launch_bounds__(kAccThreads) accumulate_kernel(const __grid_constant__ AccParams A) {
    __shared__ double w64[kChunk][kQB];
    __shared__ float4 w32[kChunk][kQB / 4];
    __shared__ double scale[kQB];
    __shared__ int idx[kChunk];
    __shared__ float cnorm[kChunk][4];       // 2 A / (M (M - 1)) per layer, 0 when M < 2
    const int4 ch = A.chunks[blockIdx.y];
    const int q0 = blockIdx.z * kQB;
    const int nql = min(kQB, A.nq - q0);
    for (int i = threadIdx.x; i < ch.z; i += kAccThreads) {
        const int n = A.order[ch.y + i];
        idx[i] = n;
#pragma unroll
        for (int j = 0; j < kQB; ++j) w64[i][j] = j < nql ? A.W[(long long)(q0 + j) * A.count + n] : 0.0;
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const double M = (double)A.pop[(long long)n * 4 + l];
            cnorm[i][l] = M >= 2.0 ? (float)(2.0 * A.area / (M * (M - 1.0))) : 0.0f;
        }
    }
    __syncthreads();
    {   // largest weight of each query state in the chunk: warp w takes states w, w + 4
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        for (int j = warp; j < kQB; j += kAccThreads / 32) {
            double mx = 0.0;
            for (int i = lane; i < ch.z; i += 32) mx = fmax(mx, w64[i][j]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (lane == 0) scale[j] = mx;
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < ch.z * kQB; t += kAccThreads) {
        const int i = t / kQB, j = t - i * kQB;
        reinterpret_cast<float*>(&w32[i][0])[j] = scale[j] > 0.0 ? (float)(w64[i][j] / scale[j]) : 0.0f;
    }
    __syncthreads();
    const int cols = A.rho_stride + A.pair_stride;
    const int col = 2 * (blockIdx.x * kAccThreads + threadIdx.x);
    if (col >= cols) return;
    float acc0[kQB], acc1[kQB];
#pragma unroll
    for (int j = 0; j < kQB; ++j) acc0[j] = acc1[j] = 0.0f;
    auto add = [&](int i, float v0, float v1) {
        const float4 wa = w32[i][0], wb = w32[i][1];
        const float w[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
#pragma unroll
        for (int j = 0; j < kQB; ++j) {
            acc0[j] = fmaf(w[j], v0, acc0[j]);
            acc1[j] = fmaf(w[j], v1, acc1[j]);
        }
    };
    constexpr int U = 8;
    if (col < A.rho_stride) {
        const unsigned* base = reinterpret_cast<const unsigned*>(A.rho) + col / 2;
        const long long rs = A.rho_stride / 2;
        int i = 0;
        for (; i + U <= ch.z; i += U) {
            unsigned v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) v[u] = __ldg(base + (long long)idx[i + u] * rs);
#pragma unroll
            for (int u = 0; u < U; ++u) add(i + u, (float)(v[u] & 0xffffu), (float)(v[u] >> 16));
        }
        for (; i < ch.z; ++i) {
            const unsigned v = __ldg(base + (long long)idx[i] * rs);
            add(i, (float)(v & 0xffffu), (float)(v >> 16));
        }
    } else {
        const int c = col - A.rho_stride;
        const int l0 = min(c / A.n_r, 3), l1 = min((c + 1) / A.n_r, 3);
        const uint2* base = reinterpret_cast<const uint2*>(A.pairs + c);
        const long long rs = A.pair_stride / 2;
        int i = 0;
        for (; i + U <= ch.z; i += U) {
            uint2 v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) v[u] = __ldg(base + (long long)idx[i + u] * rs);
#pragma unroll
            for (int u = 0; u < U; ++u) add(i + u, (float)v[u].x * cnorm[i + u][l0], (float)v[u].y * cnorm[i + u][l1]);
        }
        for (; i < ch.z; ++i) {
            const uint2 v = __ldg(base + (long long)idx[i] * rs);
            add(i, (float)v.x * cnorm[i][l0], (float)v.y * cnorm[i][l1]);
        }
    }
    double* out = A.Jp + ((long long)blockIdx.y * A.nq + q0) * cols + col;
    for (int j = 0; j < nql; ++j) {
        out[(long long)j * cols] = (double)acc0[j] * scale[j];
        out[(long long)j * cols + 1] = (double)acc1[j] * scale[j];
    }
}

// J[q][ph][col] = sum of the phase's chunk partials, in chunk order.
__global__ void reduce_chunks_kernel(const double* Jp, const int* first_chunk, int nq, int P, int cols, double* J) {
    const long long tot = (long long)nq * P * cols;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
         t += (long long)gridDim.x * blockDim.x) {
        const int col = (int)(t % cols);
        const long long qp = t / cols;
        const int ph = (int)(qp % P), q = (int)(qp / P);
        double v = 0.0;
        for (int c = first_chunk[ph]; c < first_chunk[ph + 1]; ++c) v += Jp[((long long)c * nq + q) * cols + col];
        J[t] = v;
    }
}

regc_status fail(regc_handle* h, cudaError_t e) { return handle_cuda_fail(h, e); }

}  // namespace

extern "C" {

regc_status regc_structure_init(regc_handle* h, const regc_structure_spec* spec) {
    if (h && h->P.gc2) return REGC_EINVAL;   // structure samples with one grand-canonical species only
    if (!h || !spec) return REGC_EINVAL;
    if (h->sticky != REGC_OK) return h->sticky;
    const regc_structure_spec& s = *spec;
    if (s.n_z < 1 || s.n_z > 4096 || !(s.dz > 0.0f) || !std::isfinite(s.dz) || s.n_layers < 0 || s.n_layers > 4 ||
        s.n_r < 1 || s.n_r > 4096 || !(s.dr > 0.0f) || !std::isfinite(s.dr) || s.capacity < 1)
        return REGC_EINVAL;
    // lateral distances up to the inscribed radius of the cell, where the
    // nearest image in the cell frame is the nearest image
    const double sh = h->P.g.shear;
    if (!((double)s.n_r * s.dr <= 0.5 * std::min((double)h->Lx / sqrt(1.0 + sh * sh), (double)h->Ly)))
        return REGC_EINVAL;
    for (int l = 0; l < s.n_layers; ++l)
        if (!(s.layer_lo[l] < s.layer_hi[l])) return REGC_EINVAL;
    const size_t smem = sample_smem(h->nmax, s.n_z, s.n_layers, s.n_r);
    if (smem > kMaxSmemStructure) return REGC_EINVAL;
    StructureStore& st = h->stc;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return fail(h, e);
    if (st.block) {
        cudaFree(st.block);
        st = StructureStore{};
    }
    const size_t cap = (size_t)s.capacity;
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t b_state = up(cap * 4), b_nb = up(cap * 4), b_e = up(cap * 8), b_pop = up(cap * 16);
    const int rho_stride = (s.n_z + 7) & ~7, pair_stride = (s.n_layers * s.n_r + 3) & ~3;
    const size_t b_rho = up(cap * rho_stride * 2), b_pairs = up(cap * (size_t)pair_stride * 4);
    const size_t nh = (size_t)h->nmax + 1;
    const size_t b_key = up(nh * 8), b_bn = up(nh * 4), b_bx = up(nh * (size_t)h->nmax * 12);
    void* block = nullptr;
    e = cudaMalloc(&block, b_state + b_nb + b_e + b_pop + b_rho + b_pairs + b_key + b_bn + b_bx);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return REGC_ENOMEM;
    }
    char* c = static_cast<char*>(block);
    st.block = block;
    st.state = reinterpret_cast<int32_t*>(c);
    st.nb = reinterpret_cast<int32_t*>(c + b_state);
    st.energy = reinterpret_cast<double*>(c + b_state + b_nb);
    st.pop = reinterpret_cast<int32_t*>(c + b_state + b_nb + b_e);
    st.rho = reinterpret_cast<uint16_t*>(c + b_state + b_nb + b_e + b_pop);
    st.pairs = reinterpret_cast<uint32_t*>(c + b_state + b_nb + b_e + b_pop + b_rho);
    char* c2 = c + b_state + b_nb + b_e + b_pop + b_rho + b_pairs;
    st.best_key = reinterpret_cast<long long*>(c2);
    st.best_n = reinterpret_cast<int32_t*>(c2 + b_key);
    st.best_xyz = reinterpret_cast<float*>(c2 + b_key + b_bn);
    e = cudaMemsetAsync(st.best_key, 0x7f, nh * 8, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(st.best_n, 0, nh * 4, h->stream);
    if (e != cudaSuccess) return fail(h, e);
    st.n_z = s.n_z;
    st.rho_stride = rho_stride;
    st.pair_stride = pair_stride;
    st.n_layers = s.n_layers;
    st.n_r = s.n_r;
    st.dz = s.dz;
    st.dr = s.dr;
    st.inv_dz = (float)(1.0 / (double)s.dz);
    st.inv_dr = (float)(1.0 / (double)s.dr);
    for (int l = 0; l < 4; ++l) {
        st.layer_lo[l] = l < s.n_layers ? s.layer_lo[l] : 0.0f;
        st.layer_hi[l] = l < s.n_layers ? s.layer_hi[l] : 0.0f;
    }
    st.cap = s.capacity;
    st.count = 0;
    st.smem = smem;
    e = cudaFuncSetAttribute(structure_sample_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return fail(h, e);
}

regc_status regc_structure_sample(regc_handle* h) {
    NvtxRange nvtx_("regc_structure_sample");
    if (!h) return REGC_EINVAL;
    if (h->sticky != REGC_OK) return h->sticky;
    StructureStore& st = h->stc;
    if (!st.block || h->need_walkers || h->sharded() || st.count + h->S > st.cap) return REGC_EINVAL;
    SampleParams P;
    P.pos = h->P.pos;
    P.n = h->P.n;
    P.efix = h->P.efix;
    P.sow = h->P.state_of_walker;
    P.nmax = h->nmax;
    P.n_cluster = h->P.n_cluster;
    P.Lx = h->P.g.Lx;
    P.Ly = h->P.g.Ly;
    P.hLx = h->P.g.hLx;
    P.hLy = h->P.g.hLy;
    P.z_lo = h->P.g.z_lo;
    P.shear = h->P.g.shear;
    P.n_z = st.n_z;
    P.inv_dz = st.inv_dz;
    P.n_layers = st.n_layers;
    for (int l = 0; l < 4; ++l) {
        P.layer_lo[l] = st.layer_lo[l];
        P.layer_hi[l] = st.layer_hi[l];
    }
    P.n_r = st.n_r;
    P.inv_dr = st.inv_dr;
    P.rho_stride = st.rho_stride;
    P.pair_stride = st.pair_stride;
    P.base = st.count;
    P.state = st.state;
    P.nb = st.nb;
    P.energy = st.energy;
    P.pop = st.pop;
    P.rho = st.rho;
    P.pairs = st.pairs;
    P.best_key = st.best_key;
    structure_sample_kernel<<<h->S, kSampleThreads, st.smem, h->stream>>>(P);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        best_config_kernel<<<h->S, 128, 0, h->stream>>>(h->P.pos, h->P.n, h->P.efix, h->nmax, h->P.n_cluster,
                                                         st.best_key, st.best_xyz, st.best_n);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return fail(h, e);
    st.count += h->S;
    return REGC_OK;
}

regc_status regc_structure_timing(regc_handle* h, double* ms_mbar, double* ms_weights, double* ms_accumulate,
                                  double* bytes_accumulate) {
    if (!h) return REGC_EINVAL;
    if (ms_mbar) *ms_mbar = h->stc.last_ms[0];
    if (ms_weights) *ms_weights = h->stc.last_ms[1];
    if (ms_accumulate) *ms_accumulate = h->stc.last_ms[2];
    if (bytes_accumulate) *bytes_accumulate = h->stc.last_bytes;
    return REGC_OK;
}

regc_status regc_structure_count(regc_handle* h, int64_t* n_samples) {
    if (!h || !n_samples) return REGC_EINVAL;
    *n_samples = h->stc.count;
    return REGC_OK;
}

regc_status regc_structure_reset(regc_handle* h) {
    if (!h) return REGC_EINVAL;
    if (h->sticky != REGC_OK) return h->sticky;
    h->stc.count = 0;
    if (h->stc.block) {
        const cudaError_t e = cudaMemsetAsync(h->stc.best_key, 0x7f, ((size_t)h->nmax + 1) * 8, h->stream);
        if (e != cudaSuccess) return fail(h, e);
    }
    return REGC_OK;
}

regc_status regc_aiat(regc_handle* h, int nq, const double* mu_q, double* e_min, double* dG, int32_t* phase) {
    if (!h || nq < 0 || (nq > 0 && !mu_q)) return REGC_EINVAL;
    if (h->sticky != REGC_OK) return h->sticky;
    const StructureStore& st = h->stc;
    if (!st.block) return REGC_EINVAL;
    for (int q = 0; q < nq; ++q)
        if (!std::isfinite(mu_q[q])) return REGC_EINVAL;
    const int nh = h->nmax + 1;
    std::vector<long long> key(nh);
    cudaError_t e = cudaMemcpyAsync(key.data(), st.best_key, nh * 8, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return fail(h, e);
    std::vector<double> em(nh);
    for (int n = 0; n < nh; ++n)
        em[n] = key[n] == kKeyEmpty ? NAN : (double)(key[n] >> 16) * kFixUnit;   // arithmetic shift: floor
    if (e_min) std::copy(em.begin(), em.end(), e_min);
    // Eq. aiTherm with F ~ the lowest sampled energy and F of the pristine
    // slab 0 (the frozen slab's own energy is not part of E)
    for (int q = 0; q < nq; ++q) {
        int best = -1;
        double bv = INFINITY;
        for (int n = 0; n < nh; ++n) {
            const double v = std::isnan(em[n]) ? INFINITY : em[n] - (double)n * mu_q[q];
            if (dG) dG[(size_t)q * nh + n] = v;
            if (v < bv) {
                bv = v;
                best = n;
            }
        }
        if (phase) phase[q] = best;
    }
    return REGC_OK;
}

regc_status regc_aiat_config(regc_handle* h, int n_b, float* xyz, int32_t* n) {
    if (!h || !xyz || !n) return REGC_EINVAL;
    if (h->sticky != REGC_OK) return h->sticky;
    const StructureStore& st = h->stc;
    if (!st.block || n_b < 0 || n_b > h->nmax) return REGC_EINVAL;
    long long key = 0;
    int32_t cnt = 0;
    cudaError_t e = cudaMemcpyAsync(&key, st.best_key + n_b, 8, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&cnt, st.best_n + n_b, 4, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return fail(h, e);
    if (key == kKeyEmpty) return REGC_EINVAL;
    *n = cnt;
    if (cnt > 0) {
        e = cudaMemcpyAsync(xyz, st.best_xyz + (size_t)n_b * h->nmax * 3, (size_t)cnt * 12, cudaMemcpyDeviceToHost,
                            h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return fail(h, e);
    }
    return REGC_OK;
}

regc_status regc_structure_get(regc_handle* h, int64_t first, int64_t count, int32_t* state, int32_t* n,
                               double* energy, uint16_t* rho, uint32_t* pairs, int32_t* pop) {
    if (!h) return REGC_EINVAL;
    if (h->sticky != REGC_OK) return h->sticky;
    const StructureStore& st = h->stc;
    if (!st.block || first < 0 || count < 0 || first + count > st.count) return REGC_EINVAL;
    if (count == 0) return REGC_OK;
    cudaError_t e = cudaSuccess;
    auto get = [&](void* dst, const void* src, size_t bytes) {
        if (dst && e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, h->stream);
    };
    const size_t nlr = (size_t)st.n_layers * st.n_r;
    get(state, st.state + first, (size_t)count * 4);
    get(n, st.nb + first, (size_t)count * 4);
    get(energy, st.energy + first, (size_t)count * 8);
    if (rho && e == cudaSuccess)
        e = cudaMemcpy2DAsync(rho, st.n_z * 2, st.rho + first * st.rho_stride, st.rho_stride * 2, st.n_z * 2, count,
                              cudaMemcpyDeviceToHost, h->stream);
    if (nlr && pairs && e == cudaSuccess)
        e = cudaMemcpy2DAsync(pairs, nlr * 4, st.pairs + first * st.pair_stride, st.pair_stride * 4, nlr * 4, count,
                              cudaMemcpyDeviceToHost, h->stream);
    if (pop) {
        std::vector<int32_t> p4((size_t)count * 4);
        get(p4.data(), st.pop + first * 4, (size_t)count * 16);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e == cudaSuccess)
            for (int64_t i = 0; i < count; ++i)
                for (int l = 0; l < st.n_layers; ++l) pop[i * st.n_layers + l] = p4[i * 4 + l];
    }
    if (e != cudaSuccess) return fail(h, e);
    return handle_sync_check(h);
}

regc_status regc_structure_reweight(regc_handle* h, int nq, const double* kT_q, const double* mu_q, int n_lo,
                                    int n_hi, double tol, int max_iter, double* p, double* rho, double* gxy,
                                    double* f_states, int* iters) {
    NvtxRange nvtx_("regc_structure_reweight");
    if (!h || nq < 1 || !kT_q || !mu_q || n_lo < 0 || n_hi < n_lo || max_iter < 1 || !(tol > 0.0)) return REGC_EINVAL;
    if (h->sticky != REGC_OK) return h->sticky;
    const StructureStore& st = h->stc;
    const long long count = st.count;
    if (!st.block || count < 1) return REGC_EINVAL;
    for (int q = 0; q < nq; ++q)
        if (!(kT_q[q] > 0.0) || !std::isfinite(kT_q[q]) || !std::isfinite(mu_q[q])) return REGC_EINVAL;
    const int S = h->S;
    const int n_top = std::min(n_hi, h->nmax);
    const int P = n_hi - n_lo + 1;
    const int cols = st.rho_stride + st.pair_stride;       // padded columns of the sums
    cudaStream_t s = h->stream;

    // group the samples by phase (stable: sample order within a phase)
    std::vector<int32_t> nb(count);
    std::vector<double> en(count);
    cudaError_t e = cudaMemcpyAsync(nb.data(), st.nb, count * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(en.data(), st.energy, count * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(h, e);
    // samples with the same (N_B, E) -- bit-identical energies, as every empty
    // walker has -- have the same weight at every state: they are pooled into
    // one MBAR bin with their count, exactly as the equations allow
    std::vector<int32_t> bin_of(count);
    std::vector<int32_t> bN;
    std::vector<double> bE, blnH;
    {
        std::vector<int32_t> ix(count);
        for (long long i = 0; i < count; ++i) ix[i] = (int32_t)i;
        std::sort(ix.begin(), ix.end(), [&](int32_t x, int32_t y) {
            return nb[x] != nb[y] ? nb[x] < nb[y] : (en[x] != en[y] ? en[x] < en[y] : x < y);
        });
        long long run = 0;
        for (long long i = 0; i < count; ++i) {
            const int32_t k = ix[i];
            if (i == 0 || nb[k] != bN.back() || en[k] != bE.back()) {
                if (i > 0) blnH.push_back(log((double)run));
                bN.push_back(nb[k]);
                bE.push_back(en[k]);
                run = 0;
            }
            bin_of[k] = (int32_t)(bN.size() - 1);
            ++run;
        }
        blnH.push_back(log((double)run));
    }
    const long long B = (long long)bN.size();
    std::vector<long long> offset(P + 1, 0);
    for (long long i = 0; i < count; ++i)
        if (nb[i] >= n_lo && nb[i] <= n_hi) offset[nb[i] - n_lo + 1] += 1;
    for (int i = 0; i < P; ++i) offset[i + 1] += offset[i];
    std::vector<int32_t> order(std::max<long long>(offset[P], 1));
    {
        std::vector<long long> next(offset.begin(), offset.end() - 1);
        for (long long i = 0; i < count; ++i)
            if (nb[i] >= n_lo && nb[i] <= n_hi) order[next[nb[i] - n_lo]++] = (int32_t)i;
    }
    // chunks of at most kChunk samples of one phase
    std::vector<int4> chunks;
    std::vector<int> first_chunk(P + 1, 0);
    for (int i = 0; i < P; ++i) {
        first_chunk[i] = (int)chunks.size();
        for (long long b = offset[i]; b < offset[i + 1]; b += kChunk)
            chunks.push_back(make_int4(i, (int)b, (int)std::min<long long>(kChunk, offset[i + 1] - b), 0));
    }
    first_chunk[P] = (int)chunks.size();
    const int n_chunks = std::max(1, (int)chunks.size());
    if (chunks.empty()) chunks.push_back(make_int4(0, 0, 0, 0));
    std::vector<double> a_q(nq), c_q(nq);
    for (int q = 0; q < nq; ++q) {
        a_q[q] = 1.0 / kT_q[q];
        c_q[q] = 3.0 * (log(h->lambda0) - 0.5 * log(kT_q[q])) - a_q[q] * mu_q[q];
    }

    // device scratch, one allocation
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t nh = (size_t)h->nmax + 1;
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t o = off; off += up(bytes); return o; };
    const size_t o_a = take(S * 8), o_c = take(S * 8), o_lnom = take(S * 8), o_om = take(S * 8), o_f = take(S * 8),
                 o_fn = take(S * 8), o_del = take(8), o_stt = take(8), o_lnH = take(B * 8), o_D = take(B * 8),
                 o_en = take(B * 8), o_dh = take(B * 4), o_bN = take(B * 4), o_bE = take(B * 8),
                 o_map = take(count * 4),
                 o_aq = take(nq * 8), o_cq = take(nq * 8), o_fq = take(nq * 8), o_pN = take(nq * nh * 8),
                 o_W = take((size_t)nq * count * 8), o_ord = take(order.size() * 4),
                 o_ch = take(chunks.size() * sizeof(int4)), o_fc = take((P + 1) * 4),
                 o_Jp = take((size_t)n_chunks * nq * cols * 8), o_J = take((size_t)nq * P * cols * 8),
                 o_rs = take((B + 1) * 4), o_rsc = take(mbar_runs_scratch((int)B) * 8);
    char* d = nullptr;
    e = cudaMallocAsync(reinterpret_cast<void**>(&d), off, s);
    if (e != cudaSuccess) return fail(h, e);
    double* d_a = reinterpret_cast<double*>(d + o_a);
    double* d_c = reinterpret_cast<double*>(d + o_c);
    double* d_lnom = reinterpret_cast<double*>(d + o_lnom);
    double* d_om = reinterpret_cast<double*>(d + o_om);
    double* d_f = reinterpret_cast<double*>(d + o_f);
    double* d_fn = reinterpret_cast<double*>(d + o_fn);
    double* d_del = reinterpret_cast<double*>(d + o_del);
    int* d_stt = reinterpret_cast<int*>(d + o_stt);
    double* d_lnH = reinterpret_cast<double*>(d + o_lnH);
    int32_t* d_bN = reinterpret_cast<int32_t*>(d + o_bN);
    double* d_bE = reinterpret_cast<double*>(d + o_bE);
    int32_t* d_map = reinterpret_cast<int32_t*>(d + o_map);
    double* d_D = reinterpret_cast<double*>(d + o_D);
    float2* d_en = reinterpret_cast<float2*>(d + o_en);
    float* d_dh = reinterpret_cast<float*>(d + o_dh);
    double* d_aq = reinterpret_cast<double*>(d + o_aq);
    double* d_cq = reinterpret_cast<double*>(d + o_cq);
    double* d_fq = reinterpret_cast<double*>(d + o_fq);
    double* d_pN = reinterpret_cast<double*>(d + o_pN);
    double* d_W = reinterpret_cast<double*>(d + o_W);
    int32_t* d_ord = reinterpret_cast<int32_t*>(d + o_ord);
    int4* d_ch = reinterpret_cast<int4*>(d + o_ch);
    int* d_fc = reinterpret_cast<int*>(d + o_fc);
    double* d_Jp = reinterpret_cast<double*>(d + o_Jp);
    double* d_J = reinterpret_cast<double*>(d + o_J);

    int it = 0;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaEventCreate(&ev[i]);
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_om, 0, S * 8, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_lnH, blnH.data(), B * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_bN, bN.data(), B * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_bE, bE.data(), B * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_map, bin_of.data(), count * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        count_states_kernel<<<std::max(1, (int)std::min<long long>((count + 255) / 256, 4096)), 256, 0, s>>>(
            st.state, count, d_om);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = mbar_prep_states(S, h->d_kT_state, h->d_mu_state, h->lambda0, d_om, nullptr, d_a, d_c,
                                               d_lnom, s);
    MbarDev m{S, (int)B, d_a, d_c, d_lnom, d_bN, d_bE, d_lnH, d_f, d_fn, d_D, d_en, d_dh, d_del, d_stt};
    if (count > 0x7fffffffLL) e = cudaErrorInvalidValue;
    if (e == cudaSuccess) e = mbar_solve_dev(m, tol, max_iter, &it, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_aq, a_q.data(), nq * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_cq, c_q.data(), nq * 8, cudaMemcpyHostToDevice, s);
    int n_runs = 0;   // the bins are sorted by (N_B, E): a run is a row of one N_B
    if (e == cudaSuccess)
        e = mbar_runs_dev(m, reinterpret_cast<long long*>(d + o_rsc), reinterpret_cast<int*>(d + o_rs), &n_runs, s);
    if (e == cudaSuccess) {
        m.run_start = reinterpret_cast<int*>(d + o_rs);
        m.n_runs = n_runs;
        e = mbar_query_dev(m, nq, d_aq, d_cq, h->nmax, nullptr, d_pN, d_fq, s);
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
    if (e == cudaSuccess) {
        const long long tot = (long long)nq * count;
        weights_kernel<<<(int)std::min<long long>((tot + 255) / 256, 65536), 256, 0, s>>>(
            st.nb, st.energy, d_map, d_D, count, nq, d_aq, d_cq, d_fq, d_W);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_ord, order.data(), order.size() * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_ch, chunks.data(), chunks.size() * sizeof(int4), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_fc, first_chunk.data(), (P + 1) * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaEventRecord(ev[2], s);
    if (e == cudaSuccess) {
        AccParams A{d_ord, d_ch, st.rho, st.pairs, st.pop, d_W, count, st.rho_stride, st.pair_stride,
                    std::max(st.n_r, 1), nq, (double)h->Lx * (double)h->Ly, d_Jp};
        const dim3 grid((cols / 2 + kAccThreads - 1) / kAccThreads, n_chunks, (nq + kQB - 1) / kQB);
        accumulate_kernel<<<grid, kAccThreads, 0, s>>>(A);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        const long long tot = (long long)nq * P * cols;
        reduce_chunks_kernel<<<(int)std::min<long long>((tot + 255) / 256, 65536), 256, 0, s>>>(d_Jp, d_fc, nq, P,
                                                                                             cols, d_J);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev[3], s);
    std::vector<double> J((size_t)nq * P * cols), pN((size_t)nq * nh);
    if (e == cudaSuccess) e = cudaMemcpyAsync(J.data(), d_J, J.size() * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(pN.data(), d_pN, pN.size() * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && f_states) e = cudaMemcpyAsync(f_states, d_f, S * 8, cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(d, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) {
        float ms[3] = {0, 0, 0};
        for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]);
        StructureStore& sm = h->stc;
        for (int i = 0; i < 3; ++i) sm.last_ms[i] = ms[i];
        // every row of a phase in range once per pass of kQB query states, with
        // its population and index, its weights, and the sums written (the
        // per-chunk partial sums are the implementation's, not counted)
        const double row = (double)st.rho_stride * 2 + (double)st.pair_stride * 4 + 16 + 4;
        const int passes = (nq + kQB - 1) / kQB;
        sm.last_bytes = (double)offset[P] * (row * passes + 8.0 * nq) +
                        (double)nq * P * (st.n_z + st.n_layers * st.n_r) * 8;
    }
    for (int i = 0; i < 4; ++i)
        if (ev[i]) cudaEventDestroy(ev[i]);
    if (e != cudaSuccess) return fail(h, e);
    if (iters) *iters = it;

    // normalise: densities per unit volume, g_xy per unit shell area, within the phase
    const double area = (double)h->Lx * (double)h->Ly;
    const double dz = st.dz, dr = st.dr;
    for (int q = 0; q < nq; ++q)
        for (int i = 0; i < P; ++i) {
            const int nbv = n_lo + i;
            const double pi_q = nbv <= n_top ? pN[(size_t)q * nh + nbv] : 0.0;
            if (p) p[(size_t)q * P + i] = pi_q;
            const double* Jr = &J[((size_t)q * P + i) * cols];
            if (rho)
                for (int k = 0; k < st.n_z; ++k)
                    rho[((size_t)q * P + i) * st.n_z + k] = pi_q > 0.0 ? Jr[k] / (pi_q * area * dz) : 0.0;
            if (gxy)
                for (int l = 0; l < st.n_layers; ++l)
                    for (int k = 0; k < st.n_r; ++k) {
                        const double shell = kPi * dr * dr * ((k + 1.0) * (k + 1.0) - (double)k * k);
                        gxy[(((size_t)q * P + i) * st.n_layers + l) * st.n_r + k] =
                            pi_q > 0.0 ? Jr[st.rho_stride + l * st.n_r + k] / (pi_q * shell) : 0.0;
                    }
        }
    return handle_sync_check(h);
}

}  // extern "C"
