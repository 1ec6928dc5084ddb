// regc_api.cu -- the C ABI of the REGC library (host side).
//
// Validates arguments, derives the per-state constants of the acceptance
// rules (Sec. II.A.1, Eq. Ngrand), lays out the device state, and launches the
// kernels of sweep.cu, exchange.cu and mbar.cu on the handle's stream.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "handle.h"
#include "launch.h"
#include "mbar.h"

using namespace regc;


namespace {

constexpr size_t kMaxSmem = 232448;  // 227 KB per block on sm_103a

regc_status cuda_fail(regc_handle* h, cudaError_t e) {
    if (e == cudaSuccess) return REGC_OK;
    if (h && h->sticky == REGC_OK) h->sticky = (e == cudaErrorMemoryAllocation) ? REGC_ENOMEM : REGC_ECUDA;
    return e == cudaErrorMemoryAllocation ? REGC_ENOMEM : REGC_ECUDA;
}

template <class T>
regc_status dalloc(regc_handle* h, T** p, size_t count) {
    void* v = nullptr;
    const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    cudaError_t e = cudaMalloc(&v, bytes);
    if (e != cudaSuccess) return cuda_fail(h, e);
    h->allocs.push_back(v);
    e = cudaMemsetAsync(v, 0, bytes, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e);
    *p = static_cast<T*>(v);
    return REGC_OK;
}

template <class T>
regc_status upload(regc_handle* h, T* dst, const T* src, size_t count) {
    if (count == 0) return REGC_OK;
    return cuda_fail(h, cudaMemcpyAsync(dst, src, count * sizeof(T), cudaMemcpyHostToDevice, h->stream));
}

// Synchronise and fold the device error word into the sticky status.
regc_status sync_check(regc_handle* h) {
    if (h->sticky != REGC_OK) return h->sticky;
    int* flag = static_cast<int*>(h->h_stage);   // pinned: the copy stays asynchronous
    cudaError_t e = cudaMemcpyAsync(flag, h->d_error, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e);
    const int err = *flag;
    if (err & ERR_TIMEOUT) h->sticky = REGC_ETIMEOUT;
    else if (err & ERR_CAPACITY) h->sticky = REGC_ECAPACITY;
    else if (err & ERR_NUMERIC) h->sticky = REGC_ENUMERIC;
    return h->sticky;
}

int cells_along(double len, double rc) {
    const int n = (int)floor(len / (rc * 1.00001));
    return n < 1 ? 1 : n;
}

// Hard-core guard radius^2 of a pair type: pairs closer than this have
// phi > T = 1e6 max(eps_max, kT_max, 1), so every move creating one has an
// acceptance probability far below 2^-33 and is rejected outright; the guard
// also keeps every accepted pair term inside the fixed-point range.
float hard_core_r2(double eps, double sigma, double T) {
    if (eps <= 0.0) return 0.0f;
    double lo = 1e-3, hi = 1.0;   // x = r / sigma
    for (int it = 0; it < 200; ++it) {
        const double x = 0.5 * (lo + hi);
        const double s6 = 1.0 / pow(x, 6.0);
        const double phi = 4.0 * eps * (s6 * s6 - s6);
        if (phi > T) lo = x;
        else hi = x;
    }
    const double r = lo * sigma;
    return (float)(r * r);
}

}  // namespace

regc_status handle_sync_check(regc_handle* h) { return sync_check(h); }

regc_status handle_cuda_fail(regc_handle* h, cudaError_t e) { return cuda_fail(h, e); }

extern "C" {

const char* regc_status_string(regc_status s) {
    switch (s) {
        case REGC_OK: return "ok";
        case REGC_EINVAL: return "invalid argument";
        case REGC_ENOMEM: return "out of memory";
        case REGC_ECUDA: return "CUDA error";
        case REGC_ETIMEOUT: return "device wait timed out";
        case REGC_ECAPACITY: return "cell-list capacity exceeded";
        case REGC_ENUMERIC: return "non-finite or out-of-range energy";
    }
    return "unknown status";
}

void regc_free(regc_handle* h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    for (void* p : h->allocs) cudaFree(p);
    if (h->stc.block) cudaFree(h->stc.block);
    if (h->hE_block) cudaFree(h->hE_block);
    if (h->h_stage) cudaFreeHost(h->h_stage);
    delete h;
}

}  // extern "C"

namespace {

regc_status init_grid(const regc_potential* pot, const regc_surface* surf, const regc_grid_spec* grid,
                      const regc_species2* sp2, uint64_t seed, void* cuda_stream, regc_handle** out) {
    if (!out) return REGC_EINVAL;
    *out = nullptr;
    if (!pot || !surf || !grid) return REGC_EINVAL;
    const int K = sp2 ? sp2->K : 1;
    if (sp2) {
        if (sp2->type < 1 || sp2->type >= pot->n_types || sp2->K < 1 || !sp2->mu || !(sp2->lambda0 > 0.0))
            return REGC_EINVAL;
        for (int k = 0; k < sp2->K; ++k)
            if (!std::isfinite(sp2->mu[k])) return REGC_EINVAL;
    }
    // ---- validation
    const int nt = pot->n_types;
    if (nt < 1 || nt > 4 || !(pot->rc > 0.0f)) return REGC_EINVAL;
    double eps_max = 0.0;
    for (int i = 0; i < nt; ++i)
        for (int j = 0; j < nt; ++j) {
            if (!(pot->eps[i][j] >= 0.0f) || !(pot->eps[i][j] <= 2000.0f) || !(pot->sigma[i][j] > 0.0f))
                return REGC_EINVAL;
            eps_max = std::max(eps_max, (double)pot->eps[i][j]);
        }
    const double rc = pot->rc;
    // with a sheared cell, every partner within rc is the nearest image in the
    // cell frame when rc sqrt(1 + shear^2) <= Lx / 2 and rc <= Ly / 2
    const double shear = surf->shear;
    if (!std::isfinite(shear) || !(fabs(shear) <= 1.0)) return REGC_EINVAL;
    const double su = sqrt(1.0 + shear * shear);
    if (!(surf->Lx >= 2 * rc * su) || !(surf->Ly >= 2 * rc) || !(surf->z_hi > surf->z_lo)) return REGC_EINVAL;
    if (surf->periodic_z && (!(surf->Lz >= 2 * rc) || surf->z_lo != 0.0f || surf->z_hi != surf->Lz))
        return REGC_EINVAL;
    if (surf->n_atoms < 0 || (surf->n_atoms > 0 && (!surf->xyz || !surf->type))) return REGC_EINVAL;
    for (int a = 0; a < surf->n_atoms; ++a) {
        const float* r = surf->xyz + 3 * a;
        if (surf->type[a] < 1 || surf->type[a] >= nt) return REGC_EINVAL;
        if (!(r[0] >= 0.0f && r[0] < surf->Lx && r[1] >= 0.0f && r[1] < surf->Ly) || !std::isfinite(r[2]))
            return REGC_EINVAL;
    }
    if (grid->L < 1 || grid->M < 1 || (long long)grid->L * grid->M * K > 65536 || !grid->kT || !grid->mu)
        return REGC_EINVAL;
    double kT_max = 0.0;
    for (int l = 0; l < grid->L; ++l) {
        if (!(grid->kT[l] > 0.0) || !(grid->kT[l] <= 2000.0)) return REGC_EINVAL;
        kT_max = std::max(kT_max, grid->kT[l]);
    }
    for (int m = 0; m < grid->M; ++m)
        if (!std::isfinite(grid->mu[m])) return REGC_EINVAL;
    if (grid->nmax < 1 || grid->nmax > 4096 || grid->moves_per_sweep < 1 || grid->moves_per_sweep > 1024)
        return REGC_EINVAL;
    if (!(grid->max_disp >= 0.0f) || !(grid->p_disp >= 0.0 && grid->p_disp <= 1.0) || !(grid->lambda0 > 0.0))
        return REGC_EINVAL;
    if (!(grid->e_bin > 0.0) || grid->n_e_bins < 1 || !std::isfinite(grid->e_lo)) return REGC_EINVAL;
    const long long hist_rows = sp2 ? (long long)(grid->nmax + 1) * (grid->nmax + 1) : grid->nmax + 1;
    if (hist_rows * grid->n_e_bins > (1LL << 31)) return REGC_EINVAL;

    // ---- geometry of the cell list
    const int periodic_z = surf->periodic_z ? 1 : 0;
    const double hz = periodic_z ? surf->Lz : (double)surf->z_hi - (double)surf->z_lo;
    CellGrid cg{};
    cg.ncx = cells_along(surf->Lx, rc * su);   // the cell frame's u-width reaches rc sqrt(1 + shear^2)
    cg.ncy = cells_along(surf->Ly, rc);
    cg.ncz = cells_along(hz, rc);
    if ((long long)cg.ncx * cg.ncy * cg.ncz > 65535) return REGC_EINVAL;
    cg.ncell = cg.ncx * cg.ncy * cg.ncz;
    cg.icx = (float)(cg.ncx / (double)surf->Lx);
    cg.icy = (float)(cg.ncy / (double)surf->Ly);
    cg.icz = (float)(cg.ncz / hz);
    const double vcell = (double)surf->Lx / cg.ncx * ((double)surf->Ly / cg.ncy) * (hz / cg.ncz);
    cg.cap = std::min(grid->nmax, std::max(8, (int)ceil(1.6 * vcell) + 8));
    if (!(fabs(grid->e_lo) < 4294967296.0) || !(grid->e_bin * kFixPerUnit >= 1.0) ||
        !(grid->e_bin < 4294967296.0))
        return REGC_EINVAL;
    // warps per walker = moves evaluated speculatively per round (1, 2 or 4).
    // With many walkers per SM one is best: on the 1024-replica fcc(111)
    // workload two and four warps run at 0.58x and 0.44x of one (instruction
    // fetch and the round barriers outweigh the kept evaluations).  With about
    // one walker per SM the issue slots are idle and speculation pays: 160
    // replicas of the LJ A18 system run 1.33x faster with four warps; at 256
    // fcc(111) replicas (1.7 per SM) two warps gain 3 % and four lose 18 %.
    // REGC_WARPS_PER_WALKER overrides the choice.
    int W = 1;
    {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0) {
            const long long n_rep = (long long)grid->L * grid->M;
            if (4 * n_rep <= 5LL * sms) W = 4;
            else if (n_rep <= 2LL * sms) W = 2;
        }
    }
    if (const char* env = getenv("REGC_WARPS_PER_WALKER")) {
        const int v = atoi(env);
        if (v == 1 || v == 2 || v == 4) W = v;
    }
    while (W > 1 && sweep_smem_per_walker(grid->nmax, cg.ncell, cg.cap, W) > kMaxSmem) W /= 2;
    const size_t spw = sweep_smem_per_walker(grid->nmax, cg.ncell, cg.cap, W);
    if (spw > kMaxSmem) return REGC_EINVAL;

    regc_handle* h = new (std::nothrow) regc_handle;
    if (!h) return REGC_ENOMEM;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    h->L = grid->L;
    h->M = grid->M;
    h->K = K;
    h->n_dir = K > 1 ? 5 : 4;
    h->hist_rows = hist_rows;
    h->S = grid->L * grid->M * K;
    h->nmax = grid->nmax;
    h->mps = grid->moves_per_sweep;
    h->n_e_bins = grid->n_e_bins;
    h->lambda0 = grid->lambda0;
    h->e_lo = grid->e_lo;
    h->e_bin = grid->e_bin;
    h->Lx = surf->Lx;
    h->Ly = surf->Ly;
    h->Lz = surf->Lz;
    h->z_lo = surf->z_lo;
    h->z_hi = surf->z_hi;
    h->periodic_z = periodic_z;
    h->smem_per_walker = spw;
    const int S = h->S;

    // ---- per-state constants of the acceptance rules
    const double V = (double)surf->Lx * (double)surf->Ly * ((double)surf->z_hi - (double)surf->z_lo);
    const double lnV = log(V);
    std::vector<double> beta(S), c_ins(S), c_del(S), bmu(S), lnbeta(S), c_ins2(S), c_del2(S), bmu2(S);
    h->kT_state.resize(S);
    h->mu_state.resize(S);
    h->mu2_state.clear();
    for (int s = 0; s < S; ++s) {
        // state s = (l M + m) K + k: kT[l], mu[m], and mu2[k] of a second species
        const double kT = grid->kT[s / (grid->M * K)], mu = grid->mu[(s / K) % grid->M];
        const double b = 1.0 / kT;
        const double lnL = log(grid->lambda0) - 0.5 * log(kT);
        beta[s] = b;
        c_ins[s] = lnV - 3.0 * lnL + b * mu;
        c_del[s] = 3.0 * lnL - lnV - b * mu;
        bmu[s] = b * mu;
        lnbeta[s] = log(b);
        h->kT_state[s] = kT;
        h->mu_state[s] = mu;
        if (sp2) {
            const double mu2 = sp2->mu[s % K];
            const double lnL2 = log(sp2->lambda0) - 0.5 * log(kT);
            c_ins2[s] = lnV - 3.0 * lnL2 + b * mu2;
            c_del2[s] = 3.0 * lnL2 - lnV - b * mu2;
            bmu2[s] = b * mu2;
            h->mu2_state.push_back(mu2);
        }
    }
    if (sp2) h->lambda0_2 = sp2->lambda0;
    std::vector<double> ln_tab(grid->nmax + 2, 0.0);
    for (int k = 1; k < grid->nmax + 2; ++k) ln_tab[k] = log((double)k);
    std::vector<float> beta_f(S), cins_f(S), cdel_f(S), ln_f(grid->nmax + 2);
    for (int s = 0; s < S; ++s) {
        beta_f[s] = (float)beta[s];
        cins_f[s] = (float)c_ins[s];
        cdel_f[s] = (float)c_del[s];
    }
    for (size_t k = 0; k < ln_tab.size(); ++k) ln_f[k] = (float)ln_tab[k];

    // ---- surface columns (atoms within rc of any point of a column)
    SurfaceTab st{};
    st.nsx = std::max(1, (int)floor(surf->Lx / 0.6));
    st.nsy = std::max(1, (int)floor(surf->Ly / 0.6));
    st.isx = (float)(st.nsx / (double)surf->Lx);
    st.isy = (float)(st.nsy / (double)surf->Ly);
    const double wx = (double)surf->Lx / st.nsx, wy = (double)surf->Ly / st.nsy;
    const double reach = rc * 1.0001 + 1e-4;
    const double reach_u = reach * su;
    std::vector<float4> all(surf->n_atoms);
    double zmax = -INFINITY;
    std::vector<int> relevant;
    for (int a = 0; a < surf->n_atoms; ++a) {
        const float* r = surf->xyz + 3 * a;
        all[a] = make_float4(r[0], r[1], r[2], (float)surf->type[a]);
        if (periodic_z || r[2] > surf->z_lo - reach) {
            relevant.push_back(a);
            zmax = std::max(zmax, (double)r[2]);
        }
    }
    st.z_reach = relevant.empty() ? -INFINITY : (float)(zmax + rc * 1.00001 + 1e-4);
    // Each column lists every periodic image of every relevant atom that comes
    // within reach of the column.  An image at x_a - Lx is stored shifted (exact
    // when x_a >= Lx/2, and the image is out of reach otherwise); an image at
    // x_a + Lx is stored unshifted with a flag that shifts the query by -Lx
    // instead (exact for every query that can reach it).  Likewise for y and,
    // in a periodic box, z.
    std::vector<std::vector<float4>> cols(st.nsx * st.nsy);
    const int nzi = periodic_z ? 1 : 0;
    for (int iy = 0; iy < st.nsy; ++iy)
        for (int ix = 0; ix < st.nsx; ++ix) {
            const double x0 = ix * wx, x1 = (ix + 1) * wx, y0 = iy * wy, y1 = (iy + 1) * wy;
            for (int a : relevant) {
                const float* r = surf->xyz + 3 * a;
                for (int sx = -1; sx <= 1; ++sx)
                    for (int sy = -1; sy <= 1; ++sy)
                        for (int sz = -nzi; sz <= nzi; ++sz) {
                            const double ax = (double)r[0] + sx * (double)surf->Lx;
                            const double ay = (double)r[1] + sy * (double)surf->Ly;
                            const double ex = std::max(0.0, std::max(x0 - ax, ax - x1));
                            const double ey = std::max(0.0, std::max(y0 - ay, ay - y1));
                            if (shear == 0.0 ? ex * ex + ey * ey >= reach * reach : (ex >= reach_u || ey >= reach))
                                continue;
                            unsigned bits = (unsigned)surf->type[a];
                            float bx = r[0], by = r[1], bz = r[2];
                            if (sx < 0) bx = r[0] - surf->Lx;
                            if (sx > 0) bits |= 4u;
                            if (sy < 0) by = r[1] - surf->Ly;
                            if (sy > 0) bits |= 8u;
                            if (sz < 0) bz = r[2] - surf->Lz;
                            if (sz > 0) bits |= 16u;
                            float4 v;
                            v.x = bx;
                            v.y = by;
                            v.z = bz;
                            memcpy(&v.w, &bits, sizeof(float));
                            cols[iy * st.nsx + ix].push_back(v);
                        }
            }
        }
    // fixed-stride layout: every column padded to the same multiple of 32
    // slots with entries out of reach (z = 1e30, flag bit 5)
    size_t widest = 0;
    for (const auto& c : cols) widest = std::max(widest, c.size());
    st.stride = (int)std::max<size_t>(32, (widest + 31) / 32 * 32);
    float4 pad;
    pad.x = 0.0f;
    pad.y = 0.0f;
    pad.z = 1e30f;
    const unsigned pad_bits = 32u;
    memcpy(&pad.w, &pad_bits, sizeof(float));
    std::vector<float4> col_atoms(cols.size() * (size_t)st.stride, pad);
    for (size_t c = 0; c < cols.size(); ++c)
        std::copy(cols[c].begin(), cols[c].end(), col_atoms.begin() + c * (size_t)st.stride);

    // ---- pair tables
    const double T = 1e6 * std::max(std::max(eps_max, kT_max), 1.0);
    SweepParams& P = h->P;
    P.gg = PairTab{4.0f * pot->eps[0][0], pot->sigma[0][0] * pot->sigma[0][0],
                   hard_core_r2(pot->eps[0][0], pot->sigma[0][0], T), pot->eps[0][0]};
    for (int t = 0; t < 4; ++t) {
        const int tt = t < nt ? t : 0;
        P.gs[t] = PairTab{4.0f * pot->eps[0][tt], pot->sigma[0][tt] * pot->sigma[0][tt],
                          hard_core_r2(pot->eps[0][tt], pot->sigma[0][tt], T), pot->eps[0][tt]};
    }
    P.n_cluster = 0;
    P.gA = P.gAB = P.gg;
    for (int t = 0; t < 4; ++t) P.gsA[t] = P.gs[t];
    P.gc2 = sp2 ? 1 : 0;
    if (sp2) {
        // species B = type 0 (particles [0, N_B)), C = sp2->type: the two-species
        // tables hold B-B, B-C, C-C and the surface tables of each
        const int c = sp2->type;
        auto tab = [&](int a, int b) {
            return PairTab{4.0f * pot->eps[a][b], pot->sigma[a][b] * pot->sigma[a][b],
                           hard_core_r2(pot->eps[a][b], pot->sigma[a][b], T), pot->eps[a][b]};
        };
        P.gA = tab(0, 0);
        P.gAB = tab(0, c);
        P.gg = tab(c, c);
        for (int t = 0; t < 4; ++t) {
            const int tt = t < nt ? t : 0;
            P.gsA[t] = tab(0, tt);
            P.gs[t] = tab(c, tt);
        }
    }
    h->n_types = nt;
    memcpy(h->eps, pot->eps, sizeof(h->eps));
    memcpy(h->sigma, pot->sigma, sizeof(h->sigma));
    h->hard_core_T = T;
    P.g = Geometry{surf->Lx, surf->Ly, periodic_z ? surf->Lz : 0.0f, 0.5f * surf->Lx, 0.5f * surf->Ly,
                   periodic_z ? 0.5f * surf->Lz : 0.0f, periodic_z, surf->z_lo, surf->z_hi,
                   surf->z_hi - surf->z_lo, (float)(rc * rc), (float)rc, surf->shear};
    P.cg = cg;
    P.max_disp = grid->max_disp;
    P.th_disp = (unsigned long long)floor(grid->p_disp * 4294967296.0);
    P.S = S;
    P.w_begin = 0;
    P.w_end = S;
    P.nmax = grid->nmax;
    P.mps = grid->moves_per_sweep;
    P.key0 = (uint32_t)seed;
    P.key1 = (uint32_t)(seed >> 32);
    P.e_lo = grid->e_lo;
    P.e_bin = grid->e_bin;
    P.e_lo_fix = llround(grid->e_lo * kFixPerUnit);
    P.e_bin_fix = llround(grid->e_bin * kFixPerUnit);
    P.n_e_bins = grid->n_e_bins;
    P.smem_per_walker = (int)spw;
    P.warps_per_walker = W;

    // ---- device memory
    regc_status st_ = REGC_OK;
#define TRY(x)                         \
    do {                               \
        st_ = (x);                     \
        if (st_ != REGC_OK) {          \
            regc_free(h);              \
            return st_;                \
        }                              \
    } while (0)
    double *d_beta, *d_cins, *d_cdel, *d_ln, *d_bmu, *d_lnbeta;
    float4 *d_colat, *d_all;
    TRY(dalloc(h, &d_beta, S));
    TRY(dalloc(h, &d_cins, S));
    TRY(dalloc(h, &d_cdel, S));
    TRY(dalloc(h, &d_bmu, S));
    TRY(dalloc(h, &d_lnbeta, S));
    TRY(dalloc(h, &d_ln, ln_tab.size()));
    float *d_beta_f, *d_cins_f, *d_cdel_f, *d_ln_f;
    TRY(dalloc(h, &d_beta_f, S));
    TRY(dalloc(h, &d_cins_f, S));
    TRY(dalloc(h, &d_cdel_f, S));
    TRY(dalloc(h, &d_ln_f, ln_f.size()));
    TRY(upload(h, d_beta_f, beta_f.data(), S));
    TRY(upload(h, d_cins_f, cins_f.data(), S));
    TRY(upload(h, d_cdel_f, cdel_f.data(), S));
    TRY(upload(h, d_ln_f, ln_f.data(), ln_f.size()));
    P.beta_f = d_beta_f;
    P.c_ins_f = d_cins_f;
    P.c_del_f = d_cdel_f;
    P.ln_tab_f = d_ln_f;
    TRY(dalloc(h, &h->d_kT_state, S));
    TRY(dalloc(h, &h->d_mu_state, S));
    TRY(dalloc(h, &d_colat, col_atoms.size()));
    TRY(dalloc(h, &d_all, all.size()));
    TRY(upload(h, d_beta, beta.data(), S));
    TRY(upload(h, d_cins, c_ins.data(), S));
    TRY(upload(h, d_cdel, c_del.data(), S));
    TRY(upload(h, d_bmu, bmu.data(), S));
    TRY(upload(h, d_lnbeta, lnbeta.data(), S));
    TRY(upload(h, d_ln, ln_tab.data(), ln_tab.size()));
    TRY(upload(h, h->d_kT_state, h->kT_state.data(), S));
    TRY(upload(h, h->d_mu_state, h->mu_state.data(), S));
    TRY(upload(h, d_colat, col_atoms.data(), col_atoms.size()));
    TRY(upload(h, d_all, all.data(), all.size()));
    st.atoms = d_colat;
    st.all = d_all;
    st.n_all = surf->n_atoms;
    P.st = st;
    P.beta = d_beta;
    P.c_ins = d_cins;
    P.c_del = d_cdel;
    P.ln_tab = d_ln;
    int *d_n, *d_sow, *d_wos;
    long long *d_efix, *d_mc, *d_exc;
    float4* d_pos;
    TRY(dalloc(h, &d_pos, (size_t)S * grid->nmax));
    TRY(dalloc(h, &d_n, S));
    TRY(dalloc(h, &d_efix, S));
    TRY(dalloc(h, &d_sow, S));
    TRY(dalloc(h, &d_wos, S));
    TRY(dalloc(h, &d_mc, (size_t)S * 6));
    TRY(dalloc(h, &d_exc, (size_t)S * 2 * h->n_dir));
    TRY(dalloc(h, &P.hN, (size_t)S * (grid->nmax + 1)));
    TRY(dalloc(h, &P.omega, S));
    TRY(dalloc(h, &P.moments, (size_t)S * 4));
    TRY(dalloc(h, &P.hNE, (size_t)hist_rows * grid->n_e_bins));
    double *d_bmu2 = nullptr;
    if (sp2) {
        double *d_ci2, *d_cd2;
        float *d_ci2f, *d_cd2f;
        std::vector<float> ci2f(S), cd2f(S);
        for (int q = 0; q < S; ++q) {
            ci2f[q] = (float)c_ins2[q];
            cd2f[q] = (float)c_del2[q];
        }
        TRY(dalloc(h, &d_ci2, S));
        TRY(dalloc(h, &d_cd2, S));
        TRY(dalloc(h, &d_ci2f, S));
        TRY(dalloc(h, &d_cd2f, S));
        TRY(dalloc(h, &d_bmu2, S));
        TRY(upload(h, d_ci2, c_ins2.data(), S));
        TRY(upload(h, d_cd2, c_del2.data(), S));
        TRY(upload(h, d_ci2f, ci2f.data(), S));
        TRY(upload(h, d_cd2f, cd2f.data(), S));
        TRY(upload(h, d_bmu2, bmu2.data(), S));
        TRY(dalloc(h, &h->d_mu2_state, S));
        TRY(upload(h, h->d_mu2_state, h->mu2_state.data(), S));
        TRY(dalloc(h, &P.nb, S));
        TRY(dalloc(h, &P.hN2, (size_t)S * (grid->nmax + 1)));
        TRY(dalloc(h, &P.moments2, (size_t)S * 2));
        P.c_ins2 = d_ci2;
        P.c_del2 = d_cd2;
        P.c_ins2_f = d_ci2f;
        P.c_del2_f = d_cd2f;
    }
    TRY(dalloc(h, &P.e_out, S));
    TRY(dalloc(h, &P.pair_counts, 6));
    TRY(dalloc(h, &h->d_error, 1));
    TRY(dalloc(h, &h->d_fix, S));
    TRY(dalloc(h, &h->d_xyz, (size_t)S * grid->nmax * 3));
    if (cudaHostAlloc(&h->h_stage, 64 + (size_t)S * 8, cudaHostAllocDefault) != cudaSuccess) {
        h->h_stage = nullptr;
        regc_free(h);
        return REGC_ENOMEM;
    }
    std::vector<int> ident(S);
    for (int s = 0; s < S; ++s) ident[s] = s;
    TRY(upload(h, d_sow, ident.data(), S));
    TRY(upload(h, d_wos, ident.data(), S));
    P.pos = d_pos;
    P.n = d_n;
    P.efix = d_efix;
    P.state_of_walker = d_sow;
    P.move_counts = d_mc;
    P.error = h->d_error;
    P.trace = nullptr;
    P.trace_steps = 0;
    P.cycle = 0;
    P.m_first = 0;
    h->X = ExchangeParams{grid->L, grid->M, P.key0, P.key1, d_beta, d_bmu, d_lnbeta, d_n, d_efix, d_sow, d_wos, d_exc,
                          K, sp2 ? P.nb : nullptr, d_bmu2};
    TRY(cuda_fail(h, cudaStreamSynchronize(h->stream)));
#undef TRY
    *out = h;
    return REGC_OK;
}

}  // namespace

extern "C" {

regc_status regc_init_grid(const regc_potential* pot, const regc_surface* surf, const regc_grid_spec* grid,
                           uint64_t seed, void* cuda_stream, regc_handle** out) {
    return init_grid(pot, surf, grid, nullptr, seed, cuda_stream, out);
}

regc_status regc_init_grid2(const regc_potential* pot, const regc_surface* surf, const regc_grid_spec* grid,
                            const regc_species2* species2, uint64_t seed, void* cuda_stream, regc_handle** out) {
    if (!species2) {
        if (out) *out = nullptr;
        return REGC_EINVAL;
    }
    return init_grid(pot, surf, grid, species2, seed, cuda_stream, out);
}

regc_status regc_sweep(regc_handle* h, int n_sweeps) {
    NvtxRange nvtx_("regc_sweep");
    if (!h || n_sweeps < 0) return REGC_EINVAL;
    if (h->sticky != REGC_OK) return h->sticky;
    if (h->need_walkers) return REGC_EINVAL;
    if (n_sweeps == 0) return REGC_OK;
    SweepParams P = h->P;
    P.t0 = h->t;
    P.n_sweeps = n_sweeps;
    P.trace = nullptr;
    P.expire_waits = h->expire_next ? 1 : 0;
    h->expire_next = false;
    const regc_status st = cuda_fail(h, launch_sweep(P, h->stream));
    if (st == REGC_OK) h->t += (uint32_t)n_sweeps;
    return st;
}

regc_status regc_test_expire_waits(regc_handle* h) {
    if (!h) return REGC_EINVAL;
    h->expire_next = true;
    return REGC_OK;
}

regc_status regc_sweep_traced(regc_handle* h, int n_sweeps, regc_move_record* trace) {
    NvtxRange nvtx_("regc_sweep_traced");
    if (!h || n_sweeps < 0 || (n_sweeps > 0 && !trace) || h->sharded()) return REGC_EINVAL;
    if (h->sticky != REGC_OK) return h->sticky;
    if (h->need_walkers) return REGC_EINVAL;
    if (n_sweeps == 0) return REGC_OK;
    const size_t n = (size_t)h->S * n_sweeps * h->mps;
    regc_move_record* d_trace = nullptr;
    regc_status st = cuda_fail(h, cudaMallocAsync(&d_trace, n * sizeof(regc_move_record), h->stream));
    if (st != REGC_OK) return st;
    SweepParams P = h->P;
    P.t0 = h->t;
    P.n_sweeps = n_sweeps;
    P.trace = d_trace;
    P.trace_steps = n_sweeps;
    st = cuda_fail(h, launch_sweep(P, h->stream));
    if (st == REGC_OK) {
        h->t += (uint32_t)n_sweeps;
        st = cuda_fail(h, cudaMemcpyAsync(trace, d_trace, n * sizeof(regc_move_record), cudaMemcpyDeviceToHost,
                                          h->stream));
    }
    cudaFreeAsync(d_trace, h->stream);
    const regc_status st2 = sync_check(h);
    return st != REGC_OK ? st : st2;
}

// The REGC cycle.  The choice of step t (particle or replica exchange) is a
// function of t alone, so the host reads the whole schedule from the Philox
// stream first and launches each run of steps between two replica exchanges
// as one sweep launch: mps = n_canonical + 1 moves per step, move 0 the
// particle exchange, skipped (m_first = 1) in a step that began with a
// replica exchange.
static regc_status run_cycle(regc_handle* h, int n_steps, double x0, int n_canonical, regc_move_record* trace,
                             int* n_exchanges) {
    if (h && h->P.gc2) return REGC_EINVAL;   // the REGC cycle with one grand-canonical species only
    if (h && h->sharded()) return REGC_EINVAL;   // its replica exchanges need every walker's N and E
    if (!h || n_steps < 0 || n_canonical < 0 || n_canonical > 1023 || !(x0 >= 0.0 && x0 <= 1.0))
        return REGC_EINVAL;
    if (h->sticky != REGC_OK) return h->sticky;
    if (h->need_walkers) return REGC_EINVAL;
    if (n_exchanges) *n_exchanges = 0;
    if (n_steps == 0) return REGC_OK;
    const unsigned long long th_gc =
        x0 >= 1.0 ? (1ull << 32) : (unsigned long long)floor(x0 * 4294967296.0);
    const int mps = n_canonical + 1;
    const size_t n_rec = (size_t)h->S * n_steps * mps;
    regc_move_record* d_trace = nullptr;
    if (trace) {
        const regc_status st = cuda_fail(h, cudaMallocAsync(&d_trace, n_rec * sizeof(regc_move_record), h->stream));
        if (st != REGC_OK) return st;
    }
    SweepParams P = h->P;
    P.cycle = 1;
    P.mps = mps;
    P.trace_steps = n_steps;
    std::vector<char> re_step(n_steps, 0);
    cudaError_t e = cudaSuccess;
    int n_ex = 0;
    auto segment = [&](int a, int len, bool skip) {
        if (e != cudaSuccess || len <= 0 || len * mps <= (skip ? 1 : 0)) return;   // no move to make
        P.t0 = h->t + (uint32_t)a;
        P.n_sweeps = len;
        P.m_first = skip ? 1 : 0;
        P.trace = d_trace ? d_trace + (size_t)a * mps : nullptr;
        e = launch_sweep(P, h->stream);
    };
    int seg = 0;
    bool seg_skip = false;
    for (int ts = 0; ts < n_steps && e == cudaSuccess; ++ts) {
        const U4 G = philox(h->t + (uint32_t)ts, 0u, 0u, 10u, P.key0, P.key1);
        if ((unsigned long long)G.x < th_gc) continue;
        re_step[ts] = 1;
        segment(seg, ts - seg, seg_skip);
        if (e == cudaSuccess) e = launch_exchange(h->X, h->e + (uint32_t)n_ex, h->stream);
        n_ex += 1;
        seg = ts;
        seg_skip = true;
    }
    segment(seg, n_steps - seg, seg_skip);
    regc_status st = cuda_fail(h, e);
    if (st == REGC_OK) {
        h->t += (uint32_t)n_steps;
        h->e += (uint32_t)n_ex;
        if (n_exchanges) *n_exchanges = n_ex;
    }
    if (d_trace) {
        if (st == REGC_OK)
            st = cuda_fail(h, cudaMemcpyAsync(trace, d_trace, n_rec * sizeof(regc_move_record),
                                              cudaMemcpyDeviceToHost, h->stream));
        cudaFreeAsync(d_trace, h->stream);
        const regc_status st2 = sync_check(h);
        if (st == REGC_OK) st = st2;
        if (st == REGC_OK) {
            // the particle exchange of a replica-exchange step is not attempted
            regc_move_record none;
            memset(&none, 0, sizeof none);
            none.type = -1;
            none.status = 4;
            for (int w = 0; w < h->S; ++w)
                for (int ts = 0; ts < n_steps; ++ts)
                    if (re_step[ts]) trace[((size_t)w * n_steps + ts) * mps] = none;
        }
    }
    return st;
}

regc_status regc_cycle(regc_handle* h, int n_steps, double x0, int n_canonical, int* n_exchanges) {
    NvtxRange nvtx_("regc_cycle");
    return run_cycle(h, n_steps, x0, n_canonical, nullptr, n_exchanges);
}

regc_status regc_cycle_traced(regc_handle* h, int n_steps, double x0, int n_canonical, regc_move_record* trace,
                              int* n_exchanges) {
    if (!trace && n_steps > 0) return REGC_EINVAL;
    return run_cycle(h, n_steps, x0, n_canonical, trace, n_exchanges);
}

regc_status regc_cycle_md(regc_handle* h, int n_steps, double x0, int md_steps, float dt, float tau,
                          int* n_exchanges) {
    NvtxRange nvtx_("regc_cycle_md");
    if (!h || n_steps < 0 || md_steps < 0 || !(x0 >= 0.0 && x0 <= 1.0) || !(dt > 0.0f) || !(tau > 0.0f) ||
        !std::isfinite(dt) || !std::isfinite(tau) || h->P.gc2 || h->sharded())
        return REGC_EINVAL;
    if (h->sticky != REGC_OK) return h->sticky;
    if (h->need_walkers) return REGC_EINVAL;
    if (md_smem(h->nmax, h->P.cg.ncell, h->P.cg.cap) > kMaxSmem) return REGC_EINVAL;
    if (n_exchanges) *n_exchanges = 0;
    int total = 0;
    for (int t = 0; t < n_steps; ++t) {
        int ex = 0;
        regc_status st = run_cycle(h, 1, x0, 0, nullptr, &ex);
        if (st == REGC_OK) st = regc_md(h, md_steps, dt, tau, nullptr);
        if (st != REGC_OK) return st;
        total += ex;
    }
    if (n_exchanges) *n_exchanges = total;
    return REGC_OK;
}

regc_status regc_md(regc_handle* h, int n_steps, float dt, float tau, float* kinetic) {
    NvtxRange nvtx_("regc_md");
    if (!h || n_steps < 0 || !(dt > 0.0f) || !(tau > 0.0f) || !std::isfinite(dt) || !std::isfinite(tau))
        return REGC_EINVAL;
    if (h->P.gc2 || h->sharded()) return REGC_EINVAL;   // MD: one grand-canonical species, every walker
    if (h->sticky != REGC_OK) return h->sticky;
    if (h->need_walkers) return REGC_EINVAL;
    if (md_smem(h->nmax, h->P.cg.ncell, h->P.cg.cap) > kMaxSmem) return REGC_EINVAL;
    float* d_kin = nullptr;
    cudaError_t e = cudaMallocAsync(&d_kin, h->S * sizeof(float), h->stream);
    if (e == cudaSuccess) e = launch_md(h->P, n_steps, dt, tau, h->md_seg, d_kin, h->stream);
    // every particle moved: the exact energies from scratch (a pair inside the
    // hard-core guard -- a time step far too long -- is a numeric error)
    if (e == cudaSuccess) e = launch_energy(h->P, h->P.efix, 2, h->stream);
    if (e == cudaSuccess && kinetic)
        e = cudaMemcpyAsync(kinetic, d_kin, h->S * sizeof(float), cudaMemcpyDeviceToHost, h->stream);
    if (d_kin) cudaFreeAsync(d_kin, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e);
    h->md_seg += 1;
    if (kinetic) return sync_check(h);
    return REGC_OK;
}

regc_status regc_set_shard(regc_handle* h, int w_begin, int w_end) {
    if (!h || w_begin < 0 || w_end > h->S || w_begin >= w_end) return REGC_EINVAL;
    if (h->sticky != REGC_OK) return h->sticky;
    h->P.w_begin = w_begin;
    h->P.w_end = w_end;
    return REGC_OK;
}

regc_status regc_get_walker_ne(regc_handle* h, int w_begin, int w_end, int32_t* n, int32_t* nb, int64_t* efix) {
    NvtxRange nvtx_("regc_get_walker_ne");
    if (!h || w_begin < 0 || w_end > h->S || w_begin > w_end || !n || !efix || (h->P.gc2 && !nb))
        return REGC_EINVAL;
    if (h->sticky != REGC_OK) return h->sticky;
    const size_t k = (size_t)(w_end - w_begin);
    if (k == 0) return REGC_OK;
    cudaError_t e = cudaMemcpyAsync(n, h->P.n + w_begin, k * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(efix, h->P.efix + w_begin, k * sizeof(int64_t), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && h->P.gc2)
        e = cudaMemcpyAsync(nb, h->P.nb + w_begin, k * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e);
    return sync_check(h);
}

regc_status regc_set_walker_ne(regc_handle* h, int w_begin, int w_end, const int32_t* n, const int32_t* nb,
                               const int64_t* efix) {
    NvtxRange nvtx_("regc_set_walker_ne");
    if (!h || w_begin < 0 || w_end > h->S || w_begin > w_end || !n || !efix || (h->P.gc2 && !nb))
        return REGC_EINVAL;
    if (h->sticky != REGC_OK) return h->sticky;
    const int k = w_end - w_begin;
    for (int i = 0; i < k; ++i) {
        if (n[i] < 0 || n[i] > h->nmax) return REGC_EINVAL;
        if (h->P.gc2 && (nb[i] < 0 || nb[i] > n[i])) return REGC_EINVAL;
    }
    if (k == 0) return REGC_OK;
    // the host buffers may be pageable: the copies complete before the call returns
    cudaError_t e = cudaMemcpyAsync(h->P.n + w_begin, n, k * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->P.efix + w_begin, efix, k * sizeof(int64_t), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && h->P.gc2)
        e = cudaMemcpyAsync(h->P.nb + w_begin, nb, k * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e);
    return sync_check(h);
}

regc_status regc_exchange(regc_handle* h) {
    NvtxRange nvtx_("regc_exchange");
    if (!h) return REGC_EINVAL;
    if (h->sticky != REGC_OK) return h->sticky;
    const regc_status st = cuda_fail(h, launch_exchange(h->X, h->e, h->stream));
    if (st == REGC_OK) h->e += 1;
    return st;
}

regc_status regc_histograms(regc_handle* h, int64_t* hN, int64_t* hNE, int64_t* omega, double* moments,
                            int64_t* e_out) {
    NvtxRange nvtx_("regc_histograms");
    if (!h) return REGC_EINVAL;
    if (h->sticky != REGC_OK) return h->sticky;
    const size_t S = h->S;
    cudaError_t e = cudaSuccess;
    auto get = [&](void* dst, const void* src, size_t bytes) {
        if (dst && e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, h->stream);
    };
    get(hN, h->P.hN, S * (h->nmax + 1) * 8);
    get(hNE, h->P.hNE, (size_t)h->hist_rows * h->n_e_bins * 8);
    get(omega, h->P.omega, S * 8);
    get(moments, h->P.moments, S * 4 * 8);
    get(e_out, h->P.e_out, S * 8);
    if (e != cudaSuccess) return cuda_fail(h, e);
    return sync_check(h);
}

regc_status regc_histograms2(regc_handle* h, int64_t* hN2, double* moments2) {
    if (!h) return REGC_EINVAL;
    if (h->sticky != REGC_OK) return h->sticky;
    if (!h->P.gc2) return REGC_EINVAL;
    cudaError_t e = cudaSuccess;
    if (hN2) e = cudaMemcpyAsync(hN2, h->P.hN2, (size_t)h->S * (h->nmax + 1) * 8, cudaMemcpyDeviceToHost, h->stream);
    if (moments2 && e == cudaSuccess)
        e = cudaMemcpyAsync(moments2, h->P.moments2, (size_t)h->S * 2 * 8, cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e);
    return sync_check(h);
}

regc_status regc_reset_histograms(regc_handle* h) {
    if (!h) return REGC_EINVAL;
    if (h->sticky != REGC_OK) return h->sticky;
    const size_t S = h->S;
    cudaError_t e = cudaSuccess;
    auto zero = [&](void* p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMemsetAsync(p, 0, bytes, h->stream);
    };
    zero(h->P.hN, S * (h->nmax + 1) * 8);
    zero(h->P.hNE, (size_t)h->hist_rows * h->n_e_bins * 8);
    if (h->P.gc2) {
        zero(h->P.hN2, S * (h->nmax + 1) * 8);
        zero(h->P.moments2, S * 2 * 8);
    }
    zero(h->P.omega, S * 8);
    zero(h->P.moments, S * 4 * 8);
    zero(h->P.e_out, S * 8);
    zero(h->P.move_counts, S * 6 * 8);
    zero(h->X.ex_counts, S * 2 * h->n_dir * 8);
    zero(h->P.pair_counts, 6 * 8);
    if (h->P.hE) zero(h->P.hE, S * (size_t)(h->P.hE_bins + 2) * 8);
    return cuda_fail(h, e);
}

regc_status regc_set_state_windows(regc_handle* h, int n_bins, double e_bin, const double* e_lo) {
    if (!h || n_bins < 0 || n_bins > (1 << 20)) return REGC_EINVAL;
    if (h->sticky != REGC_OK) return h->sticky;
    if (n_bins > 0 && !(e_bin * kFixPerUnit >= 1.0 && e_bin < 4294967296.0)) return REGC_EINVAL;
    const size_t S = h->S;
    std::vector<long long> lo_fix(S, 0);
    long long bin_fix = 0;
    if (n_bins > 0) {
        bin_fix = llround(e_bin * kFixPerUnit);
        std::vector<double> lo(S);
        if (e_lo) {
            for (size_t s = 0; s < S; ++s) lo[s] = e_lo[s];
        } else {
            // centred on each state's mean energy observed so far (0 if never observed)
            std::vector<double> mom(S * 4);
            std::vector<unsigned long long> om(S);
            cudaError_t e = cudaMemcpyAsync(mom.data(), h->P.moments, S * 4 * 8, cudaMemcpyDeviceToHost, h->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(om.data(), h->P.omega, S * 8, cudaMemcpyDeviceToHost, h->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
            if (e != cudaSuccess) return cuda_fail(h, e);
            for (size_t s = 0; s < S; ++s)
                lo[s] = (om[s] ? mom[4 * s + 2] / (double)om[s] : 0.0) - 0.5 * n_bins * ((double)bin_fix * kFixUnit);
        }
        for (size_t s = 0; s < S; ++s) {
            if (!std::isfinite(lo[s]) || !(fabs(lo[s]) < 4294967296.0)) return REGC_EINVAL;
            lo_fix[s] = llround(lo[s] * kFixPerUnit);
        }
    }
    // (re)allocate: the old block may still be read by queued sweeps
    if (h->hE_block) {
        cudaError_t e = cudaStreamSynchronize(h->stream);
        if (e == cudaSuccess) e = cudaFree(h->hE_block);
        h->hE_block = nullptr;
        h->P.hE = nullptr;
        h->P.hE_lo_fix = nullptr;
        h->P.hE_bins = 0;
        if (e != cudaSuccess) return cuda_fail(h, e);
    }
    if (n_bins == 0) return REGC_OK;
    const size_t hist_bytes = S * (size_t)(n_bins + 2) * 8;
    void* block = nullptr;
    cudaError_t e = cudaMalloc(&block, hist_bytes + S * 8);
    if (e != cudaSuccess) return cuda_fail(h, e);
    h->hE_block = block;
    h->P.hE = static_cast<unsigned long long*>(block);
    long long* d_lo = reinterpret_cast<long long*>(static_cast<char*>(block) + hist_bytes);
    h->P.hE_lo_fix = d_lo;
    h->P.hE_bin_fix = bin_fix;
    h->P.hE_bins = n_bins;
    e = cudaMemsetAsync(block, 0, hist_bytes, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_lo, lo_fix.data(), S * 8, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);   // lo_fix is a host temporary
    return cuda_fail(h, e);
}

regc_status regc_state_histograms(regc_handle* h, int64_t* hE, double* e_lo, double* e_bin) {
    if (!h) return REGC_EINVAL;
    if (h->sticky != REGC_OK) return h->sticky;
    if (!h->P.hE) return REGC_EINVAL;
    const size_t S = h->S;
    std::vector<long long> lo(S);
    cudaError_t e = cudaSuccess;
    if (hE) e = cudaMemcpyAsync(hE, h->P.hE, S * (size_t)(h->P.hE_bins + 2) * 8, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(lo.data(), h->P.hE_lo_fix, S * 8, cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e);
    const regc_status st = sync_check(h);
    if (st != REGC_OK) return st;
    if (e_lo)
        for (size_t s = 0; s < S; ++s) e_lo[s] = (double)lo[s] * kFixUnit;
    if (e_bin) *e_bin = (double)h->P.hE_bin_fix * kFixUnit;
    return REGC_OK;
}

namespace {

// The device address of a host buffer the GPU can read and write directly
// (page-locked memory, which unified addressing maps into the device's
// address space; on a Grace-Blackwell node the accesses run over NVLink-C2C),
// else null: the caller's positions are then read or written by the pack and
// unpack kernels themselves instead of through a staged copy.
void* device_view(const void* host) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

}  // namespace

regc_status regc_set_walkers(regc_handle* h, const float* pos, const int32_t* n, const int32_t* sow) {
    return regc_set_walkers2(h, pos, n, nullptr, sow);
}

regc_status regc_set_walkers2(regc_handle* h, const float* pos, const int32_t* n, const int32_t* nb,
                              const int32_t* sow) {
    NvtxRange nvtx_("regc_set_walkers2");
    if (!h || !pos || !n) return REGC_EINVAL;
    if (h->sticky != REGC_OK) return h->sticky;
    const int S = h->S, nmax = h->nmax;
    for (int w = 0; w < S; ++w)
        if (n[w] < h->P.n_cluster || n[w] > nmax || (nb && (nb[w] < 0 || nb[w] > n[w]))) return REGC_EINVAL;
    // walker of each state, built in the pinned staging area (asynchronous copy)
    int* flag = static_cast<int*>(h->h_stage);
    int* wos = reinterpret_cast<int*>(static_cast<char*>(h->h_stage) + 64);
    if (sow) {
        for (int k = 0; k < S; ++k) wos[k] = -1;
        for (int w = 0; w < S; ++w) {
            if (sow[w] < 0 || sow[w] >= S || wos[sow[w]] >= 0) return REGC_EINVAL;
            wos[sow[w]] = w;
        }
    }
    // repacking and the coordinate checks run on the device, reading a
    // page-locked caller buffer in place, else one copy of it
    const float* src = static_cast<const float*>(device_view(pos));
    cudaError_t e = cudaSuccess;
    if (!src) {
        e = cudaMemcpyAsync(h->d_xyz, pos, (size_t)S * nmax * 3 * sizeof(float), cudaMemcpyHostToDevice, h->stream);
        src = h->d_xyz;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->P.n, n, S * sizeof(int), cudaMemcpyHostToDevice, h->stream);
    // species B's counts (without them every particle is B)
    if (e == cudaSuccess && h->P.gc2)
        e = cudaMemcpyAsync(h->P.nb, nb ? nb : n, S * sizeof(int), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && sow)
        e = cudaMemcpyAsync(h->X.state_of_walker, sow, S * sizeof(int), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && sow)
        e = cudaMemcpyAsync(h->X.walker_of_state, wos, S * sizeof(int), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_error, 0, sizeof(int), h->stream);
    if (e == cudaSuccess) e = pack_walkers(src, h->P.n, S, nmax, h->P.g, h->P.pos, h->d_error, h->stream);
    if (e == cudaSuccess) e = launch_energy(h->P, h->P.efix, 1, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(flag, h->d_error, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e);
    if (*flag & (ERR_OVERLAP | ERR_INPUT)) {
        // leave a consistent state behind: no walker holds particles
        cudaMemsetAsync(h->P.n, 0, S * sizeof(int), h->stream);
        cudaMemsetAsync(h->P.efix, 0, S * sizeof(long long), h->stream);
        cudaMemsetAsync(h->d_error, 0, sizeof(int), h->stream);
        cudaStreamSynchronize(h->stream);
        h->need_walkers = h->P.n_cluster > 0;
        return REGC_EINVAL;
    }
    h->need_walkers = false;
    return REGC_OK;
}

regc_status regc_set_cluster(regc_handle* h, int n_cluster, int cluster_type) {
    if (!h || n_cluster < 0 || n_cluster >= h->nmax || h->P.gc2) return REGC_EINVAL;
    if (n_cluster > 0 && (cluster_type < 1 || cluster_type >= h->n_types)) return REGC_EINVAL;
    if (h->sticky != REGC_OK) return h->sticky;
    SweepParams& P = h->P;
    const int ct = n_cluster > 0 ? cluster_type : 0;
    auto tab = [&](int a, int b) {
        return PairTab{4.0f * h->eps[a][b], h->sigma[a][b] * h->sigma[a][b],
                       hard_core_r2(h->eps[a][b], h->sigma[a][b], h->hard_core_T), h->eps[a][b]};
    };
    P.n_cluster = n_cluster;
    P.gA = tab(ct, ct);
    P.gAB = tab(0, ct);
    for (int t = 0; t < 4; ++t) P.gsA[t] = tab(ct, t < h->n_types ? t : 0);
    // every walker must now hold the cluster: empty them until regc_set_walkers
    cudaError_t e = cudaMemsetAsync(P.n, 0, h->S * sizeof(int), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(P.efix, 0, h->S * sizeof(long long), h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    h->need_walkers = n_cluster > 0;
    return cuda_fail(h, e);
}

regc_status regc_get_walkers(regc_handle* h, float* pos, int32_t* n, double* energy, int32_t* sow) {
    return regc_get_walkers2(h, pos, n, nullptr, energy, sow);
}

regc_status regc_get_walkers2(regc_handle* h, float* pos, int32_t* n, int32_t* nb, double* energy, int32_t* sow) {
    NvtxRange nvtx_("regc_get_walkers2");
    if (!h) return REGC_EINVAL;
    if (h->sticky != REGC_OK) return h->sticky;
    if (nb && !h->P.gc2) return REGC_EINVAL;
    const int S = h->S, nmax = h->nmax;
    long long* ef = reinterpret_cast<long long*>(static_cast<char*>(h->h_stage) + 64);   // pinned
    cudaError_t e = cudaSuccess;
    if (pos) {
        // a page-locked caller buffer is written in place by the unpacking kernel
        float* dst = static_cast<float*>(device_view(pos));
        e = unpack_walkers(h->P.pos, (long long)S * nmax, nmax, dst ? h->P.n : nullptr, dst ? dst : h->d_xyz,
                           h->stream);
        if (e == cudaSuccess && !dst)
            e = cudaMemcpyAsync(pos, h->d_xyz, (size_t)S * nmax * 3 * sizeof(float), cudaMemcpyDeviceToHost,
                                h->stream);
    }
    if (n && e == cudaSuccess) e = cudaMemcpyAsync(n, h->P.n, S * sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (nb && e == cudaSuccess) e = cudaMemcpyAsync(nb, h->P.nb, S * sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (energy && e == cudaSuccess)
        e = cudaMemcpyAsync(ef, h->P.efix, S * sizeof(long long), cudaMemcpyDeviceToHost, h->stream);
    if (sow && e == cudaSuccess)
        e = cudaMemcpyAsync(sow, h->X.state_of_walker, S * sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e);
    const regc_status st = sync_check(h);
    if (st != REGC_OK) return st;
    if (energy)
        for (int w = 0; w < S; ++w) energy[w] = (double)ef[w] * kFixUnit;
    return REGC_OK;
}

regc_status regc_check_energy(regc_handle* h, double* max_drift) {
    if (!h) return REGC_EINVAL;
    if (h->sticky != REGC_OK) return h->sticky;
    regc_status st = cuda_fail(h, launch_energy(h->P, h->d_fix, 0, h->stream));
    if (st != REGC_OK) return st;
    std::vector<long long> a(h->S), b(h->S);
    cudaError_t e = cudaMemcpyAsync(a.data(), h->d_fix, h->S * 8, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b.data(), h->P.efix, h->S * 8, cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e);
    st = sync_check(h);
    if (st != REGC_OK) return st;
    double d = 0.0;
    // under a shard the other walkers' positions here are stale: only the
    // shard's walkers are checked
    for (int w = h->P.w_begin; w < h->P.w_end; ++w) d = std::max(d, fabs((double)(a[w] - b[w]) * kFixUnit));
    if (max_drift) *max_drift = d;
    return REGC_OK;
}

regc_status regc_warps_per_walker(const regc_handle* h, int* warps) {
    if (!h || !warps) return REGC_EINVAL;
    *warps = h->P.warps_per_walker;
    return REGC_OK;
}

regc_status regc_counters(regc_handle* h, int64_t* moves, int64_t* exchanges, int64_t* pairs) {
    if (!h) return REGC_EINVAL;
    if (h->sticky != REGC_OK) return h->sticky;
    cudaError_t e = cudaSuccess;
    if (moves) e = cudaMemcpyAsync(moves, h->P.move_counts, (size_t)h->S * 6 * 8, cudaMemcpyDeviceToHost, h->stream);
    if (exchanges && e == cudaSuccess)
        e = cudaMemcpyAsync(exchanges, h->X.ex_counts, (size_t)h->S * 2 * h->n_dir * 8, cudaMemcpyDeviceToHost,
                            h->stream);
    if (pairs && e == cudaSuccess)
        e = cudaMemcpyAsync(pairs, h->P.pair_counts, 6 * 8, cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e);
    return sync_check(h);
}

// ------------------------------------------------------------ checkpoint

namespace {

// Byte layout of a checkpoint: this header, then the sections of
// ckpt_sections() in order, raw.
struct CkptHeader {
    char magic[8];             // "REGCCKPT"
    uint32_t version;          // 3
    uint32_t flags;            // bit 0: surrogate present, bit 1: delayed-acceptance mode
    int32_t S, nmax, n_e_bins, n_cluster;
    uint32_t key0, key1, t, e;
    int32_t adam_t;
    uint32_t harvest_round;
    uint32_t md_seg;
    int32_t hE_bins;           // per-state energy windows (0: none)
    int64_t hE_bin_fix;
    uint64_t payload_bytes;
    uint64_t checksum;         // FNV-1a 64 of the payload
};

struct Section {
    void* dev;
    size_t bytes;
};

std::vector<Section> ckpt_sections(regc_handle* h, bool with_sur) {
    const size_t S = h->S, nb = h->nmax + 1;
    std::vector<Section> v = {
        {h->P.pos, S * h->nmax * sizeof(float4)},
        {h->P.n, S * sizeof(int)},
        {h->P.efix, S * sizeof(long long)},
        {h->X.state_of_walker, S * sizeof(int)},
        {h->X.walker_of_state, S * sizeof(int)},
        {h->P.hN, S * nb * 8},
        {h->P.hNE, (size_t)h->hist_rows * h->n_e_bins * 8},
        {h->P.omega, S * 8},
        {h->P.moments, S * 4 * 8},
        {h->P.e_out, S * 8},
        {h->P.move_counts, S * 6 * 8},
        {h->X.ex_counts, S * 2 * h->n_dir * 8},
        {h->P.pair_counts, 6 * 8},
    };
    if (h->P.gc2) {
        v.push_back({h->P.nb, S * sizeof(int)});
        v.push_back({h->P.hN2, S * nb * 8});
        v.push_back({h->P.moments2, S * 2 * 8});
    }
    if (h->P.hE) {
        v.push_back({h->P.hE, S * (size_t)(h->P.hE_bins + 2) * 8});
        v.push_back({const_cast<long long*>(h->P.hE_lo_fix), S * 8});
    }
    if (with_sur) {
        v.push_back({h->d_theta, REGC_SURROGATE_PARAMS * sizeof(float)});
        v.push_back({h->d_adam_m, REGC_SURROGATE_PARAMS * sizeof(float)});
        v.push_back({h->d_adam_v, REGC_SURROGATE_PARAMS * sizeof(float)});
    }
    return v;
}

uint64_t fnv1a(const unsigned char* p, size_t n) {
    uint64_t x = 1469598103934665603ull;
    for (size_t i = 0; i < n; ++i) {
        x ^= p[i];
        x *= 1099511628211ull;
    }
    return x;
}

regc_status surrogate_alloc(regc_handle* h);
regc_status surrogate_loaded(regc_handle* h);

}  // namespace

regc_status regc_checkpoint(regc_handle* h, void* buf, size_t capacity, size_t* length) {
    NvtxRange nvtx_("regc_checkpoint");
    if (!h || !length) return REGC_EINVAL;
    if (h->sticky != REGC_OK) return h->sticky;
    const auto secs = ckpt_sections(h, h->has_sur);
    size_t payload = 0;
    for (const auto& x : secs) payload += x.bytes;
    *length = sizeof(CkptHeader) + payload;
    if (!buf) return REGC_OK;
    if (capacity < *length) return REGC_EINVAL;
    unsigned char* out = static_cast<unsigned char*>(buf);
    unsigned char* q = out + sizeof(CkptHeader);
    cudaError_t e = cudaSuccess;
    for (const auto& x : secs) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(q, x.dev, x.bytes, cudaMemcpyDeviceToHost, h->stream);
        q += x.bytes;
    }
    if (e != cudaSuccess) return cuda_fail(h, e);
    const regc_status st = sync_check(h);
    if (st != REGC_OK) return st;
    CkptHeader hd{};
    memcpy(hd.magic, "REGCCKPT", 8);
    hd.version = 3;
    hd.flags = (h->has_sur ? 1u : 0u) | (h->P.delayed ? 2u : 0u) | (h->P.gc2 ? 4u : 0u);
    hd.S = h->S;
    hd.nmax = h->nmax;
    hd.n_e_bins = h->n_e_bins;
    hd.n_cluster = h->P.n_cluster;
    hd.key0 = h->P.key0;
    hd.key1 = h->P.key1;
    hd.t = h->t;
    hd.e = h->e;
    hd.adam_t = h->adam_t;
    hd.harvest_round = h->harvest_round;
    hd.md_seg = h->md_seg;
    hd.hE_bins = h->P.hE_bins;
    hd.hE_bin_fix = h->P.hE_bin_fix;
    hd.payload_bytes = payload;
    hd.checksum = fnv1a(out + sizeof(CkptHeader), payload);
    memcpy(out, &hd, sizeof hd);
    return REGC_OK;
}

regc_status regc_restore(regc_handle* h, const void* buf, size_t length) {
    NvtxRange nvtx_("regc_restore");
    if (!h || !buf || length < sizeof(CkptHeader)) return REGC_EINVAL;
    if (h->sticky != REGC_OK) return h->sticky;
    CkptHeader hd;
    memcpy(&hd, buf, sizeof hd);
    const unsigned char* in = static_cast<const unsigned char*>(buf);
    if (memcmp(hd.magic, "REGCCKPT", 8) != 0 || hd.version != 3) return REGC_EINVAL;
    if (hd.S != h->S || hd.nmax != h->nmax || hd.n_e_bins != h->n_e_bins || hd.n_cluster != h->P.n_cluster ||
        ((hd.flags & 4u) != 0) != (h->P.gc2 != 0) ||
        hd.key0 != h->P.key0 || hd.key1 != h->P.key1 || hd.hE_bins != h->P.hE_bins)
        return REGC_EINVAL;
    const bool with_sur = (hd.flags & 1u) != 0;
    if (with_sur) {
        const regc_status st = surrogate_alloc(h);
        if (st != REGC_OK) return st;
    }
    const auto secs = ckpt_sections(h, with_sur);
    size_t payload = 0;
    for (const auto& x : secs) payload += x.bytes;
    if (hd.payload_bytes != payload || length != sizeof(CkptHeader) + payload) return REGC_EINVAL;
    if (fnv1a(in + sizeof(CkptHeader), payload) != hd.checksum) return REGC_EINVAL;
    const unsigned char* q = in + sizeof(CkptHeader);
    cudaError_t e = cudaSuccess;
    for (const auto& x : secs) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(x.dev, q, x.bytes, cudaMemcpyHostToDevice, h->stream);
        q += x.bytes;
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_error, 0, sizeof(int), h->stream);
    if (e == cudaSuccess && with_sur) e = surrogate_pack(h->d_theta, h->sur, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e);
    h->t = hd.t;
    h->e = hd.e;
    h->adam_t = hd.adam_t;
    h->harvest_round = hd.harvest_round;
    h->md_seg = hd.md_seg;
    h->P.hE_bin_fix = hd.hE_bin_fix;
    h->P.delayed = (with_sur && (hd.flags & 2u)) ? 1 : 0;
    h->need_walkers = false;
    return REGC_OK;
}

// ------------------------------------------------------------- surrogate

namespace {

regc_status surrogate_alloc(regc_handle* h) {
    if (h->has_sur) return REGC_OK;
    const size_t np = REGC_SURROGATE_PARAMS;
    regc_status st = dalloc(h, &h->d_theta, np);
    if (st == REGC_OK) st = dalloc(h, &h->d_adam_m, np);
    if (st == REGC_OK) st = dalloc(h, &h->d_adam_v, np);
    if (st == REGC_OK) st = dalloc(h, &h->sur.w1, 64 * 16);
    if (st == REGC_OK) st = dalloc(h, &h->sur.b1, 64);
    if (st == REGC_OK) st = dalloc(h, &h->sur.w2, 64 * 64);
    if (st == REGC_OK) st = dalloc(h, &h->sur.b2, 64);
    if (st == REGC_OK) st = dalloc(h, &h->sur.w3, 64);
    if (st == REGC_OK) st = dalloc(h, &h->sur.b3, 1);
    if (st != REGC_OK) return st;
    h->P.net = SurrogateDev{h->sur.w1, h->sur.b1, h->sur.w2, h->sur.b2, h->sur.w3, h->sur.b3};
    h->has_sur = true;
    return REGC_OK;
}

// Reset the optimiser and refresh the inference copy after new master parameters.
regc_status surrogate_loaded(regc_handle* h) {
    cudaError_t e = cudaMemsetAsync(h->d_adam_m, 0, REGC_SURROGATE_PARAMS * sizeof(float), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_adam_v, 0, REGC_SURROGATE_PARAMS * sizeof(float), h->stream);
    if (e == cudaSuccess) e = surrogate_pack(h->d_theta, h->sur, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    h->adam_t = 0;
    return cuda_fail(h, e);
}

}  // namespace

regc_status regc_surrogate_init(regc_handle* h, uint64_t seed, float scale) {
    if (!h || !(scale >= 0.0f) || !std::isfinite(scale)) return REGC_EINVAL;
    if (h->sticky != REGC_OK) return h->sticky;
    const regc_status st = surrogate_alloc(h);
    if (st != REGC_OK) return st;
    const cudaError_t e = surrogate_init(h->d_theta, scale, (uint32_t)seed, (uint32_t)(seed >> 32), h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e);
    return surrogate_loaded(h);
}

regc_status regc_surrogate_set(regc_handle* h, const float* theta) {
    if (!h || !theta) return REGC_EINVAL;
    if (h->sticky != REGC_OK) return h->sticky;
    for (int i = 0; i < REGC_SURROGATE_PARAMS; ++i)
        if (!std::isfinite(theta[i])) return REGC_EINVAL;
    regc_status st = surrogate_alloc(h);
    if (st != REGC_OK) return st;
    const cudaError_t e = cudaMemcpyAsync(h->d_theta, theta, REGC_SURROGATE_PARAMS * sizeof(float),
                                          cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e);
    return surrogate_loaded(h);
}

regc_status regc_surrogate_get(regc_handle* h, float* theta) {
    if (!h || !theta) return REGC_EINVAL;
    if (h->sticky != REGC_OK) return h->sticky;
    if (!h->has_sur) return REGC_EINVAL;
    cudaError_t e = cudaMemcpyAsync(theta, h->d_theta, REGC_SURROGATE_PARAMS * sizeof(float),
                                    cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e);
    return sync_check(h);
}

regc_status regc_set_mode(regc_handle* h, int mode) {
    if (!h || (mode != 0 && mode != 1)) return REGC_EINVAL;
    if (mode == 1 && h->P.gc2) return REGC_EINVAL;   // delayed acceptance with one species only
    if (mode == 1 && !h->has_sur) return REGC_EINVAL;
    h->P.delayed = mode;
    return REGC_OK;
}

regc_status regc_surrogate_eval(regc_handle* h, int walker, int n_query, const float* xyz, float* e_out,
                                float* features) {
    if (!h || walker < 0 || walker >= h->S || n_query < 0 || (n_query > 0 && (!xyz || !e_out)) || h->P.gc2)
        return REGC_EINVAL;
    if (h->sticky != REGC_OK) return h->sticky;
    if (!h->has_sur) return REGC_EINVAL;
    if (n_query == 0) return REGC_OK;
    std::vector<float4> q(n_query);
    for (int i = 0; i < n_query; ++i) {
        const float* r = xyz + 3 * i;
        const bool okx = r[0] >= 0.0f && r[0] < h->Lx, oky = r[1] >= 0.0f && r[1] < h->Ly;
        const bool okz = h->periodic_z ? (r[2] >= 0.0f && r[2] < h->Lz) : (r[2] >= h->z_lo && r[2] <= h->z_hi);
        if (!(okx && oky && okz)) return REGC_EINVAL;
        q[i] = make_float4(r[0], r[1], r[2], 0.0f);
    }
    float4* d_q = nullptr;
    float *d_e = nullptr, *d_f = nullptr;
    cudaError_t e = cudaMallocAsync(&d_q, n_query * sizeof(float4), h->stream);
    if (e == cudaSuccess) e = cudaMallocAsync(&d_e, n_query * sizeof(float), h->stream);
    if (e == cudaSuccess) e = cudaMallocAsync(&d_f, (size_t)n_query * 16 * sizeof(float), h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_q, q.data(), n_query * sizeof(float4), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = surrogate_eval(h->P, walker, n_query, d_q, d_e, d_f, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(e_out, d_e, n_query * sizeof(float), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && features)
        e = cudaMemcpyAsync(features, d_f, (size_t)n_query * 16 * sizeof(float), cudaMemcpyDeviceToHost, h->stream);
    if (d_q) cudaFreeAsync(d_q, h->stream);
    if (d_e) cudaFreeAsync(d_e, h->stream);
    if (d_f) cudaFreeAsync(d_f, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e);
    return sync_check(h);
}

regc_status regc_surrogate_harvest(regc_handle* h, int particles, int probes, float e_clip, int capacity,
                                   int64_t* n_rows) {
    NvtxRange nvtx_("regc_surrogate_harvest");
    if (!h || particles < 0 || probes < 0 || capacity < 0 || std::isnan(e_clip) || h->P.gc2 || h->sharded())
        return REGC_EINVAL;
    if (h->sticky != REGC_OK) return h->sticky;
    if (h->ds_cap == 0) {
        if (capacity < 1) return REGC_EINVAL;
        regc_status st = dalloc(h, &h->d_X, (size_t)capacity * 16);
        if (st == REGC_OK) st = dalloc(h, &h->d_y, (size_t)capacity);
        if (st != REGC_OK) return st;
        h->ds_cap = capacity;
    } else if (capacity != 0 && capacity != h->ds_cap) {
        return REGC_EINVAL;
    }
    const long long rows = (long long)h->S * (particles + probes);
    if (rows > (1LL << 31) - 1) return REGC_EINVAL;
    const regc_status st = cuda_fail(h, surrogate_harvest(h->P, particles, probes, e_clip, h->harvest_round, h->d_X,
                                                          h->d_y, h->ds_next, h->ds_cap, h->stream));
    if (st != REGC_OK) return st;
    h->harvest_round += 1;
    h->ds_next = (int)((h->ds_next + rows) % h->ds_cap);
    h->ds_count = (int)std::min<long long>(h->ds_cap, h->ds_count + rows);
    if (n_rows) *n_rows = h->ds_count;
    return REGC_OK;
}

regc_status regc_surrogate_set_dataset(regc_handle* h, int64_t n_rows, const float* X, const float* y,
                                       int capacity) {
    if (!h || n_rows < 0 || capacity < 0 || (n_rows > 0 && (!X || !y))) return REGC_EINVAL;
    if (h->sticky != REGC_OK) return h->sticky;
    for (int64_t i = 0; i < n_rows * 16; ++i)
        if (!std::isfinite(X[i])) return REGC_EINVAL;
    for (int64_t i = 0; i < n_rows; ++i)
        if (!std::isfinite(y[i])) return REGC_EINVAL;
    if (h->ds_cap == 0) {
        if (capacity < 1 || n_rows > capacity) return REGC_EINVAL;
        regc_status st = dalloc(h, &h->d_X, (size_t)capacity * 16);
        if (st == REGC_OK) st = dalloc(h, &h->d_y, (size_t)capacity);
        if (st != REGC_OK) return st;
        h->ds_cap = capacity;
    } else if ((capacity != 0 && capacity != h->ds_cap) || n_rows > h->ds_cap) {
        return REGC_EINVAL;
    }
    cudaError_t e = cudaSuccess;
    if (n_rows > 0) {
        e = cudaMemcpyAsync(h->d_X, X, (size_t)n_rows * 16 * sizeof(float), cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h->d_y, y, (size_t)n_rows * sizeof(float), cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);   // the host rows may go away
    }
    if (e != cudaSuccess) return cuda_fail(h, e);
    h->ds_count = (int)n_rows;
    h->ds_next = (int)(n_rows % h->ds_cap);
    return REGC_OK;
}

regc_status regc_surrogate_dataset(regc_handle* h, int64_t max_rows, float* X, float* y, int64_t* n_rows) {
    if (!h) return REGC_EINVAL;
    if (h->sticky != REGC_OK) return h->sticky;
    if (n_rows) *n_rows = h->ds_count;
    if ((X || y) && max_rows < h->ds_count) return REGC_EINVAL;
    cudaError_t e = cudaSuccess;
    if (X && h->ds_count > 0)
        e = cudaMemcpyAsync(X, h->d_X, (size_t)h->ds_count * 16 * sizeof(float), cudaMemcpyDeviceToHost, h->stream);
    if (y && h->ds_count > 0 && e == cudaSuccess)
        e = cudaMemcpyAsync(y, h->d_y, (size_t)h->ds_count * sizeof(float), cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e);
    return sync_check(h);
}

regc_status regc_surrogate_train(regc_handle* h, int steps, int batch, float lr, float* loss) {
    NvtxRange nvtx_("regc_surrogate_train");
    if (!h || steps < 0 || batch < 1 || !(lr >= 0.0f) || !std::isfinite(lr)) return REGC_EINVAL;
    if (h->sticky != REGC_OK) return h->sticky;
    if (!h->has_sur || h->ds_count == 0) return REGC_EINVAL;
    if (steps == 0) return REGC_OK;
    int* d_idx = nullptr;
    float *d_part = nullptr, *d_loss = nullptr;
    cudaError_t e = cudaMallocAsync(&d_idx, batch * sizeof(int), h->stream);
    if (e == cudaSuccess) e = cudaMallocAsync(&d_part, surrogate_partial_floats(batch) * sizeof(float), h->stream);
    if (e == cudaSuccess) e = cudaMallocAsync(&d_loss, steps * sizeof(float), h->stream);
    for (int k = 0; k < steps && e == cudaSuccess; ++k) {
        h->adam_t += 1;
        e = surrogate_batch_index(d_idx, batch, h->ds_count, (uint32_t)h->adam_t, h->P.key0, h->P.key1, h->stream);
        if (e == cudaSuccess)
            e = surrogate_step(h->d_theta, h->d_X, h->d_y, d_idx, batch, d_part, nullptr, d_loss + k, h->d_theta,
                               h->d_adam_m, h->d_adam_v, h->adam_t, lr, true, h->stream);
    }
    if (e == cudaSuccess) e = surrogate_pack(h->d_theta, h->sur, h->stream);
    std::vector<float> lsum(steps);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(lsum.data(), d_loss, steps * sizeof(float), cudaMemcpyDeviceToHost, h->stream);
    if (d_idx) cudaFreeAsync(d_idx, h->stream);
    if (d_part) cudaFreeAsync(d_part, h->stream);
    if (d_loss) cudaFreeAsync(d_loss, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e);
    const regc_status st = sync_check(h);
    if (st == REGC_OK && loss)
        for (int k = 0; k < steps; ++k) loss[k] = lsum[k] / (float)batch;
    return st;
}

}  // extern "C"

namespace {

regc_status surrogate_gradient_on(int n, const float* theta, const float* X, const float* y, float* loss,
                                  float* grad, void* cuda_stream, bool tensor_cores) {
    if (n < 1 || !theta || !X || !y) return REGC_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    float *d_theta = nullptr, *d_X = nullptr, *d_y = nullptr, *d_part = nullptr, *d_grad = nullptr,
          *d_loss = nullptr;
    cudaError_t e = cudaMallocAsync(&d_theta, REGC_SURROGATE_PARAMS * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMallocAsync(&d_X, (size_t)n * 16 * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMallocAsync(&d_y, (size_t)n * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMallocAsync(&d_part, surrogate_partial_floats(n) * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMallocAsync(&d_grad, REGC_SURROGATE_PARAMS * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMallocAsync(&d_loss, sizeof(float), s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_theta, theta, REGC_SURROGATE_PARAMS * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_X, X, (size_t)n * 16 * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_y, y, (size_t)n * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = surrogate_step(d_theta, d_X, d_y, nullptr, n, d_part, d_grad, d_loss, nullptr, nullptr, nullptr, 0, 0.0f,
                           tensor_cores, s);
    float l = 0.0f;
    if (e == cudaSuccess && grad)
        e = cudaMemcpyAsync(grad, d_grad, REGC_SURROGATE_PARAMS * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&l, d_loss, sizeof(float), cudaMemcpyDeviceToHost, s);
    for (float* p : {d_theta, d_X, d_y, d_part, d_grad, d_loss})
        if (p) cudaFreeAsync(p, s);
    const cudaError_t e2 = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? REGC_ENOMEM : REGC_ECUDA;
    if (loss) *loss = l / (float)n;
    return REGC_OK;
}

}  // namespace

extern "C" {

regc_status regc_surrogate_gradient(int n, const float* theta, const float* X, const float* y, float* loss,
                                    float* grad, void* cuda_stream) {
    return surrogate_gradient_on(n, theta, X, y, loss, grad, cuda_stream, false);
}

regc_status regc_surrogate_gradient_bf16(int n, const float* theta, const float* X, const float* y, float* loss,
                                         float* grad, void* cuda_stream) {
    return surrogate_gradient_on(n, theta, X, y, loss, grad, cuda_stream, true);
}

}  // extern "C"

// ------------------------------------------------------------------- MBAR

namespace {

struct MbarBuffers {
    std::vector<void*> ptrs;
    cudaStream_t s;
    cudaError_t err = cudaSuccess;
    template <class T>
    T* get(size_t count) {
        void* p = nullptr;
        if (err == cudaSuccess) err = cudaMallocAsync(&p, std::max<size_t>(count, 1) * sizeof(T), s);
        if (err == cudaSuccess) ptrs.push_back(p);
        return static_cast<T*>(p);
    }
    ~MbarBuffers() {
        for (void* p : ptrs) cudaFreeAsync(p, s);
        cudaStreamSynchronize(s);
    }
};

// energy bins merged for the warm start of the handle's reweighting
constexpr double kWarmBins = 16.0;

regc_status status_of(cudaError_t e) {
    return e == cudaSuccess ? REGC_OK : (e == cudaErrorMemoryAllocation ? REGC_ENOMEM : REGC_ECUDA);
}

// Solve over bins already on the device, then answer Q host queries.
// The runs of equal (N, N2) of m's bins, for the query (m.run_start, m.n_runs).
cudaError_t with_runs(MbarBuffers& buf, MbarDev& m, cudaStream_t s) {
    long long* scratch = buf.get<long long>(mbar_runs_scratch(m.B));
    int* run_start = buf.get<int>(size_t(m.B) + 1);
    if (buf.err != cudaSuccess) return buf.err;
    int n_runs = 0;
    const cudaError_t e = mbar_runs_dev(m, scratch, run_start, &n_runs, s);
    if (e == cudaSuccess) {
        m.run_start = run_start;
        m.n_runs = n_runs;
    }
    return e;
}

// warm_width > 0: started from the solve coarsened to energy bins of that width.
cudaError_t solve_and_query(MbarBuffers& buf, MbarDev& m, double lambda0, double tol, int max_iter, int* iters,
                            double* f_host, double* D_host, int Q, const double* kT_q, const double* mu_q,
                            int nmax, double* N_mean, double* pN, double* f_q, double warm_width = 0.0) {
    cudaStream_t s = buf.s;
    m.f = buf.get<double>(m.S);
    m.f_new = buf.get<double>(m.S);
    m.D = buf.get<double>(m.B);
    m.EN32 = buf.get<float2>(m.B);
    m.DH32 = buf.get<float>(m.B);
    m.delta = buf.get<double>(1);
    m.state = buf.get<int>(2);
    if (buf.err != cudaSuccess) return buf.err;
    cudaError_t e = mbar_solve_warm_dev(m, warm_width, tol, max_iter, iters, s);
    if (e != cudaSuccess) return e;
    if (f_host) e = cudaMemcpyAsync(f_host, m.f, m.S * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && D_host) e = cudaMemcpyAsync(D_host, m.D, m.B * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    if (Q > 0) {
        double* d_kq = buf.get<double>(Q);
        double* d_mq = buf.get<double>(Q);
        double* a_q = buf.get<double>(Q);
        double* c_q = buf.get<double>(Q);
        double* d_nm = buf.get<double>(Q);
        double* d_pn = buf.get<double>((size_t)Q * (nmax + 1));
        double* d_fq = buf.get<double>(Q);
        if (buf.err != cudaSuccess) return buf.err;
        e = cudaMemcpyAsync(d_kq, kT_q, Q * sizeof(double), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_mq, mu_q, Q * sizeof(double), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = mbar_prep_states(Q, d_kq, d_mq, lambda0, nullptr, nullptr, a_q, c_q, nullptr, s);
        if (e == cudaSuccess) e = with_runs(buf, m, s);
        if (e == cudaSuccess) e = mbar_query_dev(m, Q, a_q, c_q, nmax, d_nm, d_pn, d_fq, s);
        if (e == cudaSuccess && N_mean) e = cudaMemcpyAsync(N_mean, d_nm, Q * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && pN)
            e = cudaMemcpyAsync(pN, d_pn, (size_t)Q * (nmax + 1) * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && f_q) e = cudaMemcpyAsync(f_q, d_fq, Q * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return e;
    }
    return cudaStreamSynchronize(s);
}

}  // namespace

extern "C" {

regc_status regc_mu_of_pressure(int n, const double* kT, const double* p, double lambda0, double* mu) {
    if (n < 0 || (n > 0 && (!kT || !p || !mu)) || !(lambda0 > 0.0) || !std::isfinite(lambda0)) return REGC_EINVAL;
    for (int i = 0; i < n; ++i)
        if (!(kT[i] > 0.0) || !(p[i] > 0.0) || !std::isfinite(kT[i]) || !std::isfinite(p[i])) return REGC_EINVAL;
    for (int i = 0; i < n; ++i) mu[i] = kT[i] * (3.0 * (log(lambda0) - 0.5 * log(kT[i])) + log(p[i] / kT[i]));
    return REGC_OK;
}

regc_status regc_pressure_of_mu(int n, const double* kT, const double* mu, double lambda0, double* p) {
    if (n < 0 || (n > 0 && (!kT || !mu || !p)) || !(lambda0 > 0.0) || !std::isfinite(lambda0)) return REGC_EINVAL;
    for (int i = 0; i < n; ++i)
        if (!(kT[i] > 0.0) || !std::isfinite(kT[i]) || !std::isfinite(mu[i])) return REGC_EINVAL;
    for (int i = 0; i < n; ++i)
        p[i] = kT[i] * exp(mu[i] / kT[i] - 3.0 * (log(lambda0) - 0.5 * log(kT[i])));
    return REGC_OK;
}

regc_status regc_reweight(regc_handle* h, int nq, const double* kT_q, const double* mu_q, double tol, int max_iter,
                          double* N_mean, double* pN, double* f_states, int* iters) {
    NvtxRange nvtx_("regc_reweight");
    if (!h || nq < 0 || (nq > 0 && (!kT_q || !mu_q)) || !(tol > 0.0) || max_iter < 1) return REGC_EINVAL;
    if (h->P.gc2) return REGC_EINVAL;   // two species: regc_reweight2
    for (int q = 0; q < nq; ++q)
        if (!(kT_q[q] > 0.0) || !std::isfinite(mu_q[q])) return REGC_EINVAL;
    regc_status st = sync_check(h);
    if (st != REGC_OK) return st;
    MbarBuffers buf;
    buf.s = h->stream;
    const long long n = (long long)(h->nmax + 1) * h->n_e_bins;
    int* scratch = buf.get<int>(compact_scratch_ints(n));
    int* d_count = buf.get<int>(1);
    if (buf.err != cudaSuccess) return status_of(buf.err);
    cudaError_t e = compact_count_dev(h->P.hNE, n, scratch, d_count, h->stream);
    int B = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&B, d_count, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return status_of(e);
    if (B == 0) return REGC_EINVAL;   // nothing observed yet
    MbarDev m{};
    m.S = h->S;
    m.B = B;
    int* N_b = buf.get<int>(B);
    double* E_b = buf.get<double>(B);
    double* lnH = buf.get<double>(B);
    double* a = buf.get<double>(h->S);
    double* c = buf.get<double>(h->S);
    double* lnom = buf.get<double>(h->S);
    if (buf.err != cudaSuccess) return status_of(buf.err);
    e = compact_write_dev(h->P.hNE, n, h->n_e_bins, h->e_lo, h->e_bin, scratch, N_b, E_b, lnH, h->stream);
    if (e == cudaSuccess)
        e = mbar_prep_states(h->S, h->d_kT_state, h->d_mu_state, h->lambda0, nullptr, h->P.omega, a, c, lnom, h->stream);
    if (e != cudaSuccess) return status_of(e);
    m.a = a;
    m.c = c;
    m.lnom = lnom;
    m.N_b = N_b;
    m.E_b = E_b;
    m.lnH = lnH;
    e = solve_and_query(buf, m, h->lambda0, tol, max_iter, iters, f_states, nullptr, nq, kT_q, mu_q, h->nmax, N_mean,
                        pN, nullptr, kWarmBins * h->e_bin);
    return status_of(e);
}

regc_status regc_reweight2(regc_handle* h, int nq, const double* kT_q, const double* mu_q, const double* mu2_q,
                           double tol, int max_iter, double* NB_mean, double* NC_mean, double* pNB, double* pNC,
                           double* f_states, int* iters) {
    NvtxRange nvtx_("regc_reweight2");
    if (!h || nq < 0 || (nq > 0 && (!kT_q || !mu_q || !mu2_q)) || !(tol > 0.0) || max_iter < 1) return REGC_EINVAL;
    if (!h->P.gc2) return REGC_EINVAL;   // one species: regc_reweight
    for (int q = 0; q < nq; ++q)
        if (!(kT_q[q] > 0.0) || !std::isfinite(kT_q[q]) || !std::isfinite(mu_q[q]) || !std::isfinite(mu2_q[q]))
            return REGC_EINVAL;
    regc_status st = sync_check(h);
    if (st != REGC_OK) return st;
    MbarBuffers buf;
    buf.s = h->stream;
    cudaStream_t s = h->stream;
    const int rows2 = h->nmax + 1;
    const long long n = h->hist_rows * h->n_e_bins;
    int* scratch = buf.get<int>(compact_scratch_ints(n));
    int* d_count = buf.get<int>(1);
    if (buf.err != cudaSuccess) return status_of(buf.err);
    cudaError_t e = compact_count_dev(h->P.hNE, n, scratch, d_count, s);
    int B = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&B, d_count, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return status_of(e);
    if (B == 0) return REGC_EINVAL;   // nothing observed yet
    MbarDev m{};
    m.S = h->S;
    m.B = B;
    int* N_b = buf.get<int>(B);
    int* N2_b = buf.get<int>(B);
    double* E_b = buf.get<double>(B);
    double* lnH = buf.get<double>(B);
    double* a = buf.get<double>(h->S);
    double* c = buf.get<double>(h->S);
    double* c2 = buf.get<double>(h->S);
    double* lnom = buf.get<double>(h->S);
    m.f = buf.get<double>(m.S);
    m.f_new = buf.get<double>(m.S);
    m.D = buf.get<double>(B);
    m.EN32 = buf.get<float2>(B);
    m.DH32 = buf.get<float>(B);
    m.N2f = buf.get<float>(B);
    m.delta = buf.get<double>(1);
    m.state = buf.get<int>(2);
    if (buf.err != cudaSuccess) return status_of(buf.err);
    e = compact_write2_dev(h->P.hNE, n, h->n_e_bins, rows2, h->e_lo, h->e_bin, scratch, N_b, N2_b, E_b, lnH, s);
    if (e == cudaSuccess)
        e = mbar_prep_states(h->S, h->d_kT_state, h->d_mu_state, h->lambda0, nullptr, h->P.omega, a, c, lnom, s);
    if (e == cudaSuccess) e = mbar_prep_states2(h->S, h->d_kT_state, h->d_mu2_state, h->lambda0_2, c2, s);
    if (e != cudaSuccess) return status_of(e);
    m.a = a;
    m.c = c;
    m.c2 = c2;
    m.lnom = lnom;
    m.N_b = N_b;
    m.N2_b = N2_b;
    m.E_b = E_b;
    m.lnH = lnH;
    e = mbar_solve_warm_dev(m, kWarmBins * h->e_bin, tol, max_iter, iters, s);
    if (e == cudaSuccess && f_states) e = cudaMemcpyAsync(f_states, m.f, m.S * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return status_of(e);
    if (nq > 0) {
        const size_t P = (size_t)nq * rows2;
        double* d_kq = buf.get<double>(nq);
        double* d_mq = buf.get<double>(nq);
        double* d_m2q = buf.get<double>(nq);
        double* a_q = buf.get<double>(nq);
        double* c_q = buf.get<double>(nq);
        double* c2_q = buf.get<double>(nq);
        double* d_nb = buf.get<double>(nq);
        double* d_nc = buf.get<double>(nq);
        double* d_pb = buf.get<double>(P);
        double* d_pc = buf.get<double>(P);
        if (buf.err != cudaSuccess) return status_of(buf.err);
        e = cudaMemcpyAsync(d_kq, kT_q, nq * sizeof(double), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_mq, mu_q, nq * sizeof(double), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_m2q, mu2_q, nq * sizeof(double), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = mbar_prep_states(nq, d_kq, d_mq, h->lambda0, nullptr, nullptr, a_q, c_q, nullptr, s);
        if (e == cudaSuccess) e = mbar_prep_states2(nq, d_kq, d_m2q, h->lambda0_2, c2_q, s);
        if (e == cudaSuccess) e = with_runs(buf, m, s);
        if (e == cudaSuccess) e = mbar_query2_dev(m, nq, a_q, c_q, c2_q, h->nmax, d_nb, d_nc, d_pb, d_pc, nullptr, s);
        if (e == cudaSuccess && NB_mean) e = cudaMemcpyAsync(NB_mean, d_nb, nq * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && NC_mean) e = cudaMemcpyAsync(NC_mean, d_nc, nq * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && pNB) e = cudaMemcpyAsync(pNB, d_pb, P * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && pNC) e = cudaMemcpyAsync(pNC, d_pc, P * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return status_of(e);
    }
    return status_of(cudaStreamSynchronize(s));
}

regc_status regc_mbar_last_info(regc_mbar_info* out) {
    if (!out) return REGC_EINVAL;
    const MbarInfo i = mbar_last_info();
    *out = regc_mbar_info{i.path, i.iterations, i.builds, i.lse_maps, i.nnz, i.S, i.B,
                          i.ms_build, i.ms_maps, i.sparse_maps, i.coarse_iterations, i.coarse_B,
                          i.coarse_builds, i.coarse_maps};
    return REGC_OK;
}

regc_status regc_mbar_solve(int S, const double* kT, const double* mu, double lambda0, const double* omega, int B,
                            const int32_t* N_b, const double* E_b, const double* H_b, double tol, int max_iter,
                            double* f, double* D, int* iters, void* cuda_stream) {
    NvtxRange nvtx_("regc_mbar_solve");
    if (S < 1 || B < 1 || !kT || !mu || !omega || !N_b || !E_b || !H_b || !(tol > 0.0) || max_iter < 1 ||
        !(lambda0 > 0.0))
        return REGC_EINVAL;
    for (int s = 0; s < S; ++s)
        if (!(kT[s] > 0.0) || !std::isfinite(mu[s]) || !(omega[s] >= 0.0)) return REGC_EINVAL;
    for (int b = 0; b < B; ++b)
        if (!(H_b[b] > 0.0) || N_b[b] < 0 || !std::isfinite(E_b[b])) return REGC_EINVAL;
    MbarBuffers buf;
    buf.s = static_cast<cudaStream_t>(cuda_stream);
    double* d_kT = buf.get<double>(S);
    double* d_mu = buf.get<double>(S);
    double* d_om = buf.get<double>(S);
    double* a = buf.get<double>(S);
    double* c = buf.get<double>(S);
    double* lnom = buf.get<double>(S);
    int* d_N = buf.get<int>(B);
    double* d_E = buf.get<double>(B);
    double* d_H = buf.get<double>(B);
    double* lnH = buf.get<double>(B);
    if (buf.err != cudaSuccess) return status_of(buf.err);
    cudaError_t e = cudaMemcpyAsync(d_kT, kT, S * sizeof(double), cudaMemcpyHostToDevice, buf.s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_mu, mu, S * sizeof(double), cudaMemcpyHostToDevice, buf.s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_om, omega, S * sizeof(double), cudaMemcpyHostToDevice, buf.s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_N, N_b, B * sizeof(int), cudaMemcpyHostToDevice, buf.s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_E, E_b, B * sizeof(double), cudaMemcpyHostToDevice, buf.s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_H, H_b, B * sizeof(double), cudaMemcpyHostToDevice, buf.s);
    if (e == cudaSuccess) e = mbar_prep_states(S, d_kT, d_mu, lambda0, d_om, nullptr, a, c, lnom, buf.s);
    if (e == cudaSuccess) e = mbar_prep_bins(B, d_H, lnH, buf.s);
    if (e != cudaSuccess) return status_of(e);
    MbarDev m{};
    m.S = S;
    m.B = B;
    m.a = a;
    m.c = c;
    m.lnom = lnom;
    m.N_b = d_N;
    m.E_b = d_E;
    m.lnH = lnH;
    e = solve_and_query(buf, m, lambda0, tol, max_iter, iters, f, D, 0, nullptr, nullptr, 0, nullptr, nullptr, nullptr);
    return status_of(e);
}

regc_status regc_mbar_query(int Q, const double* kT_q, const double* mu_q, double lambda0, int B,
                            const int32_t* N_b, const double* E_b, const double* H_b, const double* D, int nmax,
                            double* N_mean, double* pN, double* f_q, void* cuda_stream) {
    NvtxRange nvtx_("regc_mbar_query");
    if (Q < 1 || B < 1 || !kT_q || !mu_q || !N_b || !E_b || !H_b || !D || nmax < 0 || !(lambda0 > 0.0))
        return REGC_EINVAL;
    for (int q = 0; q < Q; ++q)
        if (!(kT_q[q] > 0.0) || !std::isfinite(mu_q[q])) return REGC_EINVAL;
    for (int b = 0; b < B; ++b)
        if (!(H_b[b] > 0.0) || N_b[b] < 0 || !std::isfinite(E_b[b]) || !std::isfinite(D[b])) return REGC_EINVAL;
    MbarBuffers buf;
    buf.s = static_cast<cudaStream_t>(cuda_stream);
    int* d_N = buf.get<int>(B);
    double* d_E = buf.get<double>(B);
    double* d_H = buf.get<double>(B);
    double* lnH = buf.get<double>(B);
    double* d_D = buf.get<double>(B);
    double* d_kq = buf.get<double>(Q);
    double* d_mq = buf.get<double>(Q);
    double* a_q = buf.get<double>(Q);
    double* c_q = buf.get<double>(Q);
    double* d_nm = buf.get<double>(Q);
    double* d_pn = buf.get<double>((size_t)Q * (nmax + 1));
    double* d_fq = buf.get<double>(Q);
    if (buf.err != cudaSuccess) return status_of(buf.err);
    cudaStream_t s = buf.s;
    cudaError_t e = cudaMemcpyAsync(d_N, N_b, B * sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_E, E_b, B * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_H, H_b, B * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_D, D, B * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_kq, kT_q, Q * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_mq, mu_q, Q * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = mbar_prep_bins(B, d_H, lnH, s);
    if (e == cudaSuccess) e = mbar_prep_states(Q, d_kq, d_mq, lambda0, nullptr, nullptr, a_q, c_q, nullptr, s);
    if (e != cudaSuccess) return status_of(e);
    MbarDev m{};
    m.S = 0;
    m.B = B;
    m.N_b = d_N;
    m.E_b = d_E;
    m.lnH = lnH;
    m.D = d_D;
    m.EN32 = buf.get<float2>(B);
    m.DH32 = buf.get<float>(B);
    if (buf.err != cudaSuccess) return status_of(buf.err);
    e = mbar_prep32_dev(m, s);
    if (e == cudaSuccess) e = with_runs(buf, m, s);
    if (e == cudaSuccess) e = mbar_query_dev(m, Q, a_q, c_q, nmax, d_nm, d_pn, d_fq, s);
    if (e == cudaSuccess && N_mean) e = cudaMemcpyAsync(N_mean, d_nm, Q * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && pN)
        e = cudaMemcpyAsync(pN, d_pn, (size_t)Q * (nmax + 1) * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && f_q) e = cudaMemcpyAsync(f_q, d_fq, Q * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return status_of(e);
}

}  // extern "C"
