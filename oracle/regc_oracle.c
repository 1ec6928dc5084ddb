/*
 * regc_oracle.c -- FP64 CPU oracle of the REGCMC sampler (arXiv:1908.11118).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * CPU-baseline leg of the benchmark, never by the library.  It is written
 * for a reader who checks it against the paper line by line:
 *   - every energy is a plain double sum over all partners (no cell lists,
 *     no tiling, no reordering);
 *   - every acceptance rule is the paper's equation in log form;
 *   - walkers are independent between exchanges, so the only parallelism is
 *     an OpenMP loop over walkers.
 *
 * Random numbers: one counter-based generator, Philox4x32-10 (Salmon, Moraes,
 * Dror & Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11), written
 * here from its published definition.  Block keyed by (seed), counter
 * (move k, sweep t, walker w, stream):
 *   stream 0 (block A): A0 move kind, A1..A3 displacement / insertion uniforms
 *   stream 1 (block B): B0 particle index, B1 acceptance uniform,
 *                       B2 top bit = grand-canonical direction, B3 spare
 *   stream 2: exchange type and parity, counter (e, 0, 0, 2)
 *   stream 3: exchange uniform of the pair whose lower state index is a,
 *             counter (e, a, 0, 3)
 *   stream 10: REGC cycle, particle or replica exchange at step t,
 *             counter (t, 0, 0, 10)
 *
 * Planted-mistake switches (oracle_system.mutation, zero in real use) exist so
 * that the tests can show each pin detects the mistake it is meant to catch:
 *   1   exchange: sign of the chemical-potential term flipped
 *   2   exchange: (beta_a/beta_b)^{3/2 dN} factor dropped
 *   4   insertion/removal: Lambda^1 instead of Lambda^3
 *   8   insertion: the 1/(N+1) factor dropped
 *   16  pair potential: the factor 4 dropped
 *   32  minimum image not applied along y
 *   64  removal: energy taken of particle i but particle (i+1) mod N removed
 *   128 delayed acceptance: stage 2 without the -dE~ correction
 *   256 cluster: insertion/removal ratios with the total N instead of N_B
 *   512 MD thermostat: the cross term 2 R1 sqrt(...) of the rescaled kinetic energy dropped
 *   1024 MD: forces with the wrong sign
 *   2048 REGC cycle: the two branches of the x0 choice swapped
 *   4096 REGC cycle: canonical moves drawn from the mixed move set
 *   8192 pooled (N, E) histogram: an observation counted one energy bin too high
 *   16384 per-state energy histograms: an observation counted in the row of the
 *         walker instead of the row of the walker's state
 *   32768 second species: insertion and removal of C with species B's mu and Lambda
 *   65536 second species: the exchange without the mu2 term
 *
 * Delayed acceptance (da != 0; not in the paper, Christen & Fox 2005): a move
 * is first screened with the surrogate energy change dE~ (stage 1: accept iff
 * ln u1 < the acceptance log ratio with dE~ in place of dE, u1 from B3); a
 * move that passes is accepted iff ln u2 < -beta (dE - dE~) (stage 2, u2 from
 * B1).  dE~ is built from the surrogate energy e~ of the moved particle at its
 * new and old positions, so it changes sign under the reverse move and the
 * chain keeps the distribution of Eq. Ngrand for any network weights.
 */
#define _GNU_SOURCE
#include "regc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- Philox */

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    /* Philox4x32 round (Salmon et al. 2011): two 32x32->64 multiplications
     * by the constants 0xD2511F53 and 0xCD9E8D57 act on words 0 and 2; the
     * high halves are mixed with words 1, 3 and the round key; the key is
     * advanced by the Weyl increments 0x9E3779B9, 0xBB67AE85 between rounds. */
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static void draw(const oracle_system *sys, uint32_t c0, uint32_t c1, uint32_t c2,
                 uint32_t c3, uint32_t out[4])
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)sys->seed, (uint32_t)(sys->seed >> 32)};
    oracle_philox4x32_10(ctr, key, out);
}

/* 24-bit uniform in [0, 1), exact in binary32 */
static double u24(uint32_t a) { return (double)(a >> 8) * (1.0 / 16777216.0); }
/* uniform in (0, 1) for acceptance tests */
static double u32_open(uint32_t a) { return ((double)a + 0.5) * (1.0 / 4294967296.0); }
/* round through binary32 */
static double f32(double v) { return (double)(float)v; }

/* ------------------------------------------------------------- potential */

double oracle_phi(const oracle_system *sys, int ti, int tj, double r2)
{
    /* Lennard-Jones 12-6 (Appendix, force field), truncated: zero at r >= rc */
    if (r2 >= sys->rc * sys->rc) return 0.0;
    double sig = sys->sigma[ti][tj];
    double s2 = sig * sig / r2;
    double s6 = s2 * s2 * s2;
    double pref = (sys->mutation & 16) ? 1.0 : 4.0;
    return pref * sys->eps[ti][tj] * (s6 * s6 - s6);
}

static double min_image(double d, double box)
{
    return d - box * nearbyint(d / box);
}

/* Nearest-image displacement a - b, Cartesian.  Coordinates are in the cell
 * frame (u, y, z): the lattice vectors of the cell are (Lx, 0) and
 * (shear Ly, Ly), so the Cartesian x of a cell-frame point is u + shear y
 * (shear = 0: a rectangular cell, where the reduced difference is the
 * nearest image).  In a sheared cell the nearest image is the shortest of the
 * displacements to the images of b in the nine cells around the reduced
 * difference. */
static void pair_vec(const oracle_system *sys, double xa, double ya, double za,
                     double xb, double yb, double zb, double d[3])
{
    double du = min_image(xa - xb, sys->Lx);
    double dv = (sys->mutation & 32) ? (ya - yb) : min_image(ya - yb, sys->Ly);
    double dz = sys->periodic_z ? min_image(za - zb, sys->Lz) : (za - zb);
    if (sys->shear == 0.0) {
        /* rectangular cell: the reduced difference is the nearest image */
        d[0] = du;
        d[1] = dv;
        d[2] = dz;
        return;
    }
    int jr = (sys->mutation & 32) ? 0 : 1;
    double best = INFINITY;
    for (int j = -jr; j <= jr; ++j)
        for (int i = -1; i <= 1; ++i) {
            double v = dv + j * sys->Ly;
            double x = du + i * sys->Lx + sys->shear * v;
            double r2 = x * x + v * v + dz * dz;
            if (r2 < best) {
                best = r2;
                d[0] = x;
                d[1] = v;
            }
        }
    d[2] = dz;
}

static double pair_r2(const oracle_system *sys, double xa, double ya, double za,
                      double xb, double yb, double zb)
{
    double d[3];
    pair_vec(sys, xa, ya, za, xb, yb, zb, d);
    return d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
}

/* Error scale of a pair evaluated in binary32: 4 eps [(sigma/r)^12 + (sigma/r)^6],
 * the magnitudes of the two terms whose difference is phi (they cancel near
 * r = sigma, so |phi| alone understates the rounding error). */
static void account(const oracle_system *sys, int ti, int tj, double r2, double phi,
                    double *sum_abs, double *band, int *n_pairs)
{
    double rc2 = sys->rc * sys->rc;
    (void)phi;
    if (r2 < rc2) {
        double s2 = sys->sigma[ti][tj] * sys->sigma[ti][tj] / r2;
        double s6 = s2 * s2 * s2;
        if (sum_abs) *sum_abs += 4.0 * sys->eps[ti][tj] * (s6 * s6 + s6);
        if (n_pairs) *n_pairs += 1;
    }
    if (band && fabs(r2 - rc2) < 4e-6 * rc2) {
        double sr = sys->sigma[ti][tj] / sys->rc;
        double s6 = pow(sr, 6.0);
        *band += fabs(4.0 * sys->eps[ti][tj] * (s6 * s6 - s6));
    }
}

/* Potential type of mobile particle j of a walker with nb particles of
 * species B: the cluster species for the first n_cluster particles; with a
 * second grand-canonical species, type gc2_type from index nb on; else the
 * grand-canonical species 0. */
static int species_nb(const oracle_system *sys, int j, int nb)
{
    if (j < sys->n_cluster) return sys->cluster_type;
    if (sys->gc2_type > 0 && j >= nb) return sys->gc2_type;
    return 0;
}

static int species(const oracle_system *sys, int j) { return species_nb(sys, j, 1 << 30); }

/* Interaction energy of a mobile particle at (x, y, z) with every surface atom
 * and every mobile particle j != skip (the moved particle's energy entering
 * E(R; N) in Eq. Ngrand).  The moved particle is particle `skip` (its species
 * decides the pair types) or, for skip < 0, a new grand-canonical particle. */
double oracle_particle_energy(const oracle_system *sys, const double *pos, int n,
                              double x, double y, double z, int skip,
                              double *sum_abs, double *band, int *n_pairs)
{
    return oracle_particle_energy2(sys, pos, n, n, x, y, z, skip, 0, sum_abs, band, n_pairs);
}

/* As oracle_particle_energy for a walker with nb particles of species B; a
 * new particle (skip < 0) has potential type species_new. */
double oracle_particle_energy2(const oracle_system *sys, const double *pos, int n, int nb,
                               double x, double y, double z, int skip, int species_new,
                               double *sum_abs, double *band, int *n_pairs)
{
    const int ti = skip >= 0 ? species_nb(sys, skip, nb) : species_new;
    double e = 0.0;
    for (int a = 0; a < sys->n_surf; ++a) {
        const double *ra = sys->surf_xyz + 3 * a;
        int ta = sys->surf_type[a];
        double r2 = pair_r2(sys, x, y, z, ra[0], ra[1], ra[2]);
        double phi = oracle_phi(sys, ti, ta, r2);
        account(sys, ti, ta, r2, phi, sum_abs, band, n_pairs);
        e += phi;
    }
    for (int j = 0; j < n; ++j) {
        if (j == skip) continue;
        const double *rj = pos + 3 * j;
        const int tj = species_nb(sys, j, nb);
        double r2 = pair_r2(sys, x, y, z, rj[0], rj[1], rj[2]);
        double phi = oracle_phi(sys, ti, tj, r2);
        account(sys, ti, tj, r2, phi, sum_abs, band, n_pairs);
        e += phi;
    }
    return e;
}

/* E(R; N): all mobile-mobile pairs i < j plus all mobile-surface pairs.  The
 * slab is frozen, so surface-surface pairs are constant and left out. */
double oracle_total_energy(const oracle_system *sys, const double *pos, int n)
{
    return oracle_total_energy2(sys, pos, n, n);
}

double oracle_total_energy2(const oracle_system *sys, const double *pos, int n, int nb)
{
    double e = 0.0;
    for (int i = 0; i < n; ++i) {
        const double *ri = pos + 3 * i;
        const int ti = species_nb(sys, i, nb);
        for (int a = 0; a < sys->n_surf; ++a) {
            const double *ra = sys->surf_xyz + 3 * a;
            e += oracle_phi(sys, ti, sys->surf_type[a],
                            pair_r2(sys, ri[0], ri[1], ri[2], ra[0], ra[1], ra[2]));
        }
        for (int j = i + 1; j < n; ++j) {
            const double *rj = pos + 3 * j;
            e += oracle_phi(sys, ti, species_nb(sys, j, nb),
                            pair_r2(sys, ri[0], ri[1], ri[2], rj[0], rj[1], rj[2]));
        }
    }
    return e;
}

/* ------------------------------------------------------------- surrogate */

#define SUR_NF 16
#define SUR_NH 64

static double silu(double x) { return x / (1.0 + exp(-x)); }

/* x rounded to binary32, then to the nearest bfloat16 (ties to even): the
 * precision of every layer input of the sampler's network. */
static double bf16(double x)
{
    float f = (float)x;
    uint32_t u;
    memcpy(&u, &f, 4);
    u = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
    memcpy(&f, &u, 4);
    return (double)f;
}

/* Surrogate energy e~ of a mobile particle at (x, y, z): 16 Gaussian radial
 * features over every surface atom and mobile particle j != skip within rc,
 * G_k = sum_j eps_0j exp(-eta (r_j - c_k)^2) (cos(pi r_j / rc) + 1) / 2 with
 * c_k = 0.8 + 1.7 k / 15 and eta = 1 / (2 (1.7/15)^2), then the network
 * 16 -> 64 -> 64 -> 1 with SiLU hidden layers, each layer's inputs (G, then
 * the hidden activations) rounded to bfloat16 as the sampler's network takes
 * them (its weights are bfloat16 already: sur_theta holds the inference
 * parameters).  feat, if given, receives G (not rounded). */
double oracle_surrogate_energy(const oracle_system *sys, const double *pos, int n,
                               double x, double y, double z, int skip, double *feat)
{
    const double rc = sys->rc, width = 1.7 / 15.0, eta = 1.0 / (2.0 * width * width);
    const int ti = skip >= 0 ? species(sys, skip) : 0;   /* weights eps between the moved species and j */
    double G[SUR_NF];
    for (int k = 0; k < SUR_NF; ++k) G[k] = 0.0;
    for (int j = -sys->n_surf; j < n; ++j) {
        const double *r;
        int t;
        if (j < 0) {
            r = sys->surf_xyz + 3 * (j + sys->n_surf);
            t = sys->surf_type[j + sys->n_surf];
        } else {
            if (j == skip) continue;
            r = pos + 3 * j;
            t = species(sys, j);
        }
        double d = sqrt(pair_r2(sys, x, y, z, r[0], r[1], r[2]));
        if (d >= rc) continue;
        double fc = 0.5 * (cos(M_PI * d / rc) + 1.0) * sys->eps[ti][t];
        for (int k = 0; k < SUR_NF; ++k) {
            double c = 0.8 + 1.7 * k / 15.0;
            G[k] += exp(-eta * (d - c) * (d - c)) * fc;
        }
    }
    if (feat)
        for (int k = 0; k < SUR_NF; ++k) feat[k] = G[k];
    const double *W1 = sys->sur_theta, *b1 = W1 + SUR_NF * SUR_NH, *W2 = b1 + SUR_NH;
    const double *b2 = W2 + SUR_NH * SUR_NH, *W3 = b2 + SUR_NH, *b3 = W3 + SUR_NH;
    double h1[SUR_NH], h2[SUR_NH], g16[SUR_NF];
    for (int k = 0; k < SUR_NF; ++k) g16[k] = bf16(G[k]);
    for (int u = 0; u < SUR_NH; ++u) {
        double z1 = b1[u];
        for (int k = 0; k < SUR_NF; ++k) z1 += W1[k * SUR_NH + u] * g16[k];
        h1[u] = bf16(silu(z1));
    }
    for (int v = 0; v < SUR_NH; ++v) {
        double z2 = b2[v];
        for (int u = 0; u < SUR_NH; ++u) z2 += W2[u * SUR_NH + v] * h1[u];
        h2[v] = bf16(silu(z2));
    }
    double e = b3[0];
    for (int v = 0; v < SUR_NH; ++v) e += W3[v] * h2[v];
    return e;
}

/* ---------------------------------------------------------- acceptance */

/* States s = (l M + m) K + k with K = 1 for one grand-canonical species. */
static int axis_K(const oracle_system *sys) { return (sys->gc2_type > 0 && sys->K > 1) ? sys->K : 1; }
static int n_states(const oracle_system *sys) { return sys->L * sys->M * axis_K(sys); }
static double kT_of(const oracle_system *sys, int state) { return sys->kT[state / (sys->M * axis_K(sys))]; }
static double mu_of(const oracle_system *sys, int state) { return sys->mu[(state / axis_K(sys)) % sys->M]; }
static double mu2_of(const oracle_system *sys, int state) { return sys->mu2[state % axis_K(sys)]; }

static double ln_lambda(const oracle_system *sys, double kT)
{
    /* Lambda = h / sqrt(2 pi m kT) (Eq. Ngrand); in reduced units lambda0/sqrt(kT) */
    return log(sys->lambda0) - 0.5 * log(kT);
}

static double ln_lambda2(const oracle_system *sys, double kT)
{
    return log(sys->lambda0_2) - 0.5 * log(kT);
}

static double volume(const oracle_system *sys)
{
    return sys->Lx * sys->Ly * (sys->z_hi - sys->z_lo);
}

/* log of the Metropolis acceptance ratio of a move that changes the energy by
 * dE, for a walker with n mobile particles before the move:
 *   type 0, displacement (Sec. II.A.3):   -beta dE
 *   type 1, insertion   (Sec. II.A.1):   ln[V / (Lambda^3 (n+1))] + beta (mu - dE)
 *   type 2, removal     (Sec. II.A.1):   ln[Lambda^3 n / V] - beta (mu + dE)
 * (the insertion exponent is read as beta[mu - (E_{N+1} - E_N)]). */
double oracle_log_alpha(const oracle_system *sys, int type, int state, int n, double dE)
{
    return oracle_log_alpha2(sys, type, 0, state, n, dE);
}

/* As oracle_log_alpha for a grand-canonical move of species `species` (0: B,
 * 1: C, with its own mu2 and Lambda) at a state holding n_c particles of it. */
double oracle_log_alpha2(const oracle_system *sys, int type, int species2, int state, int n, double dE)
{
    const int c = species2 && !(sys->mutation & 32768);
    double kT = kT_of(sys, state), beta = 1.0 / kT, mu = c ? mu2_of(sys, state) : mu_of(sys, state);
    double lam_pow = (sys->mutation & 4) ? 1.0 : 3.0;
    double lnL = c ? ln_lambda2(sys, kT) : ln_lambda(sys, kT);
    double lnV = log(volume(sys));
    if (type == 0) return -beta * dE;
    if (type == 1) {
        double ln_n1 = (sys->mutation & 8) ? 0.0 : log((double)(n + 1));
        return lnV - lam_pow * lnL - ln_n1 + beta * (mu - dE);
    }
    return lam_pow * lnL + log((double)n) - lnV - beta * (mu + dE);
}

/* log acceptance of swapping the configurations of states a and b (Eq. Pacc),
 * where state a holds (na, ea) and state b holds (nb, eb):
 *   1.5 (na - nb) ln(beta_a / beta_b) - (beta_a - beta_b)(eb - ea)
 *     - (beta_a mu_a - beta_b mu_b)(na - nb)
 * (the leading minus of the printed exponent is read as covering both terms). */
/* With a second species: state a holds (N_B,a, N_C,a, E_a); both thermal
 * wavelengths scale as beta^(1/2), so the Lambda factor takes the total N:
 *   1.5 (N_a - N_b) ln(beta_a / beta_b) - (beta_a - beta_b)(E_b - E_a)
 *   - (beta_a mu_a - beta_b mu_b)(N_B,a - N_B,b)
 *   - (beta_a mu2_a - beta_b mu2_b)(N_C,a - N_C,b). */
double oracle_exchange_log_alpha2(const oracle_system *sys, int sa, int sb, int nba, int nca,
                                  int nbb, int ncb, double ea, double eb)
{
    double ba = 1.0 / kT_of(sys, sa), bb = 1.0 / kT_of(sys, sb);
    double dn = (double)((nba + nca) - (nbb + ncb));
    double lam = 1.5 * dn * log(ba / bb);
    double mu_term = (ba * mu_of(sys, sa) - bb * mu_of(sys, sb)) * (double)(nba - nbb);
    if (!(sys->mutation & 65536))
        mu_term += (ba * mu2_of(sys, sa) - bb * mu2_of(sys, sb)) * (double)(nca - ncb);
    return lam - (ba - bb) * (eb - ea) - mu_term;
}

double oracle_exchange_log_alpha(const oracle_system *sys, int sa, int sb,
                                 int na, int nb, double ea, double eb)
{
    double ba = 1.0 / kT_of(sys, sa), bb = 1.0 / kT_of(sys, sb);
    double ma = mu_of(sys, sa), mb = mu_of(sys, sb);
    double dn = (double)(na - nb);
    double lam = (sys->mutation & 2) ? 0.0 : 1.5 * dn * log(ba / bb);
    double mu_term = (ba * ma - bb * mb) * dn;
    if (sys->mutation & 1) mu_term = -mu_term;
    return lam - (ba - bb) * (eb - ea) - mu_term;
}

/* ---------------------------------------------------------------- sweeps */

static void observe(const oracle_system *sys, oracle_hist *h, int state, int w, int n, int nc, double e)
{
    if (!h) return;
    if (sys->gc2_type > 0) {
        /* the second species' count; n is N_B here */
        if (h->hN2) h->hN2[(int64_t)state * (sys->nmax + 1) + nc] += 1;
        if (h->moments2) {
            h->moments2[2 * (int64_t)state] += nc;
            h->moments2[2 * (int64_t)state + 1] += (double)nc * nc;
        }
    }
    if (h->hE) {
        /* the state's own window (Sec. II.B: the observations of each state) */
        const int row = (sys->mutation & 16384) ? w : state;
        const double k = floor((e - h->hE_lo[row]) / h->hE_bin);
        const int64_t idx = k < 0.0 ? 0 : (k >= (double)h->hE_bins ? h->hE_bins + 1 : (int64_t)k + 1);
        h->hE[(int64_t)row * (h->hE_bins + 2) + idx] += 1;
    }
    int nb = sys->nmax + 1;
    if (h->hN) h->hN[(int64_t)state * nb + n] += 1;
    if (h->omega) h->omega[state] += 1;
    if (h->moments) {
        double *m = h->moments + 4 * (int64_t)state;
        m[0] += n;
        m[1] += (double)n * n;
        m[2] += e;
        m[3] += e * e;
    }
    if (h->hNE) {
        double k = floor((e - sys->e_lo) / sys->e_bin);
        if (sys->mutation & 8192) k += 1.0;
        if (k >= 0.0 && k < (double)sys->n_e_bins) {
            const int64_t row = sys->gc2_type > 0 ? (int64_t)n * (sys->nmax + 1) + nc : (int64_t)n;
            int64_t idx = row * sys->n_e_bins + (int64_t)k;
#ifdef _OPENMP
#pragma omp atomic
#endif
            h->hNE[idx] += 1;
        } else if (h->e_out) {
            h->e_out[state] += 1;
        }
    }
}

/* The particle count entering the grand-canonical ratios: N_B = N - n_cluster
 * (mutation 256: the total N). */
static int n_gc(const oracle_system *sys, int n)
{
    return (sys->mutation & 256) ? n : n - sys->n_cluster;
}

/* How a trial move picks its kind: MOVE_MIXED draws displacement or
 * particle exchange from A0 and p_disp (the sweeps); the REGC cycle fixes it,
 * MOVE_GC for its particle-exchange attempt, MOVE_DISPLACE for the canonical
 * diffusion that follows. */
enum { MOVE_MIXED = 0, MOVE_GC = 1, MOVE_DISPLACE = 2 };

/* Trial move k of sweep (or REGC step) t of walker w at the walker's state:
 * draws A = Philox((k, t, w, 0)) and B = Philox((k, t, w, 1)), evaluates the
 * move and applies it if accepted (positions, *n_io, *e_io).  mv receives its
 * record. */
static void trial_move(const oracle_system *sys, int w, double *pos, int *n_io, int *nb_io, double *e_io,
                       int state, uint32_t k, uint32_t t, int kind, oracle_move *out)
{
    const int two = sys->gc2_type > 0;
    int nb = two ? *nb_io : *n_io;   /* species B occupies [0, nb) */
    const double lx = sys->Lx, ly = sys->Ly, lz = sys->Lz;
    const double delta = f32(sys->max_disp);
    const double height = f32(sys->z_hi - sys->z_lo);
    double p = sys->p_disp < 0.0 ? 0.0 : (sys->p_disp > 1.0 ? 1.0 : sys->p_disp);
    const uint64_t th_disp = (uint64_t)floor(p * 4294967296.0);
    const double beta = 1.0 / kT_of(sys, state);
    int n = *n_io;
    double e = *e_io;
    uint32_t A[4], B[4];
    draw(sys, k, t, (uint32_t)w, 0u, A);
    draw(sys, k, t, (uint32_t)w, 1u, B);
    oracle_move mv;
    memset(&mv, 0, sizeof mv);
    mv.ln_u = log(u32_open(B[1]));
    if (kind == MOVE_DISPLACE || (kind == MOVE_MIXED && (uint64_t)A[0] < th_disp)) {
        mv.type = 0;
    } else {
        /* removal if y1 < 0.5, else insertion (Sec. II.A.1) */
        mv.type = (B[2] >> 31) == 0u ? 2 : 1;
    }
    /* with a second species, the next bit of B2 picks the species of a
     * grand-canonical move: 0 B, 1 C */
    const int gcs = (two && mv.type != 0) ? (int)((B[2] >> 30) & 1u) : 0;
    const int nc = n - nb;
    double nx = 0, ny = 0, nz = 0;  /* new position (displace/insert) */
    int i = -1;
    if (mv.type == 0) {
        /* Metropolis displacement (Sec. II.A.3): random atom, uniform
         * displacement in a cube of half-edge max_disp */
        if (n == 0) { mv.status = 1; goto decided; }
        i = (int)(((uint64_t)B[0] * (uint64_t)n) >> 32);
        mv.index = i;
        double d[3];
        for (int c = 0; c < 3; ++c) d[c] = f32(delta * f32(2.0 * u24(A[1 + c]) - 1.0));
        const double *ri = pos + 3 * i;
        nx = f32(ri[0] + d[0]);
        ny = f32(ri[1] + d[1]);
        nz = f32(ri[2] + d[2]);
        if (nx < 0.0) nx = f32(nx + lx);
        if (nx >= lx) nx = f32(nx - lx);
        if (ny < 0.0) ny = f32(ny + ly);
        if (ny >= ly) ny = f32(ny - ly);
        if (sys->periodic_z) {
            if (nz < 0.0) nz = f32(nz + lz);
            if (nz >= lz) nz = f32(nz - lz);
        } else if (nz < sys->z_lo || nz > sys->z_hi) {
            mv.status = 2;
            goto decided;
        }
        double e_new = oracle_particle_energy2(sys, pos, n, nb, nx, ny, nz, i, 0,
                                               &mv.sum_abs, &mv.band, &mv.n_pairs);
        double e_old = oracle_particle_energy2(sys, pos, n, nb, ri[0], ri[1], ri[2], i, 0,
                                               &mv.sum_abs, &mv.band, &mv.n_pairs);
        mv.dE = e_new - e_old;
        mv.log_alpha = -beta * mv.dE;
    } else if (mv.type == 1) {
        /* insertion at a uniform point of the region (Sec. II.A.1) */
        if (n == sys->nmax) { mv.status = 1; goto decided; }
        /* a new B goes to index nb (the first C moves to the end), a new C to n */
        mv.index = (two && gcs == 0) ? nb : n;
        nx = f32(lx * u24(A[1]));
        ny = f32(ly * u24(A[2]));
        nz = f32(sys->z_lo + f32(height * u24(A[3])));
        if (nx >= lx) nx = f32(nx - lx);
        if (ny >= ly) ny = f32(ny - ly);
        if (sys->periodic_z && nz >= lz) nz = f32(nz - lz);
        mv.dE = oracle_particle_energy2(sys, pos, n, nb, nx, ny, nz, -1, gcs ? sys->gc2_type : 0,
                                        &mv.sum_abs, &mv.band, &mv.n_pairs);
        mv.log_alpha = two ? oracle_log_alpha2(sys, 1, gcs, state, gcs ? nc : nb, mv.dE)
                           : oracle_log_alpha(sys, 1, state, n_gc(sys, n), mv.dE);
    } else {
        /* removal of grand-canonical particle i, (i-1)/N <= y2 < i/N
         * (Sec. II.A.1), counted among the N_B of that species */
        if (two) {
            /* uniformly among the particles of the chosen species */
            const int cnt = gcs ? nc : nb, first = gcs ? nb : 0;
            if (cnt == 0) { mv.status = 1; goto decided; }
            i = first + (int)(((uint64_t)B[0] * (uint64_t)cnt) >> 32);
        } else {
            if (n == sys->n_cluster) { mv.status = 1; goto decided; }
            i = sys->n_cluster + (int)(((uint64_t)B[0] * (uint64_t)(n - sys->n_cluster)) >> 32);
        }
        mv.index = i;
        const double *ri = pos + 3 * i;
        mv.dE = -oracle_particle_energy2(sys, pos, n, nb, ri[0], ri[1], ri[2], i, 0,
                                         &mv.sum_abs, &mv.band, &mv.n_pairs);
        mv.log_alpha = two ? oracle_log_alpha2(sys, 2, gcs, state, gcs ? nc : nb, mv.dE)
                           : oracle_log_alpha(sys, 2, state, n_gc(sys, n), mv.dE);
    }
    if (sys->da) {
        /* stage 1 with the surrogate energy change */
        if (mv.type == 0) {
            const double *ri = pos + 3 * i;
            mv.dE_sur = oracle_surrogate_energy(sys, pos, n, nx, ny, nz, i, NULL) -
                        oracle_surrogate_energy(sys, pos, n, ri[0], ri[1], ri[2], i, NULL);
        } else if (mv.type == 1) {
            mv.dE_sur = oracle_surrogate_energy(sys, pos, n, nx, ny, nz, -1, NULL);
        } else {
            const double *ri = pos + 3 * i;
            mv.dE_sur = -oracle_surrogate_energy(sys, pos, n, ri[0], ri[1], ri[2], i, NULL);
        }
        mv.ln_u1 = log(u32_open(B[3]));
        mv.stage1 = mv.ln_u1 < oracle_log_alpha(sys, mv.type, state, n_gc(sys, n), mv.dE_sur);
        /* stage 2: the exact correction */
        double corr = (sys->mutation & 128) ? 0.0 : mv.dE_sur;
        mv.accepted = mv.stage1 && mv.ln_u < -beta * (mv.dE - corr);
    } else {
        mv.accepted = mv.ln_u < mv.log_alpha;
    }
    if (mv.accepted) {
        if (mv.type == 0) {
            double *ri = pos + 3 * i;
            ri[0] = nx; ri[1] = ny; ri[2] = nz;
        } else if (mv.type == 1) {
            if (two && gcs == 0) {
                /* the first C (if any) moves to the end, the new B takes its index */
                memmove(pos + 3 * n, pos + 3 * nb, 3 * sizeof(double));
                double *rn = pos + 3 * nb;
                rn[0] = nx; rn[1] = ny; rn[2] = nz;
                nb += 1;
            } else {
                double *rn = pos + 3 * n;
                rn[0] = nx; rn[1] = ny; rn[2] = nz;
            }
            n += 1;
        } else if (two && gcs == 0) {
            /* the last B fills the gap, the last C fills the last B's index */
            memmove(pos + 3 * i, pos + 3 * (nb - 1), 3 * sizeof(double));
            memmove(pos + 3 * (nb - 1), pos + 3 * (n - 1), 3 * sizeof(double));
            nb -= 1;
            n -= 1;
        } else {
            int gone = (sys->mutation & 64) ? (i + 1) % n : i;
            memcpy(pos + 3 * gone, pos + 3 * (n - 1), 3 * sizeof(double));
            n -= 1;
        }
        e += mv.dE;
    }
decided:
    *n_io = n;
    if (two) *nb_io = nb;
    *e_io = e;
    *out = mv;
}

static void count_move(int64_t *counts, int w, const oracle_move *mv)
{
    if (!counts) return;
    counts[6 * (int64_t)w + 2 * mv->type] += 1;
    counts[6 * (int64_t)w + 2 * mv->type + 1] += mv->accepted;
}

static void sweep_walker(const oracle_system *sys, int w, double *pos, int32_t *n_ptr, int32_t *nb_ptr,
                         double *e_ptr, int state, uint32_t t0, int n_sweeps,
                         oracle_hist *hist, oracle_move *trace, int64_t *counts)
{
    int n = *n_ptr;
    int nb = nb_ptr ? *nb_ptr : n;
    double e = *e_ptr;
    for (int ts = 0; ts < n_sweeps; ++ts) {
        uint32_t t = t0 + (uint32_t)ts;
        for (int k = 0; k < sys->moves_per_sweep; ++k) {
            oracle_move mv;
            trial_move(sys, w, pos, &n, &nb, &e, state, (uint32_t)k, t, MOVE_MIXED, &mv);
            count_move(counts, w, &mv);
            if (trace) trace[((int64_t)ts * sys->moves_per_sweep + k)] = mv;
        }
        observe(sys, hist, state, w, sys->gc2_type > 0 ? nb : n - sys->n_cluster, n - nb, e);
    }
    *n_ptr = n;
    if (nb_ptr) *nb_ptr = nb;
    *e_ptr = e;
}

/* Run n_sweeps sweeps of moves_per_sweep trial moves on every walker, the
 * walkers' states held fixed (they change only at exchanges).  pos is
 * [n_walkers][nmax][3]; trace, if given, is [n_walkers][n_sweeps][moves_per_sweep];
 * counts, if given, is [n_walkers][3 move types][trials, accepts].
 * Returns 0, or -1 on invalid arguments. */
int oracle_sweeps(const oracle_system *sys, int n_walkers, double *pos, int32_t *n,
                  double *energy, const int32_t *state_of_walker, uint32_t t0,
                  int n_sweeps, oracle_hist *hist, oracle_move *trace,
                  int64_t *counts, int n_threads)
{
    if (sys->gc2_type > 0) return -1;   /* two species: oracle_sweeps2 */
    return oracle_sweeps2(sys, n_walkers, pos, n, NULL, energy, state_of_walker, t0, n_sweeps, hist, trace,
                          counts, n_threads);
}

int oracle_sweeps_range(const oracle_system *sys, int n_walkers, double *pos, int32_t *n, int32_t *nb,
                        double *energy, const int32_t *state_of_walker, uint32_t t0,
                        int n_sweeps, oracle_hist *hist, oracle_move *trace,
                        int64_t *counts, int n_threads, int w_begin, int w_end);

int oracle_sweeps2(const oracle_system *sys, int n_walkers, double *pos, int32_t *n, int32_t *nb,
                   double *energy, const int32_t *state_of_walker, uint32_t t0,
                   int n_sweeps, oracle_hist *hist, oracle_move *trace,
                   int64_t *counts, int n_threads)
{
    return oracle_sweeps_range(sys, n_walkers, pos, n, nb, energy, state_of_walker, t0, n_sweeps, hist, trace,
                               counts, n_threads, 0, n_walkers);
}

/* The sweeps of walkers [w_begin, w_end) only (the others are left as they
 * are): a process's share of a grid split over several processes. */
int oracle_sweeps_range(const oracle_system *sys, int n_walkers, double *pos, int32_t *n, int32_t *nb,
                        double *energy, const int32_t *state_of_walker, uint32_t t0,
                        int n_sweeps, oracle_hist *hist, oracle_move *trace,
                        int64_t *counts, int n_threads, int w_begin, int w_end)
{
    int S = n_states(sys);
    if (w_begin < 0 || w_end > n_walkers || w_begin > w_end) return -1;
    if (n_walkers != S || sys->nmax < 1 || sys->moves_per_sweep < 0 || n_sweeps < 0) return -1;
    if (sys->gc2_type > 0 && (!nb || sys->n_cluster > 0 || sys->da)) return -1;
    char *seen = (char *)calloc((size_t)S, 1);
    for (int w = 0; w < S; ++w) {
        int s = state_of_walker[w];
        if (s < 0 || s >= S || seen[s] || n[w] < 0 || n[w] > sys->nmax ||
            (nb && (nb[w] < 0 || nb[w] > n[w]))) {
            free(seen);
            return -1;
        }
        seen[s] = 1;
    }
    free(seen);
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int w = w_begin; w < w_end; ++w) {
        oracle_move *tr = trace ? trace + (int64_t)w * n_sweeps * sys->moves_per_sweep : NULL;
        sweep_walker(sys, w, pos + (int64_t)w * sys->nmax * 3, n + w, nb ? nb + w : NULL, energy + w,
                     state_of_walker[w], t0, n_sweeps, hist, tr, counts);
    }
    (void)n_threads;
    return 0;
}

/* ------------------------------------------------------------- exchange */

/* One collective replica-exchange attempt number e (Sec. II.A.2).  One of four
 * neighbour directions on the (T, mu) grid is drawn with probability 1/4
 * (T, mu, diagonal, anti-diagonal) together with a parity bit; every state
 * (l, m) whose row (column, for the mu direction) has that parity is paired
 * with its neighbour (l + dl, m + dm) if it exists.  Each pair swaps its
 * configurations with the probability of Eq. Pacc; a swap moves the state
 * labels of the two walkers, not their coordinates.
 * ex_counts, if given, is [S][4][attempts, accepts] indexed by the lower state.
 * Returns the number of accepted swaps, or -1 on invalid arguments. */
int oracle_exchange(const oracle_system *sys, uint32_t e, const int32_t *n,
                    const double *energy, int32_t *state_of_walker,
                    int32_t *walker_of_state, int64_t *ex_counts)
{
    if (sys->gc2_type > 0) return -1;   /* two species: oracle_exchange2 */
    return oracle_exchange2(sys, e, n, NULL, energy, state_of_walker, walker_of_state, ex_counts);
}

/* With a second species on a third axis (K > 1) a fifth direction joins the
 * four: type = (C0 * 5) >> 32, type 4 pairing (l, m, k) with (l, m, k + 1)
 * for k of the drawn parity; the other directions act in every k-slice
 * alike.  ex_counts is then [S][5][2]. */
int oracle_exchange2(const oracle_system *sys, uint32_t e, const int32_t *n, const int32_t *nb,
                     const double *energy, int32_t *state_of_walker,
                     int32_t *walker_of_state, int64_t *ex_counts)
{
    static const int DL[5] = {1, 0, 1, 1, 0};
    static const int DM[5] = {0, 1, 1, -1, 0};
    static const int DK[5] = {0, 0, 0, 0, 1};
    const int K = axis_K(sys), n_dir = K > 1 ? 5 : 4;
    int L = sys->L, M = sys->M, S = L * M * K;
    if (sys->gc2_type > 0 && !nb) return -1;
    for (int s = 0; s < S; ++s) {
        int w = walker_of_state[s];
        if (w < 0 || w >= S || state_of_walker[w] != s) return -1;
    }
    uint32_t C[4];
    draw(sys, e, 0u, 0u, 2u, C);
    int type = (int)(((uint64_t)C[0] * (uint64_t)n_dir) >> 32);
    int parity = (int)(C[1] >> 31);
    int accepted = 0;
    for (int l = 0; l < L; ++l) {
        for (int m = 0; m < M; ++m) {
          for (int k = 0; k < K; ++k) {
            int key = DK[type] ? k : (DL[type] ? l : m);
            if ((key & 1) != parity) continue;
            int l2 = l + DL[type], m2 = m + DM[type], k2 = k + DK[type];
            if (l2 < 0 || l2 >= L || m2 < 0 || m2 >= M || k2 >= K) continue;
            int a = (l * M + m) * K + k, b = (l2 * M + m2) * K + k2;
            int wa = walker_of_state[a], wb = walker_of_state[b];
            double la = nb ? oracle_exchange_log_alpha2(sys, a, b, nb[wa], n[wa] - nb[wa], nb[wb], n[wb] - nb[wb],
                                                        energy[wa], energy[wb])
                           : oracle_exchange_log_alpha(sys, a, b, n[wa], n[wb], energy[wa], energy[wb]);
            uint32_t D[4];
            draw(sys, e, (uint32_t)a, 0u, 3u, D);
            int acc = log(u32_open(D[0])) < la;
            if (ex_counts) {
                ex_counts[2 * n_dir * (int64_t)a + 2 * type] += 1;
                ex_counts[2 * n_dir * (int64_t)a + 2 * type + 1] += acc;
            }
            if (acc) {
                walker_of_state[a] = wb;
                walker_of_state[b] = wa;
                state_of_walker[wa] = b;
                state_of_walker[wb] = a;
                accepted += 1;
            }
          }
        }
    }
    return accepted;
}

/* ----------------------------------------------------------- REGC cycle */

/* The REGC cycle of Sec. II.A (Fig. 1), with the settings of Sec. III.A:
 * n_steps steps numbered t0, t0 + 1, ...  Step t draws G = Philox((t, 0, 0,
 * 10)).  If G0 < floor(x0 2^32) -- probability x0 -- every replica attempts
 * one particle exchange with the reservoir: move k = 0 of step t, an
 * insertion or a removal with equal probability (B2, as in the sweeps).
 * Otherwise one collective replica-exchange attempt is made (exchange numbers
 * e0, e0 + 1, ... in order).  Then every replica diffuses at fixed N with
 * moves k = 1 .. n_canonical of step t, all Metropolis displacements, and is
 * observed once after its last move of the step (n_canonical = 0 leaves a
 * replica-exchange step without moves and without an observation: REGCMD
 * runs its canonical diffusion as MD after the step).
 * trace, if given, is [n_walkers][n_steps][n_canonical + 1]; slot k = 0 of a
 * replica-exchange step holds type -1 and status 4 (not attempted).
 * counts and ex_counts as in oracle_sweeps and oracle_exchange.
 * Walkers are independent within a step: the loops over them are OpenMP
 * loops, as in oracle_sweeps.
 * Planted mistakes: 2048 swaps the two branches of the x0 choice; 4096 draws
 * the canonical moves from the mixed move set of the sweeps.
 * Returns the number of replica-exchange steps, or -1 on invalid arguments. */
int oracle_cycle(const oracle_system *sys, int n_walkers, double *pos, int32_t *n, double *energy,
                 int32_t *state_of_walker, int32_t *walker_of_state, uint32_t t0, uint32_t e0,
                 int n_steps, double x0, int n_canonical, oracle_hist *hist, oracle_move *trace,
                 int64_t *counts, int64_t *ex_counts)
{
    int S = sys->L * sys->M;
    if (sys->gc2_type > 0) return -1;   /* one grand-canonical species only */
    if (n_walkers != S || n_steps < 0 || n_canonical < 0 || !(x0 >= 0.0 && x0 <= 1.0)) return -1;
    for (int w = 0; w < S; ++w)
        if (n[w] < 0 || n[w] > sys->nmax || state_of_walker[w] < 0 || state_of_walker[w] >= S) return -1;
    const uint64_t th_gc = x0 >= 1.0 ? (uint64_t)1 << 32 : (uint64_t)floor(x0 * 4294967296.0);
    const int per_step = n_canonical + 1;
    const int canonical_kind = (sys->mutation & 4096) ? MOVE_MIXED : MOVE_DISPLACE;
    uint32_t e = e0;
    int n_exchange = 0;
    for (int ts = 0; ts < n_steps; ++ts) {
        const uint32_t t = t0 + (uint32_t)ts;
        uint32_t G[4];
        draw(sys, t, 0u, 0u, 10u, G);
        int gc = (uint64_t)G[0] < th_gc;
        if (sys->mutation & 2048) gc = !gc;
        if (gc) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
            for (int w = 0; w < S; ++w) {
                int nw = n[w];
                oracle_move mv;
                trial_move(sys, w, pos + (int64_t)w * sys->nmax * 3, &nw, &nw, energy + w, state_of_walker[w],
                           0u, t, MOVE_GC, &mv);
                n[w] = nw;
                count_move(counts, w, &mv);
                if (trace) trace[((int64_t)w * n_steps + ts) * per_step] = mv;
            }
        } else {
            if (oracle_exchange(sys, e, n, energy, state_of_walker, walker_of_state, ex_counts) < 0) return -1;
            e += 1;
            n_exchange += 1;
            if (trace) {
                for (int w = 0; w < S; ++w) {
                    oracle_move mv;
                    memset(&mv, 0, sizeof mv);
                    mv.type = -1;
                    mv.status = 4;
                    trace[((int64_t)w * n_steps + ts) * per_step] = mv;
                }
            }
        }
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
        for (int w = 0; w < S; ++w) {
            int nw = n[w];
            const int state = state_of_walker[w];
            double *pw = pos + (int64_t)w * sys->nmax * 3;
            for (int k = 1; k <= n_canonical; ++k) {
                oracle_move mv;
                trial_move(sys, w, pw, &nw, &nw, energy + w, state, (uint32_t)k, t, canonical_kind, &mv);
                count_move(counts, w, &mv);
                if (trace) trace[((int64_t)w * n_steps + ts) * per_step + k] = mv;
            }
            n[w] = nw;
            if (gc || n_canonical > 0) observe(sys, hist, state, w, nw - sys->n_cluster, 0, energy[w]);
        }
    }
    return n_exchange;
}

/* ------------------------------------------------------------------ MD */

/* Molecular dynamics between grand-canonical moves (REGCMD, Sec. II.A.3: the
 * canonical sampling step done by MD; Appendix: velocity Verlet with the
 * stochastic velocity rescaling thermostat).  Reduced units, unit masses.
 *
 * One segment of n_steps steps of length dt for walker w at its state's kT:
 *   - velocities are drawn from the Maxwell-Boltzmann distribution at kT
 *     (particle i: Philox counter (i, seg, w, 8), Box-Muller on words 0-1 and
 *     2-3, components x, y, z from the first three normals);
 *   - each step: the stochastic velocity rescaling thermostat of Bussi,
 *     Donadio & Parrinello (J. Chem. Phys. 126, 014101 (2007)) with time
 *     constant tau over dt on all 3N degrees of freedom (normals from
 *     counters (k, seg * n_steps + step, w, 9), k = 0, 1, ...: R1 is normal 0,
 *     the chi-square variable the sum of the squares of normals 1..3N-1), then
 *     one velocity-Verlet step: v += f dt/2, r += v dt, f = F(r), v += f dt/2;
 *   - F_i = -grad_i E: truncated LJ forces from every other particle and
 *     every surface atom within rc, nearest image;
 *   - x and y wrap periodically (z too in a periodic box); otherwise the walls
 *     at z_lo and z_hi reflect (z -> 2 z_wall - z, v_z -> -v_z);
 *   - at the end coordinates are rounded to binary32 and E is recomputed.
 * kin (if not NULL) receives the kinetic energy after the last step. */

static void normals4(const oracle_system *sys, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, double g[4])
{
    uint32_t u[4];
    draw(sys, c0, c1, c2, c3, u);
    for (int h = 0; h < 2; ++h) {
        double r = sqrt(-2.0 * log(u32_open(u[2 * h])));
        double a = 2.0 * M_PI * u32_open(u[2 * h + 1]);
        g[2 * h] = r * cos(a);
        g[2 * h + 1] = r * sin(a);
    }
}

static void md_forces(const oracle_system *sys, const double *pos, int n, double *f)
{
    const double rc2 = sys->rc * sys->rc;
    for (int i = 0; i < 3 * n; ++i) f[i] = 0.0;
    for (int i = 0; i < n; ++i) {
        const double *ri = pos + 3 * i;
        const int ti = species(sys, i);
        for (int j = -sys->n_surf; j < n; ++j) {
            if (j == i) continue;
            const double *rj;
            int tj;
            if (j < 0) {
                rj = sys->surf_xyz + 3 * (j + sys->n_surf);
                tj = sys->surf_type[j + sys->n_surf];
            } else {
                rj = pos + 3 * j;
                tj = species(sys, j);
            }
            double d[3];
            pair_vec(sys, ri[0], ri[1], ri[2], rj[0], rj[1], rj[2], d);
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 >= rc2) continue;
            double s2 = sys->sigma[ti][tj] * sys->sigma[ti][tj] / r2;
            double s6 = s2 * s2 * s2;
            /* -dphi/dr / r = 24 eps (2 s^12 - s^6) / r^2 */
            double g = 24.0 * sys->eps[ti][tj] * (2.0 * s6 * s6 - s6) / r2;
            if (sys->mutation & 1024) g = -g;
            for (int c = 0; c < 3; ++c) f[3 * i + c] += g * d[c];
        }
    }
}

static void md_walker(const oracle_system *sys, int w, double *pos, int n, double *e_ptr, int state,
                      uint32_t seg, int n_steps, double dt, double tau, double *kin)
{
    const double kT = kT_of(sys, state);
    double *v = (double *)malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    double *f = (double *)malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    const int nf = 3 * n;
    for (int i = 0; i < n; ++i) {
        double g[4];
        normals4(sys, (uint32_t)i, seg, (uint32_t)w, 8u, g);
        for (int c = 0; c < 3; ++c) v[3 * i + c] = sqrt(kT) * g[c];
    }
    md_forces(sys, pos, n, f);
    const double c_tau = exp(-dt / tau);
    for (int step = 0; step < n_steps && n > 0; ++step) {
        /* thermostat: rescale every velocity by alpha (Bussi et al.) */
        double K = 0.0;
        for (int i = 0; i < nf; ++i) K += 0.5 * v[i] * v[i];
        const double Kt = 0.5 * nf * kT;
        double r1 = 0.0, chi = 0.0;
        const uint32_t gstep = seg * (uint32_t)n_steps + (uint32_t)step;
        for (int k = 0; 4 * k < nf; ++k) {
            double g[4];
            normals4(sys, (uint32_t)k, gstep, (uint32_t)w, 9u, g);
            for (int h = 0; h < 4; ++h) {
                int idx = 4 * k + h;
                if (idx == 0) r1 = g[h];
                else if (idx < nf) chi += g[h] * g[h];
            }
        }
        if (K > 0.0) {
            double cross = (sys->mutation & 512) ? 0.0 : 2.0 * r1 * sqrt(c_tau * (1.0 - c_tau) * K * Kt / nf);
            double k_new = c_tau * K + (1.0 - c_tau) * Kt * (r1 * r1 + chi) / nf + cross;
            double alpha = sqrt(k_new / K);
            if (r1 + sqrt(c_tau * nf * K / ((1.0 - c_tau) * Kt)) < 0.0) alpha = -alpha;
            for (int i = 0; i < nf; ++i) v[i] *= alpha;
        }
        /* velocity Verlet */
        for (int i = 0; i < nf; ++i) v[i] += 0.5 * dt * f[i];
        for (int i = 0; i < n; ++i) {
            double *r = pos + 3 * i;
            /* the cell-frame u moves by vx - shear vy */
            r[0] += dt * (v[3 * i] - sys->shear * v[3 * i + 1]);
            r[1] += dt * v[3 * i + 1];
            r[2] += dt * v[3 * i + 2];
            r[0] -= sys->Lx * floor(r[0] / sys->Lx);
            r[1] -= sys->Ly * floor(r[1] / sys->Ly);
            if (sys->periodic_z) {
                r[2] -= sys->Lz * floor(r[2] / sys->Lz);
            } else {
                if (r[2] < sys->z_lo) { r[2] = 2.0 * sys->z_lo - r[2]; v[3 * i + 2] = -v[3 * i + 2]; }
                if (r[2] > sys->z_hi) { r[2] = 2.0 * sys->z_hi - r[2]; v[3 * i + 2] = -v[3 * i + 2]; }
            }
        }
        md_forces(sys, pos, n, f);
        for (int i = 0; i < nf; ++i) v[i] += 0.5 * dt * f[i];
    }
    if (kin) {
        double K = 0.0;
        for (int i = 0; i < nf; ++i) K += 0.5 * v[i] * v[i];
        *kin = K;
    }
    for (int i = 0; i < 3 * n; ++i) pos[i] = f32(pos[i]);
    for (int i = 0; i < n; ++i) {
        /* binary32 rounding may put a coordinate on the upper boundary */
        double *r = pos + 3 * i;
        if (r[0] >= f32(sys->Lx)) r[0] = 0.0;
        if (r[1] >= f32(sys->Ly)) r[1] = 0.0;
        if (sys->periodic_z && r[2] >= f32(sys->Lz)) r[2] = 0.0;
    }
    *e_ptr = oracle_total_energy(sys, pos, n);
    free(v);
    free(f);
}

int oracle_md(const oracle_system *sys, int n_walkers, double *pos, const int32_t *n, double *energy,
              const int32_t *state_of_walker, uint32_t seg, int n_steps, double dt, double tau, double *kin,
              int n_threads)
{
    int S = sys->L * sys->M;
    if (sys->gc2_type > 0) return -1;   /* one grand-canonical species only */
    if (n_walkers != S || n_steps < 0 || !(dt > 0.0) || !(tau > 0.0)) return -1;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int w = 0; w < S; ++w)
        md_walker(sys, w, pos + (int64_t)w * sys->nmax * 3, n[w], energy + w, state_of_walker[w], seg, n_steps, dt,
                  tau, kin ? kin + w : NULL);
    (void)n_threads;
    return 0;
}

/* Forces F_i = -grad_i E on the n mobile particles (the MD forces), f [n][3]. */
void oracle_forces(const oracle_system *sys, const double *pos, int n, double *f)
{
    md_forces(sys, pos, n, f);
}
