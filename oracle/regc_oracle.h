/*
 * regc_oracle.h -- FP64 CPU oracle of the replica-exchange grand-canonical
 * Monte Carlo (REGCMC) sampler of Zhou, Scheffler & Ghiringhelli,
 * "Determining Surface Phase Diagrams Including Anharmonic Effects"
 * (arXiv:1908.11118).
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle exists to check the CUDA library
 * against a plain, slow, obviously correct restatement of the method.  Only
 * the tests, the smoke check and the CPU-baseline leg of the benchmark may
 * load it.  It shares no code, header, table or constant with the CUDA path.
 *
 * Everything is double precision.  Particle coordinates are kept on values
 * that are exactly representable in binary32 (every coordinate update is
 * rounded through float), so that a binary32 implementation that performs
 * the same coordinate arithmetic holds bit-identical configurations while
 * its accept/reject decisions agree with this one.
 */
#ifndef REGC_ORACLE_H
#define REGC_ORACLE_H
#include <stdint.h>

#define ORACLE_MAX_TYPES 4

/* Problem statement: the potential, the surface, the gas region and the
 * (T, mu) grid (Sec. I: the method takes only the potential-energy function
 * and the T and mu ranges as inputs). */
typedef struct {
    /* truncated Lennard-Jones 12-6 pair potential (Appendix, force field):
     * phi(r) = 4 eps [(sigma/r)^12 - (sigma/r)^6] for r < rc, else 0.
     * Type 0 is the mobile (grand-canonical) species; surface atoms carry
     * types 1..n_types-1. */
    int    n_types;
    double eps[ORACLE_MAX_TYPES][ORACLE_MAX_TYPES];
    double sigma[ORACLE_MAX_TYPES][ORACLE_MAX_TYPES];
    double rc;
    /* box: x and y periodic; z periodic only if periodic_z */
    double Lx, Ly, Lz;
    int    periodic_z;
    /* region available to mobile particles, z_lo <= z <= z_hi (Sec. III.A:
     * insertion only in the zone above the top surface layer) */
    double z_lo, z_hi;
    /* frozen surface atoms (species A of Sec. III.A) */
    int           n_surf;
    const double *surf_xyz;   /* [n_surf][3] */
    const int    *surf_type;  /* [n_surf]    */
    /* replica grid S = L x M, state s = l*M + m (Sec. II.A.2) */
    int           L, M;
    const double *kT;         /* [L] */
    const double *mu;         /* [M] */
    double        lambda0;    /* thermal wavelength Lambda(kT) = lambda0/sqrt(kT) */
    /* move set */
    int    nmax;              /* capacity: insertion at N = nmax is rejected */
    int    moves_per_sweep;
    double max_disp;          /* half-edge of the displacement cube */
    double p_disp;            /* probability of a displacement; GC gets the rest, 50/50 */
    uint64_t seed;            /* Philox key */
    /* pooled (N, E) histogram: bin k covers [e_lo + k*e_bin, e_lo + (k+1)*e_bin) */
    double e_lo, e_bin;
    int    n_e_bins;
    /* planted-mistake switches for sensitivity tests of the pins; 0 in all
     * real use (bit meanings in regc_oracle.c) */
    int    mutation;
    /* delayed acceptance: when da != 0, sur_theta holds the 5313 parameters
     * of the surrogate network (layout in oracle/surrogate.py) */
    int           da;
    const double *sur_theta;
    /* a second mobile species (the cluster of configuration 5; not in the
     * paper): particles 0..n_cluster-1 of every walker have potential type
     * cluster_type and move only by displacement; insertion and removal act on
     * the grand-canonical species (type 0), whose count N_B = N - n_cluster
     * enters the acceptance ratios and the histograms */
    int           n_cluster;
    int           cluster_type;
    /* sheared cell: lattice vectors (Lx, 0) and (shear Ly, Ly); x coordinates
     * are the cell-frame u = x - shear y (0: rectangular) */
    double        shear;
    /* a second grand-canonical species C (more than one reactive gas, the
     * outlook of Sec. IV; gc2_type 0: none): potential type gc2_type
     * (1..n_types-1), chemical potentials mu2[K] on a third axis of the grid
     * (state s = (l M + m) K + k holds kT[l], mu[m], mu2[k]) and thermal
     * wavelength lambda0_2 / sqrt(kT).  A walker's particles [0, N_B) are
     * species B (type 0), [N_B, N) species C.  Not combined with a cluster. */
    int           gc2_type;
    int           K;
    const double *mu2;
    double        lambda0_2;
} oracle_system;

/* One trial move as the oracle executed it. */
typedef struct {
    int32_t type;       /* 0 displace, 1 insert, 2 delete */
    int32_t index;      /* particle touched (insert: the new slot N) */
    int32_t accepted;   /* 1 accepted, 0 rejected */
    int32_t status;     /* 0 energy evaluated, 1 rejected at the N boundary,
                           2 displacement left the region */
    double  dE;         /* energy change of the move (0 unless status 0) */
    double  log_alpha;  /* log of the acceptance ratio (status 0 only) */
    double  ln_u;       /* log of the acceptance uniform */
    double  sum_abs;    /* sum of 4 eps [(s/r)^12 + (s/r)^6] over pairs entering dE */
    double  band;       /* sum of |phi(rc)| over pairs with r^2 within 4e-6 rc^2 of rc^2 */
    int32_t n_pairs;    /* pairs with r < rc entering dE */
    int32_t stage1;     /* delayed acceptance: 1 if the surrogate stage accepted */
    double  dE_sur;     /* delayed acceptance: surrogate energy change */
    double  ln_u1;      /* delayed acceptance: ln of the stage-1 uniform */
} oracle_move;

/* Histograms filled once per sweep, at the walker's current state. */
/* With a cluster, N below means N_B, the grand-canonical count. */
typedef struct {
    int64_t *hN;        /* [S][nmax+1] occupation counts of N            */
    int64_t *hNE;       /* [nmax+1][n_e_bins] pooled (N, E-bin) counts   */
    int64_t *omega;     /* [S] observations per state                    */
    double  *moments;   /* [S][4]: sum N, sum N^2, sum E, sum E^2        */
    int64_t *e_out;     /* [S] observations with E outside the E window  */
    /* per-state energy histograms (NULL: none): state s has hE_bins bins of
     * width hE_bin from hE_lo[s], bin 0 below the window, k + 1 for window bin
     * k, hE_bins + 1 at or beyond its end */
    int64_t      *hE;        /* [S][hE_bins + 2] */
    const double *hE_lo;     /* [S] */
    double        hE_bin;
    int           hE_bins;
    /* second species (gc2_type != 0): occupation counts of N_C and its
     * moments; hN and moments then hold N_B, and the pooled histogram is
     * [(nmax+1)^2][n_e_bins] with row N_B (nmax+1) + N_C */
    int64_t      *hN2;       /* [S][nmax+1] */
    double       *moments2;  /* [S][2]: sum N_C, sum N_C^2 */
} oracle_hist;

#ifdef __cplusplus
extern "C" {
#endif
void   oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double oracle_phi(const oracle_system *sys, int ti, int tj, double r2);
double oracle_particle_energy(const oracle_system *sys, const double *pos, int n,
                              double x, double y, double z, int skip,
                              double *sum_abs, double *band, int *n_pairs);
double oracle_total_energy(const oracle_system *sys, const double *pos, int n);
double oracle_surrogate_energy(const oracle_system *sys, const double *pos, int n,
                               double x, double y, double z, int skip, double *feat);
double oracle_log_alpha(const oracle_system *sys, int type, int state, int n, double dE);
double oracle_exchange_log_alpha(const oracle_system *sys, int sa, int sb,
                                 int na, int nb, double ea, double eb);
int    oracle_sweeps(const oracle_system *sys, int n_walkers, double *pos, int32_t *n,
                     double *energy, const int32_t *state_of_walker, uint32_t t0,
                     int n_sweeps, oracle_hist *hist, oracle_move *trace,
                     int64_t *counts, int n_threads);
int    oracle_cycle(const oracle_system *sys, int n_walkers, double *pos, int32_t *n, double *energy,
                    int32_t *state_of_walker, int32_t *walker_of_state, uint32_t t0, uint32_t e0,
                    int n_steps, double x0, int n_canonical, oracle_hist *hist, oracle_move *trace,
                    int64_t *counts, int64_t *ex_counts);
void   oracle_forces(const oracle_system *sys, const double *pos, int n, double *f);
int    oracle_md(const oracle_system *sys, int n_walkers, double *pos, const int32_t *n, double *energy,
                 const int32_t *state_of_walker, uint32_t seg, int n_steps, double dt, double tau,
                 double *kin, int n_threads);
int    oracle_exchange(const oracle_system *sys, uint32_t e, const int32_t *n,
                       const double *energy, int32_t *state_of_walker,
                       int32_t *walker_of_state, int64_t *ex_counts);
/* Two grand-canonical species: nb [walkers] holds each walker's N_B (its
 * particles [0, N_B) are species B, the rest species C).  The exchange has a
 * fifth direction, mu2 (ex_counts [S][5][2]) when K > 1. */
double oracle_particle_energy2(const oracle_system *sys, const double *pos, int n, int nb,
                               double x, double y, double z, int skip, int species_new,
                               double *sum_abs, double *band, int *n_pairs);
double oracle_total_energy2(const oracle_system *sys, const double *pos, int n, int nb);
double oracle_log_alpha2(const oracle_system *sys, int type, int species, int state, int n_c, double dE);
double oracle_exchange_log_alpha2(const oracle_system *sys, int sa, int sb, int nba, int nca,
                                  int nbb, int ncb, double ea, double eb);
int    oracle_sweeps2(const oracle_system *sys, int n_walkers, double *pos, int32_t *n, int32_t *nb,
                      double *energy, const int32_t *state_of_walker, uint32_t t0,
                      int n_sweeps, oracle_hist *hist, oracle_move *trace,
                      int64_t *counts, int n_threads);
/* oracle_sweeps2 for walkers [w_begin, w_end) only */
int    oracle_sweeps_range(const oracle_system *sys, int n_walkers, double *pos, int32_t *n, int32_t *nb,
                           double *energy, const int32_t *state_of_walker, uint32_t t0,
                           int n_sweeps, oracle_hist *hist, oracle_move *trace,
                           int64_t *counts, int n_threads, int w_begin, int w_end);
int    oracle_exchange2(const oracle_system *sys, uint32_t e, const int32_t *n, const int32_t *nb,
                        const double *energy, int32_t *state_of_walker,
                        int32_t *walker_of_state, int64_t *ex_counts);
#ifdef __cplusplus
}
#endif
#endif
