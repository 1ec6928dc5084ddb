/*
 * regc.h -- C ABI of the GB300 (sm_103a) replica-exchange grand-canonical
 * Monte Carlo (REGCMC) library.
 *
 * Method: Y. Zhou, M. Scheffler, L. M. Ghiringhelli, "Determining Surface
 * Phase Diagrams Including Anharmonic Effects", arXiv:1908.11118.
 *   Sec. II.A    -- the REGC cycle: grand-canonical moves, replica exchange,
 *                   canonical diffusion, iterated
 *   Sec. II.A.1  -- insertion / removal and their acceptance probabilities
 *   Sec. II.A.2  -- the extended (T, mu) ensemble and the swap rule (Eq. Pacc)
 *   Sec. II.A.3  -- Metropolis displacement
 *   Sec. II.B    -- MBAR reweighting to phase diagrams (Eqs. textbook,
 *                   grandpot, normlizationconstant)
 *   Appendix     -- the Lennard-Jones 12-6 force field
 *
 * Conventions common to every entry point:
 *   - Reduced units: k_B = 1, energies in eps, lengths in sigma.
 *   - Every call returns a regc_status; nothing aborts or exits.  A CUDA error
 *     makes the handle's status sticky: later calls on that handle return it.
 *   - Pointers named host_* or documented "host" are host memory owned by the
 *     caller; inputs are copied before the call returns, outputs are written
 *     before it returns (the call synchronises its stream when it returns
 *     data).  The library allocates and frees its own device memory.
 *   - All device work of a handle is issued on the CUDA stream given to
 *     regc_init_grid (NULL = the legacy default stream).
 *   - One handle must not be used by two host threads at once.
 *
 * Move and random-number conventions (needed to reproduce a run exactly):
 *   Philox4x32-10 (Salmon et al., SC'11), key = (seed low, seed high) words.
 *   Trial move k of sweep t of walker w draws two blocks,
 *     A = Philox(ctr = (k, t, w, 0)), B = Philox(ctr = (k, t, w, 1)):
 *     A0 < floor(p_disp 2^32)      -> displacement, else grand-canonical move,
 *     B2 >> 31 == 0                -> removal, else insertion (y1 < 0.5 -> removal),
 *     i = (B0 * N) >> 32           -> particle picked by displacement / removal,
 *     U24(a) = (a >> 8) 2^-24      -> displacement d_c = max_disp (2 U24(A_{c+1}) - 1),
 *                                     insertion point (Lx U24(A1), Ly U24(A2),
 *                                     z_lo + (z_hi - z_lo) U24(A3)),
 *     u = (B1 + 0.5) 2^-32         -> accept iff ln u < ln(acceptance ratio).
 *   Coordinates are binary32 and every coordinate operation is one IEEE
 *   round-to-nearest binary32 operation, in the order written above.
 *   Exchange number e draws C = Philox((e, 0, 0, 2)) (direction (C0 * 4) >> 32,
 *   parity C1 >> 31) and, for the pair whose lower state index is a,
 *   D = Philox((e, a, 0, 3)), u = (D0 + 0.5) 2^-32.
 *   Step t of the REGC cycle (regc_cycle) chooses particle or replica
 *   exchange from Philox((t, 0, 0, 10)).
 */
#ifndef REGC_H
#define REGC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define REGC_API __attribute__((visibility("default")))
#else
#define REGC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct regc_handle regc_handle;   /* opaque; owned by the library */

typedef enum {
    REGC_OK = 0,
    REGC_EINVAL = -1,     /* an argument is out of range; nothing was changed    */
    REGC_ENOMEM = -2,     /* a device or host allocation failed                  */
    REGC_ECUDA = -3,      /* a CUDA call failed (sticky on the handle)           */
    REGC_ETIMEOUT = -4,   /* a bounded device wait gave up (sticky)              */
    REGC_ECAPACITY = -5,  /* a cell of a walker's cell list overflowed (sticky):
                             the move that needed the slot was rejected, so the
                             chain from that point on is not the exact one       */
    REGC_ENUMERIC = -6    /* a non-finite or out-of-range energy was detected    */
} regc_status;

/* Truncated Lennard-Jones 12-6 pair potential (Appendix, force field):
 * phi_ij(r) = 4 eps[ti][tj] ((sigma[ti][tj]/r)^12 - (sigma[ti][tj]/r)^6) for
 * r < rc, 0 otherwise.  Type 0 is the mobile, grand-canonical species (B of
 * Sec. III.A); frozen surface atoms carry types 1..n_types-1 (A).  Tables are
 * symmetric; entries outside n_types are ignored. */
typedef struct {
    int   n_types;          /* 1..4 */
    float eps[4][4];
    float sigma[4][4];
    float rc;               /* > 0; Lx, Ly (and Lz if periodic) must be >= 2 rc */
} regc_potential;

/* Frozen surface slab and the box (Sec. II.A.1: the subsystem of volume V in
 * contact with the reservoir; Sec. III.A: insertion only in the zone above the
 * topmost surface layer).  x and y are periodic with periods Lx, Ly.  Mobile
 * particles live in z_lo <= z <= z_hi; if periodic_z, z is periodic with period
 * Lz and the region is the whole box (z_lo = 0, z_hi = Lz required).
 * V = Lx Ly (z_hi - z_lo) enters the acceptance rules. */
typedef struct {
    int          n_atoms;   /* >= 0 */
    const float *xyz;       /* host [n_atoms][3]; x in [0, Lx), y in [0, Ly) */
    const int   *type;      /* host [n_atoms]; 1..n_types-1                  */
    float        Lx, Ly, Lz;
    int          periodic_z;
    float        z_lo, z_hi;
    float        shear;     /* |shear| <= 1; 0 for a rectangular cell.  The
                               cell's lattice vectors in the xy plane are
                               (Lx, 0) and (shear Ly, Ly) -- 1/sqrt(3) for the
                               hexagonal cell of an fcc(111) surface.  Every
                               x coordinate of the ABI (surface atoms and
                               walkers) is then the cell-frame u = x - shear y,
                               in [0, Lx); the box needs
                               rc sqrt(1 + shear^2) <= Lx / 2 and rc <= Ly / 2,
                               and a displacement move is uniform in a cube
                               of the cell frame (u, y, z). */
} regc_surface;

/* The (T, mu) grid of replicas (Sec. II.A.2: S = L x M states; state
 * s = l M + m holds (kT[l], mu[m])) and the move set. */
typedef struct {
    int           L, M;             /* L * M <= 65536 */
    const double *kT;               /* host [L], > 0  */
    const double *mu;               /* host [M]       */
    double        lambda0;          /* Lambda(kT) = lambda0 / sqrt(kT) (Eq. Ngrand) */
    int           nmax;             /* 1..4096: insertion at N = nmax is rejected   */
    int           moves_per_sweep;  /* 1..1024 trial moves per sweep                */
    float         max_disp;         /* half-edge of the displacement cube (Sec. II.A.3) */
    double        p_disp;           /* probability of a displacement move, [0, 1]   */
    double        e_lo, e_bin;      /* pooled (N, E) histogram: bin k covers        */
    int           n_e_bins;         /*   [e_lo + k e_bin, e_lo + (k+1) e_bin)       */
} regc_grid_spec;

/* One trial move, as recorded by regc_sweep_traced. */
typedef struct {
    int32_t type;        /* 0 displacement, 1 insertion, 2 removal (-1: none)      */
    int32_t index;       /* particle moved or removed; insertion: the new slot N  */
    int32_t accepted;    /* 1 if accepted                                          */
    int32_t status;      /* 0 energy evaluated, 1 rejected at N = 0 or N = nmax,
                            2 displacement left [z_lo, z_hi], 4 not attempted
                            (regc_cycle_traced; type is then -1)                   */
    double  dE;          /* energy change of the move (status 0); NaN when delayed
                            acceptance rejected the move at stage 1 (dE is then
                            never computed)                                        */
    double  log_alpha;   /* ln of the plain acceptance ratio (status 0), -inf for a
                            move inside the hard-core guard, NaN with dE           */
    double  ln_u;        /* ln of the acceptance uniform                           */
    double  sum_abs;     /* unused by the GPU path (0)                             */
    double  band;        /* unused by the GPU path (0)                             */
    int32_t n_pairs;     /* pairs with r < rc that entered dE                      */
    int32_t stage1;      /* delayed acceptance: 1 if the surrogate stage accepted
                            (always 1 otherwise)                                   */
    double  dE_sur;      /* delayed acceptance: surrogate energy change            */
    double  ln_u1;       /* ln of the stage-1 uniform (from B3)                    */
} regc_move_record;

/* Create a handle: copies the problem statement, builds the surface lookup
 * tables and the per-state constants, allocates the walker state and the
 * histograms on the device and sets every walker to N = 0 at state s = w.
 * seed keys every Philox stream.  cuda_stream is a cudaStream_t (or NULL).
 * Errors: REGC_EINVAL (bad sizes, box smaller than 2 rc, nmax beyond the
 * shared-memory budget of one walker), REGC_ENOMEM, REGC_ECUDA.  On error
 * *out is NULL. */
REGC_API regc_status regc_init_grid(const regc_potential *pot, const regc_surface *surf,
                           const regc_grid_spec *grid, uint64_t seed, void *cuda_stream,
                           regc_handle **out);

/* A second grand-canonical species C: more than one reactive gas (the
 * outlook of Sec. IV).  The grid gains a third axis: state
 * s = (l M + m) K + k holds kT[l], mu[m] of species B (type 0) and mu[k] of
 * species C, and S = L M K.  Species C is inserted and removed by the rules
 * of Sec. II.A.1 with its own chemical potential and thermal wavelength
 * Lambda_C(kT) = lambda0 / sqrt(kT); a grand-canonical move picks its species
 * by bit 30 of Philox word B2 (0: B, 1: C), then removal or insertion by bit
 * 31 as for one species; removal picks uniformly among the particles of that
 * species.  Displacement picks among all N particles.  A walker keeps its B
 * particles at indices [0, N_B) and its C particles at [N_B, N): a new B takes
 * index N_B (the C there moves to the end), a removed B's index is filled by
 * the last B and that one's by the last C; a new C is appended, a removed C
 * replaced by the last particle.  The exchange of Eq. Pacc takes both
 * species: ln alpha = 1.5 (N_a - N_b) ln(b_a / b_b) - (b_a - b_b)(E_b - E_a)
 * - (b_a mu_a - b_b mu_b)(N_B,a - N_B,b) - (b_a mu2_a - b_b mu2_b)(N_C,a - N_C,b)
 * (both wavelengths scale as b^(1/2)), and with K > 1 a fifth direction
 * along mu2 joins the four, drawn as (C0 * 5) >> 32, pairing (l, m, k) with
 * (l, m, k + 1) for k of the drawn parity (the others act within every
 * k-slice).  Histograms: hN and the moments hold N_B, regc_histograms2 gives
 * N_C's; the pooled histogram has (nmax + 1)^2 rows, row N_B (nmax + 1) + N_C.
 * Not available with two species: the cluster, delayed acceptance, MD, the
 * REGC cycle, structural samples, surrogate evaluation and harvesting, batches
 * and regc_reweight (regc_reweight2 instead). */
typedef struct {
    int           type;      /* potential type of species C, 1..n_types-1 */
    int           K;         /* >= 1; L M K <= 65536 */
    const double *mu;        /* host [K], finite */
    double        lambda0;   /* > 0 */
} regc_species2;

/* As regc_init_grid, with a second grand-canonical species.  Every walker
 * starts empty.  Errors: those of regc_init_grid, and REGC_EINVAL for a bad
 * species2 or (nmax + 1)^2 n_e_bins beyond 2^31. */
REGC_API regc_status regc_init_grid2(const regc_potential *pot, const regc_surface *surf,
                                     const regc_grid_spec *grid, const regc_species2 *species2,
                                     uint64_t seed, void *cuda_stream, regc_handle **out);

/* Run n_sweeps sweeps (n_sweeps x moves_per_sweep trial moves) on every walker
 * (Sec. II.A.1 insertion/removal, Sec. II.A.3 displacement) at the walkers'
 * current states, and observe each walker once per sweep into its state's
 * histograms: hN[s][N] += 1, omega[s] += 1, moments[s] += (N, N^2, E, E^2),
 * pooled hNE[N][bin(E)] += 1 (Sec. II.B: samples Omega_{l,m} per state).
 * Asynchronous on the handle's stream.  Errors: REGC_EINVAL (n_sweeps < 0),
 * the handle's sticky status. */
REGC_API regc_status regc_sweep(regc_handle *h, int n_sweeps);

/* Failure-detection test hook (no paper counterpart): the next regc_sweep
 * on h launches with its walkers issuing no bulk copy of their positions, so
 * each walker's bounded wait on that copy (about 1 s of clock cycles, taken
 * twice) expires, the walker stops without touching its state, and the
 * handle's status becomes REGC_ETIMEOUT (sticky), reported by the next call
 * that synchronises.  No GPU fault, trap or hang is involved: the wait ends
 * by its own budget and the CUDA context stays usable.  Errors: REGC_EINVAL
 * (h NULL). */
REGC_API regc_status regc_test_expire_waits(regc_handle *h);

/* As regc_sweep, and write one record per trial move to host memory:
 * trace is [S walkers][n_sweeps][moves_per_sweep].  Synchronous.  Intended
 * for move-by-move comparison with a reference implementation. */
REGC_API regc_status regc_sweep_traced(regc_handle *h, int n_sweeps, regc_move_record *trace);

/* REGCMD: one molecular-dynamics segment of every walker (Sec. II.A.3: the
 * canonical sampling between grand-canonical and exchange moves done by MD;
 * Appendix: velocity Verlet with the stochastic velocity rescaling thermostat
 * of Bussi, Donadio & Parrinello 2007).  Reduced units, unit masses.  Each
 * walker, at its state's kT:
 *   - velocities are drawn from the Maxwell-Boltzmann distribution (particle
 *     i: Philox counter (i, segment, walker, 8), Box-Muller);
 *   - n_steps steps: the thermostat (time constant tau, all 3N degrees of
 *     freedom, normals from counters (k, segment * n_steps + step, walker, 9)),
 *     then v += f dt/2, r += v dt, f = F(r), v += f dt/2, with F the truncated
 *     LJ forces of the other particles and the surface (binary32);
 *   - x and y are periodic (z too in a periodic box); otherwise the walls at
 *     z_lo and z_hi reflect;
 *   - the exact energies are recomputed at the end.
 * Use it in place of displacement moves (p_disp = 0) alternated with
 * regc_sweep; velocities do not persist between segments.  kinetic [S] (host,
 * may be NULL) receives each walker's kinetic energy after the last step
 * (synchronous then; asynchronous otherwise).  Errors: REGC_EINVAL (n_steps < 0,
 * dt or tau not positive, walkers missing after regc_set_cluster),
 * REGC_ENUMERIC (a pair came inside the hard-core guard: the time step is far
 * too long), REGC_ECAPACITY (a cell overflowed). */
REGC_API regc_status regc_md(regc_handle *h, int n_steps, float dt, float tau, float *kinetic);

/* One collective replica-exchange attempt (Sec. II.A.2, Eq. Pacc): a direction
 * (T, mu, diagonal, anti-diagonal) and a parity are drawn; every state of that
 * parity swaps with its neighbour in that direction with probability
 * min[1, (b_a/b_b)^{3/2 (N_a - N_b)} exp(-(b_a - b_b)(E_b - E_a)
 *                                          - (b_a mu_a - b_b mu_b)(N_a - N_b))],
 * where state a holds (N_a, E_a).  A swap exchanges the walkers' state labels.
 * Asynchronous.  The exchange counter advances by one per call. */
REGC_API regc_status regc_exchange(regc_handle *h);

/* ------------------------------------------------- one grid over several GPUs
 *
 * The paper runs its S replicas on S groups of cores that meet only at the
 * replica exchange (Sec. II.A.4); the grid splits the same way over GPUs.
 * Every process creates the same grid (same problem, seed and walkers), and
 * process r steps only its own range of walkers.  Between two exchanges the
 * walkers are independent; an exchange attempt (Sec. II.A.2, Eq. Pacc) reads
 * only every walker's N and E and moves only state labels, so before each
 * attempt the processes all-gather (N, E) of their ranges, write the other
 * ranges into their handles with regc_set_walker_ne, and call regc_exchange.
 * The exchange draws its direction, parity and uniforms from the shared Philox
 * stream, so every process takes the same decisions and keeps the same state
 * labels; configurations never move between processes.  Each process's
 * histograms count only its own walkers' observations: their sum over the
 * processes is the grid's.  With the same Philox key, sweep and exchange
 * counters, a sharded run is the single-process run walker for walker. */

/* Step only walkers [w_begin, w_end) in regc_sweep from now on (default
 * [0, S)).  Calls that need every walker's configuration refuse a handle with
 * a proper shard (REGC_EINVAL): regc_sweep_traced, regc_cycle*, regc_md,
 * regc_surrogate_harvest, regc_structure_sample and batches; regc_check_energy
 * checks the shard's walkers only.  Errors: REGC_EINVAL (0 <= w_begin <
 * w_end <= S violated). */
REGC_API regc_status regc_set_shard(regc_handle *h, int w_begin, int w_end);

/* Particle counts and exact running energies of walkers [w_begin, w_end) into
 * host buffers: n and nb [w_end - w_begin] (nb: species B, two-species handles
 * only, else may be NULL), efix [w_end - w_begin] in units of 2^-30 of the
 * energy unit (the library's exact fixed-point totals; E = efix * 2^-30).
 * Synchronous.  Errors: REGC_EINVAL (range outside [0, S], a NULL buffer). */
REGC_API regc_status regc_get_walker_ne(regc_handle *h, int w_begin, int w_end, int32_t *n, int32_t *nb,
                                        int64_t *efix);

/* Overwrite N (and N_B) and the running energies of walkers [w_begin, w_end)
 * with the values another process owns (layout as regc_get_walker_ne); their
 * positions here are left as they are, so only regc_exchange should read those
 * walkers until they are owned again.  Synchronous.  Errors: REGC_EINVAL (range
 * outside [0, S], a NULL buffer, N outside [0, nmax] or N_B outside [0, N]). */
REGC_API regc_status regc_set_walker_ne(regc_handle *h, int w_begin, int w_end, const int32_t *n,
                                        const int32_t *nb, const int64_t *efix);

/* n_steps steps of the REGC cycle (Sec. II.A and its flow chart, Fig. 1;
 * Sec. III.A uses x0 = 0.99 and ten MC moves per step).  Step t (the sweep
 * counter: steps and sweeps share it) draws G = Philox((t, 0, 0, 10)):
 *   - G0 < floor(x0 2^32) (probability x0): every walker attempts one
 *     particle exchange with the reservoir, trial move k = 0 of sweep t, an
 *     insertion or a removal with equal probability (B2 as in a sweep; A0 is
 *     not used);
 *   - otherwise one collective replica-exchange attempt, as regc_exchange
 *     (the exchange counter advances by one);
 * then every walker makes n_canonical Metropolis displacements at fixed N,
 * trial moves k = 1 .. n_canonical of sweep t (A0 not used), and is observed
 * once into its state's histograms after its last move of the step, as after
 * a sweep (with n_canonical = 0 a replica-exchange step has no move and no
 * observation).  moves_per_sweep and
 * p_disp of the grid spec play no part.  Runs between two replica exchanges
 * go to the device as one launch.  n_exchanges (host, may be NULL) receives
 * the number of replica-exchange steps.  Asynchronous.  Errors: REGC_EINVAL
 * (n_steps < 0, n_canonical outside 0..1023, x0 outside [0, 1] or NaN,
 * walkers missing after regc_set_cluster), the handle's sticky status. */
REGC_API regc_status regc_cycle(regc_handle *h, int n_steps, double x0, int n_canonical, int *n_exchanges);

/* REGCMD (Sec. II.A, Fig. 1, with MD as the canonical sampler; Appendix):
 * n_steps steps, each one step of regc_cycle with n_canonical = 0 (the x0
 * choice, then a particle-exchange attempt per walker or a collective
 * replica-exchange attempt) followed by one MD segment of md_steps steps of
 * length dt with thermostat time constant tau, as regc_md.  Walkers are
 * observed after their particle-exchange attempts.  n_exchanges (host, may
 * be NULL) receives the replica-exchange steps.  Asynchronous.  Errors: those
 * of regc_cycle and regc_md. */
REGC_API regc_status regc_cycle_md(regc_handle *h, int n_steps, double x0, int md_steps, float dt, float tau,
                                   int *n_exchanges);

/* As regc_cycle, and write one record per trial move to host memory: trace is
 * [S walkers][n_steps][n_canonical + 1], slot k of step t holding move k of
 * that step; slot 0 of a replica-exchange step is not attempted and holds
 * type -1, status 4, all else 0.  Synchronous. */
REGC_API regc_status regc_cycle_traced(regc_handle *h, int n_steps, double x0, int n_canonical,
                                       regc_move_record *trace, int *n_exchanges);

/* Copy the histograms to caller-owned host buffers (any may be NULL):
 * hN [S][nmax+1], hNE [nmax+1][n_e_bins] (with a second species
 * [(nmax+1)^2][n_e_bins], row N_B (nmax+1) + N_C), omega [S], moments [S][4]
 * (sum N, sum N^2, sum E, sum E^2), e_out [S] (observations with E outside
 * the E window).  Synchronous. */
REGC_API regc_status regc_histograms(regc_handle *h, int64_t *hN, int64_t *hNE, int64_t *omega,
                            double *moments, int64_t *e_out);

/* Second species: hN2 [S][nmax+1] occupation counts of N_C and moments2
 * [S][2] (sum N_C, sum N_C^2) per state (host, either may be NULL).
 * Synchronous.  Errors: REGC_EINVAL (one species). */
REGC_API regc_status regc_histograms2(regc_handle *h, int64_t *hN2, double *moments2);

/* Zero every histogram and counter (not the walkers). */
REGC_API regc_status regc_reset_histograms(regc_handle *h);

/* Per-state energy histograms (Sec. II.B: the observations Omega_{l,m} of
 * each state; Sec. III.A judges convergence by each state's distribution of
 * the reduced energy).  Every state s gets its own window of n_bins bins of
 * width e_bin starting at e_lo[s], plus an underflow and an overflow bin:
 * from now on each observation of a walker at state s (the same observations
 * as hN) adds one count to
 *   hE[s][0]           if E < e_lo[s],
 *   hE[s][k + 1]       if e_lo[s] + k e_bin <= E < e_lo[s] + (k + 1) e_bin,
 *   hE[s][n_bins + 1]  if E >= e_lo[s] + n_bins e_bin.
 * e_lo: host [S], or NULL to centre each state's window on the mean energy
 * observed at that state so far (moments E sum / omega; 0 for a state never
 * observed), e_lo[s] = mean - n_bins e_bin / 2.  The origins and the width are
 * rounded to the library's energy grid of 2^-30 (regc_state_histograms
 * returns the values used).  Replaces earlier windows and zeroes the
 * per-state histograms; n_bins = 0 switches them off.  regc_reset_histograms
 * zeroes them too; checkpoints carry them (restore into a handle with windows
 * of the same n_bins).  Set windows before creating a batch that holds the
 * handle.  Synchronous.  Errors: REGC_EINVAL (n_bins outside 0..2^20, e_bin
 * below 2^-30 or not finite, an origin not finite or beyond 2^32), REGC_ENOMEM. */
REGC_API regc_status regc_set_state_windows(regc_handle *h, int n_bins, double e_bin, const double *e_lo);

/* Copy the per-state energy histograms hE [S][n_bins + 2] (layout above), the
 * window origins e_lo [S] and the bin width *e_bin as the library uses them
 * (host; any may be NULL).  Synchronous.  Errors: REGC_EINVAL (no windows). */
REGC_API regc_status regc_state_histograms(regc_handle *h, int64_t *hE, double *e_lo, double *e_bin);

/* Release the handle and its device memory.  NULL is accepted. */
REGC_API void regc_free(regc_handle *h);

/* ---------------------------------------------------------- extensions */

/* Replace the walkers' configurations: pos [S][nmax][3] (binary32, x in
 * [0, Lx), y in [0, Ly), z in [z_lo, z_hi]; entries beyond n[w] ignored),
 * n [S] in 0..nmax, and optionally state_of_walker [S] (a permutation of
 * 0..S-1; NULL keeps the current labels).  Host buffers.  A page-locked
 * position buffer (cudaHostAlloc, cudaHostRegister, or PyTorch's pinned
 * memory) is read in place by the repacking kernel (on a Grace-Blackwell node
 * over NVLink-C2C, and only the first n[w] entries of each walker); any other
 * is copied to the device once.  The positions are checked and repacked on
 * the device; energies are recomputed on the device.
 * Synchronous.  Errors: REGC_EINVAL -- N out of range or not a permutation
 * (nothing changed), or a coordinate outside the region or a pair inside the
 * hard-core guard radius (every walker is then left empty, N = 0). */
REGC_API regc_status regc_set_walkers(regc_handle *h, const float *pos, const int32_t *n,
                             const int32_t *state_of_walker);

/* As regc_set_walkers with species B's counts nb [S] (0 <= nb[w] <= n[w]:
 * particles [0, nb[w]) of walker w are B, the rest C).  nb NULL (and
 * regc_set_walkers) makes every particle B. */
REGC_API regc_status regc_set_walkers2(regc_handle *h, const float *pos, const int32_t *n, const int32_t *nb,
                                       const int32_t *state_of_walker);

/* As regc_get_walkers, with species B's counts nb [S] (second species only;
 * REGC_EINVAL otherwise). */
REGC_API regc_status regc_get_walkers2(regc_handle *h, float *pos, int32_t *n, int32_t *nb, double *energy,
                                       int32_t *state_of_walker);

/* A second mobile species, the "cluster" (not in the paper; the cluster-in-
 * gas workload): particles 0..n_cluster-1 of every walker are of potential
 * type cluster_type (1..n_types-1; pairs with the grand-canonical species use
 * eps/sigma[0][cluster_type], with each other [cluster_type][cluster_type],
 * with surface type t [cluster_type][t]) and move only by displacement;
 * insertion and removal act on type 0, whose count N_B = N - n_cluster enters
 * the acceptance ratios of Sec. II.A.1 and every histogram (hN, hNE, moments
 * and the MBAR reweighting are over N_B).  Displacement picks uniformly among
 * all N particles, removal among the N_B.  The exchange of Eq. Pacc is
 * unchanged (both walkers hold the cluster, so N_a - N_b = N_B,a - N_B,b).
 * n_cluster = 0 removes the species.  Every walker is emptied: regc_sweep
 * refuses (REGC_EINVAL) until regc_set_walkers supplies walkers with
 * n[w] >= n_cluster whose first n_cluster particles are the cluster atoms.
 * Speculative warps are not used with a cluster (one warp per walker).
 * Errors: REGC_EINVAL (n_cluster outside 0..nmax-1, bad type). */
REGC_API regc_status regc_set_cluster(regc_handle *h, int n_cluster, int cluster_type);

/* Read the walkers: pos [S][nmax][3] (entries beyond N undefined), n [S],
 * energy [S] (the running total E(R; N), all mobile-mobile and mobile-surface
 * pairs), state_of_walker [S].  Any may be NULL.  Synchronous. */
REGC_API regc_status regc_get_walkers(regc_handle *h, float *pos, int32_t *n, double *energy,
                             int32_t *state_of_walker);

/* Recompute every walker's energy from scratch and report the largest
 * |running total - recomputed| in *max_drift (0 when the bookkeeping is exact).
 * The running totals are not changed.  Returns REGC_ENUMERIC if an energy is
 * not finite.  Synchronous. */
REGC_API regc_status regc_check_energy(regc_handle *h, double *max_drift);

/* Checkpoint of everything a run needs to continue exactly: walker
 * configurations, N, running energies, state labels, the Philox counters of
 * the sweeps, exchanges and MD segments, histograms, moments and counters, and (if loaded)
 * the surrogate's parameters, optimiser state and the sweep mode.  Not saved:
 * the problem statement (restore into a handle created with the same one and
 * the same seed) and the surrogate's training rows.  buf NULL: *length
 * receives the size and nothing else happens; else buf (host, capacity bytes)
 * receives the checkpoint.  Synchronous.  Errors: REGC_EINVAL (capacity too
 * small). */
REGC_API regc_status regc_checkpoint(regc_handle *h, void *buf, size_t capacity, size_t *length);

/* Continue from a checkpoint: the handle's state becomes the saved one, so
 * the following sweeps and exchanges are exactly those of the run that was
 * saved.  Errors: REGC_EINVAL (not a checkpoint, corrupted (checksum), or of
 * a handle with other sizes, cluster or seed); nothing is changed then. */
REGC_API regc_status regc_restore(regc_handle *h, const void *buf, size_t length);

/* Counters (host buffers, any may be NULL): moves [S walkers][3 types][trials,
 * accepts]; exchanges [S lower states][4 directions (5 with a second species
 * on K > 1 chemical potentials)][attempts, accepts];
 * pairs [6]: pairs within rc of the committed moves, candidate pairs whose
 * distance was evaluated (including speculative evaluations that were
 * discarded), evaluation rounds, move evaluations, moves screened by the
 * surrogate (delayed acceptance), moves that passed the screen -- summed over
 * walkers since the last reset.  Synchronous. */
REGC_API regc_status regc_counters(regc_handle *h, int64_t *moves, int64_t *exchanges, int64_t *pairs);

/* Warps that evaluate a walker's moves in the plain sweep (1, 2 or 4; moves
 * evaluated speculatively per round and committed in order, so the chain does
 * not depend on it).  Chosen at creation from the replicas per SM (4 up to two
 * per SM, 2 up to four, else 1) unless the environment variable
 * REGC_WARPS_PER_WALKER sets it; halved while one walker's shared memory
 * would not fit.  Delayed acceptance and the cluster species use one. */
REGC_API regc_status regc_warps_per_walker(const regc_handle *h, int *warps);

/* MBAR reweighting of the handle's pooled histogram (Sec. II.B).  Solves the
 * self-consistent equations of Eq. normlizationconstant over the occupied
 * (N, E) bins with the reduced potential
 *   u_s(N, E) = beta_s (E - mu_s N) + 3 N ln Lambda_s          (Eq. grandpot
 * plus the thermal-wavelength factor of Eq. Ngrand, needed across temperatures),
 * then evaluates the nq query states (kT_q, mu_q): N_mean [nq], pN [nq][nmax+1]
 * (probability of each N, Eq. textbook with chi = [N = i]).  f_states [S]
 * receives the state free energies (f_0 = 0).  Any output may be NULL.
 * Iterates until max |delta f| < tol or max_iter iterations; *iters, if not
 * NULL, receives the count.  FP64 log-sum-exp on the device.  Synchronous. */
/* The ideal-gas reservoir of Sec. III.A: beta mu = beta mu0 + ln(beta p) with
 * mu0 = kT ln Lambda^3, Lambda = lambda0 / sqrt(kT), i.e.
 *   mu = kT (3 ln Lambda + ln(p / kT)),   p = (kT / Lambda^3) exp(mu / kT),
 * p in the problem's units of energy per volume (eV / A^3 for eV and A; 1 atm
 * = 6.3242e-7 eV / A^3).  n host values in, n out.  Errors: REGC_EINVAL (n < 0,
 * a null pointer with n > 0, kT, p or lambda0 not positive, mu not finite). */
REGC_API regc_status regc_mu_of_pressure(int n, const double *kT, const double *p, double lambda0, double *mu);
REGC_API regc_status regc_pressure_of_mu(int n, const double *kT, const double *mu, double lambda0, double *p);

REGC_API regc_status regc_reweight(regc_handle *h, int nq, const double *kT_q, const double *mu_q,
                          double tol, int max_iter, double *N_mean, double *pN,
                          double *f_states, int *iters);

/* MBAR (Sec. II.B) over a two-species run (regc_init_grid2): the pooled
 * histogram's bins are (N_B, N_C, E) and the reduced potential of a state
 * (kT, mu_B, mu_C) at a bin is
 *   u = E / kT + N_B (3 ln Lambda_B - mu_B / kT) + N_C (3 ln Lambda_C - mu_C / kT),
 * Lambda_X = lambda0_X / sqrt(kT), the two-species form of Eq. 4's weight.
 * The sampled states' free energies are solved as in regc_reweight (f_states
 * [S], f_0 = 0, state s = (l M + m) K + k), then reweighted to nq host
 * queries (kT_q, mu_q, mu2_q): NB_mean, NC_mean [nq] and the marginal
 * distributions pNB, pNC [nq][nmax+1] of the two counts.  Any output may be
 * NULL.  Errors: REGC_EINVAL (a one-species handle, nq < 0, a null query
 * array with nq > 0, kT_q not positive, a query not finite, tol <= 0,
 * max_iter < 1, nothing observed yet), REGC_ENOMEM, REGC_ECUDA.  Synchronous. */
REGC_API regc_status regc_reweight2(regc_handle *h, int nq, const double *kT_q, const double *mu_q,
                                    const double *mu2_q, double tol, int max_iter, double *NB_mean,
                                    double *NC_mean, double *pNB, double *pNC, double *f_states, int *iters);

/* Structural observables (Sec. III.A, "Structural properties"): the axial
 * distribution rho(z) of the adsorbed particles, counted in slabs parallel to
 * the surface, and the lateral radial distribution g_xy(r) of the particles of
 * an adsorbate layer z0 +- dz0, kept per sample and averaged per phase by MBAR
 * (Sec. II.B, Eq. avegr).  Only the grand-canonical species is counted.
 * Bin decisions are binary32, in this order: slab k = floor((z - z_lo) *
 * inv_dz); lateral distance r = sqrt(dx dx + dy dy) with dx, dy the nearest
 * image in x and y (e = q - p, or (q - L) - p when e > L/2, or q - (p - L)
 * when e < -L/2), bin k = floor(r * inv_dr); inv_dz = 1/dz and inv_dr = 1/dr
 * rounded to binary32 once. */
typedef struct {
    int     n_z;            /* slabs, 1..4096: slab k covers z_lo + [k, k+1) dz         */
    float   dz;             /* > 0 (0.12 A in Sec. III.A)                               */
    int     n_layers;       /* 0..4 adsorbate layers for g_xy                            */
    float   layer_lo[4];    /* a particle is in layer l if layer_lo[l] <= z < layer_hi[l] */
    float   layer_hi[4];
    int     n_r;            /* 1..4096 lateral distance bins: bin k covers [k, k+1) dr   */
    float   dr;             /* > 0, with n_r dr <= min(Lx / sqrt(1 + shear^2), Ly) / 2  */
    int64_t capacity;       /* samples the device keeps; each regc_structure_sample call
                               adds one per walker                                      */
} regc_structure_spec;

/* Allocate (or replace) the handle's sample store.  Samples are not part of
 * checkpoints.  Errors: REGC_EINVAL (sizes out of range, n_r dr beyond half the
 * box, a walker's counting tables beyond 227 KB of shared memory), REGC_ENOMEM. */
REGC_API regc_status regc_structure_init(regc_handle *h, const regc_structure_spec *spec);

/* Append one sample of every walker: its state, N_B, E, slab counts and, per
 * layer, its population and pair counts.  Asynchronous.  The paper takes one
 * every 100 REGC steps.  Errors: REGC_EINVAL (no store, or the store cannot
 * hold S more samples: nothing is appended). */
REGC_API regc_status regc_structure_sample(regc_handle *h);

/* Number of samples held. */
REGC_API regc_status regc_structure_count(regc_handle *h, int64_t *n_samples);

/* Drop every sample and the lowest-energy configurations (the store stays
 * allocated). */
REGC_API regc_status regc_structure_reset(regc_handle *h);

/* Copy samples first .. first + count - 1 to host buffers (any may be NULL):
 * state [count], n [count] (N_B), energy [count], rho [count][n_z] slab counts,
 * pairs [count][n_layers][n_r] pair counts (unordered pairs), pop
 * [count][n_layers] layer populations.  Synchronous. */
REGC_API regc_status regc_structure_get(regc_handle *h, int64_t first, int64_t count, int32_t *state,
                                        int32_t *n, double *energy, uint16_t *rho, uint32_t *pairs,
                                        int32_t *pop);

/* MBAR averages per phase N_B = n_lo .. n_hi at nq query states (kT_q, mu_q),
 * over the samples held (Eq. avegr).  Each distinct (N_B, E) of the samples is
 * a bin with its count (samples with bit-identical energies, such as empty
 * walkers, share one): the MBAR equations (Eq. normlizationconstant, with the reduced
 * potential of regc_reweight) are solved over the samples for the free
 * energies of the sampled states (f_states [S], f_0 = 0), and sample n
 * weighs W_n(q) = exp(-u_q(n) - D_n + f_q) at query q (the weights of all
 * samples sum to 1).  Outputs (host, any may be NULL), phases P = n_hi - n_lo + 1:
 *   p    [nq][P]                    probability of each phase, sum of W_n over it
 *   rho  [nq][P][n_z]               sum_n W_n c_nk / (p A dz): number density
 *                                   within the phase (A = Lx Ly)
 *   gxy  [nq][P][n_layers][n_r]     sum_n W_n g_n(r_k) / p with the sample's
 *                                   g_n(r_k) = 2 A P_nk / (M_n (M_n - 1) pi
 *                                   ((k+1)^2 - k^2) dr^2) (0 when M_n < 2)
 * Eq. avegr as printed is the joint average, p times these; zero where p = 0.
 * FP64 on the device, except the weighted sums of the counts: over chunks of
 * at most 256 samples of a phase, with the chunk's largest weight factored
 * out, they are binary32 (relative error below 2e-5).  Synchronous.  Errors:
 * REGC_EINVAL (no samples, bad phase range, nq < 1). */
REGC_API regc_status regc_structure_reweight(regc_handle *h, int nq, const double *kT_q, const double *mu_q,
                                             int n_lo, int n_hi, double tol, int max_iter, double *p,
                                             double *rho, double *gxy, double *f_states, int *iters);

/* aiAT@REGC (Sec. III.A.1, Eq. aiTherm) over the samples of the structure
 * store (since its last reset): per composition N_B the lowest sampled energy
 * e_min [nmax+1] (NaN where N_B was never sampled; samples with |E| beyond
 * 65536 energy units are not tracked), and at nq chemical potentials mu_q the
 * formation free energy with every F approximated by that energy and F of
 * the pristine slab taken as 0 (the frozen slab's own energy is not part of
 * E): dG [nq][nmax+1] = e_min[n] - n mu_q (+inf where unsampled), and the
 * stable composition phase [nq] (lowest dG; ties: smaller n).  The
 * temperature enters only through mu(T, p).  Any output may be NULL.
 * Synchronous.  Errors: REGC_EINVAL (no store, mu not finite). */
REGC_API regc_status regc_aiat(regc_handle *h, int nq, const double *mu_q, double *e_min, double *dG,
                               int32_t *phase);

/* The configuration of a lowest-energy sample with N_B = n_b (among equal
 * energies, the one of the lowest walker index): xyz [n][3] (host, room for
 * nmax rows), *n its particle count (cluster atoms included).  Synchronous.
 * Errors: REGC_EINVAL (no store, n_b out of range or never sampled). */
REGC_API regc_status regc_aiat_config(regc_handle *h, int n_b, float *xyz, int32_t *n);

/* Device time of the last regc_structure_reweight (milliseconds, any pointer
 * may be NULL): the MBAR solve and query over the samples, the sample weights,
 * and the accumulation per phase, with the accumulation's algorithmic bytes
 * (every row of a phase in range read once per pass of 8 query states, with
 * its population and index, plus the weights and the sums written). */
REGC_API regc_status regc_structure_timing(regc_handle *h, double *ms_mbar, double *ms_weights,
                                           double *ms_accumulate, double *bytes_accumulate);

/* Stand-alone MBAR solve over caller-supplied pooled bins (host buffers):
 * S states (kT [S], mu [S], omega [S] observations), B bins (N_b [B], E_b [B],
 * H_b [B] > 0 counts).  Outputs f [S] (f_0 = 0) and D [B], the log denominators
 * D_b = ln sum_k omega_k exp(f_k - u_k(b)).  Runs on cuda_stream.
 * Device memory: besides O(S + B) buffers, when every omega_k > 0 the
 * iterations use the kept entries of the kernel matrix (those within e^-70
 * of the largest of their bin, stored by bin and by state: 24 bytes each),
 * allocated on the stream for the duration of the call when they fit in half
 * the free device memory (otherwise they run without it; the result is the
 * same fixed point).  regc_reweight, regc_reweight2 and
 * regc_structure_reweight solve the same way; regc_mbar_last_info reports
 * what the last solve did. */
REGC_API regc_status regc_mbar_solve(int S, const double *kT, const double *mu, double lambda0,
                            const double *omega, int B, const int32_t *N_b,
                            const double *E_b, const double *H_b, double tol,
                            int max_iter, double *f, double *D, int *iters,
                            void *cuda_stream);

/* What the calling thread's last MBAR solve (regc_mbar_solve, regc_reweight,
 * regc_reweight2, regc_structure_reweight) did: path 1 when it iterated on the
 * sparse kernel matrix, 0 on log-sum-exps only; its iterations (maps of the
 * self-consistent equations), matrix builds, maps taken on log-sum-exps (no
 * matrix, or a state without a kept entry far from the fixed point), the kept
 * entries of the last build, its S and B, the device milliseconds of the
 * matrix builds and of the maps on the matrix (CUDA events on the solve's
 * stream), and the number of those maps.  regc_reweight and regc_reweight2
 * start a problem of at least 65536 bins from the solution of the same
 * problem with 16 energy bins merged into one (solved to 1e-6; same fixed
 * point, fewer matrix builds): coarse_iterations, coarse_B, coarse_builds
 * and coarse_maps describe that solve (zero without one) and its device time
 * is included in ms_build and ms_maps.  All zero before the first solve.
 * Errors: REGC_EINVAL (out NULL). */
typedef struct {
    int32_t path;
    int32_t iterations;
    int32_t builds;
    int32_t lse_maps;
    int64_t nnz;
    int64_t S;
    int64_t B;
    double ms_build;
    double ms_maps;
    int32_t sparse_maps;
    int32_t coarse_iterations;
    int64_t coarse_B;
    int32_t coarse_builds;
    int32_t coarse_maps;
} regc_mbar_info;
REGC_API regc_status regc_mbar_last_info(regc_mbar_info *out);

/* Stand-alone MBAR query: with D [B] from regc_mbar_solve, reweight to Q
 * states; outputs N_mean [Q], pN [Q][nmax+1], f_q [Q] (any may be NULL). */
REGC_API regc_status regc_mbar_query(int Q, const double *kT_q, const double *mu_q, double lambda0,
                            int B, const int32_t *N_b, const double *E_b, const double *H_b,
                            const double *D, int nmax, double *N_mean, double *pN,
                            double *f_q, void *cuda_stream);

/* Largest problem regc_mbar_solve_static accepts. */
#define REGC_MBAR_STATIC_MAX_STATES 4096
#define REGC_MBAR_STATIC_MAX_BINS 262144

/* MBAR solve that allocates no device memory.  The paper has no counterpart:
 * this entry point exists for callers that cannot let a library allocate
 * device memory -- for example an application whose framework owns all device
 * memory through its own pooled allocator, or a loop that cannot afford the
 * device-wide synchronisation cudaMalloc and cudaFree may cause.
 * Arguments, outputs and results are those of regc_mbar_solve (host buffers).
 * The staged inputs and the work arrays live in one fixed scratch area of
 * about 12.3 MiB compiled into the library, which every GPU that loads the
 * library keeps reserved until the process exits.
 *   - S > REGC_MBAR_STATIC_MAX_STATES or B > REGC_MBAR_STATIC_MAX_BINS:
 *     REGC_EINVAL, nothing is run.
 *   - The first call on a device, with that device current, looks up the
 *     device address of the scratch area; make that first call before any
 *     stream capture.
 *   - Like regc_mbar_solve, the call waits for its stream after every map of
 *     the iteration (the Anderson step runs on the host) and returns when the
 *     results are in the host buffers.
 *   - Every call on a device shares that one scratch area, and it keeps the
 *     last call's contents (the solver clears what it needs cleared).  Calls
 *     that overlap on the GPU -- on different streams or from different host
 *     threads -- race on it: serialise them. */
REGC_API regc_status regc_mbar_solve_static(int S, const double *kT, const double *mu, double lambda0,
                                            const double *omega, int B, const int32_t *N_b,
                                            const double *E_b, const double *H_b, double tol,
                                            int max_iter, double *f, double *D, int *iters,
                                            void *cuda_stream);

/* ---------------------------------------------------- learned surrogate
 *
 * The paper has no surrogate.  These entry points add a delayed-acceptance
 * (Christen & Fox 2005) form of the sweep: every evaluated move is first
 * screened with the surrogate energy change dE~ (stage 1: accept iff
 * ln u1 < the log acceptance ratio of Sec. II.A.1 / II.A.3 with dE~ in place
 * of dE, u1 from the fourth word of the move's second Philox block); only a
 * move that passes gets its exact energy change dE and is accepted iff
 * ln u2 < -beta (dE - dE~) (stage 2, u2 the plain acceptance uniform).  dE~ is
 * e~(new) - e~(old) (insertion: e~(new); removal: -e~(old)), antisymmetric
 * under the reverse move, so the chain keeps the distribution of Eq. Ngrand
 * whatever the network's weights.
 *
 * e~(r) is a 16 -> 64 -> 64 -> 1 network with SiLU hidden layers on 16
 * Gaussian radial features of the neighbours within rc:
 *   G_k = sum_j eps_0j exp(-eta (r_j - c_k)^2) (cos(pi r_j / rc) + 1) / 2,
 *   c_k = 0.8 + 1.7 k / 15 (k = 0..15), eta = 1 / (2 (1.7 / 15)^2).
 * Parameters: REGC_SURROGATE_PARAMS binary32 values, row-major
 *   W1 [16][64], b1 [64], W2 [64][64], b2 [64], W3 [64], b3,
 * z1 = G W1 + b1, h1 = silu(z1), z2 = h1 W2 + b2, e~ = silu(z2) W3 + b3.
 * The sweep uses an inference copy with the weights rounded to bfloat16
 * (nearest, ties to even) and the biases in binary32; features and
 * activations are binary32. */
#define REGC_SURROGATE_PARAMS 5313

/* Load the surrogate's binary32 parameters theta [REGC_SURROGATE_PARAMS]
 * (host) as the training master copy, refresh the inference copy and reset
 * the optimiser's moments and step count.  Allocates the surrogate's device
 * buffers on first use.  Errors: REGC_EINVAL (NULL or non-finite value). */
REGC_API regc_status regc_surrogate_set(regc_handle *h, const float *theta);

/* Seeded initial parameters on the device: every weight normal with standard
 * deviation scale / sqrt(fan-in) (Box-Muller on Philox stream 7 keyed by
 * seed), every bias zero; as regc_surrogate_set otherwise. */
REGC_API regc_status regc_surrogate_init(regc_handle *h, uint64_t seed, float scale);

/* Copy the master parameters to theta [REGC_SURROGATE_PARAMS] (host).
 * Errors: REGC_EINVAL (no surrogate loaded).  Synchronous. */
REGC_API regc_status regc_surrogate_get(regc_handle *h, float *theta);

/* Sweep mode: 0 plain Metropolis (the default), 1 delayed acceptance with the
 * loaded surrogate (one warp per walker).  Errors: REGC_EINVAL (mode 1 with no
 * surrogate loaded, other modes). */
REGC_API regc_status regc_set_mode(regc_handle *h, int mode);

/* Surrogate energy e~ of a test particle at each of n_query positions
 * xyz [n_query][3] (host, inside the region) against every particle of
 * walker `walker` and every surface atom, nearest periodic image;
 * e_out [n_query] and, if not NULL, features [n_query][16] (host).
 * Synchronous. */
REGC_API regc_status regc_surrogate_eval(regc_handle *h, int walker, int n_query, const float *xyz,
                                         float *e_out, float *features);

/* Append training rows to the handle's data set, a ring of `capacity` rows
 * allocated on the first call (later calls pass the same capacity, or 0).
 * Each walker gives `particles` rows for particles spread evenly over its
 * index range (features of the particle against all the others and the
 * surface; target its exact interaction energy) and `probes` rows for
 * uniform random points of the region (Philox stream 5; target the energy a
 * test particle there would have); a walker with N = 0 gives probes only.
 * Targets are clipped from above at e_clip.  *n_rows (may be NULL) receives
 * the number of rows held.  Asynchronous apart from the count. */
REGC_API regc_status regc_surrogate_harvest(regc_handle *h, int particles, int probes, float e_clip,
                                            int capacity, int64_t *n_rows);

/* Replace the data set by n_rows caller rows: X [n_rows][16] features and
 * y [n_rows] targets (host, finite), stored as rows 0 .. n_rows - 1 of the
 * ring (allocated with `capacity` rows on first use, as by
 * regc_surrogate_harvest; later calls pass the same capacity, or 0); later
 * harvests continue after them.  Lets a caller train on rows of its own.
 * Synchronous.  Errors: REGC_EINVAL (n_rows beyond the capacity, a non-finite
 * value, a NULL buffer with n_rows > 0). */
REGC_API regc_status regc_surrogate_set_dataset(regc_handle *h, int64_t n_rows, const float *X, const float *y,
                                                int capacity);

/* Copy the data set (X [n][16], y [n], n = rows held, in ring order) to host
 * buffers of at least `max_rows` rows; *n_rows receives n.  Synchronous. */
REGC_API regc_status regc_surrogate_dataset(regc_handle *h, int64_t max_rows, float *X, float *y,
                                            int64_t *n_rows);

/* `steps` Adam steps (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on
 * the mean squared error of mini-batches of `batch` rows drawn uniformly from
 * the data set, on the device; then refresh the inference copy.  Adam step
 * number a (counted over the handle's life, from 1) takes row
 * (P0 * rows held) >> 32 for its i-th row, P = Philox((i, a, 0, 6)).  The
 * gradient is regc_surrogate_gradient_bf16's (tensor cores, BF16 operands,
 * FP32 accumulation); masters and optimiser moments are binary32.  loss [steps] (host, may be NULL) receives each step's mini-batch
 * loss before its update.  Errors: REGC_EINVAL (empty data set, no
 * surrogate, batch < 1).  Synchronous. */
REGC_API regc_status regc_surrogate_train(regc_handle *h, int steps, int batch, float lr, float *loss);

/* Stateless: the mean squared error of the network with parameters theta
 * [REGC_SURROGATE_PARAMS] on n rows X [n][16], y [n] (host) and its gradient
 * grad [REGC_SURROGATE_PARAMS] (host), everything in binary32 on the FP32
 * pipe.  Runs on cuda_stream.  Synchronous. */
REGC_API regc_status regc_surrogate_gradient(int n, const float *theta, const float *X, const float *y,
                                             float *loss, float *grad, void *cuda_stream);

/* As regc_surrogate_gradient, computed as regc_surrogate_train computes it:
 * every matrix product of the forward and backward passes on tensor cores
 * with bfloat16 operands (nearest, ties to even) and FP32 accumulation --
 *   z1 = bf(X) bf(W1) + b1, h1 = silu(z1), z2 = bf(h1) bf(W2) + b2,
 *   h2 = silu(z2), e = h2 . W3 + b3,
 *   dz2 = g W3 silu'(z2), dW2 = bf(h1)^T bf(dz2),
 *   dz1 = (bf(dz2) bf(W2)^T) silu'(z1), dW1 = bf(X)^T bf(dz1),
 * with g = 2 (e - y) / n and the rest (e, dW3, the bias gradients and the
 * element-wise products) in binary32. */
REGC_API regc_status regc_surrogate_gradient_bf16(int n, const float *theta, const float *X, const float *y,
                                                  float *loss, float *grad, void *cuda_stream);

/* ---------------------------------------------------------------- batch
 *
 * Many systems of uneven size stepped together (the paper runs one system at
 * a time; this is the GPU's way of filling itself with small ones).  A batch
 * groups existing handles -- each its own surface, box, (T, mu) grid and
 * Nmax -- without copying their state.  One batch step is, for every member,
 * exactly what regc_sweep(h, sweeps_per_step) followed by regc_exchange(h)
 * does, with the same Philox streams, so the results are bit-identical to
 * stepping the members one by one; only the schedule differs:
 *   - walkers are grouped into size classes by Nmax; each class runs as one
 *     persistent kernel whose warps take (system, walker) items from a queue,
 *     largest systems first, each warp one walker with its own shared memory;
 *   - the classes run as parallel branches of one captured CUDA graph,
 *     followed by one exchange attempt on every member's grid; the members'
 *     Philox counters advance on the device, so steps replay the graph;
 *   - the shape of each class's kernel (walkers per CTA, number of CTAs) is
 *     chosen by regc_batch_autotune from timed steps.
 * Members must be in plain mode (regc_set_mode 0), must outlive the batch,
 * and must not be used concurrently with it: call regc_batch_sync before
 * reading a member, and synchronise a member's own stream before running the
 * batch after stepping that member on its own (its counters are picked up). */
typedef struct regc_batch regc_batch;

/* Create a batch over handles [count] (distinct, plain mode), stepping
 * sweeps_per_step sweeps + one exchange attempt per step, on cuda_stream (a
 * cudaStream_t; NULL: a stream the batch creates, which orders with work on
 * the legacy default stream -- the legacy stream itself cannot be captured).
 * Errors: REGC_EINVAL (bad arguments, a member in delayed-acceptance mode, a
 * walker that does not fit one CTA's shared memory), REGC_ENOMEM, REGC_ECUDA,
 * or a member's sticky status.  On error *out is NULL. */
REGC_API regc_status regc_batch_create(regc_handle *const *handles, int count, int sweeps_per_step,
                                       void *cuda_stream, regc_batch **out);

/* Run n_steps steps (graph replays; the graph is captured on first use).
 * Asynchronous on the batch's stream. */
REGC_API regc_status regc_batch_run(regc_batch *b, int n_steps);

/* Time `rounds` x (number of candidate shapes) real batch steps -- each
 * class's kernel with warps per walker in 1, 2, 4 (more than one -- the
 * speculative walker -- for plain one-species classes only) times walkers per
 * CTA in 1, 2, 4, ... (CTAs of 32 ... 512 threads, while the shared memory
 * fits), CTAs = SMs x resident CTAs per SM (at most one per walker group) --
 * and keep each class's fastest shape.  The steps count as sampling steps
 * (the chains advance); every shape gives the same chains.  Synchronous. */
REGC_API regc_status regc_batch_autotune(regc_batch *b, int rounds);

/* The current plan: *n_classes size classes; for the first max_classes of
 * them nmax, walkers, walkers per CTA, warps per walker, CTAs and the last
 * measured kernel time in ms (-1 before tuning).  Output arrays may be NULL. */
REGC_API regc_status regc_batch_plan(const regc_batch *b, int max_classes, int *n_classes, int32_t *nmax,
                                     int32_t *walkers, int32_t *walkers_per_cta, int32_t *warps_per_walker,
                                     int32_t *ctas, double *ms);

/* Wait for the batch's work and fold every member's device error word into
 * its sticky status; returns the first error. */
REGC_API regc_status regc_batch_sync(regc_batch *b);

/* Release the batch (not its members).  NULL is accepted. */
REGC_API void regc_batch_free(regc_batch *b);

/* Human-readable name of a status. */
REGC_API const char *regc_status_string(regc_status s);

#ifdef __cplusplus
}
#endif
#endif /* REGC_H */
