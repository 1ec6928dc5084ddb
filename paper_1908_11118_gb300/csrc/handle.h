// handle.h -- the state behind a regc_handle (internal to the library).
#pragma once

#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "launch.h"

// An NVTX range over a library call: visible on the timeline of an Nsight
// tool attached to the process, nearly free otherwise.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

using regc::ExchangeParams;
using regc::SurrogateStore;
using regc::SweepParams;

// Samples of the structural observables (structure.cu): one device block
// holding state [cap], nb [cap], energy [cap], pop [cap][4], rho
// [cap][rho_stride] (n_z used), pairs [cap][pair_stride] (n_layers n_r used).
struct StructureStore {
    int n_z = 0, n_layers = 0, n_r = 0;
    int rho_stride = 0, pair_stride = 0;      // row strides: n_z and n_layers n_r rounded up to 16 bytes
    float dz = 0, dr = 0, inv_dz = 0, inv_dr = 0;
    float layer_lo[4] = {}, layer_hi[4] = {};
    long long cap = 0, count = 0;
    size_t smem = 0;
    void* block = nullptr;
    int32_t* state = nullptr;
    int32_t* nb = nullptr;
    double* energy = nullptr;
    int32_t* pop = nullptr;
    uint16_t* rho = nullptr;
    uint32_t* pairs = nullptr;
    // aiAT: per N_B the lowest sampled energy packed with the walker index
    // (E in 2^-30 units << 16 | walker), and that sample's configuration
    long long* best_key = nullptr;            // [nmax + 1]
    float* best_xyz = nullptr;                // [nmax + 1][nmax][3]
    int32_t* best_n = nullptr;                // [nmax + 1] particles of the configuration
    // the last reweighting: device milliseconds of the MBAR solve and query,
    // the weights and the accumulation, and the accumulation's algorithmic bytes
    double last_ms[3] = {0, 0, 0};
    double last_bytes = 0;
};

struct regc_handle {
    // a shard (regc_set_shard) steps only walkers [P.w_begin, P.w_end)
    bool sharded() const { return P.w_begin != 0 || P.w_end != S; }
    cudaStream_t stream = nullptr;
    int L = 0, M = 0, S = 0, nmax = 0, mps = 0, n_e_bins = 0;
    double lambda0 = 1.0, e_lo = 0.0, e_bin = 1.0;
    float Lx = 0, Ly = 0, Lz = 0, z_lo = 0, z_hi = 0;
    int periodic_z = 0;
    std::vector<double> kT_state, mu_state;   // per state
    double* d_kT_state = nullptr;
    double* d_mu_state = nullptr;
    SweepParams P{};
    ExchangeParams X{};
    uint32_t t = 0, e = 0;
    regc_status sticky = REGC_OK;
    std::vector<void*> allocs;
    int* d_error = nullptr;
    long long* d_fix = nullptr;               // scratch [S] for energy recomputes
    float* d_xyz = nullptr;                   // staging [S][nmax][3] for walker I/O
    void* h_stage = nullptr;                  // pinned host staging: error word, [S] energies or labels
    size_t smem_per_walker = 0;
    // learned surrogate (delayed acceptance)
    bool has_sur = false;
    float* d_theta = nullptr;                 // [5313] binary32 master parameters
    float* d_adam_m = nullptr;
    float* d_adam_v = nullptr;
    int adam_t = 0;
    SurrogateStore sur{};
    float* d_X = nullptr;                     // data set ring [cap][16]
    float* d_y = nullptr;                     // [cap]
    int ds_cap = 0, ds_count = 0, ds_next = 0;
    uint32_t harvest_round = 0;
    // the potential as given (for the cluster species' pair tables)
    int n_types = 0;
    float eps[4][4] = {}, sigma[4][4] = {};
    double hard_core_T = 0.0;
    bool need_walkers = false;                // set_cluster emptied the walkers
    uint32_t md_seg = 0;                      // MD segments run (Philox counter of the MD streams)
    StructureStore stc;                       // structural observables (empty until regc_structure_init)
    void* hE_block = nullptr;                 // per-state energy histograms [S][bins + 2] and window origins [S]
    // a second grand-canonical species (P.gc2): a third grid axis of K
    // chemical potentials; the pooled histogram then has (nmax+1)^2 rows
    int K = 1;
    int n_dir = 4;                            // exchange directions (5 with K > 1)
    long long hist_rows = 0;                  // rows of the pooled (N, E) histogram
    std::vector<double> mu2_state;            // per state: mu of species C (two species)
    double* d_mu2_state = nullptr;
    double lambda0_2 = 1.0;                   // Lambda_C at kT = 1
    bool expire_next = false;                 // regc_test_expire_waits: the next regc_sweep
};

// Synchronise the handle's stream and fold its device error word into the
// sticky status.
regc_status handle_sync_check(regc_handle* h);

// Record a CUDA error as the handle's sticky status; returns the status.
regc_status handle_cuda_fail(regc_handle* h, cudaError_t e);
