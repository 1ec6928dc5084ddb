// batch.cu -- many REGC systems of uneven size stepped together (host side).
//
// A batch groups existing handles, each its own system (surface, box, grid,
// Nmax).  Their walkers are sorted into size classes by Nmax; each class runs
// as one persistent kernel whose warps take (system, walker) items from a
// queue, largest systems first (csrc/sweep.cu: batch_sweep_kernel).  The
// classes run concurrently as parallel branches of one CUDA graph, followed by
// one exchange attempt on every system's grid; the Philox counters advance on
// the device, so the captured step replays without host work.  The shape of
// each class's kernel (walkers per CTA, CTAs) is picked by an autotuner that
// times real steps.
#include <string.h>

#include <algorithm>
#include <map>
#include <tuple>
#include <new>
#include <vector>

#include "handle.h"

using namespace regc;

namespace {

constexpr size_t kMaxSmem = 232448;  // 227 KB per block on sm_103a

struct Bucket {
    int nmax = 0;
    bool da = false;                // its systems sample with delayed acceptance
    bool cl = false;                // its systems carry a cluster species
    int region = 0;                 // dynamic shared memory per walker (bytes) at k warps per walker
    int k = 1;                      // warps per walker
    std::vector<int2> items;        // (system, walker), largest systems first
    std::vector<int> members;       // the members in the class
    int2* d_items = nullptr;
    int wpc = 1, grid = 1;          // walkers per CTA, CTAs
    double ms = -1.0;               // last measured kernel time
    struct Shape {
        int k, wpc, region;
    };
    std::vector<Shape> cand;        // feasible (warps per walker, walkers per CTA) choices
};

}  // namespace

struct regc_batch {
    cudaStream_t stream = nullptr;
    std::vector<regc_handle*> members;
    std::vector<char> member_da;    // a member's sampling mode at creation (1: delayed acceptance)
    int sweeps_per_step = 1;
    int sms = 1;
    SweepParams* d_sys = nullptr;
    ExchangeParams* d_xp = nullptr;
    uint32_t* d_ectr = nullptr;
    int* d_counters = nullptr;
    std::vector<uint32_t> t_mirror, e_mirror;   // counters as held on the device
    std::vector<SweepParams> sys_host;          // the parameters as uploaded (t0 as at the upload)
    std::vector<Bucket> buckets;
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool own_stream = false;
    regc_status sticky = REGC_OK;
};

namespace {

regc_status fail(regc_batch* b, cudaError_t e) {
    if (e == cudaSuccess) return REGC_OK;
    const regc_status st = e == cudaErrorMemoryAllocation ? REGC_ENOMEM : REGC_ECUDA;
    if (b->sticky == REGC_OK) b->sticky = st;
    return st;
}

void drop_graph(regc_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

// A member's sweep parameters as the batch runs them.
SweepParams batch_params(const regc_batch* b, const regc_handle* h) {
    SweepParams P = h->P;
    P.t0 = h->t;
    P.n_sweeps = b->sweeps_per_step;
    P.trace = nullptr;
    P.expire_waits = 0;
    return P;
}

// Upload every member's sweep and exchange parameters with its current
// Philox counters (the members may have been stepped on their own since).
cudaError_t upload_descriptors(regc_batch* b) {
    const size_t n = b->members.size();
    std::vector<SweepParams> sys(n);
    std::vector<ExchangeParams> xp(n);
    for (size_t m = 0; m < n; ++m) {
        regc_handle* h = b->members[m];
        sys[m] = batch_params(b, h);
        xp[m] = h->X;
        b->t_mirror[m] = h->t;
        b->e_mirror[m] = h->e;
    }
    b->sys_host = sys;
    cudaError_t e = cudaMemcpyAsync(b->d_sys, sys.data(), n * sizeof(SweepParams), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_xp, xp.data(), n * sizeof(ExchangeParams), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_ectr, b->e_mirror.data(), n * sizeof(uint32_t), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    return e;
}

// The members' host counters after `steps` more steps.
void advance_counters(regc_batch* b, int steps) {
    for (size_t m = 0; m < b->members.size(); ++m) {
        regc_handle* h = b->members[m];
        h->t += (uint32_t)(b->sweeps_per_step * steps);
        h->e += (uint32_t)steps;
        b->t_mirror[m] = h->t;
        b->e_mirror[m] = h->e;
    }
}

// One step on b->stream: the size classes as parallel branches (or one after
// another, timed, when ms_out is given), then every grid's exchange.
cudaError_t record_step(regc_batch* b, std::vector<double>* ms_out) {
    const int nb = (int)b->buckets.size();
    cudaError_t e = cudaMemsetAsync(b->d_counters, 0, nb * sizeof(int), b->stream);
    if (ms_out) {
        ms_out->assign(nb, 0.0);
        std::vector<cudaEvent_t> ev(nb + 1, nullptr);
        for (auto& x : ev)
            if (e == cudaSuccess) e = cudaEventCreate(&x);
        if (e == cudaSuccess) e = cudaEventRecord(ev[0], b->stream);
        for (int k = 0; k < nb && e == cudaSuccess; ++k) {
            const Bucket& q = b->buckets[k];
            e = launch_batch_sweep(b->d_sys, q.d_items, (int)q.items.size(), b->d_counters + k, q.wpc, q.k,
                                   q.grid, q.region, q.da, q.cl, b->stream);
            if (e == cudaSuccess) e = cudaEventRecord(ev[k + 1], b->stream);
        }
        if (e == cudaSuccess)
            e = launch_batch_exchange(b->d_xp, b->d_ectr, b->d_sys, (int)b->members.size(), b->sweeps_per_step,
                                      b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        for (int k = 0; k < nb && e == cudaSuccess; ++k) {
            float t = 0.f;
            e = cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
            (*ms_out)[k] = t;
        }
        for (auto& x : ev)
            if (x) cudaEventDestroy(x);
        return e;
    }
    if (e == cudaSuccess) e = cudaEventRecord(b->fork, b->stream);
    for (int k = 0; k < nb && e == cudaSuccess; ++k) {
        const Bucket& q = b->buckets[k];
        cudaStream_t s = k == 0 ? b->stream : b->side[k];
        if (k > 0) e = cudaStreamWaitEvent(s, b->fork, 0);
        if (e == cudaSuccess)
            e = launch_batch_sweep(b->d_sys, q.d_items, (int)q.items.size(), b->d_counters + k, q.wpc, q.k,
                                   q.grid, q.region, q.da, q.cl, s);
        if (e == cudaSuccess && k > 0) e = cudaEventRecord(b->join[k], s);
    }
    for (int k = 1; k < nb && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->stream, b->join[k], 0);
    if (e == cudaSuccess)
        e = launch_batch_exchange(b->d_xp, b->d_ectr, b->d_sys, (int)b->members.size(), b->sweeps_per_step,
                                  b->stream);
    return e;
}

cudaError_t build_graph(regc_batch* b) {
    drop_graph(b);
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    const cudaError_t er = record_step(b, nullptr);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->stream, &g);
    if (er != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return er;
    }
    if (e != cudaSuccess) return e;
    b->graph = g;
    return cudaGraphInstantiate(&b->exec, g, 0);
}

// Members must keep the sampling mode, Nmax and species they had at
// creation and have no errors; re-upload the descriptors if any member was
// stepped on its own since the last batch step or its parameters changed
// (per-state energy windows set, say; a retrained network is read in place).
regc_status check_members(regc_batch* b) {
    bool stale = false;
    for (size_t m = 0; m < b->members.size(); ++m) {
        regc_handle* h = b->members[m];
        if (h->sticky != REGC_OK) return h->sticky;
        if ((h->P.delayed != 0) != (b->member_da[m] != 0) || h->need_walkers || h->sharded()) return REGC_EINVAL;
        if (h->nmax != b->sys_host[m].nmax || (h->P.n_cluster > 0) != (b->sys_host[m].n_cluster > 0) ||
            h->P.gc2)
            return REGC_EINVAL;
        if (h->t != b->t_mirror[m] || h->e != b->e_mirror[m]) stale = true;
        SweepParams now = batch_params(b, h);
        now.t0 = b->sys_host[m].t0;   // the device advances t0 itself
        if (memcmp(&now, &b->sys_host[m], sizeof(SweepParams)) != 0) stale = true;
    }
    if (stale) return fail(b, upload_descriptors(b));
    return REGC_OK;
}

}  // namespace

extern "C" {

void regc_batch_free(regc_batch* b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    drop_graph(b);
    for (auto& q : b->buckets)
        if (q.d_items) cudaFree(q.d_items);
    for (auto s : b->side)
        if (s) cudaStreamDestroy(s);
    for (auto ev : b->join)
        if (ev) cudaEventDestroy(ev);
    if (b->fork) cudaEventDestroy(b->fork);
    cudaFree(b->d_sys);
    cudaFree(b->d_xp);
    cudaFree(b->d_ectr);
    cudaFree(b->d_counters);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
}

regc_status regc_batch_create(regc_handle* const* handles, int count, int sweeps_per_step, void* cuda_stream,
                              regc_batch** out) {
    if (!out) return REGC_EINVAL;
    *out = nullptr;
    if (!handles || count < 1 || sweeps_per_step < 1) return REGC_EINVAL;
    for (int i = 0; i < count; ++i) {
        if (!handles[i] || handles[i]->need_walkers || handles[i]->P.gc2 || handles[i]->sharded()) return REGC_EINVAL;
        if (handles[i]->P.delayed && !handles[i]->has_sur) return REGC_EINVAL;
        if (handles[i]->sticky != REGC_OK) return handles[i]->sticky;
        for (int j = 0; j < i; ++j)
            if (handles[j] == handles[i]) return REGC_EINVAL;
    }
    regc_batch* b = new (std::nothrow) regc_batch;
    if (!b) return REGC_ENOMEM;
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    b->members.assign(handles, handles + count);
    for (int i = 0; i < count; ++i) b->member_da.push_back(handles[i]->P.delayed ? 1 : 0);
    cudaError_t e = cudaSuccess;
    if (!b->stream) {
        // the legacy default stream cannot be captured: use a stream of our own
        // that still orders with default-stream work
        e = cudaStreamCreate(&b->stream);
        b->own_stream = e == cudaSuccess;
    }
    b->sweeps_per_step = sweeps_per_step;
    b->t_mirror.assign(count, 0);
    b->e_mirror.assign(count, 0);
    int dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    // size classes by (Nmax, sampling mode, cluster); within a class the largest systems first
    std::map<std::tuple<int, int, int>, std::vector<int>> by_nmax;
    for (int m = 0; m < count; ++m)
        by_nmax[{handles[m]->nmax, b->member_da[m], handles[m]->P.n_cluster > 0 ? 1 : 0}].push_back(m);
    for (auto it = by_nmax.rbegin(); it != by_nmax.rend(); ++it) {
        Bucket q;
        q.nmax = std::get<0>(it->first);
        q.da = std::get<1>(it->first) != 0;
        q.cl = std::get<2>(it->first) != 0;
        std::vector<int> ms = it->second;
        q.members = ms;
        std::stable_sort(ms.begin(), ms.end(), [&](int a, int c) {
            return handles[a]->P.cg.ncell * handles[a]->P.cg.cap > handles[c]->P.cg.ncell * handles[c]->P.cg.cap;
        });
        for (int m : ms)
            for (int w = 0; w < handles[m]->S; ++w) q.items.push_back(make_int2(m, w));
        b->buckets.push_back(q);
    }
    if (e == cudaSuccess) e = batch_prepare((int)kMaxSmem);
    // feasible shapes (warps per walker 1, 2, 4 -- more than one only for
    // plain one-species classes -- times walkers per CTA, CTAs of at most 16
    // warps), and the default: one warp per walker, the most resident walkers
    // per SM
    for (auto& q : b->buckets) {
        int best = 0;
        const size_t stat = batch_static_smem(q.da);
        for (int k = 1; k <= 4 && e == cudaSuccess; k *= 2) {
            if (k > 1 && (q.da || q.cl)) break;
            size_t region = 0;
            for (int m : q.members) {
                const regc_handle* h = handles[m];
                region = std::max(region, sweep_smem_per_walker(h->nmax, h->P.cg.ncell, h->P.cg.cap, k));
            }
            region = (region + 15) / 16 * 16;
            for (int wpc = 1; k * wpc <= batch_max_warps(q.da) && e == cudaSuccess; wpc *= 2) {
                if ((size_t)wpc * region + stat > kMaxSmem) break;
                const int occ = batch_occupancy(wpc, k, (int)region, q.da, q.cl);
                if (occ < 1) break;
                q.cand.push_back({k, wpc, (int)region});
                if (k == 1 && wpc * occ > best) {
                    best = wpc * occ;
                    q.k = 1;
                    q.wpc = wpc;
                    q.region = (int)region;
                }
            }
        }
        if (q.cand.empty()) e = cudaErrorInvalidValue;   // one walker does not fit
        const int occ = batch_occupancy(q.wpc, q.k, q.region, q.da, q.cl);
        const int need = (int)((q.items.size() + q.wpc - 1) / q.wpc);
        q.grid = std::max(1, std::min(need, b->sms * std::max(occ, 1)));
    }
    const int nb = (int)b->buckets.size();
    if (e == cudaSuccess) e = cudaMalloc(&b->d_sys, count * sizeof(SweepParams));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_xp, count * sizeof(ExchangeParams));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_ectr, count * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counters, nb * sizeof(int));
    for (auto& q : b->buckets) {
        if (e == cudaSuccess) e = cudaMalloc(&q.d_items, q.items.size() * sizeof(int2));
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(q.d_items, q.items.data(), q.items.size() * sizeof(int2), cudaMemcpyHostToDevice,
                                b->stream);
    }
    b->side.assign(nb, nullptr);
    b->join.assign(nb, nullptr);
    for (int k = 1; k < nb && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = upload_descriptors(b);
    if (e != cudaSuccess) {
        const regc_status st = e == cudaErrorMemoryAllocation ? REGC_ENOMEM
                               : e == cudaErrorInvalidValue   ? REGC_EINVAL
                                                              : REGC_ECUDA;
        regc_batch_free(b);
        return st;
    }
    *out = b;
    return REGC_OK;
}

regc_status regc_batch_run(regc_batch* b, int n_steps) {
    NvtxRange nvtx_("regc_batch_run");
    if (!b || n_steps < 0) return REGC_EINVAL;
    if (b->sticky != REGC_OK) return b->sticky;
    regc_status st = check_members(b);
    if (st != REGC_OK) return st;
    if (n_steps == 0) return REGC_OK;
    if (!b->exec) {
        st = fail(b, build_graph(b));
        if (st != REGC_OK) return st;
    }
    for (int k = 0; k < n_steps; ++k) {
        st = fail(b, cudaGraphLaunch(b->exec, b->stream));
        if (st != REGC_OK) return st;
        advance_counters(b, 1);
    }
    return REGC_OK;
}

regc_status regc_batch_sync(regc_batch* b) {
    if (!b) return REGC_EINVAL;
    if (b->sticky != REGC_OK) return b->sticky;
    regc_status st = fail(b, cudaStreamSynchronize(b->stream));
    if (st != REGC_OK) return st;
    for (regc_handle* h : b->members) {
        st = handle_sync_check(h);
        if (st != REGC_OK) return st;
    }
    return REGC_OK;
}

regc_status regc_batch_autotune(regc_batch* b, int rounds) {
    if (!b || rounds < 1) return REGC_EINVAL;
    if (b->sticky != REGC_OK) return b->sticky;
    regc_status st = check_members(b);
    if (st != REGC_OK) return st;
    const int nb = (int)b->buckets.size();
    size_t n_cand = 0;
    for (const auto& q : b->buckets) n_cand = std::max(n_cand, q.cand.size());
    std::vector<double> best(nb, 1e300);
    std::vector<Bucket::Shape> best_shape(nb);
    std::vector<int> best_grid(nb);
    std::vector<double> ms;
    // candidate c of every class in the same timed step; every step is a real step
    for (int r = 0; r < rounds; ++r) {
        for (size_t c = 0; c < n_cand; ++c) {
            for (auto& q : b->buckets) {
                const Bucket::Shape sh = q.cand[std::min(c, q.cand.size() - 1)];
                const int occ = batch_occupancy(sh.wpc, sh.k, sh.region, q.da, q.cl);
                const int need = (int)((q.items.size() + sh.wpc - 1) / sh.wpc);
                q.k = sh.k;
                q.wpc = sh.wpc;
                q.region = sh.region;
                q.grid = std::max(1, std::min(need, b->sms * std::max(occ, 1)));
            }
            st = fail(b, record_step(b, &ms));
            if (st != REGC_OK) return st;
            advance_counters(b, 1);
            for (int k = 0; k < nb; ++k)
                if (ms[k] < best[k]) {
                    best[k] = ms[k];
                    best_shape[k] = {b->buckets[k].k, b->buckets[k].wpc, b->buckets[k].region};
                    best_grid[k] = b->buckets[k].grid;
                }
        }
    }
    for (int k = 0; k < nb; ++k) {
        b->buckets[k].k = best_shape[k].k;
        b->buckets[k].wpc = best_shape[k].wpc;
        b->buckets[k].region = best_shape[k].region;
        b->buckets[k].grid = best_grid[k];
        b->buckets[k].ms = best[k];
    }
    drop_graph(b);
    return REGC_OK;
}

regc_status regc_batch_plan(const regc_batch* b, int max_classes, int* n_classes, int32_t* nmax, int32_t* walkers,
                            int32_t* walkers_per_cta, int32_t* warps_per_walker, int32_t* ctas, double* ms) {
    if (!b || !n_classes) return REGC_EINVAL;
    const int nb = (int)b->buckets.size();
    *n_classes = nb;
    for (int k = 0; k < nb && k < max_classes; ++k) {
        const Bucket& q = b->buckets[k];
        if (nmax) nmax[k] = q.nmax;
        if (walkers) walkers[k] = (int32_t)q.items.size();
        if (walkers_per_cta) walkers_per_cta[k] = q.wpc;
        if (warps_per_walker) warps_per_walker[k] = q.k;
        if (ctas) ctas[k] = q.grid;
        if (ms) ms[k] = q.ms;
    }
    return REGC_OK;
}

}  // extern "C"
