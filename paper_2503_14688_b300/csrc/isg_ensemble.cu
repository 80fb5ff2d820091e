// isg_ensemble.cu -- many independent replicas of uneven L in one persistent,
// graph-captured launch (the replica averages <...> of Eqs. (2)-(3) and
// Appendix B need thousands of independent realisations of a protocol).
//
// Each CTA of a persistent grid (one or more per SM) takes replicas from a
// global work counter, largest L first, copies the replica's spin planes
// into shared memory (an Ising L = 1024 lattice is 128 KiB), runs all sweeps
// of the launch there -- a __syncthreads between half-sweeps, no wait on any
// other CTA -- records observables into the ensemble's record ring, and
// writes the planes back.  The per-site keying is the one of the single
// lattice path, so replica r evolves bit for bit as a lattice created alone
// with the same seed.  Replicas too large for shared memory are swept by the
// global-memory kernels, one after another, on the same stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "isg.h"
#include "isg_internal.h"
#include "isg_philox.cuh"
#include "isg_sweep_core.cuh"

using namespace isg;

#include "isg_batch.cuh"

namespace {

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
isg_status efail(isg_status code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    return isg::report_error(code, "%s", buf);
}

isg_status ecuda(cudaError_t e, const char *what)
{
    cudaGetLastError();
    if (e == cudaErrorMemoryAllocation)
        return efail(ISG_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return efail(ISG_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define ECUDA(call, what)                                                                     \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return ecuda(e_, what);                                                           \
    } while (0)

}  // namespace

struct isg_ensemble {
    int64_t n = 0;
    std::vector<int64_t> L;
    std::vector<int32_t> model;
    std::vector<uint64_t> seed;
    double delta = 0.0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    uint8_t *planes = nullptr;
    std::vector<uint64_t> plane_off;
    std::vector<uint64_t> rec_off;
    EnsItem *d_items = nullptr;
    int32_t *d_order = nullptr;
    int32_t n_smem = 0;
    int32_t split_from = 0;   // order index of the first lattice run by half-CTA teams
    uint32_t half_words = 0;  // shared memory of one team (32-bit words); 0: no teams
    std::vector<int64_t> global_list;
    // the global-path replicas grouped by (model, L), swept by one multi-
    // lattice launch per group and half-sweep
    struct GlobalGroup {
        int32_t model;
        int64_t L;
        std::vector<uint32_t *> planes;
        std::vector<uint64_t> seeds;
        std::vector<int64_t> reps;  // replica indices
    };
    std::vector<GlobalGroup> groups;
    // per-launch arguments and work counters of the persistent launches of
    // one call (sweeps_per_launch > 0 cuts a call into several)
    int32_t *d_counter = nullptr;
    EnsArgs *d_args = nullptr;
    EnsArgs *h_args = nullptr;  // pinned
    // launch shape (isg_ensemble_autotune, isg_ensemble_set_tuning)
    bool teams = true;                 // half-CTA teams once replicas fit half the memory
    int32_t split_from_teams = 0;      // split point with teams (n_smem: no team-sized replica)
    uint32_t half_words_teams = 0;
    size_t smem_whole = 0, smem_teams = 0;
    int64_t sweeps_per_launch = 0;     // 0: one persistent launch per call
    int32_t multi_V = 0, multi_H = 0;  // multi-lattice words per thread, band rows; 0 = automatic
    IsingThr *d_ithr = nullptr, *h_ithr = nullptr;
    BcTable *d_btab = nullptr, *h_btab = nullptr;
    int64_t thr_cap = 0;
    bool any_bc = false;
    uint8_t *rec_ring = nullptr;
    uint64_t row_bytes = 0;
    int64_t rec_cap = 0, rec_head = 0, rec_count = 0;
    int64_t t = 0;
    int threads = 1024;
    int blocks = 0;
    size_t smem = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

// Largest number of launches one sweep call puts in a graph; multi-lattice
// launches carry 24 KB of parameters each, so fewer of them.
constexpr int64_t kMaxGraphLaunches = (int64_t)1 << 16;
constexpr int64_t kMaxGraphMultiLaunches = 2048;
// Most persistent launches one call is cut into.
constexpr int kMaxLaunches = 32;

// Shared memory, split point and grid of the persistent kernel for the
// current shape (threads per CTA, teams on or off).
isg_status apply_shape(isg_ensemble *e);

void free_tables(isg_ensemble *e)
{
    if (e->d_ithr) cudaFree(e->d_ithr);
    if (e->h_ithr) cudaFreeHost(e->h_ithr);
    if (e->d_btab) cudaFree(e->d_btab);
    if (e->h_btab) cudaFreeHost(e->h_btab);
    e->d_ithr = e->h_ithr = nullptr;
    e->d_btab = e->h_btab = nullptr;
    e->thr_cap = 0;
}

isg_status ensure_tables(isg_ensemble *e, int64_t n)
{
    if (n <= e->thr_cap)
        return ISG_OK;
    cudaStreamSynchronize(e->stream);
    free_tables(e);
    const int64_t cap = std::max<int64_t>(n, 64);
    ECUDA(dev_malloc(&e->d_ithr, sizeof(IsingThr) * cap), "threshold table");
    ECUDA(cudaMallocHost(&e->h_ithr, sizeof(IsingThr) * cap), "threshold table (host)");
    if (e->any_bc) {
        ECUDA(dev_malloc(&e->d_btab, sizeof(BcTable) * cap), "threshold table");
        ECUDA(cudaMallocHost(&e->h_btab, sizeof(BcTable) * cap), "threshold table (host)");
    }
    e->thr_cap = cap;
    return ISG_OK;
}

Planes replica_planes(const isg_ensemble *e, int64_t r)
{
    Planes p;
    p.base = reinterpret_cast<uint32_t *>(e->planes + e->plane_off[r]);
    p.L = e->L[r];
    p.W = e->L[r] / 64;
    p.model = e->model[r];
    return p;
}

int occupancy_blocks(int threads, size_t smem)
{
    int dev = 0, sms = 148, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ensemble, threads, smem);
    if (per_sm < 1)
        per_sm = 1;
    return sms * per_sm;
}

// Queue one launch of the shared-memory kernel over all its replicas plus
// the global-memory sweeps of the large replicas, for sweeps t .. t+n-1.
// Persistent launches of one call, sweeps t .. t+n-1: sweeps_per_launch (0 =
// all of them) per launch, rounded up to a multiple of record_every so that
// every launch's records fall on the call's record rows.
int64_t launch_sweeps(const isg_ensemble *e, int64_t n, int64_t record_every)
{
    int64_t k = e->sweeps_per_launch > 0 ? std::min(e->sweeps_per_launch, n) : n;
    if ((n + k - 1) / k > kMaxLaunches)
        k = (n + kMaxLaunches - 1) / kMaxLaunches;
    if (record_every > 0)
        k = (k + record_every - 1) / record_every * record_every;
    return std::max<int64_t>(k, 1);
}

isg_status queue_sweeps(isg_ensemble *e, int64_t n, int64_t record_every, int64_t rec_row0)
{
    cudaStream_t st = e->stream;
    if (e->n_smem > 0 && n > 0) {
        const int64_t k = launch_sweeps(e, n, record_every);
        int ci = 0;
        for (int64_t c0 = 0; c0 < n; c0 += k, ++ci) {
            EnsArgs &a = e->h_args[ci];
            a.items = e->d_items;
            a.order = e->d_order;
            a.n_order = e->n_smem;
            a.counter = e->d_counter + ci;
            a.ithr = e->d_ithr + c0;
            a.btab = e->d_btab ? e->d_btab + c0 : nullptr;
            a.rec_ring = e->rec_ring;
            a.row_bytes = e->row_bytes;
            a.rec_cap = (int32_t)e->rec_cap;
            a.rec_row0 = record_every > 0 ? (int32_t)((rec_row0 + c0 / record_every) % e->rec_cap)
                                          : (int32_t)rec_row0;
            a.t0 = (uint32_t)(e->t + c0);
            a.nsweeps = (int32_t)std::min(k, n - c0);
            a.record_every = (int32_t)record_every;
            a.half_words = e->half_words;
            a.split_from = e->split_from;
            ECUDA(cudaMemcpyAsync(e->d_args + ci, &a, sizeof(EnsArgs), cudaMemcpyHostToDevice, st),
                  "ensemble args");
            ECUDA(cudaMemsetAsync(e->d_counter + ci, 0, sizeof(int32_t), st), "work counter");
            if (injected_launch_failure())
                return ecuda(cudaErrorLaunchFailure, "ensemble launch");
            k_ensemble<<<e->blocks, e->threads, e->smem, st>>>(e->d_args + ci);
            ECUDA(cudaGetLastError(), "ensemble launch");
        }
    }
    for (int64_t i = 0; i < n && !e->groups.empty(); ++i) {
        const uint32_t t = (uint32_t)(e->t + i);
        for (int c = 0; c < 2; ++c)
            for (const auto &gr : e->groups)
                ECUDA(launch_half_sweep_multi(gr.model, gr.L, gr.planes.data(), gr.seeds.data(),
                                              (int)gr.planes.size(), t, c, e->h_ithr[i],
                                              e->h_btab ? &e->h_btab[i] : nullptr, st, e->multi_V,
                                              e->multi_H),
                      "half-sweep launch");
        if (record_every > 0 && (i + 1) % record_every == 0) {
            const int64_t row = (rec_row0 + (i + 1) / record_every - 1) % e->rec_cap;
            for (const auto &gr : e->groups) {
                std::vector<uint8_t *> recs(gr.reps.size());
                for (size_t k = 0; k < gr.reps.size(); ++k)
                    recs[k] = e->rec_ring + (uint64_t)row * e->row_bytes + e->rec_off[gr.reps[k]];
                ECUDA(launch_measure_multi(gr.model, gr.L, gr.planes.data(), recs.data(),
                                           (int)gr.planes.size(), (int64_t)t + 1, st),
                      "measure launch");
            }
        }
    }
    return ISG_OK;
}

isg_status apply_shape(isg_ensemble *e)
{
    const bool teams = e->teams && e->split_from_teams < e->n_smem;
    e->split_from = teams ? e->split_from_teams : e->n_smem;
    e->half_words = teams ? e->half_words_teams : 0;
    e->smem = teams ? e->smem_teams : e->smem_whole;
    if (e->n_smem > 0 && e->smem > 48 * 1024)
        ECUDA(cudaFuncSetAttribute(k_ensemble, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)e->smem),
              "shared memory opt-in");
    e->blocks = occupancy_blocks(e->threads, e->smem);
    if (e->exec) {  // the launch shape changed: rebuild the graph next time
        cudaGraphExecDestroy(e->exec);
        e->exec = nullptr;
    }
    return ISG_OK;
}

}  // namespace

extern "C" {

isg_status isg_ensemble_create(const isg_ensemble_desc *d, isg_ensemble **out)
{
    if (out)
        *out = nullptr;
    if (!d || !out || d->n < 1 || !d->L || !d->seed || d->record_capacity < 1)
        return efail(ISG_ERR_INVALID, "bad ensemble description");
    if (std::isnan(d->delta) || std::isinf(d->delta))
        return efail(ISG_ERR_INVALID, "delta must be finite");
    for (int64_t r = 0; r < d->n; ++r) {
        const int32_t m = d->model ? d->model[r] : ISG_ISING;
        if (isg_lattice_bytes(m, d->L[r]) == 0)
            return efail(ISG_ERR_INVALID, "replica %lld: invalid model %d or L %lld", (long long)r,
                         m, (long long)d->L[r]);
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return efail(ISG_ERR_UNSUPPORTED, "no usable CUDA device");
    }
    isg_ensemble *e = new (std::nothrow) isg_ensemble();
    if (!e)
        return efail(ISG_ERR_OOM, "host allocation failed");
    e->n = d->n;
    e->L.assign(d->L, d->L + d->n);
    e->seed.assign(d->seed, d->seed + d->n);
    e->model.resize(d->n);
    for (int64_t r = 0; r < d->n; ++r) {
        e->model[r] = d->model ? d->model[r] : ISG_ISING;
        e->any_bc |= e->model[r] == ISG_BLUME_CAPEL;
    }
    e->delta = d->delta;
    e->rec_cap = d->record_capacity;
    auto cleanup = [&](isg_status s) {
        isg_ensemble_destroy(e);
        return s;
    };
    if (d->stream) {
        e->stream = (cudaStream_t)d->stream;
    } else {
        if (cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking) != cudaSuccess)
            return cleanup(ecuda(cudaGetLastError(), "stream"));
        e->own_stream = true;
    }
    // planes: one allocation, 256-byte aligned per replica; record offsets
    uint64_t off = 0, roff = 0;
    e->plane_off.resize(d->n);
    e->rec_off.resize(d->n);
    for (int64_t r = 0; r < d->n; ++r) {
        e->plane_off[r] = off;
        off += (isg_lattice_bytes(e->model[r], e->L[r]) + 255) & ~(uint64_t)255;
        e->rec_off[r] = roff;
        roff += record_stride(e->L[r]);
    }
    e->row_bytes = (roff + 255) & ~(uint64_t)255;
    cudaError_t err = dev_malloc(&e->planes, off);
    if (err == cudaSuccess)
        err = dev_malloc(&e->rec_ring, e->row_bytes * (uint64_t)e->rec_cap);
    if (err == cudaSuccess)
        err = dev_malloc(&e->d_counter, sizeof(int32_t) * kMaxLaunches);
    if (err == cudaSuccess)
        err = dev_malloc(&e->d_args, sizeof(EnsArgs) * kMaxLaunches);
    if (err == cudaSuccess)
        err = cudaMallocHost(&e->h_args, sizeof(EnsArgs) * kMaxLaunches);
    if (err != cudaSuccess)
        return cleanup(ecuda(err, "ensemble allocation"));
    // work split: shared-memory replicas largest first; the rest global
    std::vector<int32_t> order;
    size_t smem = 0;
    for (int64_t r = 0; r < d->n; ++r) {
        const size_t need = smem_bytes_for(e->model[r], e->L[r]);
        if (need <= (size_t)kBatchSmemMax) {
            order.push_back((int32_t)r);
            smem = std::max(smem, need);
        } else {
            e->global_list.push_back(r);
        }
    }
    // largest shared-memory need first (longest-processing-time order; the
    // need grows with the work, L^2 sites at 1 or 2 bits)
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        return smem_bytes_for(e->model[a], e->L[a]) > smem_bytes_for(e->model[b], e->L[b]);
    });
    e->n_smem = (int32_t)order.size();
    for (int64_t r : e->global_list) {
        auto it = std::find_if(e->groups.begin(), e->groups.end(), [&](const isg_ensemble::GlobalGroup &gr) {
            return gr.model == e->model[r] && gr.L == e->L[r];
        });
        if (it == e->groups.end()) {
            e->groups.push_back({e->model[r], e->L[r], {}, {}, {}});
            it = e->groups.end() - 1;
        }
        it->planes.push_back(reinterpret_cast<uint32_t *>(e->planes + e->plane_off[r]));
        it->seeds.push_back(e->seed[r]);
        it->reps.push_back(r);
    }
    // lattices that fit half the largest shared-memory request run on
    // half-CTA teams (isg_batch.cuh); the request covers two of them
    const size_t half_cap = ((size_t)kBatchSmemMax / 2) & ~(size_t)15;
    e->smem_whole = smem;
    e->split_from_teams = e->n_smem;
    for (int32_t i = 0; i < e->n_smem; ++i)
        if (smem_bytes_for(e->model[order[i]], e->L[order[i]]) <= half_cap) {
            e->split_from_teams = i;
            break;
        }
    e->smem_teams = smem;
    if (e->split_from_teams < e->n_smem) {
        const size_t half_bytes = (smem_bytes_for(e->model[order[e->split_from_teams]],
                                                  e->L[order[e->split_from_teams]]) + 15) & ~(size_t)15;
        e->half_words_teams = (uint32_t)(half_bytes / 4);
        e->smem_teams = std::max(smem, 2 * half_bytes);
    }
    std::vector<EnsItem> items(d->n);
    for (int64_t r = 0; r < d->n; ++r) {
        items[r].seed = e->seed[r];
        items[r].planes = reinterpret_cast<uint32_t *>(e->planes + e->plane_off[r]);
        items[r].rec_offset = e->rec_off[r];
        items[r].L = (int32_t)e->L[r];
        items[r].model = e->model[r];
        items[r].own = 0;
    }
    err = dev_malloc(&e->d_items, sizeof(EnsItem) * d->n);
    if (err == cudaSuccess && !order.empty())
        err = dev_malloc(&e->d_order, sizeof(int32_t) * order.size());
    if (err == cudaSuccess)
        err = cudaMemcpy(e->d_items, items.data(), sizeof(EnsItem) * d->n, cudaMemcpyHostToDevice);
    if (err == cudaSuccess && !order.empty())
        err = cudaMemcpy(e->d_order, order.data(), sizeof(int32_t) * order.size(),
                         cudaMemcpyHostToDevice);
    if (err != cudaSuccess)
        return cleanup(ecuda(err, "ensemble tables"));
    e->threads = 1024;
    e->teams = e->split_from_teams < e->n_smem;
    const isg_status ss = apply_shape(e);
    if (ss != ISG_OK)
        return cleanup(ss);
    *out = e;
    return ISG_OK;
}

void isg_ensemble_destroy(isg_ensemble *e)
{
    if (!e)
        return;
    if (e->stream)
        cudaStreamSynchronize(e->stream);
    if (e->exec) cudaGraphExecDestroy(e->exec);
    if (e->graph) cudaGraphDestroy(e->graph);
    free_tables(e);
    if (e->planes) cudaFree(e->planes);
    if (e->rec_ring) cudaFree(e->rec_ring);
    if (e->d_counter) cudaFree(e->d_counter);
    if (e->d_args) cudaFree(e->d_args);
    if (e->h_args) cudaFreeHost(e->h_args);
    if (e->d_items) cudaFree(e->d_items);
    if (e->d_order) cudaFree(e->d_order);
    if (e->own_stream && e->stream) cudaStreamDestroy(e->stream);
    delete e;
}

isg_status isg_ensemble_init_random(isg_ensemble *e)
{
    if (!e)
        return efail(ISG_ERR_INVALID, "ensemble is NULL");
    for (int64_t r = 0; r < e->n; ++r) {
        PhiloxLaunch ph0, ph1;
        philox_launch_consts(e->seed[r], 0u, 2u, &ph0);
        philox_launch_consts(e->seed[r], 0u, 3u, &ph1);
        ECUDA(launch_init_random(replica_planes(e, r), ph0, ph1, e->stream), "init launch");
    }
    e->t = 0;
    e->rec_head = e->rec_count = 0;
    return ISG_OK;
}

isg_status isg_ensemble_sweep(isg_ensemble *e, int64_t n, const double *betas, double beta_const,
                              int64_t record_every)
{
    if (!e)
        return efail(ISG_ERR_INVALID, "ensemble is NULL");
    if (n < 0 || record_every < 0 || n > (int64_t)INT32_MAX)
        return efail(ISG_ERR_INVALID, "bad n or record_every");
    if (e->t + n > (int64_t)0xFFFFFFFFLL)
        return efail(ISG_ERR_INVALID, "sweep index would reach 2^32");
    const int64_t nrec = record_every > 0 ? n / record_every : 0;
    if (e->rec_count + nrec > e->rec_cap)
        return efail(ISG_ERR_BUSY, "record ring has room for %lld rows, %lld requested",
                     (long long)(e->rec_cap - e->rec_count), (long long)nrec);
    for (int64_t i = 0; i < n; ++i) {
        const double b = betas ? betas[i] : beta_const;
        if (std::isnan(b) || b < 0.0)
            return efail(ISG_ERR_INVALID, "beta[%lld] = %g is not >= 0", (long long)i, b);
    }
    if (n == 0)
        return ISG_OK;
    isg_status s = ensure_tables(e, n);
    if (s != ISG_OK)
        return s;
    // the pinned tables may still be read by a previous call's copies
    ECUDA(cudaStreamSynchronize(e->stream), "stream sync");
    for (int64_t i = 0; i < n; ++i) {
        const double b = betas ? betas[i] : beta_const;
        ising_thresholds(b, &e->h_ithr[i]);
        if (e->h_btab)
            bc_table(b, e->delta, &e->h_btab[i]);
    }
    const int64_t row0 = (e->rec_head + e->rec_count) % e->rec_cap;
    cudaStream_t st = e->stream;
    // replicas too large for shared memory cost one multi-lattice launch per
    // group and half-sweep (two per group and record: zeroing, measure);
    // beyond the limits the graph's host memory would grow with the call's
    // length, so such a call is queued on the stream directly
    int64_t multi_per_sweep = 0;
    for (const auto &gr : e->groups)
        multi_per_sweep += 2 * (((int64_t)gr.planes.size() + kMultiMax - 1) / kMultiMax);
    const int64_t multi_launches = multi_per_sweep * n;
    int64_t global_launches = multi_launches;
    if (record_every > 0)
        global_launches += multi_per_sweep * (n / record_every);  // zeroing + measure per group chunk
    if (global_launches > kMaxGraphLaunches || multi_launches > kMaxGraphMultiLaunches) {
        ECUDA(cudaMemcpyAsync(e->d_ithr, e->h_ithr, sizeof(IsingThr) * n, cudaMemcpyHostToDevice, st),
              "threshold upload");
        if (e->h_btab)
            ECUDA(cudaMemcpyAsync(e->d_btab, e->h_btab, sizeof(BcTable) * n, cudaMemcpyHostToDevice, st),
                  "threshold upload");
        isg_status qs = queue_sweeps(e, n, record_every, row0);
        if (qs != ISG_OK)
            return qs;
        e->t += n;
        e->rec_count += nrec;
        return ISG_OK;
    }
    // capture this call's device work in a graph and replay it; a later call
    // with the same shape updates the instantiated graph in place
    ECUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaError_t ce = cudaMemcpyAsync(e->d_ithr, e->h_ithr, sizeof(IsingThr) * n,
                                     cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess && e->h_btab)
        ce = cudaMemcpyAsync(e->d_btab, e->h_btab, sizeof(BcTable) * n, cudaMemcpyHostToDevice, st);
    isg_status qs = ce == cudaSuccess ? queue_sweeps(e, n, record_every, row0) : ISG_OK;
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamEndCapture(st, &g);
    if (ce != cudaSuccess || qs != ISG_OK || ee != cudaSuccess) {
        if (g)
            cudaGraphDestroy(g);
        if (qs != ISG_OK)
            return qs;
        return ecuda(ce != cudaSuccess ? ce : ee, "graph capture");
    }
    bool updated = false;
    if (e->exec) {
        cudaGraphExecUpdateResultInfo info;
        updated = cudaGraphExecUpdate(e->exec, g, &info) == cudaSuccess;
        if (!updated) {
            cudaGetLastError();
            cudaGraphExecDestroy(e->exec);
            e->exec = nullptr;
        }
    }
    if (!updated) {
        const cudaError_t ie = cudaGraphInstantiate(&e->exec, g, 0);
        if (ie != cudaSuccess) {
            cudaGraphDestroy(g);
            return ecuda(ie, "graph instantiate");
        }
    }
    if (e->graph)
        cudaGraphDestroy(e->graph);
    e->graph = g;
    ECUDA(cudaGraphLaunch(e->exec, st), "graph launch");
    e->t += n;
    e->rec_count += nrec;
    return ISG_OK;
}

isg_status isg_ensemble_read_records(isg_ensemble *e, int64_t rows, isg_obs *out, int64_t *count)
{
    if (count)
        *count = 0;
    if (!e || !out || !count || rows < 0)
        return efail(ISG_ERR_INVALID, "bad arguments");
    ECUDA(cudaStreamSynchronize(e->stream), "stream sync");
    const int64_t k = std::min(rows, e->rec_count);
    std::vector<uint8_t> buf(e->row_bytes);
    for (int64_t i = 0; i < k; ++i) {
        ECUDA(cudaMemcpy(buf.data(), e->rec_ring + (uint64_t)e->rec_head * e->row_bytes, e->row_bytes,
                         cudaMemcpyDeviceToHost),
              "record read");
        for (int64_t r = 0; r < e->n; ++r) {
            const uint8_t *rec = buf.data() + e->rec_off[r];
            int64_t hdr[4];
            memcpy(hdr, rec, sizeof(hdr));
            isg_obs &o = out[i * e->n + r];
            o.sweep = hdr[0];
            o.B = hdr[1];
            o.M = hdr[2];
            o.Q = hdr[3];
            if (o.row_sums)
                memcpy(o.row_sums, rec + 32, sizeof(int32_t) * e->L[r]);
            if (o.col_sums)
                memcpy(o.col_sums, rec + 32 + sizeof(int32_t) * e->L[r], sizeof(int32_t) * e->L[r]);
        }
        e->rec_head = (e->rec_head + 1) % e->rec_cap;
        e->rec_count -= 1;
        *count = i + 1;
    }
    return ISG_OK;
}

isg_status isg_ensemble_info(const isg_ensemble *e, int64_t *n, int64_t *sweep, int64_t *pending,
                             int32_t *threads_per_cta)
{
    if (!e)
        return efail(ISG_ERR_INVALID, "ensemble is NULL");
    if (n)
        *n = e->n;
    if (sweep)
        *sweep = e->t;
    if (pending)
        *pending = e->rec_count;
    if (threads_per_cta)
        *threads_per_cta = e->threads;
    return ISG_OK;
}

isg_status isg_ensemble_get(isg_ensemble *e, int64_t r, int8_t *out)
{
    if (!e || !out || r < 0 || r >= e->n)
        return efail(ISG_ERR_INVALID, "bad arguments");
    const Planes pl = replica_planes(e, r);
    const size_t nbytes = (size_t)pl.L * (size_t)pl.L;
    int8_t *d = nullptr;
    ECUDA(dev_malloc_async(&d, nbytes, e->stream), "staging allocation");
    cudaError_t err = launch_unpack_rect(pl, 0, 0, pl.L, pl.L, d, e->stream);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(out, d, nbytes, cudaMemcpyDeviceToHost, e->stream);
    cudaFreeAsync(d, e->stream);
    if (err == cudaSuccess)
        err = cudaStreamSynchronize(e->stream);
    if (err != cudaSuccess)
        return ecuda(err, "replica read");
    return ISG_OK;
}

isg_status isg_ensemble_get_tuning(const isg_ensemble *e, isg_ensemble_tuning *t)
{
    if (!e || !t)
        return efail(ISG_ERR_INVALID, "bad arguments");
    *t = isg_ensemble_tuning{};
    t->threads_per_cta = e->threads;
    t->half_teams = e->teams && e->split_from_teams < e->n_smem ? 1 : 0;
    t->sweeps_per_launch = e->sweeps_per_launch;
    t->multi_words = e->multi_V;
    t->multi_band = e->multi_H;
    return ISG_OK;
}

isg_status isg_ensemble_set_tuning(isg_ensemble *e, const isg_ensemble_tuning *t)
{
    if (!e || !t)
        return efail(ISG_ERR_INVALID, "bad arguments");
    if (t->threads_per_cta != 256 && t->threads_per_cta != 512 && t->threads_per_cta != 1024)
        return efail(ISG_ERR_INVALID, "threads_per_cta must be 256, 512 or 1024");
    if (t->sweeps_per_launch < 0 || t->multi_words < 0 || t->multi_words > 4 || t->multi_band < 0 ||
        t->multi_band > 64)
        return efail(ISG_ERR_INVALID, "bad launch shape");
    ECUDA(cudaStreamSynchronize(e->stream), "stream sync");
    e->threads = t->threads_per_cta;
    e->teams = t->half_teams != 0;
    e->sweeps_per_launch = t->sweeps_per_launch;
    e->multi_V = t->multi_words;
    e->multi_H = t->multi_band;
    return apply_shape(e);
}

isg_status isg_ensemble_autotune(isg_ensemble *e, int64_t sweeps, isg_ensemble_tuning *best,
                                 isg_ensemble_tuning *tried, int64_t max_tried, int64_t *n_tried)
{
    if (n_tried)
        *n_tried = 0;
    if (!e || sweeps < 1 || sweeps > INT32_MAX || max_tried < 0 || (max_tried > 0 && !tried))
        return efail(ISG_ERR_INVALID, "bad arguments");
    // time the candidates on a copy of the planes, so that the ensemble's
    // own state does not move
    isg_status s = ensure_tables(e, sweeps);
    if (s != ISG_OK)
        return s;
    ECUDA(cudaStreamSynchronize(e->stream), "stream sync");
    for (int64_t i = 0; i < sweeps; ++i)
        ising_thresholds(0.44068679350977147, &e->h_ithr[i]);
    if (e->h_btab)
        for (int64_t i = 0; i < sweeps; ++i)
            bc_table(0.59, e->delta, &e->h_btab[i]);
    size_t total = 0;
    for (int64_t r = 0; r < e->n; ++r)
        total = std::max<size_t>(total, e->plane_off[r] + isg_lattice_bytes(e->model[r], e->L[r]));
    uint8_t *copy = nullptr;
    EnsItem *items = nullptr;
    ECUDA(dev_malloc(&copy, total), "autotune copy");
    cudaError_t err = dev_malloc(&items, sizeof(EnsItem) * e->n);
    std::vector<EnsItem> h(e->n);
    if (err == cudaSuccess)
        err = cudaMemcpy(h.data(), e->d_items, sizeof(EnsItem) * e->n, cudaMemcpyDeviceToHost);
    for (int64_t r = 0; r < e->n && err == cudaSuccess; ++r)
        h[r].planes = reinterpret_cast<uint32_t *>(copy + e->plane_off[r]);
    if (err == cudaSuccess)
        err = cudaMemcpy(items, h.data(), sizeof(EnsItem) * e->n, cudaMemcpyHostToDevice);
    if (err == cudaSuccess)
        err = cudaMemcpy(copy, e->planes, total, cudaMemcpyDeviceToDevice);
    if (err == cudaSuccess)
        err = cudaMemcpy(e->d_ithr, e->h_ithr, sizeof(IsingThr) * sweeps, cudaMemcpyHostToDevice);
    if (err == cudaSuccess && e->h_btab)
        err = cudaMemcpy(e->d_btab, e->h_btab, sizeof(BcTable) * sweeps, cudaMemcpyHostToDevice);
    cudaEvent_t ea = nullptr, eb = nullptr;
    if (err == cudaSuccess)
        err = cudaEventCreate(&ea);
    if (err == cudaSuccess)
        err = cudaEventCreate(&eb);
    // the large replicas' plane pointers inside the copy
    std::vector<std::vector<uint32_t *>> gplanes;
    for (const auto &gr : e->groups) {
        gplanes.emplace_back();
        for (int64_t r : gr.reps)
            gplanes.back().push_back(reinterpret_cast<uint32_t *>(copy + e->plane_off[r]));
    }
    const int saved_threads = e->threads;
    const bool saved_teams = e->teams;
    const int64_t saved_spl = e->sweeps_per_launch;
    // time one configuration: the queued work `body`, after one warm-up run
    auto timed = [&](auto body, double *ms_out) {
        for (int rep = 0; rep < 2 && err == cudaSuccess; ++rep) {
            err = cudaEventRecord(ea, e->stream);
            if (err == cudaSuccess)
                err = body();
            if (err == cudaSuccess)
                err = cudaEventRecord(eb, e->stream);
            if (err == cudaSuccess)
                err = cudaEventSynchronize(eb);
            float ms = 0;
            if (err == cudaSuccess && rep == 1 && cudaEventElapsedTime(&ms, ea, eb) == cudaSuccess)
                *ms_out = ms;
        }
    };
    std::vector<isg_ensemble_tuning> cands;
    isg_ensemble_tuning pick{};
    pick.threads_per_cta = e->threads;
    pick.half_teams = e->teams ? 1 : 0;
    double best_a = 0.0, best_b = 0.0;
    // part 0: the persistent shared-memory kernel -- CTA size, half-CTA
    // teams, sweeps per launch
    if (e->n_smem > 0) {
        best_a = 1e300;
        const int threads_c[3] = {256, 512, 1024};
        const bool can_split = e->split_from_teams < e->n_smem;
        const int64_t spl_c[2] = {0, std::max<int64_t>(1, sweeps / 5)};
        for (int ti = 0; ti < 3 && err == cudaSuccess; ++ti)
            for (int teams = can_split ? 1 : 0; teams >= 0 && err == cudaSuccess; --teams)
                for (int si = 0; si < 2 && err == cudaSuccess; ++si) {
                    e->threads = threads_c[ti];
                    e->teams = teams != 0;
                    if (apply_shape(e) != ISG_OK) {
                        err = cudaErrorInvalidValue;
                        break;
                    }
                    const int64_t k = spl_c[si] > 0 ? std::min(spl_c[si], sweeps) : sweeps;
                    double ms = -1.0;
                    timed([&]() -> cudaError_t {
                        int ci = 0;
                        for (int64_t c0 = 0; c0 < sweeps; c0 += k, ++ci) {
                            EnsArgs a{};
                            a.items = items;
                            a.order = e->d_order;
                            a.n_order = e->n_smem;
                            a.counter = e->d_counter + (ci % kMaxLaunches);
                            a.ithr = e->d_ithr + c0;
                            a.btab = e->d_btab ? e->d_btab + c0 : nullptr;
                            a.rec_ring = e->rec_ring;
                            a.row_bytes = e->row_bytes;
                            a.rec_cap = (int32_t)e->rec_cap;
                            a.t0 = (uint32_t)c0;
                            a.nsweeps = (int32_t)std::min(k, sweeps - c0);
                            a.half_words = e->half_words;
                            a.split_from = e->split_from;
                            e->h_args[ci % kMaxLaunches] = a;
                            cudaError_t x = cudaMemcpyAsync(e->d_args + (ci % kMaxLaunches), &e->h_args[ci % kMaxLaunches],
                                                            sizeof(EnsArgs), cudaMemcpyHostToDevice, e->stream);
                            if (x == cudaSuccess)
                                x = cudaMemsetAsync(e->d_counter + (ci % kMaxLaunches), 0, sizeof(int32_t), e->stream);
                            if (x != cudaSuccess)
                                return x;
                            k_ensemble<<<e->blocks, e->threads, e->smem, e->stream>>>(e->d_args + (ci % kMaxLaunches));
                            x = cudaGetLastError();
                            if (x == cudaSuccess && ci % kMaxLaunches == kMaxLaunches - 1)
                                x = cudaStreamSynchronize(e->stream);  // pinned arguments reused
                            if (x != cudaSuccess)
                                return x;
                        }
                        return cudaSuccess;
                    }, &ms);
                    isg_ensemble_tuning c{};
                    c.threads_per_cta = e->threads;
                    c.half_teams = teams;
                    c.sweeps_per_launch = spl_c[si];
                    c.ms = ms;
                    c.part = 0;
                    cands.push_back(c);
                    if (ms >= 0 && ms < best_a) {
                        best_a = ms;
                        pick.threads_per_cta = c.threads_per_cta;
                        pick.half_teams = c.half_teams;
                        pick.sweeps_per_launch = c.sweeps_per_launch;
                    }
                }
    }
    // part 1: the multi-lattice launches of the large replicas -- words per
    // thread and band rows
    if (!e->groups.empty() && err == cudaSuccess) {
        best_b = 1e300;
        const int V_c[4] = {0, 1, 2, 4};
        const int H_c[4] = {0, 16, 32, 64};
        for (int vi = 0; vi < 4 && err == cudaSuccess; ++vi)
            for (int hi = 0; hi < 4 && err == cudaSuccess; ++hi) {
                double ms = -1.0;
                timed([&]() -> cudaError_t {
                    for (int64_t i = 0; i < sweeps; ++i)
                        for (int c = 0; c < 2; ++c)
                            for (size_t g = 0; g < e->groups.size(); ++g) {
                                const auto &gr = e->groups[g];
                                const cudaError_t x = launch_half_sweep_multi(
                                    gr.model, gr.L, gplanes[g].data(), gr.seeds.data(),
                                    (int)gplanes[g].size(), (uint32_t)i, c, e->h_ithr[i],
                                    e->h_btab ? &e->h_btab[i] : nullptr, e->stream, V_c[vi], H_c[hi]);
                                if (x != cudaSuccess)
                                    return x;
                            }
                    return cudaSuccess;
                }, &ms);
                isg_ensemble_tuning c{};
                c.threads_per_cta = pick.threads_per_cta;
                c.half_teams = pick.half_teams;
                c.sweeps_per_launch = pick.sweeps_per_launch;
                c.multi_words = V_c[vi];
                c.multi_band = H_c[hi];
                c.ms = ms;
                c.part = 1;
                cands.push_back(c);
                if (ms >= 0 && ms < best_b) {
                    best_b = ms;
                    pick.multi_words = V_c[vi];
                    pick.multi_band = H_c[hi];
                }
            }
    }
    if (ea) cudaEventDestroy(ea);
    if (eb) cudaEventDestroy(eb);
    cudaStreamSynchronize(e->stream);
    cudaFree(copy);
    cudaFree(items);
    if (err != cudaSuccess) {
        e->threads = saved_threads;
        e->teams = saved_teams;
        e->sweeps_per_launch = saved_spl;
        apply_shape(e);
        return ecuda(err, "autotune");
    }
    e->threads = pick.threads_per_cta;
    e->teams = pick.half_teams != 0;
    e->sweeps_per_launch = pick.sweeps_per_launch;
    e->multi_V = pick.multi_words;
    e->multi_H = pick.multi_band;
    s = apply_shape(e);
    if (s != ISG_OK)
        return s;
    pick.ms = best_a + best_b;
    if (best)
        *best = pick;
    const int64_t n = std::min<int64_t>(max_tried, (int64_t)cands.size());
    for (int64_t i = 0; i < n; ++i)
        tried[i] = cands[(size_t)i];
    if (n_tried)
        *n_tried = (int64_t)cands.size();
    return ISG_OK;
}

}  // extern "C"
