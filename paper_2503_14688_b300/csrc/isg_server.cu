// isg_server.cu -- a request server with continuous batching for the paper's
// protocols: each request is one lattice (Ising or Blume-Capel, its own L,
// seed and bath schedule beta(t) -- the pre-cooling protocol's T1 -> T2 of
// Table II, or any stepped bath), run for its number of sweeps.
//
// Scheduling works in rounds.  At each round the server
//   1. retires requests whose device work has finished (completion times from
//      CUDA events on the device timeline),
//   2. admits queued requests whose arrival time has passed, in arrival order,
//      while the device-memory budget and the slot count allow, and starts
//      them (hot start),
//   3. advances every running request by up to `chunk_sweeps` sweeps: the
//      requests whose lattice fits in shared memory share ONE persistent
//      launch of the batch kernel (isg_batch.cuh; each CTA takes whole
//      lattices); larger requests run the single-lattice kernels on streams of
//      their own, overlapping that launch.
// Requests arriving while others run join at the next round.  The keying of
// the random numbers by (seed, sweep, colour, site) makes every result
// independent of what else runs and of where chunks are cut.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <new>
#include <vector>

#include "isg.h"
#include "isg_batch.cuh"
#include "isg_internal.h"

using namespace isg;

namespace {

isg_status sfail(isg_status code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    return isg::report_error(code, "%s", buf);
}

isg_status scuda(cudaError_t e, const char *what)
{
    cudaGetLastError();
    if (e == cudaErrorMemoryAllocation)
        return sfail(ISG_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return sfail(ISG_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define SCUDA(call, what)                                                                     \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return scuda(e_, what);                                                           \
    } while (0)

constexpr int kSmemLimit = kBatchSmemMax;

struct Request {
    uint64_t id = 0;
    int32_t model = 0;
    int64_t L = 0;
    uint64_t seed = 0;
    double delta = 0.0;
    int64_t n_sweeps = 0;
    std::vector<int64_t> t_start;
    std::vector<double> beta;
    int64_t record_every = 0;
    int32_t keep = 0;
    double t_arrival = 0, t_admit = -1, t_done = -1;
    double deadline = 0;           // server clock; <= 0: none
    int32_t state = ISG_REQ_QUEUED;
    int32_t error = ISG_OK;        // the status that failed it (ISG_REQ_FAILED)
    int64_t queued_sweeps = 0;  // sweeps queued on the device so far
    bool finish_queued = false;
    bool small = false;
    size_t bytes = 0;
    int64_t final_obs[4] = {0, 0, 0, 0};  // [sweep, B, M, Q] once done
    int32_t final_slot = -1;              // slot of the server's pinned final array
    // device resources while admitted
    uint32_t *planes = nullptr;
    uint8_t *recs = nullptr;  // periodic records, then one final record
    int64_t rec_cap = 0;      // periodic records
    int64_t rec_read = 0;     // periodic records already read by the caller
    cudaStream_t stream = nullptr;  // own stream (large requests)
    int32_t stream_prio = 0;        // its priority (smaller lattices: higher)
    cudaEvent_t done = nullptr;
    // large requests: events after their last two chunks; a chunk is queued
    // only once the one two before it has finished, so at most two chunks
    // are ever in flight (cancellation and deadlines act within them)
    cudaEvent_t chunk_ev[2] = {nullptr, nullptr};
    int64_t chunks_queued = 0;
    bool freed = true;
};

double beta_at(const Request &r, int64_t t)
{
    int64_t k = 0;
    while (k + 1 < (int64_t)r.t_start.size() && r.t_start[k + 1] <= t)
        ++k;
    return r.beta[k];
}

}  // namespace

struct isg_server {
    size_t budget = 0, used = 0;
    int32_t max_active = 0;
    int64_t chunk = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::chrono::steady_clock::time_point h0;
    cudaEvent_t ev0 = nullptr;
    uint64_t next_id = 1;
    std::map<uint64_t, std::unique_ptr<Request>> reqs;
    std::deque<uint64_t> queue;      // arrival order
    std::vector<uint64_t> active;    // admitted, not finished
    // idle request streams by priority; priorities run from prio_least
    // (largest lattices) to prio_greatest (numerically lower)
    std::map<int32_t, std::vector<cudaStream_t>> free_streams;
    int32_t prio_least = 0, prio_greatest = 0;
    std::vector<int32_t> free_final_slots;
    int64_t *h_finals = nullptr;     // pinned, 4 int64 per slot (max_active slots)
    // double-buffered launch buffers of the batch kernel (one set per round parity)
    EnsItem *d_items[2] = {nullptr, nullptr}, *h_items[2] = {nullptr, nullptr};
    int32_t *d_order[2] = {nullptr, nullptr}, *h_order[2] = {nullptr, nullptr};
    EnsArgs *d_args[2] = {nullptr, nullptr}, *h_args[2] = {nullptr, nullptr};
    IsingThr *d_ithr[2] = {nullptr, nullptr}, *h_ithr[2] = {nullptr, nullptr};
    BcTable *d_btab[2] = {nullptr, nullptr}, *h_btab[2] = {nullptr, nullptr};
    int32_t *d_counter = nullptr;
    cudaEvent_t round_done[2] = {nullptr, nullptr};
    int64_t round = 0;
    int threads = 1024;
    int blocks = 0;
    double flips_done = 0;
};

namespace {

double clock_now(const isg_server *s)
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->h0).count();
}

cudaStream_t req_stream(const isg_server *s, const Request &r)
{
    return r.small ? s->stream : r.stream;
}

void release_device(isg_server *s, Request &r)
{
    if (r.freed)
        return;
    cudaStream_t st = req_stream(s, r);
    if (r.planes) cudaFreeAsync(r.planes, st);
    if (r.recs) cudaFreeAsync(r.recs, st);
    if (r.stream)
        s->free_streams[r.stream_prio].push_back(r.stream);
    r.planes = nullptr;
    r.recs = nullptr;
    r.stream = nullptr;
    s->used -= r.bytes;
    r.freed = true;
}

size_t request_bytes(const Request &r)
{
    return isg_lattice_bytes(r.model, r.L) + record_stride(r.L) * (size_t)(r.rec_cap + 1);
}

// Stream priority of a large request: the lattices of 2^28 sites or more
// (L = 16384) take the least priority and every halving of L one step more,
// so that the short launches of mid-size requests are scheduled ahead of
// the remaining blocks of the largest ones (the batch of small requests
// runs at the greatest priority).  Scheduling only: results do not depend
// on it.
int32_t request_priority(const isg_server *s, const Request &r)
{
    int steps = 0;
    for (int64_t l = r.L; l < 16384 && steps < 30; l *= 2)
        ++steps;
    const int32_t p = s->prio_least - steps;  // greater priority = numerically lower
    const int32_t floor_p = std::min(s->prio_greatest + 1, s->prio_least);  // the batch keeps the greatest
    return std::max(p, floor_p);
}

isg_status admit(isg_server *s, Request &r)
{
    if (!r.small) {
        r.stream_prio = request_priority(s, r);
        std::vector<cudaStream_t> &pool = s->free_streams[r.stream_prio];
        if (!pool.empty()) {
            r.stream = pool.back();
            pool.pop_back();
        } else {
            SCUDA(cudaStreamCreateWithPriority(&r.stream, cudaStreamNonBlocking, r.stream_prio),
                  "request stream");
        }
    }
    cudaStream_t st = req_stream(s, r);
    cudaError_t e = dev_malloc_async(&r.planes, isg_lattice_bytes(r.model, r.L), st);
    if (e == cudaSuccess)
        e = dev_malloc_async(&r.recs, record_stride(r.L) * (size_t)(r.rec_cap + 1), st);
    r.freed = false;
    s->used += r.bytes;
    if (e != cudaSuccess) {
        release_device(s, r);
        return scuda(e, "request allocation");
    }
    if (!r.done)
        SCUDA(cudaEventCreate(&r.done), "request event");
    for (int k = 0; k < 2 && !r.small; ++k)
        if (!r.chunk_ev[k])
            SCUDA(cudaEventCreateWithFlags(&r.chunk_ev[k], cudaEventDisableTiming), "chunk event");
    Planes pl{r.planes, r.L, r.L / 64, r.model};
    PhiloxLaunch ph0, ph1;
    philox_launch_consts(r.seed, 0u, 2u, &ph0);
    philox_launch_consts(r.seed, 0u, 3u, &ph1);
    SCUDA(launch_init_random(pl, ph0, ph1, st), "request init");
    r.final_slot = s->free_final_slots.back();
    s->free_final_slots.pop_back();
    r.state = ISG_REQ_RUNNING;
    r.t_admit = clock_now(s);
    return ISG_OK;
}

// Queue the end of a request: the final observables and its completion event.
isg_status queue_finish(isg_server *s, Request &r)
{
    cudaStream_t st = req_stream(s, r);
    Planes pl{r.planes, r.L, r.L / 64, r.model};
    uint8_t *fin = r.recs + record_stride(r.L) * (size_t)r.rec_cap;
    SCUDA(cudaMemsetAsync(fin, 0, record_stride(r.L), st), "final record clear");
    SCUDA(launch_measure(pl, fin, r.n_sweeps, st), "final measure");
    SCUDA(cudaMemcpyAsync(s->h_finals + 4 * r.final_slot, fin, 4 * sizeof(int64_t),
                          cudaMemcpyDeviceToHost, st), "final record read");
    SCUDA(cudaEventRecord(r.done, st), "completion event");
    r.finish_queued = true;
    return ISG_OK;
}

// Take a queued or running request out of the schedule for good: cancelled
// by the caller, past its deadline, or failed (its allocation or a launch).
// A running request's queued device work is waited for (its stream: at most
// one chunk), so that nothing still reads its memory when it is freed and
// its final-record slot is reused.
void drop(isg_server *s, Request &r, int32_t state, int32_t error)
{
    auto q = std::find(s->queue.begin(), s->queue.end(), r.id);
    if (q != s->queue.end())
        s->queue.erase(q);
    auto a = std::find(s->active.begin(), s->active.end(), r.id);
    if (a != s->active.end()) {
        s->active.erase(a);
        cudaStreamSynchronize(req_stream(s, r));
        cudaGetLastError();
        release_device(s, r);
        if (r.final_slot >= 0) {
            s->free_final_slots.push_back(r.final_slot);
            r.final_slot = -1;
        }
    }
    r.state = state;
    r.error = error;
    r.t_done = clock_now(s);
}

isg_status run_round(isg_server *s)
{
    const double now = clock_now(s);
    // 1. retire requests whose final copy has landed
    for (size_t i = 0; i < s->active.size();) {
        Request &r = *s->reqs[s->active[i]];
        if (r.finish_queued && cudaEventQuery(r.done) == cudaSuccess) {
            if (s->h_finals[4 * r.final_slot] == kRecordFailed) {
                // the final record pass ran out of time: the request fails
                drop(s, r, ISG_REQ_FAILED, ISG_ERR_DEVICE_TIMEOUT);
                continue;
            }
            float ms = 0;
            cudaEventElapsedTime(&ms, s->ev0, r.done);
            r.t_done = 1e-3 * ms;
            memcpy(r.final_obs, s->h_finals + 4 * r.final_slot, sizeof(r.final_obs));
            s->free_final_slots.push_back(r.final_slot);
            r.final_slot = -1;
            r.state = ISG_REQ_DONE;
            s->flips_done += (double)r.L * (double)r.L * (double)r.n_sweeps;
            if (!r.keep)
                release_device(s, r);
            s->active.erase(s->active.begin() + i);
        } else {
            cudaGetLastError();  // not ready yet
            ++i;
        }
    }
    // requests past their deadline leave the schedule (queued or running)
    std::vector<uint64_t> late;
    for (uint64_t id : s->queue)
        if (s->reqs[id]->deadline > 0 && now > s->reqs[id]->deadline)
            late.push_back(id);
    for (uint64_t id : s->active)
        if (s->reqs[id]->deadline > 0 && now > s->reqs[id]->deadline)
            late.push_back(id);
    for (uint64_t id : late)
        drop(s, *s->reqs[id], ISG_REQ_EXPIRED, ISG_OK);
    // 2. admit in arrival order while slots and the memory budget allow; a
    // request whose allocation fails is failed alone
    while (!s->queue.empty() && (int32_t)s->active.size() < s->max_active) {
        Request &r = *s->reqs[s->queue.front()];
        if (r.t_arrival > now || s->used + r.bytes > s->budget)
            break;
        s->queue.pop_front();
        s->active.push_back(r.id);
        const isg_status st = admit(s, r);
        if (st != ISG_OK)
            drop(s, r, ISG_REQ_FAILED, st);
    }
    // 3. advance every running request by one chunk
    const int buf = (int)(s->round & 1);
    if (s->round >= 2)  // this parity's host buffers were last read by round - 2
        SCUDA(cudaEventSynchronize(s->round_done[buf]), "round sync");
    std::vector<std::pair<int64_t, int32_t>> batch;  // (work, item)
    std::vector<uint64_t> batch_ids;                  // request of each item
    std::vector<std::pair<uint64_t, isg_status>> failed;
    int32_t n_items = 0;
    for (uint64_t id : s->active) {
        Request &r = *s->reqs[id];
        if (r.queued_sweeps >= r.n_sweeps)
            continue;
        if (!r.small && r.chunks_queued >= 2 &&
            cudaEventQuery(r.chunk_ev[r.chunks_queued & 1]) != cudaSuccess) {
            cudaGetLastError();  // not ready: two chunks still in flight
            continue;
        }
        const int64_t n = std::min(s->chunk, r.n_sweeps - r.queued_sweeps);
        const int64_t t0 = r.queued_sweeps;
        if (r.small) {
            const int32_t slot = n_items;
            IsingThr *hi = s->h_ithr[buf] + (size_t)slot * s->chunk;
            BcTable *hb = s->h_btab[buf] + (size_t)slot * s->chunk;
            double last = NAN;
            for (int64_t i = 0; i < n; ++i) {
                const double b = beta_at(r, t0 + i);
                if (r.model == ISG_ISING) {
                    if (b == last)
                        hi[i] = hi[i - 1];
                    else
                        ising_thresholds(b, &hi[i]);
                } else {
                    if (b == last)
                        hb[i] = hb[i - 1];
                    else
                        bc_table(b, r.delta, &hb[i]);
                }
                last = b;
            }
            if (r.model == ISG_ISING)
                SCUDA(cudaMemcpyAsync(s->d_ithr[buf] + (size_t)slot * s->chunk, hi,
                                      sizeof(IsingThr) * n, cudaMemcpyHostToDevice, s->stream),
                      "thresholds");
            else
                SCUDA(cudaMemcpyAsync(s->d_btab[buf] + (size_t)slot * s->chunk, hb,
                                      sizeof(BcTable) * n, cudaMemcpyHostToDevice, s->stream),
                      "thresholds");
            EnsItem &it = s->h_items[buf][slot];
            it = EnsItem{};
            it.seed = r.seed;
            it.planes = r.planes;
            it.L = (int32_t)r.L;
            it.model = r.model;
            it.own = 1;
            it.t0 = (uint32_t)t0;
            it.nsweeps = (int32_t)n;
            // chunks are multiples of record_every (checked at submit), so the
            // kernel's count from the chunk start hits the request's multiples
            it.record_every = (int32_t)r.record_every;
            it.rec_row0 = r.record_every > 0 ? (int32_t)(t0 / r.record_every) : 0;
            it.ithr = s->d_ithr[buf] + (size_t)slot * s->chunk;
            it.btab = s->d_btab[buf] + (size_t)slot * s->chunk;
            it.rec_base = r.recs;
            it.rec_pitch = record_stride(r.L);
            it.rec_cap = (int32_t)std::max<int64_t>(r.rec_cap, 1);
            batch.emplace_back(r.L * r.L * (r.model + 1), slot);
            batch_ids.push_back(id);
            ++n_items;
        } else {
            Planes pl{r.planes, r.L, r.L / 64, r.model};
            double last = NAN;
            IsingThr ithr{};
            BcTable tab;
            for (int64_t i = 0; i < n; ++i) {
                const int64_t t = t0 + i;
                const double b = beta_at(r, t);
                if (b != last) {
                    if (r.model == ISG_ISING)
                        ising_thresholds(b, &ithr);
                    else
                        bc_table(b, r.delta, &tab);
                    last = b;
                }
                cudaError_t e = cudaSuccess;
                for (int c = 0; c < 2 && e == cudaSuccess; ++c) {
                    PhiloxLaunch ph;
                    philox_launch_consts(r.seed, (uint32_t)t, (uint32_t)c, &ph);
                    e = launch_half_sweep(pl, c, ph, ithr, r.model == ISG_ISING ? nullptr : &tab,
                                          r.stream);
                }
                if (e == cudaSuccess && r.record_every > 0 && (t + 1) % r.record_every == 0) {
                    uint8_t *rec = r.recs + record_stride(r.L) * (size_t)((t + 1) / r.record_every - 1);
                    e = cudaMemsetAsync(rec, 0, record_stride(r.L), r.stream);
                    if (e == cudaSuccess)
                        e = launch_measure(pl, rec, t + 1, r.stream);
                }
                if (e != cudaSuccess) {
                    failed.push_back({id, scuda(e, "request launch")});
                    break;
                }
            }
            cudaEventRecord(r.chunk_ev[r.chunks_queued & 1], r.stream);
            r.chunks_queued += 1;
        }
        r.queued_sweeps += n;
    }
    if (n_items > 0) {
        std::sort(batch.begin(), batch.end(), [](const std::pair<int64_t, int32_t> &a,
                                                 const std::pair<int64_t, int32_t> &b) {
            return a.first > b.first;
        });
        for (int32_t i = 0; i < n_items; ++i)
            s->h_order[buf][i] = batch[i].second;
        EnsArgs &a = *s->h_args[buf];
        a = EnsArgs{};
        a.items = s->d_items[buf];
        a.order = s->d_order[buf];
        a.n_order = n_items;
        a.counter = s->d_counter + buf;
        SCUDA(cudaMemcpyAsync(s->d_items[buf], s->h_items[buf], sizeof(EnsItem) * n_items,
                              cudaMemcpyHostToDevice, s->stream), "items");
        SCUDA(cudaMemcpyAsync(s->d_order[buf], s->h_order[buf], sizeof(int32_t) * n_items,
                              cudaMemcpyHostToDevice, s->stream), "order");
        SCUDA(cudaMemcpyAsync(s->d_args[buf], s->h_args[buf], sizeof(EnsArgs),
                              cudaMemcpyHostToDevice, s->stream), "args");
        SCUDA(cudaMemsetAsync(s->d_counter + buf, 0, sizeof(int32_t), s->stream), "counter");
        cudaError_t e = cudaErrorLaunchFailure;
        if (!injected_launch_failure()) {
            k_ensemble<<<s->blocks, s->threads, (size_t)kSmemLimit, s->stream>>>(s->d_args[buf]);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) {  // every request of this batch fails
            const isg_status st = scuda(e, "batch launch");
            for (uint64_t id : batch_ids)
                failed.push_back({id, st});
        }
    }
    for (const auto &f : failed)
        drop(s, *s->reqs[f.first], ISG_REQ_FAILED, f.second);
    // queue the finish of requests whose last chunk went out
    for (uint64_t id : s->active) {
        Request &r = *s->reqs[id];
        if (r.queued_sweeps == r.n_sweeps && !r.finish_queued) {
            isg_status st = queue_finish(s, r);
            if (st != ISG_OK)
                return st;
        }
    }
    SCUDA(cudaEventRecord(s->round_done[buf], s->stream), "round event");
    s->round += 1;
    return ISG_OK;
}

}  // namespace

extern "C" {

isg_status isg_server_create(const isg_server_desc *d, isg_server **out)
{
    if (out)
        *out = nullptr;
    if (!d || !out || d->max_active < 1 || d->chunk_sweeps < 1 || d->hbm_budget == 0)
        return sfail(ISG_ERR_INVALID, "bad server description");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return sfail(ISG_ERR_UNSUPPORTED, "no usable CUDA device");
    }
    isg_server *s = new (std::nothrow) isg_server();
    if (!s)
        return sfail(ISG_ERR_OOM, "host allocation failed");
    auto cleanup = [&](isg_status st) {
        isg_server_destroy(s);
        return st;
    };
    s->max_active = d->max_active;
    s->chunk = d->chunk_sweeps;
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    s->budget = std::min(d->hbm_budget, free_b);
    if (cudaDeviceGetStreamPriorityRange(&s->prio_least, &s->prio_greatest) != cudaSuccess) {
        cudaGetLastError();
        s->prio_least = s->prio_greatest = 0;
    }
    if (d->stream) {
        s->stream = (cudaStream_t)d->stream;
    } else {
        if (cudaStreamCreateWithPriority(&s->stream, cudaStreamNonBlocking, s->prio_greatest) != cudaSuccess)
            return cleanup(scuda(cudaGetLastError(), "stream"));
        s->own_stream = true;
    }
    const size_t na = (size_t)s->max_active;
    const size_t nt = na * (size_t)s->chunk;
    cudaError_t e = dev_malloc(&s->d_counter, sizeof(int32_t) * 2);
    if (e == cudaSuccess)
        e = cudaMallocHost(&s->h_finals, sizeof(int64_t) * 4 * na);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = dev_malloc(&s->d_items[k], sizeof(EnsItem) * na);
        if (e == cudaSuccess) e = cudaMallocHost(&s->h_items[k], sizeof(EnsItem) * na);
        if (e == cudaSuccess) e = dev_malloc(&s->d_order[k], sizeof(int32_t) * na);
        if (e == cudaSuccess) e = cudaMallocHost(&s->h_order[k], sizeof(int32_t) * na);
        if (e == cudaSuccess) e = dev_malloc(&s->d_args[k], sizeof(EnsArgs));
        if (e == cudaSuccess) e = cudaMallocHost(&s->h_args[k], sizeof(EnsArgs));
        if (e == cudaSuccess) e = dev_malloc(&s->d_ithr[k], sizeof(IsingThr) * nt);
        if (e == cudaSuccess) e = cudaMallocHost(&s->h_ithr[k], sizeof(IsingThr) * nt);
        if (e == cudaSuccess) e = dev_malloc(&s->d_btab[k], sizeof(BcTable) * nt);
        if (e == cudaSuccess) e = cudaMallocHost(&s->h_btab[k], sizeof(BcTable) * nt);
        if (e == cudaSuccess) e = cudaEventCreate(&s->round_done[k]);
    }
    for (int32_t k = 0; k < s->max_active; ++k)
        s->free_final_slots.push_back(k);
    if (e == cudaSuccess)
        e = cudaEventCreate(&s->ev0);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_ensemble, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    if (e != cudaSuccess)
        return cleanup(scuda(e, "server allocation"));
    int dev = 0, sms = 148, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ensemble, s->threads, kSmemLimit);
    s->blocks = sms * std::max(per_sm, 1);
    cudaStreamSynchronize(s->stream);
    cudaEventRecord(s->ev0, s->stream);
    cudaEventSynchronize(s->ev0);
    s->h0 = std::chrono::steady_clock::now();
    *out = s;
    return ISG_OK;
}

void isg_server_destroy(isg_server *s)
{
    if (!s)
        return;
    cudaDeviceSynchronize();
    for (auto &kv : s->reqs) {
        Request &r = *kv.second;
        release_device(s, r);
        if (r.done) cudaEventDestroy(r.done);
        for (cudaEvent_t ev : r.chunk_ev)
            if (ev) cudaEventDestroy(ev);
    }
    cudaDeviceSynchronize();
    for (auto &kv : s->free_streams)
        for (cudaStream_t st : kv.second)
            cudaStreamDestroy(st);
    if (s->d_counter) cudaFree(s->d_counter);
    if (s->h_finals) cudaFreeHost(s->h_finals);
    for (int k = 0; k < 2; ++k) {
        if (s->d_items[k]) cudaFree(s->d_items[k]);
        if (s->h_items[k]) cudaFreeHost(s->h_items[k]);
        if (s->d_order[k]) cudaFree(s->d_order[k]);
        if (s->h_order[k]) cudaFreeHost(s->h_order[k]);
        if (s->d_args[k]) cudaFree(s->d_args[k]);
        if (s->h_args[k]) cudaFreeHost(s->h_args[k]);
        if (s->d_ithr[k]) cudaFree(s->d_ithr[k]);
        if (s->h_ithr[k]) cudaFreeHost(s->h_ithr[k]);
        if (s->d_btab[k]) cudaFree(s->d_btab[k]);
        if (s->h_btab[k]) cudaFreeHost(s->h_btab[k]);
        if (s->round_done[k]) cudaEventDestroy(s->round_done[k]);
    }
    if (s->ev0) cudaEventDestroy(s->ev0);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

double isg_server_clock(const isg_server *s) { return s ? clock_now(s) : NAN; }

isg_status isg_server_submit(isg_server *s, const isg_request *q, uint64_t *id)
{
    if (id)
        *id = 0;
    if (!s || !q || !id)
        return sfail(ISG_ERR_INVALID, "bad arguments");
    if (isg_lattice_bytes(q->model, q->L) == 0)
        return sfail(ISG_ERR_INVALID, "request L %lld: must be a valid lattice side (a multiple "
                     "of 64)", (long long)q->L);
    if (q->n_sweeps < 1 || q->n_sweeps > (int64_t)0xFFFFFFFFLL || q->record_every < 0)
        return sfail(ISG_ERR_INVALID, "bad n_sweeps or record_every");
    if (q->n_pieces < 1 || !q->t_start || !q->beta || q->t_start[0] != 0)
        return sfail(ISG_ERR_INVALID, "the schedule must start at sweep 0");
    for (int64_t k = 0; k < q->n_pieces; ++k) {
        if (std::isnan(q->beta[k]) || q->beta[k] < 0.0)
            return sfail(ISG_ERR_INVALID, "schedule beta[%lld] is not >= 0", (long long)k);
        if (k > 0 && q->t_start[k] <= q->t_start[k - 1])
            return sfail(ISG_ERR_INVALID, "schedule t_start must increase");
    }
    if (std::isnan(q->delta) || std::isinf(q->delta))
        return sfail(ISG_ERR_INVALID, "delta must be finite");
    auto r = std::make_unique<Request>();
    r->id = s->next_id++;
    r->model = q->model;
    r->L = q->L;
    r->seed = q->seed;
    r->delta = q->model == ISG_BLUME_CAPEL ? q->delta : 0.0;
    r->n_sweeps = q->n_sweeps;
    r->t_start.assign(q->t_start, q->t_start + q->n_pieces);
    r->beta.assign(q->beta, q->beta + q->n_pieces);
    r->record_every = q->record_every;
    r->keep = q->keep_result;
    r->t_arrival = q->arrival_time >= 0 ? q->arrival_time : clock_now(s);
    r->deadline = q->deadline > 0 ? q->deadline : 0;
    r->small = smem_bytes_for(r->model, r->L) <= (size_t)kSmemLimit;
    r->rec_cap = q->record_every > 0 ? q->n_sweeps / q->record_every : 0;
    // batched requests record inside the kernel at multiples of record_every
    // counted from each chunk's start: keep chunks aligned to record_every
    if (r->small && q->record_every > 0 && s->chunk % q->record_every != 0)
        return sfail(ISG_ERR_INVALID, "record_every %lld must divide the server's chunk %lld",
                     (long long)q->record_every, (long long)s->chunk);
    r->bytes = request_bytes(*r);
    if (r->bytes > s->budget)
        return sfail(ISG_ERR_OOM, "request needs %zu bytes, the budget is %zu", r->bytes, s->budget);
    *id = r->id;
    s->queue.push_back(r->id);
    s->reqs.emplace(r->id, std::move(r));
    return ISG_OK;
}

isg_status isg_server_step(isg_server *s, int32_t *active, int32_t *queued)
{
    if (!s)
        return sfail(ISG_ERR_INVALID, "server is NULL");
    isg_status st = run_round(s);
    if (active)
        *active = (int32_t)s->active.size();
    if (queued)
        *queued = (int32_t)s->queue.size();
    return st;
}

isg_status isg_server_drain(isg_server *s)
{
    if (!s)
        return sfail(ISG_ERR_INVALID, "server is NULL");
    while (!s->active.empty() || !s->queue.empty()) {
        isg_status st = run_round(s);
        if (st != ISG_OK)
            return st;
        if (s->active.empty() && !s->queue.empty()) {
            // nothing runs: wait for the next arrival
            const double next = s->reqs[s->queue.front()]->t_arrival;
            while (clock_now(s) < next) {
            }
        } else if (!s->active.empty()) {
            bool all_queued = true;
            for (uint64_t id : s->active)
                all_queued &= s->reqs[id]->queued_sweeps == s->reqs[id]->n_sweeps;
            if (all_queued && s->queue.empty())
                cudaDeviceSynchronize();
        }
    }
    return ISG_OK;
}

isg_status isg_server_poll(isg_server *s, uint64_t id, isg_result *out)
{
    if (!s || !out)
        return sfail(ISG_ERR_INVALID, "bad arguments");
    auto it = s->reqs.find(id);
    if (it == s->reqs.end())
        return sfail(ISG_ERR_INVALID, "unknown request %llu", (unsigned long long)id);
    const Request &r = *it->second;
    out->state = r.state;
    out->sweeps_done = r.state == ISG_REQ_DONE ? r.n_sweeps : 0;
    out->B = out->M = out->Q = 0;
    if (r.state == ISG_REQ_DONE) {
        out->B = r.final_obs[1];
        out->M = r.final_obs[2];
        out->Q = r.final_obs[3];
    }
    out->t_arrival = r.t_arrival;
    out->t_admit = r.t_admit;
    out->t_done = r.t_done;
    out->records = r.state == ISG_REQ_DONE ? r.rec_cap - r.rec_read : 0;
    out->error = r.error;
    return ISG_OK;
}

isg_status isg_server_cancel(isg_server *s, uint64_t id)
{
    if (!s)
        return sfail(ISG_ERR_INVALID, "server is NULL");
    auto it = s->reqs.find(id);
    if (it == s->reqs.end())
        return sfail(ISG_ERR_INVALID, "unknown request %llu", (unsigned long long)id);
    Request &r = *it->second;
    if (r.state != ISG_REQ_QUEUED && r.state != ISG_REQ_RUNNING)
        return sfail(ISG_ERR_INVALID, "request %llu has already left the schedule (state %d)",
                     (unsigned long long)id, r.state);
    drop(s, r, ISG_REQ_CANCELLED, ISG_OK);
    return ISG_OK;
}

isg_status isg_server_read_records(isg_server *s, uint64_t id, isg_obs *out, int64_t max,
                                   int64_t *count)
{
    if (count)
        *count = 0;
    if (!s || !out || !count || max < 0)
        return sfail(ISG_ERR_INVALID, "bad arguments");
    auto it = s->reqs.find(id);
    if (it == s->reqs.end())
        return sfail(ISG_ERR_INVALID, "unknown request %llu", (unsigned long long)id);
    Request &r = *it->second;
    if (r.state != ISG_REQ_DONE || r.freed)
        return sfail(ISG_ERR_INVALID, "request %llu is not finished with its result kept",
                     (unsigned long long)id);
    const size_t stride = record_stride(r.L);
    const int64_t n = std::min(max, r.rec_cap - r.rec_read);
    for (int64_t i = 0; i < n; ++i) {
        const uint8_t *slot = r.recs + stride * (size_t)(r.rec_read + i);
        int64_t hdr[4];
        SCUDA(cudaMemcpy(hdr, slot, sizeof(hdr), cudaMemcpyDeviceToHost), "record read");
        if (hdr[0] == kRecordFailed) {
            r.rec_read += i + 1;  // dropped
            return sfail(ISG_ERR_DEVICE_TIMEOUT, "record %lld of request %llu: its pass ran out of time",
                         (long long)(r.rec_read - 1), (unsigned long long)id);
        }
        out[i].sweep = hdr[0];
        out[i].B = hdr[1];
        out[i].M = hdr[2];
        out[i].Q = hdr[3];
        if (out[i].row_sums)
            SCUDA(cudaMemcpy(out[i].row_sums, slot + 32, 4 * r.L, cudaMemcpyDeviceToHost), "row sums");
        if (out[i].col_sums)
            SCUDA(cudaMemcpy(out[i].col_sums, slot + 32 + 4 * r.L, 4 * r.L, cudaMemcpyDeviceToHost),
                  "column sums");
        *count = i + 1;
    }
    r.rec_read += n;
    return ISG_OK;
}

isg_status isg_server_get_lattice(isg_server *s, uint64_t id, int8_t *out)
{
    if (!s || !out)
        return sfail(ISG_ERR_INVALID, "bad arguments");
    auto it = s->reqs.find(id);
    if (it == s->reqs.end())
        return sfail(ISG_ERR_INVALID, "unknown request %llu", (unsigned long long)id);
    Request &r = *it->second;
    if (r.state != ISG_REQ_DONE || r.freed)
        return sfail(ISG_ERR_INVALID, "request %llu is not finished with its result kept",
                     (unsigned long long)id);
    Planes pl{r.planes, r.L, r.L / 64, r.model};
    const size_t n = (size_t)r.L * (size_t)r.L;
    int8_t *d = nullptr;
    SCUDA(dev_malloc(&d, n), "staging allocation");
    cudaError_t e = launch_unpack_rect(pl, 0, 0, r.L, r.L, d, s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, d, n, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s->stream);
    cudaFree(d);
    if (e != cudaSuccess)
        return scuda(e, "lattice read");
    return ISG_OK;
}

isg_status isg_server_release(isg_server *s, uint64_t id)
{
    if (!s)
        return sfail(ISG_ERR_INVALID, "server is NULL");
    auto it = s->reqs.find(id);
    if (it == s->reqs.end())
        return sfail(ISG_ERR_INVALID, "unknown request %llu", (unsigned long long)id);
    if (it->second->state != ISG_REQ_DONE)
        return sfail(ISG_ERR_BUSY, "request %llu has not finished", (unsigned long long)id);
    release_device(s, *it->second);
    return ISG_OK;
}

isg_status isg_server_stats(const isg_server *s, double *flips_done, size_t *bytes_in_use,
                            size_t *budget)
{
    if (!s)
        return sfail(ISG_ERR_INVALID, "server is NULL");
    if (flips_done)
        *flips_done = s->flips_done;
    if (bytes_in_use)
        *bytes_in_use = s->used;
    if (budget)
        *budget = s->budget;
    return ISG_OK;
}

}  // extern "C"
