// isg_api.cu -- the C ABI of libisg (declared in include/isg.h): lattice
// objects, the sweep driver (constant beta, per-sweep beta(t), piecewise
// schedules), the on-device record ring and the host-side reads.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <new>
#include <vector>

#include "isg.h"
#include "isg_internal.h"

using namespace isg;

namespace {

thread_local char g_err[512] = "";

isg_status fail(isg_status code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

isg_status cuda_fail(cudaError_t e, const char *what)
{
    if (e == cudaErrorMemoryAllocation)
        return fail(ISG_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver)
        return fail(ISG_ERR_UNSUPPORTED, "%s: %s", what, cudaGetErrorString(e));
    return fail(ISG_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define ISG_CUDA(call, what)                                                                  \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return cuda_fail(e_, what);                                                       \
    } while (0)

bool valid_L(int32_t model, int64_t L)
{
    if (model != ISG_ISING && model != ISG_BLUME_CAPEL)
        return false;
    const int64_t maxL = model == ISG_ISING ? (int64_t)1 << 20 : (int64_t)1 << 19;
    return L >= 64 && L % 64 == 0 && L <= maxL;
}

bool valid_beta(double b) { return !std::isnan(b) && b >= 0.0; }

}  // namespace

namespace isg {

namespace {
// armed injections: the count of events still to pass before the failing
// one (0 = disarmed)
std::atomic<int64_t> g_inject_alloc{0}, g_inject_launch{0}, g_inject_wait{0};

bool take(std::atomic<int64_t> &counter)
{
    int64_t v = counter.load();
    while (v > 0) {
        if (counter.compare_exchange_weak(v, v - 1))
            return v == 1;
    }
    return false;
}
}  // namespace

cudaError_t dev_malloc_raw(void **p, size_t bytes)
{
    if (take(g_inject_alloc)) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

cudaError_t dev_malloc_async_raw(void **p, size_t bytes, cudaStream_t st)
{
    if (take(g_inject_alloc)) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMallocAsync(p, bytes, st);
}

bool injected_launch_failure() { return take(g_inject_launch); }

bool injected_wait_failure() { return take(g_inject_wait); }

int32_t report_error(int32_t code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

}  // namespace isg

struct isg_lattice {
    int32_t model;
    int64_t L, W;
    uint64_t seed;
    double delta;
    cudaStream_t stream;
    uint32_t *planes;
    bool owns_planes;
    uint8_t *records;        // rec_cap ring slots + 1 private slot for isg_measure
    int64_t rec_cap, rec_head, rec_count;
    size_t rec_stride;
    int64_t t;               // sweeps done
    int32_t *d_flag;
    int device;
    uint32_t *sw_labels = nullptr;  // Swendsen-Wang labels (allocated on first use)
    int64_t sw_count = 0;           // Swendsen-Wang iterations done
    // thresholds of the last beta a half-sweep used (NaN: none yet)
    double thr_beta = std::numeric_limits<double>::quiet_NaN();
    IsingThr thr_ising{};
    BcTable thr_bc{};
};

namespace {

Planes planes_of(const isg_lattice *lat)
{
    Planes p;
    p.base = lat->planes;
    p.L = lat->L;
    p.W = lat->W;
    p.model = lat->model;
    return p;
}

isg_status check_device(void)
{
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0) {
        cudaGetLastError();
        return fail(ISG_ERR_UNSUPPORTED, "no usable CUDA device (%s)",
                    e == cudaSuccess ? "device count 0" : cudaGetErrorString(e));
    }
    return ISG_OK;
}

isg_status queue_half(isg_lattice *lat, int colour, double beta)
{
    PhiloxLaunch ph;
    philox_launch_consts(lat->seed, (uint32_t)lat->t, (uint32_t)colour, &ph);
    if (!(beta == lat->thr_beta)) {  // both colours and constant-beta runs reuse the table
        if (lat->model == ISG_ISING)
            ising_thresholds(beta, &lat->thr_ising);
        else
            bc_table(beta, lat->delta, &lat->thr_bc);
        lat->thr_beta = beta;
    }
    const BcTable *tp = lat->model == ISG_ISING ? nullptr : &lat->thr_bc;
    ISG_CUDA(launch_half_sweep(planes_of(lat), colour, ph, lat->thr_ising, tp, lat->stream),
             "half-sweep launch");
    if (colour == 1)
        lat->t += 1;
    return ISG_OK;
}

isg_status queue_record(isg_lattice *lat, uint8_t *slot)
{
    ISG_CUDA(cudaMemsetAsync(slot, 0, lat->rec_stride, lat->stream), "record clear");
    ISG_CUDA(launch_measure(planes_of(lat), slot, lat->t, lat->stream), "measure launch");
    return ISG_OK;
}

isg_status push_record(isg_lattice *lat)
{
    if (lat->rec_count >= lat->rec_cap)
        return fail(ISG_ERR_BUSY, "record ring full (%lld records pending)", (long long)lat->rec_count);
    uint8_t *slot = lat->records + (size_t)((lat->rec_head + lat->rec_count) % lat->rec_cap) * lat->rec_stride;
    isg_status s = queue_record(lat, slot);
    if (s == ISG_OK)
        lat->rec_count += 1;
    return s;
}

isg_status copy_record(const isg_lattice *lat, const uint8_t *slot, isg_obs *out)
{
    int64_t hdr[4];
    ISG_CUDA(cudaMemcpy(hdr, slot, sizeof(hdr), cudaMemcpyDeviceToHost), "record read");
    if (hdr[0] == kRecordFailed)
        return fail(ISG_ERR_DEVICE_TIMEOUT, "the record pass ran out of time waiting for its row copies");
    out->sweep = hdr[0];
    out->B = hdr[1];
    out->M = hdr[2];
    out->Q = hdr[3];
    const int32_t *R = reinterpret_cast<const int32_t *>(slot + 32);
    if (out->row_sums)
        ISG_CUDA(cudaMemcpy(out->row_sums, R, sizeof(int32_t) * lat->L, cudaMemcpyDeviceToHost),
                 "row sums read");
    if (out->col_sums)
        ISG_CUDA(cudaMemcpy(out->col_sums, R + lat->L, sizeof(int32_t) * lat->L,
                            cudaMemcpyDeviceToHost),
                 "column sums read");
    return ISG_OK;
}

isg_status sweep_impl(isg_lattice *lat, int64_t n, const double *betas, double beta_const,
                      const isg_schedule *sched, int64_t record_every)
{
    if (!lat)
        return fail(ISG_ERR_INVALID, "lattice is NULL");
    if (n < 0 || record_every < 0)
        return fail(ISG_ERR_INVALID, "n and record_every must be >= 0");
    if (lat->t + n > (int64_t)0xFFFFFFFFLL)
        return fail(ISG_ERR_INVALID, "sweep index would reach 2^32");
    std::vector<double> beta((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        double b = beta_const;
        if (betas) {
            b = betas[i];
        } else if (sched) {
            const int64_t t = lat->t + i;
            if (sched->n_pieces < 1 || !sched->t_start || !sched->beta || sched->t_start[0] > t)
                return fail(ISG_ERR_INVALID, "schedule does not cover sweep %lld", (long long)t);
            int64_t k = 0;
            while (k + 1 < sched->n_pieces && sched->t_start[k + 1] <= t)
                ++k;
            b = sched->beta[k];
        }
        if (!valid_beta(b))
            return fail(ISG_ERR_INVALID, "beta[%lld] = %g is not >= 0", (long long)i, b);
        beta[(size_t)i] = b;
    }
    if (sched)
        for (int64_t k = 1; k < sched->n_pieces; ++k)
            if (sched->t_start[k] <= sched->t_start[k - 1])
                return fail(ISG_ERR_INVALID, "schedule t_start must increase");
    const int64_t nrec = record_every > 0 ? n / record_every : 0;
    if (lat->rec_count + nrec > lat->rec_cap)
        return fail(ISG_ERR_BUSY, "record ring has room for %lld records, %lld requested",
                    (long long)(lat->rec_cap - lat->rec_count), (long long)nrec);
    for (int64_t i = 0; i < n; ++i) {
        isg_status s = queue_half(lat, 0, beta[(size_t)i]);
        if (s == ISG_OK)
            s = queue_half(lat, 1, beta[(size_t)i]);
        if (s == ISG_OK && record_every > 0 && (i + 1) % record_every == 0)
            s = push_record(lat);
        if (s != ISG_OK)
            return s;
    }
    return ISG_OK;
}

}  // namespace

extern "C" {

isg_status isg_debug_inject(int32_t what, int64_t after)
{
    if (after < 0)
        return fail(ISG_ERR_INVALID, "after must be >= 0");
    if (what == ISG_INJECT_ALLOC)
        isg::g_inject_alloc.store(after);
    else if (what == ISG_INJECT_LAUNCH)
        isg::g_inject_launch.store(after);
    else if (what == ISG_INJECT_WAIT)
        isg::g_inject_wait.store(after);
    else
        return fail(ISG_ERR_INVALID, "unknown injection %d", what);
    return ISG_OK;
}

size_t isg_lattice_bytes(int32_t model, int64_t L)
{
    if (!valid_L(model, L))
        return 0;
    return (size_t)L * (size_t)L / (model == ISG_ISING ? 8 : 4);
}

isg_status isg_lattice_create(const isg_lattice_desc *desc, isg_lattice **out)
{
    if (out)
        *out = nullptr;
    if (!desc || !out)
        return fail(ISG_ERR_INVALID, "desc and out must not be NULL");
    if (!valid_L(desc->model, desc->L))
        return fail(ISG_ERR_INVALID, "invalid model %d or L %lld (L must be a multiple of 64 in "
                    "[64, 2^20] for Ising, [64, 2^19] for Blume-Capel)", desc->model,
                    (long long)desc->L);
    if (desc->record_capacity < 1)
        return fail(ISG_ERR_INVALID, "record_capacity must be >= 1");
    if (std::isnan(desc->delta) || std::isinf(desc->delta))
        return fail(ISG_ERR_INVALID, "delta must be finite");
    const size_t bytes = isg_lattice_bytes(desc->model, desc->L);
    if (desc->device_buf && desc->device_buf_bytes < bytes)
        return fail(ISG_ERR_INVALID, "device_buf holds %zu bytes, %zu needed",
                    desc->device_buf_bytes, bytes);
    if (desc->device_buf && ((uintptr_t)desc->device_buf % 16) != 0)
        return fail(ISG_ERR_INVALID, "device_buf must be 16-byte aligned");
    isg_status st = check_device();
    if (st != ISG_OK)
        return st;
    isg_lattice *lat = new (std::nothrow) isg_lattice();
    if (!lat)
        return fail(ISG_ERR_OOM, "host allocation failed");
    lat->model = desc->model;
    lat->L = desc->L;
    lat->W = desc->L / 64;
    lat->seed = desc->seed;
    lat->delta = desc->model == ISG_BLUME_CAPEL ? desc->delta : 0.0;
    lat->stream = (cudaStream_t)desc->stream;
    lat->rec_cap = desc->record_capacity;
    lat->rec_stride = record_stride(desc->L);
    cudaGetDevice(&lat->device);
    cudaError_t e = cudaSuccess;
    if (desc->device_buf) {
        lat->planes = (uint32_t *)desc->device_buf;
        lat->owns_planes = false;
    } else {
        e = dev_malloc(&lat->planes, bytes);
        lat->owns_planes = true;
    }
    if (e == cudaSuccess)
        e = dev_malloc(&lat->records, lat->rec_stride * (size_t)(lat->rec_cap + 1));
    if (e == cudaSuccess)
        e = dev_malloc(&lat->d_flag, sizeof(int32_t));
    if (e != cudaSuccess) {
        isg_status s = cuda_fail(e, "lattice allocation");
        cudaGetLastError();
        isg_lattice_destroy(lat);
        return s;
    }
    *out = lat;
    return ISG_OK;
}

void isg_lattice_destroy(isg_lattice *lat)
{
    if (!lat)
        return;
    cudaStreamSynchronize(lat->stream);
    if (lat->owns_planes && lat->planes)
        cudaFree(lat->planes);
    if (lat->records)
        cudaFree(lat->records);
    if (lat->d_flag)
        cudaFree(lat->d_flag);
    if (lat->sw_labels)
        cudaFree(lat->sw_labels);
    delete lat;
}

isg_status isg_lattice_init_random(isg_lattice *lat)
{
    if (!lat)
        return fail(ISG_ERR_INVALID, "lattice is NULL");
    PhiloxLaunch ph0, ph1;
    philox_launch_consts(lat->seed, 0u, 2u, &ph0);
    philox_launch_consts(lat->seed, 0u, 3u, &ph1);
    ISG_CUDA(launch_init_random(planes_of(lat), ph0, ph1, lat->stream), "init launch");
    lat->t = 0;
    lat->sw_count = 0;
    lat->rec_head = lat->rec_count = 0;
    return ISG_OK;
}

isg_status isg_lattice_init_uniform(isg_lattice *lat, int8_t value)
{
    if (!lat)
        return fail(ISG_ERR_INVALID, "lattice is NULL");
    const bool ok = value == 1 || value == -1 || (value == 0 && lat->model == ISG_BLUME_CAPEL);
    if (!ok)
        return fail(ISG_ERR_INVALID, "value %d is not a spin of this model", value);
    ISG_CUDA(launch_init_uniform(planes_of(lat), value, lat->stream), "init launch");
    lat->t = 0;
    lat->sw_count = 0;
    lat->rec_head = lat->rec_count = 0;
    return ISG_OK;
}

isg_status isg_lattice_set(isg_lattice *lat, const int8_t *host, int64_t t)
{
    if (!lat || !host)
        return fail(ISG_ERR_INVALID, "lattice and host must not be NULL");
    if (t < 0 || t > (int64_t)0xFFFFFFFFLL)
        return fail(ISG_ERR_INVALID, "sweep index %lld out of range", (long long)t);
    const size_t n = (size_t)lat->L * (size_t)lat->L;
    int8_t *d = nullptr;
    ISG_CUDA(dev_malloc_async(&d, n, lat->stream), "staging allocation");
    isg_status s = ISG_OK;
    int32_t bad = 0;
    cudaError_t e = cudaMemcpyAsync(d, host, n, cudaMemcpyHostToDevice, lat->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(lat->d_flag, 0, sizeof(int32_t), lat->stream);
    if (e == cudaSuccess)
        e = launch_pack(planes_of(lat), d, lat->d_flag, lat->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&bad, lat->d_flag, sizeof(int32_t), cudaMemcpyDeviceToHost, lat->stream);
    cudaFreeAsync(d, lat->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(lat->stream);
    if (e != cudaSuccess)
        return cuda_fail(e, "lattice set");
    if (bad)
        s = fail(ISG_ERR_INVALID, "a value is outside the model's spin set (lattice now undefined)");
    lat->t = t;
    lat->rec_head = lat->rec_count = 0;
    return s;
}

isg_status isg_lattice_get_rect(isg_lattice *lat, int64_t y0, int64_t x0, int64_t h, int64_t w,
                                int8_t *out)
{
    if (!lat || !out)
        return fail(ISG_ERR_INVALID, "lattice and out must not be NULL");
    if (y0 < 0 || x0 < 0 || h < 0 || w < 0 || h > lat->L || w > lat->L)
        return fail(ISG_ERR_INVALID, "bad window");
    const size_t n = (size_t)h * (size_t)w;
    if (n == 0)
        return ISG_OK;
    int8_t *d = nullptr;
    ISG_CUDA(dev_malloc_async(&d, n, lat->stream), "staging allocation");
    cudaError_t e = launch_unpack_rect(planes_of(lat), y0 % lat->L, x0 % lat->L, h, w, d, lat->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, d, n, cudaMemcpyDeviceToHost, lat->stream);
    cudaFreeAsync(d, lat->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(lat->stream);
    if (e != cudaSuccess)
        return cuda_fail(e, "lattice get");
    return ISG_OK;
}

isg_status isg_lattice_get(isg_lattice *lat, int8_t *out)
{
    if (!lat)
        return fail(ISG_ERR_INVALID, "lattice is NULL");
    return isg_lattice_get_rect(lat, 0, 0, lat->L, lat->L, out);
}

isg_status isg_lattice_info(const isg_lattice *lat, int64_t *sweep, int64_t *L, int32_t *model,
                            uint64_t *seed)
{
    if (!lat)
        return fail(ISG_ERR_INVALID, "lattice is NULL");
    if (sweep)
        *sweep = lat->t;
    if (L)
        *L = lat->L;
    if (model)
        *model = lat->model;
    if (seed)
        *seed = lat->seed;
    return ISG_OK;
}

isg_status isg_sweep(isg_lattice *lat, int64_t n, const double *betas, double beta_const,
                     int64_t record_every)
{
    if (!betas && !valid_beta(beta_const))
        return fail(ISG_ERR_INVALID, "beta_const = %g is not >= 0", beta_const);
    return sweep_impl(lat, n, betas, beta_const, nullptr, record_every);
}

isg_status isg_sweep_schedule(isg_lattice *lat, int64_t n, const isg_schedule *sched,
                              int64_t record_every)
{
    if (!sched)
        return fail(ISG_ERR_INVALID, "schedule is NULL");
    return sweep_impl(lat, n, nullptr, 0.0, sched, record_every);
}

isg_status isg_half_sweep(isg_lattice *lat, int32_t colour, double beta)
{
    if (!lat)
        return fail(ISG_ERR_INVALID, "lattice is NULL");
    if (colour != 0 && colour != 1)
        return fail(ISG_ERR_INVALID, "colour must be 0 or 1");
    if (!valid_beta(beta))
        return fail(ISG_ERR_INVALID, "beta = %g is not >= 0", beta);
    if (lat->t >= (int64_t)0xFFFFFFFFLL)
        return fail(ISG_ERR_INVALID, "sweep index would reach 2^32");
    return queue_half(lat, colour, beta);
}

isg_status isg_record(isg_lattice *lat)
{
    if (!lat)
        return fail(ISG_ERR_INVALID, "lattice is NULL");
    return push_record(lat);
}

isg_status isg_pending_records(const isg_lattice *lat, int64_t *count)
{
    if (!lat || !count)
        return fail(ISG_ERR_INVALID, "lattice and count must not be NULL");
    *count = lat->rec_count;
    return ISG_OK;
}

isg_status isg_read_records(isg_lattice *lat, isg_obs *out, int64_t max, int64_t *count)
{
    if (count)
        *count = 0;
    if (!lat || !out || !count || max < 0)
        return fail(ISG_ERR_INVALID, "bad arguments");
    ISG_CUDA(cudaStreamSynchronize(lat->stream), "stream sync");
    const int64_t n = max < lat->rec_count ? max : lat->rec_count;
    for (int64_t i = 0; i < n; ++i) {
        const uint8_t *slot = lat->records + (size_t)lat->rec_head * lat->rec_stride;
        isg_status s = copy_record(lat, slot, &out[i]);
        if (s == ISG_ERR_DEVICE_TIMEOUT) {  // a failed record is dropped
            lat->rec_head = (lat->rec_head + 1) % lat->rec_cap;
            lat->rec_count -= 1;
        }
        if (s != ISG_OK)
            return s;
        lat->rec_head = (lat->rec_head + 1) % lat->rec_cap;
        lat->rec_count -= 1;
        *count = i + 1;
    }
    return ISG_OK;
}

isg_status isg_measure(isg_lattice *lat, isg_obs *out)
{
    if (!lat || !out)
        return fail(ISG_ERR_INVALID, "lattice and out must not be NULL");
    uint8_t *slot = lat->records + (size_t)lat->rec_cap * lat->rec_stride;
    isg_status s = queue_record(lat, slot);
    if (s != ISG_OK)
        return s;
    ISG_CUDA(cudaStreamSynchronize(lat->stream), "stream sync");
    return copy_record(lat, slot, out);
}

namespace {

struct FileHeader {
    char magic[8];
    int32_t model;
    int32_t zero;
    int64_t L;
    uint64_t seed;
    double delta;
    int64_t sweep;
    uint64_t plane_bytes;
    uint64_t pad;
};
static_assert(sizeof(FileHeader) == 64, "checkpoint header is 64 bytes");
const char kMagic[8] = {'I', 'S', 'G', 'L', 'A', 'T', '0', '1'};
constexpr size_t kChunk = (size_t)64 << 20;

}  // namespace

isg_status isg_save(isg_lattice *lat, const char *path)
{
    if (!lat || !path)
        return fail(ISG_ERR_INVALID, "lattice and path must not be NULL");
    FileHeader h{};
    memcpy(h.magic, kMagic, 8);
    h.model = lat->model;
    h.L = lat->L;
    h.seed = lat->seed;
    h.delta = lat->delta;
    h.sweep = lat->t;
    h.pad = (uint64_t)lat->sw_count;
    h.plane_bytes = isg_lattice_bytes(lat->model, lat->L);
    ISG_CUDA(cudaStreamSynchronize(lat->stream), "stream sync");
    FILE *f = fopen(path, "wb");
    if (!f)
        return fail(ISG_ERR_INVALID, "cannot open %s for writing", path);
    void *bounce = nullptr;
    cudaError_t e = cudaMallocHost(&bounce, kChunk);
    bool ok = e == cudaSuccess && fwrite(&h, sizeof(h), 1, f) == 1;
    const uint8_t *src = reinterpret_cast<const uint8_t *>(lat->planes);
    for (uint64_t done = 0; ok && done < h.plane_bytes;) {
        const size_t n = (size_t)std::min<uint64_t>(kChunk, h.plane_bytes - done);
        e = cudaMemcpy(bounce, src + done, n, cudaMemcpyDeviceToHost);
        ok = e == cudaSuccess && fwrite(bounce, 1, n, f) == n;
        done += n;
    }
    if (bounce)
        cudaFreeHost(bounce);
    ok = (fclose(f) == 0) && ok;
    if (e != cudaSuccess)
        return cuda_fail(e, "checkpoint copy");
    if (!ok)
        return fail(ISG_ERR_INVALID, "write to %s failed", path);
    return ISG_OK;
}

isg_status isg_load(const char *path, void *stream, int64_t record_capacity, isg_lattice **out)
{
    if (out)
        *out = nullptr;
    if (!path || !out)
        return fail(ISG_ERR_INVALID, "path and out must not be NULL");
    FILE *f = fopen(path, "rb");
    if (!f)
        return fail(ISG_ERR_INVALID, "cannot open %s", path);
    FileHeader h{};
    if (fread(&h, sizeof(h), 1, f) != 1 || memcmp(h.magic, kMagic, 8) != 0 ||
        !valid_L(h.model, h.L) || h.plane_bytes != isg_lattice_bytes(h.model, h.L) ||
        h.sweep < 0 || h.sweep > (int64_t)0xFFFFFFFFLL) {
        fclose(f);
        return fail(ISG_ERR_INVALID, "%s is not a lattice checkpoint", path);
    }
    isg_lattice_desc d{};
    d.model = h.model;
    d.L = h.L;
    d.seed = h.seed;
    d.delta = h.delta;
    d.stream = stream;
    d.record_capacity = record_capacity;
    isg_lattice *lat = nullptr;
    isg_status st = isg_lattice_create(&d, &lat);
    if (st != ISG_OK) {
        fclose(f);
        return st;
    }
    void *bounce = nullptr;
    cudaError_t e = cudaMallocHost(&bounce, kChunk);
    bool ok = e == cudaSuccess;
    uint8_t *dst = reinterpret_cast<uint8_t *>(lat->planes);
    for (uint64_t done = 0; ok && done < h.plane_bytes;) {
        const size_t n = (size_t)std::min<uint64_t>(kChunk, h.plane_bytes - done);
        ok = fread(bounce, 1, n, f) == n;
        if (ok) {
            e = cudaMemcpy(dst + done, bounce, n, cudaMemcpyHostToDevice);
            ok = e == cudaSuccess;
        }
        done += n;
    }
    if (bounce)
        cudaFreeHost(bounce);
    fclose(f);
    if (!ok) {
        isg_lattice_destroy(lat);
        if (e != cudaSuccess)
            return cuda_fail(e, "checkpoint copy");
        return fail(ISG_ERR_INVALID, "%s is truncated", path);
    }
    lat->t = h.sweep;
    lat->sw_count = (int64_t)h.pad;
    *out = lat;
    return ISG_OK;
}

isg_status isg_correlation(isg_lattice *lat, int64_t nr, const int64_t *r, int64_t *out_x,
                           int64_t *out_y)
{
    if (!lat || nr < 0 || (nr > 0 && (!r || !out_x || !out_y)) || nr > (1 << 20))
        return fail(ISG_ERR_INVALID, "bad arguments");
    for (int64_t k = 0; k < nr; ++k)
        if (r[k] < 0 || r[k] >= lat->L)
            return fail(ISG_ERR_INVALID, "distance r[%lld] = %lld outside [0, L)", (long long)k,
                        (long long)r[k]);
    if (nr == 0)
        return ISG_OK;
    int64_t *d_r = nullptr;
    unsigned long long *d_out = nullptr;
    ISG_CUDA(dev_malloc_async(&d_r, sizeof(int64_t) * nr, lat->stream), "staging allocation");
    cudaError_t e = dev_malloc_async(&d_out, sizeof(unsigned long long) * 2 * nr, lat->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_r, r, sizeof(int64_t) * nr, cudaMemcpyHostToDevice, lat->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(d_out, 0, sizeof(unsigned long long) * 2 * nr, lat->stream);
    if (e == cudaSuccess)
        e = launch_correlation(planes_of(lat), (int)nr, d_r, d_out, lat->stream);
    std::vector<int64_t> h((size_t)(2 * nr));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h.data(), d_out, sizeof(int64_t) * 2 * nr, cudaMemcpyDeviceToHost,
                            lat->stream);
    cudaFreeAsync(d_r, lat->stream);
    if (d_out)
        cudaFreeAsync(d_out, lat->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(lat->stream);
    if (e != cudaSuccess)
        return cuda_fail(e, "correlation");
    for (int64_t k = 0; k < nr; ++k) {
        out_x[k] = h[(size_t)k];
        out_y[k] = h[(size_t)(nr + k)];
    }
    return ISG_OK;
}

double isg_xi_integral(int64_t n, const double *r, const double *c, double r_cut)
{
    return xi_integral_fp64(n, r, c, r_cut);
}

double isg_xi2(int64_t n, int64_t L, const int64_t *M, const int32_t *R, const int32_t *C)
{
    return xi2_fp64(n, L, M, R, C);
}

double isg_energy_density(const isg_obs *obs, int64_t L, double delta)
{
    if (!obs || L < 1)
        return NAN;
    return (-(double)obs->B + delta * (double)obs->Q) / ((double)L * (double)L);
}

const char *isg_last_error(void) { return g_err; }

}  // extern "C"

isg_status isg_swendsen_wang(isg_lattice *lat, double beta)
{
    if (!lat)
        return fail(ISG_ERR_INVALID, "lattice is NULL");
    if (!(beta >= 0.0) || !std::isfinite(beta))
        return fail(ISG_ERR_INVALID, "beta must be finite and >= 0 (got %g)", beta);
    if (lat->L > ISG_SW_MAX_L)
        return fail(ISG_ERR_INVALID, "Swendsen-Wang labels need L <= %d (L = %lld)", ISG_SW_MAX_L,
                    (long long)lat->L);
    if (lat->sw_count > (int64_t)0xFFFFFFFFLL)
        return fail(ISG_ERR_INVALID, "Swendsen-Wang iteration count exceeds 2^32");
    const int64_t n = lat->L * lat->L;
    if (!lat->sw_labels)
        ISG_CUDA(dev_malloc(&lat->sw_labels, sizeof(uint32_t) * (size_t)n), "label allocation");
    PhiloxLaunch px, py, pc;
    const uint32_t k = (uint32_t)lat->sw_count;
    philox_launch_consts(lat->seed, k, 4u, &px);
    philox_launch_consts(lat->seed, k, 5u, &py);
    philox_launch_consts(lat->seed, k, 6u, &pc);
    int32_t bad = 0;
    cudaError_t e = cudaMemsetAsync(lat->d_flag, 0, sizeof(int32_t), lat->stream);
    if (e == cudaSuccess)
        e = launch_swendsen_wang(planes_of(lat), lat->sw_labels, px, py, pc, sw_threshold(beta),
                                 lat->d_flag, lat->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&bad, lat->d_flag, sizeof(int32_t), cudaMemcpyDeviceToHost, lat->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(lat->stream);
    if (e != cudaSuccess)
        return cuda_fail(e, "Swendsen-Wang");
    if (bad)
        return fail(ISG_ERR_DEVICE_TIMEOUT, "Swendsen-Wang union-find exceeded its bound (%d)", bad);
    ++lat->sw_count;
    return ISG_OK;
}

isg_status isg_sw_labels(isg_lattice *lat, int32_t *out)
{
    if (!lat || !out)
        return fail(ISG_ERR_INVALID, "lattice and out must not be NULL");
    if (!lat->sw_labels || lat->sw_count == 0)
        return fail(ISG_ERR_INVALID, "no Swendsen-Wang iteration has run on this lattice");
    const int64_t n = lat->L * lat->L;
    ISG_CUDA(cudaMemcpyAsync(out, lat->sw_labels, sizeof(int32_t) * (size_t)n,
                             cudaMemcpyDeviceToHost, lat->stream), "label copy");
    ISG_CUDA(cudaStreamSynchronize(lat->stream), "label copy");
    for (int64_t i = 0; i < n; ++i)
        out[i] &= 0x7FFFFFFF;
    return ISG_OK;
}

isg_status isg_sw_iterations(const isg_lattice *lat, int64_t *count)
{
    if (!lat || !count)
        return fail(ISG_ERR_INVALID, "lattice and count must not be NULL");
    *count = lat->sw_count;
    return ISG_OK;
}
