// isg_slab.cu -- row slabs of one lattice: the domain decomposition with
// which the paper spreads a single lattice over many GPUs (Introduction;
// Table I, the L = 2^22 runs on 64 GPUs).
//
// A slab owns the global rows y0 .. y0 + rows - 1 of an L x L lattice and
// keeps, per colour plane, one halo row above and one below.  A half-sweep of
// colour c reads only the other colour's plane, so it needs that plane's two
// halo rows -- the edge rows of the neighbouring slabs -- to be current: the
// caller (one process per slab) moves them between slabs before each
// half-sweep (isg_slab_edges on the sender, isg_slab_set_halos on the
// receiver).  Random numbers are keyed by the global site, so the union of
// the slabs evolves bit for bit as the whole lattice does.  The observables
// of a slab are the parts the whole lattice's sums are made of: B over the
// four bonds of each owned colour-1 site (every bond has one colour-1 end;
// the first and last rows reach into the colour-0 halos, which are current
// after a sweep), M, Q, its rows' sums, and its partial column sums.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <limits>
#include <new>

#include "isg.h"
#include "isg_internal.h"

using namespace isg;

struct isg_slab {
    int32_t model = 0;
    int64_t L = 0, W = 0, rows = 0, y0 = 0;
    uint64_t seed = 0;
    double delta = 0.0;
    cudaStream_t stream = nullptr;
    uint32_t *planes = nullptr;
    uint8_t *record = nullptr;
    int32_t *d_flag = nullptr;
    int64_t t = 0;
    double thr_beta = std::numeric_limits<double>::quiet_NaN();
    IsingThr thr_ising{};
    BcTable thr_bc{};
};

namespace {

isg_status slab_cuda(cudaError_t e, const char *what)
{
    cudaGetLastError();
    if (e == cudaErrorMemoryAllocation)
        return report_error(ISG_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver)
        return report_error(ISG_ERR_UNSUPPORTED, "%s: %s", what, cudaGetErrorString(e));
    return report_error(ISG_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define SLAB_CUDA(call, what)                                                                 \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return slab_cuda(e_, what);                                                       \
    } while (0)

SlabPlanes planes_of(const isg_slab *s)
{
    SlabPlanes p;
    p.base = s->planes;
    p.L = s->L;
    p.W = s->W;
    p.rows = s->rows;
    p.y0 = s->y0;
    p.model = s->model;
    return p;
}

int nplanes(int32_t model) { return model == ISG_ISING ? 2 : 4; }

size_t plane_words(const isg_slab *s) { return (size_t)(s->rows + 2) * (size_t)s->W; }

size_t record_bytes(const isg_slab *s) { return 32 + 4 * (size_t)s->rows + 4 * (size_t)s->L; }

// True when p is memory that only the host can address (pageable or pinned
// host memory, as opposed to device or managed memory).
bool host_memory(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return a.type == cudaMemoryTypeUnregistered || a.type == cudaMemoryTypeHost;
}

// Copy one row of colour c's plane(s) (local buffer row `row`) to or from
// `ext` (W words per plane; Blume-Capel: the n words, then the p words).
cudaError_t copy_row(isg_slab *s, int colour, int64_t row, void *ext, bool to_ext)
{
    const size_t rb = 4 * (size_t)s->W;
    const int k0 = s->model == ISG_ISING ? colour : 2 * colour;
    const int nk = s->model == ISG_ISING ? 1 : 2;
    for (int k = 0; k < nk; ++k) {
        uint32_t *plane_row = s->planes + (size_t)(k0 + k) * plane_words(s) + (size_t)row * s->W;
        char *e = static_cast<char *>(ext) + k * rb;
        const cudaError_t err = to_ext ? cudaMemcpyAsync(e, plane_row, rb, cudaMemcpyDefault, s->stream)
                                       : cudaMemcpyAsync(plane_row, e, rb, cudaMemcpyDefault, s->stream);
        if (err != cudaSuccess)
            return err;
    }
    return cudaSuccess;
}

}  // namespace

extern "C" {

size_t isg_slab_edge_bytes(int32_t model, int64_t L)
{
    if (isg_lattice_bytes(model, L) == 0)
        return 0;
    return (size_t)(L / 64) * 4 * (model == ISG_ISING ? 1 : 2);
}

isg_status isg_slab_create(const isg_slab_desc *d, isg_slab **out)
{
    if (out)
        *out = nullptr;
    if (!d || !out)
        return report_error(ISG_ERR_INVALID, "desc and out must not be NULL");
    if (isg_lattice_bytes(d->model, d->L) == 0)
        return report_error(ISG_ERR_INVALID, "invalid model %d or L %lld", d->model, (long long)d->L);
    if (d->rows < 16 || d->rows % 16 != 0 || d->y0 < 0 || d->y0 % 16 != 0 || d->y0 + d->rows > d->L)
        return report_error(ISG_ERR_INVALID,
                            "slab rows %lld at y0 %lld: both must be multiples of 16, rows >= 16, "
                            "y0 + rows <= L = %lld", (long long)d->rows, (long long)d->y0,
                            (long long)d->L);
    if (std::isnan(d->delta) || std::isinf(d->delta))
        return report_error(ISG_ERR_INVALID, "delta must be finite");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return report_error(ISG_ERR_UNSUPPORTED, "no usable CUDA device");
    }
    isg_slab *s = new (std::nothrow) isg_slab();
    if (!s)
        return report_error(ISG_ERR_OOM, "host allocation failed");
    s->model = d->model;
    s->L = d->L;
    s->W = d->L / 64;
    s->rows = d->rows;
    s->y0 = d->y0;
    s->seed = d->seed;
    s->delta = d->model == ISG_BLUME_CAPEL ? d->delta : 0.0;
    s->stream = (cudaStream_t)d->stream;
    cudaError_t e = dev_malloc(&s->planes, 4 * plane_words(s) * nplanes(s->model));
    if (e == cudaSuccess)
        e = dev_malloc(&s->record, record_bytes(s));
    if (e == cudaSuccess)
        e = dev_malloc(&s->d_flag, sizeof(int32_t));
    // halo rows start as zero words until the first isg_slab_set_halos
    if (e == cudaSuccess)
        e = cudaMemsetAsync(s->planes, 0, 4 * plane_words(s) * nplanes(s->model), s->stream);
    if (e != cudaSuccess) {
        const isg_status st = slab_cuda(e, "slab allocation");
        isg_slab_destroy(s);
        return st;
    }
    *out = s;
    return ISG_OK;
}

void isg_slab_destroy(isg_slab *s)
{
    if (!s)
        return;
    cudaStreamSynchronize(s->stream);
    if (s->planes)
        cudaFree(s->planes);
    if (s->record)
        cudaFree(s->record);
    if (s->d_flag)
        cudaFree(s->d_flag);
    delete s;
}

isg_status isg_slab_init_random(isg_slab *s)
{
    if (!s)
        return report_error(ISG_ERR_INVALID, "slab is NULL");
    PhiloxLaunch ph0, ph1;
    philox_launch_consts(s->seed, 0u, 2u, &ph0);
    philox_launch_consts(s->seed, 0u, 3u, &ph1);
    SLAB_CUDA(launch_slab_init_random(planes_of(s), ph0, ph1, s->stream), "slab init");
    s->t = 0;
    return ISG_OK;
}

isg_status isg_slab_set(isg_slab *s, const int8_t *host, int64_t t)
{
    if (!s || !host)
        return report_error(ISG_ERR_INVALID, "slab and host must not be NULL");
    if (t < 0 || t > (int64_t)0xFFFFFFFFLL)
        return report_error(ISG_ERR_INVALID, "sweep index %lld out of range", (long long)t);
    const size_t n = (size_t)s->rows * (size_t)s->L;
    int8_t *d = nullptr;
    SLAB_CUDA(dev_malloc_async(&d, n, s->stream), "staging allocation");
    int32_t bad = 0;
    cudaError_t e = cudaMemcpyAsync(d, host, n, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(s->d_flag, 0, sizeof(int32_t), s->stream);
    if (e == cudaSuccess)
        e = launch_slab_convert(planes_of(s), d, 1, s->d_flag, s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&bad, s->d_flag, sizeof(int32_t), cudaMemcpyDeviceToHost, s->stream);
    cudaFreeAsync(d, s->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess)
        return slab_cuda(e, "slab set");
    s->t = t;
    if (bad)
        return report_error(ISG_ERR_INVALID, "a value is outside the model's spin set (slab now undefined)");
    return ISG_OK;
}

isg_status isg_slab_get(isg_slab *s, int8_t *out)
{
    if (!s || !out)
        return report_error(ISG_ERR_INVALID, "slab and out must not be NULL");
    const size_t n = (size_t)s->rows * (size_t)s->L;
    int8_t *d = nullptr;
    SLAB_CUDA(dev_malloc_async(&d, n, s->stream), "staging allocation");
    cudaError_t e = launch_slab_convert(planes_of(s), d, 0, nullptr, s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, d, n, cudaMemcpyDeviceToHost, s->stream);
    cudaFreeAsync(d, s->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess)
        return slab_cuda(e, "slab get");
    return ISG_OK;
}

isg_status isg_slab_edges(isg_slab *s, int32_t colour, void *first, void *last)
{
    if (!s || !first || !last || (colour != 0 && colour != 1))
        return report_error(ISG_ERR_INVALID, "bad slab, colour or edge buffer");
    SLAB_CUDA(copy_row(s, colour, 1, first, true), "edge row copy");
    SLAB_CUDA(copy_row(s, colour, s->rows, last, true), "edge row copy");
    if (host_memory(first) || host_memory(last))
        SLAB_CUDA(cudaStreamSynchronize(s->stream), "edge row copy");
    return ISG_OK;
}

isg_status isg_slab_set_halos(isg_slab *s, int32_t colour, const void *above, const void *below)
{
    if (!s || !above || !below || (colour != 0 && colour != 1))
        return report_error(ISG_ERR_INVALID, "bad slab, colour or halo buffer");
    SLAB_CUDA(copy_row(s, colour, 0, const_cast<void *>(above), false), "halo row copy");
    SLAB_CUDA(copy_row(s, colour, s->rows + 1, const_cast<void *>(below), false), "halo row copy");
    if (host_memory(above) || host_memory(below))
        SLAB_CUDA(cudaStreamSynchronize(s->stream), "halo row copy");
    return ISG_OK;
}

isg_status isg_slab_half_sweep(isg_slab *s, int32_t colour, double beta)
{
    if (!s || (colour != 0 && colour != 1))
        return report_error(ISG_ERR_INVALID, "bad slab or colour");
    if (std::isnan(beta) || beta < 0.0)
        return report_error(ISG_ERR_INVALID, "beta = %g is not >= 0", beta);
    if (s->t >= (int64_t)0xFFFFFFFFLL)
        return report_error(ISG_ERR_INVALID, "sweep index would reach 2^32");
    PhiloxLaunch ph;
    philox_launch_consts(s->seed, (uint32_t)s->t, (uint32_t)colour, &ph);
    if (!(beta == s->thr_beta)) {
        if (s->model == ISG_ISING)
            ising_thresholds(beta, &s->thr_ising);
        else
            bc_table(beta, s->delta, &s->thr_bc);
        s->thr_beta = beta;
    }
    SLAB_CUDA(launch_half_sweep_slab(planes_of(s), colour, ph, s->thr_ising,
                                     s->model == ISG_ISING ? nullptr : &s->thr_bc, s->stream),
              "slab half-sweep launch");
    if (colour == 1)
        s->t += 1;
    return ISG_OK;
}

isg_status isg_slab_measure(isg_slab *s, isg_obs *out)
{
    if (!s || !out)
        return report_error(ISG_ERR_INVALID, "slab and out must not be NULL");
    SLAB_CUDA(cudaMemsetAsync(s->record, 0, record_bytes(s), s->stream), "record clear");
    SLAB_CUDA(launch_measure_slab(planes_of(s), s->record, s->t, s->stream), "slab measure launch");
    int64_t hdr[4];
    SLAB_CUDA(cudaMemcpyAsync(hdr, s->record, sizeof(hdr), cudaMemcpyDeviceToHost, s->stream),
              "record read");
    if (out->row_sums)
        SLAB_CUDA(cudaMemcpyAsync(out->row_sums, s->record + 32, 4 * (size_t)s->rows,
                                  cudaMemcpyDeviceToHost, s->stream), "row sums read");
    if (out->col_sums)
        SLAB_CUDA(cudaMemcpyAsync(out->col_sums, s->record + 32 + 4 * (size_t)s->rows,
                                  4 * (size_t)s->L, cudaMemcpyDeviceToHost, s->stream),
                  "column sums read");
    SLAB_CUDA(cudaStreamSynchronize(s->stream), "slab measure");
    out->sweep = hdr[0];
    out->B = hdr[1];
    out->M = hdr[2];
    out->Q = hdr[3];
    return ISG_OK;
}

isg_status isg_slab_info(const isg_slab *s, int64_t *sweep, int64_t *L, int64_t *y0, int64_t *rows,
                         int32_t *model)
{
    if (!s)
        return report_error(ISG_ERR_INVALID, "slab is NULL");
    if (sweep)
        *sweep = s->t;
    if (L)
        *L = s->L;
    if (y0)
        *y0 = s->y0;
    if (rows)
        *rows = s->rows;
    if (model)
        *model = s->model;
    return ISG_OK;
}

}  // extern "C"
