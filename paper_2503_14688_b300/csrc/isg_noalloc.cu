// isg_noalloc.cu -- observables of caller-held spin planes, allocating nothing.
//
// isg_measure accumulates B, M, Q and the row/column sums with atomics into a
// record slot that the lattice allocated when it was created.  Some callers
// cannot get device memory at the point where they need a measurement: a
// process whose device memory is entirely handed out by its own pool
// allocator (where a raw cudaMalloc fails or fragments the pool), or a
// latency-sensitive loop that runs many lattices on concurrent streams and
// cannot afford cudaMalloc/cudaFree, which may synchronise the whole device.
// For them, isg_measure_planes_noalloc runs the same measure kernel with its
// accumulation record in a fixed array that lives in this library's device
// image, so the call itself allocates nothing.
//
// The array is sized for L <= ISG_NOALLOC_MAX_L (one record: 32 + 8 L
// bytes, 2 MiB + 32 bytes); every GPU on which the library's kernels are
// loaded holds it until the process exits.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "isg.h"
#include "isg_internal.h"

// One record of the largest accepted lattice: int64 [sweep, B, M, Q], then
// int32 R[L] and C[L].
static __device__ __align__(256) unsigned char isg_noalloc_scratch[32 + 8 * (size_t)ISG_NOALLOC_MAX_L];

namespace {

constexpr int kMaxDevices = 128;
std::mutex g_setup_mutex;
void *g_scratch_addr[kMaxDevices] = {};  // device address of the array, per device

// The device address of isg_noalloc_scratch on the current device.  The
// symbol's name is only a host-side stand-in, so its address is looked up
// once per device (with that device current) and remembered for the life
// of the process; a device reset (cudaDeviceReset, or the primary context
// torn down and created again) would leave the remembered address stale.
isg_status scratch_address(void **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return isg::report_error(ISG_ERR_UNSUPPORTED, "no usable CUDA device (%s)",
                                 cudaGetErrorString(e));
    }
    if (dev < 0 || dev >= kMaxDevices)
        return isg::report_error(ISG_ERR_UNSUPPORTED, "device ordinal %d not supported", dev);
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, isg_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return isg::report_error(ISG_ERR_CUDA, "cudaGetSymbolAddress of the static scratch "
                                     "array failed on device %d: %s", dev,
                                     cudaGetErrorString(e));
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return ISG_OK;
}

}  // namespace

extern "C" isg_status isg_measure_planes_noalloc(int32_t model, int64_t L, const void *d_planes,
                                                 void *stream, int64_t sweep, isg_obs *out)
{
    if (!out || !d_planes)
        return isg::report_error(ISG_ERR_INVALID, "d_planes and out must not be NULL");
    if (model != ISG_ISING && model != ISG_BLUME_CAPEL)
        return isg::report_error(ISG_ERR_INVALID, "unknown model %d", model);
    if (L < 64 || L % 64 != 0)
        return isg::report_error(ISG_ERR_INVALID, "L = %lld must be a multiple of 64, >= 64",
                                 (long long)L);
    if (L > ISG_NOALLOC_MAX_L)
        return isg::report_error(ISG_ERR_INVALID,
                                 "L = %lld exceeds the static scratch limit of this entry point "
                                 "(L <= %lld); use isg_measure for larger lattices",
                                 (long long)L, (long long)ISG_NOALLOC_MAX_L);
    if ((uintptr_t)d_planes % 16 != 0)
        return isg::report_error(ISG_ERR_INVALID, "d_planes must be 16-byte aligned");

    void *scratch = nullptr;
    isg_status st = scratch_address(&scratch);
    if (st != ISG_OK)
        return st;

    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = isg::record_stride(L);
    isg::Planes pl;
    pl.base = (uint32_t *)d_planes;  // read only
    pl.L = L;
    pl.W = L / 64;
    pl.model = model;

    // The array keeps the previous call's sums: clear this call's record first.
    cudaError_t e = cudaMemsetAsync(scratch, 0, bytes, s);
    const bool queued = e == cudaSuccess;  // from here on, work on the array may be in flight
    if (e == cudaSuccess)
        e = isg::launch_measure(pl, scratch, sweep, s);
    int64_t hdr[4] = {0, 0, 0, 0};
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hdr, scratch, sizeof(hdr), cudaMemcpyDeviceToHost, s);
    const unsigned char *sums = (const unsigned char *)scratch + 32;
    if (e == cudaSuccess && out->row_sums)
        e = cudaMemcpyAsync(out->row_sums, sums, sizeof(int32_t) * (size_t)L,
                            cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && out->col_sums)
        e = cudaMemcpyAsync(out->col_sums, sums + sizeof(int32_t) * (size_t)L,
                            sizeof(int32_t) * (size_t)L, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        // No call returns while its work on the shared array may still run:
        // a following call on another stream would otherwise race with it.
        if (queued) {
            cudaStreamSynchronize(s);
            cudaGetLastError();
        }
        return isg::report_error(ISG_ERR_CUDA, "isg_measure_planes_noalloc: %s",
                                 cudaGetErrorString(e));
    }
    if (hdr[0] == isg::kRecordFailed)
        return isg::report_error(ISG_ERR_DEVICE_TIMEOUT,
                                 "isg_measure_planes_noalloc: the record pass ran out of time");
    out->sweep = hdr[0];
    out->B = hdr[1];
    out->M = hdr[2];
    out->Q = hdr[3];
    return ISG_OK;
}
