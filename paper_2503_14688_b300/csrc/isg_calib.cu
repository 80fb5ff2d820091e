// isg_calib.cu -- integer-throughput calibration kernels (libisg_calib.so).
//
// The sweep is bound by integer arithmetic, not by memory, so its roofline
// needs the sustained rate of the instruction classes it uses.  Each kernel
// below runs 8 independent dependency chains per thread of one operation
// class, long enough to amortise launch cost; the host divides operations by
// time.  Kinds:
//   0  32x32 -> 64 multiply (both halves used), plus one xor to fold them
//   1  32x32 -> high 32 bits only (plus one xor)
//   2  32x32 -> low 32 bits (multiply-add)
//   3  three-input xor
//   4  three-input add
//   5  one Philox4x32-10 evaluation (counter increments, keys from params)
#include <cuda_runtime.h>

#include <cstdint>

namespace {

constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;

template <int KIND>
__global__ void k_calib(uint32_t *sink, int iters, uint32_t k0, uint32_t k1)
{
    uint32_t x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
        x[i] = threadIdx.x * 8 + i + blockIdx.x * 977u;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if constexpr (KIND == 0) {
                const uint64_t p = (uint64_t)M0 * x[i];
                x[i] = (uint32_t)(p >> 32) ^ (uint32_t)p;
            } else if constexpr (KIND == 1) {
                x[i] = __umulhi(M0, x[i]) ^ k0;
            } else if constexpr (KIND == 2) {
                x[i] = x[i] * M1 + k1;
            } else if constexpr (KIND == 3) {
                x[i] = x[i] ^ x[(i + 1) & 7] ^ k0;
            } else if constexpr (KIND == 4) {
                x[i] = x[i] + x[(i + 3) & 7] + k1;
            }
        }
        if constexpr (KIND == 5) {
            // two interleaved Philox evaluations per iteration (4 outputs each)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint32_t c0 = x[4 * h] + it, c1 = x[4 * h + 1], c2 = x[4 * h + 2], c3 = x[4 * h + 3];
                uint32_t a = k0, b = k1;
#pragma unroll
                for (int r = 0; r < 10; ++r) {
                    const uint64_t p0 = (uint64_t)M0 * c0, p1 = (uint64_t)M1 * c2;
                    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ a;
                    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ b;
                    c1 = (uint32_t)p1;
                    c3 = (uint32_t)p0;
                    c0 = n0;
                    c2 = n2;
                    a += 0x9E3779B9u;
                    b += 0xBB67AE85u;
                }
                x[4 * h] ^= c0;
                x[4 * h + 1] ^= c1;
                x[4 * h + 2] ^= c2;
                x[4 * h + 3] ^= c3;
            }
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i)
        acc ^= x[i];
    if (acc == 0x12345678u)  // practically never; keeps the chains alive
        sink[blockIdx.x] = acc;
}

}  // namespace

extern "C" {

// Run kind `kind` with grid (blocks x threads) for `iters` iterations and
// return the kernel time in milliseconds (CUDA events), or a negative value
// on error.  sink: device buffer of >= blocks uint32.
float isg_calib_run(int kind, int blocks, int threads, int iters, void *sink)
{
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)
        return -1.0f;
    uint32_t *s = (uint32_t *)sink;
    cudaEventRecord(a);
    switch (kind) {
    case 0: k_calib<0><<<blocks, threads>>>(s, iters, 1u, 2u); break;
    case 1: k_calib<1><<<blocks, threads>>>(s, iters, 1u, 2u); break;
    case 2: k_calib<2><<<blocks, threads>>>(s, iters, 1u, 2u); break;
    case 3: k_calib<3><<<blocks, threads>>>(s, iters, 1u, 2u); break;
    case 4: k_calib<4><<<blocks, threads>>>(s, iters, 1u, 2u); break;
    case 5: k_calib<5><<<blocks, threads>>>(s, iters, 1u, 2u); break;
    default: return -2.0f;
    }
    cudaEventRecord(b);
    if (cudaEventSynchronize(b) != cudaSuccess)
        return -3.0f;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return cudaGetLastError() == cudaSuccess ? ms : -4.0f;
}

}  // extern "C"
