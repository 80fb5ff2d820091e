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
//   6  compare u >= thr shifted into an accumulator by sub.cc + addc
//   7  funnel shift by one (shf.l)
//   8  shift left by one, or-ed with a top bit (plain C)
//   9  two-input add
//  10  byte permute (prmt)
//  11  compare accumulated in plain C: acc + acc + (u >= thr)
//  12  compare as the borrow bit from logic ops, shifted in by a funnel shift
//  13  the Ising word update of the sweep (32 sites, no memory traffic)
//  14  the sweep's Philox calls alone (folded first rounds, 4 sites each)
// Together with per-pipe instruction counters (a profiler run of the same
// command) these show which execution pipe each operation class uses.
#include <cuda_runtime.h>

#include <cstdint>

#include "isg_sweep_core.cuh"

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
            } else if constexpr (KIND == 6) {
                x[i] = isg::shift_in_not_below(x[i], x[(i + 1) & 7], k0);
            } else if constexpr (KIND == 7) {
                x[i] = __funnelshift_l(x[(i + 1) & 7], x[i], 1);
            } else if constexpr (KIND == 8) {
                x[i] = (x[i] << 1) | (x[(i + 1) & 7] >> 31);
            } else if constexpr (KIND == 9) {
                x[i] = x[i] + x[(i + 1) & 7];
            } else if constexpr (KIND == 10) {
                x[i] = __byte_perm(x[i], x[(i + 1) & 7], 0x6541u);
            } else if constexpr (KIND == 11) {
                x[i] = x[i] + x[i] + (uint32_t)(x[(i + 1) & 7] >= k0);
            } else if constexpr (KIND == 12) {
                const uint32_t u = x[(i + 1) & 7], d = u - k0;
                const uint32_t borrow = (~u & k0) | (~(u ^ k0) & d);
                x[i] = __funnelshift_l(borrow, x[i], 1);
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

// Kinds 13..18: the sweep's own per-word arithmetic on register data.
//   13  Ising word update (32 sites), 48 registers (the sweep kernel's budget)
//   14  the sweep's Philox calls alone, 8 unrolled per word, 48 registers
//   15  as 14, calls not unrolled
//   16  as 14, four calls per word step
//   17  as 14, up to 128 registers
//   18  unfolded Philox4x32-10 (20 multiplies), 8 unrolled, 48 registers
template <int KIND>
__device__ __forceinline__ void calib_word_body(uint32_t *sink, int iters, uint32_t k0, uint32_t k1)
{
    const isg::PhiloxLaunch pc = isg::philox_consts_device(0x2503146880000000ull ^ k0, 7u, 1u);
    isg::IsingThr thr;
    thr.thr4 = 0x2BEDD0D9u ^ k1;
    thr.thr8 = 0x0784B2A1u ^ k1;
    thr.full4 = thr.full8 = 0u;
    uint32_t t = threadIdx.x * 0x9E3779B9u, up = blockIdx.x * 0x85EBCA6Bu, dn = t ^ 0x5bd1e995u;
    uint32_t same = up + 0x27d4eb2fu;
    uint64_t q = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) * 8;
    for (int it = 0; it < iters; ++it) {
        if constexpr (KIND == 13) {
            const uint32_t side = isg::side_word(same, up, it & 1);
            const uint32_t n = isg::ising_word_update(t, up, dn, same, side, q, pc, thr);
            up = dn;
            dn = same;
            same = t;
            t = n;
        } else if constexpr (KIND == 18) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                uint32_t c0 = (uint32_t)q + i, c1 = (uint32_t)(q >> 32), c2 = 7u, c3 = 1u;
#pragma unroll
                for (int r = 0; r < 10; ++r) {
                    const uint64_t p0 = (uint64_t)M0 * c0, p1 = (uint64_t)M1 * c2;
                    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ pc.rk0[r];
                    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ pc.rk1[r];
                    c1 = (uint32_t)p1;
                    c3 = (uint32_t)p0;
                    c0 = n0;
                    c2 = n2;
                }
                t ^= c0 ^ c1;
                up ^= c2 ^ c3;
            }
        } else {
            const isg::PhiloxWordPart wp = isg::philox_word_part(pc, (uint32_t)(q >> 32));
            constexpr int kStep = KIND == 16 ? 2 : 1;
            if constexpr (KIND == 15) {
#pragma unroll 1
                for (int i = 0; i < 8; ++i) {
                    uint32_t r0, r1, r2, r3;
                    isg::philox_site4(pc, wp, (uint32_t)q + i, r0, r1, r2, r3);
                    t ^= r0 ^ r1;
                    up ^= r2 ^ r3;
                }
            } else {
#pragma unroll
                for (int i = 0; i < 8 / kStep; ++i) {
                    uint32_t r0, r1, r2, r3;
                    isg::philox_site4(pc, wp, (uint32_t)q + i, r0, r1, r2, r3);
                    t ^= r0 ^ r1;
                    up ^= r2 ^ r3;
                }
            }
        }
        q += 8ull * 148 * 2048;
    }
    if ((t ^ up ^ dn ^ same) == 0x12345678u)
        sink[blockIdx.x] = t;
}

template <int KIND>
__global__ void __launch_bounds__(256, 5) k_calib_word(uint32_t *sink, int iters, uint32_t k0, uint32_t k1)
{
    calib_word_body<KIND>(sink, iters, k0, k1);
}

template <int KIND>
__global__ void __launch_bounds__(256, 2) k_calib_word_wide(uint32_t *sink, int iters, uint32_t k0,
                                                            uint32_t k1)
{
    calib_word_body<KIND>(sink, iters, k0, k1);
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
    case 6: k_calib<6><<<blocks, threads>>>(s, iters, 0x80000000u, 2u); break;
    case 7: k_calib<7><<<blocks, threads>>>(s, iters, 1u, 2u); break;
    case 8: k_calib<8><<<blocks, threads>>>(s, iters, 1u, 2u); break;
    case 9: k_calib<9><<<blocks, threads>>>(s, iters, 1u, 2u); break;
    case 10: k_calib<10><<<blocks, threads>>>(s, iters, 1u, 2u); break;
    case 11: k_calib<11><<<blocks, threads>>>(s, iters, 0x80000000u, 2u); break;
    case 12: k_calib<12><<<blocks, threads>>>(s, iters, 0x80000000u, 2u); break;
    case 13: k_calib_word<13><<<blocks, threads>>>(s, iters, 1u, 2u); break;
    case 14: k_calib_word<14><<<blocks, threads>>>(s, iters, 1u, 2u); break;
    case 15: k_calib_word<15><<<blocks, threads>>>(s, iters, 1u, 2u); break;
    case 16: k_calib_word<16><<<blocks, threads>>>(s, iters, 1u, 2u); break;
    case 17: k_calib_word_wide<14><<<blocks, threads>>>(s, iters, 1u, 2u); break;
    case 18: k_calib_word<18><<<blocks, threads>>>(s, iters, 1u, 2u); break;
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
