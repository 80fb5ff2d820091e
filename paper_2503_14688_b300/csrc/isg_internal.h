// isg_internal.h -- types shared by the host side of libisg and its kernels.
// Not part of the public ABI (that is include/isg.h).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace isg {

// Philox4x32-10 multipliers and Weyl key increments (Salmon et al., SC'11).
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

// Launch-uniform part of the per-site Philox evaluation.  For a launch the
// counter words 2 and 3 (sweep index, colour tag) and the key are fixed, so
// half of the first round and a quarter of the second are the same for every
// site; the host folds them here once per launch.
struct PhiloxLaunch {
    uint32_t rk0[10];  // round keys, word 0: key0 + r * W0
    uint32_t rk1[10];  // round keys, word 1: key1 + r * W1
    uint32_t r0_c0;    // round 0: hi(M1 * w2) ^ rk0[0]   (xor hi32(j>>2) per word)
    uint32_t r0_c2x;   // round 0: w3 ^ rk1[0]            (xor hi(M0 * lo32(j>>2)))
    uint32_t r1_c0x;   // round 1: lo(M1 * w2) ^ rk0[1]   (xor hi(M1 * c2'))
};

// Ising acceptance: a site with c anti-aligned neighbours has dE = 8 - 4c;
// c >= 2 always flips, c = 1 flips iff u < thr4, c = 0 iff u < thr8.  A
// threshold equal to 2^32 (always accept) is carried as full = ~0u.
struct IsingThr {
    uint32_t thr4, thr8;
    uint32_t full4, full8;
};

// Blume-Capel acceptance table: entry (g & 7) | p << 3 | n << 4 | (g >> 3) << 5
// | b << 6 for the current value s (n = s != 0, p = s > 0), the proposal bit
// b and g = h + 4 in [0, 8] (h = neighbour sum): the bits the half-sweep
// gathers per site from its bit-planes.  The rule is v < thr31 with
// v = u >> 1 and thr31 = rne(2^31 p) (2^31 = always).
//   full = 1 (every thr31 >= 1): entry = 2 thr31 - 1 (mod 2^32), and the
//            site accepts iff u <= entry -- the same decision, since
//            u = 2 v + b;
//   full = 0 (some move can never be accepted): entry = thr31, accept iff
//            (u >> 1) < entry.
// Entries of no state (p without n, g > 8) are unused.
constexpr int kBcTableSize = 128;
struct BcTable {
    uint32_t thr[kBcTableSize];
    uint32_t full;
};
__host__ __device__ constexpr int bc_entry(int n, int p, int b, int g)
{
    return (g & 7) | (p << 3) | (n << 4) | ((g >> 3) << 5) | (b << 6);
}

// Device-side description of one lattice's spin planes.
//   Ising:        plane(c)    = base + c * L * W          (bit = s > 0)
//   Blume-Capel:  plane(c, 0) = base + (2c) * L * W       (n: s != 0)
//                 plane(c, 1) = base + (2c + 1) * L * W   (p: s > 0, 0 if s = 0)
// W = L / 64 words per row; bit b of word w of row y is the site with
// same-colour row index i = 32 w + b, x = 2 i + ((c ^ y) & 1).
struct Planes {
    uint32_t *base;
    int64_t L;
    int64_t W;
    int32_t model;
};

// Device-side description of one row slab of an L x L lattice (domain
// decomposition): the owned global rows y0 .. y0 + rows - 1.  Each plane
// holds rows + 2 rows of W = L / 64 words (row 0: halo above, global row
// y0 - 1 mod L; rows 1 .. rows: owned; row rows + 1: halo below, global row
// y0 + rows mod L); planes are (rows + 2) W words apart, in the order of
// Planes.
struct SlabPlanes {
    uint32_t *base;
    int64_t L;
    int64_t W;
    int64_t rows;
    int64_t y0;
    int32_t model;
};

// Record layout in device memory: int64 [sweep, B, M, Q] then int32 R[L],
// int32 C[L].
inline size_t record_stride(int64_t L) { return 32 + 8 * (size_t)L; }

// ---- host helpers (isg_host.cpp) ----
void philox_launch_consts(uint64_t seed, uint32_t w2, uint32_t w3, PhiloxLaunch *out);
void ising_thresholds(double beta, IsingThr *out);
void bc_table(double beta, double delta, BcTable *out);
double xi2_fp64(int64_t n, int64_t L, const int64_t *M, const int32_t *R, const int32_t *C);
double xi_integral_fp64(int64_t n, const double *r, const double *c, double r_cut);
// Swendsen-Wang bond threshold rne(2^32 (1 - e^{-2 beta})), 2^32 = always.
uint64_t sw_threshold(double beta);

// ---- fault injection (isg_debug_inject, isg_api.cu) ----
// Every device allocation of the library goes through dev_malloc /
// dev_malloc_async, and every kernel launch of the sweep paths first asks
// injected_launch_failure(): an armed injection makes the k-th such event
// fail -- the allocation reports cudaErrorMemoryAllocation without
// allocating, the launch is skipped and reports cudaErrorLaunchFailure -- so
// the error paths can be tested on the host, with no device fault.
cudaError_t dev_malloc_raw(void **p, size_t bytes);
cudaError_t dev_malloc_async_raw(void **p, size_t bytes, cudaStream_t st);
bool injected_launch_failure();
// An armed ISG_INJECT_WAIT: the k-th streamed record pass under-delivers the
// bytes it announces in one block, so that its bounded waits run out.
bool injected_wait_failure();
// Sweep field of a record whose pass gave up waiting (a bounded wait ran
// out); the host reports ISG_ERR_DEVICE_TIMEOUT when it reads one.
constexpr int64_t kRecordFailed = INT64_MIN;
template <class T>
cudaError_t dev_malloc(T **p, size_t bytes)
{
    return dev_malloc_raw(reinterpret_cast<void **>(p), bytes);
}
template <class T>
cudaError_t dev_malloc_async(T **p, size_t bytes, cudaStream_t st)
{
    return dev_malloc_async_raw(reinterpret_cast<void **>(p), bytes, st);
}

// ---- error reporting shared by the C-ABI files (isg_api.cu) ----
// Stores a printf-style message for isg_last_error() and returns code.
int32_t report_error(int32_t code, const char *fmt, ...);

// ---- kernel launchers (isg_kernels.cu); return the launch error ----
cudaError_t launch_init_random(const Planes &pl, const PhiloxLaunch &ph0, const PhiloxLaunch &ph1,
                               cudaStream_t st);
// One Swendsen-Wang iteration (isg_sw.cu): labels lab (L*L uint32), Philox
// constants of the +x bonds, +y bonds and cluster coins, bond threshold, a
// device error flag raised when a bounded loop runs out.
cudaError_t launch_swendsen_wang(const Planes &pl, uint32_t *lab, const PhiloxLaunch &px,
                                 const PhiloxLaunch &py, const PhiloxLaunch &pc, uint64_t thr,
                                 int32_t *err, cudaStream_t st);
cudaError_t launch_init_uniform(const Planes &pl, int value, cudaStream_t st);
cudaError_t launch_half_sweep(const Planes &pl, int colour, const PhiloxLaunch &ph,
                              const IsingThr &ithr, const BcTable *btab, cudaStream_t st);
cudaError_t launch_measure(const Planes &pl, void *record, int64_t sweep, cudaStream_t st);
// One half-sweep of colour `colour` at sweep t of n lattices of one model
// and side L (planes[i], seeds[i]) in as few launches as the kernel
// parameters allow (kMultiMax lattices each); same results as n single
// launches.
constexpr int kMultiMax = 240;  // lattices per launch: 240 x 100 B of parameters
// Records (zeroed here first) of n lattices of one model and side L after
// sweep `sweep`, in as few launches as the kernel parameters allow.
cudaError_t launch_measure_multi(int model, int64_t L, uint32_t *const *planes, uint8_t *const *recs, int n,
                                 int64_t sweep, cudaStream_t st);
// V_set / H_set: words per thread and band rows (0: chosen from L and n).
cudaError_t launch_half_sweep_multi(int model, int64_t L, uint32_t *const *planes, const uint64_t *seeds,
                                    int n, uint32_t t, int colour, const IsingThr &ithr,
                                    const BcTable *btab, cudaStream_t st, int V_set = 0,
                                    int H_set = 0);
cudaError_t launch_correlation(const Planes &pl, int nr, const int64_t *d_r, unsigned long long *d_out,
                               cudaStream_t st);
cudaError_t launch_pack(const Planes &pl, const int8_t *d_spins, int32_t *d_bad, cudaStream_t st);
// Row slabs (isg_slab.cu): half-sweep of the owned rows with the halo rows of
// the neighbour colour; record (int64 [sweep, B, M, Q], int32 R[rows], int32
// C[L]) of the owned rows, zeroed beforehand; hot start with global keys;
// owned rows <-> rows x L bytes.
cudaError_t launch_half_sweep_slab(const SlabPlanes &sp, int colour, const PhiloxLaunch &ph,
                                   const IsingThr &ithr, const BcTable *btab, cudaStream_t st);
cudaError_t launch_measure_slab(const SlabPlanes &sp, void *record, int64_t sweep, cudaStream_t st);
cudaError_t launch_slab_init_random(const SlabPlanes &sp, const PhiloxLaunch &ph0, const PhiloxLaunch &ph1,
                                    cudaStream_t st);
cudaError_t launch_slab_convert(const SlabPlanes &sp, int8_t *d_spins, int to_planes, int32_t *d_bad,
                                cudaStream_t st);
cudaError_t launch_unpack_rect(const Planes &pl, int64_t y0, int64_t x0, int64_t h, int64_t w,
                               int8_t *d_out, cudaStream_t st);

}  // namespace isg
