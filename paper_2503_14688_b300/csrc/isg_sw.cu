// isg_sw.cu -- one Swendsen-Wang iteration of the s = +-1 spins on the
// bit-packed lattice (Appendix B: the Blume-Capel equilibrium runs combine
// Swendsen-Wang cluster updates restricted to s = +-1 with Metropolis sweeps;
// for Ising every site takes part).
//
// Definition (shared with the oracle only through its statement):
//   bond (i, j), j the +x (d = 0) or +y (d = 1) neighbour of site
//   i = y L + x, is active iff s_i = s_j != 0 and u < thr, thr =
//   rne(2^32 (1 - e^{-2 beta})) (2^32: always); u = word i & 3 of
//   Philox4x32-10 with counter (lo(i >> 2), hi(i >> 2), k, 4 + d), k the
//   lattice's count of earlier iterations.  A cluster (connected component of
//   active bonds) is labelled by its smallest site index r and flips iff word
//   r & 3 of counter (lo(r >> 2), hi(r >> 2), k, 6) is >= 2^31.
//
// GPU layout: one uint32 label per site (row-major, L <= 2^15 so labels fit
// 30 bits; bit 31 carries a root's coin after pass 3).  Passes:
//   1. k_sw_local_w:  one warp per 32 x 32 tile (four tiles per block).
//                     The warp first loads the tile's spins into shared
//                     memory, then walks its rows in order: a lane computes
//                     each Philox call and shares its words by shuffle; the
//                     row's horizontal runs come from a ballot of its +x
//                     bonds (a site's run starts one past the last unbonded
//                     position to its left); the vertical bonds to the row
//                     above join runs by a lock-free union-find in shared
//                     memory whose links always point from the larger root
//                     to the smaller (atomicMin).  Each label becomes the
//                     global index of its local root.  (Against one block
//                     per tile with all rows at once: 7.0 vs 11.9 ms per
//                     iteration at L = 16384 -- no block barriers, shallow
//                     trees, 64 tiles in flight per SM instead of 4.)
//   2. k_sw_boundary: bonds crossing a tile edge, joined the same way in
//                     global memory.  Every final root is the smallest index
//                     of its component whatever the execution order: the
//                     labels are deterministic.
//   3. k_sw_resolve:  per 4 sites, label := root; a root draws its coin
//                     into bit 31.
//   4. k_sw_flip:     per row and word index, both colours' words (64
//                     consecutive sites): flip the sites whose root has
//                     bit 31 (Ising: s -> -s; Blume-Capel: p ^= 1 where n).
// Every loop is bounded; a bound that runs out raises the lattice's device
// error flag (never expected: root chains strictly decrease).
#include <cuda_runtime.h>

#include <cstdint>

#include "isg_internal.h"
#include "isg_philox.cuh"

namespace isg {
namespace {

constexpr uint32_t kCoinBit = 0x80000000u;
constexpr uint32_t kLabelMask = 0x7FFFFFFFu;
constexpr int kUnionBudget = 1 << 20;
constexpr int kFindBudget = 1 << 24;

// Spin at (x, y) from the colour planes: Ising bit 1 = +1; Blume-Capel
// planes n (s != 0) and p (s > 0).
__device__ __forceinline__ int spin_at(const Planes &pl, int64_t x, int64_t y)
{
    const int c = (int)((x + y) & 1);
    const int64_t k = x >> 1;
    const int64_t LW = pl.L * pl.W;
    const int64_t off = y * pl.W + (k >> 5);
    const uint32_t bit = (uint32_t)(k & 31);
    if (pl.model == 0)
        return ((__ldg(pl.base + (int64_t)c * LW + off) >> bit) & 1u) ? 1 : -1;
    const uint32_t n = (__ldg(pl.base + (int64_t)(2 * c) * LW + off) >> bit) & 1u;
    const uint32_t p = (__ldg(pl.base + (int64_t)(2 * c + 1) * LW + off) >> bit) & 1u;
    return n ? (p ? 1 : -1) : 0;
}

// Root of i by following parent links.  With kHalve, path halving: a node
// is re-pointed to its grandparent.  While links are being made that is
// benign (the store is always an ancestor, and a link it overwrites is
// re-joined by the union loop, which continues from the parent it saw).  It
// is not used while labels are being finalised: a halving store landing
// after a site's root was written would replace the root by an ancestor.
template <bool kHalve>
__device__ __forceinline__ uint32_t find_root(uint32_t *lab, uint32_t i, int &budget)
{
    while (budget-- > 0) {
        const uint32_t p = __ldcg(lab + i);
        if (p == i)
            return i;
        const uint32_t g = __ldcg(lab + p);
        if (kHalve && g != p)
            __stcg(lab + i, g);
        i = g;
    }
    return i;
}

// Join the components of a and b (lock-free: a failed atomicMin means the
// node was re-linked meanwhile; continue from its new parent).
__device__ __forceinline__ bool unite(uint32_t *lab, uint32_t a, uint32_t b)
{
    int find_budget = kFindBudget;
    for (int it = 0; it < kUnionBudget; ++it) {
        a = find_root<true>(lab, a, find_budget);
        b = find_root<true>(lab, b, find_budget);
        if (a == b)
            return find_budget > 0;
        if (a < b) {
            const uint32_t old = atomicMin(lab + b, a);
            if (old == b)
                return find_budget > 0;
            b = old;
        } else {
            const uint32_t old = atomicMin(lab + a, b);
            if (old == a)
                return find_budget > 0;
            a = old;
        }
    }
    return false;
}

// --- pass 1: union-find inside 32 x kTileH tiles, in shared memory -------
// Bonds whose both ends lie in a tile are joined here; local indices
// r * 32 + tx are ordered like the global ones, so each local root is the
// smallest global index of its local component.  Every site's label becomes
// the global index of its local root (roots keep their own index).
constexpr int kTile = 32;   // tile width (one warp per tile row)
#ifndef ISG_SW_TILE_H
#define ISG_SW_TILE_H 32
#endif
constexpr int kTileH = ISG_SW_TILE_H;  // tile height (rows walked by one warp)
static_assert(kTileH >= 2 && kTileH <= 32, "tile height");

__device__ __forceinline__ uint32_t find_local(volatile uint32_t *ls, uint32_t i, int &budget)
{
    while (budget-- > 0) {
        const uint32_t p = ls[i];
        if (p == i)
            return i;
        const uint32_t g = ls[p];
        if (g != p)
            ls[i] = g;
        i = g;
    }
    return i;
}

__device__ __forceinline__ bool unite_local(uint32_t *ls, uint32_t a, uint32_t b)
{
    int budget = kFindBudget;
    volatile uint32_t *v = ls;
    for (int it = 0; it < kUnionBudget; ++it) {
        a = find_local(v, a, budget);
        b = find_local(v, b, budget);
        if (a == b)
            return budget > 0;
        if (a < b) {
            const uint32_t old = atomicMin(ls + b, a);
            if (old == b)
                return budget > 0;
            b = old;
        } else {
            const uint32_t old = atomicMin(ls + a, b);
            if (old == a)
                return budget > 0;
            a = old;
        }
    }
    return false;
}

// One warp per 32 x kTileH tile, rows walked in order (see pass 1 above).
constexpr int kWarpsPerBlock = 4;

__global__ void __launch_bounds__(32 * kWarpsPerBlock) k_sw_local_w(Planes pl, uint32_t *lab,
                                                                   PhiloxLaunch px, PhiloxLaunch py,
                                                                   uint32_t thr, int full,
                                                                   int32_t *err)
{
    __shared__ uint32_t s_all[kWarpsPerBlock][kTileH * kTile];
    __shared__ int8_t s_sp[kWarpsPerBlock][kTileH][kTile];
    const int wid = threadIdx.x >> 5, tx = threadIdx.x & 31;
    const int64_t L = pl.L;
    const int64_t tiles_x = L / kTile, n_tiles = tiles_x * (L / kTileH);
    const int64_t tile = (int64_t)blockIdx.x * kWarpsPerBlock + wid;
    if (tile >= n_tiles)
        return;  // whole warp
    const int64_t bx = tile % tiles_x, by = tile / tiles_x;
    uint32_t *sl = s_all[wid];
    const int64_t x = bx * kTile + tx;
    bool ok = true;
    int s_prev = 0;
    uint32_t uy_prev = 0, hm_prev = 0;
    // all spins of the tile first: independent loads, issued together
#pragma unroll 8
    for (int r = 0; r < kTileH; ++r)
        s_sp[wid][r][tx] = (int8_t)spin_at(pl, x, by * kTileH + r);
    __syncwarp();
    // The bond words of two rows come from one Philox call per lane: lane
    // 16 h + 2 m + d draws for sites 4m .. 4m+3 of row r2 + h, the +x bonds
    // (stream px) for d = 0 and the +y bonds (py) for d = 1.
    const int hsel = tx >> 4, jsel = tx & 15;
    const PhiloxLaunch &pc = (jsel & 1) ? py : px;
    uint32_t w[4];
#pragma unroll 1
    for (int r = 0; r < kTileH; ++r) {
        const int64_t y = by * kTileH + r;
        const int sv = s_sp[wid][r][tx];
        if ((r & 1) == 0) {
            const int64_t g = ((y + hsel) * L + bx * kTile + 4 * (jsel >> 1)) >> 2;
            philox_site4(pc, philox_word_part(pc, (uint32_t)((uint64_t)g >> 32)), (uint32_t)g, w[0],
                         w[1], w[2], w[3]);
        }
        const int src = 16 * (r & 1) + 2 * (tx >> 2);
        uint32_t ux = 0, uy = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t a = __shfl_sync(0xFFFFFFFFu, w[k], src);
            const uint32_t b = __shfl_sync(0xFFFFFFFFu, w[k], src + 1);
            if ((tx & 3) == k) {
                ux = a;
                uy = b;
            }
        }
        const int sr = __shfl_down_sync(0xFFFFFFFFu, sv, 1);
        const bool hb = tx + 1 < kTile && sv != 0 && sr == sv && (full || ux < thr);
        const uint32_t hm = __ballot_sync(0xFFFFFFFFu, hb);
        const uint32_t z = ~hm & ((1u << tx) - 1u);
        const int start = z ? 32 - __clz(z) : 0;
        sl[r * kTile + tx] = (uint32_t)(r * kTile + start);
        __syncwarp();
        if (r > 0) {
            const bool vb = s_prev != 0 && s_prev == sv && (full || uy_prev < thr);
            const uint32_t vm = __ballot_sync(0xFFFFFFFFu, vb);
            const bool dup = tx > 0 && ((vm >> (tx - 1)) & 1u) && ((hm_prev >> (tx - 1)) & 1u) &&
                             ((hm >> (tx - 1)) & 1u);
            if (vb && !dup)
                ok &= unite_local(sl, (uint32_t)((r - 1) * kTile + tx), (uint32_t)(r * kTile + tx));
            __syncwarp();
        }
        s_prev = sv;
        uy_prev = uy;
        hm_prev = hm;
    }
    __syncwarp();
#pragma unroll 1
    for (int r = 0; r < kTileH; ++r) {
        int budget = kFindBudget;
        uint32_t q = (uint32_t)(r * kTile + tx);
        while (budget-- > 0) {
            const uint32_t p = sl[q];
            if (p == q)
                break;
            q = p;
        }
        ok &= budget > 0;
        const int64_t y = by * kTileH + r;
        lab[y * L + x] = (uint32_t)((by * kTileH + (q >> 5)) * L + bx * kTile + (q & 31));
    }
    if (!ok)
        atomicOr(err, 1);
}

// --- pass 2: bonds that cross a tile edge, joined in global memory --------
// Per tile: 32 +x bonds leaving its right column (word 3 of the site's
// Philox call) and 32 +y bonds leaving its bottom row (8 calls of 4 words).
__global__ void k_sw_boundary(Planes pl, uint32_t *lab, PhiloxLaunch px, PhiloxLaunch py,
                              uint32_t thr, int full, int32_t *err)
{
    const int64_t L = pl.L;
    const int64_t tiles_x = L / kTile, tiles_y = L / kTileH;
    constexpr int kPer = kTileH + 8;  // right-column rows + bottom-row groups of 4
    const int64_t items = tiles_x * tiles_y * kPer;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < items;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t tile = t / kPer;
        const int e = (int)(t - tile * kPer);
        const int64_t bx = tile % tiles_x, by = tile / tiles_x;
        bool ok = true;
        if (e < kTileH) {  // right column, row e: bond to the next tile's first column
            const int64_t y = by * kTileH + e, x = bx * kTile + kTile - 1;
            const int64_t xr = x + 1 == L ? 0 : x + 1;
            const int sv = spin_at(pl, x, y);
            if (sv != 0 && spin_at(pl, xr, y) == sv) {
                const int64_t g = (y * L + x) >> 2;
                uint32_t u[4];
                philox_site4(px, philox_word_part(px, (uint32_t)((uint64_t)g >> 32)), (uint32_t)g,
                             u[0], u[1], u[2], u[3]);
                if (full || u[3] < thr)
                    ok = unite(lab, (uint32_t)(y * L + x), (uint32_t)(y * L + xr));
            }
        } else {  // bottom row, sites 4 (e - kTileH) .. +3: bonds to the next tile's first row
            const int64_t y = by * kTileH + kTileH - 1, x0 = bx * kTile + 4 * (e - kTileH);
            const int64_t yd = y + 1 == L ? 0 : y + 1;
            int sv[4], sd[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                sv[j] = spin_at(pl, x0 + j, y);
                sd[j] = spin_at(pl, x0 + j, yd);
            }
            if (((sv[0] != 0) & (sd[0] == sv[0])) | ((sv[1] != 0) & (sd[1] == sv[1])) |
                ((sv[2] != 0) & (sd[2] == sv[2])) | ((sv[3] != 0) & (sd[3] == sv[3]))) {
                const int64_t g = (y * L + x0) >> 2;
                uint32_t u[4];
                philox_site4(py, philox_word_part(py, (uint32_t)((uint64_t)g >> 32)), (uint32_t)g,
                             u[0], u[1], u[2], u[3]);
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (sv[j] != 0 && sd[j] == sv[j] && (full || u[j] < thr))
                        ok &= unite(lab, (uint32_t)(y * L + x0 + j), (uint32_t)(yd * L + x0 + j));
            }
        }
        if (!ok)
            atomicOr(err, 1);
    }
}

// --- pass 3: final labels and coins ---------------------------------------
// Per 4 consecutive sites: each label becomes its root (read-only walk; bit
// 31, set meanwhile on roots by other threads, is masked off); a site that
// is its own root draws its coin (one Philox call per 4 sites, only where a
// root is present) into bit 31.
__global__ void k_sw_resolve(uint32_t *lab, int64_t n, PhiloxLaunch pc, int32_t *err)
{
    const int64_t groups = n / 4;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < groups;
         g += (int64_t)gridDim.x * blockDim.x) {
        uint32_t r[4];
        bool root_any = false, ok = true;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            uint32_t i = (uint32_t)(4 * g + j);
            int budget = kFindBudget;
            while (budget-- > 0) {
                const uint32_t p = __ldcg(lab + i) & kLabelMask;
                if (p == i)
                    break;
                i = p;
            }
            ok &= budget > 0;
            r[j] = i;
            root_any |= i == (uint32_t)(4 * g + j);
        }
        if (root_any) {
            uint32_t u[4];
            philox_site4(pc, philox_word_part(pc, (uint32_t)((uint64_t)g >> 32)), (uint32_t)g, u[0],
                         u[1], u[2], u[3]);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (r[j] == (uint32_t)(4 * g + j) && u[j] >= kCoinBit)
                    r[j] |= kCoinBit;
        }
        reinterpret_cast<uint4 *>(lab)[g] = make_uint4(r[0], r[1], r[2], r[3]);
        if (!ok)
            atomicOr(err, 2);
    }
}

// --- pass 4: flips ---------------------------------------------------------
// Per row y and word index w: the two colour words of index w hold the 64
// sites x = 64 w .. 64 w + 63, read once as 16 uint4 labels.
__global__ void k_sw_flip(Planes pl, const uint32_t *__restrict__ lab)
{
    const int64_t L = pl.L, W = pl.W, LW = L * W;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < LW;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t y = t / W, w = t - y * W;
        const uint4 *row = reinterpret_cast<const uint4 *>(lab + y * L + 64 * w);
        uint32_t m_even = 0, m_odd = 0;  // by x parity: bit b = site x = 64 w + 2 b (+1)
#pragma unroll 4
        for (int q = 0; q < 16; ++q) {
            const uint4 v = row[q];
            const uint32_t c0 = __ldg(lab + (v.x & kLabelMask)) >> 31;
            const uint32_t c1 = __ldg(lab + (v.y & kLabelMask)) >> 31;
            const uint32_t c2 = __ldg(lab + (v.z & kLabelMask)) >> 31;
            const uint32_t c3 = __ldg(lab + (v.w & kLabelMask)) >> 31;
            m_even |= (c0 << (2 * q)) | (c2 << (2 * q + 1));
            m_odd |= (c1 << (2 * q)) | (c3 << (2 * q + 1));
        }
        // colour c holds x parity (c ^ y) & 1
        const int yp = (int)(y & 1);
        const uint32_t m0 = yp ? m_odd : m_even, m1 = yp ? m_even : m_odd;
        if (pl.model == 0) {
            pl.base[t] ^= m0;
            pl.base[LW + t] ^= m1;
        } else {
            pl.base[LW + t] ^= m0 & pl.base[t];
            pl.base[3 * LW + t] ^= m1 & pl.base[2 * LW + t];
        }
    }
}

unsigned grid_for(int64_t items, int threads)
{
    const int64_t want = (items + threads - 1) / threads;
    const int64_t cap = 148LL * 16;
    return (unsigned)(want < 1 ? 1 : (want > cap ? cap : want));
}

}  // namespace

cudaError_t launch_swendsen_wang(const Planes &pl, uint32_t *lab, const PhiloxLaunch &px,
                                 const PhiloxLaunch &py, const PhiloxLaunch &pc, uint64_t thr,
                                 int32_t *err, cudaStream_t st)
{
    const int64_t n = pl.L * pl.L;
    const int th = 256;
    const int full = thr >= (1ull << 32) ? 1 : 0;
    const int64_t tiles = (pl.L / kTile) * (pl.L / kTileH);
    k_sw_local_w<<<(unsigned)((tiles + kWarpsPerBlock - 1) / kWarpsPerBlock), 32 * kWarpsPerBlock, 0,
                   st>>>(pl, lab, px, py, (uint32_t)thr, full, err);
    k_sw_boundary<<<grid_for(tiles * (kTileH + 8), th), th, 0, st>>>(pl, lab, px, py,
                                                                      (uint32_t)thr, full, err);
    k_sw_resolve<<<grid_for(n / 4, th), th, 0, st>>>(lab, n, pc, err);
    k_sw_flip<<<grid_for(pl.L * pl.W, th), th, 0, st>>>(pl, lab);
    return cudaGetLastError();
}

}  // namespace isg
