// isg_kernels.cu -- sm_103a kernels of libisg.
//
//   k_init_random    hot start ("Thermal protocols": T = infinity start)
//   k_init_uniform   cold start
//   k_ising_half     Ising half-sweep of one colour (Introduction: Metropolis
//                    with checkerboard decomposition and multispin coding)
//   k_bc_half        Blume-Capel half-sweep of one colour (Eq. (1))
//   k_measure        B, M, Q and row/column sums (Eqs. (2)-(3); Appendix B)
//   k_pack / k_unpack_rect   byte-per-site <-> bit-plane conversion
//
// Layout (see Planes in isg_internal.h): one bit per site and colour plane,
// 32 same-colour sites of one row per 32-bit word.  For a target word at
// (row y, word w) of colour c the four neighbours of its 32 sites are, in
// the other colour's plane: row y-1 word w (up), row y+1 word w (down), row
// y word w (same), and row y word w shifted by one site toward the left when
// (c ^ y) & 1 == 0 or toward the right otherwise (the "side" word).
//
// Every kernel is integer-only: no tensor cores, nothing here is a
// contraction.  The sweep kernels are bound by the integer issue rate of the
// Philox evaluations (one per four sites) and the threshold compares.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "isg_bulk.cuh"
#include "isg_internal.h"
#include "isg_philox.cuh"
#include "isg_sweep_core.cuh"

namespace isg {

namespace {

constexpr int kSweepThreads = 128;
constexpr int kSweepMinBlocks = 6;   // 80 registers: 24 warps per SM, four words interleaved
constexpr int kBcThreads = 256;
constexpr int kBcMinBlocks = 2;      // 128 registers: 16 warps per SM, two words interleaved
constexpr int kMeasureThreads = 256;

template <int V>
struct Words {
    uint32_t v[V];
};

template <int V>
__device__ __forceinline__ Words<V> load_words(const uint32_t *__restrict__ p)
{
    Words<V> r;
    if constexpr (V == 4) {
        const uint4 q = __ldg(reinterpret_cast<const uint4 *>(p));
        r.v[0] = q.x;
        r.v[1] = q.y;
        r.v[2] = q.z;
        r.v[3] = q.w;
    } else if constexpr (V == 2) {
        const uint2 q = __ldg(reinterpret_cast<const uint2 *>(p));
        r.v[0] = q.x;
        r.v[1] = q.y;
    } else {
        r.v[0] = __ldg(p);
    }
    return r;
}

template <int V>
__device__ __forceinline__ Words<V> load_words_rw(const uint32_t *p)
{
    Words<V> r;
    if constexpr (V == 4) {
        const uint4 q = *reinterpret_cast<const uint4 *>(p);
        r.v[0] = q.x;
        r.v[1] = q.y;
        r.v[2] = q.z;
        r.v[3] = q.w;
    } else if constexpr (V == 2) {
        const uint2 q = *reinterpret_cast<const uint2 *>(p);
        r.v[0] = q.x;
        r.v[1] = q.y;
    } else {
        r.v[0] = *p;
    }
    return r;
}

template <int V>
__device__ __forceinline__ void store_words(uint32_t *p, const Words<V> &r)
{
    if constexpr (V == 4) {
        *reinterpret_cast<uint4 *>(p) = make_uint4(r.v[0], r.v[1], r.v[2], r.v[3]);
    } else if constexpr (V == 2) {
        *reinterpret_cast<uint2 *>(p) = make_uint2(r.v[0], r.v[1]);
    } else {
        *p = r.v[0];
    }
}

// The side neighbours of the V target words: for parity 0 each site's
// other horizontal neighbour is one site to the left (bit b-1, or bit 31 of
// the previous word), for parity 1 one site to the right.
template <int V>
__device__ __forceinline__ Words<V> side_words(const Words<V> &S, uint32_t edge, int parity)
{
    Words<V> X;
    if (parity == 0) {
#pragma unroll
        for (int v = 0; v < V; ++v)
            X.v[v] = (S.v[v] << 1) | ((v > 0 ? S.v[v - 1] : edge) >> 31);
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v)
            X.v[v] = (S.v[v] >> 1) | ((v < V - 1 ? S.v[v + 1] : edge) << 31);
    }
    return X;
}

// ---------------------------------------------------------------------------
// Hot start: site random word from the counter (lo(q), hi(q), 0, c | 2).
// One thread per word of either colour plane.
// ---------------------------------------------------------------------------
__global__ void k_init_random(Planes pl, PhiloxLaunch ph0, PhiloxLaunch ph1)
{
    const int64_t words = pl.L * pl.W;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= 2 * words)
        return;
    const int c = gid >= words;
    const int64_t wi = c ? gid - words : gid;  // y * W + w
    const int64_t y = wi / pl.W, w = wi - y * pl.W;
    const PhiloxLaunch &pc = c ? ph1 : ph0;
    const uint64_t q0 = (uint64_t)y * (uint64_t)(pl.L / 8) + 8u * (uint64_t)w;
    const PhiloxWordPart wp = philox_word_part(pc, (uint32_t)(q0 >> 32));
    uint32_t bits_n = 0, bits_p = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        uint32_t r[4];
        philox_site4(pc, wp, (uint32_t)q0 + i, r[0], r[1], r[2], r[3]);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int b = 4 * i + k;
            if (pl.model == 0) {
                bits_p |= (r[k] >> 31) << b;
            } else {
                const uint32_t v = (uint32_t)(((uint64_t)r[k] * 3u) >> 32);  // 0,1,2 -> s = v-1
                bits_n |= (uint32_t)(v != 1) << b;
                bits_p |= (uint32_t)(v == 2) << b;
            }
        }
    }
    const int64_t LW = pl.L * pl.W;
    if (pl.model == 0) {
        pl.base[(int64_t)c * LW + wi] = bits_p;
    } else {
        pl.base[(int64_t)(2 * c) * LW + wi] = bits_n;
        pl.base[(int64_t)(2 * c + 1) * LW + wi] = bits_p;
    }
}

__global__ void k_init_uniform(Planes pl, int value)
{
    const int64_t n = (pl.model == 0 ? 2 : 4) * pl.L * pl.W;
    const int64_t LW = pl.L * pl.W;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t word;
        if (pl.model == 0) {
            word = value > 0 ? ~0u : 0u;
        } else {
            const bool is_p = (i / LW) & 1;
            word = is_p ? (value > 0 ? ~0u : 0u) : (value != 0 ? ~0u : 0u);
        }
        pl.base[i] = word;
    }
}

// ---------------------------------------------------------------------------
// Ising half-sweep.  A thread owns V consecutive words (32 V sites) of a
// band of H rows of the target colour and walks down the band, keeping the
// up/same/down neighbour words in registers (each neighbour word is loaded
// once per band plus two halo rows).
// ---------------------------------------------------------------------------
//
// kWrap = true: the whole periodic lattice (Li = L rows, rows wrap).
// kWrap = false: a row slab of a larger lattice (domain decomposition): Li
// rows starting at global row yg0, whose neighbour plane has one halo row
// above row 0 and one below row Li - 1 (the neighbouring slabs' edge rows);
// parity and random keys follow the global row.  Lx is the lattice side
// (the row width in sites), which sets the Philox counter's row stride.
template <int V, bool kWrap = true>
__device__ __forceinline__ void ising_half_band(uint32_t g, uint32_t *__restrict__ tgt,
                                                const uint32_t *__restrict__ nbr, uint32_t Li,
                                                uint32_t Wi, int colour, int H, const PhiloxLaunch &pc,
                                                const IsingThr &thr, uint32_t yg0 = 0)
{
    // threads enumerate (row band, V-word group) pairs, groups fastest, so
    // every block is full whatever the row width; rows and words fit 32 bits
    const uint32_t tpr = Wi / V;
    const uint32_t band = g / tpr;
    const uint32_t w0 = (g - band * tpr) * V;
    const uint32_t y0 = band * (uint32_t)H;
    if (y0 >= Li)
        return;
    const uint32_t y1 = y0 + H < Li ? y0 + H : Li;
    // L / 8 Philox counters per row (the periodic lattice has Li = L rows)
    const uint64_t qrow = kWrap ? (uint64_t)(Li / 8) : (uint64_t)(Wi * 8);
    // edge words of the two parities (periodic in the row)
    const uint32_t e_left = w0 == 0 ? Wi - 1 : w0 - 1;
    const uint32_t e_right = w0 + V == Wi ? 0 : w0 + V;

    const uint32_t *nrow = nbr + (uint64_t)y0 * Wi;
    uint32_t *trow = tgt + (uint64_t)y0 * Wi;
    Words<V> U = load_words<V>(kWrap ? nbr + (uint64_t)(y0 == 0 ? Li - 1 : y0 - 1) * Wi + w0
                                     : nrow - Wi + w0);
    Words<V> S = load_words<V>(nrow + w0);
    for (uint32_t y = y0; y < y1; ++y) {
        const uint32_t *ndown = (kWrap && y + 1 == Li) ? nbr : nrow + Wi;
        const Words<V> D = load_words<V>(ndown + w0);
        const uint32_t yg = kWrap ? y : y + yg0;
        const int parity = (colour ^ (int)yg) & 1;
        const uint32_t edge = __ldg(nrow + (parity == 0 ? e_left : e_right));
        const Words<V> X = side_words<V>(S, edge, parity);
        Words<V> T = load_words_rw<V>(trow + w0);
        const uint64_t qy = (uint64_t)yg * qrow + 8u * w0;
        ising_words_update<V>(T.v, U.v, D.v, S.v, X.v, qy, pc, thr);  // the V words interleaved
        store_words<V>(trow + w0, T);
        U = S;
        S = D;
        nrow += Wi;
        trow += Wi;
    }
}

template <int V>
__global__ void __launch_bounds__(kSweepThreads, V == 4 ? kSweepMinBlocks : 8)
    k_ising_half(uint32_t *__restrict__ tgt, const uint32_t *__restrict__ nbr, int64_t L,
                 int64_t W, int colour, int H, PhiloxLaunch pc, IsingThr thr)
{
    ising_half_band<V>(blockIdx.x * blockDim.x + threadIdx.x, tgt, nbr, (uint32_t)L, (uint32_t)W,
                       colour, H, pc, thr);
}

// Many lattices of one side L in one launch (the ensemble's replicas too
// large for shared memory): lattice blockIdx.y of the launch, its planes and
// Philox constants in the kernel parameters, so both stay uniform per block.
struct MultiArgs {
    PhiloxLaunch pc[kMultiMax];
    uint32_t *planes[kMultiMax];
};

template <int V>
__global__ void __launch_bounds__(kSweepThreads, V == 4 ? kSweepMinBlocks : 8)
    k_ising_half_multi(int64_t L, int colour, int H, IsingThr thr, const __grid_constant__ MultiArgs a)
{
    const int r = blockIdx.y;
    const uint32_t Li = (uint32_t)L, Wi = (uint32_t)(L / 64);
    const uint64_t LW = (uint64_t)Li * Wi;
    ising_half_band<V>(blockIdx.x * blockDim.x + threadIdx.x, a.planes[r] + colour * LW,
                       a.planes[r] + (1 - colour) * LW, Li, Wi, colour, H, a.pc[r], thr);
}

// ---------------------------------------------------------------------------
// Blume-Capel half-sweep.  Two bit-planes per colour: n (s != 0) and p (s > 0).
// The neighbour field h + 4 = #(+1 neighbours) + #(neighbours != -1) is a
// bit-sliced sum of eight indicator words (four bits g0..g3); the six
// planes g0..g3, p, n are transposed into one index byte per site, and each
// site looks its threshold up in the table of BcTable, indexed by that byte
// and its proposal bit, held in shared memory.
// ---------------------------------------------------------------------------
// kWrap and yg0 as for ising_half_band; L is the number of rows swept.
template <int V, bool kFull, bool kWrap = true>
__device__ __forceinline__ void bc_half_band(int64_t g, uint32_t *__restrict__ tn_plane,
                                             uint32_t *__restrict__ tp_plane,
                                             const uint32_t *__restrict__ nn_plane,
                                             const uint32_t *__restrict__ np_plane, int64_t L,
                                             int64_t W, int colour, int H, const PhiloxLaunch &pc,
                                             const uint32_t *s_thr, uint32_t yg0 = 0)
{
    // rows and words fit 32 bits; row pointers advance by one row per step
    const uint32_t Li = (uint32_t)L, Wi = (uint32_t)W;
    const uint32_t tpr = Wi / V;
    const uint32_t band = (uint32_t)(g / tpr);
    const uint32_t w0 = ((uint32_t)g - band * tpr) * V;
    const uint32_t y0 = band * (uint32_t)H;
    if (y0 >= Li)
        return;
    const uint32_t y1 = y0 + H < Li ? y0 + H : Li;
    // L / 8 Philox counters per row (the periodic lattice has Li = L rows)
    const uint64_t qrow = kWrap ? (uint64_t)(Li / 8) : (uint64_t)(Wi * 8);
    const uint32_t e_left = w0 == 0 ? Wi - 1 : w0 - 1;
    const uint32_t e_right = w0 + V == Wi ? 0 : w0 + V;
    const int64_t dpn = np_plane - nn_plane, dtp = tp_plane - tn_plane;  // occupancy -> sign plane

    const uint32_t *nrow = nn_plane + (uint64_t)y0 * Wi;
    const uint32_t *nup = kWrap ? nn_plane + (uint64_t)(y0 == 0 ? Li - 1 : y0 - 1) * Wi : nrow - Wi;
    Words<V> Un = load_words<V>(nup + w0);
    Words<V> Up = load_words<V>(nup + dpn + w0);
    uint32_t *trow = tn_plane + (uint64_t)y0 * Wi;
    Words<V> Sn = load_words<V>(nrow + w0);
    Words<V> Sp = load_words<V>(nrow + dpn + w0);
    for (uint32_t y = y0; y < y1; ++y) {
        const uint32_t *ndown = (kWrap && y + 1 == Li) ? nn_plane : nrow + Wi;
        const Words<V> Dn = load_words<V>(ndown + w0);
        const Words<V> Dp = load_words<V>(ndown + dpn + w0);
        const uint32_t yg = kWrap ? y : y + yg0;
        const int parity = (colour ^ (int)yg) & 1;
        const uint32_t *edge = nrow + (parity == 0 ? e_left : e_right);
        const Words<V> Xn = side_words<V>(Sn, __ldg(edge), parity);
        const Words<V> Xp = side_words<V>(Sp, __ldg(edge + dpn), parity);
        Words<V> Tn = load_words_rw<V>(trow + w0);
        Words<V> Tp = load_words_rw<V>(trow + dtp + w0);
        if constexpr (V == 2) {
            // the two words interleaved (bc_word_update2)
            const uint32_t nbn[2][4] = {{Un.v[0], Dn.v[0], Sn.v[0], Xn.v[0]},
                                        {Un.v[1], Dn.v[1], Sn.v[1], Xn.v[1]}};
            const uint32_t nbp[2][4] = {{Up.v[0], Dp.v[0], Sp.v[0], Xp.v[0]},
                                        {Up.v[1], Dp.v[1], Sp.v[1], Xp.v[1]}};
            uint32_t nn[2] = {Tn.v[0], Tn.v[1]}, pp[2] = {Tp.v[0], Tp.v[1]};
            const uint64_t q0 = (uint64_t)yg * qrow + 8u * (uint64_t)w0;
            bc_word_update2<kFull>(nn, pp, nbn, nbp, q0, q0 + 8u, pc, s_thr);
            Tn.v[0] = nn[0];
            Tn.v[1] = nn[1];
            Tp.v[0] = pp[0];
            Tp.v[1] = pp[1];
        } else {
            const uint32_t nbn[4] = {Un.v[0], Dn.v[0], Sn.v[0], Xn.v[0]};
            const uint32_t nbp[4] = {Up.v[0], Dp.v[0], Sp.v[0], Xp.v[0]};
            const uint64_t q0 = (uint64_t)yg * qrow + 8u * (uint64_t)w0;
            bc_word_update<kFull>(Tn.v[0], Tp.v[0], nbn, nbp, q0, pc, s_thr);
        }
        store_words<V>(trow + w0, Tn);
        store_words<V>(trow + dtp + w0, Tp);
        Un = Sn;
        Up = Sp;
        Sn = Dn;
        Sp = Dp;
        nrow += Wi;
        trow += Wi;
    }
}

template <int V, bool kFull>
__global__ void __launch_bounds__(kBcThreads, kBcMinBlocks)
    k_bc_half(uint32_t *__restrict__ tn_plane, uint32_t *__restrict__ tp_plane,
              const uint32_t *__restrict__ nn_plane, const uint32_t *__restrict__ np_plane,
              int64_t L, int64_t W, int colour, int H, PhiloxLaunch pc, BcTable tab)
{
    __shared__ uint32_t s_thr[kBcTableSize];
    for (int i = threadIdx.x; i < kBcTableSize; i += blockDim.x)
        s_thr[i] = tab.thr[i];
    __syncthreads();
    bc_half_band<V, kFull>((int64_t)blockIdx.x * blockDim.x + threadIdx.x, tn_plane, tp_plane,
                           nn_plane, np_plane, L, W, colour, H, pc, s_thr);
}

// Blume-Capel lattices of one side L in one launch (see k_ising_half_multi).
template <int V, bool kFull>
__global__ void __launch_bounds__(kBcThreads, kBcMinBlocks)
    k_bc_half_multi(int64_t L, int colour, int H, BcTable tab, const __grid_constant__ MultiArgs a)
{
    __shared__ uint32_t s_thr[kBcTableSize];
    for (int i = threadIdx.x; i < kBcTableSize; i += blockDim.x)
        s_thr[i] = tab.thr[i];
    __syncthreads();
    const int r = blockIdx.y;
    const int64_t W = L / 64, LW = L * W;
    uint32_t *tn = a.planes[r] + (int64_t)(2 * colour) * LW;
    const uint32_t *nn = a.planes[r] + (int64_t)(2 * (1 - colour)) * LW;
    bc_half_band<V, kFull>((int64_t)blockIdx.x * blockDim.x + threadIdx.x, tn, tn + LW, nn, nn + LW,
                           L, W, colour, H, a.pc[r], s_thr);
}

// ---------------------------------------------------------------------------
// Observables.  A thread owns one word column w of both colours over a band
// of H rows (a multiple of 16), walked in groups of four rows whose loads are
// issued together.  Bonds: every bond joins a colour-0 and a colour-1 site,
// so B = sum over colour-1 sites of s * (sum of its four colour-0
// neighbours).  Row sums: the 32 lanes of a warp share the row; one warp
// reduction per row into a shared-memory array for the band, then one global
// atomic per row and block.  Column sums: per bit position, carry-save
// (Harley-Seal) counters of the +1 (and for Blume-Capel the -1) sites, split
// by column parity; every 16 rows the carry of weight 16 ripples into a
// bit-sliced high counter.  At the end of the band each column's count is
// read out and added atomically.
// ---------------------------------------------------------------------------
constexpr int kMeasureBand = 8192;  // rows per band at most
// blocks per SM the launch bounds ask for, per model
constexpr int kMeasureBlocksIsing = 3, kMeasureBlocksBc = 3;  // 80 registers each
constexpr int kHighBits = 10;       // high counter: multiples of 16 up to 16 * 1023

struct ColumnCounter {
    uint32_t ones, twos, fours, eights;
    uint32_t high[kHighBits];
    uint32_t fa, ea;  // pending carries of weight 4 and 8 inside a 16-row block
};

__device__ __forceinline__ void csa(uint32_t &acc, uint32_t b, uint32_t c, uint32_t &carry)
{
    const uint32_t u = acc ^ b;
    carry = (acc & b) | (u & c);
    acc = u ^ c;
}

// Add the four words of one 4-row group; g = group index within the 16-row
// block (0..3).
__device__ __forceinline__ void cc_add4(ColumnCounter &k, uint32_t w0, uint32_t w1, uint32_t w2,
                                        uint32_t w3, int g)
{
    uint32_t ta, tb, f;
    csa(k.ones, w0, w1, ta);
    csa(k.ones, w2, w3, tb);
    csa(k.twos, ta, tb, f);
    if ((g & 1) == 0) {
        k.fa = f;
        return;
    }
    uint32_t e;
    csa(k.fours, k.fa, f, e);
    if (g == 1) {
        k.ea = e;
        return;
    }
    uint32_t sixteen;
    csa(k.eights, k.ea, e, sixteen);
#pragma unroll
    for (int l = 0; l < kHighBits; ++l) {
        const uint32_t c = k.high[l] & sixteen;
        k.high[l] ^= sixteen;
        sixteen = c;
    }
}

__device__ __forceinline__ int cc_get(const ColumnCounter &k, int bit)
{
    int v = (int)((k.ones >> bit) & 1u) + 2 * (int)((k.twos >> bit) & 1u) +
            4 * (int)((k.fours >> bit) & 1u) + 8 * (int)((k.eights >> bit) & 1u);
    int h = 0;
#pragma unroll
    for (int l = 0; l < kHighBits; ++l)
        h |= (int)((k.high[l] >> bit) & 1u) << l;
    return v + 16 * h;
}

__device__ __forceinline__ void cc_zero(ColumnCounter &k)
{
    k.ones = k.twos = k.fours = k.eights = k.fa = k.ea = 0;
#pragma unroll
    for (int l = 0; l < kHighBits; ++l)
        k.high[l] = 0;
}

// Blume-Capel column counter of s + 1 in {0, 1, 2}: per row a word of the
// zero sites (weight 1) and a word of the +1 sites (weight 2), so that one
// counter per column parity replaces separate +1 and -1 counters.  Levels
// of weight 1 .. 32 in carry-save form; a carry of weight 64 leaves every
// 16 rows into the bit-sliced high counter (a band's count is at most
// 2 x 8192 = 64 x 256).
constexpr int kHighBitsW = 9;
struct WColumnCounter {
    uint32_t l1, l2, l4, l8, l16, l32;
    uint32_t high[kHighBitsW];
    uint32_t e16, f32;  // pending carries of weight 16 and 32 inside a 16-row block
};

// Add one 4-row group: zero-site words z (weight 1) and +1-site words p
// (weight 2); g = group index within the 16-row block (0..3).
__device__ __forceinline__ void wcc_add4(WColumnCounter &k, const uint32_t (&z)[4], const uint32_t (&p)[4], int g)
{
    uint32_t a, b, c1, c2, c3, d1, e;
    csa(k.l1, z[0], z[1], a);
    csa(k.l1, z[2], z[3], b);
    csa(k.l2, a, b, c1);
    csa(k.l2, p[0], p[1], c2);
    csa(k.l2, p[2], p[3], c3);
    csa(k.l4, c1, c2, d1);
    const uint32_t d2 = k.l4 & c3;
    k.l4 ^= c3;
    csa(k.l8, d1, d2, e);
    if ((g & 1) == 0) {
        k.e16 = e;
        return;
    }
    uint32_t f;
    csa(k.l16, k.e16, e, f);
    if (g == 1) {
        k.f32 = f;
        return;
    }
    uint32_t c64;
    csa(k.l32, k.f32, f, c64);
#pragma unroll
    for (int l = 0; l < kHighBitsW; ++l) {
        const uint32_t c = k.high[l] & c64;
        k.high[l] ^= c64;
        c64 = c;
    }
}

__device__ __forceinline__ int wcc_get(const WColumnCounter &k, int bit)
{
    int v = (int)((k.l1 >> bit) & 1u) + 2 * (int)((k.l2 >> bit) & 1u) + 4 * (int)((k.l4 >> bit) & 1u) +
            8 * (int)((k.l8 >> bit) & 1u) + 16 * (int)((k.l16 >> bit) & 1u) + 32 * (int)((k.l32 >> bit) & 1u);
    int h = 0;
#pragma unroll
    for (int l = 0; l < kHighBitsW; ++l)
        h |= (int)((k.high[l] >> bit) & 1u) << l;
    return v + 64 * h;
}

__device__ __forceinline__ void wcc_zero(WColumnCounter &k)
{
    k.l1 = k.l2 = k.l4 = k.l8 = k.l16 = k.l32 = k.e16 = k.f32 = 0;
#pragma unroll
    for (int l = 0; l < kHighBitsW; ++l)
        k.high[l] = 0;
}

// The running state of one thread's walk down its word column: the
// accumulators, the colour-0 rows above (U) and beside (S) the current
// colour-1 row, and the column counters of the even / odd columns (Ising:
// +1 sites; Blume-Capel: s + 1).
struct MeasureState {
    int accB, accM, accQ;
    uint32_t Up, Sp, Un, Sn;
    ColumnCounter ce_p, co_p;   // Ising
    WColumnCounter ce_w, co_w;  // Blume-Capel
};

template <int MODEL>
__device__ __forceinline__ void measure_init(MeasureState &m)
{
    m.accB = m.accM = m.accQ = 0;
    m.Up = m.Sp = m.Un = m.Sn = 0;
    if (MODEL == 0) {
        cc_zero(m.ce_p);
        cc_zero(m.co_p);
    } else {
        wcc_zero(m.ce_w);
        wcc_zero(m.co_w);
    }
}

// Row values in raw form: a thread's part of a row sum is, for Ising,
// 2 raw - 64 with raw = the +1 sites among its 64 (raw = 32 for a lane with
// no column), and for Blume-Capel raw - 64 with raw = 64 + (+1 sites) -
// (-1 sites) (64 for a lane with no column): always in [0, 128], so that
// two rows' warp sums fit the 16-bit halves of one word.
template <int MODEL>
__device__ __forceinline__ int raw_to_row(int raw_sum, int lanes)
{
    return MODEL == 0 ? 2 * raw_sum - 64 * lanes : raw_sum - 64 * lanes;
}

// One group of four rows (row r has parity r & 1): per row the colour-1
// target words Tp (Tn), the colour-0 row below Dp (Dn) and the colour-0
// side word Ep (En) of the row itself.  Bonds, magnetisation (raw) and
// occupancy go to the accumulators, each row's raw value to raw[r] for the
// caller's row reduction, and the column counters advance (g = the group's
// index within its 16-row block).
template <int MODEL>
__device__ __forceinline__ void measure_group(MeasureState &m, const uint32_t (&Tp)[4],
                                              const uint32_t (&Dp)[4], const uint32_t (&Ep)[4],
                                              const uint32_t (&Tn)[4], const uint32_t (&Dn)[4],
                                              const uint32_t (&En)[4], bool active, int (&raw)[4], int g)
{
    uint32_t evp[4], odp[4], evz[4], odz[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const bool odd = r & 1;
        const uint32_t Xp = odd ? (m.Sp << 1) | (Ep[r] >> 31) : (m.Sp >> 1) | (Ep[r] << 31);
        if (MODEL == 0) {
            const uint32_t T = Tp[r];
            const int anti = __popc(T ^ m.Up) + __popc(T ^ Dp[r]) + __popc(T ^ m.Sp) + __popc(T ^ Xp);
            m.accB += 128 - 2 * anti;
            raw[r] = active ? __popc(T) + __popc(m.Sp) : 32;
            evp[r] = odd ? T : m.Sp;
            odp[r] = odd ? m.Sp : T;
        } else {
            const uint32_t Xn = odd ? (m.Sn << 1) | (En[r] >> 31) : (m.Sn >> 1) | (En[r] << 31);
            const uint32_t Tn_ = Tn[r], Tp_ = Tp[r];
            const uint32_t nb[4] = {m.Un, Dn[r], m.Sn, Xn}, pb[4] = {m.Up, Dp[r], m.Sp, Xp};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t both = Tn_ & nb[k];
                m.accB += __popc(both) - 2 * __popc(both & (Tp_ ^ pb[k]));
            }
            const uint32_t plus1 = Tn_ & Tp_, plus0 = m.Sn & m.Sp;
            // (+1) - (-1) = 2 (+1) - (occupied); the occupied count is Q's
            const int occ = __popc(Tn_) + __popc(m.Sn);
            m.accQ += occ;
            raw[r] = active ? 64 + 2 * (__popc(plus1) + __popc(plus0)) - occ : 64;
            evp[r] = odd ? plus1 : plus0;
            odp[r] = odd ? plus0 : plus1;
            evz[r] = odd ? ~Tn_ : ~m.Sn;  // zero sites
            odz[r] = odd ? ~m.Sn : ~Tn_;
            m.Un = m.Sn;
            m.Sn = Dn[r];
        }
        m.accM += raw[r];
        m.Up = m.Sp;
        m.Sp = Dp[r];
    }
    if (MODEL == 0) {
        cc_add4(m.ce_p, evp[0], evp[1], evp[2], evp[3], g);
        cc_add4(m.co_p, odp[0], odp[1], odp[2], odp[3], g);
    } else {
        wcc_add4(m.ce_w, evz, evp, g);
        wcc_add4(m.co_w, odz, odp, g);
    }
}

// End of a band of `rows` rows: B, M, Q summed per warp into the record
// header, and every column's count (one site per row of the band) added to
// C.  Every lane of the warp takes part.
template <int MODEL>
__device__ __forceinline__ void measure_finish(MeasureState &m, bool active, int rows, int64_t wc,
                                               int64_t *__restrict__ rec_hdr, int32_t *__restrict__ C)
{
    m.accM = raw_to_row<MODEL>(m.accM, rows);  // raw over the band's rows -> its part of M
    if (!active)
        m.accB = m.accM = m.accQ = 0;
    if (MODEL == 0)
        m.accQ = active ? 64 * rows : 0;
    const int accB = __reduce_add_sync(0xFFFFFFFFu, m.accB);
    const int accM = __reduce_add_sync(0xFFFFFFFFu, m.accM);
    const int accQ = __reduce_add_sync(0xFFFFFFFFu, m.accQ);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(reinterpret_cast<unsigned long long *>(rec_hdr + 1), (unsigned long long)(int64_t)accB);
        atomicAdd(reinterpret_cast<unsigned long long *>(rec_hdr + 2), (unsigned long long)(int64_t)accM);
        atomicAdd(reinterpret_cast<unsigned long long *>(rec_hdr + 3), (unsigned long long)(int64_t)accQ);
    }
    if (active) {
#pragma unroll 4
        for (int b = 0; b < 32; ++b) {
            const int64_t xe = 2 * (32 * wc + b);
            int ve, vo;
            if (MODEL == 0) {
                ve = 2 * cc_get(m.ce_p, b) - rows;
                vo = 2 * cc_get(m.co_p, b) - rows;
            } else {  // the counters hold the sum of s + 1
                ve = wcc_get(m.ce_w, b) - rows;
                vo = wcc_get(m.co_w, b) - rows;
            }
            if (ve)
                atomicAdd(&C[xe], ve);
            if (vo)
                atomicAdd(&C[xe + 1], vo);
        }
    }
}

// base: row 0 of plane 0; L rows of W words per plane, planes LW words
// apart.  kWrap = true: the periodic lattice (L rows).  kWrap = false: a row
// slab whose planes have a halo row above row 0 and below row L - 1, which
// stand in for the wrap (its first global row must be a multiple of 16).
template <int MODEL, bool kWrap = true>
__device__ __forceinline__ void measure_band(const uint32_t *base, int64_t L, int64_t W, int64_t LW,
                                             int H, int64_t *__restrict__ rec_hdr,
                                             int32_t *__restrict__ R, int32_t *__restrict__ C,
                                             int64_t sweep, int32_t *s_row)
{
    const int64_t y0 = (int64_t)blockIdx.y * H;
    const int rows = (int)((y0 + H < L ? y0 + H : L) - y0);  // a multiple of 16
    for (int i = threadIdx.x; i < rows; i += blockDim.x)
        s_row[i] = 0;
    __syncthreads();
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0)
        rec_hdr[0] = sweep;

    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = w < W;
    const int64_t wc = active ? w : 0;
    // plane pointers: colour-0 / colour-1 sign planes (and occupancy planes)
    const uint32_t *p0 = MODEL == 0 ? base : base + LW;
    const uint32_t *p1 = MODEL == 0 ? base + LW : base + 3 * LW;
    const uint32_t *n0 = base, *n1 = base + 2 * LW;  // Blume-Capel only
    const int64_t wl = wc == 0 ? W - 1 : wc - 1, wr = wc + 1 == W ? 0 : wc + 1;

    MeasureState m;
    measure_init<MODEL>(m);
    const int64_t yup = (kWrap && y0 == 0) ? L - 1 : y0 - 1;
    if (active) {
        m.Up = __ldg(p0 + yup * W + wc);
        m.Sp = __ldg(p0 + y0 * W + wc);
        if (MODEL == 1) {
            m.Un = __ldg(n0 + yup * W + wc);
            m.Sn = __ldg(n0 + y0 * W + wc);
        }
    }
    // Bands start at multiples of 16 rows and groups at multiples of 4, so row
    // yg + r has parity r & 1 (known at compile time) and the only periodic
    // wrap is the down neighbour of row L - 1.  Column pointers; the edge word
    // of the colour-1 site is to the left on odd rows, to the right on even.
    const uint32_t *p0c = p0 + wc, *p1c = p1 + wc;
    const uint32_t *n0c = n0 + wc, *n1c = n1 + wc;
    const int64_t off_l = wl - wc, off_r = wr - wc;
    const uint32_t *t1 = p1c + y0 * W, *t0 = p0c + y0 * W;  // the band's first row
    // The band is walked in 4-row groups, all loads of a group (Ising: of
    // two groups) issued before any is used.
    struct Group {
        uint32_t Tp[4], Dp[4], Ep[4], Tn[4], Dn[4], En[4];
    };
    const int ngroups = rows / 4;  // even: a band has a multiple of 16 rows
    auto load = [&](Group &G, int gg) {
        const uint32_t *g1 = t1 + (int64_t)(4 * gg) * W, *g0p = t0 + (int64_t)(4 * gg) * W;
        const bool last = kWrap && y0 + 4 * gg + 4 == L;  // row + 3 wraps to row 0
        if (active) {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const uint32_t *down = (r == 3 && last) ? p0c : g0p + (r + 1) * W;
                const uint32_t *edge = g0p + r * W + ((r & 1) ? off_l : off_r);
                G.Tp[r] = __ldg(g1 + r * W);
                G.Dp[r] = __ldg(down);
                G.Ep[r] = __ldg(edge);
                if (MODEL == 1) {
                    const int64_t d_nb = n0c - p0c;  // occupancy planes: fixed offset
                    G.Tn[r] = __ldg(g1 + r * W + (n1c - p1c));
                    G.Dn[r] = __ldg(down + d_nb);
                    G.En[r] = __ldg(edge + d_nb);
                }
            }
        } else {
#pragma unroll
            for (int r = 0; r < 4; ++r)
                G.Tp[r] = G.Dp[r] = G.Ep[r] = G.Tn[r] = G.Dn[r] = G.En[r] = 0;
        }
    };
    auto process = [&](const Group &G, int gg) {
        int raw[4];
        measure_group<MODEL>(m, G.Tp, G.Dp, G.Ep, G.Tn, G.Dn, G.En, active, raw, gg & 3);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int rs = __reduce_add_sync(0xFFFFFFFFu, raw[r]);
            if ((threadIdx.x & 31) == 0)
                atomicAdd(&s_row[4 * gg + r], raw_to_row<MODEL>(rs, 32));
        }
    };
    Group A, B;
    if (MODEL == 0) {
        // two groups' loads go out together, then both are processed (a
        // prefetch of the next pair while processing was 17% slower)
#pragma unroll 1
        for (int gg = 0; gg < ngroups; gg += 2) {
            load(A, gg);
            load(B, gg + 1);
            process(A, gg);
            process(B, gg + 1);
        }
    } else {
        // Blume-Capel loads twice the words per group: one group at a
        // time, so that the kernel stays within its registers
#pragma unroll 1
        for (int gg = 0; gg < ngroups; ++gg) {
            load(A, gg);
            process(A, gg);
        }
    }
    measure_finish<MODEL>(m, active, rows, wc, rec_hdr, C);
    __syncthreads();
    for (int i = threadIdx.x; i < rows; i += blockDim.x)
        if (s_row[i])
            atomicAdd(&R[y0 + i], s_row[i]);
}

template <int MODEL>
__global__ void __launch_bounds__(kMeasureThreads, MODEL == 0 ? kMeasureBlocksIsing : kMeasureBlocksBc)
    k_measure(Planes pl, int H, int64_t *__restrict__ rec_hdr, int32_t *__restrict__ R,
              int32_t *__restrict__ C, int64_t sweep)
{
    __shared__ int32_t s_row[kMeasureBand];
    measure_band<MODEL>(pl.base, pl.L, pl.W, pl.L * pl.W, H, rec_hdr, R, C, sweep, s_row);
}

// ---------------------------------------------------------------------------
// The record pass with its rows streamed into shared memory by the copy
// engine (k_measure_stream): the walk and arithmetic of k_measure
// (measure_group / measure_finish), for lattices whose rows split into
// whole segments of kStreamSeg words (L a multiple of 16384).  A block has
// one consumer thread per word of its segment (8 warps) and one producer
// warp, whose lane 0 copies 4-row groups into a ring of shared-memory
// stages, completing on the stage's `full` mbarrier: per plane one tiled
// copy of a 4-row box through a tensor map of the planes (away from the
// row ends and the periodic wrap), else one 1D bulk copy per row.  Per row
// a stage holds the colour-1 target segment and the colour-0 row below it
// with kStreamHalo words on each side: the side neighbours of the
// segment's edge words, taken from the row's other end at the periodic
// wrap.  Consumer warps release a stage through its `empty` mbarrier; each
// leaves the warp sums of the group's four raw row values in shared memory,
// two rows to a word (16-bit halves), and the producer adds them to R
// before it refills the stage.  Every wait is bounded (kStreamWaitNs); one
// that runs out marks the record failed (sweep field INT64_MIN, read by the
// host as ISG_ERR_DEVICE_TIMEOUT), and the producer waits (bounded) for its
// copies in flight before the block returns.
// ---------------------------------------------------------------------------
constexpr int kStreamSeg = 256;   // words per segment: one consumer thread each
constexpr int kStreamHalo = 4;    // 16 bytes, the bulk-copy granule
constexpr int kStreamRowD = kStreamSeg + 2 * kStreamHalo;
constexpr int kStreamThreads = kStreamSeg + 32;
constexpr uint64_t kStreamWaitNs = 2000000000ull;

template <int MODEL>
struct StreamShape {
    static constexpr int kPlanes = MODEL == 0 ? 1 : 2;   // sign (and occupancy) planes per colour
    static constexpr int kStages = MODEL == 0 ? 8 : 4;  // 66.6 KB of stages either way
    // per plane: the 4 colour-1 rows, then the 4 colour-0 rows below them
    // (the layouts of the two tiled boxes; every block 128-byte aligned)
    static constexpr int kPlaneWords = 4 * (kStreamSeg + kStreamRowD);
    static constexpr int kStageWords = kPlanes * kPlaneWords;
    static constexpr uint32_t kStageBytes = 4u * kStageWords;
    // stages, then kStages full and kStages empty barriers, then per stage and
    // consumer warp its two packed row-pair sums
    static constexpr size_t kSmem = (size_t)kStages * kStageBytes + 16 * kStages + 64 * kStages;
    // word offsets in a stage: colour-1 plane q of row r; colour-0 plane q
    // of the row below row r (halo words included)
    static __device__ __forceinline__ int t_off(int r, int q) { return q * kPlaneWords + r * kStreamSeg; }
    static __device__ __forceinline__ int d_off(int r, int q)
    {
        return q * kPlaneWords + 4 * kStreamSeg + r * kStreamRowD;
    }
};

__device__ __forceinline__ void mark_record_failed(int64_t *rec_hdr)
{
    atomicExch(reinterpret_cast<unsigned long long *>(rec_hdr), (unsigned long long)INT64_MIN);
}

// The producer (one thread): copies of group gg go to stage gg % kStages;
// c0[q] / c1[q]: colour-0 / colour-1 plane q (0: sign, 1: occupancy).
// tmT / tmD (used when tmap): tensor maps of all planes as (W / 2) x L x
// planes 8-byte elements with boxes of 128 x 4 x 1 (colour-1 rows) and
// 132 x 4 x 1 (colour-0 rows with halos).  tx_extra (0 except under
// ISG_INJECT_WAIT): bytes announced for the first group on top of those
// copied, so that its waits run out.
template <int MODEL>
__device__ void stream_produce(uint32_t sbase, uint32_t full0, uint32_t empty0, const uint32_t *s_part,
                               const uint32_t *const (&c0)[2], const uint32_t *const (&c1)[2], int64_t L,
                               int64_t W, int64_t y0, int64_t seg0, int ngroups, int32_t *__restrict__ R,
                               int64_t *rec_hdr, uint32_t tx_extra, const CUtensorMap *tmT,
                               const CUtensorMap *tmD, bool tmap)
{
    using S = StreamShape<MODEL>;
    // plane index in the tensor maps: colour-0 / colour-1 sign (and occupancy)
    const int z0[2] = {MODEL == 0 ? 0 : 1, 0}, z1[2] = {MODEL == 0 ? 1 : 3, 2};
    const bool inner = seg0 >= kStreamHalo && seg0 + kStreamSeg + kStreamHalo <= W;
    const int64_t left = seg0 >= kStreamHalo ? seg0 - kStreamHalo : W - kStreamHalo;
    const int64_t right = seg0 + kStreamSeg < W ? seg0 + kStreamSeg : 0;
    int issued = 0;
    bool ok = true;
    for (int gg = 0; gg < ngroups + S::kStages; ++gg) {
        const int s = gg % S::kStages;
        if (gg >= S::kStages) {
            const int done = gg - S::kStages;  // the group the consumers release from stage s
            if (done >= ngroups)
                break;
            if (!mbar_wait(empty0 + 8u * s, (uint32_t)((done / S::kStages) & 1), kStreamWaitNs)) {
                ok = false;
                break;
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint32_t tot = 0;  // halves stay below 2^16: 8 warps x 32 lanes x 128
#pragma unroll
                for (int w = 0; w < kStreamSeg / 32; ++w)
                    tot += s_part[2 * (s * (kStreamSeg / 32) + w) + h];
                const int64_t y = y0 + 4 * done + 2 * h;
                const int v0 = raw_to_row<MODEL>((int)(tot & 0xFFFFu), kStreamSeg);
                const int v1 = raw_to_row<MODEL>((int)(tot >> 16), kStreamSeg);
                if (v0)
                    atomicAdd(&R[y], v0);
                if (v1)
                    atomicAdd(&R[y + 1], v1);
            }
        }
        if (gg < ngroups) {
            const uint32_t full = full0 + 8u * s;
            const uint32_t st = sbase + (uint32_t)s * S::kStageBytes;
            mbar_expect_tx(full, S::kStageBytes + (gg == 0 ? tx_extra : 0u));
            const int64_t yg = y0 + 4 * gg;
            if (tmap && inner && yg + 4 < L) {
#pragma unroll
                for (int q = 0; q < S::kPlanes; ++q) {
                    tensor_load_3d(st + 4u * S::t_off(0, q), tmT, (int)(seg0 / 2), (int)yg, z1[q], full);
                    tensor_load_3d(st + 4u * S::d_off(0, q), tmD, (int)(seg0 / 2) - kStreamHalo / 2, (int)yg + 1,
                                   z0[q], full);
                }
                issued = gg + 1;
                continue;
            }
#pragma unroll 1
            for (int r = 0; r < 4; ++r) {
                const int64_t y = y0 + 4 * gg + r, yd = y + 1 == L ? 0 : y + 1;
#pragma unroll
                for (int q = 0; q < S::kPlanes; ++q) {
                    bulk_load(st + 4u * S::t_off(r, q), c1[q] + y * W + seg0, 4u * kStreamSeg, full);
                    const uint32_t d = st + 4u * S::d_off(r, q);
                    const uint32_t *row = c0[q] + yd * W;
                    if (inner) {
                        bulk_load(d, row + seg0 - kStreamHalo, 4u * kStreamRowD, full);
                    } else {
                        bulk_load(d, row + left, 4u * kStreamHalo, full);
                        bulk_load(d + 4u * kStreamHalo, row + seg0, 4u * kStreamSeg, full);
                        bulk_load(d + 4u * (kStreamHalo + kStreamSeg), row + right, 4u * kStreamHalo, full);
                    }
                }
            }
            issued = gg + 1;
        }
    }
    if (!ok) {
        mark_record_failed(rec_hdr);
        // the latest group issued into each stage must have landed before
        // the block's shared memory goes away
        for (int s = 0; s < S::kStages && s < issued; ++s) {
            const int last = s + S::kStages * ((issued - 1 - s) / S::kStages);
            mbar_wait(full0 + 8u * s, (uint32_t)((last / S::kStages) & 1), kStreamWaitNs);
        }
    }
}

template <int MODEL>
__global__ void __launch_bounds__(kStreamThreads, 3)  // 3 blocks per SM: 71 / 72 registers
    k_measure_stream(Planes pl, int H, int64_t *__restrict__ rec_hdr, int32_t *__restrict__ R,
                     int32_t *__restrict__ C, int64_t sweep, uint32_t tx_extra,
                     const __grid_constant__ CUtensorMap tmT, const __grid_constant__ CUtensorMap tmD, int tmap)
{
    using S = StreamShape<MODEL>;
    extern __shared__ __align__(128) uint32_t smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + S::kStages * S::kStageWords);
    uint32_t *s_part = reinterpret_cast<uint32_t *>(bars + 2 * S::kStages);
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + S::kStages);
    const int64_t L = pl.L, W = pl.W, LW = L * W;
    const int64_t y0 = (int64_t)blockIdx.y * H;
    const int rows = (int)((y0 + H < L ? y0 + H : L) - y0);  // a multiple of 16
    const int ngroups = rows / 4;
    const int64_t seg0 = (int64_t)blockIdx.x * kStreamSeg;
    const uint32_t *const c0[2] = {MODEL == 0 ? pl.base : pl.base + LW, pl.base};
    const uint32_t *const c1[2] = {MODEL == 0 ? pl.base + LW : pl.base + 3 * LW, pl.base + 2 * LW};
    if (threadIdx.x == 0) {
        for (int s = 0; s < S::kStages; ++s) {
            mbar_init(full0 + 8u * s, 1);
            mbar_init(empty0 + 8u * s, kStreamSeg / 32);
        }
        mbar_fence_init();
        if (blockIdx.x == 0 && blockIdx.y == 0)  // the slot is zeroed; a failure mark stays
            atomicCAS(reinterpret_cast<unsigned long long *>(rec_hdr), 0ull, (unsigned long long)sweep);
    }
    __syncthreads();
    if (threadIdx.x >= kStreamSeg) {
        if (threadIdx.x == kStreamSeg)
            stream_produce<MODEL>(smem_u32(smem), full0, empty0, s_part, c0, c1, L, W, y0, seg0, ngroups, R,
                                  rec_hdr, blockIdx.x == 0 && blockIdx.y == 0 ? tx_extra : 0u, &tmT, &tmD,
                                  tmap != 0);
        return;
    }
    const int t = threadIdx.x;
    const int64_t wc = seg0 + t;
    const int64_t wr = wc + 1 == W ? 0 : wc + 1;
    const int64_t yup = y0 == 0 ? L - 1 : y0 - 1;
    MeasureState m;
    measure_init<MODEL>(m);
    m.Up = __ldg(c0[0] + yup * W + wc);
    m.Sp = __ldg(c0[0] + y0 * W + wc);
    // side word of the next group's first row (even: to the right)
    uint32_t Ecp = __ldg(c0[0] + y0 * W + wr), Ecn = 0;
    if (MODEL == 1) {
        m.Un = __ldg(c0[1] + yup * W + wc);
        m.Sn = __ldg(c0[1] + y0 * W + wc);
        Ecn = __ldg(c0[1] + y0 * W + wr);
    }
    const int warp = t >> 5, lane = t & 31;
    // 16 rows (four groups, one 16-row block of the column counters) per
    // iteration: a band has a multiple of 16 rows, and kStages is a
    // multiple of 4, so the four groups take consecutive stages of one phase
#pragma unroll 1
    for (int gb = 0; gb < ngroups; gb += 4) {
        const uint32_t parity = (uint32_t)((gb / S::kStages) & 1);
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const int s = gb % S::kStages + g;
            // the warp gives up as one (its lanes meet in warp reductions below)
            const bool landed = mbar_wait(full0 + 8u * s, parity, kStreamWaitNs);
            if (__any_sync(0xFFFFFFFFu, !landed)) {
                if (lane == 0)
                    mark_record_failed(rec_hdr);
                return;
            }
            const uint32_t *st = smem + s * S::kStageWords;
            uint32_t Tp[4], Dp[4], Ep[4], Tn[4], Dn[4], En[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                Tp[r] = st[S::t_off(r, 0) + t];
                Dp[r] = st[S::d_off(r, 0) + kStreamHalo + t];
                // the row's own colour-0 words are the previous row's "below"
                Ep[r] = r == 0 ? Ecp : st[S::d_off(r - 1, 0) + kStreamHalo + t + ((r & 1) ? -1 : 1)];
                if (MODEL == 1) {
                    Tn[r] = st[S::t_off(r, 1) + t];
                    Dn[r] = st[S::d_off(r, 1) + kStreamHalo + t];
                    En[r] = r == 0 ? Ecn : st[S::d_off(r - 1, 1) + kStreamHalo + t + ((r & 1) ? -1 : 1)];
                } else {
                    Tn[r] = Dn[r] = En[r] = 0;
                }
            }
            Ecp = st[S::d_off(3, 0) + kStreamHalo + t + 1];
            if (MODEL == 1)
                Ecn = st[S::d_off(3, 1) + kStreamHalo + t + 1];
            int raw[4];
            measure_group<MODEL>(m, Tp, Dp, Ep, Tn, Dn, En, true, raw, g);
            const uint32_t p01 = __reduce_add_sync(0xFFFFFFFFu, (uint32_t)raw[0] | ((uint32_t)raw[1] << 16));
            const uint32_t p23 = __reduce_add_sync(0xFFFFFFFFu, (uint32_t)raw[2] | ((uint32_t)raw[3] << 16));
            if (lane == 0) {
                *reinterpret_cast<uint2 *>(s_part + 2 * (s * (kStreamSeg / 32) + warp)) = make_uint2(p01, p23);
                mbar_arrive(empty0 + 8u * s);
            }
            __syncwarp();
        }
    }
    measure_finish<MODEL>(m, true, rows, wc, rec_hdr, C);
}

// Records of many lattices of one side L in one launch (the ensemble's
// replicas too large for shared memory): lattice blockIdx.z, its planes and
// its record slot (zeroed beforehand) in the kernel parameters.
struct MeasureMultiArgs {
    uint32_t *planes[kMultiMax];
    uint8_t *rec[kMultiMax];
};

template <int MODEL>
__global__ void __launch_bounds__(kMeasureThreads, MODEL == 0 ? kMeasureBlocksIsing : kMeasureBlocksBc)
    k_measure_multi(int64_t L, int H, int64_t sweep, const __grid_constant__ MeasureMultiArgs a)
{
    __shared__ int32_t s_row[kMeasureBand];
    const int r = blockIdx.z;
    int64_t *hdr = reinterpret_cast<int64_t *>(a.rec[r]);
    int32_t *R = reinterpret_cast<int32_t *>(hdr + 4);
    measure_band<MODEL>(a.planes[r], L, L / 64, L * (L / 64), H, hdr, R, R + L, sweep, s_row);
}

// Zero the record slots of a multi-lattice measure launch.
__global__ void k_zero_records(const __grid_constant__ MeasureMultiArgs a, int n, uint32_t words)
{
    for (int r = blockIdx.y; r < n; r += gridDim.y) {
        uint32_t *p = reinterpret_cast<uint32_t *>(a.rec[r]);
        for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < words; i += gridDim.x * blockDim.x)
            p[i] = 0u;
    }
}

// ---------------------------------------------------------------------------
// Row slabs of a lattice (domain decomposition, Introduction: the paper
// splits one lattice over many GPUs).  A slab's planes hold rows + 2 rows of
// W words each: row 0 is the halo above (global row y0 - 1, periodic), rows
// 1 .. rows the owned rows y0 .. y0 + rows - 1, row rows + 1 the halo below
// (global row y0 + rows).  The half-sweep and the observables are the band
// walks above with the halo rows in place of the periodic wrap and the
// global row for parity and random keys.
// ---------------------------------------------------------------------------
template <int V>
__global__ void __launch_bounds__(kSweepThreads, V == 4 ? kSweepMinBlocks : 8)
    k_ising_half_slab(uint32_t *__restrict__ tgt, const uint32_t *__restrict__ nbr, int64_t rows,
                      int64_t W, int colour, int H, PhiloxLaunch pc, IsingThr thr, uint32_t yg0)
{
    ising_half_band<V, false>(blockIdx.x * blockDim.x + threadIdx.x, tgt, nbr, (uint32_t)rows,
                              (uint32_t)W, colour, H, pc, thr, yg0);
}

template <int V, bool kFull>
__global__ void __launch_bounds__(kBcThreads, kBcMinBlocks)
    k_bc_half_slab(uint32_t *__restrict__ tn_plane, uint32_t *__restrict__ tp_plane,
                   const uint32_t *__restrict__ nn_plane, const uint32_t *__restrict__ np_plane,
                   int64_t rows, int64_t W, int colour, int H, PhiloxLaunch pc, BcTable tab,
                   uint32_t yg0)
{
    __shared__ uint32_t s_thr[kBcTableSize];
    for (int i = threadIdx.x; i < kBcTableSize; i += blockDim.x)
        s_thr[i] = tab.thr[i];
    __syncthreads();
    bc_half_band<V, kFull, false>((int64_t)blockIdx.x * blockDim.x + threadIdx.x, tn_plane, tp_plane,
                                  nn_plane, np_plane, rows, W, colour, H, pc, s_thr, yg0);
}

template <int MODEL>
__global__ void __launch_bounds__(kMeasureThreads, MODEL == 0 ? kMeasureBlocksIsing : kMeasureBlocksBc)
    k_measure_slab(const uint32_t *base, int64_t rows, int64_t W, int H, int64_t *__restrict__ rec_hdr,
                   int32_t *__restrict__ R, int32_t *__restrict__ C, int64_t sweep)
{
    __shared__ int32_t s_row[kMeasureBand];
    measure_band<MODEL, false>(base + W, rows, W, (rows + 2) * W, H, rec_hdr, R, C, sweep, s_row);
}

// Hot start of the owned rows (global keys) and byte <-> plane conversion of
// the owned rows.  One thread per word of an owned row of either colour.
__global__ void k_slab_init_random(SlabPlanes sp, PhiloxLaunch ph0, PhiloxLaunch ph1)
{
    const int64_t words = sp.rows * sp.W;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= 2 * words)
        return;
    const int c = gid >= words;
    const int64_t wi = c ? gid - words : gid;  // local row * W + w
    const int64_t yl = wi / sp.W, w = wi - yl * sp.W;
    const PhiloxLaunch &pc = c ? ph1 : ph0;
    const uint64_t q0 = (uint64_t)(sp.y0 + yl) * (uint64_t)(sp.L / 8) + 8u * (uint64_t)w;
    const PhiloxWordPart wp = philox_word_part(pc, (uint32_t)(q0 >> 32));
    uint32_t bits_n = 0, bits_p = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        uint32_t r[4];
        philox_site4(pc, wp, (uint32_t)q0 + i, r[0], r[1], r[2], r[3]);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int b = 4 * i + k;
            if (sp.model == 0) {
                bits_p |= (r[k] >> 31) << b;
            } else {
                const uint32_t v = (uint32_t)(((uint64_t)r[k] * 3u) >> 32);  // 0,1,2 -> s = v-1
                bits_n |= (uint32_t)(v != 1) << b;
                bits_p |= (uint32_t)(v == 2) << b;
            }
        }
    }
    const int64_t PS = (sp.rows + 2) * sp.W, off = sp.W + wi;
    if (sp.model == 0) {
        sp.base[(int64_t)c * PS + off] = bits_p;
    } else {
        sp.base[(int64_t)(2 * c) * PS + off] = bits_n;
        sp.base[(int64_t)(2 * c + 1) * PS + off] = bits_p;
    }
}

// s: rows x L bytes (row-major, owned rows); to_planes = 1 packs s into the
// planes (flagging values outside the model's set), 0 unpacks.
__global__ void k_slab_convert(SlabPlanes sp, int8_t *s, int to_planes, int32_t *bad)
{
    const int64_t words = sp.rows * sp.W;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= 2 * words)
        return;
    const int c = gid >= words;
    const int64_t wi = c ? gid - words : gid;
    const int64_t yl = wi / sp.W, w = wi - yl * sp.W;
    const int par = (c ^ (int)((sp.y0 + yl) & 1)) & 1;
    const int64_t PS = (sp.rows + 2) * sp.W, off = sp.W + wi;
    uint32_t *pn = sp.base + (int64_t)(sp.model == 0 ? c : 2 * c) * PS + off;
    uint32_t *pp = sp.base + (int64_t)(sp.model == 0 ? c : 2 * c + 1) * PS + off;
    int8_t *row = s + yl * sp.L;
    if (to_planes) {
        uint32_t bn = 0, bp = 0;
        for (int b = 0; b < 32; ++b) {
            const int v = row[2 * (32 * w + b) + par];
            if (sp.model == 0 ? (v != 1 && v != -1) : (v < -1 || v > 1))
                atomicExch(bad, 1);
            bn |= (uint32_t)(v != 0) << b;
            bp |= (uint32_t)(v > 0) << b;
        }
        *pp = bp;
        if (sp.model != 0)
            *pn = bn;
    } else {
        const uint32_t bp = *pp, bn = sp.model == 0 ? ~0u : *pn;
        for (int b = 0; b < 32; ++b) {
            const int on = (bn >> b) & 1, up = (bp >> b) & 1;
            row[2 * (32 * w + b) + par] = (int8_t)(sp.model == 0 ? (up ? 1 : -1) : (on ? (up ? 1 : -1) : 0));
        }
    }
}

// ---------------------------------------------------------------------------
// Correlation function along the axes (Eq. (2)): for each distance r of a
// list, Sx(r) = sum s(x,y) s(x+r,y) and Sy(r) = sum s(x,y) s(x,y+r), exact.
// A thread owns one word column w of one colour plane c over a band of rows.
//   vertical:   the partner of (c, y, w) is word w of row y+r in plane
//               c ^ (r & 1) (same same-colour index);
//   horizontal: the partner row is row y of plane c ^ (r & 1), shifted by
//               k = r/2 sites (r even) or (r-1)/2 + p (r odd, p = (c^y) & 1),
//               taken with a funnel shift across the word boundary.
// A pair contributes s s' = 1 - 2 [bits differ] (Ising) or
// n n' (1 - 2 (p ^ p')) (Blume-Capel), counted with popcounts.
// ---------------------------------------------------------------------------
// A Blume-Capel word pair: sum of n n' (1 - 2 (p ^ p')) over its 32 sites.
__device__ __forceinline__ int bc_pair_sum(uint32_t an, uint32_t ap, uint32_t bn, uint32_t bp)
{
    const uint32_t both = an & bn;
    return __popc(both) - 2 * __popc(both & (ap ^ bp));
}

// Ising rows y_s .. y_s + n - 1 of one band segment in which the vertical
// partner row y + r does not wrap: own words at own + i W, the partner
// plane's rows at hrow + i W, the vertical partners at vrow + i W.  Rows of
// even i (the parity of y_s) take the horizontal partner words (a0, b0)
// shifted by s0, rows of odd i (a1, b1, s1).  Adds the differing vertical
// pairs to mv and the differing horizontal pairs to mh.  Four rows per
// step with all their loads issued first and their parity known at
// compile time.
__device__ __forceinline__ void corr_ising_rows(const uint32_t *own, const uint32_t *hrow, const uint32_t *vrow,
                                                int n, int64_t W, int64_t a0, int64_t b0, unsigned s0,
                                                int64_t a1, int64_t b1, unsigned s1, int &mv, int &mh)
{
    int i = 0;
#pragma unroll 1
    for (; i + 4 <= n; i += 4) {
        uint32_t A[4], V[4], H1[4], H2[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            A[j] = __ldg(own + j * W);
            V[j] = __ldg(vrow + j * W);
            H1[j] = __ldg(hrow + j * W + ((j & 1) ? a1 : a0));
            H2[j] = __ldg(hrow + j * W + ((j & 1) ? b1 : b0));
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            mv += __popc(A[j] ^ V[j]);
            mh += __popc(A[j] ^ __funnelshift_r(H1[j], H2[j], (j & 1) ? s1 : s0));
        }
        own += 4 * W;
        hrow += 4 * W;
        vrow += 4 * W;
    }
    for (; i < n; ++i) {
        const bool odd = i & 1;
        const uint32_t a = __ldg(own);
        mv += __popc(a ^ __ldg(vrow));
        mh += __popc(a ^ __funnelshift_r(__ldg(hrow + (odd ? a1 : a0)), __ldg(hrow + (odd ? b1 : b0)),
                                         odd ? s1 : s0));
        own += W;
        hrow += W;
        vrow += W;
    }
}

template <int MODEL>
__global__ void __launch_bounds__(kMeasureThreads)
    k_correlation(Planes pl, int H, int nr, const int64_t *__restrict__ rlist,
                  unsigned long long *__restrict__ out)
{
    const int64_t L = pl.L, W = pl.W, LW = L * W;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = gid < 2 * W;
    const int c = active ? (int)(gid / W) : 0;
    const int64_t w = active ? gid - (int64_t)c * W : 0;
    const int64_t y0 = (int64_t)blockIdx.y * H;
    const int64_t y1 = y0 + H < L ? y0 + H : L;
    const int64_t half = L / 2;
    // sign plane (Ising: the only plane) and occupancy plane of colour cc
    auto sgn = [&](int cc) { return pl.base + (MODEL == 0 ? cc : 2 * cc + 1) * LW; };
    auto occ = [&](int cc) { return pl.base + (2 * cc) * LW; };
    __shared__ long long s_red[2][kMeasureThreads / 32];
    for (int k = 0; k < nr; ++k) {
        const int64_t r = rlist[k];
        const int cp = c ^ (int)(r & 1);
        int ax = 0, ay = 0;
        if (active && MODEL == 0) {
            // Ising.  Horizontal partner of row parity q = (c ^ y) & 1: bits
            // i + kk of the same row of plane cp, i.e. two words w1, w2
            // shifted by sh
            auto split = [&](int q, int64_t &a, int64_t &b, unsigned &sh) {
                int64_t kk = (r & 1) ? (r - 1) / 2 + q : r / 2;
                if (kk >= half)
                    kk -= half;
                a = w + (kk >> 5);
                if (a >= W)
                    a -= W;
                b = a + 1 == W ? 0 : a + 1;
                sh = (unsigned)(kk & 31);
            };
            int64_t w1e, w2e, w1o, w2o;
            unsigned oe, oo;
            split(0, w1e, w2e, oe);
            split(1, w1o, w2o, oo);
            // the band in at most two segments, split where the vertical
            // partner row y + r wraps to y + r - L, so that no row checks
            const int64_t y_wrap = L - r;
            int rows = 0, mv = 0, mh = 0;  // rows walked; differing vertical / horizontal pairs
#pragma unroll 1
            for (int sgm = 0; sgm < 2; ++sgm) {
                const int64_t ys = sgm == 0 ? y0 : (y0 > y_wrap ? y0 : y_wrap);
                const int64_t ye = sgm == 0 ? (y1 < y_wrap ? y1 : y_wrap) : y1;
                if (ye <= ys)
                    continue;
                const bool p = (c ^ (int)ys) & 1;  // parity of the segment's first row
                const uint32_t *own = sgn(c) + ys * W + w, *hr = sgn(cp) + ys * W;
                const uint32_t *vr = sgn(cp) + (ys + r - (sgm ? L : 0)) * W + w;
                const int n = (int)(ye - ys);
                corr_ising_rows(own, hr, vr, n, W, p ? w1o : w1e, p ? w2o : w2e, p ? oo : oe, p ? w1e : w1o,
                                p ? w2e : w2o, p ? oe : oo, mv, mh);
                rows += n;
            }
            // 32 pairs per row and axis: s s' = 1 - 2 [bits differ]
            ax = 32 * rows - 2 * mh;
            ay = 32 * rows - 2 * mv;
        } else if (active) {
            // Blume-Capel: per-row 64-bit row products (row pointers took it
            // from 40 to 128 registers and made it 24% slower; the Ising
            // walk's segments and four-row steps made it 10% slower at
            // L = 2^19, where it is nearer the memory bound)
            const uint32_t *os = sgn(c), *on = occ(c), *ps = sgn(cp), *pn = occ(cp);
            for (int64_t y = y0; y < y1; ++y) {
                const uint32_t a_p = __ldg(os + y * W + w);
                const uint32_t a_n = MODEL == 1 ? __ldg(on + y * W + w) : 0u;
                // vertical partner
                int64_t yv = y + r;
                if (yv >= L)
                    yv -= L;
                const uint32_t v_p = __ldg(ps + yv * W + w);
                const uint32_t v_n = MODEL == 1 ? __ldg(pn + yv * W + w) : 0u;
                ay += bc_pair_sum(a_n, a_p, v_n, v_p);
                // horizontal partner: bits i + kk of row y of plane cp
                int64_t kk = (r & 1) ? (r - 1) / 2 + ((c ^ (int)y) & 1) : r / 2;
                if (kk >= half)
                    kk -= half;
                int64_t w1 = w + (kk >> 5);
                if (w1 >= W)
                    w1 -= W;
                const int64_t w2 = w1 + 1 == W ? 0 : w1 + 1;
                const unsigned o = (unsigned)(kk & 31);
                const uint32_t h_p = __funnelshift_r(__ldg(ps + y * W + w1), __ldg(ps + y * W + w2), o);
                const uint32_t h_n = MODEL == 1
                                         ? __funnelshift_r(__ldg(pn + y * W + w1), __ldg(pn + y * W + w2), o)
                                         : 0u;
                ax += bc_pair_sum(a_n, a_p, h_n, h_p);
            }
        }
        long long sx = __reduce_add_sync(0xFFFFFFFFu, ax);
        long long sy = __reduce_add_sync(0xFFFFFFFFu, ay);
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (lane == 0) {
            s_red[0][warp] = sx;
            s_red[1][warp] = sy;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            long long tx = 0, ty = 0;
            for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
                tx += s_red[0][i];
                ty += s_red[1][i];
            }
            atomicAdd(&out[k], (unsigned long long)tx);
            atomicAdd(&out[nr + k], (unsigned long long)ty);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Byte-per-site <-> planes.
// ---------------------------------------------------------------------------
__global__ void k_pack(Planes pl, const int8_t *__restrict__ s, int32_t *bad)
{
    const int64_t LW = pl.L * pl.W;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= 2 * LW)
        return;
    const int c = gid >= LW;
    const int64_t wi = c ? gid - LW : gid;
    const int64_t y = wi / pl.W, w = wi - y * pl.W;
    const int par = (c ^ (int)y) & 1;
    uint32_t bn = 0, bp = 0;
    for (int b = 0; b < 32; ++b) {
        const int64_t x = 2 * (32 * w + b) + par;
        const int v = s[y * pl.L + x];
        if (pl.model == 0) {
            if (v != 1 && v != -1)
                atomicExch(bad, 1);
            bp |= (uint32_t)(v > 0) << b;
        } else {
            if (v < -1 || v > 1)
                atomicExch(bad, 1);
            bn |= (uint32_t)(v != 0) << b;
            bp |= (uint32_t)(v > 0) << b;
        }
    }
    if (pl.model == 0) {
        pl.base[(int64_t)c * LW + wi] = bp;
    } else {
        pl.base[(int64_t)(2 * c) * LW + wi] = bn;
        pl.base[(int64_t)(2 * c + 1) * LW + wi] = bp;
    }
}

__global__ void k_unpack_rect(Planes pl, int64_t y0, int64_t x0, int64_t h, int64_t w,
                              int8_t *__restrict__ out)
{
    const int64_t LW = pl.L * pl.W;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= h * w)
        return;
    const int64_t i = gid / w, j = gid - i * w;
    const int64_t y = (y0 + i) % pl.L, x = (x0 + j) % pl.L;
    const int c = (int)((x + y) & 1);
    const int64_t si = x >> 1;  // same-colour index within the row
    const int64_t word = y * pl.W + (si >> 5);
    const int bit = (int)(si & 31);
    int v;
    if (pl.model == 0) {
        v = ((pl.base[(int64_t)c * LW + word] >> bit) & 1u) ? 1 : -1;
    } else {
        const uint32_t n = (pl.base[(int64_t)(2 * c) * LW + word] >> bit) & 1u;
        const uint32_t p = (pl.base[(int64_t)(2 * c + 1) * LW + word] >> bit) & 1u;
        v = n ? (p ? 1 : -1) : 0;
    }
    out[gid] = (int8_t)v;
}

// Rows per thread for a sweep launch: at most 64, fewer while the grid would
// give less than `waves` waves of resident blocks (blocks_per_sm blocks of
// `threads` threads on each of the 148 SMs).  Ising: eight waves of its
// 128-thread blocks; Blume-Capel: two waves of its 256-thread blocks (taller
// bands: at L = 16384, 919 vs 830 flips/ns with the Ising rule).
int sweep_band(int64_t L, int64_t threads_per_row, int blocks_per_sm = kSweepMinBlocks,
               int threads = kSweepThreads, int waves = 8)
{
    const int64_t want_threads = 148LL * blocks_per_sm * threads * waves;
    int H = 64;
    while (H > 1 && threads_per_row * ((L + H - 1) / H) < want_threads)
        H >>= 1;
    return H;
}

unsigned sweep_blocks(int64_t L, int64_t threads_per_row, int H)
{
    const int64_t threads = threads_per_row * ((L + H - 1) / H);
    return (unsigned)((threads + kSweepThreads - 1) / kSweepThreads);
}

template <int V>
cudaError_t launch_ising(const Planes &pl, int colour, const PhiloxLaunch &ph, const IsingThr &thr,
                         cudaStream_t st)
{
    const int64_t LW = pl.L * pl.W;
    uint32_t *tgt = pl.base + (int64_t)colour * LW;
    const uint32_t *nbr = pl.base + (int64_t)(1 - colour) * LW;
    const int64_t tpr = pl.W / V;
    const int H = sweep_band(pl.L, tpr);
    k_ising_half<V><<<sweep_blocks(pl.L, tpr, H), kSweepThreads, 0, st>>>(tgt, nbr, pl.L, pl.W, colour, H, ph, thr);
    return cudaGetLastError();
}

template <int V>
cudaError_t launch_bc(const Planes &pl, int colour, const PhiloxLaunch &ph, const BcTable &tab,
                      cudaStream_t st)
{
    const int64_t LW = pl.L * pl.W;
    uint32_t *tn = pl.base + (int64_t)(2 * colour) * LW;
    uint32_t *tp = tn + LW;
    const uint32_t *nn = pl.base + (int64_t)(2 * (1 - colour)) * LW;
    const uint32_t *np = nn + LW;
    const int64_t tpr = pl.W / V;
    const int H = sweep_band(pl.L, tpr, kBcMinBlocks, kBcThreads, 2);
    const int64_t threads = tpr * ((pl.L + H - 1) / H);
    const unsigned blocks = (unsigned)((threads + kBcThreads - 1) / kBcThreads);
    if (tab.full)
        k_bc_half<V, true><<<blocks, kBcThreads, 0, st>>>(tn, tp, nn, np, pl.L, pl.W, colour, H, ph, tab);
    else
        k_bc_half<V, false><<<blocks, kBcThreads, 0, st>>>(tn, tp, nn, np, pl.L, pl.W, colour, H, ph, tab);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_init_random(const Planes &pl, const PhiloxLaunch &ph0, const PhiloxLaunch &ph1,
                               cudaStream_t st)
{
    const int64_t n = 2 * pl.L * pl.W;
    const int threads = 256;
    k_init_random<<<(unsigned)((n + threads - 1) / threads), threads, 0, st>>>(pl, ph0, ph1);
    return cudaGetLastError();
}

cudaError_t launch_init_uniform(const Planes &pl, int value, cudaStream_t st)
{
    k_init_uniform<<<148 * 8, 256, 0, st>>>(pl, value);
    return cudaGetLastError();
}

// Words per thread: the most that still gives `waves` full waves of
// resident blocks with one-row bands, and that divides the row.  A lattice
// of a few thousand rows has too few threads at four words per thread:
// Ising L = 2048 runs at 511 instead of 341 flips/ns with one word per
// thread, L = 4096 at 837 instead of 819; from L = 8192 on four words win
// (1261 against 1171 with one).
int words_per_thread(int64_t L, int64_t W, int vmax, int blocks_per_sm, int threads, int waves)
{
    for (int V = vmax; V > 1; V >>= 1)
        if (W % V == 0 && (W / V) * L >= 148LL * blocks_per_sm * threads * waves)
            return V;
    return 1;
}

cudaError_t launch_half_sweep(const Planes &pl, int colour, const PhiloxLaunch &ph,
                              const IsingThr &ithr, const BcTable *btab, cudaStream_t st)
{
    if (injected_launch_failure())
        return cudaErrorLaunchFailure;
    if (pl.model == 0) {
        const int V = words_per_thread(pl.L, pl.W, 4, kSweepMinBlocks, kSweepThreads, 1);
        if (V == 4)
            return launch_ising<4>(pl, colour, ph, ithr, st);
        if (V == 2)
            return launch_ising<2>(pl, colour, ph, ithr, st);
        return launch_ising<1>(pl, colour, ph, ithr, st);
    }
    // Blume-Capel: at most two words per thread (more threads in flight than
    // four at the same 80 registers: 137 vs 148 ms per half-sweep at
    // L = 2^19, 919 vs 898 flips/ns at L = 16384)
    if (words_per_thread(pl.L, pl.W, 2, kBcMinBlocks, kBcThreads, 1) == 2)
        return launch_bc<2>(pl, colour, ph, *btab, st);
    return launch_bc<1>(pl, colour, ph, *btab, st);
}

cudaError_t launch_half_sweep_multi(int model, int64_t L, uint32_t *const *planes, const uint64_t *seeds,
                                    int n, uint32_t t, int colour, const IsingThr &ithr,
                                    const BcTable *btab, cudaStream_t st, int V_set, int H_set)
{
    const int64_t W = L / 64;
    if (injected_launch_failure())
        return cudaErrorLaunchFailure;
    for (int i0 = 0; i0 < n; i0 += kMultiMax) {
        const int m = n - i0 < kMultiMax ? n - i0 : kMultiMax;
        MultiArgs a;
        for (int i = 0; i < m; ++i) {
            philox_launch_consts(seeds[i0 + i], t, (uint32_t)colour, &a.pc[i]);
            a.planes[i] = planes[i0 + i];
        }
        if (model == 0) {
            const int V = ((V_set == 1 || V_set == 2 || V_set == 4) && W % V_set == 0)
                              ? V_set : (W % 4 == 0 ? 4 : (W % 2 == 0 ? 2 : 1));
            const int64_t tpr = W / V;
            // the band height that fills the GPU for one lattice, taller
            // while the m lattices of the launch still fill the waves
            int H = sweep_band(L, tpr);
            while (H < 64 && tpr * ((L + 2 * H - 1) / (2 * H)) * m >= 148LL * kSweepMinBlocks * kSweepThreads * 8)
                H *= 2;
            if (H_set > 0)
                H = H_set;
            const dim3 grid(sweep_blocks(L, tpr, H), (unsigned)m);
            if (V == 4)
                k_ising_half_multi<4><<<grid, kSweepThreads, 0, st>>>(L, colour, H, ithr, a);
            else if (V == 2)
                k_ising_half_multi<2><<<grid, kSweepThreads, 0, st>>>(L, colour, H, ithr, a);
            else
                k_ising_half_multi<1><<<grid, kSweepThreads, 0, st>>>(L, colour, H, ithr, a);
        } else {
            const int V = ((V_set == 1 || V_set == 2) && W % V_set == 0) ? V_set : (W % 2 == 0 ? 2 : 1);
            const int64_t tpr = W / V;
            int H = sweep_band(L, tpr, kBcMinBlocks, kBcThreads, 2);
            while (H < 64 && tpr * ((L + 2 * H - 1) / (2 * H)) * m >= 148LL * kBcMinBlocks * kBcThreads * 2)
                H *= 2;
            if (H_set > 0)
                H = H_set;
            const int64_t threads = tpr * ((L + H - 1) / H);
            const dim3 grid((unsigned)((threads + kBcThreads - 1) / kBcThreads), (unsigned)m);
            if (V == 2) {
                if (btab->full)
                    k_bc_half_multi<2, true><<<grid, kBcThreads, 0, st>>>(L, colour, H, *btab, a);
                else
                    k_bc_half_multi<2, false><<<grid, kBcThreads, 0, st>>>(L, colour, H, *btab, a);
            } else {
                if (btab->full)
                    k_bc_half_multi<1, true><<<grid, kBcThreads, 0, st>>>(L, colour, H, *btab, a);
                else
                    k_bc_half_multi<1, false><<<grid, kBcThreads, 0, st>>>(L, colour, H, *btab, a);
            }
        }
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

// The driver's tensor-map encoder, looked up once through the runtime (no
// link against the driver library); null if this driver lacks it.
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
        }
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

// Tensor maps of a lattice's planes for k_measure_stream: (W / 2) x L x
// planes elements of 8 bytes, boxes of 128 x 4 x 1 (colour-1 rows) and
// 132 x 4 x 1 (colour-0 rows with 2-element halos).  False if they cannot be
// made; the pass then copies every row with 1D bulk copies.
static bool stream_tensor_maps(const Planes &pl, CUtensorMap *tmT, CUtensorMap *tmD)
{
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc)
        return false;
    const cuuint64_t dims[3] = {(cuuint64_t)(pl.W / 2), (cuuint64_t)pl.L, (cuuint64_t)(pl.model == 0 ? 2 : 4)};
    const cuuint64_t strides[2] = {(cuuint64_t)pl.W * 4, (cuuint64_t)pl.L * (cuuint64_t)pl.W * 4};
    const cuuint32_t boxT[3] = {kStreamSeg / 2, 4, 1}, boxD[3] = {kStreamRowD / 2, 4, 1}, one[3] = {1, 1, 1};
    for (int k = 0; k < 2; ++k) {
        const CUresult r = enc(k == 0 ? tmT : tmD, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, pl.base, dims, strides,
                               k == 0 ? boxT : boxD, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
                               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS)
            return false;
    }
    return true;
}

cudaError_t launch_measure(const Planes &pl, void *record, int64_t sweep, cudaStream_t st)
{
    int64_t *hdr = reinterpret_cast<int64_t *>(record);
    int32_t *R = reinterpret_cast<int32_t *>(hdr + 4);
    int32_t *C = R + pl.L;
    // band height: a multiple of 16 (L is a multiple of 64, so every band,
    // the last included, has a multiple of 16 rows), as tall as possible
    // (fewer column atomics) while the grid still has a few blocks per SM
    const int64_t bx = (pl.W + kMeasureThreads - 1) / kMeasureThreads;
    int64_t H = pl.L < kMeasureBand ? pl.L : kMeasureBand;
    while (H % 32 == 0 && bx * ((pl.L + H - 1) / H) < 148 * 4)
        H >>= 1;
    const dim3 grid((unsigned)bx, (unsigned)((pl.L + H - 1) / H));
    if (pl.W % kStreamSeg == 0 && (reinterpret_cast<uintptr_t>(pl.base) & 15u) == 0) {
        // whole segments (and the 16-byte aligned planes bulk copies need):
        // the streamed pass, on the same grid, one segment per block; if its
        // shared memory cannot be had, the register walk below (same sums)
        const cudaError_t ea = pl.model == 0
                                   ? cudaFuncSetAttribute(k_measure_stream<0>,
                                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                          (int)StreamShape<0>::kSmem)
                                   : cudaFuncSetAttribute(k_measure_stream<1>,
                                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                          (int)StreamShape<1>::kSmem);
        if (ea == cudaSuccess) {
            const uint32_t extra = injected_wait_failure() ? 16u : 0u;
            CUtensorMap tmT, tmD;
            const int tmap = stream_tensor_maps(pl, &tmT, &tmD) ? 1 : 0;
            if (pl.model == 0)
                k_measure_stream<0><<<grid, kStreamThreads, StreamShape<0>::kSmem, st>>>(
                    pl, (int)H, hdr, R, C, sweep, extra, tmT, tmD, tmap);
            else
                k_measure_stream<1><<<grid, kStreamThreads, StreamShape<1>::kSmem, st>>>(
                    pl, (int)H, hdr, R, C, sweep, extra, tmT, tmD, tmap);
            return cudaGetLastError();
        }
        cudaGetLastError();
    }
    if (pl.model == 0)
        k_measure<0><<<grid, kMeasureThreads, 0, st>>>(pl, (int)H, hdr, R, C, sweep);
    else
        k_measure<1><<<grid, kMeasureThreads, 0, st>>>(pl, (int)H, hdr, R, C, sweep);
    return cudaGetLastError();
}

cudaError_t launch_measure_multi(int model, int64_t L, uint32_t *const *planes, uint8_t *const *recs, int n,
                                 int64_t sweep, cudaStream_t st)
{
    const int64_t W = L / 64;
    const int64_t bx = (W + kMeasureThreads - 1) / kMeasureThreads;
    for (int i0 = 0; i0 < n; i0 += kMultiMax) {
        const int m = n - i0 < kMultiMax ? n - i0 : kMultiMax;
        MeasureMultiArgs a;
        for (int i = 0; i < m; ++i) {
            a.planes[i] = planes[i0 + i];
            a.rec[i] = recs[i0 + i];
        }
        const uint32_t words = (uint32_t)(record_stride(L) / 4);
        k_zero_records<<<dim3((words + 255) / 256, (unsigned)m), 256, 0, st>>>(a, m, words);
        // band height as for one lattice, taller while the m lattices keep
        // a few blocks per SM (fewer column atomics)
        int64_t H = L < kMeasureBand ? L : kMeasureBand;
        while (H % 32 == 0 && bx * ((L + H - 1) / H) * m < 148 * 4)
            H >>= 1;
        const dim3 grid((unsigned)bx, (unsigned)((L + H - 1) / H), (unsigned)m);
        if (model == 0)
            k_measure_multi<0><<<grid, kMeasureThreads, 0, st>>>(L, (int)H, sweep, a);
        else
            k_measure_multi<1><<<grid, kMeasureThreads, 0, st>>>(L, (int)H, sweep, a);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

cudaError_t launch_half_sweep_slab(const SlabPlanes &sp, int colour, const PhiloxLaunch &ph,
                                   const IsingThr &ithr, const BcTable *btab, cudaStream_t st)
{
    if (injected_launch_failure())
        return cudaErrorLaunchFailure;
    const int64_t PS = (sp.rows + 2) * sp.W;
    const uint32_t yg0 = (uint32_t)sp.y0;
    if (sp.model == 0) {
        uint32_t *tgt = sp.base + (int64_t)colour * PS + sp.W;
        const uint32_t *nbr = sp.base + (int64_t)(1 - colour) * PS + sp.W;
        const int V = words_per_thread(sp.rows, sp.W, 4, kSweepMinBlocks, kSweepThreads, 1);
        const int64_t tpr = sp.W / V;
        const int H = sweep_band(sp.rows, tpr);
        const unsigned blocks = sweep_blocks(sp.rows, tpr, H);
        if (V == 4)
            k_ising_half_slab<4><<<blocks, kSweepThreads, 0, st>>>(tgt, nbr, sp.rows, sp.W, colour, H, ph, ithr, yg0);
        else if (V == 2)
            k_ising_half_slab<2><<<blocks, kSweepThreads, 0, st>>>(tgt, nbr, sp.rows, sp.W, colour, H, ph, ithr, yg0);
        else
            k_ising_half_slab<1><<<blocks, kSweepThreads, 0, st>>>(tgt, nbr, sp.rows, sp.W, colour, H, ph, ithr, yg0);
        return cudaGetLastError();
    }
    uint32_t *tn = sp.base + (int64_t)(2 * colour) * PS + sp.W;
    uint32_t *tp = tn + PS;
    const uint32_t *nn = sp.base + (int64_t)(2 * (1 - colour)) * PS + sp.W;
    const uint32_t *np = nn + PS;
    const int V = words_per_thread(sp.rows, sp.W, 2, kBcMinBlocks, kBcThreads, 1) == 2 ? 2 : 1;
    const int64_t tpr = sp.W / V;
    const int H = sweep_band(sp.rows, tpr, kBcMinBlocks, kBcThreads, 2);
    const int64_t threads = tpr * ((sp.rows + H - 1) / H);
    const unsigned blocks = (unsigned)((threads + kBcThreads - 1) / kBcThreads);
    if (V == 2) {
        if (btab->full)
            k_bc_half_slab<2, true><<<blocks, kBcThreads, 0, st>>>(tn, tp, nn, np, sp.rows, sp.W, colour, H, ph, *btab, yg0);
        else
            k_bc_half_slab<2, false><<<blocks, kBcThreads, 0, st>>>(tn, tp, nn, np, sp.rows, sp.W, colour, H, ph, *btab, yg0);
    } else {
        if (btab->full)
            k_bc_half_slab<1, true><<<blocks, kBcThreads, 0, st>>>(tn, tp, nn, np, sp.rows, sp.W, colour, H, ph, *btab, yg0);
        else
            k_bc_half_slab<1, false><<<blocks, kBcThreads, 0, st>>>(tn, tp, nn, np, sp.rows, sp.W, colour, H, ph, *btab, yg0);
    }
    return cudaGetLastError();
}

cudaError_t launch_measure_slab(const SlabPlanes &sp, void *record, int64_t sweep, cudaStream_t st)
{
    int64_t *hdr = reinterpret_cast<int64_t *>(record);
    int32_t *R = reinterpret_cast<int32_t *>(hdr + 4);
    int32_t *C = R + sp.rows;
    // band height: a multiple of 16 (rows is one), as in launch_measure
    const int64_t bx = (sp.W + kMeasureThreads - 1) / kMeasureThreads;
    int64_t H = sp.rows < kMeasureBand ? sp.rows : kMeasureBand;
    while (H % 32 == 0 && bx * ((sp.rows + H - 1) / H) < 148 * 4)
        H >>= 1;
    const dim3 grid((unsigned)bx, (unsigned)((sp.rows + H - 1) / H));
    if (sp.model == 0)
        k_measure_slab<0><<<grid, kMeasureThreads, 0, st>>>(sp.base, sp.rows, sp.W, (int)H, hdr, R, C, sweep);
    else
        k_measure_slab<1><<<grid, kMeasureThreads, 0, st>>>(sp.base, sp.rows, sp.W, (int)H, hdr, R, C, sweep);
    return cudaGetLastError();
}

cudaError_t launch_slab_init_random(const SlabPlanes &sp, const PhiloxLaunch &ph0, const PhiloxLaunch &ph1,
                                    cudaStream_t st)
{
    const int64_t n = 2 * sp.rows * sp.W;
    k_slab_init_random<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(sp, ph0, ph1);
    return cudaGetLastError();
}

cudaError_t launch_slab_convert(const SlabPlanes &sp, int8_t *d_spins, int to_planes, int32_t *d_bad,
                                cudaStream_t st)
{
    const int64_t n = 2 * sp.rows * sp.W;
    k_slab_convert<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(sp, d_spins, to_planes, d_bad);
    return cudaGetLastError();
}

cudaError_t launch_correlation(const Planes &pl, int nr, const int64_t *d_r, unsigned long long *d_out,
                               cudaStream_t st)
{
    const int64_t bx = (2 * pl.W + kMeasureThreads - 1) / kMeasureThreads;
    int64_t H = pl.L < 4096 ? pl.L : 4096;
    while (H > 1 && bx * ((pl.L + H - 1) / H) < 148 * 8)
        H >>= 1;
    const dim3 grid((unsigned)bx, (unsigned)((pl.L + H - 1) / H));
    if (pl.model == 0)
        k_correlation<0><<<grid, kMeasureThreads, 0, st>>>(pl, (int)H, nr, d_r, d_out);
    else
        k_correlation<1><<<grid, kMeasureThreads, 0, st>>>(pl, (int)H, nr, d_r, d_out);
    return cudaGetLastError();
}

cudaError_t launch_pack(const Planes &pl, const int8_t *d_spins, int32_t *d_bad, cudaStream_t st)
{
    const int64_t n = 2 * pl.L * pl.W;
    k_pack<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(pl, d_spins, d_bad);
    return cudaGetLastError();
}

cudaError_t launch_unpack_rect(const Planes &pl, int64_t y0, int64_t x0, int64_t h, int64_t w,
                               int8_t *d_out, cudaStream_t st)
{
    const int64_t n = h * w;
    if (n == 0)
        return cudaSuccess;
    k_unpack_rect<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(pl, y0, x0, h, w, d_out);
    return cudaGetLastError();
}

}  // namespace isg
