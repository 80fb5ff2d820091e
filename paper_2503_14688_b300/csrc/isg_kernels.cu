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
#include <cuda_runtime.h>

#include <cstdint>

#include "isg_internal.h"
#include "isg_philox.cuh"

namespace isg {

namespace {

constexpr int kSweepThreads = 128;
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

// Index of the word adjacent to the V-word group starting at w0 on the side
// that parity needs, with periodic wrap.
__device__ __forceinline__ int64_t edge_word(int64_t w0, int V, int64_t W, int parity)
{
    if (parity == 0)
        return w0 == 0 ? W - 1 : w0 - 1;
    return w0 + V == W ? 0 : w0 + V;
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
template <int V>
__global__ void __launch_bounds__(kSweepThreads)
    k_ising_half(uint32_t *__restrict__ tgt, const uint32_t *__restrict__ nbr, int64_t L,
                 int64_t W, int colour, int H, PhiloxLaunch pc, IsingThr thr)
{
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * V;
    const int64_t y0 = (int64_t)blockIdx.y * H;
    if (w0 >= W || y0 >= L)
        return;
    const int64_t y1 = y0 + H < L ? y0 + H : L;
    const uint64_t qrow = (uint64_t)(L / 8);

    Words<V> U = load_words<V>(nbr + (y0 == 0 ? L - 1 : y0 - 1) * W + w0);
    Words<V> S = load_words<V>(nbr + y0 * W + w0);
    for (int64_t y = y0; y < y1; ++y) {
        const int64_t yd = y + 1 == L ? 0 : y + 1;
        const Words<V> D = load_words<V>(nbr + yd * W + w0);
        const int parity = (colour ^ (int)y) & 1;
        const uint32_t edge = __ldg(nbr + y * W + edge_word(w0, V, W, parity));
        const Words<V> X = side_words<V>(S, edge, parity);
        Words<V> T = load_words_rw<V>(tgt + y * W + w0);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const uint64_t q0 = (uint64_t)y * qrow + 8u * (uint64_t)(w0 + v);
            const PhiloxWordPart wp = philox_word_part(pc, (uint32_t)(q0 >> 32));
            uint32_t a4 = 0, a8 = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                uint32_t r[4];
                philox_site4(pc, wp, (uint32_t)q0 + i, r[0], r[1], r[2], r[3]);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    a4 |= (uint32_t)(r[k] < thr.thr4) << (4 * i + k);
                    a8 |= (uint32_t)(r[k] < thr.thr8) << (4 * i + k);
                }
            }
            a4 |= thr.full4;
            a8 |= thr.full8;
            const uint32_t t = T.v[v];
            // anti-aligned neighbour indicators and their bit-sliced count
            const uint32_t a = t ^ U.v[v], b = t ^ D.v[v], d = t ^ S.v[v], e = t ^ X.v[v];
            const uint32_t s1 = a ^ b ^ d;
            const uint32_t c1 = (a & b) | (d & (a ^ b));
            const uint32_t s = s1 ^ e;         // count = s + 2 (c1 + c2)
            const uint32_t c2 = s1 & e;
            const uint32_t ge2 = c1 | c2;      // dE <= 0: always flip
            const uint32_t flip = ge2 | (~ge2 & ((s & a4) | (~s & a8)));
            T.v[v] = t ^ flip;
        }
        store_words<V>(tgt + y * W + w0, T);
        U = S;
        S = D;
    }
}

// ---------------------------------------------------------------------------
// Blume-Capel half-sweep.  Two bit-planes per colour: n (s != 0) and p (s > 0).
// The neighbour field h + 4 = #(+1 neighbours) + #(neighbours != -1) is a
// bit-sliced sum of eight indicator words (four bits g0..g3); each site
// then looks its threshold up in a 128-entry table indexed by
// (n, p, proposal bit, h + 4) held in shared memory.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void full_add(uint32_t a, uint32_t b, uint32_t c, uint32_t &s,
                                         uint32_t &cy)
{
    s = a ^ b ^ c;
    cy = (a & b) | (c & (a ^ b));
}

template <int V>
__global__ void __launch_bounds__(kSweepThreads)
    k_bc_half(uint32_t *__restrict__ tn_plane, uint32_t *__restrict__ tp_plane,
              const uint32_t *__restrict__ nn_plane, const uint32_t *__restrict__ np_plane,
              int64_t L, int64_t W, int colour, int H, PhiloxLaunch pc, BcTable tab)
{
    __shared__ uint32_t s_thr[kBcTableSize];
    for (int i = threadIdx.x; i < kBcTableSize; i += blockDim.x)
        s_thr[i] = tab.thr[i];
    __syncthreads();

    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * V;
    const int64_t y0 = (int64_t)blockIdx.y * H;
    if (w0 >= W || y0 >= L)
        return;
    const int64_t y1 = y0 + H < L ? y0 + H : L;
    const uint64_t qrow = (uint64_t)(L / 8);
    const int64_t yu0 = y0 == 0 ? L - 1 : y0 - 1;

    Words<V> Un = load_words<V>(nn_plane + yu0 * W + w0);
    Words<V> Up = load_words<V>(np_plane + yu0 * W + w0);
    Words<V> Sn = load_words<V>(nn_plane + y0 * W + w0);
    Words<V> Sp = load_words<V>(np_plane + y0 * W + w0);
    for (int64_t y = y0; y < y1; ++y) {
        const int64_t yd = y + 1 == L ? 0 : y + 1;
        const Words<V> Dn = load_words<V>(nn_plane + yd * W + w0);
        const Words<V> Dp = load_words<V>(np_plane + yd * W + w0);
        const int parity = (colour ^ (int)y) & 1;
        const int64_t ew = y * W + edge_word(w0, V, W, parity);
        const Words<V> Xn = side_words<V>(Sn, __ldg(nn_plane + ew), parity);
        const Words<V> Xp = side_words<V>(Sp, __ldg(np_plane + ew), parity);
        Words<V> Tn = load_words_rw<V>(tn_plane + y * W + w0);
        Words<V> Tp = load_words_rw<V>(tp_plane + y * W + w0);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            // eight indicators: s_i = +1 (n & p), s_i != -1 (~n | p)
            const uint32_t x0 = Un.v[v] & Up.v[v], x1 = ~Un.v[v] | Up.v[v];
            const uint32_t x2 = Dn.v[v] & Dp.v[v], x3 = ~Dn.v[v] | Dp.v[v];
            const uint32_t x4 = Sn.v[v] & Sp.v[v], x5 = ~Sn.v[v] | Sp.v[v];
            const uint32_t x6 = Xn.v[v] & Xp.v[v], x7 = ~Xn.v[v] | Xp.v[v];
            uint32_t sa, ca, sb, cb, sc, cc, g0, cd, se, ce, g1, cf;
            full_add(x0, x1, x2, sa, ca);
            full_add(x3, x4, x5, sb, cb);
            full_add(sa, sb, x6, sc, cc);
            g0 = sc ^ x7;
            cd = sc & x7;
            full_add(ca, cb, cc, se, ce);   // weight-2 column
            g1 = se ^ cd;
            cf = se & cd;
            const uint32_t g2 = ce ^ cf;     // weight-4 column
            const uint32_t g3 = ce & cf;     // only when h + 4 = 8

            const uint32_t n = Tn.v[v], p = Tp.v[v];
            const uint64_t q0 = (uint64_t)y * qrow + 8u * (uint64_t)(w0 + v);
            const PhiloxWordPart wp = philox_word_part(pc, (uint32_t)(q0 >> 32));
            uint32_t acc = 0, bits = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                uint32_t r[4];
                philox_site4(pc, wp, (uint32_t)q0 + i, r[0], r[1], r[2], r[3]);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int bi = 4 * i + k;
                    const uint32_t bb = r[k] & 1u;
                    const uint32_t idx = (((n >> bi) & 1u) << 6) | (((p >> bi) & 1u) << 5) |
                                         (bb << 4) | (((g3 >> bi) & 1u) << 3) |
                                         (((g2 >> bi) & 1u) << 2) | (((g1 >> bi) & 1u) << 1) |
                                         ((g0 >> bi) & 1u);
                    acc |= (uint32_t)((r[k] >> 1) < s_thr[idx]) << bi;
                    bits |= bb << bi;
                }
            }
            // proposed value: p' = b & ~(n & p), n' = ~n | (p ^ b)
            const uint32_t np2 = bits & ~(n & p);
            const uint32_t nn2 = ~n | (p ^ bits);
            Tn.v[v] = n ^ (acc & (n ^ nn2));
            Tp.v[v] = p ^ (acc & (p ^ np2));
        }
        store_words<V>(tn_plane + y * W + w0, Tn);
        store_words<V>(tp_plane + y * W + w0, Tp);
        Un = Sn;
        Up = Sp;
        Sn = Dn;
        Sp = Dp;
    }
}

// ---------------------------------------------------------------------------
// Observables.  A thread owns one word column w of both colours over a band
// of H rows.  Bonds: every bond joins a colour-0 and a colour-1 site, so
// B = sum over colour-1 sites of s * (sum of its four colour-0 neighbours).
// Row sums: a warp's lanes share the row, reduced by shuffles into a
// shared-memory array for the band, then one global atomic per row and block.
// Column sums: per bit position, vertical bit-sliced counters of the +1 (and
// for Blume-Capel the -1) sites, split by column parity; at the end of the
// band they are read out per column and added atomically.
// ---------------------------------------------------------------------------
constexpr int kCountBits = 13;  // band height < 2^13
constexpr int kMeasureBand = 4096;

__device__ __forceinline__ void vcount_add(uint32_t (&c)[kCountBits], uint32_t x)
{
#pragma unroll
    for (int l = 0; l < kCountBits; ++l) {
        const uint32_t carry = c[l] & x;
        c[l] ^= x;
        x = carry;
        if (x == 0)
            break;
    }
}

__device__ __forceinline__ int vcount_get(const uint32_t (&c)[kCountBits], int bit)
{
    int v = 0;
#pragma unroll
    for (int l = 0; l < kCountBits; ++l)
        v |= (int)((c[l] >> bit) & 1u) << l;
    return v;
}

__device__ __forceinline__ int64_t warp_sum64(int64_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

__device__ __forceinline__ int warp_sum32(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

template <int MODEL>
__global__ void __launch_bounds__(kMeasureThreads)
    k_measure(Planes pl, int H, int64_t *__restrict__ rec_hdr, int32_t *__restrict__ R,
              int32_t *__restrict__ C, int64_t sweep)
{
    __shared__ int32_t s_row[kMeasureBand];
    const int64_t L = pl.L, W = pl.W, LW = L * W;
    const int64_t y0 = (int64_t)blockIdx.y * H;
    const int64_t y1 = y0 + H < L ? y0 + H : L;
    for (int i = threadIdx.x; i < H; i += blockDim.x)
        s_row[i] = 0;
    __syncthreads();
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0)
        rec_hdr[0] = sweep;

    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = w < W && y0 < L;
    const int64_t wc = active ? w : 0;
    // plane pointers: colour c, bit-plane k
    const uint32_t *n0 = pl.base, *n1, *p0, *p1;
    if (MODEL == 0) {
        p0 = pl.base;
        p1 = pl.base + LW;
        n0 = n1 = nullptr;
    } else {
        n0 = pl.base;
        p0 = pl.base + LW;
        n1 = pl.base + 2 * LW;
        p1 = pl.base + 3 * LW;
    }
    int64_t accB = 0, accM = 0, accQ = 0;
    uint32_t ce_p[kCountBits] = {}, co_p[kCountBits] = {};
    uint32_t ce_m[kCountBits] = {}, co_m[kCountBits] = {};
    const int64_t yup = y0 == 0 ? L - 1 : y0 - 1;
    uint32_t Up = 0, Sp = 0, Un = ~0u, Sn = ~0u;
    if (active) {
        Up = __ldg(p0 + yup * W + wc);
        Sp = __ldg(p0 + y0 * W + wc);
        if (MODEL == 1) {
            Un = __ldg(n0 + yup * W + wc);
            Sn = __ldg(n0 + y0 * W + wc);
        }
    }
    for (int64_t y = y0; y < y1; ++y) {
        int rowpart = 0;
        if (active) {
            const int64_t yd = y + 1 == L ? 0 : y + 1;
            const int par1 = (1 ^ (int)y) & 1;  // colour-1 parity of row y
            const int64_t ew = y * W + edge_word(wc, 1, W, par1);
            const uint32_t Dp = __ldg(p0 + yd * W + wc);
            const uint32_t Xp = par1 == 0 ? (Sp << 1) | (__ldg(p0 + ew) >> 31)
                                          : (Sp >> 1) | (__ldg(p0 + ew) << 31);
            const uint32_t Tp = __ldg(p1 + y * W + wc);
            if (MODEL == 0) {
                const int anti = __popc(Tp ^ Up) + __popc(Tp ^ Dp) + __popc(Tp ^ Sp) +
                                 __popc(Tp ^ Xp);
                accB += 128 - 2 * anti;
                const int ones = __popc(Tp) + __popc(Sp);
                rowpart = 2 * ones - 64;
                const uint32_t E = (y & 1) ? Tp : Sp, O = (y & 1) ? Sp : Tp;
                vcount_add(ce_p, E);
                vcount_add(co_p, O);
                Up = Sp;
                Sp = Dp;
            } else {
                const uint32_t Dn = __ldg(n0 + yd * W + wc);
                const uint32_t Xn = par1 == 0 ? (Sn << 1) | (__ldg(n0 + ew) >> 31)
                                              : (Sn >> 1) | (__ldg(n0 + ew) << 31);
                const uint32_t Tn = __ldg(n1 + y * W + wc);
                const uint32_t nb[4] = {Un, Dn, Sn, Xn}, pb[4] = {Up, Dp, Sp, Xp};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint32_t both = Tn & nb[k];
                    accB += __popc(both) - 2 * __popc(both & (Tp ^ pb[k]));
                }
                const uint32_t plus1 = Tn & Tp, minus1 = Tn & ~Tp;
                const uint32_t plus0 = Sn & Sp, minus0 = Sn & ~Sp;
                rowpart = __popc(plus1) + __popc(plus0) - __popc(minus1) - __popc(minus0);
                accQ += __popc(Tn) + __popc(Sn);
                const bool odd = y & 1;
                vcount_add(ce_p, odd ? plus1 : plus0);
                vcount_add(co_p, odd ? plus0 : plus1);
                vcount_add(ce_m, odd ? minus1 : minus0);
                vcount_add(co_m, odd ? minus0 : minus1);
                Un = Sn;
                Sn = Dn;
                Up = Sp;
                Sp = Dp;
            }
            accM += rowpart;
        }
        const int rs = warp_sum32(rowpart);
        if ((threadIdx.x & 31) == 0 && y < y1)
            atomicAdd(&s_row[y - y0], rs);
    }
    if (MODEL == 0)
        accQ = active ? 64 * (y1 - y0) : 0;
    accB = warp_sum64(accB);
    accM = warp_sum64(accM);
    accQ = warp_sum64(accQ);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(reinterpret_cast<unsigned long long *>(rec_hdr + 1), (unsigned long long)accB);
        atomicAdd(reinterpret_cast<unsigned long long *>(rec_hdr + 2), (unsigned long long)accM);
        atomicAdd(reinterpret_cast<unsigned long long *>(rec_hdr + 3), (unsigned long long)accQ);
    }
    if (active) {
        const int rows = (int)(y1 - y0);
        // rows of each column parity in the band: even columns take colour 0
        // on even rows and colour 1 on odd rows, so every column gets one
        // site per row.
#pragma unroll 4
        for (int b = 0; b < 32; ++b) {
            const int64_t xe = 2 * (32 * wc + b);
            int ve, vo;
            if (MODEL == 0) {
                ve = 2 * vcount_get(ce_p, b) - rows;
                vo = 2 * vcount_get(co_p, b) - rows;
            } else {
                ve = vcount_get(ce_p, b) - vcount_get(ce_m, b);
                vo = vcount_get(co_p, b) - vcount_get(co_m, b);
            }
            if (ve)
                atomicAdd(&C[xe], ve);
            if (vo)
                atomicAdd(&C[xe + 1], vo);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < (int)(y1 - y0); i += blockDim.x)
        if (s_row[i])
            atomicAdd(&R[y0 + i], s_row[i]);
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

// Rows per thread for a sweep launch: enough threads to fill the GPU a few
// times over, at most 64 rows per band.
int sweep_band(int64_t L, int64_t threads_per_row)
{
    int H = 64;
    while (H > 1 && (L / H) * threads_per_row < 148LL * 2048)
        H >>= 1;
    return H;
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
    const dim3 grid((unsigned)((tpr + kSweepThreads - 1) / kSweepThreads),
                    (unsigned)((pl.L + H - 1) / H));
    k_ising_half<V><<<grid, kSweepThreads, 0, st>>>(tgt, nbr, pl.L, pl.W, colour, H, ph, thr);
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
    const int H = sweep_band(pl.L, tpr);
    const dim3 grid((unsigned)((tpr + kSweepThreads - 1) / kSweepThreads),
                    (unsigned)((pl.L + H - 1) / H));
    k_bc_half<V><<<grid, kSweepThreads, 0, st>>>(tn, tp, nn, np, pl.L, pl.W, colour, H, ph, tab);
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

cudaError_t launch_half_sweep(const Planes &pl, int colour, const PhiloxLaunch &ph,
                              const IsingThr &ithr, const BcTable *btab, cudaStream_t st)
{
    const int V = (pl.W % 4 == 0) ? 4 : (pl.W % 2 == 0 ? 2 : 1);
    if (pl.model == 0) {
        if (V == 4)
            return launch_ising<4>(pl, colour, ph, ithr, st);
        if (V == 2)
            return launch_ising<2>(pl, colour, ph, ithr, st);
        return launch_ising<1>(pl, colour, ph, ithr, st);
    }
    if (V == 4)
        return launch_bc<4>(pl, colour, ph, *btab, st);
    if (V == 2)
        return launch_bc<2>(pl, colour, ph, *btab, st);
    return launch_bc<1>(pl, colour, ph, *btab, st);
}

cudaError_t launch_measure(const Planes &pl, void *record, int64_t sweep, cudaStream_t st)
{
    int64_t *hdr = reinterpret_cast<int64_t *>(record);
    int32_t *R = reinterpret_cast<int32_t *>(hdr + 4);
    int32_t *C = R + pl.L;
    const int H = (int)(pl.L < kMeasureBand ? pl.L : kMeasureBand);
    const dim3 grid((unsigned)((pl.W + kMeasureThreads - 1) / kMeasureThreads),
                    (unsigned)((pl.L + H - 1) / H));
    if (pl.model == 0)
        k_measure<0><<<grid, kMeasureThreads, 0, st>>>(pl, H, hdr, R, C, sweep);
    else
        k_measure<1><<<grid, kMeasureThreads, 0, st>>>(pl, H, hdr, R, C, sweep);
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
