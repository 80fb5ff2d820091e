// isg_sweep_core.cuh -- the per-word Metropolis update shared by the global
// half-sweep kernels (isg_kernels.cu) and the shared-memory ensemble kernel
// (isg_ensemble.cu).
//
// A "word" is 32 same-colour sites of one row (bit b = same-colour index
// 32 w + b).  Its four neighbour words come from the other colour's plane:
// up (row y-1), down (row y+1), same (row y) and side (row y shifted by one
// site; see side_word).  q0 = j0 >> 2 is the Philox counter of its first
// site, j0 = y L/2 + 32 w; the eight Philox calls of the word use q0 .. q0+7.
#pragma once

#include <cstdint>

#include "isg_internal.h"
#include "isg_philox.cuh"

namespace isg {

// The side neighbour word: for parity (c ^ y) & 1 == 0 each site's other
// horizontal neighbour is one site to the left (bit b-1, or bit 31 of the
// previous word `edge`); for parity 1 one site to the right (bit b+1, or
// bit 0 of the next word).
__device__ __forceinline__ uint32_t side_word(uint32_t same, uint32_t edge, int parity)
{
    return parity == 0 ? (same << 1) | (edge >> 31) : (same >> 1) | (edge << 31);
}

// acc * 2 + (u >= thr): the compare is the borrow of u - thr, shifted into the
// accumulator by an add-with-carry -- two integer instructions per compare.
__device__ __forceinline__ uint32_t shift_in_not_below(uint32_t acc, uint32_t u, uint32_t thr)
{
    uint32_t out;
    asm("{\n\t.reg .u32 d;\n\tsub.cc.u32 d, %1, %2;\n\taddc.u32 %0, %3, %3;\n\t}"
        : "=r"(out)
        : "r"(u), "r"(thr), "r"(acc));
    return out;
}

// Launch-uniform Philox constants for counter words (w2, w3) -- the device
// twin of the host's philox_launch_consts, for kernels whose key or sweep
// index is not a launch parameter.
__device__ __forceinline__ PhiloxLaunch philox_consts_device(uint64_t seed, uint32_t w2, uint32_t w3)
{
    PhiloxLaunch pc;
    const uint32_t key0 = (uint32_t)seed, key1 = (uint32_t)(seed >> 32);
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        pc.rk0[r] = key0 + (uint32_t)r * kPhiloxW0;
        pc.rk1[r] = key1 + (uint32_t)r * kPhiloxW1;
    }
    const uint64_t m1w2 = (uint64_t)kPhiloxM1 * (uint64_t)w2;
    pc.r0_c0 = (uint32_t)(m1w2 >> 32) ^ pc.rk0[0];
    pc.r0_c2x = w3 ^ pc.rk1[0];
    pc.r1_c0x = (uint32_t)m1w2 ^ pc.rk0[1];
    return pc;
}

// Ising flip mask of a target word from its reject masks (bit set iff the
// site's word is >= thr4 / thr8) and its four neighbour words.  A site with
// c anti-aligned neighbours has dE = 8 - 4c (Eq. (1), J = 1): c >= 2 always
// flips, c = 1 flips iff u < thr4, c = 0 iff u < thr8.
__device__ __forceinline__ uint32_t ising_flips(uint32_t t, uint32_t up, uint32_t dn, uint32_t same,
                                                uint32_t side, uint32_t r4, uint32_t r8,
                                                const IsingThr &thr)
{
    const uint32_t a4 = ~r4 | thr.full4;
    const uint32_t a8 = ~r8 | thr.full8;
    // anti-aligned neighbour indicators and their bit-sliced count
    const uint32_t a = t ^ up, b = t ^ dn, d = t ^ same, e = t ^ side;
    const uint32_t s1 = a ^ b ^ d;
    const uint32_t c1 = (a & b) | (d & (a ^ b));
    const uint32_t s = s1 ^ e;  // count = s + 2 (c1 + c2)
    const uint32_t c2 = s1 & e;
    const uint32_t ge2 = c1 | c2;  // dE <= 0: always flip
    return ge2 | (~ge2 & ((s & a4) | (~s & a8)));
}

// Ising: new target word (one word at a time; the shared-memory ensemble).
__device__ __forceinline__ uint32_t ising_word_update(uint32_t t, uint32_t up, uint32_t dn,
                                                      uint32_t same, uint32_t side, uint64_t q0,
                                                      const PhiloxLaunch &pc, const IsingThr &thr)
{
    const PhiloxWordPart wp = philox_word_part(pc, (uint32_t)(q0 >> 32));
    // reject masks, bit b set iff site b's word >= the threshold: one chain
    // over the 32 sites, site 31 first, so no per-call merge is needed
    uint32_t r4 = 0, r8 = 0;
#pragma unroll
    for (int i = 7; i >= 0; --i) {
        uint32_t r[4];
        philox_site4(pc, wp, (uint32_t)q0 + i, r[0], r[1], r[2], r[3]);
#pragma unroll
        for (int k = 3; k >= 0; --k) {
            r4 = shift_in_not_below(r4, r[k], thr.thr4);
            r8 = shift_in_not_below(r8, r[k], thr.thr8);
        }
    }
    return t ^ ising_flips(t, up, dn, same, side, r4, r8, thr);
}

// Ising: N consecutive target words of one row (counters q0, q0 + 8, ...),
// their Philox calls and compare chains interleaved so that each thread
// has N independent chains in flight (four words: 1.7% faster than one
// after another at L = 2^20).
template <int N>
__device__ __forceinline__ void ising_words_update(uint32_t (&t)[N], const uint32_t (&up)[N],
                                                   const uint32_t (&dn)[N], const uint32_t (&same)[N],
                                                   const uint32_t (&side)[N], uint64_t q0,
                                                   const PhiloxLaunch &pc, const IsingThr &thr)
{
    PhiloxWordPart wp[N];
    uint32_t r4[N], r8[N];
#pragma unroll
    for (int v = 0; v < N; ++v) {
        wp[v] = philox_word_part(pc, (uint32_t)((q0 + 8u * v) >> 32));
        r4[v] = r8[v] = 0;
    }
#pragma unroll
    for (int i = 7; i >= 0; --i) {
        uint32_t r[N][4];
#pragma unroll
        for (int v = 0; v < N; ++v)
            philox_site4(pc, wp[v], (uint32_t)(q0 + 8u * v) + i, r[v][0], r[v][1], r[v][2], r[v][3]);
#pragma unroll
        for (int k = 3; k >= 0; --k) {
#pragma unroll
            for (int v = 0; v < N; ++v) {
                r4[v] = shift_in_not_below(r4[v], r[v][k], thr.thr4);
                r8[v] = shift_in_not_below(r8[v], r[v][k], thr.thr8);
            }
        }
    }
#pragma unroll
    for (int v = 0; v < N; ++v)
        t[v] ^= ising_flips(t[v], up[v], dn[v], same[v], side[v], r4[v], r8[v], thr);
}

__device__ __forceinline__ void full_add(uint32_t a, uint32_t b, uint32_t c, uint32_t &s,
                                         uint32_t &cy)
{
    s = a ^ b ^ c;
    cy = (a & b) | (c & (a ^ b));
}

// Blume-Capel per-site threshold lookup.  A site's table entry (BcTable,
// bc_entry) has the bits (g0, g1, g2, p, n, g3, b): the field g = h + 4 in
// four bits, the spin planes p, n and the proposal bit b = u & 1.  As a byte
// offset into the u32 table that is 4 * (low six bits) + 256 b.
//
// The six planes g0..g2, p, n, g3 are known before the random numbers.
// Their bits become one byte per site -- plane bits at byte bits 2..7, so
// the byte is already the entry's offset -- by transposing, within each byte
// column, the bit matrix of 8 plane words x 32 sites: three exchange stages,
// each swapping one bit of the word index with one bit of the bit position
// between pairs of words.  Site s = 4i + k (Philox call i, output word k)
// then sits in word 2k + (i & 1), byte i >> 1.  Per site one byte permute
// joins the index byte with b at bit 8.  (Two more stages that gathered each
// call's four sites into one word cost 16 byte permutes per word for
// nothing: the byte permute picks any byte of any word.)

// Exchange between words a (index bit 0) and c (index bit 1) of the
// position bit of value d (mask m: positions where that bit is 0): a's bits
// at the positions outside m trade places with c's bits d lower.  (A
// select-by-mask form with one op fewer per pair measured 1% slower.)
__device__ __forceinline__ void bit_exchange(uint32_t &a, uint32_t &c, int d, uint32_t m)
{
    const uint32_t t = ((a >> d) ^ c) & m;
    c ^= t;
    a ^= t << d;
}

// Index bytes of the 32 sites: site 4i + k in byte i >> 1 of o[2k + (i & 1)],
// bits 2..7 = (g0, g1, g2, p, n, g3).  The word index starts as the byte bit
// each plane is headed for, in the order the stages leave it (plane word j
// ends at byte bit 4 (j & 1) + 2 ((j >> 2) & 1) + ((j >> 1) & 1)), so words
// 0 and 2, headed for bits 0 and 1, start at zero.
__device__ __forceinline__ void bc_index_bytes(uint32_t g0, uint32_t g1, uint32_t g2, uint32_t g3,
                                               uint32_t p, uint32_t n, uint32_t (&o)[8])
{
    o[1] = g2;
    o[3] = p;
    o[5] = n;
    o[7] = g3;
    // word bit 2 <-> position bit 1 (the partners of g0 and g1 are zero)
    o[0] = (g0 << 2) & 0xCCCCCCCCu;
    o[4] = g0 & 0xCCCCCCCCu;
    o[2] = (g1 << 2) & 0xCCCCCCCCu;
    o[6] = g1 & 0xCCCCCCCCu;
    bit_exchange(o[1], o[5], 2, 0x33333333u);
    bit_exchange(o[3], o[7], 2, 0x33333333u);
    // word bit 1 <-> position bit 0
    bit_exchange(o[0], o[2], 1, 0x55555555u);
    bit_exchange(o[1], o[3], 1, 0x55555555u);
    bit_exchange(o[4], o[6], 1, 0x55555555u);
    bit_exchange(o[5], o[7], 1, 0x55555555u);
    // word bit 0 <-> position bit 2
    bit_exchange(o[0], o[1], 4, 0x0F0F0F0Fu);
    bit_exchange(o[2], o[3], 4, 0x0F0F0F0Fu);
    bit_exchange(o[4], o[5], 4, 0x0F0F0F0Fu);
    bit_exchange(o[6], o[7], 4, 0x0F0F0F0Fu);
}

// Blume-Capel: new (n, p) target words.  Neighbour planes nbn/nbp hold the
// up, down, same and side words.  The field h + 4 = #(+1 neighbours) +
// #(neighbours != -1) is summed bit-sliced into g0..g3.  kFull: a site
// accepts iff u <= its entry; otherwise iff (u >> 1) < its entry (BcTable).
// Proposal: p' = b & ~(n & p), n' = ~n | (p ^ b) with b = u & 1.
template <bool kFull>
__device__ __forceinline__ void bc_word_update(uint32_t &n, uint32_t &p, const uint32_t (&nbn)[4],
                                               const uint32_t (&nbp)[4], uint64_t q0,
                                               const PhiloxLaunch &pc, const uint32_t *s_thr)
{
    // eight indicators: s_i = +1 (n & p), s_i != -1 (~n | p)
    const uint32_t x0 = nbn[0] & nbp[0], x1 = ~nbn[0] | nbp[0];
    const uint32_t x2 = nbn[1] & nbp[1], x3 = ~nbn[1] | nbp[1];
    const uint32_t x4 = nbn[2] & nbp[2], x5 = ~nbn[2] | nbp[2];
    const uint32_t x6 = nbn[3] & nbp[3], x7 = ~nbn[3] | nbp[3];
    uint32_t sa, ca, sb, cb, sc, cc, se, ce;
    full_add(x0, x1, x2, sa, ca);
    full_add(x3, x4, x5, sb, cb);
    full_add(sa, sb, x6, sc, cc);
    const uint32_t g0 = sc ^ x7, cd = sc & x7;
    full_add(ca, cb, cc, se, ce);  // weight-2 column
    const uint32_t g1 = se ^ cd, cf = se & cd;
    const uint32_t g2 = ce ^ cf;  // weight-4 column
    const uint32_t g3 = ce & cf;  // only when h + 4 = 8
    uint32_t idx[8];
    bc_index_bytes(g0, g1, g2, g3, p, n, idx);

    const char *thr_bytes = reinterpret_cast<const char *>(s_thr);
    const PhiloxWordPart wp = philox_word_part(pc, (uint32_t)(q0 >> 32));
    // one chain over the 32 sites, site 31 first: acc ends with site b at
    // bit b; bits (a right funnel shift) with site b at bit 31 - b
    uint32_t acc = 0, bits = 0;
#pragma unroll
    for (int i = 7; i >= 0; --i) {
        uint32_t r[4];
        philox_site4(pc, wp, (uint32_t)q0 + i, r[0], r[1], r[2], r[3]);
#pragma unroll
        for (int kk = 3; kk >= 0; --kk) {
            // the site's entry offset (byte i >> 1 of idx[2 kk + (i & 1)]) and
            // bit 0 of u (b) at bit 8
            const uint32_t off =
                __byte_perm(idx[2 * kk + (i & 1)], r[kk], 0x0040u | (uint32_t)(i >> 1)) & 0x1FCu;
            const uint32_t thr = *reinterpret_cast<const uint32_t *>(thr_bytes + off);
            if (kFull)
                acc = shift_in_not_below(acc, thr, r[kk]);       // + (entry >= u): accept
            else
                acc = shift_in_not_below(acc, r[kk] >> 1, thr);  // + (v >= entry): reject
            bits = __funnelshift_r(bits, r[kk], 1);
        }
    }
    const uint32_t accept = kFull ? acc : ~acc;
    bits = __brev(bits);
    const uint32_t np2 = bits & ~(n & p);
    const uint32_t nn2 = ~n | (p ^ bits);
    const uint32_t n_old = n, p_old = p;
    n = n_old ^ (accept & (n_old ^ nn2));
    p = p_old ^ (accept & (p_old ^ np2));
}

// Blume-Capel, two target words of one row side by side: the same update as
// bc_word_update, with the Philox calls and per-site steps of the two words
// interleaved, so that each warp has two independent chains in flight
// (16 warps per SM at 128 registers this way beat 24 warps at 80 registers
// one word at a time by 2.7%).
template <bool kFull>
__device__ __forceinline__ void bc_word_update2(uint32_t (&n)[2], uint32_t (&p)[2],
                                                const uint32_t (&nbn)[2][4], const uint32_t (&nbp)[2][4],
                                                uint64_t q0a, uint64_t q0b, const PhiloxLaunch &pc,
                                                const uint32_t *s_thr)
{
    uint32_t idx[2][8];
#pragma unroll
    for (int v = 0; v < 2; ++v) {
        const uint32_t x0 = nbn[v][0] & nbp[v][0], x1 = ~nbn[v][0] | nbp[v][0];
        const uint32_t x2 = nbn[v][1] & nbp[v][1], x3 = ~nbn[v][1] | nbp[v][1];
        const uint32_t x4 = nbn[v][2] & nbp[v][2], x5 = ~nbn[v][2] | nbp[v][2];
        const uint32_t x6 = nbn[v][3] & nbp[v][3], x7 = ~nbn[v][3] | nbp[v][3];
        uint32_t sa, ca, sb, cb, sc, cc, se, ce;
        full_add(x0, x1, x2, sa, ca);
        full_add(x3, x4, x5, sb, cb);
        full_add(sa, sb, x6, sc, cc);
        const uint32_t g0 = sc ^ x7, cd = sc & x7;
        full_add(ca, cb, cc, se, ce);
        const uint32_t g1 = se ^ cd, cf = se & cd;
        const uint32_t g2 = ce ^ cf;
        const uint32_t g3 = ce & cf;
        bc_index_bytes(g0, g1, g2, g3, p[v], n[v], idx[v]);
    }
    const char *thr_bytes = reinterpret_cast<const char *>(s_thr);
    const PhiloxWordPart wpa = philox_word_part(pc, (uint32_t)(q0a >> 32));
    const PhiloxWordPart wpb = philox_word_part(pc, (uint32_t)(q0b >> 32));
    uint32_t acc[2] = {0, 0}, bits[2] = {0, 0};
#pragma unroll
    for (int i = 7; i >= 0; --i) {
        uint32_t r[2][4];
        philox_site4(pc, wpa, (uint32_t)q0a + i, r[0][0], r[0][1], r[0][2], r[0][3]);
        philox_site4(pc, wpb, (uint32_t)q0b + i, r[1][0], r[1][1], r[1][2], r[1][3]);
#pragma unroll
        for (int kk = 3; kk >= 0; --kk) {
#pragma unroll
            for (int v = 0; v < 2; ++v) {
                const uint32_t off =
                    __byte_perm(idx[v][2 * kk + (i & 1)], r[v][kk], 0x0040u | (uint32_t)(i >> 1)) & 0x1FCu;
                const uint32_t thr = *reinterpret_cast<const uint32_t *>(thr_bytes + off);
                if (kFull)
                    acc[v] = shift_in_not_below(acc[v], thr, r[v][kk]);
                else
                    acc[v] = shift_in_not_below(acc[v], r[v][kk] >> 1, thr);
                bits[v] = __funnelshift_r(bits[v], r[v][kk], 1);
            }
        }
    }
#pragma unroll
    for (int v = 0; v < 2; ++v) {
        const uint32_t accept = kFull ? acc[v] : ~acc[v];
        const uint32_t b = __brev(bits[v]);
        const uint32_t np2 = b & ~(n[v] & p[v]);
        const uint32_t nn2 = ~n[v] | (p[v] ^ b);
        const uint32_t n_old = n[v], p_old = p[v];
        n[v] = n_old ^ (accept & (n_old ^ nn2));
        p[v] = p_old ^ (accept & (p_old ^ np2));
    }
}

}  // namespace isg
