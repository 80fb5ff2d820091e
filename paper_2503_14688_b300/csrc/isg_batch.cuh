// isg_batch.cuh -- the persistent shared-memory kernel that sweeps many
// independent lattices in one launch, shared by the replica ensemble
// (isg_ensemble.cu) and the request server (isg_server.cu).
//
// Each CTA takes whole lattices from a global work counter (in the order the
// host gives, largest first), copies the lattice's spin planes into shared
// memory, runs its sweeps there with a barrier between half-sweeps -- no
// wait on any other CTA -- records observables, and writes the planes back.
// Once the counter reaches the lattices that fit half the CTA's shared
// memory, the CTA splits into two teams of half its threads, each with its
// own half of the shared memory and its own named barrier, which take
// lattices independently: while one team runs the last, partly idle round of
// a half-sweep, the other keeps the SM's pipes busy.  Included by one
// translation unit each (anonymous namespace).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "isg.h"
#include "isg_internal.h"
#include "isg_philox.cuh"
#include "isg_sweep_core.cuh"

namespace isg {
namespace {

// Dynamic shared memory the batch kernel may ask for: the sm_100-family
// per-block opt-in maximum (227 KiB) less room for its static shared memory.
constexpr int kBatchSmemMax = 227 * 1024 - 1024;

constexpr int kCounterBits = 8;  // column counters in the shared-memory measure

struct EnsItem {
    uint64_t seed;
    uint32_t *planes;     // the replica's planes in global memory
    uint64_t rec_offset;  // byte offset of its record inside a record row
    int32_t L;
    int32_t model;
    // own == 1: this item's sweep range, thresholds and record buffer below
    // replace the launch-wide ones of EnsArgs (independent requests)
    int32_t own;
    uint32_t t0;
    int32_t nsweeps;
    int32_t record_every;
    const IsingThr *ithr;
    const BcTable *btab;
    uint8_t *rec_base;    // record k goes to rec_base + ((rec_row0 + k) % rec_cap) * rec_pitch
    uint64_t rec_pitch;
    int32_t rec_cap;
    int32_t rec_row0;
};

struct EnsArgs {
    const EnsItem *items;
    const int32_t *order;  // replica indices, shared-memory path, largest first
    int32_t n_order;
    int32_t *counter;      // work counter, zero at launch
    const IsingThr *ithr;  // per sweep of this launch
    const BcTable *btab;   // per sweep of this launch (Blume-Capel), may be null
    uint8_t *rec_ring;
    uint64_t row_bytes;
    int32_t rec_cap;
    int32_t rec_row0;      // ring row of this launch's first record
    uint32_t t0;
    int32_t nsweeps;
    int32_t record_every;
    // half_words > 0: order entries from split_from on need at most
    // half_words 32-bit words of shared memory and run on half-CTA teams
    uint32_t half_words;
    int32_t split_from;
};

// The threads that work on one lattice.  kHalf = false: the whole CTA,
// synchronised by __syncthreads.  kHalf = true: one of two teams of half the
// CTA (team 0 = the lower threads), synchronised by named barrier 1 + team.
// Every field derives from threadIdx.x and blockDim.x, so the compiler can
// recompute it instead of keeping it in a register.
template <bool kHalf>
struct Team {
    __device__ __forceinline__ int nt() const { return kHalf ? (int)(blockDim.x >> 1) : (int)blockDim.x; }
    __device__ __forceinline__ int team() const { return kHalf ? (int)(threadIdx.x >= (blockDim.x >> 1)) : 0; }
    __device__ __forceinline__ int tid() const { return (int)threadIdx.x - team() * nt(); }
    __device__ __forceinline__ void sync() const
    {
        if (kHalf)
            asm volatile("bar.sync %0, %1;" ::"r"(1 + team()), "r"(nt()) : "memory");
        else
            __syncthreads();
    }
};

size_t smem_bytes_for(int32_t model, int64_t L)
{
    const size_t planes = (size_t)L * (size_t)L / (model == ISG_ISING ? 8 : 4);
    return planes + 8 * (size_t)L + 4 * kBcTableSize + 64;
}

// ---------------------------------------------------------------------------
// Observables of the replica held in shared memory (after a full sweep).
// ---------------------------------------------------------------------------
template <int MODEL, bool kHalf>
__device__ void smem_measure(const Team<kHalf> &team, const uint32_t *P, int L, int W, int32_t *R_s,
                             int32_t *C_s, unsigned long long *acc, uint8_t *rec, int64_t sweep)
{
    const int tid = team.tid(), nt = team.nt();
    const int LW = L * W;
    for (int i = tid; i < L; i += nt) {
        R_s[i] = 0;
        C_s[i] = 0;
    }
    if (tid < 3)
        acc[tid] = 0;
    team.sync();
    const uint32_t *p0 = MODEL == 0 ? P : P + LW;
    const uint32_t *p1 = MODEL == 0 ? P + LW : P + 3 * LW;
    const uint32_t *n0 = P, *n1 = P + 2 * LW;
    int b = 0, m = 0, q = 0;
    // bonds, magnetisation, row sums: one colour-1 word with its colour-0 neighbours
    for (int i = tid; i < LW; i += nt) {
        const int y = i / W, w = i - y * W;
        const int yu = y == 0 ? L - 1 : y - 1, yd = y + 1 == L ? 0 : y + 1;
        const int par = (1 ^ y) & 1;
        const int ew = par == 0 ? (w == 0 ? W - 1 : w - 1) : (w + 1 == W ? 0 : w + 1);
        const uint32_t Tp = p1[i], Sp = p0[i];
        const uint32_t Xp = side_word(Sp, p0[y * W + ew], par);
        const uint32_t Up = p0[yu * W + w], Dp = p0[yd * W + w];
        int rp;
        if (MODEL == 0) {
            const int anti = __popc(Tp ^ Up) + __popc(Tp ^ Dp) + __popc(Tp ^ Sp) + __popc(Tp ^ Xp);
            b += 128 - 2 * anti;
            rp = 2 * (__popc(Tp) + __popc(Sp)) - 64;
        } else {
            const uint32_t Tn = n1[i], Sn = n0[i];
            const uint32_t Xn = side_word(Sn, n0[y * W + ew], par);
            const uint32_t nb[4] = {n0[yu * W + w], n0[yd * W + w], Sn, Xn};
            const uint32_t pb[4] = {Up, Dp, Sp, Xp};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t both = Tn & nb[k];
                b += __popc(both) - 2 * __popc(both & (Tp ^ pb[k]));
            }
            rp = __popc(Tn & Tp) + __popc(Sn & Sp) - __popc(Tn & ~Tp) - __popc(Sn & ~Sp);
            q += __popc(Tn) + __popc(Sn);
        }
        m += rp;
        atomicAdd(&R_s[y], rp);
    }
    if (MODEL == 0)
        q = 0;
    b = __reduce_add_sync(0xFFFFFFFFu, b);
    m = __reduce_add_sync(0xFFFFFFFFu, m);
    q = __reduce_add_sync(0xFFFFFFFFu, q);
    if ((tid & 31) == 0) {
        atomicAdd(&acc[0], (unsigned long long)(long long)b);
        atomicAdd(&acc[1], (unsigned long long)(long long)m);
        atomicAdd(&acc[2], (unsigned long long)(long long)q);
    }
    // column sums: thread (g, w) counts rows [g R_g, (g+1) R_g) of word column w
    const int G = nt / W > 0 ? nt / W : 1;
    const int Rg = (L + G - 1) / G;
    if (tid < G * W) {
        const int g = tid / W, w = tid - g * W;
        const int ya = g * Rg, yb = min(L, ya + Rg);
        uint32_t ep[kCounterBits] = {}, op[kCounterBits] = {};
        uint32_t em[kCounterBits] = {}, om[kCounterBits] = {};
        for (int y = ya; y < yb; ++y) {
            const bool odd = y & 1;
            uint32_t e_p, o_p, e_m = 0, o_m = 0;
            if (MODEL == 0) {
                e_p = odd ? p1[y * W + w] : p0[y * W + w];
                o_p = odd ? p0[y * W + w] : p1[y * W + w];
            } else {
                const uint32_t a_n = n0[y * W + w], a_p = p0[y * W + w];
                const uint32_t c_n = n1[y * W + w], c_p = p1[y * W + w];
                const uint32_t plus0 = a_n & a_p, minus0 = a_n & ~a_p;
                const uint32_t plus1 = c_n & c_p, minus1 = c_n & ~c_p;
                e_p = odd ? plus1 : plus0;
                o_p = odd ? plus0 : plus1;
                e_m = odd ? minus1 : minus0;
                o_m = odd ? minus0 : minus1;
            }
            uint32_t x;
            x = e_p;
            for (int l = 0; l < kCounterBits && x; ++l) { const uint32_t c = ep[l] & x; ep[l] ^= x; x = c; }
            x = o_p;
            for (int l = 0; l < kCounterBits && x; ++l) { const uint32_t c = op[l] & x; op[l] ^= x; x = c; }
            if (MODEL == 1) {
                x = e_m;
                for (int l = 0; l < kCounterBits && x; ++l) { const uint32_t c = em[l] & x; em[l] ^= x; x = c; }
                x = o_m;
                for (int l = 0; l < kCounterBits && x; ++l) { const uint32_t c = om[l] & x; om[l] ^= x; x = c; }
            }
        }
        const int rows = yb > ya ? yb - ya : 0;
        for (int bit = 0; bit < 32; ++bit) {
            int ce = 0, co = 0, cem = 0, com = 0;
#pragma unroll
            for (int l = 0; l < kCounterBits; ++l) {
                ce |= (int)((ep[l] >> bit) & 1u) << l;
                co |= (int)((op[l] >> bit) & 1u) << l;
                if (MODEL == 1) {
                    cem |= (int)((em[l] >> bit) & 1u) << l;
                    com |= (int)((om[l] >> bit) & 1u) << l;
                }
            }
            const int x = 2 * (32 * w + bit);
            const int ve = MODEL == 0 ? 2 * ce - rows : ce - cem;
            const int vo = MODEL == 0 ? 2 * co - rows : co - com;
            if (ve)
                atomicAdd(&C_s[x], ve);
            if (vo)
                atomicAdd(&C_s[x + 1], vo);
        }
    }
    team.sync();
    int64_t *hdr = reinterpret_cast<int64_t *>(rec);
    int32_t *R = reinterpret_cast<int32_t *>(rec + 32);
    int32_t *C = R + L;
    if (tid == 0) {
        hdr[0] = sweep;
        hdr[1] = (int64_t)acc[0];
        hdr[2] = (int64_t)acc[1];
        hdr[3] = MODEL == 0 ? (int64_t)L * L : (int64_t)acc[2];
    }
    for (int i = tid; i < L; i += nt) {
        R[i] = R_s[i];
        C[i] = C_s[i];
    }
    team.sync();
}

// One Blume-Capel colour of a replica held in shared memory; the threads
// walk its words from (y, w) in steps of (dy, dw).
template <bool kFull>
__device__ __forceinline__ void bc_smem_colour(uint32_t *P, int L, int W, int c, int y, int w,
                                               int dy, int dw, uint64_t qrow,
                                               const PhiloxLaunch &pc, const uint32_t *s_thr)
{
    const int LW = L * W;
    const uint32_t *nbn = P + 2 * (1 - c) * LW, *nbp = nbn + LW;
    uint32_t *tn = P + 2 * c * LW, *tp = tn + LW;
    while (y < L) {
        const int yu = y == 0 ? L - 1 : y - 1, yd = y + 1 == L ? 0 : y + 1;
        const int par = (c ^ y) & 1;
        const int ew = par == 0 ? (w == 0 ? W - 1 : w - 1) : (w + 1 == W ? 0 : w + 1);
        const uint32_t sn = nbn[y * W + w], sp = nbp[y * W + w];
        const uint32_t nn[4] = {nbn[yu * W + w], nbn[yd * W + w], sn,
                                side_word(sn, nbn[y * W + ew], par)};
        const uint32_t pp[4] = {nbp[yu * W + w], nbp[yd * W + w], sp,
                                side_word(sp, nbp[y * W + ew], par)};
        uint32_t n = tn[y * W + w], p = tp[y * W + w];
        const uint64_t q0 = (uint64_t)y * qrow + 8u * (uint64_t)w;
        bc_word_update<kFull>(n, p, nn, pp, q0, pc, s_thr);
        tn[y * W + w] = n;
        tp[y * W + w] = p;
        w += dw;
        y += dy;
        if (w >= W) {
            w -= W;
            ++y;
        }
    }
}

template <int MODEL, bool kHalf>
__device__ void run_replica(const EnsItem &it, const EnsArgs &a, uint32_t *smem, const Team<kHalf> &team)
{
    const int tid = team.tid(), nt = team.nt();
    const int L = it.L, W = L / 64, LW = L * W;
    const int nplanes = MODEL == 0 ? 2 : 4;
    uint32_t *P = smem;
    int32_t *R_s = reinterpret_cast<int32_t *>(P + nplanes * LW);
    int32_t *C_s = R_s + L;
    uint32_t *s_thr = reinterpret_cast<uint32_t *>(C_s + L);
    unsigned long long *acc = reinterpret_cast<unsigned long long *>(s_thr + kBcTableSize);

    const uint4 *g4 = reinterpret_cast<const uint4 *>(it.planes);
    uint4 *s4 = reinterpret_cast<uint4 *>(P);
    for (int i = tid; i < nplanes * LW / 4; i += nt)
        s4[i] = g4[i];
    team.sync();

    const int dy = nt / W, dw = nt - (nt / W) * W;
    const uint64_t qrow = (uint64_t)(L / 8);
    const uint32_t t0 = it.own ? it.t0 : a.t0;
    const int nsweeps = it.own ? it.nsweeps : a.nsweeps;
    const int record_every = it.own ? it.record_every : a.record_every;
    const IsingThr *ithr = it.own ? it.ithr : a.ithr;
    const BcTable *btab = it.own ? it.btab : a.btab;
    uint8_t *rec_base = it.own ? it.rec_base : a.rec_ring + it.rec_offset;
    const uint64_t rec_pitch = it.own ? it.rec_pitch : a.row_bytes;
    const int rec_cap = it.own ? it.rec_cap : a.rec_cap;
    const int rec_row0 = it.own ? it.rec_row0 : a.rec_row0;
    for (int s = 0; s < nsweeps; ++s) {
        const uint32_t t = t0 + (uint32_t)s;
        bool bc_full = false;
        if (MODEL == 1) {
            for (int i = tid; i < kBcTableSize; i += nt)
                s_thr[i] = btab[s].thr[i];
            bc_full = btab[s].full != 0;
            team.sync();
        }
        for (int c = 0; c < 2; ++c) {
            const PhiloxLaunch pc = philox_consts_device(it.seed, t, (uint32_t)c);
            int y = tid / W, w = tid - (tid / W) * W;
            if (MODEL == 0) {
                const IsingThr thr = ithr[s];
                const uint32_t *nb = P + (1 - c) * LW;
                uint32_t *tg = P + c * LW;
                while (y < L) {
                    const int yu = y == 0 ? L - 1 : y - 1, yd = y + 1 == L ? 0 : y + 1;
                    const int par = (c ^ y) & 1;
                    const int ew = par == 0 ? (w == 0 ? W - 1 : w - 1) : (w + 1 == W ? 0 : w + 1);
                    const uint32_t same = nb[y * W + w];
                    const uint32_t X = side_word(same, nb[y * W + ew], par);
                    const uint64_t q0 = (uint64_t)y * qrow + 8u * (uint64_t)w;
                    tg[y * W + w] = ising_word_update(tg[y * W + w], nb[yu * W + w], nb[yd * W + w],
                                                      same, X, q0, pc, thr);
                    w += dw;
                    y += dy;
                    if (w >= W) {
                        w -= W;
                        ++y;
                    }
                }
            } else if (bc_full) {
                bc_smem_colour<true>(P, L, W, c, y, w, dy, dw, qrow, pc, s_thr);
            } else {
                bc_smem_colour<false>(P, L, W, c, y, w, dy, dw, qrow, pc, s_thr);
            }
            team.sync();
        }
        if (record_every > 0 && (s + 1) % record_every == 0) {
            const int k = (s + 1) / record_every - 1;
            const int row = (rec_row0 + k) % rec_cap;
            uint8_t *rec = rec_base + (uint64_t)row * rec_pitch;
            smem_measure<MODEL, kHalf>(team, P, L, W, R_s, C_s, acc, rec, (int64_t)t + 1);
        }
    }
    uint4 *o4 = reinterpret_cast<uint4 *>(it.planes);
    for (int i = tid; i < nplanes * LW / 4; i += nt)
        o4[i] = s4[i];
    team.sync();
}

template <bool kHalf>
__device__ __forceinline__ void run_item(const EnsArgs &a, int item, uint32_t *smem)
{
    const EnsItem it = a.items[a.order[item]];
    const Team<kHalf> team;
    if (it.model == 0)
        run_replica<0, kHalf>(it, a, smem, team);
    else
        run_replica<1, kHalf>(it, a, smem, team);
}

__global__ void __launch_bounds__(1024, 1) k_ensemble(const EnsArgs *__restrict__ args)
{
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ int s_item[3];
    const EnsArgs a = *args;
    const bool split = a.half_words > 0 && blockDim.x % 64 == 0;
    int item;
    // whole-CTA lattices (all of them without a split)
    for (;;) {
        if (threadIdx.x == 0)
            s_item[0] = atomicAdd(a.counter, 1);
        __syncthreads();
        item = s_item[0];
        __syncthreads();
        if (item >= a.n_order)
            return;
        if (split && item >= a.split_from)
            break;
        run_item<false>(a, item, smem);
    }
    // two teams from here on; team 0 starts with the lattice just taken.
    // Control flow below is uniform within a team (the item comes from the
    // team's shared slot), so each named barrier sees all of its warps.
    const Team<true> team;
    const int g = team.team();
    uint32_t *tsm = smem + (size_t)g * a.half_words;
    int mine = g == 0 ? item : -1;
    for (;;) {
        if (mine < 0) {
            if (team.tid() == 0)
                s_item[1 + g] = atomicAdd(a.counter, 1);
            team.sync();
            mine = s_item[1 + g];
            team.sync();
        }
        if (mine >= a.n_order)
            return;
        run_item<true>(a, mine, tsm);
        mine = -1;
    }
}

}  // namespace
}  // namespace isg
