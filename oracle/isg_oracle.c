/*
 * isg_oracle.c -- the reference CPU implementation (the "oracle") of the
 * checkerboard single-spin-flip Metropolis sweep of the 2D spin-1/2 Ising and
 * spin-1 Blume-Capel models, and of the observables tracked per sweep.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * includes this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark load it.  It shares no code, header, table or constant
 * generator with the CUDA path: its Philox, its acceptance thresholds, its
 * observables and its xi_2 are written here, once, from the definitions.
 *
 * Plain and slow on purpose: one int8_t per site, one Philox evaluation per
 * site (the generator is stateless, so the four output words of a call are
 * recomputed for each of the four sites that share its counter), the update
 * rule applied literally, site by site, in the order stated below.
 *
 * Sources (the paper: "Universal exotic dynamics in critical mesoscopic
 * systems", arXiv 2503.14688):
 *   - Eq. (1): H = -J sum_<xy> s_x s_y + Delta sum_x s_x^2, s in {-1,0,+1}
 *     (Blume-Capel; Ising is s in {-1,+1}), L x L square lattice, periodic.
 *   - Introduction: the update is Metropolis, made parallel by a checkerboard
 *     decomposition (and multispin coding, which is a GPU layout matter and
 *     plays no role here).
 *   - Table I caption: the unit of time is one full-lattice Metropolis sweep.
 *   - Appendix B: the random numbers are 32-bit integers.
 *   - "Thermal protocols": a run starts from T = infinity, i.e. a fully
 *     disordered configuration.
 *   - Eqs. (2)-(3): C(r;t) and E(t) = C(1,0) + C(0,1) (the nearest-neighbour
 *     bond sum), read with the sign of the Hamiltonian (E_eq(T_c) = -sqrt 2).
 *   - Appendix B: M(k), chi(k) and the second-moment correlation length
 *     xi_2 = sqrt(chi(0)/chi(k_min) - 1) / (2 sin(pi/L)).
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   - Colour c(x,y) = (x+y) & 1; a sweep updates colour 0 then colour 1, both
 *     halves with the same beta and the same sweep index t.  Within a colour
 *     the sites are visited in row-major order and updated in place.  For even
 *     L this is exactly the parallel checkerboard (same-colour sites are never
 *     neighbours); for odd L (used only by tiny enumeration checks) it is a
 *     valid sequential Metropolis chain.
 *   - Random word of site (x,y) at sweep t: Philox4x32-10 (Salmon, Moraes,
 *     Dror & Shaw, SC'11) with key (lo32(seed), hi32(seed)) and counter
 *     (lo32(j>>2), hi32(j>>2), t, c), output word j & 3, where
 *     j = (y*L + x) >> 1 is the same-colour index.  The hot start uses the
 *     counter (lo32(j>>2), hi32(j>>2), 0, c | 2).
 *   - Acceptance of a proposal with energy change dE: always if dE <= 0; for
 *     dE > 0 Ising accepts iff (uint64)u < rne(2^32 exp(-beta dE)), and
 *     Blume-Capel iff (u >> 1) < rne(2^31 exp(-beta dE)); exp is the host FP64
 *     libm exp, rne = round to nearest even (llrint).
 *   - Blume-Capel proposal: b = u & 1 picks s' as the (b+1)-th smallest of the
 *     two values different from s (s=-1 -> {0,+1}[b], s=0 -> {-1,+1}[b],
 *     s=+1 -> {-1,0}[b]); dE = -J (s'-s) h + Delta (s'^2 - s^2), J = 1.
 *   - Hot start: Ising s = +1 iff u >= 2^31; Blume-Capel s = ((u*3) >> 32) - 1.
 *   - xi_2 is an ensemble quantity: S_0 = M^2 and S_k (the mean of |M(k)|^2
 *     over k = (2pi/L,0) and (0,2pi/L)) are averaged over replicas first.
 *     The FP64 operation order is fixed (see oracle_xi2) so that two
 *     implementations fed the same integers agree to the last bit.
 *
 * Build: gcc -O2 -fPIC -shared -fopenmp -ffp-contract=off (oracle/build.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_ISING 0
#define ORACLE_BLUME_CAPEL 1

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, written from its published definition (SC'11).            */
/* ------------------------------------------------------------------------ */

/* One Philox4x32 round: two 32x32->64 multiplies and a Feistel-like mix.   */
static void philox_round(uint32_t c[4], const uint32_t k[2])
{
    const uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    const uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    const uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
    const uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
    const uint32_t n0 = hi1 ^ c[1] ^ k[0];
    const uint32_t n1 = lo1;
    const uint32_t n2 = hi0 ^ c[3] ^ k[1];
    const uint32_t n3 = lo0;
    c[0] = n0;
    c[1] = n1;
    c[2] = n2;
    c[3] = n3;
}

/* Ten rounds; the key is bumped by the Weyl constants before rounds 2..10.  */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k[0] += 0x9E3779B9u;
            k[1] += 0xBB67AE85u;
        }
        philox_round(c, k);
    }
    out[0] = c[0];
    out[1] = c[1];
    out[2] = c[2];
    out[3] = c[3];
}

/* The 32-bit random word of same-colour index j for counter words (w2, w3). */
static uint32_t site_word(uint64_t seed, uint64_t j, uint32_t w2, uint32_t w3)
{
    const uint64_t q = j >> 2;
    const uint32_t ctr[4] = {(uint32_t)q, (uint32_t)(q >> 32), w2, w3};
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    oracle_philox4x32_10(ctr, key, out);
    return out[j & 3u];
}

uint32_t oracle_site_random(uint64_t seed, uint64_t j, uint32_t w2, uint32_t w3)
{
    return site_word(seed, j, w2, w3);
}

/* ------------------------------------------------------------------------ */
/* Acceptance thresholds (Appendix B: 32-bit integer random numbers).        */
/* ------------------------------------------------------------------------ */

/* rne(2^bits * exp(-beta dE)); only called for dE > 0.                      */
static uint64_t threshold_bits(double beta, double dE, int bits)
{
    const double p = exp(-beta * dE);
    return (uint64_t)llrint(ldexp(p, bits));
}

uint64_t oracle_threshold(double beta, double dE, int bits)
{
    if (dE <= 0.0)
        return (uint64_t)1 << bits;
    return threshold_bits(beta, dE, bits);
}

/* Energy change of the Blume-Capel move s -> s2 in local field h (J = 1).   */
static double bc_delta_energy(int s, int s2, int h, double delta)
{
    return (double)(-(s2 - s) * h) + delta * (double)(s2 * s2 - s * s);
}

/* The proposal s' picked by the bit b (the (b+1)-th smallest other value).  */
int oracle_bc_proposal(int s, int b)
{
    if (s == -1)
        return b ? +1 : 0;
    if (s == 0)
        return b ? +1 : -1;
    return b ? 0 : -1;
}

/* ------------------------------------------------------------------------ */
/* Lattice: s[y*L + x], x,y in [0,L), periodic neighbours.                   */
/* ------------------------------------------------------------------------ */

static inline int64_t up1(int64_t a, int64_t L) { return a + 1 == L ? 0 : a + 1; }
static inline int64_t dn1(int64_t a, int64_t L) { return a == 0 ? L - 1 : a - 1; }

/* Hot start: the T = infinity (beta = 0) Boltzmann measure ("Thermal
 * protocols": the direct quench starts from a fully disordered state).      */
int oracle_init_random(int8_t *s, int64_t L, int model, uint64_t seed)
{
    if (!s || L < 2 || (model != ORACLE_ISING && model != ORACLE_BLUME_CAPEL))
        return -1;
    for (int64_t y = 0; y < L; ++y) {
        for (int64_t x = 0; x < L; ++x) {
            const uint64_t idx = (uint64_t)(y * L + x);
            const uint32_t c = (uint32_t)((x + y) & 1);
            const uint32_t u = site_word(seed, idx >> 1, 0u, c | 2u);
            if (model == ORACLE_ISING)
                s[idx] = (int8_t)(u >= 0x80000000u ? 1 : -1);
            else
                s[idx] = (int8_t)((int)(((uint64_t)u * 3u) >> 32) - 1);
        }
    }
    return 0;
}

/* One Metropolis update of site (x,y) with random word u.                   */
static void update_site(int8_t *s, int64_t L, int64_t x, int64_t y, int model,
                        double beta, double delta, uint32_t u)
{
    const int64_t idx = y * L + x;
    const int si = s[idx];
    const int h = s[y * L + up1(x, L)] + s[y * L + dn1(x, L)] +
                  s[up1(y, L) * L + x] + s[dn1(y, L) * L + x];
    if (model == ORACLE_ISING) {
        /* Flip s -> -s: dE = 2 J s h (Eq. (1) with s^2 = 1).              */
        const double dE = (double)(2 * si * h);
        int accept = 1;
        if (dE > 0.0)
            accept = (uint64_t)u < threshold_bits(beta, dE, 32);
        if (accept)
            s[idx] = (int8_t)(-si);
    } else {
        const int b = (int)(u & 1u);
        const int s2 = oracle_bc_proposal(si, b);
        const double dE = bc_delta_energy(si, s2, h, delta);
        int accept = 1;
        if (dE > 0.0)
            accept = (uint64_t)(u >> 1) < threshold_bits(beta, dE, 31);
        if (accept)
            s[idx] = (int8_t)s2;
    }
}

/* Half-sweep of colour c at sweep index t: every site with (x+y)&1 == c,
 * row-major, in place.  For even L rows of one colour are independent, so
 * they may be split among threads without changing the result.             */
static void half_sweep(int8_t *s, int64_t L, int model, double beta, double delta,
                       uint64_t seed, uint64_t t, int c, int nthreads)
{
    const int par = (L % 2 == 0) && nthreads > 1;
    (void)par;
#pragma omp parallel for schedule(static) num_threads(nthreads) if (par)
    for (int64_t y = 0; y < L; ++y) {
        for (int64_t x = (int64_t)((c + y) & 1); x < L; x += 2) {
            const uint64_t j = (uint64_t)(y * L + x) >> 1;
            const uint32_t u = site_word(seed, j, (uint32_t)t, (uint32_t)c);
            update_site(s, L, x, y, model, beta, delta, u);
        }
    }
}

/* For odd L the same-colour sites of one row are not all independent of
 * each other across the periodic seam, so the visit order matters; the
 * sequential version below is the definition for any L.                     */
static void half_sweep_sequential(int8_t *s, int64_t L, int model, double beta,
                                  double delta, uint64_t seed, uint64_t t, int c)
{
    for (int64_t y = 0; y < L; ++y)
        for (int64_t x = 0; x < L; ++x)
            if (((x + y) & 1) == c) {
                const uint64_t j = (uint64_t)(y * L + x) >> 1;
                const uint32_t u = site_word(seed, j, (uint32_t)t, (uint32_t)c);
                update_site(s, L, x, y, model, beta, delta, u);
            }
}

/* ------------------------------------------------------------------------ */
/* Observables (Eqs. (2)-(3); Appendix B).                                   */
/* ------------------------------------------------------------------------ */

/* bmq[0] = B = sum_x s_x (s_{x+e1} + s_{x+e2}) (bond sum, so that the energy
 * per spin is (-J B + Delta Q) / L^2), bmq[1] = M = sum s, bmq[2] = Q =
 * sum s^2; R[y] = sum_x s(x,y), C[x] = sum_y s(x,y).  R or C may be NULL.   */
int oracle_measure(const int8_t *s, int64_t L, int64_t *bmq, int32_t *R, int32_t *C)
{
    if (!s || !bmq || L < 1)
        return -1;
    int64_t B = 0, M = 0, Q = 0;
    if (C)
        for (int64_t x = 0; x < L; ++x)
            C[x] = 0;
    for (int64_t y = 0; y < L; ++y) {
        int64_t row = 0;
        for (int64_t x = 0; x < L; ++x) {
            const int v = s[y * L + x];
            B += (int64_t)v * (s[y * L + up1(x, L)] + s[up1(y, L) * L + x]);
            M += v;
            Q += v * v;
            row += v;
            if (C)
                C[x] += v;
        }
        if (R)
            R[y] = (int32_t)row;
    }
    bmq[0] = B;
    bmq[1] = M;
    bmq[2] = Q;
    return 0;
}

/* Run n sweeps t0 .. t0+n-1 with inverse temperature betas[i] for sweep
 * t0+i.  If record_every > 0, after every sweep i with (i+1) % record_every
 * == 0 the observables are appended: rec_bmq[3*r..], rec_R[L*r..],
 * rec_C[L*r..] (rec_R / rec_C may be NULL).  nthreads > 1 splits the rows of
 * a colour among OpenMP threads (even L only; the result does not change).
 * sequential != 0 forces the row-major sequential visit order (required for
 * odd L).  Returns the number of records written, or -1 on bad arguments.   */
int64_t oracle_run(int8_t *s, int64_t L, int model, uint64_t seed, uint64_t t0,
                   int64_t n, const double *betas, double delta, int64_t record_every,
                   int64_t *rec_bmq, int32_t *rec_R, int32_t *rec_C, int nthreads,
                   int sequential)
{
    if (!s || L < 2 || n < 0 || !betas ||
        (model != ORACLE_ISING && model != ORACLE_BLUME_CAPEL))
        return -1;
    if (L % 2 != 0)
        sequential = 1;
    int64_t nrec = 0;
    for (int64_t i = 0; i < n; ++i) {
        const uint64_t t = t0 + (uint64_t)i;
        for (int c = 0; c < 2; ++c) {
            if (sequential)
                half_sweep_sequential(s, L, model, betas[i], delta, seed, t, c);
            else
                half_sweep(s, L, model, betas[i], delta, seed, t, c, nthreads);
        }
        if (record_every > 0 && (i + 1) % record_every == 0) {
            oracle_measure(s, L, rec_bmq + 3 * nrec, rec_R ? rec_R + L * nrec : NULL,
                           rec_C ? rec_C + L * nrec : NULL);
            ++nrec;
        }
    }
    return nrec;
}

/* ------------------------------------------------------------------------ */
/* Second-moment correlation length (Appendix B).                            */
/* ------------------------------------------------------------------------ */

/* Neumaier-compensated running sum.                                         */
typedef struct {
    double sum, comp;
} ksum;

static void ksum_add(ksum *a, double v)
{
    const double t = a->sum + v;
    if (fabs(a->sum) >= fabs(v))
        a->comp += (a->sum - t) + v;
    else
        a->comp += (v - t) + a->sum;
    a->sum = t;
}

static double ksum_value(const ksum *a) { return a->sum + a->comp; }

/* Twiddles w[x] = cos(2 pi x / L), v[x] = sin(2 pi x / L).  For L % 8 == 0
 * libm is called for x in [0, L/8] only and the other octants are filled by
 * the exact symmetries of cos and sin, so that e.g. w[L/4] is exactly 0;
 * otherwise libm is called for every x.                                      */
static void twiddles(int64_t L, double *w, double *v)
{
    const double two_pi = 2.0 * M_PI;
    if (L % 8 != 0) {
        for (int64_t x = 0; x < L; ++x) {
            const double a = two_pi * (double)x / (double)L;
            w[x] = cos(a);
            v[x] = sin(a);
        }
        return;
    }
    const int64_t e = L / 8, q = L / 4, h = L / 2;
    for (int64_t x = 0; x <= e; ++x) {
        const double a = two_pi * (double)x / (double)L;
        w[x] = cos(a);
        v[x] = sin(a);
    }
    for (int64_t x = e + 1; x <= q; ++x) { /* cos(pi/2 - a) = sin(a)         */
        w[x] = v[q - x];
        v[x] = w[q - x];
    }
    for (int64_t x = q + 1; x <= h; ++x) { /* cos(pi - a) = -cos(a)          */
        w[x] = -w[h - x];
        v[x] = v[h - x];
    }
    for (int64_t x = h + 1; x < L; ++x) { /* cos(2pi - a) = cos(a)           */
        w[x] = w[L - x];
        v[x] = -v[L - x];
    }
}

/* |sum_x f[x] e^{i 2 pi x / L}|^2 with compensated sums in index order.     */
static double fourier_power(const int32_t *f, int64_t L, const double *w, const double *v)
{
    ksum re = {0.0, 0.0}, im = {0.0, 0.0};
    for (int64_t x = 0; x < L; ++x) {
        ksum_add(&re, (double)f[x] * w[x]);
        ksum_add(&im, (double)f[x] * v[x]);
    }
    const double r = ksum_value(&re), i = ksum_value(&im);
    return r * r + i * i;
}

/* Ensemble xi_2 from n replicas of one sweep: M[r], R[r*L + y], C[r*L + x].
 *   S_0(r) = M_r^2 (exact, __int128), S_k(r) = (|M(k_x)|^2 + |M(k_y)|^2)/2
 *   with M(k_x) from the column sums and M(k_y) from the row sums;
 *   <S_0> = (double)(sum_r S_0(r)) / n, <S_k> = (compensated sum_r S_k) / n;
 *   xi_2 = sqrt(<S_0>/<S_k> - 1) / (2 sin(pi/L)).
 * NaN if <S_0> <= <S_k> or n < 1; +inf if <S_k> == 0 < <S_0>.               */
double oracle_xi2(int64_t n, int64_t L, const int64_t *M, const int32_t *R, const int32_t *C)
{
    if (n < 1 || L < 2 || !M || !R || !C)
        return NAN;
    double *w = (double *)malloc(sizeof(double) * (size_t)L);
    double *v = (double *)malloc(sizeof(double) * (size_t)L);
    if (!w || !v) {
        free(w);
        free(v);
        return NAN;
    }
    twiddles(L, w, v);
    __int128 s0 = 0;
    ksum sk = {0.0, 0.0};
    for (int64_t r = 0; r < n; ++r) {
        s0 += (__int128)M[r] * (__int128)M[r];
        const double px = fourier_power(C + r * L, L, w, v);
        const double py = fourier_power(R + r * L, L, w, v);
        ksum_add(&sk, 0.5 * (px + py));
    }
    free(w);
    free(v);
    const double s0avg = (double)s0 / (double)n;
    const double skavg = ksum_value(&sk) / (double)n;
    if (!(s0avg > skavg))
        return NAN;
    if (skavg == 0.0)
        return INFINITY;
    return sqrt(s0avg / skavg - 1.0) / (2.0 * sin(M_PI / (double)L));
}

/* ------------------------------------------------------------------------ */
/* Windows of a large lattice (light-cone checks).                           */
/* ------------------------------------------------------------------------ */

/* Hot start of the h x w window with corner (y0, x0) of the L x L lattice:
 * s[i*w + j] is site ((x0 + j) mod L, (y0 + i) mod L), drawn exactly as
 * oracle_init_random draws it (global colour and same-colour index).       */
int oracle_window_init(int8_t *s, int64_t h, int64_t w, int64_t y0, int64_t x0, int64_t L,
                       int model, uint64_t seed)
{
    if (!s || h < 1 || w < 1 || L < 2 || (model != ORACLE_ISING && model != ORACLE_BLUME_CAPEL))
        return -1;
    for (int64_t i = 0; i < h; ++i) {
        const int64_t y = (y0 + i) % L;
        for (int64_t j = 0; j < w; ++j) {
            const int64_t x = (x0 + j) % L;
            const uint64_t idx = (uint64_t)(y * L + x);
            const uint32_t c = (uint32_t)((x + y) & 1);
            const uint32_t u = site_word(seed, idx >> 1, 0u, c | 2u);
            if (model == ORACLE_ISING)
                s[i * w + j] = (int8_t)(u >= 0x80000000u ? 1 : -1);
            else
                s[i * w + j] = (int8_t)((int)(((uint64_t)u * 3u) >> 32) - 1);
        }
    }
    return 0;
}

/* n sweeps t0 .. t0+n-1 of the window: every site except the outer ring is
 * updated with the random word and colour of its global position; the ring
 * is held fixed (it stands for the unknown rest of the lattice).  After n
 * sweeps the sites at distance > 2n from the ring are exactly those of the
 * full lattice (each half-sweep lets an error move one site).  L even.     */
int oracle_window_run(int8_t *s, int64_t h, int64_t w, int64_t y0, int64_t x0, int64_t L,
                      int model, uint64_t seed, uint64_t t0, int64_t n, const double *betas,
                      double delta)
{
    if (!s || h < 3 || w < 3 || L < 2 || L % 2 != 0 || n < 0 || !betas ||
        (model != ORACLE_ISING && model != ORACLE_BLUME_CAPEL))
        return -1;
    for (int64_t k = 0; k < n; ++k) {
        const uint64_t t = t0 + (uint64_t)k;
        for (int c = 0; c < 2; ++c) {
            for (int64_t i = 1; i < h - 1; ++i) {
                const int64_t y = (y0 + i) % L;
                for (int64_t j = 1; j < w - 1; ++j) {
                    const int64_t x = (x0 + j) % L;
                    if ((int)((x + y) & 1) != c)
                        continue;
                    const uint64_t jj = (uint64_t)(y * L + x) >> 1;
                    const uint32_t u = site_word(seed, jj, (uint32_t)t, (uint32_t)c);
                    const int64_t id = i * w + j;
                    const int si = s[id];
                    const int hsum = s[id - 1] + s[id + 1] + s[id - w] + s[id + w];
                    if (model == ORACLE_ISING) {
                        const double dE = (double)(2 * si * hsum);
                        int accept = 1;
                        if (dE > 0.0)
                            accept = (uint64_t)u < threshold_bits(betas[k], dE, 32);
                        if (accept)
                            s[id] = (int8_t)(-si);
                    } else {
                        const int s2 = oracle_bc_proposal(si, (int)(u & 1u));
                        const double dE = bc_delta_energy(si, s2, hsum, delta);
                        int accept = 1;
                        if (dE > 0.0)
                            accept = (uint64_t)(u >> 1) < threshold_bits(betas[k], dE, 31);
                        if (accept)
                            s[id] = (int8_t)s2;
                    }
                }
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Row slabs of a lattice (domain decomposition, Introduction: the paper     */
/* runs one lattice on many GPUs, each holding a part of it).                */
/* ------------------------------------------------------------------------ */

/* Value of a site after its Metropolis update: current value si, neighbour
 * sum h, random word u (Eq. (1) with J = 1; the acceptance and proposal
 * rules stated at the top of this file).                                   */
static int metropolis_new_value(int si, int h, uint32_t u, int model, double beta, double delta)
{
    if (model == ORACLE_ISING) {
        const double dE = (double)(2 * si * h);
        if (dE > 0.0 && !((uint64_t)u < threshold_bits(beta, dE, 32)))
            return si;
        return -si;
    }
    const int s2 = oracle_bc_proposal(si, (int)(u & 1u));
    const double dE = bc_delta_energy(si, s2, h, delta);
    if (dE > 0.0 && !((uint64_t)(u >> 1) < threshold_bits(beta, dE, 31)))
        return si;
    return s2;
}

/* s holds rows + 2 rows of L sites: row 0 is global row y0 - 1 (mod L), rows
 * 1 .. rows are the owned global rows y0 .. y0 + rows - 1, row rows + 1 is
 * global row y0 + rows (mod L).  Half-sweep of colour c at sweep t: every
 * owned site with (x + y) & 1 == c (y the global row), row-major, in place,
 * with its global random word; x is periodic, rows 0 and rows + 1 are only
 * read.                                                                    */
int oracle_slab_half_sweep(int8_t *s, int64_t rows, int64_t L, int64_t y0, int model,
                           uint64_t seed, uint64_t t, int c, double beta, double delta)
{
    if (!s || rows < 1 || L < 2 || L % 2 != 0 || y0 < 0 || y0 + rows > L || (c != 0 && c != 1) ||
        (model != ORACLE_ISING && model != ORACLE_BLUME_CAPEL))
        return -1;
    for (int64_t i = 1; i <= rows; ++i) {
        const int64_t y = y0 + i - 1;
        for (int64_t x = 0; x < L; ++x) {
            if ((int)((x + y) & 1) != c)
                continue;
            const int64_t id = i * L + x;
            const int h = s[i * L + dn1(x, L)] + s[i * L + up1(x, L)] + s[(i - 1) * L + x] +
                          s[(i + 1) * L + x];
            const uint64_t j = (uint64_t)(y * L + x) >> 1;
            const uint32_t u = site_word(seed, j, (uint32_t)t, (uint32_t)c);
            s[id] = (int8_t)metropolis_new_value(s[id], h, u, model, beta, delta);
        }
    }
    return 0;
}

/* The owned rows' part of the observables of oracle_measure: B over the
 * bonds of owned sites to +x and +y (the last owned row's +y neighbours are
 * row rows + 1), M, Q, R[i] for owned row i, and C[x] summed over the owned
 * rows only.                                                               */
int oracle_slab_measure(const int8_t *s, int64_t rows, int64_t L, int64_t *bmq, int32_t *R,
                        int32_t *C)
{
    if (!s || !bmq || rows < 1 || L < 1)
        return -1;
    int64_t B = 0, M = 0, Q = 0;
    if (C)
        for (int64_t x = 0; x < L; ++x)
            C[x] = 0;
    for (int64_t i = 1; i <= rows; ++i) {
        int64_t row = 0;
        for (int64_t x = 0; x < L; ++x) {
            const int v = s[i * L + x];
            B += (int64_t)v * (s[i * L + up1(x, L)] + s[(i + 1) * L + x]);
            M += v;
            Q += v * v;
            row += v;
            if (C)
                C[x] += v;
        }
        if (R)
            R[i - 1] = (int32_t)row;
    }
    bmq[0] = B;
    bmq[1] = M;
    bmq[2] = Q;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Correlation function along the lattice axes (Eq. (2)).                   */
/* ------------------------------------------------------------------------ */

/* For each distance r[k] (0 <= r[k] < L): sx[k] = sum_{x,y} s(x,y) s(x+r,y)
 * and sy[k] = sum_{x,y} s(x,y) s(x,y+r), periodic.  C((r,0)) = sx / L^2 and
 * C((0,r)) = sy / L^2.                                                     */
int oracle_correlation(const int8_t *s, int64_t L, int64_t nr, const int64_t *r, int64_t *sx,
                       int64_t *sy)
{
    if (!s || L < 1 || nr < 0 || (nr > 0 && (!r || !sx || !sy)))
        return -1;
    for (int64_t k = 0; k < nr; ++k) {
        if (r[k] < 0 || r[k] >= L)
            return -1;
        int64_t ax = 0, ay = 0;
        for (int64_t y = 0; y < L; ++y) {
            const int64_t y2 = (y + r[k]) % L;
            for (int64_t x = 0; x < L; ++x) {
                const int v = s[y * L + x];
                ax += v * s[y * L + (x + r[k]) % L];
                ay += v * s[y2 * L + x];
            }
        }
        sx[k] = ax;
        sy[k] = ay;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Swendsen-Wang iteration restricted to the sites with s = +-1 (Appendix B: */
/* the Blume-Capel equilibrium runs combine Swendsen-Wang cluster updates of */
/* the +-1 spins with Metropolis sweeps, which change s^2; for Ising every  */
/* site takes part).                                                         */
/*                                                                           */
/* Readings where the paper is silent:                                       */
/*   - Bond (i, j), j the +x (d = 0) or +y (d = 1) neighbour of site         */
/*     i = y*L + x, is active iff s_i = s_j != 0 and (uint64)u < thr, with  */
/*     thr = rne(2^32 p), p = 1 - exp(-2 beta) (J = 1; the energy of an      */
/*     aligned +-1 pair is 2 below an anti-aligned one) computed as          */
/*     -expm1(-2 beta), and u the Philox4x32-10 word i & 3 of counter        */
/*     (lo32(i>>2), hi32(i>>2), k, 4 + d), key (lo32(seed), hi32(seed)),     */
/*     k = the number of Swendsen-Wang iterations done before on this        */
/*     lattice.  Counter word 3 >= 4 keeps these draws apart from the        */
/*     sweep (0, 1) and hot-start (2, 3) draws.                              */
/*   - A cluster is a connected component of active bonds; its label is its */
/*     smallest site index r.  It flips (s -> -s on all its sites) iff the   */
/*     word r & 3 of counter (lo32(r>>2), hi32(r>>2), k, 6) is >= 2^31.     */
/*   - Sites with s = 0 are never bonded and never flip (label = own index). */
/* ------------------------------------------------------------------------ */

static int64_t uf_root(int64_t *parent, int64_t i)
{
    while (parent[i] != i)
        i = parent[i];
    return i;
}

/* Join the components of a and b: the larger root points to the smaller,  */
/* so every root is the smallest index of its component.                    */
static void uf_unite(int64_t *parent, int64_t a, int64_t b)
{
    a = uf_root(parent, a);
    b = uf_root(parent, b);
    if (a < b)
        parent[b] = a;
    else if (b < a)
        parent[a] = b;
}

uint64_t oracle_sw_threshold(double beta)
{
    return (uint64_t)llrint(ldexp(-expm1(-2.0 * beta), 32));
}

static uint32_t full_index_word(uint64_t seed, uint64_t i, uint32_t k, uint32_t w3)
{
    const uint64_t q = i >> 2;
    const uint32_t ctr[4] = {(uint32_t)q, (uint32_t)(q >> 32), k, w3};
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    oracle_philox4x32_10(ctr, key, out);
    return out[i & 3u];
}

/* One iteration on s (L x L, updated in place).  labels (L*L, may be NULL)
 * receives each site's cluster label.  Returns the number of clusters of
 * +-1 sites, or -1 on bad arguments.                                        */
int64_t oracle_swendsen_wang(int8_t *s, int64_t L, uint64_t seed, uint64_t k, double beta,
                             int64_t *labels)
{
    if (!s || L < 2 || !(beta >= 0.0) || k > 0xFFFFFFFFull)
        return -1;
    const int64_t N = L * L;
    const uint64_t thr = oracle_sw_threshold(beta);
    int64_t *parent = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    if (!parent)
        return -1;
    for (int64_t i = 0; i < N; ++i)
        parent[i] = i;
    for (int64_t y = 0; y < L; ++y)
        for (int64_t x = 0; x < L; ++x) {
            const int64_t i = y * L + x;
            if (s[i] == 0)
                continue;
            const int64_t jx = y * L + up1(x, L), jy = up1(y, L) * L + x;
            if (s[jx] == s[i] && (uint64_t)full_index_word(seed, (uint64_t)i, (uint32_t)k, 4) < thr)
                uf_unite(parent, i, jx);
            if (s[jy] == s[i] && (uint64_t)full_index_word(seed, (uint64_t)i, (uint32_t)k, 5) < thr)
                uf_unite(parent, i, jy);
        }
    int64_t clusters = 0;
    for (int64_t i = 0; i < N; ++i) {
        parent[i] = uf_root(parent, i);
        if (s[i] != 0 && parent[i] == i)
            ++clusters;
    }
    if (labels)
        memcpy(labels, parent, sizeof(int64_t) * (size_t)N);
    for (int64_t i = 0; i < N; ++i)
        if (s[i] != 0 && full_index_word(seed, (uint64_t)parent[i], (uint32_t)k, 6) >= 0x80000000u)
            s[i] = (int8_t)-s[i];
    free(parent);
    return clusters;
}
