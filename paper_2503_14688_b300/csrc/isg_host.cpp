// isg_host.cpp -- host-side arithmetic of libisg: Philox launch constants,
// the integer acceptance thresholds (Introduction: Metropolis; Appendix B:
// 32-bit integer random numbers) and the FP64 second-moment correlation
// length (Appendix B).
//
// Compiled with -ffp-contract=off: the threshold and xi_2 expressions below
// are evaluated exactly as written, one IEEE operation at a time, so that any
// other program that writes the same definitions in the same order obtains
// the same bits.
#include <cmath>
#include <cstdint>
#include <vector>

#include "isg_internal.h"

namespace isg {

void philox_launch_consts(uint64_t seed, uint32_t w2, uint32_t w3, PhiloxLaunch *out)
{
    const uint32_t key0 = (uint32_t)seed, key1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        out->rk0[r] = key0 + (uint32_t)r * kPhiloxW0;
        out->rk1[r] = key1 + (uint32_t)r * kPhiloxW1;
    }
    const uint64_t m1w2 = (uint64_t)kPhiloxM1 * (uint64_t)w2;
    out->r0_c0 = (uint32_t)(m1w2 >> 32) ^ out->rk0[0];
    out->r0_c2x = w3 ^ out->rk1[0];
    out->r1_c0x = (uint32_t)m1w2 ^ out->rk0[1];
}

// rne(2^bits * exp(-beta * dE)) for dE > 0.
static uint64_t grid_threshold(double beta, double dE, int bits)
{
    const double p = std::exp(-beta * dE);
    return (uint64_t)std::llrint(std::ldexp(p, bits));
}

void ising_thresholds(double beta, IsingThr *out)
{
    // dE = 2 s h = 8 - 4c for c anti-aligned neighbours; only c = 0, 1 are uphill.
    const uint64_t t4 = grid_threshold(beta, 4.0, 32);
    const uint64_t t8 = grid_threshold(beta, 8.0, 32);
    const uint64_t two32 = (uint64_t)1 << 32;
    out->full4 = t4 >= two32 ? ~0u : 0u;
    out->full8 = t8 >= two32 ? ~0u : 0u;
    out->thr4 = t4 >= two32 ? 0xFFFFFFFFu : (uint32_t)t4;
    out->thr8 = t8 >= two32 ? 0xFFFFFFFFu : (uint32_t)t8;
}

// The value proposed from s by the bit b: the (b+1)-th smallest of the two
// values different from s.
static int bc_proposed(int s, int b)
{
    if (s < 0)
        return b ? 1 : 0;
    if (s == 0)
        return b ? 1 : -1;
    return b ? 0 : -1;
}

void bc_table(double beta, double delta, BcTable *out)
{
    const uint32_t always = 0x80000000u;  // (u >> 1) < 2^31 for every u
    for (int i = 0; i < kBcTableSize; ++i)
        out->thr[i] = always;
    uint32_t lowest = always;
    for (int s = -1; s <= 1; ++s) {
        const int n = s != 0, p = s > 0;
        for (int b = 0; b < 2; ++b) {
            const int s2 = bc_proposed(s, b);
            for (int g = 0; g <= 8; ++g) {
                const int h = g - 4;
                // Eq. (1) with J = 1: dE = -(s' - s) h + Delta (s'^2 - s^2)
                const double dE = (double)(-(s2 - s) * h) + delta * (double)(s2 * s2 - s * s);
                uint32_t thr = always;
                if (dE > 0.0)
                    thr = (uint32_t)grid_threshold(beta, dE, 31);
                out->thr[bc_entry(n, p, b, g)] = thr;
                lowest = thr < lowest ? thr : lowest;
            }
        }
    }
    // v < thr31  <=>  u = 2 v + b <= 2 thr31 - 1, representable unless thr31 = 0
    out->full = lowest >= 1u;
    if (out->full)
        for (int i = 0; i < kBcTableSize; ++i)
            out->thr[i] = 2u * out->thr[i] - 1u;
}

// ---------------------------------------------------------------------------
// xi_2 (Appendix B).  Fixed operation order:
//   twiddles cos/sin(2 pi x / L) from libm on x in [0, L/8] (all x when L is
//   not a multiple of 8), the other octants by the exact symmetries;
//   Re and Im of sum_x f[x] e^{i 2 pi x/L} as Neumaier-compensated sums in
//   index order; S_k = 0.5 * (P_col + P_row); S_0 summed exactly in 128-bit
//   integers; replica S_k summed with Neumaier in replica order.
// ---------------------------------------------------------------------------
namespace {

struct Compensated {
    double sum = 0.0, comp = 0.0;
    void add(double v)
    {
        const double t = sum + v;
        if (std::fabs(sum) >= std::fabs(v))
            comp += (sum - t) + v;
        else
            comp += (v - t) + sum;
        sum = t;
    }
    double value() const { return sum + comp; }
};

void make_twiddles(int64_t L, std::vector<double> &c, std::vector<double> &s)
{
    c.assign((size_t)L, 0.0);
    s.assign((size_t)L, 0.0);
    const double two_pi = 2.0 * M_PI;
    if (L % 8 != 0) {
        for (int64_t x = 0; x < L; ++x) {
            const double a = two_pi * (double)x / (double)L;
            c[x] = std::cos(a);
            s[x] = std::sin(a);
        }
        return;
    }
    const int64_t oct = L / 8, quad = L / 4, half = L / 2;
    for (int64_t x = 0; x <= oct; ++x) {
        const double a = two_pi * (double)x / (double)L;
        c[x] = std::cos(a);
        s[x] = std::sin(a);
    }
    for (int64_t x = oct + 1; x <= quad; ++x) {
        c[x] = s[quad - x];
        s[x] = c[quad - x];
    }
    for (int64_t x = quad + 1; x <= half; ++x) {
        c[x] = -c[half - x];
        s[x] = s[half - x];
    }
    for (int64_t x = half + 1; x < L; ++x) {
        c[x] = c[L - x];
        s[x] = -s[L - x];
    }
}

double mode_power(const int32_t *f, int64_t L, const std::vector<double> &c,
                  const std::vector<double> &s)
{
    Compensated re, im;
    for (int64_t x = 0; x < L; ++x) {
        re.add((double)f[x] * c[x]);
        im.add((double)f[x] * s[x]);
    }
    const double r = re.value(), i = im.value();
    return r * r + i * i;
}

}  // namespace

double xi2_fp64(int64_t n, int64_t L, const int64_t *M, const int32_t *R, const int32_t *C)
{
    if (n < 1 || L < 2 || !M || !R || !C)
        return NAN;
    std::vector<double> c, s;
    make_twiddles(L, c, s);
    __int128 s0 = 0;
    Compensated sk;
    for (int64_t r = 0; r < n; ++r) {
        s0 += (__int128)M[r] * (__int128)M[r];
        const double pc = mode_power(C + r * L, L, c, s);
        const double pr = mode_power(R + r * L, L, c, s);
        sk.add(0.5 * (pc + pr));
    }
    const double s0avg = (double)s0 / (double)n;
    const double skavg = sk.value() / (double)n;
    if (!(s0avg > skavg))
        return NAN;
    if (skavg == 0.0)
        return INFINITY;
    return std::sqrt(s0avg / skavg - 1.0) / (2.0 * std::sin(M_PI / (double)L));
}

// Swendsen-Wang bond threshold (Appendix B): rne(2^32 p), p the probability
// that a bond between aligned +-1 neighbours is active.
uint64_t sw_threshold(double beta)
{
    // p = 1 - e^{-2 beta} (J = 1: aligned +-1 neighbours lie 2 below
    // anti-aligned ones), evaluated as -expm1(-2 beta)
    return (uint64_t)std::llrint(std::ldexp(-std::expm1(-2.0 * beta), 32));
}

// Integral coherence length (Appendix C): xi = I2 / I1 with
// I_n = int_0^{r_cut} r^n C(r) dr, by the trapezoid rule over the sampled
// distances r[0] < r[1] < ... (those beyond r_cut are ignored).
double xi_integral_fp64(int64_t n, const double *r, const double *c, double r_cut)
{
    if (n < 2 || !r || !c)
        return NAN;
    double i1 = 0.0, i2 = 0.0;
    for (int64_t k = 1; k < n && r[k] <= r_cut; ++k) {
        const double h = r[k] - r[k - 1];
        if (!(h > 0.0))
            return NAN;
        i1 += 0.5 * h * (r[k - 1] * c[k - 1] + r[k] * c[k]);
        i2 += 0.5 * h * (r[k - 1] * r[k - 1] * c[k - 1] + r[k] * r[k] * c[k]);
    }
    if (!(i1 > 0.0))
        return NAN;
    return i2 / i1;
}

}  // namespace isg
