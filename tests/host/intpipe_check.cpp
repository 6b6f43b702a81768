/* Host build of the integer-pipe FP64 helpers compared with the host's IEEE
 * arithmetic: gf_dadd_int(x, y) and gf_dadd_int_any(x, y) against x + y
 * (bits, NaN as NaN) over same-sign pairs at every exponent gap,
 * round-to-even ties, carries into the next binade, zeros, subnormals,
 * overflow and random bit patterns;
 * gf_udiv32 against '/' over edge and random operands (exhaustive over
 * [0, 2^31) for two divisors).  Prints "<name> checked N mismatches M". */
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include "gf_intpipe.cuh"

static uint64_t B(double x) { uint64_t b; memcpy(&b, &x, 8); return b; }
static double D(uint64_t b) { double x; memcpy(&x, &b, 8); return x; }

static long n_add = 0, bad_add = 0;
static void add_case(double x, double y)
{
    volatile double vx = x, vy = y;
    const double want = vx + vy;
    /* the entry point (short path for small exponent gaps) and the
     * any-gap path on its own */
    const double got[2] = {gf_dadd_int(x, y), gf_dadd_int_any(x, y)};
    for (int p = 0; p < 2; p++) {
        n_add++;
        const bool ok = (std::isnan(want) && std::isnan(got[p])) || B(want) == B(got[p]);
        if (!ok) {
            if (bad_add < 10)
                printf("dadd%s mismatch %a + %a: got %a want %a\n", p ? "_any" : "", x, y, got[p], want);
            bad_add++;
        }
    }
}

int main(int argc, char **argv)
{
    const long scale = argc > 1 ? atol(argv[1]) : 1;
    std::mt19937_64 rng(12345);
    auto u53 = [&] { return rng() & 0x000fffffffffffffull; };
    /* same-sign pairs, every exponent gap 0..70, several binades */
    for (long it = 0; it < 200000 * scale; it++) {
        const uint64_t ea = 1 + rng() % 2046, gap = rng() % 71;
        const uint64_t eb = ea > gap ? ea - gap : 1;
        const uint64_t s = (rng() & 1) ? 0x8000000000000000ull : 0;
        add_case(D(s | (ea << 52) | u53()), D(s | (eb << 52) | u53()));
        add_case(D(s | (eb << 52) | u53()), D(s | (ea << 52) | u53()));
    }
    /* the Jacobi range: sums of values in [0, 6) */
    std::uniform_real_distribution<double> U(0.0, 6.0);
    for (long it = 0; it < 1000000 * scale; it++)
        add_case(U(rng), U(rng));
    /* ties and near-ties: y = half an ulp of x, +-1 ulp around it */
    for (long it = 0; it < 100000 * scale; it++) {
        const uint64_t ea = 60 + rng() % 1900;
        const double x = D((ea << 52) | u53());
        for (int k = 52; k <= 54; k++) {
            const double h = D((ea - k) << 52);
            add_case(x, h);
            add_case(x, D(B(h) + 1));
            add_case(x, D(B(h) - 1));
            add_case(-x, -h);
        }
    }
    /* exponent gaps 1..10 whose dropped bits are exactly one half: the ties
     * of the short path, with and without a carry into the next binade */
    for (long it = 0; it < 200000 * scale; it++) {
        const uint64_t d = 1 + rng() % 10, ea = 20 + rng() % 2020;
        const uint64_t low = (1ull << d) - 1;
        const uint64_t fb = (u53() & ~low) | (1ull << (d - 1));
        add_case(D((ea << 52) | u53()), D(((ea - d) << 52) | fb));
        add_case(D(((ea - d) << 52) | fb), D((ea << 52) | u53()));
    }
    /* carries into the next binade, and all-ones significands */
    for (long it = 0; it < 100000 * scale; it++) {
        const uint64_t ea = 1 + rng() % 2046;
        add_case(D((ea << 52) | 0x000fffffffffffffull), D((ea << 52) | u53()));
        add_case(D((ea << 52) | 0x000fffffffffffffull), D(((ea > 53 ? ea - 53 : 1) << 52) | u53()));
    }
    /* specials and edges (the FP64 fallback or the zero shortcut) */
    const double sp[] = {0.0, -0.0, 1.0, -1.0, INFINITY, -INFINITY, NAN, 5e-324, -5e-324, 2.2250738585072014e-308,
                         2.2250738585072009e-308, 1.7976931348623157e308, -1.7976931348623157e308, 8.98846567431158e307,
                         4.49423283715579e307, 0x1.fffffffffffffp1022, 0x1p1023, 0x1p-1022, 0x1.8p-1022, 3.0, 0.5};
    for (double x : sp)
        for (double y : sp)
            add_case(x, y);
    /* random bit patterns: every category mixed */
    for (long it = 0; it < 2000000 * scale; it++)
        add_case(D(rng()), D(rng()));
    /* fabs */
    long bad_abs = 0;
    for (long it = 0; it < 100000; it++) {
        const double x = D(rng());
        if (B(gf_fabs_int(x)) != (B(x) & 0x7fffffffffffffffull))
            bad_abs++;
    }
    printf("dadd checked %ld mismatches %ld\n", n_add, bad_add);
    printf("fabs checked %d mismatches %ld\n", 100000, bad_abs);
    /* udiv32 */
    long n_div = 0, bad_div = 0;
    auto div_case = [&](uint32_t x, uint32_t d, const gf_udiv32 &q) {
        n_div++;
        if (q.div(x) != x / d) {
            if (bad_div < 10)
                printf("udiv mismatch %u / %u: got %u\n", x, d, q.div(x));
            bad_div++;
        }
    };
    std::vector<uint32_t> ds = {1, 2, 3, 5, 6, 7, 31, 32, 33, 254, 255, 256, 257, 1289, 1290, 65025, 65536, 1664100,
                                (1u << 30) - 1, 1u << 30, (1u << 30) + 1, 0x7fffffffu};
    for (int k = 0; k < 2000; k++)
        ds.push_back(1u + (uint32_t)(rng() % 0x7fffffffu));
    for (uint32_t d : ds) {
        const gf_udiv32 q = gf_udiv32::make(d);
        for (uint32_t x : {0u, 1u, d - 1u, d, d + 1u, 0x7fffffffu, 0x7ffffffeu})
            if (x < 0x80000000u)
                div_case(x, d, q);
        for (int k = 0; k < 2000; k++) {
            const uint32_t x = (uint32_t)(rng() & 0x7fffffffu);
            div_case(x, d, q);
            const uint64_t mult = (uint64_t)(x / d) * d;
            if (mult >= 1 && mult - 1 < 0x80000000ull)
                div_case((uint32_t)(mult - 1), d, q);
        }
    }
    for (uint32_t d : {255u, 65025u}) {
        const gf_udiv32 q = gf_udiv32::make(d);
        for (uint32_t x = 0; x < 0x80000000u; x++) {
            if (q.div(x) != x / d) {
                bad_div++;
                break;
            }
        }
        n_div += 0x80000000l;
    }
    printf("udiv checked %ld mismatches %ld\n", n_div, bad_div);
    return 0;
}
