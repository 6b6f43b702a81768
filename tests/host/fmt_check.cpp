/* The printf landing pad's to_chars fast path against snprintf with the same
 * conversion: every accepted conversion and length modifier, random words,
 * doubles across the exponent range, exact ties and integer edge values.
 * Prints "fmt checked N fast F mismatches M". */
#include <cfloat>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <string>
#include <vector>
#include "fmt_fast.h"

struct Spec {
    const char *fmt;
    char conv;
    const char *len;
    int prec;
    int kind;  /* 0 int-like (word), 1 double */
};

int main()
{
    const Spec specs[] = {
        {"%d", 'd', "", -1, 0},     {"%i", 'i', "", -1, 0},     {"%hd", 'd', "h", -1, 0},   {"%hhd", 'd', "hh", -1, 0},
        {"%ld", 'd', "l", -1, 0},   {"%lld", 'd', "ll", -1, 0}, {"%zd", 'd', "z", -1, 0},   {"%u", 'u', "", -1, 0},
        {"%lu", 'u', "l", -1, 0},   {"%llu", 'u', "ll", -1, 0}, {"%hu", 'u', "h", -1, 0},   {"%hhu", 'u', "hh", -1, 0},
        {"%x", 'x', "", -1, 0},     {"%lx", 'x', "l", -1, 0},   {"%llx", 'x', "ll", -1, 0}, {"%hx", 'x', "h", -1, 0},
        {"%o", 'o', "", -1, 0},     {"%llo", 'o', "ll", -1, 0}, {"%e", 'e', "", -1, 1},     {"%.0e", 'e', "", 0, 1},
        {"%.3e", 'e', "", 3, 1},    {"%.6e", 'e', "", 6, 1},    {"%.17e", 'e', "", 17, 1},  {"%le", 'e', "l", -1, 1},
        {"%f", 'f', "", -1, 1},     {"%.0f", 'f', "", 0, 1},    {"%.3f", 'f', "", 3, 1},    {"%.10f", 'f', "", 10, 1},
        {"%lf", 'f', "l", -1, 1},   {"%g", 'g', "", -1, 1},     {"%.1g", 'g', "", 1, 1},    {"%.3g", 'g', "", 3, 1},
        {"%.6g", 'g', "", 6, 1},    {"%.15g", 'g', "", 15, 1},  {"%.17g", 'g', "", 17, 1},  {"%.25g", 'g', "", 25, 1},
        {"%lg", 'g', "l", -1, 1},   {"%.1e", 'e', "", 1, 1},    {"%.16e", 'e', "", 16, 1},  {"%.9e", 'e', "", 9, 1},
        {"%.1f", 'f', "", 1, 1},    {"%.2f", 'f', "", 2, 1},    {"%.6f", 'f', "", 6, 1},    {"%.17f", 'f', "", 17, 1},
        {"%.2g", 'g', "", 2, 1},    {"%.12g", 'g', "", 12, 1},  {"%.16g", 'g', "", 16, 1},
    };
    std::mt19937_64 rng(7);
    std::vector<uint64_t> words = {0, 1, 2, 9, 10, 15, 16, 255, 256, 65535, 65536, 0x7fffffffull, 0x80000000ull,
                                   0xffffffffull, 0x100000000ull, (uint64_t)LLONG_MAX, (uint64_t)LLONG_MIN, ~0ull,
                                   (uint64_t)-1ll, (uint64_t)-128ll, (uint64_t)-32768ll};
    for (int k = 0; k < 20000; k++)
        words.push_back(rng() >> (rng() % 64));
    std::vector<double> dbls = {0.0, -0.0, 0.5, 1.5, 2.5, -2.5, 0.125, 0.0625, 1e-5, 1e-4, 1e15, 1e16, 1e17, 1e21,
                                1e22, 1e23, 123456.5, 999999.5, 9.9999995, 0.00001234, DBL_MAX, DBL_MIN, 5e-324,
                                -DBL_MAX, 1.0 / 3.0, 2.0 / 3.0, 1e300, 1e-300, 4503599627370496.5, 0.1, 0.2, 0.3};
    std::uniform_real_distribution<double> U(-1.0, 1.0);
    for (int k = 0; k < 40000; k++) {
        const int e = (int)(rng() % 640) - 330;
        dbls.push_back(std::ldexp(U(rng), (int)(e * 3.3219)));
        uint64_t b = rng();
        double d;
        memcpy(&d, &b, 8);
        dbls.push_back(d);
        dbls.push_back((double)(int64_t)(rng() % 2000001) / 1000.0 - 1000.0);   /* short decimals, ties for %.0f */
    }
    /* near powers of ten and the decimal carries they invite */
    for (int k = -320; k <= 308; k++) {
        const double p = std::pow(10.0, k);
        if (!(p > 0) || !std::isfinite(p))
            continue;
        double q = p;
        for (int j = 0; j < 4; j++) {
            dbls.push_back(q);
            q = std::nextafter(q, 0.0);
        }
        q = p;
        for (int j = 0; j < 4; j++) {
            q = std::nextafter(q, INFINITY);
            dbls.push_back(q);
        }
        dbls.push_back(p * 9.5);
        dbls.push_back(p * 9.95);
        dbls.push_back(p * 9.9999999999999995);
        dbls.push_back(p * 0.99999999999999999);
    }
    /* integers up to 2^64, exact halves at every scale, short decimals */
    for (int k = 0; k < 20000; k++) {
        dbls.push_back((double)(rng() >> (rng() % 64)));
        dbls.push_back(std::ldexp((double)(2 * (rng() % 1000000) + 1), -(int)(rng() % 60)));
        dbls.push_back((double)(int64_t)(rng() % 200000001) / 1e6);
    }
    long n = 0, fast = 0, bad = 0;
    char a[1024], b[1024];
    for (const Spec &s : specs) {
        const size_t cnt = s.kind ? dbls.size() : words.size();
        for (size_t k = 0; k < cnt; k++) {
            uint64_t w;
            int want_n;
            if (s.kind) {
                memcpy(&w, &dbls[k], 8);
                want_n = snprintf(a, sizeof a, s.fmt, dbls[k]);
            } else {
                w = words[k];
                const bool ll = s.len[0] == 'l' || s.len[0] == 'z';
                want_n = ll ? snprintf(a, sizeof a, s.fmt, (long long)w)
                            : (s.len[0] == 'h' && s.len[1] == 'h')
                                  ? snprintf(a, sizeof a, s.fmt, (int)(signed char)w)
                                  : s.len[0] == 'h' ? snprintf(a, sizeof a, s.fmt, (int)(short)w)
                                                    : snprintf(a, sizeof a, s.fmt, (int)w);
            }
            n++;
            int got_n = 0;
            if (!gfh::fmt_fast(s.conv, s.len, s.prec, w, s.kind == 1, b, sizeof b, &got_n))
                continue;
            fast++;
            if (want_n >= (int)sizeof a || got_n != want_n || memcmp(a, b, (size_t)got_n) != 0) {
                if (bad < 10)
                    printf("mismatch %s: want [%.*s] got [%.*s]\n", s.fmt, want_n, a, got_n, b);
                bad++;
            }
        }
    }
    /* the fixed-precision path alone: whatever it accepts must match */
    long dn = 0, dacc = 0;
    const int precs[] = {0, 1, 2, 3, 5, 6, 9, 12, 15, 16, 17};
    const char convs[] = {'e', 'f', 'g'};
    for (const char c : convs)
        for (const int p : precs)
            for (const double d : dbls) {
                if (!std::isfinite(d))
                    continue;
                char f[16];
                snprintf(f, sizeof f, "%%.%d%c", p, c);
                const int want_n = snprintf(a, sizeof a, f, d);
                uint64_t bits;
                memcpy(&bits, &d, 8);
                const int got_n = gfh::dtoa::format(c, p, bits, b);
                dn++;
                if (got_n <= 0)
                    continue;
                dacc++;
                if (got_n != want_n || memcmp(a, b, (size_t)got_n) != 0) {
                    if (bad < 20)
                        printf("dtoa mismatch %s of %a: want [%.*s] got [%.*s]\n", f, d, want_n, a, got_n, b);
                    bad++;
                }
            }
    printf("dtoa checked %ld accepted %ld\n", dn, dacc);
    printf("fmt checked %ld fast %ld mismatches %ld\n", n, fast, bad);
    return 0;
}
