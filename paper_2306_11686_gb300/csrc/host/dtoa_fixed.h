/*
 * Fixed-precision decimal conversion of binary64 for the printf landing pad:
 * %.Pe, %.Pf and %.Pg (P up to 17 significant digits), the same characters
 * as the C library's correctly rounded conversion in the "C" locale.
 *
 * A finite x != 0 is m * 2^e exactly (53-bit m).  The conversion needs
 * N = round-half-even(x * 10^k) for one k (the digit count of %e/%g fixes k
 * from the decimal exponent; %f has k = P).  10^k comes from a table of
 * 128-bit significands, each the exact power truncated to 128 bits and built
 * once from exact big-integer arithmetic (no floating point), so the product
 * m * c (at most 181 bits) is within a relative 2^-126 below the exact
 * x * 10^k.  When N fits in 64 bits that error is below 2^-62 of the last
 * digit, and the rounding direction is exact unless the fraction lies within
 * that distance of one half.  Those rare near-ties -- and exact ties -- are
 * left to the caller's exact path (std::to_chars), as are zero, P beyond the
 * supported range and results too long for 64 bits.
 *
 * The digits follow from N with integer arithmetic; the layout rules are
 * those of the C standard's fprintf: %e's exponent has at least two digits,
 * %g takes the %e form when the exponent X of that form is below -4 or at
 * least P, and otherwise the %f form with P - 1 - X decimals, and in both
 * drops trailing zeros of the fraction and a bare decimal point.
 */
#ifndef GF_DTOA_FIXED_H
#define GF_DTOA_FIXED_H

#include <cstdint>
#include <cmath>
#include <cstring>
#include <vector>

namespace gfh {
namespace dtoa {

typedef unsigned __int128 u128;

/* 10^k = (hi:lo) * 2^s * (1 + t), 0 <= t < 2^-126, hi's top bit set */
struct P10 {
    uint64_t hi, lo;
    int32_t s;
};

static const int KMIN = -360, KMAX = 360;

/* little-endian 64-bit limbs */
typedef std::vector<uint64_t> Big;

inline int big_bits(const Big &b)
{
    for (size_t i = b.size(); i-- > 0;)
        if (b[i])
            return (int)(64 * i) + 64 - __builtin_clzll(b[i]);
    return 0;
}

/* bits [from, from + 128) of b */
inline u128 big_window(const Big &b, int from)
{
    u128 r = 0;
    for (int i = 127; i >= 0; i--) {
        const int bit = from + i;
        const uint64_t v = bit >= 0 && (size_t)(bit / 64) < b.size() ? (b[(size_t)bit / 64] >> (bit % 64)) & 1u : 0u;
        r = (r << 1) | v;
    }
    return r;
}

inline void big_mul10(Big &b)
{
    uint64_t carry = 0;
    for (uint64_t &x : b) {
        const u128 t = (u128)x * 10u + carry;
        x = (uint64_t)t;
        carry = (uint64_t)(t >> 64);
    }
    if (carry)
        b.push_back(carry);
}

inline void big_div10(Big &b)
{
    u128 rem = 0;
    for (size_t i = b.size(); i-- > 0;) {
        const u128 cur = (rem << 64) | b[i];
        b[i] = (uint64_t)(cur / 10u);
        rem = cur % 10u;
    }
    while (!b.empty() && b.back() == 0)
        b.pop_back();
}

/* the table, built on first use: for k >= 0 the top 128 bits of the integer
 * 10^k; for k < 0 the top 128 bits of floor(2^B / 10^-k) with B large
 * enough that at least 128 bits remain */
inline const P10 *table()
{
    static const std::vector<P10> t = [] {
        std::vector<P10> v((size_t)(KMAX - KMIN + 1));
        Big b{1};
        for (int k = 0; k <= KMAX; k++) {
            const int L = big_bits(b);
            const u128 c = big_window(b, L - 128);
            v[(size_t)(k - KMIN)] = {(uint64_t)(c >> 64), (uint64_t)c, L - 128};
            big_mul10(b);
        }
        const int B = 1536;                       /* 10^360 < 2^1196: 340 bits remain at k = -360 */
        Big q((size_t)B / 64 + 1, 0);
        q.back() = 1;                             /* 2^B */
        for (int k = -1; k >= KMIN; k--) {
            big_div10(q);
            const int L = big_bits(q);
            const u128 c = big_window(q, L - 128);
            v[(size_t)(k - KMIN)] = {(uint64_t)(c >> 64), (uint64_t)c, L - 128 - B};
        }
        return v;
    }();
    return t.data() - KMIN;
}

/* x = m 2^e with m in [2^52, 2^53).  Sets *N = round-half-even(x 10^k) and
 * *F = floor(x 10^k) (to within one unit where the fraction is within 2^-62
 * of a whole number), and returns true; returns false when N would not fit
 * in 64 bits, k is outside the table, or the fraction is too close to one
 * half to call. */
inline bool scaled_round(uint64_t m, int e, int k, uint64_t *N, uint64_t *F = nullptr)
{
    if (k < KMIN || k > KMAX)
        return false;
    const P10 &c = table()[k];
    /* P = m * (hi:lo), 181 bits at most: three limbs */
    const u128 a = (u128)m * c.lo, b = (u128)m * c.hi;
    const uint64_t p0 = (uint64_t)a;
    const u128 mid = (a >> 64) + (uint64_t)b;
    const uint64_t p1 = (uint64_t)mid;
    const uint64_t p2 = (uint64_t)(b >> 64) + (uint64_t)(mid >> 64);
    /* x 10^k ~ P 2^(e + s): sh fraction bits */
    const int sh = -(e + c.s);
    if (sh <= 64 || sh > 191)
        return false;
    /* integer part P >> sh must fit in 64 bits: P < 2^(sh + 64) */
    uint64_t I;
    u128 W;                                   /* the 128 fraction bits below the point */
    if (sh >= 128) {
        const int t = sh - 128;               /* 0 .. 63 */
        if (t == 0) {
            I = p2;
            W = ((u128)p1 << 64) | p0;
        } else {
            I = p2 >> t;
            W = ((u128)((p2 << (64 - t)) | (p1 >> t)) << 64) | ((p1 << (64 - t)) | (p0 >> t));
        }
    } else {                                  /* 65 .. 127: P >> sh from limbs 1 and 2 */
        const int t = sh - 64;                /* 1 .. 63 */
        if (p2 >> t)
            return false;
        I = (p2 << (64 - t)) | (p1 >> t);
        W = (((u128)p1 << 64) | p0) << (128 - sh);
    }
    /* P underestimates: the exact fraction lies in [W, W + 2^66] in units of
     * 2^-128 (2^-62 of the last digit, plus the bits below W) */
    const u128 HALF = (u128)1 << 127, MARGIN = ((u128)1 << 66) + 1;
    if (F)
        *F = I;
    if (W > HALF)
        I++;
    else if (W + MARGIN >= HALF)
        return false;
    if (I < (uint64_t)(W > HALF))             /* wrapped past 2^64 */
        return false;
    *N = I;
    return true;
}

/* decompose finite x != 0: |x| = m 2^e, m in [2^52, 2^53) */
inline void decompose(uint64_t bits, uint64_t *m, int *e)
{
    const uint64_t frac = bits & ((1ull << 52) - 1);
    const int ex = (int)((bits >> 52) & 0x7ff);
    if (ex) {
        *m = frac | (1ull << 52);
        *e = ex - 1075;
    } else {                                  /* subnormal: normalise */
        const int z = __builtin_clzll(frac) - 11;
        *m = frac << z;
        *e = -1074 - z;
    }
}

static const uint64_t POW10[20] = {1ull,
                                   10ull,
                                   100ull,
                                   1000ull,
                                   10000ull,
                                   100000ull,
                                   1000000ull,
                                   10000000ull,
                                   100000000ull,
                                   1000000000ull,
                                   10000000000ull,
                                   100000000000ull,
                                   1000000000000ull,
                                   10000000000000ull,
                                   100000000000000ull,
                                   1000000000000000ull,
                                   10000000000000000ull,
                                   100000000000000000ull,
                                   1000000000000000000ull,
                                   10000000000000000000ull};

/* the doubles nearest 10^k (to within an ulp), for the exponent estimate */
inline const double *pow10_dbl()
{
    static const std::vector<double> t = [] {
        std::vector<double> v((size_t)(KMAX - KMIN + 1));
        const P10 *c = table();
        for (int k = KMIN; k <= KMAX; k++)
            v[(size_t)(k - KMIN)] = std::ldexp((double)c[k].hi, c[k].s + 64);
        return v;
    }();
    return t.data() - KMIN;
}

/* D significant digits of |x| (1 <= D <= 18): N in [10^(D-1), 10^D) and
 * the decimal exponent X with |x| ~ N 10^(X - D + 1) */
inline bool sig_digits(uint64_t m, int e, double ax, int D, uint64_t *N, int *X)
{
    /* floor(log10 2^(e + 52)) is X or X - 1; the comparison with the double
     * nearest the next power of ten picks between them (a miss at the very
     * boundary is caught below) */
    int E = ((e + 52) * 78913) >> 18;
    if (E + 1 <= KMAX && ax >= pow10_dbl()[E + 1])
        E++;
    uint64_t n, fl;
    /* the exponent is right when the unrounded value lies in [10^(D-1), 10^D):
     * judged on the floor, since rounding alone can reach either bound */
    for (int tries = 0;; tries++) {
        if (tries == 3 || !scaled_round(m, e, D - 1 - E, &n, &fl))
            return false;
        if (fl >= POW10[D])
            E++;
        else if (fl < POW10[D - 1])
            E--;
        else
            break;
    }
    if (n == POW10[D]) {                      /* rounding carried into a new digit */
        n = POW10[D - 1];
        E++;
    }
    *N = n;
    *X = E;
    return true;
}

/* "00" .. "99" */
static const char DIG2[201] =
    "0001020304050607080910111213141516171819"
    "2021222324252627282930313233343536373839"
    "4041424344454647484950515253545556575859"
    "6061626364656667686970717273747576777879"
    "8081828384858687888990919293949596979899";

/* the digits of v < 10^len, len <= 8, into p[0..len) (leading zeros kept) */
inline void put_digits8(char *p, uint32_t v, int len)
{
    int i = len;
    while (i >= 2) {
        const uint32_t q = v / 100u;
        i -= 2;
        memcpy(p + i, DIG2 + 2 * (v - q * 100u), 2);
        v = q;
    }
    if (i)
        p[0] = (char)('0' + v);
}

/* the decimal digits of v, exactly `len` of them (leading zeros kept):
 * the low eight and the rest as two independent chains */
inline void put_digits(char *p, uint64_t v, int len)
{
    if (len <= 8) {
        put_digits8(p, (uint32_t)v, len);
        return;
    }
    const uint64_t hi = v / 100000000u;
    put_digits8(p + len - 8, (uint32_t)(v - hi * 100000000u), 8);
    if (len <= 16) {
        put_digits8(p, (uint32_t)hi, len - 8);
    } else {
        const uint64_t top = hi / 100000000u;
        put_digits8(p + len - 16, (uint32_t)(hi - top * 100000000u), 8);
        put_digits8(p, (uint32_t)top, len - 16);
    }
}

inline int ndigits(uint64_t v)
{
    int d = 1;
    while (d < 20 && v >= POW10[d])
        d++;
    return d;
}

inline char *put_exp(char *p, int X)
{
    *p++ = 'e';
    *p++ = X < 0 ? '-' : '+';
    const int a = X < 0 ? -X : X;
    if (a >= 100)
        *p++ = (char)('0' + a / 100);
    *p++ = (char)('0' + a / 10 % 10);
    *p++ = (char)('0' + a % 10);
    return p;
}

/*
 * %.Pe, %.Pf or %.Pg of the finite double with these bits into buf (at least
 * 64 bytes).  Returns the length, or 0 to leave the value to an exact
 * general routine.
 */
inline int format(char conv, int P, uint64_t bits, char *buf)
{
    if ((bits & ~(1ull << 63)) == 0 || P < 0)
        return 0;                             /* zero: the general routine */
    uint64_t m;
    int e;
    decompose(bits, &m, &e);
    double ax;
    {
        const uint64_t ab = bits & ~(1ull << 63);
        memcpy(&ax, &ab, 8);
    }
    char *p = buf;
    if (bits >> 63)
        *p++ = '-';
    if (conv == 'e') {
        if (P > 17)
            return 0;
        uint64_t N;
        int X;
        if (!sig_digits(m, e, ax, P + 1, &N, &X))
            return 0;
        char d[20];
        put_digits(d, N, P + 1);
        *p++ = d[0];
        if (P) {
            *p++ = '.';
            memcpy(p, d + 1, (size_t)P);
            p += P;
        }
        p = put_exp(p, X);
        return (int)(p - buf);
    }
    if (conv == 'f') {
        if (P > 17)
            return 0;
        uint64_t N;
        if (!scaled_round(m, e, P, &N) || N >= POW10[19])
            return 0;
        const int nd = ndigits(N);
        const int ip = nd > P ? nd - P : 1;   /* integer digits printed */
        char d[24];
        put_digits(d, N, ip + P);             /* zero-padded to the point */
        memcpy(p, d, (size_t)ip);
        p += ip;
        if (P) {
            *p++ = '.';
            memcpy(p, d + ip, (size_t)P);
            p += P;
        }
        return (int)(p - buf);
    }
    if (conv == 'g') {
        const int D = P == 0 ? 1 : P;
        if (D > 17)
            return 0;
        uint64_t N;
        int X;
        if (!sig_digits(m, e, ax, D, &N, &X))
            return 0;
        char d[20];
        put_digits(d, N, D);
        int sig = D;                          /* digits left after dropping trailing zeros */
        while (sig > 1 && d[sig - 1] == '0')
            sig--;
        if (X < -4 || X >= D) {               /* the %e form */
            *p++ = d[0];
            if (sig > 1) {
                *p++ = '.';
                memcpy(p, d + 1, (size_t)(sig - 1));
                p += sig - 1;
            }
            p = put_exp(p, X);
        } else if (X >= 0) {                  /* digits 0..X before the point */
            memcpy(p, d, (size_t)(X + 1));
            p += X + 1;
            if (sig > X + 1) {
                *p++ = '.';
                memcpy(p, d + X + 1, (size_t)(sig - X - 1));
                p += sig - X - 1;
            }
        } else {                              /* 0.000ddd */
            *p++ = '0';
            *p++ = '.';
            for (int z = 0; z < -X - 1; z++)
                *p++ = '0';
            memcpy(p, d, (size_t)sig);
            p += sig;
        }
        return (int)(p - buf);
    }
    return 0;
}

} // namespace dtoa
} // namespace gfh
#endif
