/*
 * ORACLE (test infrastructure only).  Only tests/, __graft_entry__.smoke() and
 * bench.py's cpu_baseline leg may build, call or run anything under oracle/.
 *
 * Exactly rounded sum of binary64 values.  The paper leaves reductions in
 * multi-team regions unimplemented (Sec. 4.3), so the reduction added here is
 * checked against the plain definition: the real-number sum of the inputs,
 * rounded once to nearest-even.  The method is a Kulisch-style long
 * accumulator: every finite double is m * 2^e with an integer |m| < 2^53 and
 * e >= -1074, so all of them are integers in units of 2^-1074 and their sum is
 * held exactly in a fixed-point big integer (70 limbs of 32 bits, bit 0 worth
 * 2^-1074, headroom above 2^1024 for 2^40 terms), then rounded once.
 *
 *   exact_sum file.bin      prints  "naive %.17g\nexact %.17g\nabsum %.17g\n"
 *
 * naive is the left-to-right serial sum; absum is the exactly rounded sum of
 * |x_i| (the scale of the error bound of a compensated sum).  Non-finite
 * inputs are rejected.
 */
#include <stdio.h>
#include <stdlib.h>
#include <stdint.h>
#include <string.h>
#include <math.h>

#define LIMBS 70

typedef struct {
    int64_t d[LIMBS];   /* d[k] holds a signed multiple of 2^(32k) in units of 2^-1074 */
    long pending;       /* additions since the last carry normalisation */
} kacc;

static void kacc_norm(kacc *a)
{
    for (int k = 0; k < LIMBS - 1; k++) {
        int64_t carry = a->d[k] >> 32;          /* arithmetic shift: floor division */
        a->d[k] -= carry * ((int64_t)1 << 32);
        a->d[k + 1] += carry;
    }
    a->pending = 0;
}

static void kacc_add(kacc *a, double x)
{
    if (x == 0.0)
        return;
    int e;
    double fr = frexp(fabs(x), &e);             /* |x| = fr * 2^e, fr in [0.5, 1) */
    /* integer mantissa m = fr * 2^53 and exponent of its unit: |x| = m * 2^(e-53) */
    uint64_t m = (uint64_t)ldexp(fr, 53);
    int p = e - 53 + 1074;                      /* bit position of m's unit */
    if (p < 0) {                                /* subnormal: m has trailing zeros */
        m >>= -p;
        p = 0;
    }
    int k = p / 32, s = p % 32;
    unsigned __int128 w = (unsigned __int128)m << s;
    int64_t sign = x < 0 ? -1 : 1;
    for (int t = 0; t < 3 && k + t < LIMBS; t++) {
        a->d[k + t] += sign * (int64_t)(uint32_t)(w & 0xFFFFFFFFu);
        w >>= 32;
    }
    if (++a->pending >= (1L << 29))
        kacc_norm(a);
}

/* bit b of the non-negative normalised magnitude */
static int getbit(const uint32_t *mag, int b)
{
    return (mag[b / 32] >> (b % 32)) & 1u;
}

static double kacc_round(kacc *a)
{
    kacc_norm(a);
    uint32_t mag[LIMBS];
    int neg = a->d[LIMBS - 1] < 0;
    /* two's complement magnitude */
    uint64_t borrow = 0;
    if (!neg) {
        for (int k = 0; k < LIMBS; k++)
            mag[k] = (uint32_t)a->d[k];
    } else {
        /* magnitude = -value: invert limbs (value = sum d[k] 2^32k with d[k] in [0,2^32) except top) */
        uint64_t c = 1;
        for (int k = 0; k < LIMBS; k++) {
            uint64_t v = (uint64_t)(~(uint32_t)a->d[k]) + c;
            mag[k] = (uint32_t)v;
            c = v >> 32;
        }
    }
    (void)borrow;
    int top = -1;
    for (int b = LIMBS * 32 - 1; b >= 0; b--)
        if (getbit(mag, b)) {
            top = b;
            break;
        }
    if (top < 0)
        return 0.0;
    double r;
    if (top < 53) {
        uint64_t v = 0;
        for (int b = top; b >= 0; b--)
            v = (v << 1) | getbit(mag, b);
        r = ldexp((double)v, -1074);            /* exact: multiple of 2^-1074 below 2^-1021 */
    } else {
        int shift = top - 52;
        uint64_t mant = 0;
        for (int b = top; b >= shift; b--)
            mant = (mant << 1) | getbit(mag, b);
        int rnd = getbit(mag, shift - 1);
        int sticky = 0;
        for (int b = shift - 2; b >= 0 && !sticky; b--)
            sticky = getbit(mag, b);
        if (rnd && (sticky || (mant & 1)))
            mant++;
        if (mant == (1ull << 53)) {
            mant >>= 1;
            shift++;
        }
        r = ldexp((double)mant, shift - 1074);
    }
    return neg ? -r : r;
}

int main(int argc, char **argv)
{
    if (argc != 2) {
        fprintf(stderr, "usage: exact_sum file.bin\n");
        return 2;
    }
    FILE *f = fopen(argv[1], "rb");
    if (!f) {
        fprintf(stderr, "exact_sum: cannot open %s\n", argv[1]);
        return 2;
    }
    static kacc acc, aacc;
    memset(&acc, 0, sizeof acc);
    memset(&aacc, 0, sizeof aacc);
    double naive = 0.0, buf[4096];
    size_t got;
    while ((got = fread(buf, sizeof(double), 4096, f)) > 0) {
        for (size_t i = 0; i < got; i++) {
            if (!isfinite(buf[i])) {
                fprintf(stderr, "exact_sum: non-finite input\n");
                return 3;
            }
            naive += buf[i];
            kacc_add(&acc, buf[i]);
            kacc_add(&aacc, fabs(buf[i]));
        }
    }
    fclose(f);
    printf("naive %.17g\nexact %.17g\nabsum %.17g\n", naive, kacc_round(&acc), kacc_round(&aacc));
    return 0;
}
