/*
 * The decimal fast path of gf_strtod, for host and device (the host build is
 * what the CPU tests compare with the C library's strtod).
 *
 * A decimal string with at most 15 significant digits and a decimal exponent
 * of magnitude at most 22 is converted exactly: the digits and the power of
 * ten are both exact doubles, so one IEEE multiply or divide rounds once
 * (Clinger's fast path, W. D. Clinger, "How to read floating point numbers
 * accurately", PLDI 1990).  Anything else -- more digits, larger exponents,
 * hex floats, inf/nan, no number at all -- returns false and the caller takes
 * the exact host conversion.
 */
#ifndef GF_STRTOD_FAST_H
#define GF_STRTOD_FAST_H

#if defined(__CUDACC__)
#define GF_HD __host__ __device__
#else
#define GF_HD
#endif

GF_HD inline double gf_mul_rn(double a, double b)
{
#ifdef __CUDA_ARCH__
    return __dmul_rn(a, b);
#else
    volatile double r = a * b;                  /* one rounded product, never contracted */
    return r;
#endif
}

GF_HD inline double gf_div_rn(double a, double b)
{
#ifdef __CUDA_ARCH__
    return __ddiv_rn(a, b);
#else
    volatile double r = a / b;
    return r;
#endif
}

/* true: *out is the correctly rounded value of the number at the start of
 * str (after white space) and *end points past it, as strtod would set it */
GF_HD inline bool gf_strtod_fast(const char *str, double *out, const char **end)
{
    const char *p = str;
    while (*p == ' ' || *p == '\t' || *p == '\n' || *p == '\r' || *p == '\f' || *p == '\v')
        p++;
    bool neg = false;
    if (*p == '+' || *p == '-')
        neg = (*p++ == '-');
    if (p[0] == '0' && (p[1] == 'x' || p[1] == 'X'))
        return false;                           /* hex float: the leading 0 is not the number */
    unsigned long long mant = 0;
    int digits = 0, exp10 = 0;
    bool any = false;
    for (; *p >= '0' && *p <= '9'; p++) {
        any = true;
        if (mant == 0 && *p == '0')
            continue;                           /* leading zeros are not significant */
        if (digits == 15)
            return false;
        mant = mant * 10 + (unsigned)(*p - '0');
        digits++;
    }
    if (*p == '.') {
        p++;
        for (; *p >= '0' && *p <= '9'; p++) {
            any = true;
            if (mant == 0 && *p == '0') {
                exp10--;
                continue;
            }
            if (digits == 15)
                return false;
            mant = mant * 10 + (unsigned)(*p - '0');
            digits++;
            exp10--;
        }
    }
    if (!any)
        return false;                           /* inf, nan or no number: the host decides */
    if (*p == 'e' || *p == 'E') {
        const char *q = p + 1;
        bool eneg = false;
        if (*q == '+' || *q == '-')
            eneg = (*q++ == '-');
        if (*q >= '0' && *q <= '9') {           /* else the exponent is not part of the number */
            int e = 0;
            for (; *q >= '0' && *q <= '9'; q++)
                e = e < 100000 ? e * 10 + (*q - '0') : e;
            exp10 += eneg ? -e : e;
            p = q;
        }
    }
    if (mant == 0)
        exp10 = 0;                              /* zero with any exponent is zero */
    if (exp10 < -22 || exp10 > 22)
        return false;
    const int ae = exp10 < 0 ? -exp10 : exp10;
    double p10 = 1.0;                           /* 10^k for k <= 22 is exact, and so is each step */
    for (int k = 0; k < ae; k++)
        p10 = gf_mul_rn(p10, 10.0);
    double v = (double)mant;                    /* exact: mant < 10^15 < 2^53 */
    v = exp10 >= 0 ? gf_mul_rn(v, p10) : gf_div_rn(v, p10);
    *out = neg ? -v : v;
    *end = p;
    return true;
}

#endif
