/*
 * FP64 results computed on the integer pipe, bit for bit the IEEE ones.
 *
 * GB300 retires FP64 instructions at 2 lanes per clock per SM and integer
 * ALU instructions at 64 (16 per clock on each of the 4 sub-partitions).
 * A loop whose FP64 instructions saturate their pipe (a stencil of adds,
 * say) leaves the integer pipe partly idle; moving some of its correctly
 * rounded operations onto integer instructions splits the work between the
 * two pipes without changing any result.  An emulated add costs tens of
 * ALU instructions (more pipe time than one FP64 add), so it pays only for
 * the share of the adds the integer pipe has room for.
 *
 *   gf_div6_int(x)     x / 6.0, round to nearest even;
 *   gf_dadd_int(x, y)  x + y, round to nearest even, for operands of the same
 *                      sign (or one of them zero); other cases (opposite
 *                      signs, both zero, subnormal, inf, NaN, results near
 *                      overflow) take the FP64 add;
 *   gf_fabs_int(x)     |x| as a sign-bit clear the compiler cannot turn back
 *                      into an FP64 instruction;
 *   gf_udiv32          floor(x / d) for x < 2^31 by one 32x32->64 multiply
 *                      and a shift (T. Granlund, P. Montgomery, "Division by
 *                      invariant integers using multiplication", PLDI 1994).
 *
 * The add follows the textbook same-sign path (e.g. J.-M. Muller et al.,
 * "Handbook of Floating-Point Arithmetic", Ch. 7): the significands, widened
 * by 10 guard bits, are aligned with a sticky bit, added, renormalised by at
 * most one position, and rounded to nearest even on the guard bits.  Small
 * exponent gaps, where no bit falls below the guard bits, skip the sticky
 * and form the exact sum directly.
 * Everything is host+device so the CPU tests can compare it with the host's
 * IEEE arithmetic over many operands.
 */
#ifndef GF_INTPIPE_CUH
#define GF_INTPIPE_CUH
#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define GF_IP_HD __host__ __device__ __forceinline__
#else
#define GF_IP_HD inline
#endif

/* The moves between FP64 and integer registers are opaque to the compiler:
 * otherwise it recognises a sign-bit mask of a reinterpreted double as fabs,
 * a sign-bit merge as copysign, a magnitude test as an FP64 compare, and
 * emits those on the FP64 pipe this code is meant to leave alone. */
GF_IP_HD uint64_t gf_ip_bits(double x)
{
#ifdef __CUDA_ARCH__
    uint64_t b;
    asm("mov.b64 %0, %1;" : "=l"(b) : "d"(x));
    return b;
#else
    uint64_t b;
    memcpy(&b, &x, 8);
    return b;
#endif
}

GF_IP_HD double gf_ip_double(uint64_t b)
{
#ifdef __CUDA_ARCH__
    double x;
    asm("mov.b64 %0, %1;" : "=d"(x) : "l"(b));
    return x;
#else
    double x;
    memcpy(&x, &b, 8);
    return x;
#endif
}

/* the FP64 add for the cases the integer path leaves out */
#ifdef __CUDA_ARCH__
static __device__ __noinline__ double gf_ip_dadd_hw(double x, double y) { return __dadd_rn(x, y); }
#else
static inline double gf_ip_dadd_hw(double x, double y)
{
    volatile double r = x + y;
    return r;
}
#endif

/* the same-sign add at any exponent gap (the textbook path) */
GF_IP_HD double gf_dadd_int_any(double x, double y)
{
    const uint64_t SIGN = 0x8000000000000000ull, FRAC = 0x000fffffffffffffull, HID = 1ull << 52;
    uint64_t a = gf_ip_bits(x), b = gf_ip_bits(y);
    if ((a & ~SIGN) < (b & ~SIGN)) {             /* a: the operand of larger magnitude */
        const uint64_t t = a;
        a = b;
        b = t;
    }
    const uint64_t am = a & ~SIGN, bm = b & ~SIGN;
    if (bm == 0 && am != 0)                      /* x + 0 = x for x != 0, either zero */
        return gf_ip_double(a);
    const uint32_t ea = (uint32_t)(am >> 52), eb = (uint32_t)(bm >> 52);
    /* same sign, b normal (so a too), a at most 2^1022 so the sum stays finite
     * or rounds straight to inf */
    if (((a ^ b) & SIGN) || eb == 0 || ea > 2045u)
        return gf_ip_dadd_hw(x, y);
    const uint32_t d = ea - eb;
    const uint64_t ma = ((am & FRAC) | HID) << 10;          /* [2^62, 2^63) */
    uint64_t mb = ((bm & FRAC) | HID) << 10;
    if (d >= 63u)
        mb = 1;                                  /* all of it below the guard bits: sticky only */
    else if (d)
        mb = (mb >> d) | ((mb << (64u - d)) != 0 ? 1u : 0u);
    uint64_t s = ma + mb;                        /* < 2^64 */
    uint64_t e = ea;
    if (s >> 63) {                               /* carry out: one position right, keep the sticky */
        s = (s >> 1) | (s & 1u);
        e++;
    }
    uint64_t m = s >> 10;                        /* [2^52, 2^53) */
    const uint32_t g = (uint32_t)s & 0x3ffu;     /* the 10 guard bits, sticky in the lowest */
    m += (g > 0x200u || (g == 0x200u && (m & 1u))) ? 1u : 0u;
    /* (e - 1) 2^52 + m: a carry of the rounding into 2^53 moves into the
     * exponent (and from 2046 into the inf encoding) */
    return gf_ip_double((a & SIGN) | (((e - 1u) << 52) + m));
}

/* x + y, round to nearest even.  Exponent gaps up to 10 (neighbouring grid
 * values nearly always) take a shorter path: in units of the smaller
 * operand's ulp the exact sum S = ma 2^d + mb fits in 64 bits, so it is
 * formed exactly and rounded once, by s = d or d + 1 positions (one more
 * when S carries into the next binade).  Everything else takes the path
 * above. */
GF_IP_HD double gf_dadd_int(double x, double y)
{
    const uint64_t SIGN = 0x8000000000000000ull, FRAC = 0x000fffffffffffffull, HID = 1ull << 52;
    uint64_t a = gf_ip_bits(x), b = gf_ip_bits(y);
    if ((a & ~SIGN) < (b & ~SIGN)) {
        const uint64_t t = a;
        a = b;
        b = t;
    }
    const uint64_t am = a & ~SIGN, bm = b & ~SIGN;
    const uint32_t ea = (uint32_t)(am >> 52), eb = (uint32_t)(bm >> 52);
    const uint32_t d = ea - eb;
    if (((a ^ b) & SIGN) || eb == 0 || ea > 2045u || d > 10u)
        return gf_dadd_int_any(x, y);
    const uint64_t ma = (am & FRAC) | HID, mb = (bm & FRAC) | HID;
    const uint64_t S = (ma << d) + mb;                 /* < 2^64, exact */
    const uint32_t s = d + (uint32_t)(S >> (53u + d)); /* 1 .. 11 (d = 0 always carries) */
    uint64_t q = S >> s;                               /* [2^52, 2^53) */
    const uint32_t rem = (uint32_t)S & ((1u << s) - 1u), half = 1u << (s - 1u);
    q += (rem > half || (rem == half && (q & 1u))) ? 1u : 0u;
    /* the result is q 2^(eb + s - 1075): biased exponent eb + s, and a
     * rounding carry of q into 2^53 moves into the exponent as above */
    return gf_ip_double((a & SIGN) | (((uint64_t)(eb + s - 1u) << 52) + q));
}

GF_IP_HD double gf_fabs_int(double x)
{
    return gf_ip_double(gf_ip_bits(x) & 0x7fffffffffffffffull);
}

/*
 * The same quotient on the integer pipe (GB300's integer rate is many times
 * its FP64 rate).  For normal x = m 2^(E-52) with integer m in [2^52, 2^53):
 *
 *   x / 6 = (m 2^k / 3) 2^(E-53-k),   k = 2 if m < 3 * 2^51, else k = 1,
 *
 * which puts the exact quotient q* = m 2^k / 3 in [2^52, 2^53).  With
 * q = floor(q*) and r = m 2^k - 3q in {0, 1, 2}, the discarded fraction is
 * r/3 in {0, 1/3, 2/3}: never exactly one half, so round-to-nearest-even is
 * "add one iff r = 2", and q + 1 stays below 2^53 (its largest case,
 * m = 3 * 2^51 - 1, gives q = 2^53 - 2).  The biased exponent of the result
 * is E_biased - 1 - k; results that would be subnormal, and inputs that are
 * zero, subnormal, inf or NaN, take the IEEE division.  The tests compare it
 * bit for bit with the hardware division on the CPU and the GPU.
 */
GF_IP_HD double gf_div6_int(double x)
{
    const uint64_t b = gf_ip_bits(x);
    const uint32_t eb = (uint32_t)(b >> 52) & 0x7ffu;
    if (eb - 4u > 2042u)                        /* zero, subnormal, tiny results, inf, NaN */
        return x / 6.0;
    const uint64_t m = (b & 0xfffffffffffffull) | (1ull << 52);
    const uint32_t k = m < (3ull << 51) ? 2u : 1u;
    const uint64_t n = m << k;                  /* < 3 * 2^53 */
#ifdef __CUDA_ARCH__
    const uint64_t q = __umul64hi(n, 0xAAAAAAAAAAAAAAABull) >> 1;   /* floor(n / 3) */
#else
    const uint64_t q = (uint64_t)(((unsigned __int128)n * 0xAAAAAAAAAAAAAAABull) >> 65);
#endif
    const uint64_t r = n - 3ull * q;
    const uint64_t mq = q + (r == 2ull ? 1ull : 0ull);
    return gf_ip_double((b & 0x8000000000000000ull) | ((uint64_t)(eb - 1u - k) << 52) | (mq & 0xfffffffffffffull));
}

/* floor(x / d) for 0 <= x < 2^31 and 1 <= d < 2^31:
 * k = 31 + ceil(log2 d), M = ceil(2^k / d) < 2^32; then M d - 2^k < d, so
 * x (M d - 2^k) < 2^31 d <= 2^k and floor(x M / 2^k) = floor(x / d). */
struct gf_udiv32 {
    uint32_t m, k;
    GF_IP_HD static gf_udiv32 make(uint32_t d)
    {
        uint32_t l = 0;
        while (l < 31u && (1u << l) < d)
            l++;
        gf_udiv32 r;
        r.k = 31u + l;
        r.m = (uint32_t)(((1ull << r.k) + d - 1u) / d);
        return r;
    }
    GF_IP_HD uint32_t div(uint32_t x) const { return (uint32_t)(((uint64_t)x * m) >> k); }
};

#endif
