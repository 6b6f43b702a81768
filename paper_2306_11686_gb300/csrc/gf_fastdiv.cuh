/*
 * Correctly rounded division by the constant 6.0 in three FP64 operations
 * (the integer-pipe version, gf_div6_int, is in gf_intpipe.cuh).
 *
 * GB300 issues FP64 instructions at a small fraction of its other rates, and
 * a general IEEE double division costs several of them; a compiler may
 * replace a division by a constant with any sequence that returns the same
 * correctly rounded quotient.  This one is Markstein's correction step
 * (P. Markstein, "Computation of elementary functions on the IBM RISC
 * System/6000 processor", IBM J. Res. Dev. 34(1), 1990):
 *
 *   r = RN(1/6),  q = RN(x r),  rho = x - 6 q  (exact in one FMA),
 *   result = RN(q + rho r).
 *
 * Why it is exact here, for normal x with no overflow or underflow on the way
 * (|x| in [2^-1000, 2^1000]):
 *  - q is within 1.5 ulp(q) of x/6, so x - 6q is a small integer multiple of
 *    ulp(q) and is representable: the FMA computes it without error;
 *  - q + rho r = x/6 + (x/6 - q) (6r - 1), off x/6 by less than 2^-52 ulp;
 *  - x/6 is never a rounding midpoint (6 times a midpoint is an odd multiple
 *    of ulp(q), while x is a multiple of 4 ulp(q)), and any other quotient is
 *    at least ulp(q)/6 from one, so both round to the same double.
 * Every other x (0, subnormal, huge, inf, NaN) takes the IEEE division.
 * The tests compare it bit for bit with x / 6.0 over many binades.
 */
#ifndef GF_FASTDIV_CUH
#define GF_FASTDIV_CUH

/* out of line, so that no part of the general division is hoisted into the
 * fast path */
static __device__ __noinline__ double gf_div6_ieee(double x) { return x / 6.0; }

__device__ __forceinline__ double gf_div6_rn(double x)
{
    const double r = 1.0 / 6.0;                      /* folded at compile time: RN(1/6) */
    const unsigned e = (unsigned)((__double_as_longlong(x) >> 52) & 0x7ff);
    if (e - 23u > 2000u)                             /* outside [2^-1000, 2^1001): IEEE path */
        return gf_div6_ieee(x);
    const double q = __dmul_rn(x, r);
    const double rho = __fma_rn(q, -6.0, x);        /* x - 6q, exact; the sign sits on the constant */
    return __fma_rn(rho, r, q);
}

#endif
