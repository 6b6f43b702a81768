/*
 * Fast path of the host printf landing pad for the plainest conversions.
 *
 * A conversion with no flags, no field width and no '*' -- %d %i %u %x %o
 * (any length modifier, no precision) and %e %f %g with an optional
 * precision -- is formatted by std::to_chars, whose output the C++ standard
 * defines as that of printf with the same conversion and precision in the
 * "C" locale.  Non-finite values, %g with precision 0, long double, and
 * anything that does not fit the buffer return false, and the caller uses
 * snprintf.  glibc's printf converts doubles with multi-precision
 * arithmetic; to_chars (Ryu-printf in libstdc++) is several times faster,
 * which matters when one device warp ships 32 formatted calls per slot.
 * Doubles at precisions up to 17 digits first try dtoa::format
 * (dtoa_fixed.h), a 128-bit table-driven conversion that is faster again
 * and declines the cases it cannot decide exactly.
 */
#ifndef GF_FMT_FAST_H
#define GF_FMT_FAST_H

#include <charconv>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "dtoa_fixed.h"

namespace gfh {

/* len: the length modifier ("", "h", "hh", "l", "ll", "j", "z", "t", "q", "L");
 * prec: -1 if the spec has none; w: the argument word; is_f64: the argument
 * was passed as a double.  On true, buf[0..*n) holds the conversion. */
inline bool fmt_fast(char conv, const char *len, int prec, uint64_t w, bool is_f64, char *buf, size_t cap, int *n)
{
    std::to_chars_result r;
    char *const end = buf + cap;
    switch (conv) {
    case 'd':
    case 'i': {
        if (prec >= 0)
            return false;
        long long v;
        if (len[0] == 'l' || len[0] == 'j' || len[0] == 'z' || len[0] == 't' || len[0] == 'q')
            v = (long long)w;                       /* long and long long are 64-bit here */
        else if (len[0] == 'h' && len[1] == 'h')
            v = (signed char)w;
        else if (len[0] == 'h')
            v = (short)w;
        else if (len[0] == 0)
            v = (int)w;
        else
            return false;
        r = std::to_chars(buf, end, v);
        break;
    }
    case 'u':
    case 'x':
    case 'o': {
        if (prec >= 0)
            return false;
        unsigned long long v;
        if (len[0] == 'l' || len[0] == 'j' || len[0] == 'z' || len[0] == 't' || len[0] == 'q')
            v = (unsigned long long)w;
        else if (len[0] == 'h' && len[1] == 'h')
            v = (unsigned char)w;
        else if (len[0] == 'h')
            v = (unsigned short)w;
        else if (len[0] == 0)
            v = (unsigned)w;
        else
            return false;
        r = std::to_chars(buf, end, v, conv == 'u' ? 10 : conv == 'x' ? 16 : 8);
        break;
    }
    case 'e':
    case 'f':
    case 'g': {
        if (len[0] == 'L' || (len[0] && len[0] != 'l'))
            return false;
        double d;
        if (is_f64)
            memcpy(&d, &w, 8);
        else
            d = (double)(int64_t)w;
        const int p = prec < 0 ? 6 : prec;
        if (!std::isfinite(d) || (conv == 'g' && p == 0))
            return false;
        if (cap >= 64) {                        /* the fixed-precision path, exact or declined */
            uint64_t bits;
            memcpy(&bits, &d, 8);
            const int k = dtoa::format(conv, p, bits, buf);
            if (k > 0) {
                *n = k;
                return true;
            }
        }
        const std::chars_format f = conv == 'e' ? std::chars_format::scientific
                                    : conv == 'f' ? std::chars_format::fixed
                                                  : std::chars_format::general;
        r = std::to_chars(buf, end, d, f, p);
        break;
    }
    default:
        return false;
    }
    if (r.ec != std::errc())
        return false;
    *n = (int)(r.ptr - buf);
    return true;
}

} // namespace gfh

#endif
