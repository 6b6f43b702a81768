/*
 * More of the partial GPU libc (paper Sec. 3.4: functions that run natively
 * without an RPC -- the paper names strtod, rand and realloc).
 *
 * gf_srand / gf_rand: the generator behind glibc's rand() (the default
 * TYPE_3 additive feedback generator), from its published description
 * (P. Selinger, "The GLIBC pseudo-random number generator"): r0 = seed;
 * r_i = 16807 r_{i-1} mod (2^31 - 1) for i = 1..30 (Schrage's method);
 * r_i = r_{i-31} for i = 31..33; r_i = r_{i-31} + r_{i-3} mod 2^32 after;
 * output k is r_{k+344} >> 1.  A program therefore sees the same sequence on
 * the GPU as on the host.  The state is the program's; calls from a region
 * are serialised by a lock (as glibc's rand() locks), so their interleaving
 * across threads is unspecified.
 *
 * gf_realloc: in place when the heap block already has room, otherwise
 * malloc + copy + free; realloc(NULL, n) = malloc(n); realloc(p, 0) frees p
 * and returns NULL.
 *
 * gf_strtod: decimal strings with at most 15 significant digits and a
 * decimal exponent of magnitude at most 22 are converted natively, exactly:
 * the digits and the power of ten are both exact doubles, so one IEEE
 * multiply or divide rounds once (Clinger's fast path, W. D. Clinger, "How to
 * read floating point numbers accurately", PLDI 1990).  Everything else
 * (more digits, large exponents, hex floats, inf/nan) goes to the host's
 * strtod by RPC, so every result is the correctly rounded one.
 */
#ifndef GF_DEVICE_LIBC_CUH
#define GF_DEVICE_LIBC_CUH

#include "gf_device.cuh"
#include "gf_strtod_fast.h"

namespace gfd {
struct rand_state {
    int32_t r[34];               /* the last 31 (of 34) values, ring indexed by pos */
    uint32_t pos, lock, seeded;
};
__device__ inline rand_state *rstate() { return (rand_state *)&s_st->rand_words[0]; }

__device__ inline void rand_lock(rand_state *s)
{
    if (is_initial_thread())
        return;
    for (int k = 0; k < (1 << 22); k++) {
        if (atomicCAS(&s->lock, 0u, 1u) == 0u) {
            __threadfence();
            return;
        }
        __nanosleep(64);
    }
}
__device__ inline void rand_unlock(rand_state *s)
{
    if (is_initial_thread())
        return;
    __threadfence();
    atomicExch(&s->lock, 0u);
}

__device__ inline int32_t rand_next(rand_state *s)
{
    /* ring of 34: r_i = r_{i-31} + r_{i-3} */
    const uint32_t i = s->pos;
    const int32_t v = (int32_t)((uint32_t)s->r[(i + 34 - 31) % 34] + (uint32_t)s->r[(i + 34 - 3) % 34]);
    s->r[i % 34] = v;
    s->pos = (i + 1) % 34;
    return v;
}

__device__ inline void srand_locked(rand_state *s, uint32_t seed)
{
    int32_t r[34];
    r[0] = (int32_t)(seed ? seed : 1u);
    for (int i = 1; i < 31; i++) {
        const int32_t hi = r[i - 1] / 127773, lo = r[i - 1] % 127773;
        int32_t w = 16807 * lo - 2836 * hi;
        if (w < 0)
            w += 2147483647;
        r[i] = w;
    }
    for (int i = 31; i < 34; i++)
        r[i] = r[i - 31];
    for (int i = 0; i < 34; i++)
        s->r[i] = r[i];
    s->pos = 0;                  /* next value written overwrites r[0] = r_34 */
    for (int k = 34; k < 344; k++)
        rand_next(s);
    s->seeded = 1;
}
} // namespace gfd

__device__ inline void gf_srand(unsigned seed)
{
    gfd::rand_state *s = gfd::rstate();
    gfd::rand_lock(s);
    gfd::srand_locked(s, seed);
    gfd::rand_unlock(s);
}

__device__ inline int gf_rand()
{
    gfd::rand_state *s = gfd::rstate();
    gfd::rand_lock(s);
    if (!s->seeded)
        gfd::srand_locked(s, 1u);             /* C: rand() before srand() behaves as srand(1) */
    const int v = (int)((uint32_t)gfd::rand_next(s) >> 1);
    gfd::rand_unlock(s);
    return v;
}

__device__ inline void *gf_realloc(void *p, size_t n)
{
    if (!p)
        return gf_malloc(n);
    if (n == 0) {
        gf_free(p);
        return nullptr;
    }
    const uint64_t cap = gf_heap_block_size(p);
    if (cap && n <= cap)
        return p;
    void *q = gf_malloc(n);
    if (!q)
        return nullptr;
    const uint64_t keep = cap < n ? cap : n;
    const unsigned char *s = (const unsigned char *)p;
    unsigned char *d = (unsigned char *)q;
    if (!(((uintptr_t)s | (uintptr_t)d | keep) & 15u)) {
        for (uint64_t k = 0; k < keep / 16; k++)
            ((uint4 *)d)[k] = ((const uint4 *)s)[k];
    } else {
        for (uint64_t k = 0; k < keep; k++)
            d[k] = s[k];
    }
    gf_free(p);
    return q;
}

__device__ inline double gf_strtod(const char *str, char **endptr)
{
    double v;
    const char *end;
    if (gf_strtod_fast(str, &v, &end)) {
        if (endptr)
            *endptr = (char *)end;
        return v;
    }
    /* exact slow path on the host: value bits returned, consumed length written back */
    long long used = 0;
    int st = 0;
    const long long bits = gfd::rpc(GF_OP_STRTOD, nullptr, &st, str, gf_ref_write(&used, 8, 0));
    if (endptr)
        *endptr = (char *)str + (st == GF_OK ? used : 0);
    return st == GF_OK ? __longlong_as_double(bits) : 0.0;
}

#endif
