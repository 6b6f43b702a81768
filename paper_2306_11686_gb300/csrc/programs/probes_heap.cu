/*
 * Small programs that expose one runtime mechanism each, for the GPU tests:
 * the device heap's audit, its large path and its exhaustion behaviour.
 */
#include "../gf_device.cuh"
#include "../gf_fastdiv.cuh"
#include "../gf_intpipe.cuh"

/* heap_audit n per                  buffers: 0 = uint32 sizes[n*per], 1 = uint64 ptrs[n*per], 2 = uint64 info[4]
 * Every iteration allocates `per` blocks and keeps them live; the host audits
 * the (ptr, size) set, then a second region frees everything and a third
 * allocates again to check reuse. */
GF_MAIN(heap_audit)(int argc, char **argv)
{
    if (argc < 3)
        return 2;
    const long long n = gf_atoll(argv[1]);
    const int per = (int)gf_atoll(argv[2]);
    const unsigned *sz = (const unsigned *)gf_buffer(0);
    unsigned long long *ptr = (unsigned long long *)gf_buffer(1);
    unsigned long long *info = (unsigned long long *)gf_buffer(2);
    if (!sz || !ptr || !info)
        return 2;
    int rc = gf_parallel_for(0, n, GF_SCHED_STATIC, 1, [=](int64_t i) {
        for (int j = 0; j < per; j++) {
            const unsigned s = sz[i * per + j];
            unsigned long long *p = (unsigned long long *)gf_malloc(s);
            ptr[i * per + j] = (unsigned long long)p;
            if (p) {
                p[0] = (unsigned long long)(i * per + j);
                p[(s / 8) - 1] = ~(unsigned long long)(i * per + j);
            }
        }
    });
    /* every block still holds its tags: nobody else was handed overlapping memory */
    unsigned long long bad = 0;
    gf_reduce<long long, GF_RED_SUM>(0, n * per, GF_SCHED_STATIC, 1, [=](int64_t q) -> long long {
        unsigned long long *p = (unsigned long long *)ptr[q];
        if (!p)
            return 0;
        const unsigned s = sz[q];
        return (p[0] != (unsigned long long)q || p[(s / 8) - 1] != ~(unsigned long long)q) ? 1 : 0;
    }, (long long *)&bad);
    info[0] = bad;
    info[1] = gfd::s_st->heap.live_bytes;
    rc |= gf_parallel_for(0, n * per, GF_SCHED_STATIC, 1, [=](int64_t q) { gf_free((void *)ptr[q]); });
    info[2] = gfd::s_st->heap.live_bytes;
    /* allocate again: freed blocks come back */
    unsigned long long again = 0;
    gf_reduce<long long, GF_RED_SUM>(0, n * per, GF_SCHED_STATIC, 1, [=](int64_t q) -> long long {
        void *p = gf_malloc(sz[q]);
        const long long ok = p ? 1 : 0;
        gf_free(p);
        return ok;
    }, (long long *)&again);
    info[3] = again;
    return rc ? 10 : 0;
}

/* heap_big nbytes count            initial-thread large allocations; buffer 0 = uint64 ptrs[count] */
GF_MAIN(heap_big)(int argc, char **argv)
{
    if (argc < 3)
        return 2;
    const unsigned long long nb = (unsigned long long)gf_atoll(argv[1]);
    const int count = (int)gf_atoll(argv[2]);
    unsigned long long *out = (unsigned long long *)gf_buffer(0);
    for (int k = 0; k < count; k++)
        out[k] = (unsigned long long)gf_malloc(nb);
    gf_free((void *)out[1]);     /* hole in the middle, then reuse it */
    out[count] = (unsigned long long)gf_malloc(nb);
    for (int k = 0; k < count; k++)
        if (k != 1)
            gf_free((void *)out[k]);
    gf_free((void *)out[count]);
    out[count + 1] = (unsigned long long)gf_malloc(nb * count);   /* everything merged back */
    gf_free((void *)out[count + 1]);
    gf_free((void *)0x1234);     /* foreign pointer: counted, ignored */
    return 0;
}

/* heap_exhaust T per bytes          buffers: 0 = uint64 ptrs[2 * T * per]
 * Phase 1: T threads each allocate `per` blocks of `bytes` until the small
 * heap is exhausted (NULLs from then on); all of them are freed; phase 2
 * allocates the same way again, which can only be served from the freed
 * blocks on the per-lane stacks of every SM (no fresh slab is left); then
 * everything is freed again. */
GF_MAIN(heap_exhaust)(int argc, char **argv)
{
    if (argc < 4)
        return 2;
    const long long T = gf_atoll(argv[1]), per = gf_atoll(argv[2]);
    const size_t bytes = (size_t)gf_atoll(argv[3]);
    unsigned long long *ptrs = (unsigned long long *)gf_buffer(0);
    if (T < 1 || per < 1 || !ptrs || gf_buffer_bytes(0) < (uint64_t)(2 * T * per) * 8)
        return 2;
    for (int phase = 0; phase < 2; phase++) {
        unsigned long long *out = ptrs + (size_t)phase * T * per;
        if (gf_parallel_for(0, T, GF_SCHED_STATIC, 1, [=](int64_t t) {
                for (long long j = 0; j < per; j++) {
                    void *p = gf_malloc(bytes);
                    if (p)
                        *(volatile unsigned long long *)p = (unsigned long long)(t * per + j);
                    out[t * per + j] = (unsigned long long)p;
                }
            }))
            return 10;
        if (gf_parallel_for(0, T * per, GF_SCHED_STATIC, 1, [=](int64_t i) {
                void *p = (void *)out[i];
                if (p && *(volatile unsigned long long *)p != (unsigned long long)i)
                    out[i] |= 1ull;            /* a block shared by two owners: flag it */
                gf_free(p);
            }))
            return 11;
    }
    return 0;
}
