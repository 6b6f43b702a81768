/*
 * Small programs that expose one runtime mechanism each, for the GPU tests:
 * schedules, reductions, the cross-block barrier, RPC landing pads, the heap
 * audit and the bounded-wait error path.
 */
#include "../gf_device.cuh"
#include "../gf_fastdiv.cuh"
#include "../gf_intpipe.cuh"

/* sched_probe b e sched chunk      buffers: 0 = int32 hits[e-b], 1 = int64 owner[e-b], 2 = int64 info[2]
 * Every iteration records which continuous thread id ran it. */
GF_MAIN(sched_probe)(int argc, char **argv)
{
    if (argc < 5)
        return 2;
    const long long b = gf_atoll(argv[1]), e = gf_atoll(argv[2]);
    const int sched = (int)gf_atoll(argv[3]);
    const long long chunk = gf_atoll(argv[4]);
    int *hits = (int *)gf_buffer(0);
    long long *owner = (long long *)gf_buffer(1);
    long long *info = (long long *)gf_buffer(2);
    if (!hits || !owner || !info)
        return 2;
    info[0] = 0;
    int rc = gf_parallel_for(b, e, sched, chunk, [=](int64_t i) {
        atomicAdd(&hits[i - b], 1);
        owner[i - b] = gf_thread_num();
        if (i == b)
            info[0] = gf_num_threads();
    });
    info[1] = gf_num_threads();   /* the initial thread outside a region: a team of 1 */
    return rc ? 10 : 0;
}

/* reduce_probe n sched chunk       buffers: 0 = double x[n], 1 = int64 v[n], 2 = out[6] */
GF_MAIN(reduce_probe)(int argc, char **argv)
{
    if (argc < 4)
        return 2;
    const long long n = gf_atoll(argv[1]);
    const int sched = (int)gf_atoll(argv[2]);
    const long long chunk = gf_atoll(argv[3]);
    const double *x = (const double *)gf_buffer(0);
    const long long *v = (const long long *)gf_buffer(1);
    uint64_t *out = (uint64_t *)gf_buffer(2);
    if (!x || !v || !out)
        return 2;
    double d;
    long long l;
    int rc = 0;
    rc |= gf_reduce<double, GF_RED_SUM>(0, n, sched, chunk, [=](int64_t i) { return x[i]; }, &d);
    out[0] = __double_as_longlong(d);
    rc |= gf_reduce<double, GF_RED_MIN>(0, n, sched, chunk, [=](int64_t i) { return x[i]; }, &d);
    out[1] = __double_as_longlong(d);
    rc |= gf_reduce<double, GF_RED_MAX>(0, n, sched, chunk, [=](int64_t i) { return x[i]; }, &d);
    out[2] = __double_as_longlong(d);
    rc |= gf_reduce<long long, GF_RED_SUM>(0, n, sched, chunk, [=](int64_t i) { return v[i]; }, &l);
    out[3] = (uint64_t)l;
    rc |= gf_reduce<long long, GF_RED_MIN>(0, n, sched, chunk, [=](int64_t i) { return v[i]; }, &l);
    out[4] = (uint64_t)l;
    rc |= gf_reduce<long long, GF_RED_MAX>(0, n, sched, chunk, [=](int64_t i) { return v[i]; }, &l);
    out[5] = (uint64_t)l;
    return rc ? 10 : 0;
}

/* range_probe b e                  buffer 0 = int64 out[4]
 * Static chunk-1 loops over [b, e) with a large base: the count, the sum of
 * i - b, min and max of i, as integer reductions (a trampoline of its own
 * below 2^31 iterations, the generic 64-bit loop above). */
GF_MAIN(range_probe)(int argc, char **argv)
{
    if (argc < 3)
        return 2;
    const long long b = gf_atoll(argv[1]), e = gf_atoll(argv[2]);
    long long *out = (long long *)gf_buffer(0);
    if (!out)
        return 2;
    long long r;
    int rc = 0;
    rc |= gf_reduce<long long, GF_RED_SUM>(b, e, GF_SCHED_STATIC, 1, [=](int64_t i) { return 1ll; }, &r);
    out[0] = r;
    rc |= gf_reduce<long long, GF_RED_SUM>(b, e, GF_SCHED_STATIC, 1, [=](int64_t i) { return (long long)(i - b); }, &r);
    out[1] = r;
    rc |= gf_reduce<long long, GF_RED_MIN>(b, e, GF_SCHED_STATIC, 1, [=](int64_t i) { return (long long)i; }, &r);
    out[2] = r;
    rc |= gf_reduce<long long, GF_RED_MAX>(b, e, GF_SCHED_STATIC, 1, [=](int64_t i) { return (long long)i; }, &r);
    out[3] = r;
    return rc ? 10 : 0;
}

/* barrier_probe rounds             buffers: 0 = int64 a[T], 1 = int64 errors[1]
 * Each worker writes its slot, crosses the grid barrier, and reads a slot
 * written by a thread of another block; any stale value counts an error. */
GF_MAIN(barrier_probe)(int argc, char **argv)
{
    if (argc < 2)
        return 2;
    const int rounds = (int)gf_atoll(argv[1]);
    long long *a = (long long *)gf_buffer(0);
    unsigned long long *err = (unsigned long long *)gf_buffer(1);
    if (!a || !err)
        return 2;
    const int T = (int)(gfd::s_st->nblocks * gfd::s_st->block_dim - 32);
    if (gf_buffer_bytes(0) < (uint64_t)T * 8)
        return 3;
    int rc = gf_parallel_for(0, T, GF_SCHED_STATIC, 1, [=](int64_t t) {
        const int64_t other = (t + 1 + 3 * GF_BLOCK) % T;
        for (int r = 0; r < rounds; r++) {
            a[t] = (long long)r * 1000003ll + t;
            __threadfence();
            if (gf_barrier())
                atomicAdd(err, 1000000ull);
            if (*(volatile long long *)&a[other] != (long long)r * 1000003ll + other)
                atomicAdd(err, 1ull);
            if (gf_barrier())
                atomicAdd(err, 1000000ull);
        }
    });
    return rc ? 10 : 0;
}

/*
 * rpc_probe path_small path_big nbig      buffers: 0 = int64 results[32], 1 = bytes big[nbig]
 * Exercises every landing pad; results[] receives the host return values.
 */
GF_MAIN(rpc_probe)(int argc, char **argv)
{
    if (argc < 4)
        return 2;
    long long *res = (long long *)gf_buffer(0);
    unsigned char *big = (unsigned char *)gf_buffer(1);
    const long long nbig = gf_atoll(argv[3]);
    if (!res || !big)
        return 2;
    int k = 0;
    res[k++] = gf_printf("int %d %i %u %x %X %o|\n", -42, 7, 4000000000u, 255u, 3054u, 8u);
    res[k++] = gf_printf("long %ld %lld %llu %lx\n", -5000000000l, 123456789012345ll, 18446744073709551615ull,
                         0xdeadbeefcafeul);
    res[k++] = gf_printf("dbl %f %e %g %.17g %10.3f|%-8.2e|%+.0f\n", 3.14159, -1.5e-300, 1e100, 0.1, 2.5, 12345.678, 2.5);
    res[k++] = gf_printf("str [%s] [%10s] [%-6s] [%.3s] %c%c %%\n", "hello", "right", "left", "truncate", 'o', 'k');
    res[k++] = gf_printf("star [%*d] [%-*d] [%.*f]\n", 6, 42, 5, 7, 3, 1.0 / 3.0);
    res[k++] = gf_printf("no args\n");
    GF_FILE f = gf_fopen(argv[1], "w");
    res[k++] = f != 0;
    res[k++] = gf_fprintf(f, "to file %d %s\n", 99, "ok");
    const char blob[] = "0123456789abcdef";
    res[k++] = (long long)gf_fwrite(blob, 1, 16, f);
    res[k++] = gf_fclose(f);
    GF_FILE g = gf_fopen(argv[2], "wb");
    res[k++] = (long long)gf_fwrite(big, 1, (size_t)nbig, g);   /* DMA path */
    res[k++] = gf_fclose(g);
    /* read both back: small inline and large DMA */
    char back[64];
    for (int q = 0; q < 64; q++)
        back[q] = 0;
    GF_FILE r = gf_fopen(argv[1], "r");
    res[k++] = (long long)gf_fread(back, 1, 20, r);
    gf_fclose(r);
    long long sum = 0;
    for (int q = 0; q < 20; q++)
        sum = sum * 31 + (unsigned char)back[q];
    res[k++] = sum;
    for (long long q = 0; q < nbig; q++)
        big[q] = 0;
    GF_FILE r2 = gf_fopen(argv[2], "rb");
    res[k++] = (long long)gf_fread(big, 1, (size_t)nbig, r2);
    gf_fclose(r2);
    const char *hv = gf_getenv("GF_PROBE_VAR");
    res[k++] = hv ? (long long)gf_strlen(hv) : -1;
    res[k++] = hv ? (long long)hv[0] : -1;
    res[k++] = gf_getenv("GF_PROBE_UNSET_VAR") ? 1 : 0;
    const long long c0 = gf_clock();
    const long long c1 = gf_clock();
    res[k++] = c1 >= c0 ? 1 : 0;
    res[k++] = gf_fopen("/nonexistent-dir/x", "r") == 0 ? 1 : 0;
    res[k++] = k;
    return 0;
}

/* rpc_storm nthreads calls          every iteration prints `calls` lines "t <i> k <k> v <double>" */
GF_MAIN(rpc_storm)(int argc, char **argv)
{
    if (argc < 3)
        return 2;
    const long long n = gf_atoll(argv[1]);
    const int calls = (int)gf_atoll(argv[2]);
    unsigned long long *bad = (unsigned long long *)gf_buffer(0);
    int rc = gf_parallel_for(0, n, GF_SCHED_STATIC, 1, [=](int64_t i) {
        for (int k = 0; k < calls; k++) {
            const int r = gf_printf("t %lld k %d v %.6e\n", (long long)i, k, (double)i * 0.5 + k);
            if (r <= 0 && bad)
                atomicAdd(bad, 1ull);
        }
    });
    return rc ? 10 : 0;
}

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

/* link_probe bytes reps dir         buffers: 0 = device bytes, 1 = int64 ns[reps]
 * Times `reps` grid-wide copies of `bytes` between device memory and the
 * context's bulk arena (pinned host memory mapped into the device): dir 0 =
 * device stores into host memory (the fwrite path), dir 1 = device loads
 * from host memory (the fread path).  ns[r] = device time of copy r. */
GF_MAIN(link_probe)(int argc, char **argv)
{
    if (argc < 4)
        return 2;
    const uint64_t bytes = (uint64_t)gf_atoll(argv[1]);
    const int reps = (int)gf_atoll(argv[2]), dir = (int)gf_atoll(argv[3]);
    uint8_t *dev = (uint8_t *)gf_buffer(0);
    long long *ns = (long long *)gf_buffer(1);
    uint8_t *host = (uint8_t *)gfd::s_st->bulk_dev;
    if (!dev || !ns || !host || bytes > gfd::s_st->bulk_bytes || gf_buffer_bytes(0) < bytes ||
        gf_buffer_bytes(1) < (uint64_t)reps * 8)
        return 2;
    for (int r = 0; r < reps; r++) {
        const uint64_t t0 = gfd::now_ns();
        const int rc = dir == 0 ? gfd::copy_region(host, dev, bytes) : gfd::copy_region(dev, host, bytes);
        ns[r] = (long long)(gfd::now_ns() - t0);
        if (rc)
            return 10;
    }
    return 0;
}

/* rpc_latency n mode                buffers: 0 = int64 ns[n]
 * One thread makes n RPCs in a row, each timed on the device: mode 0 =
 * clock() (an empty round trip), mode 1 = fprintf(f, "fread reads: %s\n",
 * buffer) with a 128-byte buffer and f = /dev/null -- the call the paper
 * times 1000 times for its RPC cost breakdown (Sec. 5, "RPC Performance"). */
GF_MAIN(rpc_latency)(int argc, char **argv)
{
    if (argc < 3)
        return 2;
    const long long n = gf_atoll(argv[1]);
    const int mode = (int)gf_atoll(argv[2]);
    long long *ns = (long long *)gf_buffer(0);
    if (n < 1 || !ns || gf_buffer_bytes(0) < (uint64_t)n * 8)
        return 2;
    char *buf = (char *)gf_malloc(128);
    if (!buf)
        return 4;
    for (int k = 0; k < 127; k++)
        buf[k] = (char)('a' + k % 26);
    buf[127] = 0;
    GF_FILE f = mode ? gf_fopen("/dev/null", "w") : (GF_FILE)0;
    if (mode && !f)
        return 3;
    for (long long k = 0; k < n; k++) {
        const uint64_t t0 = gfd::now_ns();
        if (mode)
            gf_fprintf(f, "fread reads: %s\n", buf);
        else
            gf_clock();
        ns[k] = (long long)(gfd::now_ns() - t0);
    }
    if (f)
        gf_fclose(f);
    gf_free(buf);
    return 0;
}

/* rpc_timeout                      the host does not serve: the call must come back with GF_ETIMEDOUT */
GF_MAIN(rpc_timeout)(int argc, char **argv)
{
    int st = 0;
    gfd::rpc(GF_OP_CLOCK, nullptr, &st);
    return st == GF_ETIMEDOUT ? 1 : (st == GF_OK ? 0 : 2);
}

/* div6_probe n                     buffers: 0 = double x[n],
 *                                   1 = double out[3n]: (x / 6.0, gf_div6_rn(x), gf_div6_int(x)) */
GF_MAIN(div6_probe)(int argc, char **argv)
{
    const long long n = gf_atoll(argv[1]);
    const double *x = (const double *)gf_buffer(0);
    double *out = (double *)gf_buffer(1);
    return gf_parallel_for(0, n, GF_SCHED_STATIC, 1, [=](int64_t i) {
        const double v = x[i];
        out[3 * i] = v / 6.0;
        out[3 * i + 1] = gf_div6_rn(v);
        out[3 * i + 2] = gf_div6_int(v);
    }) ? 10 : 0;
}

/* dadd_probe n                     buffers: 0 = double x[n], 1 = double y[n],
 *                                   2 = double out[2n]: (x + y on the FP64 pipe, gf_dadd_int(x, y)) */
GF_MAIN(dadd_probe)(int argc, char **argv)
{
    const long long n = gf_atoll(argv[1]);
    const double *x = (const double *)gf_buffer(0);
    const double *y = (const double *)gf_buffer(1);
    double *out = (double *)gf_buffer(2);
    return gf_parallel_for(0, n, GF_SCHED_STATIC, 1, [=](int64_t i) {
        out[2 * i] = __dadd_rn(x[i], y[i]);
        out[2 * i + 1] = gf_dadd_int(x[i], y[i]);
    }) ? 10 : 0;
}

/* fwrite_modes path nbytes          buffer 0 = bytes; appends the buffer twice ("ab": in-order path),
 * then writes it once more at offset 0 of a fresh file ("wb": parallel path) followed by a small tail */
GF_MAIN(fwrite_modes)(int argc, char **argv)
{
    if (argc < 3)
        return 2;
    const unsigned char *b = (const unsigned char *)gf_buffer(0);
    const long long n = gf_atoll(argv[2]);
    GF_FILE f = gf_fopen(argv[1], "ab");
    if (!f)
        return 3;
    long long w = (long long)gf_fwrite(b, 1, (size_t)n, f);
    w += (long long)gf_fwrite(b, 1, (size_t)n, f);
    gf_fclose(f);
    return w == 2 * n ? 0 : 4;
}

/*
 * fig4_probe opcode               buffer 0 = int64 out[8]
 * The call site of the paper's worked example (Fig. 4),
 *     r = fscanf(fd, "%f %i %i", &s.f, s.a ? &i : &s.b, p);
 * issued to a user landing pad: fd by value (an opaque FILE*), the format as a
 * read-only reference, &s.f readwrite with the whole struct at offset
 * offsetof(f), &i write-only (s.a != 0), and p -- an interior pointer no
 * analysis pins down -- looked up in the device heap at run time.
 */
struct fig4_S {
    int a, b;
    float f;
};
GF_MAIN(fig4_probe)(int argc, char **argv)
{
    if (argc < 2)
        return 2;
    const unsigned op = (unsigned)gf_atoll(argv[1]);
    long long *out = (long long *)gf_buffer(0);
    fig4_S s;
    s.a = 1;
    s.b = 2;
    s.f = 0.5f;
    int i = -1;
    int *blk = (int *)gf_malloc(16);
    if (!blk || !out)
        return 3;
    blk[0] = 10;
    blk[1] = 11;
    blk[2] = 12;
    blk[3] = 13;
    int *p = blk + 1;
    const char *fmt = "%f %i %i";
    const unsigned long long fd = 0xF11E0ull;
    int st = 0;
    long long r;
    if (s.a)
        r = gf_rpc(op, &st, fd, gf_ref_read(fmt, 9, 0), gf_ref_readwrite(&s, sizeof(fig4_S), offsetof(fig4_S, f)),
                   gf_ref_write(&i, sizeof(int), 0), gf_ref_lookup(p));
    else
        r = gf_rpc(op, &st, fd, gf_ref_read(fmt, 9, 0), gf_ref_readwrite(&s, sizeof(fig4_S), offsetof(fig4_S, f)),
                   gf_ref_readwrite(&s, sizeof(fig4_S), offsetof(fig4_S, b)), gf_ref_lookup(p));
    out[0] = r;
    out[1] = st;
    out[2] = __float_as_int(s.f);
    out[3] = s.a;
    out[4] = s.b;
    out[5] = i;
    out[6] = blk[1];
    out[7] = blk[0] + 100 * blk[2] + 10000 * blk[3];
    gf_free(blk);
    return 0;
}
