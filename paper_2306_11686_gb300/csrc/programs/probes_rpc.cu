/*
 * Small programs that expose one runtime mechanism each, for the GPU tests:
 * RPC landing pads, call storms, the host link, round-trip latency and the
 * bounded-wait error path.
 */
#include "../gf_device.cuh"
#include "../gf_fastdiv.cuh"
#include "../gf_intpipe.cuh"

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

/* rpc_diverge n                      buffers: 0 = int32 returns[n]
 * Odd and even iterations print from two different call sites with one
 * format, so the lanes of a warp reach the call as two separate groups (the
 * shared-slot path lets the second join the first's slot). */
__device__ const char rpc_diverge_fmt[] = "d %lld %d\n";
GF_MAIN(rpc_diverge)(int argc, char **argv)
{
    if (argc < 2)
        return 2;
    const long long n = gf_atoll(argv[1]);
    int *ret = (int *)gf_buffer(0);
    if (!ret || gf_buffer_bytes(0) < (uint64_t)n * 4)
        return 2;
    return gf_parallel_for(0, n, GF_SCHED_STATIC, 1, [=](int64_t i) {
        int r;
        if (i & 1)
            r = gf_printf(rpc_diverge_fmt, (long long)i, 1);
        else
            r = gf_printf(rpc_diverge_fmt, (long long)i, 0);
        ret[i] = r;
    }) ? 10 : 0;
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
        if (mode) {
            const int r = gf_fprintf(f, "fread reads: %s\n", buf);   /* reading the result: a full round trip */
            (void)r;
        } else
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

/*
 * main_printf_batch [path]   buffers: 0 = int64 results[8]
 * The initial thread's buffered printf: 100 lines of one format (three full
 * batches and a partial one), a line of another format with a string, a
 * result read in its own statement, a non-printf call (clock) in between, a
 * record too large for the buffer, 40 lines of a third format, a result
 * read only after a later call (-1 by contract), 50 buffered fprintf lines
 * to a file closed right after them (path given), then main returns with
 * records still buffered.  Every line must appear once, in program order.
 */
GF_MAIN(main_printf_batch)(int argc, char **argv)
{
    long long *res = (long long *)gf_buffer(0);
    if (!res)
        return 2;
    for (int k = 0; k < 100; k++)
        gf_printf("a %d\n", k);
    gf_printf("b %s %d\n", "str", -1);
    res[0] = (int)gf_printf("c %d\n", 7);               /* read at once: 4 */
    res[1] = gf_clock() >= 0 ? 1 : 0;
    char big[1400];
    for (int k = 0; k < 1399; k++)
        big[k] = (char)('a' + k % 26);
    big[1399] = 0;
    res[2] = (int)gf_printf("big %s\n", big);            /* larger than the buffer: 1404 */
    gf_call_result late = gf_printf("d %d %.17g\n", 0, 0.5);
    for (int k = 1; k < 40; k++)
        gf_printf("d %d %.17g\n", k, k * 0.25);
    res[3] = gf_clock() >= 0 ? 1 : 0;
    res[4] = (int)late;                                   /* its batch already went: -1 */
    if (argc > 1) {                                       /* buffered fprintf, then fclose at once */
        GF_FILE f = gf_fopen(argv[1], "w");
        if (!f)
            return 3;
        for (int k = 0; k < 50; k++)
            gf_fprintf(f, "f %d %s\n", k, "x");
        res[5] = gf_fclose(f);
    }
    gf_printf("e %d\n", 1);
    gf_printf("e %d\n", 2);                              /* left buffered when main returns */
    return 0;
}
