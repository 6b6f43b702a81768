/*
 * Small programs that expose one runtime mechanism each, for the GPU tests:
 * schedules, reductions, static chunk-1 ranges and the cross-block barrier.
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
