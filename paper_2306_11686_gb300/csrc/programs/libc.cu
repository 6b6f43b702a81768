/*
 * Programs for the native device libc additions (rand, realloc, strtod) and
 * the paper's interleaved-layout experiment (HeCBench "interleaved", Sec.
 * 5.3: the same loop over an array of structs vs a struct of arrays).
 */
#include "../gf_device.cuh"
#include "../gf_device_libc.cuh"

/* libc_probe seed nrand nstr
 * buffers: 0 = int32 rnd[nrand], 1 = char strs[], 2 = int64 str_off[nstr],
 *          3 = double val[nstr], 4 = int64 used[nstr], 5 = int64 rea[8] */
GF_MAIN(libc_probe)(int argc, char **argv)
{
    if (argc < 4)
        return 2;
    const unsigned seed = (unsigned)gf_atoll(argv[1]);
    const int nrand = (int)gf_atoll(argv[2]);
    const long long nstr = gf_atoll(argv[3]);
    int *rnd = (int *)gf_buffer(0);
    const char *strs = (const char *)gf_buffer(1);
    const long long *soff = (const long long *)gf_buffer(2);
    double *val = (double *)gf_buffer(3);
    long long *used = (long long *)gf_buffer(4);
    long long *rea = (long long *)gf_buffer(5);
    if (!rnd || !rea)
        return 2;
    gf_srand(seed);
    for (int k = 0; k < nrand; k++)
        rnd[k] = gf_rand();
    /* strtod from every thread of a region (fast path native, the rest by RPC) */
    if (nstr > 0 && gf_parallel_for(0, nstr, GF_SCHED_STATIC, 1, [=](int64_t k) {
            char *end = nullptr;
            const char *s = strs + soff[k];
            val[k] = gf_strtod(s, &end);
            used[k] = end - s;
        }))
        return 10;
    /* realloc: in place inside a block, moved across classes, NULL and 0 cases */
    unsigned char *p = (unsigned char *)gf_malloc(24);
    for (int k = 0; k < 24; k++)
        p[k] = (unsigned char)(k + 1);
    unsigned char *q = (unsigned char *)gf_realloc(p, 30);       /* 32-byte class: stays */
    rea[0] = q == p;
    unsigned char *r = (unsigned char *)gf_realloc(q, 1000);     /* moves, keeps the bytes */
    long long same = 1;
    for (int k = 0; k < 24; k++)
        same &= r[k] == (unsigned char)(k + 1);
    rea[1] = r != q;
    rea[2] = same;
    unsigned char *s = (unsigned char *)gf_realloc(nullptr, 10);
    rea[3] = s != nullptr;
    rea[4] = gf_realloc(s, 0) == nullptr;
    unsigned char *big = (unsigned char *)gf_realloc(r, 200000);  /* into the large path */
    same = 1;
    for (int k = 0; k < 24; k++)
        same &= big[k] == (unsigned char)(k + 1);
    rea[5] = same;
    gf_free(big);
    return 0;
}

/* interleave layout n             buffers: 0 = double aos[4n] {a,b,c,d}, 1..4 = double a[n], b[n], c[n], d[n],
 *                                 5 = double out[n]; layout 0 = array of structs, 1 = struct of arrays */
GF_MAIN(interleave)(int argc, char **argv)
{
    if (argc < 3)
        return 2;
    const int layout = (int)gf_atoll(argv[1]);
    const long long n = gf_atoll(argv[2]);
    const double *aos = (const double *)gf_buffer(0);
    const double *a = (const double *)gf_buffer(1), *b = (const double *)gf_buffer(2);
    const double *c = (const double *)gf_buffer(3), *d = (const double *)gf_buffer(4);
    double *out = (double *)gf_buffer(5);
    if (!out)
        return 2;
    if (layout == 0)
        return gf_parallel_for(0, n, GF_SCHED_STATIC, 1, [=](int64_t i) {
                   const double *s = aos + 4 * i;
                   out[i] = s[0] + s[1] * s[2] - s[3];
               }) ? 10 : 0;
    return gf_parallel_for(0, n, GF_SCHED_STATIC, 1, [=](int64_t i) { out[i] = a[i] + b[i] * c[i] - d[i]; }) ? 10
                                                                                                                : 0;
}
