/*
 * The served legacy program: R passes of a CSR SpMV y = A x (then x = y)
 * whose row iterations issue libc requests at seeded positions -- fwrite of
 * self-describing records (16-byte header + payload from the device heap),
 * printf, clock, getenv.  Many instances run at once under the serving loop
 * (continuous batching: each takes a free program instance -- its ring
 * segment and heap arena -- and others are admitted as instances free up).
 *
 *   spmv_serve prog R n out_path
 *   buffers: 0 = int64 rowptr[n+1], 1 = int32 col[nnz], 2 = double val[nnz],
 *            3 = double x[n] (in: x0, out: the last y), 4 = double y[n] (scratch),
 *            5 = int64 req[2 nreq] {pass << 32 | row, kind | size << 8} sorted,
 *            6 = int64 results[nreq]
 */
#include "../gf_device.cuh"

static __device__ __forceinline__ uint64_t serve_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;   /* SplitMix64 finaliser */
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* one row's sum, y_i = sum of val_j x[col_j] in CSR order, one rounding
 * each, as in the serial program; values and columns read two at a time
 * (16-byte and 8-byte loads from an even index), the gathers of eight
 * nonzeros in flight together.  The matrix is constant for the whole
 * program (read-only loads); x was written by the previous pass, so it
 * takes ordinary loads. */
static __device__ __forceinline__ double spmv_row(const long long *rowptr, const int *col, const double *val,
                                                  const double *xs, bool vec, long long i)
{
    double s = 0.0;
    const long long j0 = __ldg(rowptr + i), j1 = __ldg(rowptr + i + 1);
    long long j = j0;
    if (vec) {
        if ((j & 1) && j < j1) {
            s = s + __ldg(val + j) * xs[__ldg(col + j)];
            j++;
        }
#pragma unroll 4
        for (; j + 1 < j1; j += 2) {
            const double2 v = __ldg((const double2 *)(val + j));
            const int2 c = __ldg((const int2 *)(col + j));
            const double x0 = xs[c.x], x1 = xs[c.y];
            s = s + v.x * x0;
            s = s + v.y * x1;
        }
    }
#pragma unroll 8
    for (; j < j1; j++)
        s = s + __ldg(val + j) * xs[__ldg(col + j)];
    return s;
}

/* the libc requests of row i in pass rr (all of them after its sum, as in
 * the serial program) */
static __device__ __noinline__ void serve_requests(const long long *req, long long *res, const unsigned *mark,
                                                   long long qa, long long qb, unsigned prog, int rr, long long i,
                                                   double s, GF_FILE f)
{
    if (!((mark[i >> 5] >> (i & 31)) & 1u))
        return;
    const long long key = ((long long)rr << 32) | (long long)i;
    long long lo = qa, hi = qb;                 /* first request with key >= (pass, row) */
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if (req[2 * mid] < key)
            lo = mid + 1;
        else
            hi = mid;
    }
    for (long long q = lo; q < qb && req[2 * q] == key; q++) {
        const int kind = (int)(req[2 * q + 1] & 0xff);
        const unsigned size = (unsigned)(req[2 * q + 1] >> 8);
        if (kind == 0) {
            const unsigned long long words = (size + 7) / 8;
            unsigned long long *b = (unsigned long long *)gf_malloc(16 + 8 * words);
            if (!b) {
                res[q] = -2;
                continue;
            }
            b[0] = (unsigned long long)prog | ((unsigned long long)rr << 32);
            b[1] = (unsigned long long)i | ((unsigned long long)size << 32);
            const uint64_t k0 = serve_mix(((uint64_t)prog << 40) ^ ((uint64_t)rr << 32) ^ (uint64_t)i);
            for (unsigned long long w = 0; w < words; w++)
                b[2 + w] = serve_mix(k0 + w * 0x9E3779B97F4A7C15ull);
            res[q] = (long long)gf_fwrite(b, 1, 16 + (size_t)size, f);
            gf_free(b);
        } else if (kind == 1) {
            res[q] = gf_printf("p %d r %d row %d y %.17g\n", (int)prog, rr, (int)i, s);
        } else if (kind == 2) {
            res[q] = gf_clock();
        } else {
            char name[16] = "GF_SERVE_VAR0";
            name[12] = (char)('0' + (int)(i % 3));
            const char *v = gf_getenv(name);
            res[q] = v ? (long long)gf_strlen(v) : -1;
        }
    }
}

/* compiled for 4 resident blocks per SM (64 registers): each of the
 * concurrent instances gets a quarter of the co-resident blocks' worth of
 * warps more for its latency-bound gathers (measured: 77.0 k vs 72.8 k
 * served calls/s, admission-to-done p50 0.25 s vs 0.28 s at 1 block per SM) */
GF_MAIN_BOUNDS(spmv_serve, 4)(int argc, char **argv)
{
    if (argc < 5)
        return 2;
    const unsigned prog = (unsigned)gf_atoll(argv[1]);
    const int R = (int)gf_atoll(argv[2]);
    const long long n = gf_atoll(argv[3]);
    const long long *rowptr = (const long long *)gf_buffer(0);
    const int *col = (const int *)gf_buffer(1);
    const double *val = (const double *)gf_buffer(2);
    double *xb = (double *)gf_buffer(3);
    double *yb = (double *)gf_buffer(4);
    const long long *req = (const long long *)gf_buffer(5);
    long long *res = (long long *)gf_buffer(6);
    const long long nreq = (long long)(gf_buffer_bytes(5) / 16);
    if (!rowptr || !col || !val || !xb || !yb || (nreq && (!req || !res)))
        return 2;
    GF_FILE f = gf_fopen(argv[4], "wb");
    if (!f)
        return 3;
    /* one bit per row: set for the rows that issue a request in this pass, so
     * a row without one skips the request search with a single load */
    const long long nw = (n + 31) / 32;
    unsigned *mark = (unsigned *)gf_malloc((size_t)(nw > 0 ? nw : 1) * 4);
    if (!mark)
        return 4;
    if (gf_parallel_for(0, nw, GF_SCHED_STATIC, 1, [=](int64_t w) { mark[w] = 0u; }))
        return 10;
    double *x = xb, *y = yb;
    long long q0 = 0;
    /* paired loads need 16-byte aligned values and 8-byte aligned columns */
    const bool vec = ((uintptr_t)val & 15u) == 0 && ((uintptr_t)col & 7u) == 0;
    for (int r = 0; r < R; r++) {
        long long q1 = q0;
        while (q1 < nreq && (req[2 * q1] >> 32) == r)
            q1++;
        const long long qa = q0, qb = q1;
        const int rr = r;
        const double *xs = x;
        double *ys = y;
        if (qb > qa && gf_parallel_for(qa, qb, GF_SCHED_STATIC, 1, [=](int64_t q) {
                const unsigned row = (unsigned)(req[2 * q] & 0xffffffffll);
                atomicOr(&mark[row >> 5], 1u << (row & 31));
            }))
            return 10;
        /* the row loop keeps only the sum; the requests (malloc, record
         * generation, RPC) live out of line, so their code and registers
         * stay out of the loop over the nonzeros */
        const int rc = gf_parallel_for(0, n, GF_SCHED_STATIC, 1, [=](int64_t i) {
            const double s = spmv_row(rowptr, col, val, xs, vec, i);
            ys[i] = s;
            if (qa == qb)
                return;
            serve_requests(req, res, mark, qa, qb, prog, rr, i, s, f);
        });
        if (rc)
            return 10;
        if (qb > qa && gf_parallel_for(qa, qb, GF_SCHED_STATIC, 1, [=](int64_t q) {
                mark[(unsigned)(req[2 * q] & 0xffffffffll) >> 5] = 0u;   /* clear for the next pass */
            }))
            return 10;
        q0 = q1;
        double *t = x;
        x = y;
        y = t;
    }
    if (x != xb) {                                       /* the last y lives in the scratch buffer */
        const double *src = x;
        if (gf_parallel_for(0, n, GF_SCHED_STATIC, 1, [=](int64_t i) { xb[i] = src[i]; }))
            return 10;
    }
    gf_fclose(f);
    gf_free(mark);
    return 0;
}
