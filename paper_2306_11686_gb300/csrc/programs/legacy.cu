/*
 * Legacy-style programs run whole on the GPU (paper Sec. 1: the CPU program
 * is not restructured; its serial part runs on one thread, its parallel loops
 * on the whole device, its libc calls through RPC or the device libc).
 *
 * Each is the device twin of a serial C program; the same computation in
 * plain C with the real libc is what a run must reproduce.
 */
#include "../gf_device.cuh"
#include "../gf_fastdiv.cuh"
#include "../gf_intpipe.cuh"

/*
 * axpy_sum N out_path            buffers: 0 = x (N doubles), 1 = y (N doubles, updated)
 *
 *   y[i] = 2.5*x[i] + y[i] over [0, N), printf("%d %.17g\n", i, y[i]) when i % 1024 == 0;
 *   s = sum of y (worksharing reduction), printf("sum %.17g\n", s);
 *   fopen / fwrite(y) / fclose.
 */
GF_MAIN(axpy_sum)(int argc, char **argv)
{
    if (argc < 3)
        return 2;
    const long long n = gf_atoll(argv[1]);
    const double *x = (const double *)gf_buffer(0);
    double *y = (double *)gf_buffer(1);
    if (n < 0 || (n > 0 && (!x || !y)) || gf_buffer_bytes(0) < (uint64_t)n * 8 ||
        gf_buffer_bytes(1) < (uint64_t)n * 8)
        return 2;
    int rc = gf_parallel_for(0, n, GF_SCHED_STATIC, 1, [=](int64_t i) {
        const double v = 2.5 * x[i] + y[i];
        y[i] = v;
        if (i % 1024 == 0)
            gf_printf("%d %.17g\n", (int)i, v);
    });
    if (rc)
        return 10;
    double s = 0.0;
    rc = gf_reduce<double, GF_RED_SUM>(0, n, GF_SCHED_STATIC, 1, [=](int64_t i) { return y[i]; }, &s);
    if (rc)
        return 11;
    gf_printf("sum %.17g\n", s);
    GF_FILE f = gf_fopen(argv[2], "wb");
    if (!f)
        return 3;
    if (gf_fwrite(y, sizeof(double), (size_t)n, f) != (size_t)n)
        return 3;
    gf_fclose(f);
    return 0;
}

/*
 * One Jacobi sweep: the six-neighbour average of the interior into un, 0 on
 * the boundary, and the max residual |un - u| over the grid as a max
 * reduction.  The five neighbour adds keep the serial program's order; the
 * first INT_ADDS of them run on the integer pipe and the rest on the FP64
 * pipe (every one correctly rounded, so the split changes no bit of the
 * result, only which pipe does the work), as do the division by 6 and the
 * absolute value.  The flat index is split into (i, j, k) by multiplication
 * with an invariant-divisor magic number.
 */
template <int INT_ADDS>
__device__ int jacobi_sweep(const double *u, double *un, uint32_t nn, gf_udiv32 dn, uint64_t cells, double *res)
{
    const uint32_t sk = nn * nn;
    return gf_reduce<double, GF_RED_MAX>(
        0, (int64_t)cells, GF_SCHED_STATIC, 1,
        [=](int64_t c64) -> double {
            const uint32_t c = (uint32_t)c64;
            /* i - 1, j - 1, k - 1 wrap to 2^32 - 1 at 0, so one unsigned
             * compare of their maximum finds every boundary cell */
            const uint32_t jk = dn.div(c), im1 = c - 1u - jk * nn;
            const uint32_t k = dn.div(jk), jm1 = jk - 1u - k * nn;
            if (max(im1, max(jm1, k - 1u)) >= nn - 2u) {
                un[c] = 0.0;
                return 0.0;
            }
            /* u is not written during the sweep: read-only loads, which may be
             * issued ahead of the previous iteration's store to un */
            const double nb[6] = {__ldg(u + c - 1),  __ldg(u + c + 1),  __ldg(u + c - nn),
                                  __ldg(u + c + nn), __ldg(u + c - sk), __ldg(u + c + sk)};
            double v = nb[0];
#pragma unroll
            for (int t = 1; t < 6; t++)
                v = t <= INT_ADDS ? gf_dadd_int(v, nb[t]) : __dadd_rn(v, nb[t]);
            v = gf_div6_int(v);               /* == v / 6.0, bit for bit */
            un[c] = v;
            return gf_fabs_int(__dadd_rn(v, -__ldg(u + c)));
        },
        res);
}

/*
 * The same sweep written with the k loop inside the parallel loop: work item
 * t is the column (i, j) over planes [k0, k0 + kseg), t = (k0 / kseg) * n^2 +
 * j * n + i, so consecutive items are consecutive i (coalesced).  Walking up
 * the column, the k - 1 and k neighbours of a point are the values loaded for
 * the previous point, so each point loads five values instead of seven, and
 * the index split and boundary test are paid once per column segment.  Every
 * point's arithmetic and its order are those of jacobi_sweep, so the grid
 * and the residual are the same bits.
 */
template <int INT_ADDS>
__device__ int jacobi_sweep_col(const double *u, double *un, uint32_t nn, gf_udiv32 dn, gf_udiv32 dsk, uint32_t kseg,
                                double *res)
{
    const uint32_t sk = nn * nn;
    const uint32_t nseg = (nn + kseg - 1) / kseg;
    return gf_reduce<double, GF_RED_MAX>(
        0, (int64_t)nseg * sk, GF_SCHED_STATIC, 1,
        [=](int64_t t64) -> double {
            const uint32_t t = (uint32_t)t64;
            const uint32_t seg = dsk.div(t), ij = t - seg * sk;
            const uint32_t j = dn.div(ij), im1 = ij - 1u - j * nn;
            const uint32_t k0 = seg * kseg, k1 = min(k0 + kseg, nn);
            double *o = un + ij;
            if (max(im1, j - 1u) >= nn - 2u) {            /* a boundary column */
                for (uint32_t k = k0; k < k1; k++)
                    o[(size_t)k * sk] = 0.0;
                return 0.0;
            }
            const double *c = u + ij;
            uint32_t k = k0;
            if (k == 0) {                                  /* the bottom boundary plane */
                o[0] = 0.0;
                k = 1;
            }
            const uint32_t kend = min(k1, nn - 1u);
            long long best = 0;                            /* bits of the largest |un - u|, +0 to start */
            if (k < kend) {
                double um = __ldg(c + (size_t)(k - 1) * sk), u0 = __ldg(c + (size_t)k * sk);
                for (; k < kend; k++) {
                    const double *p = c + (size_t)k * sk;
                    const double up = __ldg(p + sk);
                    const double nb[6] = {__ldg(p - 1), __ldg(p + 1), __ldg(p - nn), __ldg(p + nn), um, up};
                    double v = nb[0];
#pragma unroll
                    for (int q = 1; q < 6; q++)
                        v = q <= INT_ADDS ? gf_dadd_int(v, nb[q]) : __dadd_rn(v, nb[q]);
                    v = gf_div6_int(v);
                    o[(size_t)k * sk] = v;
                    /* |un - u| >= 0: its bits order as the values do; NaN is skipped, as the reduction does */
                    const long long b = __double_as_longlong(gf_fabs_int(__dadd_rn(v, -u0)));
                    if (b <= 0x7ff0000000000000ll && b > best)
                        best = b;
                    um = u0;
                    u0 = up;
                }
            }
            if (k1 == nn && nn > 1)                        /* the top boundary plane */
                o[(size_t)(nn - 1) * sk] = 0.0;
            return __longlong_as_double(best);
        },
        res);
}

/*
 * jacobi n sweeps out_path [int_adds [kseg]]   buffers: 0 = input grid (n^3 doubles, i fastest)
 *
 * Laplace Jacobi sweeps with the six-neighbour average, boundary written as 0,
 * a fresh grid from the device heap every sweep (old one freed after the
 * swap), the max residual over the interior fused into the sweep as a max
 * reduction, one printf per sweep, the final grid fwrite'd.  int_adds (0..5,
 * default 1) is how many of the five neighbour adds run on the integer pipe;
 * kseg (default 0) > 0 runs the sweep as columns of kseg planes
 * (jacobi_sweep_col) instead of one parallel iteration per point.
 * Compiled for 4 resident blocks per SM (64 registers): the sweep waits on
 * L2 more than on any pipe, and more warps hide that latency.
 */
GF_MAIN_BOUNDS(jacobi, 4)(int argc, char **argv)
{
    if (argc < 4)
        return 2;
    const long long n = gf_atoll(argv[1]);
    const int sweeps = (int)gf_atoll(argv[2]);
    const int int_adds = argc > 4 ? (int)gf_atoll(argv[4]) : 1;
    const long long kseg = argc > 5 ? gf_atoll(argv[5]) : 0;
    const double *u0 = (const double *)gf_buffer(0);
    const uint64_t cells = (uint64_t)n * n * n;
    if (n < 1 || n > 1290 || !u0 || gf_buffer_bytes(0) < cells * 8 || int_adds < 0 || int_adds > 5 || kseg < 0 ||
        kseg > n)
        return 2;
    const uint32_t nn = (uint32_t)n;
    const double *u = u0;
    double *owned = nullptr;
    /* the index split's magic numbers: loop invariants, made once */
    const gf_udiv32 dn = gf_udiv32::make(nn), dsk = gf_udiv32::make(nn * nn);
    for (int s = 1; s <= sweeps; s++) {
        double *un = (double *)gf_malloc(cells * sizeof(double));
        if (!un) {
            gf_printf("jacobi: out of device heap at sweep %d\n", s);
            return 4;
        }
        double res = 0.0;
        int rc;
        if (kseg > 0) {
            const uint32_t ks = (uint32_t)kseg;
            switch (int_adds) {
            case 0: rc = jacobi_sweep_col<0>(u, un, nn, dn, dsk, ks, &res); break;
            case 1: rc = jacobi_sweep_col<1>(u, un, nn, dn, dsk, ks, &res); break;
            case 2: rc = jacobi_sweep_col<2>(u, un, nn, dn, dsk, ks, &res); break;
            case 3: rc = jacobi_sweep_col<3>(u, un, nn, dn, dsk, ks, &res); break;
            case 4: rc = jacobi_sweep_col<4>(u, un, nn, dn, dsk, ks, &res); break;
            default: rc = jacobi_sweep_col<5>(u, un, nn, dn, dsk, ks, &res); break;
            }
        } else {
            switch (int_adds) {
            case 0: rc = jacobi_sweep<0>(u, un, nn, dn, cells, &res); break;
            case 1: rc = jacobi_sweep<1>(u, un, nn, dn, cells, &res); break;
            case 2: rc = jacobi_sweep<2>(u, un, nn, dn, cells, &res); break;
            case 3: rc = jacobi_sweep<3>(u, un, nn, dn, cells, &res); break;
            case 4: rc = jacobi_sweep<4>(u, un, nn, dn, cells, &res); break;
            default: rc = jacobi_sweep<5>(u, un, nn, dn, cells, &res); break;
            }
        }
        if (rc)
            return 10;
        gf_printf("%d %.17g\n", s, res);
        if (owned)
            gf_free(owned);
        owned = un;
        u = un;
    }
    if (argv[3][0] == '-' && argv[3][1] == 0) {      /* "-": keep the grid, write nothing (profiling) */
        if (owned)
            gf_free(owned);
        return 0;
    }
    GF_FILE f = gf_fopen(argv[3], "wb");
    if (!f)
        return 3;
    const size_t w = gf_fwrite(u, sizeof(double), (size_t)cells, f);
    gf_fclose(f);
    if (owned)
        gf_free(owned);
    return w == cells ? 0 : 3;
}
