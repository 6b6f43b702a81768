/*
 * Small programs that expose one runtime mechanism each, for the GPU tests:
 * the integer-pipe FP64 helpers, fwrite modes and the paper's Fig. 4 call site.
 */
#include "../gf_device.cuh"
#include "../gf_fastdiv.cuh"
#include "../gf_intpipe.cuh"

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
 * fig4_probe opcode [array]       buffer 0 = int64 out[8]
 * The call site of the paper's worked example (Fig. 4),
 *     r = fscanf(fd, "%f %i %i", &s.f, s.a ? &i : &s.b, p);
 * issued to a user landing pad: fd by value (an opaque FILE*), the format as a
 * read-only reference, &s.f readwrite with the whole struct at offset
 * offsetof(f), &i write-only (s.a != 0), and p -- an interior pointer no
 * analysis pins down -- looked up in the device heap at run time.
 * With "array" the same call goes through the array form of gf_rpc, the
 * arguments described one by one in gf_arg records.
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
    if (argc > 2 && argv[2][0] == 'a') {
        gf_arg args[5];
        memset(args, 0, sizeof args);
        args[0].tag = GF_T_U64;                       /* the FILE*, by value (as its 64 bits) */
        args[0].word = fd;
        args[1].tag = GF_T_BLOB_R;                    /* the format, read only */
        args[1].ptr = fmt;
        args[1].bytes = 9;
        args[2].tag = GF_T_BLOB_RW;                   /* &s.f: the whole struct, readwrite */
        args[2].ptr = &s;
        args[2].bytes = sizeof(fig4_S);
        args[2].off = offsetof(fig4_S, f);
        if (s.a) {                                    /* &i: write only */
            args[3].tag = GF_T_BLOB_W;
            args[3].ptr = &i;
            args[3].bytes = sizeof(int);
        } else {
            args[3].tag = GF_T_BLOB_RW;
            args[3].ptr = &s;
            args[3].bytes = sizeof(fig4_S);
            args[3].off = offsetof(fig4_S, b);
        }
        uint64_t base = 0, size = 0;                  /* p: its object found at run time */
        if (gf_find_obj(p, &base, &size)) {
            args[4].tag = GF_T_BLOB_RW;
            args[4].ptr = (const void *)base;
            args[4].bytes = (uint32_t)size;
            args[4].off = (uint32_t)((uint64_t)p - base);
        } else {
            args[4].tag = GF_T_PTR;
            args[4].word = (uint64_t)p;
        }
        int64_t r64 = 0;
        st = gf_rpc(op, args, 5, &r64);
        r = r64;
    } else if (s.a)
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

/* axpy_width w          buffers: 0 = n (int64), 1 = x, 2 = y, 3 = z (n doubles each)
 * z = 2.5 x + y as one static chunk-1 region with w = 1 (8-byte accesses)
 * or w = 2 (16-byte double2 accesses from an even index, scalar tail): the
 * same loop with the access width as the only difference.  axpy_width is
 * compiled with the register count left to the compiler, axpy_width4 and
 * axpy_width8 for 4 and 8 resident blocks per SM (64 and 32 registers). */
static __device__ int axpy_width_main(int argc, char **argv)
{
    if (argc < 2)
        return 2;
    const int w = (int)gf_atoll(argv[1]);
    const long long *np = (const long long *)gf_buffer(0);
    if (!np || *np < 0)
        return 2;
    const long long n = *np;
    if (n == 0)
        return 0;
    const double *x = (const double *)gf_buffer(1), *y = (const double *)gf_buffer(2);
    double *z = (double *)gf_buffer(3);
    if (!x || !y || !z || gf_buffer_bytes(1) < (uint64_t)n * 8 || gf_buffer_bytes(2) < (uint64_t)n * 8 ||
        gf_buffer_bytes(3) < (uint64_t)n * 8)
        return 2;
    if (w == 1)
        return gf_parallel_for(0, n, GF_SCHED_STATIC, 1, [=](int64_t i) { z[i] = 2.5 * x[i] + y[i]; }) ? 10 : 0;
    if (((uintptr_t)x | (uintptr_t)y | (uintptr_t)z) & 15)
        return 2;
    const double2 *x2 = (const double2 *)x, *y2 = (const double2 *)y;
    double2 *z2 = (double2 *)z;
    if (gf_parallel_for(0, n / 2, GF_SCHED_STATIC, 1, [=](int64_t i) {
            const double2 a = x2[i], b = y2[i];
            z2[i] = make_double2(2.5 * a.x + b.x, 2.5 * a.y + b.y);
        }))
        return 10;
    if (n & 1)
        z[n - 1] = 2.5 * x[n - 1] + y[n - 1];
    return 0;
}
GF_MAIN_BOUNDS(axpy_width, 1)(int argc, char **argv) { return axpy_width_main(argc, argv); }
GF_MAIN_BOUNDS(axpy_width4, 4)(int argc, char **argv) { return axpy_width_main(argc, argv); }
GF_MAIN_BOUNDS(axpy_width8, 8)(int argc, char **argv) { return axpy_width_main(argc, argv); }
