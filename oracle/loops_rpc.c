/*
 * ORACLE (test infrastructure only).  Only tests/, __graft_entry__.smoke() and
 * bench.py's cpu_baseline leg may build, call or run anything under oracle/.
 *
 * Many independent legacy loops whose bodies also call libc: serial, in order,
 * with the real printf, malloc and free (the paper runs such calls by RPC and
 * from a device heap inside parallel regions, Sec. 3.2 and 3.4):
 *
 *   for k in 0..n-1:
 *     for i in 0..trip_k-1:
 *       v = a_k * x[off_k + i] + y[off_k + i]          (two roundings)
 *       if i % 4096 == 0:
 *         w = malloc(64 << (k % 8))                     (64 B .. 8 KiB)
 *         w[0] = v; w[last] = -v; v = w[0]; free(w)     (the value passes through the block)
 *         printf("%d %lld %.17g\n", k, i, v)
 *       z[off_k + i] = v
 *
 * Elements of z outside every loop keep the value read from z_in.
 *
 *   loops_rpc n trips.bin a.bin off.bin x.bin y.bin z_in.bin z_out.bin total
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

static void *load(const char *p, size_t bytes)
{
    void *m = malloc(bytes ? bytes : 1);
    FILE *f = fopen(p, "rb");
    if (!m || !f || fread(m, 1, bytes, f) != bytes) {
        fprintf(stderr, "loops_rpc: cannot read %s\n", p);
        exit(2);
    }
    fclose(f);
    return m;
}

int main(int argc, char **argv)
{
    if (argc != 10) {
        fprintf(stderr, "usage: loops_rpc n trips.bin a.bin off.bin x.bin y.bin z_in.bin z_out.bin total\n");
        return 2;
    }
    const int n = atoi(argv[1]);
    const long total = atol(argv[9]);
    int64_t *trips = load(argv[2], (size_t)n * 8);
    double *a = load(argv[3], (size_t)n * 8);
    int64_t *off = load(argv[4], (size_t)n * 8);
    double *x = load(argv[5], (size_t)total * 8);
    double *y = load(argv[6], (size_t)total * 8);
    double *z = load(argv[7], (size_t)total * 8);
    for (int k = 0; k < n; k++)
        for (int64_t i = 0; i < trips[k]; i++) {
            double v = a[k] * x[off[k] + i] + y[off[k] + i];
            if (i % 4096 == 0) {
                const size_t words = ((size_t)64 << (k % 8)) / 8;
                double *w = malloc(words * 8);
                if (!w)
                    return 4;
                w[0] = v;
                w[words - 1] = -v;
                v = w[0];
                free(w);
                printf("%d %lld %.17g\n", k, (long long)i, v);
            }
            z[off[k] + i] = v;
        }
    FILE *f = fopen(argv[8], "wb");
    if (!f || fwrite(z, 8, (size_t)total, f) != (size_t)total)
        return 3;
    fclose(f);
    return 0;
}
