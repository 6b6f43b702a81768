/*
 * ORACLE (test infrastructure only).  Only tests/, __graft_entry__.smoke() and
 * bench.py's cpu_baseline leg may build, call or run anything under oracle/.
 *
 * The plain legacy program, run serially on the host with the real libc.  GPU
 * First executes an unmodified CPU program faithfully on the GPU (Sec. 1 and
 * Sec. 3.1, Fig. 1), so the expected result of the GPU run is simply what this
 * serial program prints and writes.
 *
 *   axpy_sum N x.bin y.bin out.bin
 *
 * 1. y[i] = 2.5*x[i] + y[i] for i in [0, N), printing "%d %.17g\n" (i, y[i])
 *    for every i with i % 1024 == 0 (one line per 1024 iterations);
 * 2. s = sum of y[i] in index order, printed as "sum %.17g\n";
 * 3. y written with fopen/fwrite/fclose to out.bin.
 * Build with -ffp-contract=off: the multiply and the add round separately.
 */
#include <stdio.h>
#include <stdlib.h>

static double *read_f64(const char *path, long n)
{
    double *a = malloc((size_t)n * sizeof(double));
    FILE *f = fopen(path, "rb");
    if (!a || !f || fread(a, sizeof(double), (size_t)n, f) != (size_t)n) {
        fprintf(stderr, "axpy_sum: cannot read %s\n", path);
        exit(2);
    }
    fclose(f);
    return a;
}

int main(int argc, char **argv)
{
    if (argc != 5) {
        fprintf(stderr, "usage: axpy_sum N x.bin y.bin out.bin\n");
        return 2;
    }
    long n = atol(argv[1]);
    double *x = read_f64(argv[2], n);
    double *y = read_f64(argv[3], n);

    for (long i = 0; i < n; i++) {
        y[i] = 2.5 * x[i] + y[i];
        if (i % 1024 == 0)
            printf("%d %.17g\n", (int)i, y[i]);
    }
    double s = 0.0;
    for (long i = 0; i < n; i++)
        s += y[i];
    printf("sum %.17g\n", s);

    FILE *f = fopen(argv[4], "wb");
    if (!f || fwrite(y, sizeof(double), (size_t)n, f) != (size_t)n) {
        fprintf(stderr, "axpy_sum: cannot write %s\n", argv[4]);
        return 3;
    }
    fclose(f);
    free(x);
    free(y);
    return 0;
}
