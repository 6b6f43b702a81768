/*
 * ORACLE (test infrastructure only).  Only tests/, __graft_entry__.smoke() and
 * bench.py's cpu_baseline leg may build, call or run anything under oracle/.
 *
 * Legacy 3-D Jacobi program, serial, real libc.  The paper's hypterm stencil
 * regions (Sec. 5.3, HeCBench) are the shape this stands in for; the paper
 * does not define a "7-point Jacobi", so the reading used here is Laplace's
 * equation (no source term) with the six-neighbour average:
 *
 *   u'[k][j][i] = (u[i-1] + u[i+1] + u[j-1] + u[j+1] + u[k-1] + u[k+1]) / 6.0
 *
 * with the additions in exactly that left-to-right order, for every interior
 * point 1..n-2 of each axis, and u' = 0 on the boundary.  Each sweep takes a
 * fresh grid from malloc and frees the old one after the swap; the residual is
 * max |u' - u| over the interior, printed "%d %.17g\n" (sweep, residual) with
 * sweeps numbered from 1.  After the last sweep the grid is fwrite'd.
 *
 *   jacobi n sweeps in.bin out.bin        (grid index ((k*n)+j)*n+i, i fastest)
 */
#include <stdio.h>
#include <stdlib.h>
#include <math.h>

int main(int argc, char **argv)
{
    if (argc != 5) {
        fprintf(stderr, "usage: jacobi n sweeps in.bin out.bin\n");
        return 2;
    }
    long n = atol(argv[1]);
    int sweeps = atoi(argv[2]);
    size_t cells = (size_t)n * n * n;
    double *u = malloc(cells * sizeof(double));
    FILE *f = fopen(argv[3], "rb");
    if (!u || !f || fread(u, sizeof(double), cells, f) != cells) {
        fprintf(stderr, "jacobi: cannot read %s\n", argv[3]);
        return 2;
    }
    fclose(f);

    const long sj = n, sk = n * n;
    for (int s = 1; s <= sweeps; s++) {
        double *un = malloc(cells * sizeof(double));
        if (!un) {
            fprintf(stderr, "jacobi: out of memory\n");
            return 4;
        }
        double res = 0.0;
        /* ignored by the plain build (the oracle); the -fopenmp build of this
         * same file is only a timed all-core CPU baseline, never a parity
         * reference: max is order-independent, so its output is the same */
#pragma omp parallel for collapse(2) reduction(max : res)
        for (long k = 0; k < n; k++)
            for (long j = 0; j < n; j++)
                for (long i = 0; i < n; i++) {
                    long c = k * sk + j * sj + i;
                    if (i == 0 || j == 0 || k == 0 || i == n - 1 || j == n - 1 || k == n - 1) {
                        un[c] = 0.0;
                        continue;
                    }
                    double v = u[c - 1] + u[c + 1];
                    v = v + u[c - sj];
                    v = v + u[c + sj];
                    v = v + u[c - sk];
                    v = v + u[c + sk];
                    v = v / 6.0;
                    un[c] = v;
                    double d = fabs(v - u[c]);
                    if (d > res)
                        res = d;
                }
        printf("%d %.17g\n", s, res);
        free(u);
        u = un;
    }

    f = fopen(argv[4], "wb");
    if (!f || fwrite(u, sizeof(double), cells, f) != cells) {
        fprintf(stderr, "jacobi: cannot write %s\n", argv[4]);
        return 3;
    }
    fclose(f);
    free(u);
    return 0;
}
