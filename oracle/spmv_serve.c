/*
 * ORACLE (test infrastructure only).  Only tests/, __graft_entry__.smoke() and
 * bench.py's cpu_baseline leg may build, call or run anything under oracle/.
 *
 * One "served" legacy program: R passes of a CSR sparse matrix-vector product
 * y = A x (then x = y), with libc requests issued at seeded row positions.
 * It stands for the paper's AMGmk / page-rank style regions (Sec. 5.3) plus
 * libc calls from inside them (Sec. 3.2).
 *
 *   y_i = sum over j in [rowptr_i, rowptr_{i+1}) of val_j * x[col_j], in CSR
 *   order, each product and sum rounded separately (-ffp-contract=off).
 *
 * Request q (sorted by pass, then row) fires in pass pass_q after row row_q
 * is computed.  type = kind | size << 8:
 *   kind 0 fwrite: a record of 16 + size bytes to the program's file:
 *          header {u32 prog, u32 pass, u32 row, u32 size} then size payload
 *          bytes, byte b = low byte of mix(key + (b / 8) * GOLDEN) >> (8 (b % 8)),
 *          key = mix(prog << 40 ^ pass << 32 ^ row); result = items written
 *   kind 1 printf("p %d r %d row %d y %.17g\n", prog, pass, row, y_row); result = chars
 *   kind 2 clock(); result = its value (not comparable across runs)
 *   kind 3 getenv(name) with name = "GF_SERVE_VAR" followed by (row % 3);
 *          result = strlen(value) or -1 when unset
 * mix = SplitMix64 finaliser, GOLDEN = 0x9E3779B97F4A7C15.
 *
 *   spmv_serve prog R n nnz nreq rowptr.bin col.bin val.bin x.bin req.bin out_y.bin records.bin results.bin
 *   (req.bin: nreq x {int64 pass << 32 | row, int64 type})
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

static uint64_t mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static void *load(const char *p, size_t bytes)
{
    void *m = malloc(bytes ? bytes : 1);
    FILE *f = fopen(p, "rb");
    if (!m || !f || fread(m, 1, bytes, f) != bytes) {
        fprintf(stderr, "spmv_serve: cannot read %s\n", p);
        exit(2);
    }
    fclose(f);
    return m;
}

int main(int argc, char **argv)
{
    if (argc != 14) {
        fprintf(stderr, "usage: spmv_serve prog R n nnz nreq rowptr col val x req out_y records results\n");
        return 2;
    }
    const uint32_t prog = (uint32_t)atol(argv[1]);
    const int R = atoi(argv[2]);
    const long n = atol(argv[3]), nnz = atol(argv[4]), nreq = atol(argv[5]);
    int64_t *rowptr = load(argv[6], (size_t)(n + 1) * 8);
    int32_t *col = load(argv[7], (size_t)nnz * 4);
    double *val = load(argv[8], (size_t)nnz * 8);
    double *x = load(argv[9], (size_t)n * 8);
    int64_t *req = load(argv[10], (size_t)nreq * 16);
    double *y = malloc((size_t)n * 8);
    int64_t *res = calloc((size_t)(nreq ? nreq : 1), 8);
    FILE *rec = fopen(argv[12], "wb");
    if (!y || !res || !rec)
        return 2;
    long q = 0;
    for (int r = 0; r < R; r++) {
        for (long i = 0; i < n; i++) {
            double s = 0.0;
            for (int64_t j = rowptr[i]; j < rowptr[i + 1]; j++)
                s = s + val[j] * x[col[j]];
            y[i] = s;
            while (q < nreq && (req[2 * q] >> 32) == r && (req[2 * q] & 0xffffffff) == i) {
                const int kind = (int)(req[2 * q + 1] & 0xff);
                const uint32_t size = (uint32_t)(req[2 * q + 1] >> 8);
                if (kind == 0) {
                    unsigned char *b = malloc(16 + (size_t)size);
                    const uint32_t hdr[4] = {prog, (uint32_t)r, (uint32_t)i, size};
                    memcpy(b, hdr, 16);
                    const uint64_t key = mix(((uint64_t)prog << 40) ^ ((uint64_t)r << 32) ^ (uint64_t)i);
                    for (uint32_t k = 0; k < size; k++)
                        b[16 + k] = (unsigned char)(mix(key + (uint64_t)(k / 8) * 0x9E3779B97F4A7C15ull) >> (8 * (k % 8)));
                    res[q] = (int64_t)fwrite(b, 1, 16 + (size_t)size, rec);
                    free(b);
                } else if (kind == 1) {
                    res[q] = printf("p %d r %d row %d y %.17g\n", (int)prog, r, (int)i, s);
                } else if (kind == 2) {
                    res[q] = (int64_t)clock();
                } else {
                    char name[32];
                    snprintf(name, sizeof name, "GF_SERVE_VAR%d", (int)(i % 3));
                    const char *v = getenv(name);
                    res[q] = v ? (int64_t)strlen(v) : -1;
                }
                q++;
            }
        }
        double *t = x;
        x = y;
        y = t;
    }
    fclose(rec);
    FILE *f = fopen(argv[11], "wb");
    if (!f || fwrite(x, 8, (size_t)n, f) != (size_t)n)
        return 3;
    fclose(f);
    f = fopen(argv[13], "wb");
    if (!f || fwrite(res, 8, (size_t)(nreq ? nreq : 0), f) != (size_t)nreq)
        return 3;
    fclose(f);
    return 0;
}
