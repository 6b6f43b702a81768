/*
 * ORACLE (test infrastructure only).  Only tests/, __graft_entry__.smoke() and
 * bench.py's cpu_baseline leg may build, call or run anything under oracle/.
 *
 * RPC / heap stress program, serial, real libc.  It stands in for the
 * allocation pattern the paper measures (Sec. 5.1: every thread of every team
 * allocates, uses and frees) combined with libc calls from inside a parallel
 * loop (Sec. 3.2).  For each iteration t in [0, T) ("device thread" t):
 *
 *   for j in 0..7:
 *     s = sizes[8t + j]  (bytes, 16..65536);  w = s / 8 words
 *     h = mix(8t + j + 1), mix = the SplitMix64 finaliser (xor-shift 30,
 *         multiply 0xBF58476D1CE4E5B9, xor-shift 27, multiply
 *         0x94D049BB133111EB, xor-shift 31)
 *     p = malloc(s); p[0] = h; p[w/2] = h ^ 0x5555555555555555; p[w-1] = ~h
 *     cs ^= p[0] ^ p[w/2] ^ p[w-1] ^ (8t + j)      (read back, then free(p))
 *     j = 0: printf("%d %d\n", t, j)
 *     j = 1: printf("%d %.17g\n", t, t * 0.25 + 1)
 *     j = 2: printf("%lld %.6e\n", t * 1000003, (double)h * 1e-12)
 *     j = 3: printf("%d %x %.3f\n", t, (unsigned)h, (h & 0xffff) / 7.0)
 *   checksum[t] = cs
 *
 *   stress T sizes.bin checksums.bin      prints the lines, then "fail %d\n"
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

static uint64_t mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

int main(int argc, char **argv)
{
    if (argc != 4) {
        fprintf(stderr, "usage: stress T sizes.bin checksums.bin\n");
        return 2;
    }
    long T = atol(argv[1]);
    uint32_t *sizes = malloc((size_t)T * 8 * sizeof(uint32_t));
    uint64_t *cs = malloc((size_t)T * sizeof(uint64_t));
    FILE *f = fopen(argv[2], "rb");
    if (!sizes || !cs || !f || fread(sizes, sizeof(uint32_t), (size_t)T * 8, f) != (size_t)T * 8) {
        fprintf(stderr, "stress: cannot read %s\n", argv[2]);
        return 2;
    }
    fclose(f);
    int fail = 0;
    for (long t = 0; t < T; t++) {
        uint64_t c = 0;
        for (int j = 0; j < 8; j++) {
            const uint32_t s = sizes[8 * t + j];
            const uint64_t w = s / 8;
            const uint64_t h = mix((uint64_t)(8 * t + j + 1));
            uint64_t *p = malloc(s);
            if (!p) {
                fail++;
                continue;
            }
            p[0] = h;
            p[w / 2] = h ^ 0x5555555555555555ull;
            p[w - 1] = ~h;
            c ^= p[0] ^ p[w / 2] ^ p[w - 1] ^ (uint64_t)(8 * t + j);
            free(p);
            switch (j) {
            case 0:
                printf("%d %d\n", (int)t, j);
                break;
            case 1:
                printf("%d %.17g\n", (int)t, (double)t * 0.25 + 1.0);
                break;
            case 2:
                printf("%lld %.6e\n", (long long)t * 1000003ll, (double)h * 1e-12);
                break;
            case 3:
                printf("%d %x %.3f\n", (int)t, (unsigned)h, (double)(h & 0xffff) / 7.0);
                break;
            }
        }
        cs[t] = c;
    }
    printf("fail %d\n", fail);
    f = fopen(argv[3], "wb");
    if (!f || fwrite(cs, sizeof(uint64_t), (size_t)T, f) != (size_t)T)
        return 3;
    fclose(f);
    free(sizes);
    free(cs);
    return 0;
}
