/*
 * ORACLE (test infrastructure only).  Only tests/, __graft_entry__.smoke() and
 * bench.py's cpu_baseline leg may build, call or run anything under oracle/.
 *
 * One synthetic legacy loop, serial (the launch-shape tuning workload):
 *   for i in [0, trip):
 *     h   = mix(seed + i * 0x9E3779B97F4A7C15)      (SplitMix64 finaliser)
 *     acc = 0f; for k < bytes/8: acc = acc + (float)x[k * trip + i]
 *     v = acc; flops times: v = fmaf(v, 1.0001f, 0.5f)
 *     if ((uint32)h < div_thresh): flops times: v = fmaf(v, 0.9999f, -0.25f)
 *     (if ((uint32)(h >> 32) < rpc_thresh) the program calls clock(); the
 *      value does not enter the result)
 *     z[i] = (double)v
 * fmaf is the C99 fused multiply-add, rounded once.
 *
 *   synth trip bytes flops div_thresh rpc_thresh seed x.bin z.bin
 *   prints "rpc %ld\n": how many iterations made the clock() call
 */
#include <math.h>
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
    if (argc != 9) {
        fprintf(stderr, "usage: synth trip bytes flops div_thresh rpc_thresh seed x.bin z.bin\n");
        return 2;
    }
    const long trip = atol(argv[1]);
    const unsigned nwords = (unsigned)atol(argv[2]) / 8, flops = (unsigned)atol(argv[3]);
    const uint32_t div_t = (uint32_t)strtoul(argv[4], 0, 10), rpc_t = (uint32_t)strtoul(argv[5], 0, 10);
    const uint64_t seed = strtoull(argv[6], 0, 10);
    const size_t nx = (size_t)nwords * (size_t)trip;
    double *x = malloc((nx ? nx : 1) * sizeof(double));
    double *z = malloc((trip ? trip : 1) * sizeof(double));
    FILE *f = fopen(argv[7], "rb");
    if (!x || !z || !f || fread(x, sizeof(double), nx, f) != nx) {
        fprintf(stderr, "synth: cannot read %s\n", argv[7]);
        return 2;
    }
    fclose(f);
    long rpc = 0;
    for (long i = 0; i < trip; i++) {
        const uint64_t h = mix(seed + (uint64_t)i * 0x9E3779B97F4A7C15ull);
        float acc = 0.0f;
        for (unsigned k = 0; k < nwords; k++)
            acc = acc + (float)x[(size_t)k * trip + i];
        float v = acc;
        for (unsigned q = 0; q < flops; q++)
            v = fmaf(v, 1.0001f, 0.5f);
        if ((uint32_t)h < div_t)
            for (unsigned q = 0; q < flops; q++)
                v = fmaf(v, 0.9999f, -0.25f);
        if ((uint32_t)(h >> 32) < rpc_t)
            rpc++;
        z[i] = (double)v;
    }
    printf("rpc %ld\n", rpc);
    f = fopen(argv[8], "wb");
    if (!f || fwrite(z, sizeof(double), (size_t)trip, f) != (size_t)trip)
        return 3;
    fclose(f);
    return 0;
}
