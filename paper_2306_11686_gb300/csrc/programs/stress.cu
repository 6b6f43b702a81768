/*
 * RPC / heap stress program (device twin of the serial C stress program).
 *
 * Every iteration t of one parallel loop stands for a "device thread": it
 * makes 8 malloc/free pairs of log-uniform sizes (16 B .. 64 KiB), tags each
 * block at its first, middle and last word, reads the tags back into an XOR
 * checksum, and issues 4 printf calls cycling through int / double formats.
 * This is the paper's allocator stress (Sec. 5.1: every thread allocates,
 * uses and frees) together with libc calls from inside a parallel region
 * (Sec. 3.2), so the heap and the warp-aggregated RPC are exercised at once.
 *
 *   stress T                 buffers: 0 = uint32 sizes[8T], 1 = uint64 checksums[T],
 *                                     2 = int64 fail count [1]
 */
#include "../gf_device.cuh"

static __device__ __forceinline__ uint64_t stress_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;   /* SplitMix64 finaliser */
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

GF_MAIN(stress)(int argc, char **argv)
{
    if (argc < 2)
        return 2;
    const long long T = gf_atoll(argv[1]);
    const unsigned *sizes = (const unsigned *)gf_buffer(0);
    unsigned long long *cs = (unsigned long long *)gf_buffer(1);
    unsigned long long *fails = (unsigned long long *)gf_buffer(2);
    if (!sizes || !cs || !fails || gf_buffer_bytes(0) < (uint64_t)T * 32 || gf_buffer_bytes(1) < (uint64_t)T * 8)
        return 2;
    const int rc = gf_parallel_for(0, T, GF_SCHED_STATIC, 1, [=](int64_t t) {
        unsigned long long c = 0;
        for (int j = 0; j < 8; j++) {
            const unsigned s = sizes[8 * t + j];
            const unsigned long long w = s / 8;
            const unsigned long long h = stress_mix((unsigned long long)(8 * t + j + 1));
            unsigned long long *p = (unsigned long long *)gf_malloc(s);
            if (!p) {
                atomicAdd(fails, 1ull);
                continue;
            }
            p[0] = h;
            p[w / 2] = h ^ 0x5555555555555555ull;
            p[w - 1] = ~h;
            c ^= p[0] ^ p[w / 2] ^ p[w - 1] ^ (unsigned long long)(8 * t + j);
            gf_free(p);
            switch (j) {
            case 0:
                gf_printf("%d %d\n", (int)t, j);
                break;
            case 1:
                gf_printf("%d %.17g\n", (int)t, (double)t * 0.25 + 1.0);
                break;
            case 2:
                gf_printf("%lld %.6e\n", (long long)t * 1000003ll, (double)h * 1e-12);
                break;
            case 3:
                gf_printf("%d %x %.3f\n", (int)t, (unsigned)h, (double)(h & 0xffff) / 7.0);
                break;
            }
        }
        cs[t] = c;
    });
    gf_printf("fail %d\n", (int)*(volatile unsigned long long *)fails);
    return rc ? 10 : 0;
}

/*
 * heap_only T                buffers: 0 = uint32 sizes[8T], 1 = uint64 checksums[T], 2 = int64 fail [1]
 * The heap half of the stress program alone (no printf), to time alloc/free pairs.
 * Compiled with the register count left to the compiler (2 blocks per SM):
 * more resident warps only add contention on the per-lane free stacks
 * (571 M pairs/s there, 368 M at 4 blocks per SM).
 */
GF_MAIN_BOUNDS(heap_only, 1)(int argc, char **argv)
{
    const long long T = gf_atoll(argv[1]);
    const unsigned *sizes = (const unsigned *)gf_buffer(0);
    unsigned long long *cs = (unsigned long long *)gf_buffer(1);
    unsigned long long *fails = (unsigned long long *)gf_buffer(2);
    if (!sizes || !cs || !fails)
        return 2;
    return gf_parallel_for(0, T, GF_SCHED_STATIC, 1, [=](int64_t t) {
        unsigned long long c = 0;
        for (int j = 0; j < 8; j++) {
            const unsigned s = sizes[8 * t + j];
            const unsigned long long w = s / 8;
            const unsigned long long h = stress_mix((unsigned long long)(8 * t + j + 1));
            unsigned long long *p = (unsigned long long *)gf_malloc(s);
            if (!p) {
                atomicAdd(fails, 1ull);
                continue;
            }
            p[0] = h;
            p[w / 2] = h ^ 0x5555555555555555ull;
            p[w - 1] = ~h;
            c ^= p[0] ^ p[w / 2] ^ p[w - 1] ^ (unsigned long long)(8 * t + j);
            gf_free(p);
        }
        cs[t] = c;
    }) ? 10 : 0;
}

/* printf_only T              the RPC half alone: 4 printf per iteration, formats as in stress.
 * Compiled with the register count left to the compiler (2 blocks per SM):
 * its calls are bound by the ring and the host, and more resident warps
 * only lengthen the queue for slots (one slot per calling thread: 9.1 M
 * calls/s there, 4.4 M at 4 blocks per SM). */
GF_MAIN_BOUNDS(printf_only, 1)(int argc, char **argv)
{
    const long long T = gf_atoll(argv[1]);
    return gf_parallel_for(0, T, GF_SCHED_STATIC, 1, [=](int64_t t) {
        const unsigned long long h1 = stress_mix((unsigned long long)(8 * t + 3));
        const unsigned long long h2 = stress_mix((unsigned long long)(8 * t + 4));
        gf_printf("%d %d\n", (int)t, 0);
        gf_printf("%d %.17g\n", (int)t, (double)t * 0.25 + 1.0);
        gf_printf("%lld %.6e\n", (long long)t * 1000003ll, (double)h1 * 1e-12);
        gf_printf("%d %x %.3f\n", (int)t, (unsigned)h2, (double)(h2 & 0xffff) / 7.0);
    }) ? 10 : 0;
}
