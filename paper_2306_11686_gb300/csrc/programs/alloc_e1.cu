/*
 * The paper's allocator experiment (Sec. 5.1, Fig. 6): `teams` blocks of
 * `threads` threads; every thread allocates at kernel start, uses the block
 * briefly and frees it.  Allocators compared: the runtime's slab heap, the
 * paper's balanced allocator (N = 32 thread slots x M = 16 team slots, as in
 * the paper's figure), the paper's generic allocator, and CUDA's own device
 * malloc (the paper's baseline, "NVIDIA malloc").
 */
#include <stdio.h>

#include <algorithm>

#include "../gf_device.cuh"
#include "../gf_internal.h"
#include "../gf_paper_alloc.cuh"

#define E1_RATIO 4        /* first-chunk ratio (the paper calls it configurable; value not given) */

template <int KIND>
__global__ void __launch_bounds__(256) e1_kernel(gf_state *S, gfpa::balanced B, gfpa::generic G, uint32_t bytes,
                                                 unsigned long long *fails)
{
    if (KIND == 0) {
        if (threadIdx.x == 0) {
            gfd::block_setup(S, 1);    /* not a program kernel: every thread is a worker */
        }
        __syncthreads();
    }
    const unsigned long long tag = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x + 1;
    void *p;
    if (KIND == 0)
        p = gf_malloc(bytes);
    else if (KIND == 1)
        p = gfpa::balanced_malloc(B, threadIdx.x, blockIdx.x, bytes);
    else if (KIND == 2)
        p = gfpa::generic_malloc(G, bytes);
    else
        p = malloc(bytes);
    if (p) {
        volatile unsigned long long *q = (volatile unsigned long long *)p;
        q[0] = tag;
        if (q[0] != tag)
            atomicAdd(fails, 1ull << 32);
    } else {
        atomicAdd(fails, 1ull);
    }
    if (KIND == 0)
        gf_free(p);
    else if (KIND == 1)
        gfpa::balanced_free(B, threadIdx.x, blockIdx.x, p);
    else if (KIND == 2)
        gfpa::generic_free(G, p);
    else
        free(p);
}

/*
 * balanced_probe                  buffer 0 = int64 out[16]
 * The chunk life cycle of the paper's Fig. 5 on one chunk of the balanced
 * allocator: three entries; freeing the middle one leaves the watermark;
 * freeing the top one reclaims it and, chained, the middle one; the next
 * allocation lands where the middle entry was; a full chunk reuses a freed
 * entry by walking the entries.
 */
GF_MAIN(balanced_probe)(int argc, char **argv)
{
    long long *out = (long long *)gf_buffer(0);
    unsigned char *arena = (unsigned char *)gf_malloc(1 << 20);
    gfpa::chunk_state *st = (gfpa::chunk_state *)gf_malloc(256);
    if (!out || !arena || !st)
        return 2;
    for (int k = 0; k < 256 / 4; k++)
        ((unsigned *)st)[k] = 0;
    gfpa::balanced B;
    B.arena = arena;
    B.st = st;
    B.N = 2;
    B.M = 1;
    B.chunk = 1024;
    B.ratio = 2;                                   /* chunk (0, 0) is 2048 B, chunk (1, 0) 1024 B */
    unsigned char *base = B.base(1, 0);
    unsigned char *a = (unsigned char *)gfpa::balanced_malloc(B, 1, 0, 100);   /* thread 1 -> chunk 1 */
    unsigned char *b = (unsigned char *)gfpa::balanced_malloc(B, 1, 0, 200);
    unsigned char *c = (unsigned char *)gfpa::balanced_malloc(B, 1, 0, 50);
    out[0] = a - base;
    out[1] = b - base;
    out[2] = c - base;
    out[3] = st[1].top;
    gfpa::balanced_free(B, 1, 0, b);
    out[4] = st[1].top;                            /* middle freed: watermark stays */
    gfpa::balanced_free(B, 1, 0, c);
    out[5] = st[1].top;                            /* top freed: reclaims c and, chained, b */
    unsigned char *d = (unsigned char *)gfpa::balanced_malloc(B, 1, 0, 100);
    out[6] = d - base;
    /* fill the chunk, free one entry in the middle, then ask for a smaller block */
    unsigned char *blocks[64];
    int nb = 0;
    for (; nb < 64; nb++) {
        blocks[nb] = (unsigned char *)gfpa::balanced_malloc(B, 1, 0, 48);
        if (!blocks[nb])
            break;
    }
    out[7] = nb;                                   /* how many 48 B entries still fitted */
    gfpa::balanced_free(B, 1, 0, blocks[2]);
    unsigned char *e = (unsigned char *)gfpa::balanced_malloc(B, 1, 0, 32);
    out[8] = e - base;
    out[9] = blocks[2] - base;
    out[10] = (long long)(uintptr_t)gfpa::balanced_malloc(B, 1, 0, 48);   /* full again: NULL */
    out[11] = (long long)((unsigned char *)gfpa::balanced_malloc(B, 0, 0, 1500) - B.base(0, 0));   /* big first chunk */
    out[12] = (long long)(uintptr_t)gfpa::balanced_malloc(B, 1, 0, 1500);                       /* too big for chunk 1 */
    gf_free(arena);
    gf_free(st);
    return 0;
}

extern "C" GF_API int gf_alloc_e1(gf_ctx *ctx, int kind, uint32_t teams, uint32_t threads, uint32_t bytes, int reps,
                                  void *stream, float *ms, uint64_t *fails)
{
    if (!ctx || kind < 0 || kind > 3 || !teams || !threads || threads > 256 || !bytes || reps < 1 || !ms)
        return GF_EINVAL;
    static bool cuda_heap_set = false;
    if (kind == 3 && !cuda_heap_set) {
        size_t cur = 0;
        cudaDeviceGetLimit(&cur, cudaLimitMallocHeapSize);
        if (cur < (1ull << 30) && cudaDeviceSetLimit(cudaLimitMallocHeapSize, 1ull << 30) != cudaSuccess)
            return GF_ECUDA;
        cuda_heap_set = true;
    }
    int idx = -1;
    gf_state *S = gf_inst_acquire(ctx, stream, 1, &idx);
    if (!S)
        return GF_EBUSY;
    unsigned char *arena = nullptr;
    uint64_t arena_bytes = 0;
    gf_inst_heap(ctx, idx, (void **)&arena, &arena_bytes);
    unsigned char *scratch = (unsigned char *)gf_inst_scratch(ctx, idx);
    cudaStream_t st = (cudaStream_t)stream;
    gfpa::balanced B;
    B.N = 32;
    B.M = 16;
    B.ratio = E1_RATIO;
    B.arena = arena;
    B.st = (gfpa::chunk_state *)(scratch + 64);
    B.chunk = (uint32_t)std::min<uint64_t>(arena_bytes / ((uint64_t)B.M * (B.ratio + B.N - 1)), 0xfff00000ull) & ~15u;
    gfpa::generic G;
    G.arena = arena;
    G.bytes = std::min<uint64_t>(arena_bytes, 0xfff00000ull);
    G.st = (gfpa::chunk_state *)(scratch + 64);
    unsigned long long *d_fails = (unsigned long long *)scratch;
    const size_t state_bytes = 64 + (size_t)B.N * B.M * sizeof(gfpa::chunk_state);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = GF_OK;
    float total = 0;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        rc = GF_ECUDA;
    for (int r = 0; r <= reps && rc == GF_OK; r++) {
        /* a fresh allocator every launch (the slab heap was reset when the instance was taken) */
        if (cudaMemsetAsync(scratch, 0, state_bytes, st) != cudaSuccess) {
            rc = GF_ECUDA;
            break;
        }
        cudaEventRecord(e0, st);
        switch (kind) {
        case 0: e1_kernel<0><<<teams, threads, 0, st>>>(S, B, G, bytes, d_fails); break;
        case 1: e1_kernel<1><<<teams, threads, 0, st>>>(S, B, G, bytes, d_fails); break;
        case 2: e1_kernel<2><<<teams, threads, 0, st>>>(S, B, G, bytes, d_fails); break;
        default: e1_kernel<3><<<teams, threads, 0, st>>>(S, B, G, bytes, d_fails); break;
        }
        cudaEventRecord(e1, st);
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
            rc = GF_ECUDA;
            break;
        }
        float t = 0;
        cudaEventElapsedTime(&t, e0, e1);
        if (r > 0)
            total += t;
    }
    if (rc == GF_OK) {
        *ms = total / reps;
        if (fails)
            cudaMemcpy(fails, d_fails, 8, cudaMemcpyDeviceToHost);
    }
    if (e0)
        cudaEventDestroy(e0);
    if (e1)
        cudaEventDestroy(e1);
    cudaStreamSynchronize(st);
    gf_inst_release(ctx, idx);
    return rc;
}
