/*
 * Synthetic legacy loops for launch-configuration tuning (the learned-model
 * pattern added on top of the paper, whose evaluation shows that the team
 * count chosen for an offloaded region changes its speed, Sec. 5.3).
 *
 * Iteration i of a loop with parameters (trip, bytes, flops, div, rpc, seed):
 *   h   = SplitMix64 finaliser of (seed + i * 0x9E3779B97F4A7C15)
 *   acc = sum over k < bytes/8 of (float)x[k * trip + i]     (k-th coalesced stream)
 *   v   = acc; flops times v = fmaf(v, 1.0001f, 0.5f)       (dependent FP32 chain)
 *   if (uint32)h < div_thresh: flops times v = fmaf(v, 0.9999f, -0.25f)   (divergent branch)
 *   if (uint32)(h >> 32) < rpc_thresh: clock() by RPC to the host
 *   z[i] = (double)v
 * The FMA chain is FP32 so that both memory-bound and compute-bound loops
 * exist on GB300 (its FP64 rate would make nearly every loop compute-bound).
 *
 * Launch shape: grid x block threads; warps take work items of `chunk`
 * iterations (lanes stride over an item), round robin (static) or from a
 * shared counter (dynamic).
 */
#include <vector>

#include "../gf_device.cuh"
#include "../gf_internal.h"

struct SynthP {
    int64_t trip, chunk;
    uint32_t nwords, flops, div_thresh, rpc_thresh;
    uint64_t seed;
    int sched;
};

static __device__ __forceinline__ uint64_t synth_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void __launch_bounds__(1024) synth_kernel(SynthP P, const double *__restrict__ x, double *__restrict__ z,
                                                     gf_state *S, unsigned long long *counter)
{
    if (threadIdx.x == 0) {
        gfd::block_setup(S, 1);    /* not a program kernel: every thread is a worker */
    }
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u;
    const int64_t items = (P.trip + P.chunk - 1) / P.chunk;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int64_t it = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    for (;;) {
        if (P.sched == GF_SCHED_DYNAMIC) {
            unsigned long long v = 0;
            if (lane == 0)
                v = atomicAdd(counter, 1ull);
            it = (int64_t)__shfl_sync(0xffffffffu, v, 0);
        }
        if (it >= items)
            break;
        const int64_t i0 = it * P.chunk;
        const int64_t i1 = i0 + P.chunk < P.trip ? i0 + P.chunk : P.trip;
        for (int64_t i = i0 + lane; i < i1; i += 32) {
            const uint64_t h = synth_mix(P.seed + (uint64_t)i * 0x9E3779B97F4A7C15ull);
            float acc = 0.0f;
            for (uint32_t k = 0; k < P.nwords; k++)
                acc = acc + (float)x[(int64_t)k * P.trip + i];
            float v = acc;
            for (uint32_t f = 0; f < P.flops; f++)
                v = __fmaf_rn(v, 1.0001f, 0.5f);
            if ((uint32_t)h < P.div_thresh)
                for (uint32_t f = 0; f < P.flops; f++)
                    v = __fmaf_rn(v, 0.9999f, -0.25f);
            if ((uint32_t)(h >> 32) < P.rpc_thresh) {
                const long long c = gf_clock();
                if (c == -12345)      /* never: the value must not change the result */
                    v = 0.0f;
            }
            z[i] = (double)v;
        }
        if (P.sched != GF_SCHED_DYNAMIC)
            it += nw;
    }
}

static int synth_check(const gf_synth_loop *L, uint64_t xlen, const gf_shape *sh)
{
    if (!L || L->trip < 0 || L->bytes < 8 || L->bytes % 8 || L->bytes > 4096 || !sh || !sh->grid || !sh->block ||
        sh->block % 32 || sh->block > 1024 || !sh->chunk)
        return GF_EINVAL;
    if ((uint64_t)(L->bytes / 8) * (uint64_t)L->trip > xlen)
        return GF_EINVAL;
    return GF_OK;
}

static SynthP synth_params(const gf_synth_loop *L, const gf_shape *sh)
{
    SynthP P;
    P.trip = L->trip;
    P.chunk = sh->chunk;
    P.nwords = L->bytes / 8;
    P.flops = L->flops;
    P.div_thresh = L->div_thresh;
    P.rpc_thresh = L->rpc_thresh;
    P.seed = L->seed;
    P.sched = (int)sh->sched;
    return P;
}

/* One run of one synthetic loop with one launch shape (asynchronous on `stream`). */
extern "C" GF_API int gf_synth_run(gf_ctx *ctx, const gf_synth_loop *L, const double *x, uint64_t xlen, double *z,
                                   const gf_shape *sh, void *stream)
{
    float ms = 0;
    return gf_synth_time(ctx, L, x, xlen, z, sh, 1, 0, stream, &ms);
}

/*
 * Times `nshapes` launch shapes of one loop: per shape one warm-up run, then
 * `reps` timed runs (CUDA events on `stream`); ms[s] = the fastest.  With
 * reps = 0 each shape runs once, untimed.  A program instance of the context
 * is borrowed for the call, so loops with RPCs are served.
 */
extern "C" GF_API int gf_synth_time(gf_ctx *ctx, const gf_synth_loop *L, const double *x, uint64_t xlen, double *z,
                                    const gf_shape *shapes, int nshapes, int reps, void *stream, float *ms)
{
    if (!ctx || !x || !z || !shapes || nshapes < 1 || reps < 0 || !ms)
        return GF_EINVAL;
    for (int s = 0; s < nshapes; s++)
        if (synth_check(L, xlen, &shapes[s]) != GF_OK)
            return GF_EINVAL;
    if (L->rpc_thresh && gf_ctx_server_threads(ctx) == 0)
        return GF_EINVAL;   /* nobody would answer the loop's RPCs */
    int idx = -1;
    gf_state *S = gf_inst_acquire(ctx, stream, 1, &idx);
    if (!S)
        return GF_EBUSY;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = GF_OK;
    unsigned long long *counter = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    /* the dynamic-schedule counter lives in the instance's reduction partials (device scratch) */
    counter = (unsigned long long *)gf_inst_scratch(ctx, idx);
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        rc = GF_ECUDA;
    for (int s = 0; s < nshapes && rc == GF_OK; s++) {
        const SynthP P = synth_params(L, &shapes[s]);
        float best = 1e30f;
        for (int r = 0; r <= reps && rc == GF_OK; r++) {
            if (cudaMemsetAsync(counter, 0, 8, st) != cudaSuccess) {
                rc = GF_ECUDA;
                break;
            }
            if (r > 0)
                cudaEventRecord(e0, st);
            synth_kernel<<<shapes[s].grid, shapes[s].block, 0, st>>>(P, x, z, S, counter);
            if (cudaGetLastError() != cudaSuccess) {
                rc = GF_ECUDA;
                break;
            }
            if (r > 0) {
                cudaEventRecord(e1, st);
                if (cudaEventSynchronize(e1) != cudaSuccess) {
                    rc = GF_ECUDA;
                    break;
                }
                float t = 0;
                cudaEventElapsedTime(&t, e0, e1);
                best = t < best ? t : best;
            }
        }
        ms[s] = reps ? best : 0.0f;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess && rc == GF_OK)
        rc = GF_ECUDA;
    int err = 0;
    if (rc == GF_OK && cudaMemcpy(&err, &S->error, sizeof err, cudaMemcpyDeviceToHost) == cudaSuccess && err)
        rc = err;
    if (e0)
        cudaEventDestroy(e0);
    if (e1)
        cudaEventDestroy(e1);
    gf_inst_release(ctx, idx);
    return rc;
}
