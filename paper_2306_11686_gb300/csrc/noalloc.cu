/*
 * gf_reduce_f64_noalloc: the worksharing reduction without any allocation.
 *
 * Who needs it: code that cannot create a gf_ctx or call cudaMalloc -- for
 * example a library running under another framework's fixed memory budget or
 * inside its pool allocator's lock, code that must not change the device's
 * memory footprint, or a caller that only needs one reduction and cannot pay
 * for a context (a context reserves a device heap arena, a pinned RPC ring and
 * per-instance state).  Such callers pass their input and output buffers and
 * nothing else is allocated on their behalf.
 *
 * Same algorithm as a gf_reduce region: per-thread accumulation (Neumaier
 * compensation for sums), xor-shuffle warp tree, shared-memory block tree, one
 * partial per block; the last block to finish merges the partials with a
 * strided per-thread pass (thread t takes partials t, t + 256, ...) followed
 * by the same warp and block trees.  The per-block partials and the
 * last-block ticket live in one file-scope device array, gf_noalloc_scratch,
 * instead of context memory.  The combine order depends only on the grid, so
 * a SUM gives the same bits on every run with the same `blocks`; the default
 * grid follows the device (SMs x occupancy), so callers that need identical
 * bits on every GPU pass `blocks` explicitly.
 *
 * Limits and sharing:
 *  - at most GF_NOALLOC_MAX_BLOCKS blocks (the scratch holds one 16-byte
 *    partial per block): 2048 blocks, 32 KiB of partials plus a 256-byte
 *    counter line, held by every GPU that loads this library until exit;
 *  - every call uses the same array; it keeps the last call's contents, and
 *    the ticket counter is cleared (cudaMemsetAsync, no allocation) before each
 *    launch.  Calls that overlap on the GPU (different streams, or different
 *    host threads on the same device) race on the array and give wrong
 *    results: serialise them;
 *  - the first call on a device looks up the array's device address with
 *    cudaGetSymbolAddress (with that device current) and caches it.
 */
#include <cuda_runtime.h>
#include <functional>
#include <mutex>
#include <stdio.h>

#include "gf_device.cuh"

#define GF_NOALLOC_MAX_BLOCKS 2048
#define GF_NOALLOC_SCRATCH_BYTES (GF_NOALLOC_MAX_BLOCKS * 16 + 256)
#define GF_NOALLOC_MAX_DEVICES 64

/* partials[0 .. 2*MAX_BLOCKS) as uint64 words, then the ticket counter */
static __device__ __align__(256) unsigned char gf_noalloc_scratch[GF_NOALLOC_SCRATCH_BYTES];

template <int OP>
__global__ void __launch_bounds__(256) noalloc_reduce_kernel(const double *x, int64_t n, double *out,
                                                             unsigned char *scratch)
{
    uint64_t *part = (uint64_t *)scratch;
    unsigned *ticket = (unsigned *)(scratch + GF_NOALLOC_MAX_BLOCKS * 16);
    __shared__ uint64_t sred[8][2];
    __shared__ unsigned last;
    const unsigned warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    gfd::acc<double, OP> a;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a.add(x[i]);
    a = gfd::warp_tree(a);
    if (lane == 0)
        a.to_words(sred[warp]);
    __syncthreads();
    if (warp == 0) {
        gfd::acc<double, OP> b;
        if (lane < (blockDim.x >> 5))
            b.from_words(sred[lane]);
        b = gfd::warp_tree(b);
        if (lane == 0) {
            uint64_t w[2];
            b.to_words(w);
            part[2 * blockIdx.x] = w[0];
            part[2 * blockIdx.x + 1] = w[1];
            __threadfence();
            last = atomicAdd(ticket, 1u) == gridDim.x - 1;
        }
    }
    __syncthreads();
    if (!last)
        return;
    __threadfence();
    gfd::acc<double, OP> c;
    for (unsigned k = threadIdx.x; k < gridDim.x; k += blockDim.x) {
        gfd::acc<double, OP> p;
        uint64_t w[2] = {gfd::ld_vol64(part + 2 * k), gfd::ld_vol64(part + 2 * k + 1)};
        p.from_words(w);
        c.merge(p);
    }
    c = gfd::warp_tree(c);
    if (lane == 0)
        c.to_words(sred[warp]);
    __syncthreads();
    if (warp == 0) {
        gfd::acc<double, OP> d;
        if (lane < (blockDim.x >> 5))
            d.from_words(sred[lane]);
        d = gfd::warp_tree(d);
        if (lane == 0)
            *out = d.result();
    }
}

namespace {
struct DevSetup {
    std::once_flag once;
    void *scratch = nullptr;
    int blocks = 0;
    int rc = GF_OK;
};
DevSetup g_dev[GF_NOALLOC_MAX_DEVICES];

/* once per device, with that device current: the array's device address and the default grid */
void setup(DevSetup &d, int dev)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, gf_noalloc_scratch);
    if (e != cudaSuccess) {
        fprintf(stderr, "gf_reduce_f64_noalloc: cudaGetSymbolAddress failed on device %d: %s\n", dev,
                cudaGetErrorString(e));
        d.rc = GF_ECUDA;
        return;
    }
    int sms = 0, occ = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, noalloc_reduce_kernel<GF_RED_SUM>, 256, 0) !=
            cudaSuccess) {
        d.rc = GF_ECUDA;
        return;
    }
    int b = sms * (occ > 0 ? occ : 1);
    d.blocks = b < GF_NOALLOC_MAX_BLOCKS ? b : GF_NOALLOC_MAX_BLOCKS;
    d.scratch = p;
}
} // namespace

extern "C" GF_API int gf_reduce_f64_noalloc(const double *x, int64_t n, int op, double *out, uint32_t blocks,
                                            void *stream)
{
    if (!out || n < 0 || (n > 0 && !x) || (op != GF_RED_SUM && op != GF_RED_MIN && op != GF_RED_MAX))
        return GF_EINVAL;
    if (blocks > GF_NOALLOC_MAX_BLOCKS) {
        fprintf(stderr, "gf_reduce_f64_noalloc: %u blocks requested, the static scratch holds at most %d\n", blocks,
                GF_NOALLOC_MAX_BLOCKS);
        return GF_EINVAL;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= GF_NOALLOC_MAX_DEVICES)
        return GF_ECUDA;
    DevSetup &d = g_dev[dev];
    std::call_once(d.once, setup, std::ref(d), dev);
    if (d.rc != GF_OK)
        return d.rc;
    const unsigned grid = blocks ? blocks : (unsigned)d.blocks;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char *scr = (unsigned char *)d.scratch;
    if (cudaMemsetAsync(scr + GF_NOALLOC_MAX_BLOCKS * 16, 0, sizeof(unsigned), s) != cudaSuccess)
        return GF_ECUDA;
    /* cudaLaunchKernel reports this launch's own status: an error left
     * pending on the caller's thread by earlier work is neither read nor
     * cleared here */
    const void *fn = op == GF_RED_SUM   ? (const void *)noalloc_reduce_kernel<GF_RED_SUM>
                     : op == GF_RED_MIN ? (const void *)noalloc_reduce_kernel<GF_RED_MIN>
                                        : (const void *)noalloc_reduce_kernel<GF_RED_MAX>;
    void *args[4] = {(void *)&x, (void *)&n, (void *)&out, (void *)&scr};
    return cudaLaunchKernel(fn, dim3(grid), dim3(256), args, 0, s) == cudaSuccess ? GF_OK : GF_ECUDA;
}
