/*
 * Many independent legacy loops (the batching pattern added on top of the
 * paper's runtime): z_k[i] = a_k * x_k[i] + y_k[i] for k = 0 .. n-1, each
 * loop a slice [off_k, off_k + trip_k) of shared x, y, z arrays.
 *
 * Three ways to run them:
 *  - `loops 0 ...`: the plain runtime, one parallel region per loop (each
 *    region ends with the initial thread waiting for every block);
 *  - `loops 1 ...`: ONE batched region, warps pull (loop, chunk) work items;
 *  - gf_axpy_batch_graph: one CUDA graph with one kernel node per loop, each
 *    with its own launch shape (the kernel-split view: the host launches a
 *    multi-team kernel per region, paper Sec. 3.3, Fig. 3), launched once.
 */
#include <vector>

#include "../gf_device.cuh"
#include "../gf_internal.h"

/* loops mode n chunk sched         buffers: 0 = int64 trips[n], 1 = double a[n], 2 = int64 off[n],
 *                                  3 = double x[], 4 = double y[], 5 = double z[], 6 = int64 prefix[n+1] */
/* memory-bound: compiled for 8 resident blocks per SM (2048 threads) so more
 * loads are in flight; its serial part makes no RPC, so little spills */
GF_MAIN_BOUNDS(loops, 8)(int argc, char **argv)
{
    if (argc < 5)
        return 2;
    const int mode = (int)gf_atoll(argv[1]);
    const int n = (int)gf_atoll(argv[2]);
    const long long chunk = gf_atoll(argv[3]);
    const int sched = (int)gf_atoll(argv[4]);
    const long long *trips = (const long long *)gf_buffer(0);
    const double *a = (const double *)gf_buffer(1);
    const long long *off = (const long long *)gf_buffer(2);
    const double *x = (const double *)gf_buffer(3);
    const double *y = (const double *)gf_buffer(4);
    double *z = (double *)gf_buffer(5);
    long long *prefix = (long long *)gf_buffer(6);
    if (!trips || !a || !off || !x || !y || !z || !prefix)
        return 2;
    if (mode == 0) {
        for (int k = 0; k < n; k++) {
            const double ak = a[k];
            const double *xk = x + off[k];
            const double *yk = y + off[k];
            double *zk = z + off[k];
            if (gf_parallel_for(0, trips[k], GF_SCHED_STATIC, 1, [=](int64_t i) { zk[i] = ak * xk[i] + yk[i]; }))
                return 10;
        }
        return 0;
    }
    return gf_parallel_for_batch(n, (const int64_t *)trips, (int64_t *)prefix, chunk, sched,
                                 [=](int k, int64_t i) {
                                     const long long o = off[k];
                                     z[o + i] = a[k] * x[o + i] + y[o + i];
                                 })
               ? 10
               : 0;
}

/*
 * The same loops with libc inside their bodies: every 4096th iteration of
 * loop k takes a block of 64 << (k % 8) bytes from the device heap, passes
 * the element's value through it, frees it, and prints
 * "k i value" by RPC; every loop's RPC traffic shares the program's one ring.
 *
 * loops_rpc mode n chunk sched    buffers as `loops`, plus 7 = int64 fails[1]
 *                                 (heap blocks not granted or corrupted)
 * mode 0: one region per loop; mode 1: one batched region.
 */
/* the libc part of an iteration (every 4096th), out of line so that its
 * code and registers stay out of the loop every other iteration runs */
static __device__ __noinline__ double loop_rpc_libc(int k, int64_t i, double v, unsigned long long *fails)
{
    const unsigned long long words = (64ull << (k & 7)) / 8;
    double *w = (double *)gf_malloc(words * 8);
    if (!w) {
        atomicAdd(fails, 1ull);
    } else {
        w[0] = v;
        w[words - 1] = -v;
        const double r = w[0];
        if (w[words - 1] != -r)
            atomicAdd(fails, 1ull);
        v = r;
        gf_free(w);
    }
    gf_printf("%d %lld %.17g\n", k, (long long)i, v);
    return v;
}

struct loop_rpc_body {
    const double *x, *y;
    double *z;
    unsigned long long *fails;
    __device__ __forceinline__ void operator()(int k, double a, long long o, int64_t i) const
    {
        double v = a * x[o + i] + y[o + i];
        if ((i & 4095) == 0)
            v = loop_rpc_libc(k, i, v, fails);
        z[o + i] = v;
    }
};

GF_MAIN_BOUNDS(loops_rpc, 4)(int argc, char **argv)
{
    if (argc < 5)
        return 2;
    const int mode = (int)gf_atoll(argv[1]);
    const int n = (int)gf_atoll(argv[2]);
    const long long chunk = gf_atoll(argv[3]);
    const int sched = (int)gf_atoll(argv[4]);
    const long long *trips = (const long long *)gf_buffer(0);
    const double *a = (const double *)gf_buffer(1);
    const long long *off = (const long long *)gf_buffer(2);
    loop_rpc_body B{(const double *)gf_buffer(3), (const double *)gf_buffer(4), (double *)gf_buffer(5),
                    (unsigned long long *)gf_buffer(7)};
    long long *prefix = (long long *)gf_buffer(6);
    if (!trips || !a || !off || !B.x || !B.y || !B.z || !prefix || !B.fails)
        return 2;
    if (mode == 0) {
        for (int k = 0; k < n; k++) {
            const double ak = a[k];
            const long long o = off[k];
            if (gf_parallel_for(0, trips[k], GF_SCHED_STATIC, 1, [=](int64_t i) { B(k, ak, o, i); }))
                return 10;
        }
        return 0;
    }
    return gf_parallel_for_batch(n, (const int64_t *)trips, (int64_t *)prefix, chunk, sched,
                                 [=](int k, int64_t i) { B(k, a[k], off[k], i); })
               ? 10
               : 0;
}

/* ------------------------------------------------------------------ graph mode */
__global__ void __launch_bounds__(1024) axpy_loop_kernel(const double *__restrict__ x, const double *__restrict__ y,
                                                          double *__restrict__ z, double a, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        z[i] = a * x[i] + y[i];
}

/* A loop of loops_rpc as its own kernel: the runtime's device state of a
 * borrowed program instance serves its heap and RPC calls. */
__global__ void __launch_bounds__(GF_BLOCK) loop_rpc_kernel(loop_rpc_body B, double a, long long o, int64_t n,
                                                             int k, gf_state *S)
{
    if (threadIdx.x == 0) {
        gfd::block_setup(S, 1);    /* not a program kernel: every thread is a worker */
    }
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        B(k, a, o, i);
}

/*
 * One CUDA graph, one kernel node per loop (no dependencies between nodes, so
 * the GPU may run them concurrently), per-loop grid and block (NULL: a grid
 * covering the loop once at 256 threads, capped at 8 blocks per SM).
 * Replays the graph `reps` times on `stream` and stores the mean milliseconds
 * per replay in *ms (CUDA events on that stream).
 */
extern "C" GF_API int gf_axpy_batch_graph(int n, const int64_t *trips, const double *a, const int64_t *off,
                                          const double *x, const double *y, double *z, const uint32_t *grid,
                                          const uint32_t *block, int reps, void *stream, float *ms)
{
    if (n <= 0 || !trips || !a || !off || !x || !y || !z || reps < 1)
        return GF_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))
        return GF_ECUDA;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = GF_OK;
    std::vector<void *> keep;
    if (cudaGraphCreate(&g, 0) != cudaSuccess)
        return GF_ECUDA;
    struct Args {
        const double *x, *y;
        double *z;
        double a;
        int64_t n;
        void *p[5];
    };
    std::vector<Args> args((size_t)n);
    for (int k = 0; k < n && rc == GF_OK; k++) {
        Args &A = args[(size_t)k];
        A.x = x + off[k];
        A.y = y + off[k];
        A.z = z + off[k];
        A.a = a[k];
        A.n = trips[k];
        A.p[0] = &A.x;
        A.p[1] = &A.y;
        A.p[2] = &A.z;
        A.p[3] = &A.a;
        A.p[4] = &A.n;
        const uint32_t bl = block && block[k] ? block[k] : 256;
        uint64_t gr = grid && grid[k] ? grid[k] : (uint64_t)((trips[k] + bl - 1) / bl);
        if (gr < 1)
            gr = 1;
        if (gr > (uint64_t)sms * 8)
            gr = (uint64_t)sms * 8;
        cudaKernelNodeParams kp = {};
        kp.func = (void *)axpy_loop_kernel;
        kp.gridDim = dim3((unsigned)gr);
        kp.blockDim = dim3(bl);
        kp.sharedMemBytes = 0;
        kp.kernelParams = A.p;
        kp.extra = nullptr;
        cudaGraphNode_t node;
        if (cudaGraphAddKernelNode(&node, g, nullptr, 0, &kp) != cudaSuccess)
            rc = GF_ECUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (rc == GF_OK && (cudaGraphInstantiate(&ge, g, 0) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
                        cudaEventCreate(&e1) != cudaSuccess))
        rc = GF_ECUDA;
    if (rc == GF_OK && cudaGraphLaunch(ge, s) != cudaSuccess)   /* warm-up replay */
        rc = GF_ECUDA;
    if (rc == GF_OK) {
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps; r++)
            cudaGraphLaunch(ge, s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess)
            rc = GF_ECUDA;
        float t = 0;
        cudaEventElapsedTime(&t, e0, e1);
        if (ms)
            *ms = t / reps;
    }
    if (e0)
        cudaEventDestroy(e0);
    if (e1)
        cudaEventDestroy(e1);
    if (ge)
        cudaGraphExecDestroy(ge);
    cudaGraphDestroy(g);
    return rc;
}

/*
 * The graph form of loops_rpc: one kernel node per loop with grid[k] x
 * block[k] threads (either array may be NULL: 256 threads, enough blocks to
 * cover the loop up to 8 per SM; at most GF_BLOCK = 256 threads, the warps
 * the device heap's per-block hand-off area holds).  The loops' heap and RPC calls go through a
 * program instance of ctx borrowed for the call (its heap quota and ring;
 * the context's server threads answer).  The graph is replayed `warmup`
 * times untimed, then `reps` times timed on `stream`; *ms = mean
 * milliseconds per timed replay.  Every replay prints its lines again.
 * Errors: GF_EINVAL, GF_EBUSY (no instance free), GF_ECUDA, or the device
 * error of the loops' calls (GF_ETIMEDOUT, GF_ERING).
 */
extern "C" GF_API int gf_loops_rpc_graph(gf_ctx *ctx, int n, const int64_t *trips, const double *a, const int64_t *off,
                                         const double *x, const double *y, double *z, unsigned long long *fails,
                                         const uint32_t *grid, const uint32_t *block, int warmup, int reps,
                                         void *stream, float *ms)
{
    if (!ctx || n <= 0 || !trips || !a || !off || !x || !y || !z || !fails || warmup < 0 || reps < 0 ||
        warmup + reps < 1 || gf_ctx_server_threads(ctx) == 0)
        return GF_EINVAL;
    for (int k = 0; k < n; k++)
        if ((block && block[k] && (block[k] % 32 || block[k] > GF_BLOCK)) || trips[k] < 0)
            return GF_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))
        return GF_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    int idx = -1;
    gf_state *S = gf_inst_acquire(ctx, stream, 1, &idx);
    if (!S)
        return GF_EBUSY;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = GF_OK;
    struct Args {
        loop_rpc_body B;
        double a;
        long long o;
        int64_t n;
        int k;
        gf_state *S;
        void *p[6];
    };
    std::vector<Args> args((size_t)n);
    if (cudaGraphCreate(&g, 0) != cudaSuccess)
        rc = GF_ECUDA;
    for (int k = 0; k < n && rc == GF_OK; k++) {
        Args &A = args[(size_t)k];
        A.B = loop_rpc_body{x, y, z, fails};
        A.a = a[k];
        A.o = off[k];
        A.n = trips[k];
        A.k = k;
        A.S = S;
        A.p[0] = &A.B;
        A.p[1] = &A.a;
        A.p[2] = &A.o;
        A.p[3] = &A.n;
        A.p[4] = &A.k;
        A.p[5] = &A.S;
        const uint32_t bl = block && block[k] ? block[k] : 256;
        uint64_t gr = grid && grid[k] ? grid[k] : (uint64_t)((trips[k] + bl - 1) / bl);
        if (gr < 1)
            gr = 1;
        if (gr > (uint64_t)sms * 8)
            gr = (uint64_t)sms * 8;
        cudaKernelNodeParams kp = {};
        kp.func = (void *)loop_rpc_kernel;
        kp.gridDim = dim3((unsigned)gr);
        kp.blockDim = dim3(bl);
        kp.sharedMemBytes = 0;
        kp.kernelParams = A.p;
        kp.extra = nullptr;
        cudaGraphNode_t node;
        if (cudaGraphAddKernelNode(&node, g, nullptr, 0, &kp) != cudaSuccess)
            rc = GF_ECUDA;
    }
    if (rc == GF_OK && (cudaGraphInstantiate(&ge, g, 0) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
                        cudaEventCreate(&e1) != cudaSuccess))
        rc = GF_ECUDA;
    for (int r = 0; r < warmup && rc == GF_OK; r++)
        if (cudaGraphLaunch(ge, s) != cudaSuccess)
            rc = GF_ECUDA;
    if (rc == GF_OK && reps > 0) {
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps; r++)
            if (cudaGraphLaunch(ge, s) != cudaSuccess)
                rc = GF_ECUDA;
        cudaEventRecord(e1, s);
    }
    if (cudaStreamSynchronize(s) != cudaSuccess && rc == GF_OK)
        rc = GF_ECUDA;
    if (rc == GF_OK && reps > 0 && ms) {
        float t = 0;
        cudaEventElapsedTime(&t, e0, e1);
        *ms = t / reps;
    }
    int err = 0;
    if (rc == GF_OK && cudaMemcpy(&err, &S->error, sizeof err, cudaMemcpyDeviceToHost) == cudaSuccess && err)
        rc = err;
    if (e0)
        cudaEventDestroy(e0);
    if (e1)
        cudaEventDestroy(e1);
    if (ge)
        cudaGraphExecDestroy(ge);
    if (g)
        cudaGraphDestroy(g);
    gf_inst_release(ctx, idx);
    return rc;
}
