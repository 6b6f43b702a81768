/*
 * gf.h -- C ABI of the GPU-First runtime for GB300 (sm_103a).
 *
 * What the library does (paper: "GPU First -- Execution of Legacy CPU Codes on
 * GPUs", Sec. 1 and Sec. 3, Fig. 1): a legacy-style program runs WHOLE on one
 * GPU.  Its serial part runs on one initial thread, its parallel-for regions
 * are workshared over every SM (Sec. 3.3), malloc/free are served by a device
 * heap (Sec. 3.4) and libc calls the GPU cannot make (printf, fopen, fwrite,
 * fread, fclose, clock, getenv) are forwarded to a host server by RPC
 * (Sec. 3.2).  Programs are written against the device header gf_device.cuh
 * and registered by name with GF_MAIN(name); this header is the host side.
 *
 * Conventions for every function below:
 *  - return 0 (GF_OK) on success or a negative GF_E* code; nothing aborts;
 *  - pointers are plain host pointers unless the argument says "device";
 *    a cudaStream_t travels as void*;
 *  - the context owns every buffer it allocates; caller buffers stay the
 *    caller's.  Functions are thread-safe per context unless noted.
 */
#ifndef GF_H
#define GF_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define GF_API __attribute__((visibility("default")))
#else
#define GF_API
#endif

/* ------------------------------------------------------------------ errors */
#define GF_OK 0
#define GF_EINVAL -1       /* bad argument, unknown handle, record larger than a ring slot  */
#define GF_ENOMEM -2       /* device heap, ring or host allocation exhausted                */
#define GF_ERING -3        /* no ring slot became free within the timeout                   */
#define GF_ETIMEDOUT -4    /* the host (or a region / barrier) did not answer in time       */
#define GF_EHOST -5        /* a host landing pad failed                                     */
#define GF_ECUDA -6        /* a CUDA runtime call failed                                    */
#define GF_ENOENT -7       /* no program registered under that name                         */
#define GF_EBUSY -8        /* no free program instance (admission refused)                  */

/* ------------------------------------------------------------------ types */
typedef struct gf_ctx gf_ctx;          /* runtime context: ring, heap, server, instances   */
typedef struct gf_handle gf_handle;    /* one launched program                             */
typedef int32_t gf_program;            /* registry id from gf_program_lookup               */

/* Runtime configuration.  Fill with gf_config_default, then override. */
typedef struct gf_config {
    uint64_t heap_bytes;          /* default heap quota of a program (default 4 GiB)               */
    uint32_t heap_small_pct;      /* percent of the arena for the small-size slabs (default 50)    */
    uint32_t ring_slots;          /* default ring-slot quota of a program, power of two (4096)     */
    uint32_t slot_bytes;          /* bytes per slot, multiple of 64, >= 1024 (default 4096)        */
    uint32_t aggregate;           /* 1 = warp-aggregated RPC, 0 = one slot per calling thread      */
    uint32_t server_threads;      /* host RPC server threads started by gf_init (default 1;
                                     0 = the caller serves with gf_rpc_serve / gf_wait)            */
    uint32_t max_programs;        /* program instances that may run at once (default 1): each has
                                     its state, reduction partials, format cache and bulk arena  */
    uint32_t grid;                /* blocks per program launch, 0 = SMs x occupancy / max_programs */
    int64_t timeout_ns;           /* bound of every device wait (default 30 s)                     */
    void *stream;                 /* cudaStream_t for gf_run_main (NULL = a stream of the context) */
    const char *stdout_path;      /* where device printf goes (NULL = this process's stdout)       */
    uint32_t fmt_cache;           /* format-string cache entries per instance, power of two (4096) */
    int32_t device;               /* CUDA device ordinal (-1 = current device)                    */
    uint64_t bulk_bytes;          /* pinned, device-mapped staging arena per instance for large
                                     fwrite/fread from the serial part (default 64 MiB; 0 = DMA) */
    uint32_t split_regions;       /* 0 (default): regions run on the program's persistent grid.
                                     1: the paper's kernel split (Sec. 3.3, Fig. 3), kept as a
                                     comparator -- the program kernel is one block, and each
                                     parallel region is an RPC on which the host server launches
                                     the region as its own kernel (on a stream of the instance)
                                     while the initial thread waits for its blocks to finish.
                                     Needs server_threads >= 1.  A region kernel cannot start
                                     under a profiler that serialises kernels (ncu): the program
                                     then times out waiting for it. */
    uint32_t pad0;
    uint64_t heap_pool_bytes;     /* device heap shared by all running programs: a launch takes its
                                     heap quota from it (0 = heap_bytes x max_programs; both
                                     rounded up to whole 256 KiB slabs)                          */
    uint32_t ring_pool_slots;     /* ring slots shared by all running programs: a launch takes its
                                     ring quota from it (0 = ring_slots x max_programs)           */
    uint32_t pad1;
} gf_config;

/* Memory a launch asks for (gf_launch_q).  Zero fields take the context's
 * defaults (gf_config.heap_bytes, gf_config.ring_slots).  The heap quota is
 * rounded up to 256 KiB and split like a whole arena (heap_small_pct); the
 * ring quota is a power of two, at least the number of server threads. */
typedef struct gf_quota {
    uint64_t heap_bytes;
    uint32_t ring_slots;
    uint32_t pad;
} gf_quota;

/* A buffer mapped into the program before main (the loader's job, paper
 * Sec. 3.1).  Device pointers are used in place.  Host pointers are copied to
 * device memory before launch when dir has GF_BUF_IN and copied back after the
 * program ends when dir has GF_BUF_OUT.  The program reads them with
 * gf_buffer(i) / gf_buffer_bytes(i). */
#define GF_BUF_IN 1u
#define GF_BUF_OUT 2u
typedef struct gf_buf {
    void *ptr;
    uint64_t bytes;
    uint32_t dir;
    uint32_t pad;
} gf_buf;

/* Counters of the last program waited for on this context (host fields
 * accumulate over the context's life). */
#define GF_NOPS 16
/* Built-in opcodes, the index of rpc_calls / rpc_slots: 1 printf / fprintf,
 * 2 fopen, 3 fwrite, 4 fclose, 5 clock, 6 getenv, 7 fread, 8 fflush,
 * 9 strtod (the device's slow path), 10 region launch (kernel split only). */
typedef struct gf_stats {
    uint64_t rpc_calls[GF_NOPS];  /* lane records per opcode (index = GF_OP_*)               */
    uint64_t rpc_slots[GF_NOPS];  /* ring slots per opcode (calls / slots = aggregation)    */
    uint64_t rpc_wait_ns;         /* device time leaders spent waiting for the host        */
    double rpc_p50_ns;            /* device round-trip latency percentiles (claim -> done) of
                                     calls whose caller waited (not deferred printf)        */
    double rpc_p99_ns;
    uint64_t regions;             /* parallel regions run                                   */
    uint64_t region_ns;           /* device time inside regions (publish -> all blocks done) */
    uint64_t heap_alloc, heap_free, heap_fail, heap_bad_free;
    uint64_t heap_live_bytes, heap_high_water;
    uint64_t main_ns;             /* device time from main() entry to return               */
    uint64_t host_slots;          /* slots the host served (cumulative)                    */
    uint64_t host_records;        /* lane records the host served (cumulative)             */
    uint64_t host_ns;             /* host time inside landing pads (cumulative)            */
    uint64_t host_dma_bytes;      /* bytes moved by DMA for fwrite/fread (cumulative)      */
    int32_t grid, block;          /* launch shape of the last program                      */
    int32_t error;                /* first device-side error of the last program           */
    int32_t exit_code;
    uint64_t heap_ns;             /* the initial thread's time inside malloc / free        */
    uint64_t copy_regions;        /* regions that moved large fwrite/fread data through the
                                     bulk arena (included in regions)                      */
    uint64_t copy_ns;             /* their device time (included in region_ns)             */
    uint64_t host_ring_bytes;     /* ring bytes the host served: records written by the device,
                                     8-byte returns read back (cumulative)                  */
    uint64_t t_start_ns, t_end_ns;/* device %globaltimer at main's entry and return (one clock
                                     for all programs on the device: intervals can be compared) */
    uint64_t heap_quota;          /* heap bytes the program was admitted with              */
    uint64_t ring_quota;          /* ring slots the program was admitted with              */
    uint64_t rpc_wait_op_ns[GF_NOPS]; /* rpc_wait_ns split by opcode                        */
    uint64_t rpc_client_ns;       /* the initial thread's time inside RPC calls outside the
                                     waits (packing, slot claim, publication, collection)   */
} gf_stats;

/* Host landing pad for a user opcode (>= 256).  `rec` points at the lane
 * record (layout in gf_layout.h: gf_rec_hdr, tags, words, tail); the return
 * value is handed back to the calling lane.  Write-mode reference arguments
 * may be modified in place in the record's tail; they are copied back. */
typedef int64_t (*gf_host_fn)(void *user, uint32_t opcode, void *rec);

typedef struct gf_serve_opts {
    int64_t timeout_ns;           /* return GF_ETIMEDOUT after this long (<= 0: no limit)   */
    volatile int32_t *stop;       /* return GF_OK when *stop becomes nonzero (may be NULL)  */
} gf_serve_opts;

/* ------------------------------------------------------------------ lifecycle */

/* Fill *cfg with the defaults listed in gf_config. */
GF_API void gf_config_default(gf_config *cfg);

/* Create a context on the configured device: device heap arenas, the pinned
 * and device-mapped RPC ring, per-instance program state, DMA staging and the
 * host server threads.  cfg may be NULL (defaults).  *out receives the
 * context.  Errors: GF_EINVAL (bad sizes), GF_ENOMEM, GF_ECUDA. */
GF_API int gf_init(const gf_config *cfg, gf_ctx **out);

/* Stop the server threads, close files the programs left open, free all
 * context memory.  Programs still running are waited for first.  NULL is a
 * no-op returning GF_OK. */
GF_API int gf_finalize(gf_ctx *ctx);

/* Registry id of the program registered as GF_MAIN(name).  GF_ENOENT if none. */
GF_API int gf_program_lookup(gf_ctx *ctx, const char *name, gf_program *out);

/* ------------------------------------------------------------------ running programs */

/* The loader (paper Sec. 3.1: map argv to the device, start the RPC server,
 * call main on the GPU): copy argv (and host buffers marked GF_BUF_IN) to the
 * device, launch the program's persistent cooperative grid on cfg.stream,
 * serve its RPCs until main returns, copy GF_BUF_OUT host buffers back and
 * store main's return value in *exit_code.  Blocking.  argv strings are copied
 * (at most 64 KiB in total); bufs may be NULL when nbufs is 0 (at most 16).
 * Returns GF_OK, or the first device error (GF_ETIMEDOUT, GF_ERING, ...),
 * GF_EBUSY when every instance is taken, GF_ECUDA on a launch failure. */
GF_API int gf_run_main(gf_ctx *ctx, gf_program prog, int argc, const char *const *argv,
                       const gf_buf *bufs, int nbufs, int *exit_code);

/* Asynchronous launch for serving and batching: like gf_run_main up to the
 * kernel launch, on `stream` (NULL = cfg.stream) with `grid` blocks (0 = the
 * configured share), with the default heap and ring quotas.  *h receives the
 * handle.  GF_EBUSY when the program cannot be admitted now. */
GF_API int gf_launch(gf_ctx *ctx, gf_program prog, int argc, const char *const *argv,
                     const gf_buf *bufs, int nbufs, void *stream, uint32_t grid, gf_handle **h);

/* gf_launch with explicit quotas (q may be NULL = defaults).  Admission by
 * ring and heap memory: the program starts only when a free instance, its
 * heap quota (from the context's heap pool) and its ring quota (from the ring
 * pool) are all available; otherwise nothing is taken and GF_EBUSY returns,
 * and the caller retries after a running program has been collected with
 * gf_wait.  GF_EINVAL when a quota exceeds its whole pool (it could never be
 * admitted) or the ring quota is not a power of two. */
GF_API int gf_launch_q(gf_ctx *ctx, gf_program prog, int argc, const char *const *argv,
                       const gf_buf *bufs, int nbufs, void *stream, uint32_t grid, const gf_quota *q,
                       gf_handle **h);

/* 1 if the program behind h has finished (its kernel completed), else 0. */
GF_API int gf_done(gf_handle *h);

/* Wait for the program behind h (serving its RPCs when the context has no
 * server threads), copy back GF_BUF_OUT host buffers, release the instance and
 * free h.  timeout_ns <= 0 waits without limit; on GF_ETIMEDOUT h stays valid. */
GF_API int gf_wait(gf_handle *h, int *exit_code, int64_t timeout_ns);

/* Serve RPCs of all running programs in the calling thread until none is
 * running, *opts->stop becomes nonzero, or the timeout passes. */
GF_API int gf_rpc_serve(gf_ctx *ctx, const gf_serve_opts *opts);

/* Register a host landing pad for opcode >= 256 (device: gf_rpc(opcode, ...)). */
GF_API int gf_rpc_register(gf_ctx *ctx, uint32_t opcode, gf_host_fn fn, void *user);

/* Inside a landing pad: argument k of the lane record `rec`.  *tag gets the
 * argument kind ('i','u','l','L','d' integers and doubles, 'p' an opaque value
 * such as FILE*, 's' string, 'b' / 'w' / 'x' a read / write / readwrite
 * reference), *word its 8-byte value.  For references (paper Sec. 3.2,
 * Fig. 4) the whole underlying object was copied into the record: *ptr
 * points into that host copy at the argument's offset, *bytes is the
 * object's size and *off the offset; write and readwrite objects are copied
 * back to the device after the pad returns.  Any output pointer may be NULL.
 * Returns 0, or -1 when k is out of range. */
GF_API int gf_rec_arg(const void *rec, int k, uint8_t *tag, uint64_t *word, void **ptr, uint32_t *bytes,
                      uint32_t *off);

/* Counters of the last program waited for (see gf_stats). */
GF_API int gf_get_stats(gf_ctx *ctx, gf_stats *out);

/* Static message for an error code. */
GF_API const char *gf_strerror(int err);

/* ------------------------------------------------------------------ batching */

/* Graph form of a batch of independent loops (the paper's kernel split, Sec.
 * 3.3 and Fig. 3, where each parallel region becomes a multi-team kernel the
 * host launches): n axpy loops z[off_k + i] = a_k * x[off_k + i] +
 * y[off_k + i], i < trips[k], become one CUDA graph with one kernel node per
 * loop (no edges, so loops may overlap), each with grid[k] x block[k] threads
 * (either array may be NULL: 256 threads, enough blocks to cover the loop up
 * to 8 per SM).  x, y, z are device arrays; trips, a, off, grid, block are
 * host arrays of n entries.  The graph is built, replayed once to warm up,
 * then `reps` times on `stream`; *ms receives the mean milliseconds per
 * replay.  Errors: GF_EINVAL, GF_ECUDA. */
GF_API int gf_axpy_batch_graph(int n, const int64_t *trips, const double *a, const int64_t *off, const double *x,
                               const double *y, double *z, const uint32_t *grid, const uint32_t *block, int reps,
                               void *stream, float *ms);

/* The graph form of loops that call libc (the loops_rpc program's body):
 * loop k computes z[off_k + i] = a_k * x[off_k + i] + y[off_k + i] for
 * i < trips[k], and every 4096th iteration passes the value through a device
 * heap block of 64 << (k % 8) bytes and prints "k i value" by RPC.  One CUDA
 * graph with one kernel node per loop, each with grid[k] x block[k] threads
 * (either array may be NULL: 256 threads, enough blocks to cover the loop up
 * to 8 per SM; block a multiple of 32, <= 256: the device heap's per-block
 * hand-off area holds 8 warps).  A program instance of ctx
 * (its heap quota and ring; answered by the context's server threads, at
 * least one) is borrowed for the call.  `warmup` untimed replays, then `reps`
 * timed ones on `stream`; *ms (may be NULL) = mean ms per timed replay.
 * Every replay prints its lines again.  x, y, z and fails (uint64 count of
 * heap blocks not granted or corrupted) are device memory; trips, a, off,
 * grid, block are host arrays of n entries.  Errors: GF_EINVAL, GF_EBUSY,
 * GF_ECUDA, or a device error of the loops' calls. */
GF_API int gf_loops_rpc_graph(gf_ctx *ctx, int n, const int64_t *trips, const double *a, const int64_t *off,
                              const double *x, const double *y, double *z, unsigned long long *fails,
                              const uint32_t *grid, const uint32_t *block, int warmup, int reps, void *stream,
                              float *ms);

/* ------------------------------------------------------------------ launch-shape tuning */

/* A synthetic legacy loop (the learned-model workload): per iteration it reads
 * `bytes` (8..4096, multiple of 8) as bytes/8 coalesced FP64 streams of x,
 * runs a dependent chain of `flops` FP32 FMAs, a second chain when the
 * iteration's hash falls below div_thresh (divergent branch; fraction =
 * div_thresh / 2^32), calls clock() on the host by RPC when another hash
 * falls below rpc_thresh (rate = rpc_thresh / 2^32), and writes z[i]. */
typedef struct gf_synth_loop {
    int64_t trip;
    uint32_t bytes, flops;
    uint32_t div_thresh, rpc_thresh;
    uint64_t seed;
} gf_synth_loop;

/* A launch shape: grid x block threads (block a multiple of 32, <= 1024);
 * warps take work items of `chunk` iterations, sched GF 0 = round robin,
 * 1 = shared counter. */
typedef struct gf_shape {
    uint32_t grid, block, chunk, sched;
} gf_shape;

/* Run loop L once with shape *sh (x: device, >= trip * bytes/8 doubles of
 * xlen; z: device, >= trip doubles).  Borrows a program instance of ctx for
 * the loop's RPCs; waits for completion.  Errors: GF_EINVAL (bad loop or
 * shape, x too short, RPCs without server threads), GF_EBUSY, GF_ECUDA, or a
 * device error (GF_ETIMEDOUT, GF_ERING). */
GF_API int gf_synth_run(gf_ctx *ctx, const gf_synth_loop *L, const double *x, uint64_t xlen, double *z,
                        const gf_shape *sh, void *stream);

/* Time loop L under nshapes shapes: per shape one warm-up run and `reps`
 * timed runs (CUDA events on `stream`); ms[s] = the fastest, in ms. */
GF_API int gf_synth_time(gf_ctx *ctx, const gf_synth_loop *L, const double *x, uint64_t xlen, double *z,
                         const gf_shape *shapes, int nshapes, int reps, void *stream, float *ms);

/* The model's input features of (loop, shape), written to out[GF_TUNE_NFEAT]:
 * log2 trip, log2 bytes, log2 flops, divergent fraction, 1000 x RPC rate,
 * log2(grid / sms), log2 block, log2 chunk, sched.  Host only; training and
 * inference both use this function, so they cannot disagree. */
#define GF_TUNE_NFEAT 9
GF_API void gf_tune_features(const gf_synth_loop *L, const gf_shape *sh, uint32_t sms, float *out);

/* FP32 MLP forward pass on the host: normalise each of the nin inputs with
 * (x - mean) / std, `depth` hidden layers of `width` ReLU units, one linear
 * output.  params = mean[nin], std[nin], then per hidden layer W (width x in,
 * row major) and b[width], then w_out[width], b_out.  x is n x nin, y gets n
 * outputs.  Returns GF_EINVAL for bad sizes. */
GF_API int gf_mlp_forward(const float *params, int nin, int width, int depth, const float *x, int n, float *y);

/* Learned launch shape: the index of the shape with the smallest predicted
 * log-time for loop L among shapes[0..nshapes) (the model predicts log
 * milliseconds from gf_tune_features).  Writes it to *best. */
GF_API int gf_mlp_choose(const float *params, int width, int depth, const gf_synth_loop *L, const gf_shape *shapes,
                         int nshapes, uint32_t sms, int *best);

/* The k shapes with the smallest predicted times, fastest first, in idx[k]:
 * the candidates a tuner times when it refines the model's choice with k
 * measured runs instead of measuring every shape. */
GF_API int gf_mlp_topk(const float *params, int width, int depth, const gf_synth_loop *L, const gf_shape *shapes,
                       int nshapes, uint32_t sms, int k, int *idx);

/* ------------------------------------------------------------------ allocator experiment */

/* The paper's allocator stress (Sec. 5.1, Fig. 6): `teams` blocks of
 * `threads` (<= 256) threads; every thread allocates `bytes` at kernel start,
 * writes and reads its block, and frees it.  kind: 0 = the runtime's slab
 * heap, 1 = the paper's balanced allocator (N = 32 thread slots x M = 16
 * team slots, first chunk 4x larger), 2 = the paper's generic allocator (two
 * lists under one lock), 3 = CUDA's device malloc (its heap limit is raised
 * to 1 GiB on first use, which must precede any other kernel that calls
 * malloc).  The paper's allocators use the heap arena of a borrowed program
 * instance.  After one warm-up launch, `reps` launches are timed on `stream`;
 * *ms = mean kernel time, *fails = NULL returns in the last launch (low 32
 * bits) plus 2^32 x corrupted blocks.  Errors: GF_EINVAL, GF_EBUSY, GF_ECUDA. */
GF_API int gf_alloc_e1(gf_ctx *ctx, int kind, uint32_t teams, uint32_t threads, uint32_t bytes, int reps,
                       void *stream, float *ms, uint64_t *fails);

/* The FP64 add throughput of the current device, for the roofline of FP64-bound
 * loops (the Jacobi sweep).  A kernel of `blocks` x 256 threads (0 = SMs x
 * resident blocks), each running eight independent chains of `iters`
 * correctly rounded FP64 adds, runs once to warm up and once timed with CUDA
 * events on `stream`.  *ms = the timed run, *adds = FP64 adds it issued
 * (thread count x iters x 8), so *adds / *ms is the measured rate at the
 * clock the GPU ran during the call.  Errors: GF_EINVAL, GF_ECUDA. */
GF_API int gf_fp64_add_rate(uint32_t blocks, int64_t iters, void *stream, float *ms, double *adds);

/* Number of SMs and resident blocks per SM that a program's grid uses at
 * `block` threads (for sizing, tests and roofline accounting). */
GF_API int gf_grid_info(gf_ctx *ctx, gf_program prog, uint32_t *sms, uint32_t *blocks_per_sm);

/* ------------------------------------------------------------------ allocation-free reduction */

/* The paper has no counterpart to this entry point; it is an addition for
 * callers that may not allocate device memory at all (code running under
 * another framework's fixed memory budget or inside its allocator, code that
 * must not change the device's footprint, or a one-off reduction that cannot
 * pay for a gf_ctx, which reserves a heap arena, a pinned ring and state).
 *
 * *out (device) = op over x[0 .. n) (device FP64), op one of GF_REDUCE_SUM,
 * GF_REDUCE_MIN, GF_REDUCE_MAX, computed by the same reduction a gf_reduce
 * region uses (compensated per-thread sums, warp / block trees, one partial
 * per block; the last block merges the partials with a strided per-thread
 * pass and the same warp / block trees), launched on `stream` (cudaStream_t,
 * NULL = legacy default) and not waited for.  blocks = 0 picks SMs x
 * resident blocks; at most 2048 blocks (larger: GF_EINVAL).  n = 0 stores
 * the identity (0, +inf, -inf).  MIN and MAX are exact.  A SUM is the same
 * bits on every run with the same `blocks`; the default grid differs between
 * GPU models, so pass `blocks` to get identical bits everywhere.
 *
 * Nothing is allocated: the per-block partials live in one static device
 * array of 32 KiB + 256 B inside this library, present on every GPU that
 * loads it until the process exits.  All calls share that array and it keeps
 * the last call's contents; the ticket that must start at zero is cleared
 * before each launch.  Calls that overlap on the GPU race on the array: do
 * not run two at once.  The first call on each device looks the array's
 * address up (cudaGetSymbolAddress, with that device current) and caches it.
 * Errors: GF_EINVAL (bad op, n < 0, NULL pointers, too many blocks),
 * GF_ECUDA (lookup, ticket clear or launch failed).  A CUDA error left
 * pending by the caller's earlier work is not read or cleared. */
#define GF_REDUCE_SUM 1
#define GF_REDUCE_MIN 2
#define GF_REDUCE_MAX 3
GF_API int gf_reduce_f64_noalloc(const double *x, int64_t n, int op, double *out, uint32_t blocks, void *stream);

#ifdef __cplusplus
}
#endif
#endif
