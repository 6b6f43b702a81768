/*
 * GPU-First device runtime for sm_103a (header-only; include it in the .cu file
 * that defines a program with GF_MAIN).
 *
 * Execution model (the paper's Sec. 2.1 and Sec. 3.3, Fig. 3): a program's
 * serial part runs on ONE initial thread; its parallel regions are workshared
 * over the threads of ALL blocks with continuous thread ids, and a barrier
 * spans all blocks.  The paper realises this with a 1-thread main kernel that
 * asks the host (by RPC) to launch a multi-team kernel per region.  Here one
 * cooperative, persistent grid (SMs x resident blocks) is launched once:
 *   - block 0, lane 0 of warp 0 is the initial thread and runs main();
 *     lanes 1..31 of that warp retire at start;
 *   - every other warp is a worker that waits in a state machine (the paper's
 *     generic-mode worker loop, Sec. 3.3) on an epoch word, runs the published
 *     region through a trampoline, and reports completion per block;
 *   - no host round trip per region: a region costs one release store, one
 *     acquire poll per block and one counter increment per block.
 *
 * Reductions (sum/min/max over double and int64) extend the paper, which does
 * not rewrite reduction clauses (Sec. 4.3): per-thread accumulation (Neumaier
 * compensation for double sums) -> xor-shuffle warp tree -> shared-memory
 * block tree -> one partial per block -> the last block to finish combines all
 * partials in block-index order.  For a fixed grid the result is the same on
 * every run.
 *
 * Every wait is bounded by %globaltimer against gf_state.timeout_ns and ends
 * with an error status (GF_ETIMEDOUT / GF_ERING); nothing here traps.
 */
#ifndef GF_DEVICE_CUH
#define GF_DEVICE_CUH

#include <stdint.h>
#include <cuda_runtime.h>
#include <type_traits>
#include "gf_layout.h"
#include "gf_errors.h"

#ifndef GF_BLOCK
#define GF_BLOCK 256
#endif
/* default minimum resident blocks per SM a program's persistent kernel is
 * compiled for: 4 (at most 64 registers).  A legacy loop streams from HBM
 * with as many loads in flight as the SM holds warps: one axpy region over
 * 2^28 doubles reached 45% of the measured copy peak at the 2 blocks per SM
 * the compiler's own register choice left, 76% at 4 and 85% at 8 (90% at 4
 * with 16-byte accesses).  Programs ask for another count with
 * GF_MAIN_BOUNDS(name, n): the batched loops use 8. */
#ifndef GF_MIN_BLOCKS
#define GF_MIN_BLOCKS 4
#endif
#define GF_MAX_WARPS (GF_BLOCK / 32)

typedef uint64_t GF_FILE;   /* opaque host FILE* (paper Sec. 3.2: never dereferenced on the device) */

namespace gfd {

/* ------------------------------------------------------------ per-block state */
__shared__ gf_state *s_st;                 /* this program's state                     */
__shared__ uint32_t s_epoch;               /* epoch seen by this block's poller         */
__shared__ uint32_t s_last;                /* this block combines the reduction         */
__shared__ uint32_t s_abort;               /* this block's workers give up (idle bound) */
__shared__ uint32_t s_kr;                  /* 1 outside a program's persistent kernel (a
                                              region kernel of the split, a standalone
                                              kernel): every thread is a worker, none is
                                              the initial thread, ids have no offset   */
__shared__ uint64_t s_red[GF_MAX_WARPS][2];/* per-warp reduction partials               */
__shared__ uint64_t s_xfer[GF_MAX_WARPS][32]; /* per-warp lane hand-off (heap, rpc)    */
/* the initial thread's own bookkeeping, kept in its block's shared memory so
 * that its serial part pays no global-memory round trip for it: */
__shared__ uint32_t s_done_target;         /* blocks done when the current region ends   */
__shared__ uint32_t s_main_epoch;          /* the last epoch the initial thread published */
__shared__ unsigned long long s_pend_t1;   /* deferred call: ticket + 1, 0 = none        */
__shared__ unsigned long long s_pend_key;  /* ... and the format it shipped (0: none)    */
__shared__ unsigned long long s_done_t1;   /* last deferred call collected with its value */
__shared__ long long s_done_val;
__shared__ unsigned long long s_known_key; /* a format the host is known to have         */
/* printf records of the initial thread waiting to share one ring slot (the
 * stdio buffer of the serial part): the records, their count and bytes, the
 * format they share and whether it ships with them, and the sequence numbers
 * that name each buffered call */
#define GF_PBUF_WORDS 128
__shared__ uint64_t s_pb[GF_PBUF_WORDS];
__shared__ uint32_t s_pb_n, s_pb_bytes, s_pb_fbytes, s_pend_n;
__shared__ unsigned long long s_pb_key;    /* format (device address) of the buffered records */
__shared__ const char *s_pb_fmt;
__shared__ unsigned long long s_pb_seq;    /* sequence number of the next buffered call        */
__shared__ unsigned long long s_pend_seq0; /* first sequence number in the pending slot, 0: one
                                              unbuffered call                                 */

/* how long the initial thread polls a region's end without sleeping, and
 * the workers poll for the next region with short sleeps */
#define GF_REGION_SPIN_NS 20000u

/* ------------------------------------------------------------ PTX helpers */
__device__ __forceinline__ uint64_t now_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ uint32_t ld_acq_gpu(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_rel_gpu(uint32_t *p, uint32_t v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_acq_sys64(const uint64_t *p)
{
    uint64_t v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_rel_sys64(uint64_t *p, uint64_t v)
{
    asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_vol64(const uint64_t *p)
{
    uint64_t v;
    asm volatile("ld.volatile.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void bar_workers(uint32_t n)
{
    asm volatile("bar.sync 1, %0;" ::"r"(n) : "memory");
}
__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}
__device__ __forceinline__ uint32_t smid()
{
    uint32_t s;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(s));
    return s;
}

__device__ __forceinline__ gf_state *st() { return s_st; }

/* Thread 0 of every block of a kernel that uses the device runtime: the
 * program's state, and whether this is a program's persistent kernel
 * (kr = 0) or another kernel whose threads are all workers (kr = 1).
 * Followed by __syncthreads() in the caller. */
__device__ __forceinline__ void block_setup(gf_state *S, uint32_t kr)
{
    s_st = S;
    s_kr = kr;
    s_done_target = 0;
    s_main_epoch = 0;                         /* the state's epoch starts at 0 each launch */
    s_pend_t1 = 0;
    s_pend_key = 0;
    s_done_t1 = 0;
    s_done_val = -1;
    s_known_key = 0;
    s_pb_n = 0;
    s_pb_bytes = 0;
    s_pb_fbytes = 0;
    s_pend_n = 0;
    s_pb_key = 0;
    s_pb_fmt = nullptr;
    s_pb_seq = 1;
    s_pend_seq0 = 0;
}
__device__ __forceinline__ bool is_initial_thread() { return blockIdx.x == 0 && threadIdx.x == 0 && !s_kr; }

__device__ __forceinline__ void set_error(int e)
{
    atomicCAS((int *)&s_st->error, 0, e);
}

/* bounded spin helper: returns false on timeout */
struct backoff {
    uint64_t t0, limit;
    uint32_t ns;
    __device__ backoff(int64_t limit_ns) : t0(now_ns()), limit((uint64_t)limit_ns), ns(32) {}
    __device__ bool wait()
    {
        __nanosleep(ns);
        if (ns < 512)
            ns <<= 1;
        return now_ns() - t0 < limit;
    }
};

/* ------------------------------------------------------------ worker context */
struct wctx {
    int64_t tid;        /* continuous worker id: 0 .. nthreads-1                       */
    int64_t nthreads;
    uint32_t nbar;      /* worker threads in this block (named barrier count)          */
    uint32_t wfirst;    /* first worker warp of this block (1 in block 0, else 0)      */
    bool poller;        /* first worker thread of this block                           */
};

__device__ __forceinline__ wctx make_wctx()
{
    wctx w;
    if (s_kr) {                 /* region kernel: every thread of every block is a worker */
        w.tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        w.nthreads = (int64_t)gridDim.x * blockDim.x;
        w.nbar = blockDim.x;
        w.wfirst = 0;
        w.poller = threadIdx.x == 0;
        return w;
    }
    const bool b0 = blockIdx.x == 0;
    w.tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - 32;
    w.nthreads = (int64_t)gridDim.x * blockDim.x - 32;
    w.nbar = blockDim.x - (b0 ? 32u : 0u);
    w.wfirst = b0 ? 1u : 0u;
    w.poller = threadIdx.x == (b0 ? 32u : 0u);
    return w;
}

typedef void (*tramp_t)(const gf_region *, const wctx &);

} // namespace gfd

/* ====================================================================== thread ids */
/* Continuous ids across all blocks inside a region (paper Sec. 3.3, Fig. 3);
 * outside a region the initial thread is thread 0 of a team of 1. */
__device__ __forceinline__ int64_t gf_thread_num()
{
    if (gfd::is_initial_thread())
        return 0;
    return (int64_t)blockIdx.x * blockDim.x + threadIdx.x - (gfd::s_kr ? 0 : 32);
}
__device__ __forceinline__ int64_t gf_num_threads()
{
    if (gfd::is_initial_thread())
        return 1;
    return (int64_t)gridDim.x * blockDim.x - (gfd::s_kr ? 0 : 32);
}

/* ====================================================================== reductions */
namespace gfd {

template <class T, int OP> struct acc;

/* double sum: Neumaier compensated accumulation, double-double combine */
template <> struct acc<double, GF_RED_SUM> {
    double s, c;
    __device__ acc() : s(0.0), c(0.0) {}
    __device__ void add(double x)
    {
        double t = __dadd_rn(s, x);
        if (fabs(s) >= fabs(x))
            c = __dadd_rn(c, __dadd_rn(__dadd_rn(s, -t), x));
        else
            c = __dadd_rn(c, __dadd_rn(__dadd_rn(x, -t), s));
        s = t;
    }
    __device__ void merge(const acc &o)
    {
        double t = __dadd_rn(s, o.s);
        double bp = __dadd_rn(t, -s);
        double e = __dadd_rn(__dadd_rn(s, -__dadd_rn(t, -bp)), __dadd_rn(o.s, -bp));  /* TwoSum error */
        s = t;
        c = __dadd_rn(__dadd_rn(c, o.c), e);
    }
    __device__ double result() const { return __dadd_rn(s, c); }
    __device__ void to_words(uint64_t *w) const { w[0] = __double_as_longlong(s); w[1] = __double_as_longlong(c); }
    __device__ void from_words(const uint64_t *w) { s = __longlong_as_double(w[0]); c = __longlong_as_double(w[1]); }
    __device__ acc shfl_xor(int m) const
    {
        acc r;
        r.s = __shfl_xor_sync(0xffffffffu, s, m);
        r.c = __shfl_xor_sync(0xffffffffu, c, m);
        return r;
    }
};

/* double min / max on the integer pipe: flipping the magnitude bits of
 * negative values makes the signed 64-bit order of the bit patterns equal to
 * the IEEE order (with -0 < +0), so no FP64 instruction is spent per element
 * (GB300 issues FP64 at a small fraction of its integer rate).  NaNs are
 * skipped, as `if (x > m) m = x` skips them.  Between -0 and +0 max returns
 * +0 and min returns -0, either of which the unordered reduction allows. */
__device__ __forceinline__ long long f64_key(double x)
{
    const long long b = __double_as_longlong(x);
    return b ^ ((b >> 63) & 0x7fffffffffffffffll);
}
template <int OP> struct acc<double, OP> {
    long long k;
    __device__ acc() : k(OP == GF_RED_MIN ? 0x7ff0000000000000ll : (long long)0x800fffffffffffffull) {}
    __device__ void add_key(long long x) { k = OP == GF_RED_MIN ? (x < k ? x : k) : (x > k ? x : k); }
    __device__ void add(double x)
    {
        const long long b = __double_as_longlong(x);
        if ((b & 0x7fffffffffffffffll) <= 0x7ff0000000000000ll)      /* not a NaN */
            add_key(b ^ ((b >> 63) & 0x7fffffffffffffffll));
    }
    __device__ void merge(const acc &o) { add_key(o.k); }
    __device__ double result() const { return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffll)); }
    __device__ void to_words(uint64_t *w) const { w[0] = (uint64_t)k; w[1] = 0; }
    __device__ void from_words(const uint64_t *w) { k = (long long)w[0]; }
    __device__ acc shfl_xor(int m) const
    {
        acc r;
        r.k = __shfl_xor_sync(0xffffffffu, k, m);
        return r;
    }
};

template <int OP> struct acc<long long, OP> {
    long long v;
    __device__ acc() : v(OP == GF_RED_SUM ? 0ll : OP == GF_RED_MIN ? 0x7fffffffffffffffll : (-0x7fffffffffffffffll - 1)) {}
    __device__ void add(long long x)
    {
        if (OP == GF_RED_SUM)
            v = (long long)((unsigned long long)v + (unsigned long long)x);   /* wraps like two's complement */
        else if (OP == GF_RED_MIN ? (x < v) : (x > v))
            v = x;
    }
    __device__ void merge(const acc &o) { add(o.v); }
    __device__ long long result() const { return v; }
    __device__ void to_words(uint64_t *w) const { w[0] = (uint64_t)v; w[1] = 0; }
    __device__ void from_words(const uint64_t *w) { v = (long long)w[0]; }
    __device__ acc shfl_xor(int m) const
    {
        acc r;
        r.v = __shfl_xor_sync(0xffffffffu, v, m);
        return r;
    }
};

template <class A> __device__ __forceinline__ A warp_tree(A a)
{
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1)
        a.merge(a.shfl_xor(m));
    return a;
}

/* block + grid combine; every worker thread of the block calls this */
template <class A> __device__ void finish_reduce(A a, const wctx &w)
{
    gf_state *S = s_st;
    const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
    const uint32_t nw = w.nbar >> 5;
    a = warp_tree(a);
    if (lane == 0)
        a.to_words(s_red[warp]);
    bar_workers(w.nbar);
    if (warp == w.wfirst) {
        A b;
        if (lane < nw)
            b.from_words(s_red[w.wfirst + lane]);
        b = warp_tree(b);
        if (lane == 0) {
            uint64_t *part = (uint64_t *)S->partials + 2 * blockIdx.x;
            uint64_t wd[2];
            b.to_words(wd);
            part[0] = wd[0];
            part[1] = wd[1];
            __threadfence();
            uint32_t t = atomicAdd(&S->red_ticket, 1u);
            s_last = (t == gridDim.x - 1) ? 1u : 0u;
        }
    }
    bar_workers(w.nbar);
    if (s_last) {
        __threadfence();
        const uint64_t *part = (const uint64_t *)S->partials;
        A c;
        const uint32_t idx = threadIdx.x - w.wfirst * 32;
        for (uint32_t k = idx; k < gridDim.x; k += w.nbar) {
            A p;
            uint64_t wd[2] = {ld_vol64(part + 2 * k), ld_vol64(part + 2 * k + 1)};
            p.from_words(wd);
            c.merge(p);
        }
        c = warp_tree(c);
        if (lane == 0)
            c.to_words(s_red[warp]);
        bar_workers(w.nbar);
        if (warp == w.wfirst) {
            A d;
            if (lane < nw)
                d.from_words(s_red[w.wfirst + lane]);
            d = warp_tree(d);
            if (lane == 0)
                d.to_words(S->red_result);
        }
    }
}

/* ------------------------------------------------------------ schedules */
template <class F> __device__ __forceinline__ void run_schedule(const gf_region *rd, const wctx &w, F &f)
{
    const int64_t b = rd->b, e = rd->e, c = rd->chunk;
    if (rd->sched == GF_SCHED_STATIC) {
        if (c == 1) {
            /* two iterations in flight per thread: their dependent chains of
             * long-latency operations (FP64, loads) overlap */
#pragma unroll 2
            for (int64_t i = b + w.tid; i < e; i += w.nthreads)
                f(i);
        } else if (c <= 0) {                       /* OpenMP default: one contiguous block each */
            const int64_t n = e - b, per = (n + w.nthreads - 1) / w.nthreads;
            const int64_t lo = b + w.tid * per;
            const int64_t hi = lo + per < e ? lo + per : e;
            for (int64_t i = lo; i < hi; i++)
                f(i);
        } else {                                   /* chunks of c, round robin over threads */
            for (int64_t base = b + w.tid * c; base < e; base += w.nthreads * c) {
                const int64_t hi = base + c < e ? base + c : e;
                for (int64_t i = base; i < hi; i++)
                    f(i);
            }
        }
    } else {                                       /* dynamic: one atomic per warp grabs 32 chunks */
        const int64_t cc = c > 0 ? c : 1;
        const uint32_t lane = lane_id();
        for (;;) {
            unsigned long long base = 0;
            if (lane == 0)
                base = atomicAdd(&s_st->dyn_next, 32ull * (unsigned long long)cc);
            base = __shfl_sync(0xffffffffu, base, 0);
            if (b + (int64_t)base >= e)
                break;
            const int64_t lo = b + (int64_t)base + (int64_t)lane * cc;
            const int64_t hi = lo + cc < e ? lo + cc : e;
            for (int64_t i = lo; i < hi; i++)
                f(i);
        }
    }
}

template <class F> __device__ void tramp_for(const gf_region *rd, const wctx &w)
{
    F f = *reinterpret_cast<const F *>(rd->body);
    run_schedule(rd, w, f);
}

template <class T, int OP, class F> __device__ void tramp_reduce(const gf_region *rd, const wctx &w)
{
    F f = *reinterpret_cast<const F *>(rd->body);
    acc<T, OP> a;
    auto g = [&](int64_t i) { a.add((T)f(i)); };
    run_schedule(rd, w, g);
    finish_reduce(a, w);
}

/* The common case on its own: static schedule, chunk 1, fewer than 2^31
 * iterations.  A trampoline holding only this loop, with a 32-bit induction
 * variable (k + nthreads stays below 2^32), needs fewer registers than one
 * holding every schedule, which keeps a register-hungry body free of spill
 * reloads inside its loop. */
__device__ __forceinline__ bool static1_fits(int sched, int64_t chunk, int64_t b, int64_t e)
{
    return sched == GF_SCHED_STATIC && chunk == 1 && e - b < (int64_t)0x7fffffff;
}

template <class G> __device__ __forceinline__ void run_static1(const gf_region *rd, const wctx &w, G &g)
{
    const int64_t b = rd->b;
    const uint32_t n = (uint32_t)(rd->e - b), nth = (uint32_t)w.nthreads;
#pragma unroll 2
    for (uint32_t k = (uint32_t)w.tid; k < n; k += nth)
        g(b + (int64_t)k);
}

template <class F> __device__ void tramp_for_s1(const gf_region *rd, const wctx &w)
{
    F f = *reinterpret_cast<const F *>(rd->body);
    run_static1(rd, w, f);
}

template <class T, int OP, class F> __device__ void tramp_reduce_s1(const gf_region *rd, const wctx &w)
{
    F f = *reinterpret_cast<const F *>(rd->body);
    acc<T, OP> a;
    auto g = [&](int64_t i) { a.add((T)f(i)); };
    run_static1(rd, w, g);
    finish_reduce(a, w);
}

/* ------------------------------------------------------------ region launch (initial thread) */
/* kernel split: ask the host to launch the region kernel; its grid, or < 0 */
static __device__ int64_t split_launch(gf_state *S, int *status);

/* err: the program's error word, read by the caller before it wrote the
 * region's descriptor (the read's round trip overlaps those stores) */
static __device__ __noinline__ int run_region(gf_state *S, int32_t err)
{
    if (err)                                  /* after a timeout the workers may still be busy */
        return err;
    atomicAdd((unsigned long long *)&S->st_regions, 1ull);   /* no result needed: no round trip */
    if (S->split) {
        /* the paper's kernel split (Sec. 3.3, Fig. 3): one RPC per region, on
         * which the host launches the region as its own kernel; the initial
         * thread then waits for that kernel's blocks to finish */
        S->dyn_next = 0;
        S->red_ticket = 0;
        const uint64_t t0 = now_ns();
        __threadfence();
        int st = GF_OK;
        const int64_t grid = split_launch(S, &st);
        if (st != GF_OK || grid <= 0) {
            set_error(st != GF_OK ? st : GF_ECUDA);
            return S->error;
        }
        const uint32_t target = s_done_target + (uint32_t)grid;
        s_done_target = target;
        backoff bo(S->timeout_ns);
        while ((int32_t)(ld_acq_gpu(&S->done_blocks) - target) < 0) {
            if (now_ns() - t0 < GF_REGION_SPIN_NS)
                continue;
            if (!bo.wait()) {
                set_error(GF_ETIMEDOUT);
                return GF_ETIMEDOUT;
            }
        }
        atomicAdd((unsigned long long *)&S->st_region_ns, (unsigned long long)(now_ns() - t0));
        return GF_OK;
    }
    const uint32_t target = s_done_target + S->nblocks;
    s_done_target = target;
    S->dyn_next = 0;
    S->red_ticket = 0;
    const uint64_t t0 = now_ns();
    /* the release orders the descriptor stores above before the epoch; the
     * initial thread is the epoch's only writer, so it counts it itself */
    st_rel_gpu(&S->epoch, ++s_main_epoch);
    backoff bo(S->timeout_ns);
    while ((int32_t)(ld_acq_gpu(&S->done_blocks) - target) < 0) {
        if (now_ns() - t0 < GF_REGION_SPIN_NS)   /* most regions end within microseconds: no sleep yet */
            continue;
        if (!bo.wait()) {
            set_error(GF_ETIMEDOUT);
            return GF_ETIMEDOUT;
        }
    }
    atomicAdd((unsigned long long *)&S->st_region_ns, (unsigned long long)(now_ns() - t0));
    return GF_OK;
}

template <class F> __device__ __forceinline__ void put_body(gf_region *r, const F &body)
{
    static_assert(sizeof(F) <= GF_BODY_MAX, "loop body captures too much state");
    static_assert(std::is_trivially_copyable<F>::value, "loop body must be trivially copyable");
    const uint32_t *src = reinterpret_cast<const uint32_t *>(&body);
    uint32_t *dst = reinterpret_cast<uint32_t *>(r->body);
#pragma unroll 4
    for (uint32_t k = 0; k < (sizeof(F) + 3) / 4; k++)
        dst[k] = src[k];
}

/* ------------------------------------------------------------ worker state machine */
static __device__ __noinline__ void worker_loop(gf_state *S)
{
    const wctx w = make_wctx();
    uint32_t seen = 0;
    /* idle bound: the serial part may run long, but not forever */
    const uint64_t idle_limit = 8ull * (uint64_t)S->timeout_ns;
    for (;;) {
        if (w.poller) {
            uint32_t e;
            uint32_t ns = 32;
            const uint64_t t0 = now_ns();
            s_abort = 0;
            while ((e = ld_acq_gpu(&S->epoch)) == seen) {
                __nanosleep(ns);
                /* short sleeps while the next region is likely close */
                if (ns < (now_ns() - t0 < GF_REGION_SPIN_NS ? 64u : 256u))
                    ns <<= 1;
                if (now_ns() - t0 > idle_limit) {
                    set_error(GF_ETIMEDOUT);
                    s_abort = 1;
                    break;
                }
            }
            s_epoch = e;
        }
        bar_workers(w.nbar);
        if (s_abort)
            return;
        seen = s_epoch;
        if (*(volatile uint32_t *)&S->exit_flag)
            return;
        tramp_t fn = (tramp_t)S->region.fn;
        fn(&S->region, w);
        bar_workers(w.nbar);
        if (w.poller) {
            __threadfence();
            atomicAdd(&S->done_blocks, 1u);
        }
    }
}

} // namespace gfd

/* ====================================================================== parallel regions */
/* Worksharing loop over [b, e) (paper Sec. 3.3: `omp for` rewritten to span all
 * teams).  Called by the initial thread it runs on every worker of the grid and
 * returns when all have finished; called inside a region it runs serially in
 * the calling thread (no nested parallelism, as OpenMP's default). */
template <class F>
__device__ int gf_parallel_for(int64_t b, int64_t e, int sched, int64_t chunk, F body)
{
    if (!gfd::is_initial_thread()) {
        for (int64_t i = b; i < e; i++)
            body(i);
        return GF_OK;
    }
    if (e <= b)
        return GF_OK;
    gf_state *S = gfd::s_st;
    const int32_t err = *(volatile int32_t *)&S->error;   /* read first: its round trip overlaps the stores below */
    gf_region *r = &S->region;
    r->fn = gfd::static1_fits(sched, chunk, b, e) ? (uint64_t)(&gfd::tramp_for_s1<F>) : (uint64_t)(&gfd::tramp_for<F>);
    r->b = b;
    r->e = e;
    r->chunk = chunk;
    r->sched = sched;
    r->red = GF_RED_NONE;
    gfd::put_body(r, body);
    return gfd::run_region(S, err);
}

/* Worksharing reduction: *out = op over body(i), i in [b, e).  T is double or
 * long long; op is GF_RED_SUM, GF_RED_MIN or GF_RED_MAX.  The paper leaves
 * reduction clauses unrewritten (Sec. 4.3); this adds them. */
template <class T, int OP, class F>
__device__ int gf_reduce(int64_t b, int64_t e, int sched, int64_t chunk, F body, T *out)
{
    if (!gfd::is_initial_thread() || e <= b) {
        gfd::acc<T, OP> a;
        for (int64_t i = b; i < e; i++)
            a.add((T)body(i));
        *out = a.result();
        return GF_OK;
    }
    gf_state *S = gfd::s_st;
    const int32_t err = *(volatile int32_t *)&S->error;   /* read first: its round trip overlaps the stores below */
    gf_region *r = &S->region;
    r->fn = gfd::static1_fits(sched, chunk, b, e) ? (uint64_t)(&gfd::tramp_reduce_s1<T, OP, F>)
                                                  : (uint64_t)(&gfd::tramp_reduce<T, OP, F>);
    r->b = b;
    r->e = e;
    r->chunk = chunk;
    r->sched = sched;
    r->red = OP;
    gfd::put_body(r, body);
    int rc = gfd::run_region(S, err);
    gfd::acc<T, OP> a;
    a.from_words((const uint64_t *)S->red_result);
    *out = a.result();
    return rc;
}

/* ====================================================================== batched loops */
namespace gfd {
template <class F> struct batch_body {
    int nloops;
    const int64_t *trips;
    const int64_t *prefix;   /* first work item of each loop; prefix[nloops] = items */
    int64_t chunk;
    F f;
};

/* Each warp takes one work item (chunk of one loop) at a time -- from a
 * shared counter (dynamic) or round robin (static) -- finds its loop by
 * binary search over the item prefix, and strides its lanes over the chunk. */
template <class F> __device__ void tramp_batch(const gf_region *rd, const wctx &w)
{
    const batch_body<F> bb = *reinterpret_cast<const batch_body<F> *>(rd->body);
    const uint32_t lane = lane_id();
    const int64_t items = bb.prefix[bb.nloops];
    const int64_t warp = w.tid >> 5, nwarps = w.nthreads >> 5;
    int64_t it = warp;
    for (;;) {
        if (rd->sched == GF_SCHED_DYNAMIC) {
            unsigned long long v = 0;
            if (lane == 0)
                v = atomicAdd(&s_st->dyn_next, 1ull);
            it = (int64_t)__shfl_sync(0xffffffffu, v, 0);
        }
        if (it >= items)
            break;
        int lo = 0, hi = bb.nloops - 1;               /* last loop whose first item <= it */
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (bb.prefix[mid] <= it)
                lo = mid;
            else
                hi = mid - 1;
        }
        const int64_t i0 = (it - bb.prefix[lo]) * bb.chunk;
        const int64_t i1 = i0 + bb.chunk < bb.trips[lo] ? i0 + bb.chunk : bb.trips[lo];
        /* four iterations in flight per lane: a body's store may alias its
         * next loads, so without this each lane waits out one load latency
         * per element (4.74 -> 5.71 TB/s on the 256-loop batch) */
#pragma unroll 4
        for (int64_t i = i0 + lane; i < i1; i += 32)
            bb.f(lo, i);
        if (rd->sched != GF_SCHED_DYNAMIC)
            it += nwarps;
    }
}
} // namespace gfd

/*
 * Batching: nloops independent loops in ONE region.  Loop k runs
 * body(k, i) for i in [0, trips[k]).  Work items are chunks of `chunk`
 * iterations; a warp runs one item at a time (lanes stride over it), taken
 * from a shared counter (GF_SCHED_DYNAMIC) or round robin (GF_SCHED_STATIC).
 * Short and long loops share the grid instead of each being a region with
 * its own end-of-region wait.  `prefix` is caller-provided device memory of
 * nloops + 1 entries that receives the item prefix.  Initial thread only
 * (elsewhere the loops run serially in the caller).
 */
template <class F>
__device__ int gf_parallel_for_batch(int nloops, const int64_t *trips, int64_t *prefix, int64_t chunk, int sched,
                                     F body)
{
    if (chunk < 1)
        chunk = 1;
    if (!gfd::is_initial_thread()) {
        for (int k = 0; k < nloops; k++)
            for (int64_t i = 0; i < trips[k]; i++)
                body(k, i);
        return GF_OK;
    }
    int64_t acc = 0;
    for (int k = 0; k < nloops; k++) {
        prefix[k] = acc;
        acc += (trips[k] + chunk - 1) / chunk;
    }
    prefix[nloops] = acc;
    if (acc == 0)
        return GF_OK;
    gf_state *S = gfd::s_st;
    const int32_t err = *(volatile int32_t *)&S->error;   /* read first: its round trip overlaps the stores below */
    gf_region *r = &S->region;
    gfd::batch_body<F> bb{nloops, trips, prefix, chunk, body};
    r->fn = (uint64_t)(&gfd::tramp_batch<F>);
    r->b = 0;
    r->e = acc;
    r->chunk = chunk;
    r->sched = sched;
    r->red = GF_RED_NONE;
    gfd::put_body(r, bb);
    return gfd::run_region(S, err);
}

/* Barrier across every worker of the grid (paper Sec. 3.3: `omp barrier`
 * replaced by a cross-team barrier on global atomic counters).  Inside a
 * region all workers must call it; outside a region it is a no-op. */
static __device__ __noinline__ int gf_barrier()
{
    if (gfd::is_initial_thread())
        return GF_OK;
    gf_state *S = gfd::s_st;
    const gfd::wctx w = gfd::make_wctx();
    __shared__ int s_rc;
    gfd::bar_workers(w.nbar);
    if (w.poller) {
        s_rc = GF_OK;
        const uint32_t gen = *(volatile uint32_t *)&S->bar_gen;
        __threadfence();
        if (atomicAdd(&S->bar_count, 1u) == gridDim.x - 1) {
            S->bar_count = 0;
            __threadfence();
            gfd::st_rel_gpu(&S->bar_gen, gen + 1);
        } else {
            gfd::backoff bo(S->timeout_ns);
            while (gfd::ld_acq_gpu(&S->bar_gen) == gen)
                if (!bo.wait()) {
                    gfd::set_error(GF_ETIMEDOUT);
                    s_rc = GF_ETIMEDOUT;
                    break;
                }
        }
    }
    gfd::bar_workers(w.nbar);
    return s_rc;
}

/* ====================================================================== mapped buffers */
/* Buffers the host mapped to the device before main (the loader's job in the
 * paper, Sec. 3.1: command line and environment are moved to the device). */
__device__ __forceinline__ void *gf_buffer(int i)
{
    gf_state *S = gfd::s_st;
    return (i >= 0 && (uint32_t)i < S->nbufs) ? (void *)S->buf_ptr[i] : nullptr;
}
__device__ __forceinline__ uint64_t gf_buffer_bytes(int i)
{
    gf_state *S = gfd::s_st;
    return (i >= 0 && (uint32_t)i < S->nbufs) ? S->buf_bytes[i] : 0;
}

/* small libc pieces that run natively (partial GPU libc, paper Sec. 3.4) */
__device__ __forceinline__ uint32_t gf_strlen(const char *s)
{
    uint32_t n = 0;
    while (s[n])
        n++;
    return n;
}
__device__ __forceinline__ long long gf_atoll(const char *s)
{
    long long v = 0;
    int neg = 0;
    while (*s == ' ')
        s++;
    if (*s == '-' || *s == '+')
        neg = (*s++ == '-');
    while (*s >= '0' && *s <= '9')
        v = v * 10 + (*s++ - '0');
    return neg ? -v : v;
}

#include "gf_device_rpc.cuh"
#include "gf_device_heap.cuh"

/* ====================================================================== program kernel */
namespace gfd {

typedef int (*main_t)(int, char **);

/* MINB: resident blocks per SM the kernel is compiled for (a register cap);
 * memory-bound programs ask for more resident warps with GF_MAIN_BOUNDS. */
template <main_t MAIN, int MINB = GF_MIN_BLOCKS>
__global__ void __launch_bounds__(GF_BLOCK, MINB) program_kernel(gf_state *S, int argc, char **argv)
{
    if (threadIdx.x == 0)
        block_setup(S, 0);
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        if (threadIdx.x == 0) {
            S->t_main_start = now_ns();
            int rc = MAIN(argc, argv);
            pb_flush(S);                      /* printf records main left buffered */
            rpc_collect_deferred(S, false);   /* a printf main did not wait for */
            S->exit_code = rc;
            S->t_main_end = now_ns();
            S->main_done = 1;
            S->exit_flag = 1;
            __threadfence();
            st_rel_gpu(&S->epoch, ++s_main_epoch);
        }
        return;
    }
    worker_loop(S);
}

/*
 * The kernel split's region kernel (paper Sec. 3.3, Fig. 3), a comparator:
 * with split_regions the host server launches it for each parallel region of
 * the program.  Every thread of every block is a worker; the published region
 * runs through its trampoline, and each block counts itself in done_blocks,
 * which the initial thread waits on.  Instantiated per program, because the
 * trampoline pointers are valid only in the program's own module.
 */
template <main_t MAIN, int MINB = GF_MIN_BLOCKS>
__global__ void __launch_bounds__(GF_BLOCK, MINB) region_kernel(gf_state *S)
{
    if (threadIdx.x == 0) {
        block_setup(S, 1);
        s_abort = *(volatile int32_t *)&S->error != 0;   /* one reading for the whole block */
    }
    __syncthreads();
    if (!s_abort) {
        const wctx w = make_wctx();
        tramp_t fn = (tramp_t)S->region.fn;
        fn(&S->region, w);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(&S->done_blocks, 1u);
    }
}

} // namespace gfd

/* host-side registration of a program (name -> cooperative launcher) */
#include "gf_program.h"

#define GF_MAIN_BOUNDS(name, minb)                                                             \
    __device__ int gf_main_##name(int argc, char **argv);                                     \
    static cudaError_t gf_launch_##name(void **args, unsigned grid, unsigned block, void *stream) \
    {                                                                                          \
        return cudaLaunchCooperativeKernel((const void *)&gfd::program_kernel<gf_main_##name, minb>, \
                                           dim3(grid), dim3(block), args, 0, (cudaStream_t)stream); \
    }                                                                                          \
    static int gf_occ_##name(unsigned block)                                                   \
    {                                                                                          \
        int n = 0;                                                                             \
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(                                     \
                &n, (const void *)&gfd::program_kernel<gf_main_##name, minb>, (int)block, 0) != cudaSuccess) \
            return -1;                                                                         \
        return n;                                                                              \
    }                                                                                          \
    /* grid 0: only load the region kernel (before the program kernel runs:     \
     * a lazily loaded kernel would wait for the running program to end) */    \
    static cudaError_t gf_region_##name(void **args, unsigned grid, unsigned block, void *stream) \
    {                                                                                          \
        if (!grid) {                                                                           \
            cudaFuncAttributes fa;                                                             \
            return cudaFuncGetAttributes(&fa, (const void *)&gfd::region_kernel<gf_main_##name, minb>); \
        }                                                                                      \
        return cudaLaunchKernel((const void *)&gfd::region_kernel<gf_main_##name, minb>, dim3(grid), \
                                dim3(block), args, 0, (cudaStream_t)stream);                   \
    }                                                                                          \
    static const int gf_reg_##name =                                                           \
        gf_program_register(#name, gf_launch_##name, gf_occ_##name, gf_region_##name);        \
    __device__ int gf_main_##name

/* GF_MAIN(name)(int argc, char **argv) { ... } defines and registers a program */
#define GF_MAIN(name) GF_MAIN_BOUNDS(name, GF_MIN_BLOCKS)

#endif
