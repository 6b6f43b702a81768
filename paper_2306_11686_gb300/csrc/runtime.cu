/*
 * Host runtime: the C ABI of include/gf.h.
 *
 * The loader part follows the paper's main wrapper (Sec. 3.1): argv and the
 * mapped buffers go to the device, the RPC server runs, main starts on the
 * GPU.  GB300 specifics:
 *  - the ring lives in pinned host memory mapped into the device address space
 *    (cudaHostAllocMapped); on Grace-Blackwell the GPU reaches it coherently
 *    over NVLink-C2C, so hand-offs are single release/acquire words instead of
 *    the paper's managed-memory page traffic;
 *  - bulk fwrite/fread payloads move by copy-engine DMA on a separate stream,
 *    double-buffered through pinned staging, while the program's grid keeps
 *    running (no SM time spent copying);
 *  - the context holds one device heap pool and one ring pool; a launch takes
 *    a program instance (its state and staging) plus a heap quota and a
 *    ring-slot quota carved from the pools, so concurrent programs (serving)
 *    are isolated, and a program is admitted only when an instance, its heap
 *    quota and its ring quota are all free (otherwise GF_EBUSY).
 */
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <chrono>
#include <condition_variable>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "gf.h"
#include "gf_layout.h"
#include "gf_internal.h"
#include "gf_program.h"
#include "host/range_alloc.h"
#include "host/server.h"

#define GF_MAX_BLOCKS_PER_SM 32
#define GF_ARGV_BYTES (64u * 1024u)
#define GF_DMA_CHUNK (8ull << 20)
#define GF_DMA_LANES 8             /* independent copy-engine lanes (one per server thread, up to 8) */
#define GF_INTERN_BYTES (1u << 20)
#define GF_BLOCK_THREADS 256

/* ------------------------------------------------------------------ registry */
struct ProgEntry {
    std::string name;
    gf_launch_fn launch;
    gf_occ_fn occ;
    gf_launch_fn region;    /* the program's region kernel (kernel split) */
};
static std::mutex &reg_mu()
{
    static std::mutex m;
    return m;
}
static std::vector<ProgEntry> &registry()
{
    static std::vector<ProgEntry> r;
    return r;
}

extern "C" __attribute__((visibility("default"))) int gf_program_register(const char *name, gf_launch_fn launch,
                                                                           gf_occ_fn occ, gf_launch_fn region)
{
    std::lock_guard<std::mutex> g(reg_mu());
    registry().push_back({name, launch, occ, region});
    return (int)registry().size() - 1;
}

/* ------------------------------------------------------------------ context */
struct Staged {
    void *host;
    void *dev;
    uint64_t bytes;
    uint32_t dir;
    bool owned;
};

/* One copy-engine lane: two pinned staging buffers of GF_DMA_CHUNK bytes
 * (double buffering), a stream and its events.  Server thread t uses lane
 * t % GF_DMA_LANES, so the threads' DMAs run side by side instead of
 * queueing behind one context-wide lock. */
struct DmaLane {
    std::mutex mu;
    cudaStream_t stream = nullptr;
    void *stage[2] = {};
    cudaEvent_t ev[2] = {};
};
static thread_local int tl_dma_lane = 0;

struct Instance {
    int idx = 0;
    std::atomic<bool> busy{false};
    gf_state *d_state = nullptr;
    void *d_partials = nullptr;
    void *d_fmt = nullptr;
    uint8_t *d_heap = nullptr;      /* this launch's heap quota inside the context's pool */
    void *d_meta = nullptr, *d_heads = nullptr, *d_cur = nullptr, *d_ext = nullptr, *d_lsize = nullptr;
    uint32_t nslabs = 0, npages = 0;
    uint64_t slab_bytes = 0, large_bytes = 0;
    uint64_t heap_first = 0, heap_units = 0;    /* quota in the heap pool, in slabs */
    uint64_t ring_first = 0, ring_n = 0;        /* quota in the ring pool, in slots */
    char *d_argv = nullptr;
    uint8_t *bulk_host = nullptr;   /* pinned, device-mapped bulk arena */
    uint64_t bulk_dev = 0;
    std::vector<char> h_argv;
    gf_state h_init;     /* initial state copied to the device at launch */
    gf_state h_final;    /* state read back after the program ends       */
    uint64_t h_ext0 = 0;
    gfh::Segment seg;
    cudaEvent_t ev_done = nullptr;
    /* kernel split: the running program's region kernel, its grid and stream */
    gf_launch_fn region = nullptr;
    uint32_t region_grid = 0;
    cudaStream_t region_stream = nullptr;
};

struct gf_handle {
    gf_ctx *ctx;
    Instance *inst;
    cudaStream_t stream;
    std::vector<Staged> staged;
    uint32_t grid, block;
    bool finished = false;
};

struct gf_ctx {
    gf_config cfg;
    int device = 0, nsm = 0;
    uint8_t *ring_host = nullptr;
    uint64_t ring_dev = 0;
    size_t ring_bytes = 0;
    uint8_t *heap_pool = nullptr;   /* device heap shared out as per-launch quotas */
    uint64_t heap_pool_bytes = 0;
    uint64_t max_slabs = 0, max_pages = 0;
    RangeAlloc heap_ra, ring_ra;
    std::mutex adm_mu;              /* admission: instances, heap and ring quotas */
    std::vector<Instance *> inst;
    gfh::Server server;
    std::vector<std::thread> threads;
    std::atomic<bool> stop{false};
    std::atomic<int> nactive{0};
    std::mutex act_mu;
    std::condition_variable act_cv;
    cudaStream_t own_stream = nullptr;
    DmaLane dma[GF_DMA_LANES];
    uint8_t *intern_host = nullptr;
    uint64_t intern_dev = 0;
    size_t intern_used = 0;
    FILE *out = stdout;
    bool own_out = false;
    gfh::AsyncFile *aout = nullptr;   /* the stdout file, written by its own thread */
    std::mutex stats_mu;
    gf_stats last;
};

static int cuda_err(cudaError_t e)
{
    if (e == cudaSuccess)
        return GF_OK;
    if (e == cudaErrorMemoryAllocation)
        return GF_ENOMEM;
    return GF_ECUDA;
}
#define GF_CK(x)                                                                                    \
    do {                                                                                            \
        cudaError_t _e = (x);                                                                       \
        if (_e != cudaSuccess) {                                                                    \
            fprintf(stderr, "gf: %s failed: %s (%s:%d)\n", #x, cudaGetErrorString(_e), __FILE__, __LINE__); \
            return cuda_err(_e);                                                                    \
        }                                                                                           \
    } while (0)

extern "C" GF_API void gf_config_default(gf_config *c)
{
    memset(c, 0, sizeof *c);
    c->heap_bytes = 4ull << 30;
    c->heap_small_pct = 50;
    c->ring_slots = 4096;
    c->slot_bytes = 4096;
    c->aggregate = 1;
    c->server_threads = 1;
    c->max_programs = 1;
    c->grid = 0;
    c->timeout_ns = 30ll * 1000 * 1000 * 1000;
    c->stream = nullptr;
    c->stdout_path = nullptr;
    c->fmt_cache = 4096;
    c->bulk_bytes = 64ull << 20;
    c->split_regions = 0;
    c->pad0 = 0;
    c->device = -1;
    c->heap_pool_bytes = 0;
    c->ring_pool_slots = 0;
    c->pad1 = 0;
}

extern "C" GF_API const char *gf_strerror(int e)
{
    switch (e) {
    case GF_OK: return "ok";
    case GF_EINVAL: return "invalid argument";
    case GF_ENOMEM: return "out of memory";
    case GF_ERING: return "no RPC ring slot became free in time";
    case GF_ETIMEDOUT: return "timed out waiting for the host or for other threads";
    case GF_EHOST: return "host landing pad failed";
    case GF_ECUDA: return "CUDA runtime error";
    case GF_ENOENT: return "no such program";
    case GF_EBUSY: return "no free program instance";
    default: return "unknown error";
    }
}

static bool pow2(uint64_t x) { return x && !(x & (x - 1)); }

/* ------------------------------------------------------------------ DMA */
/*
 * Device -> host streaming through the calling server thread's lane: chunk k
 * goes to staging buffer k % 2, and the copy of chunk k overlaps the sink's
 * work on chunk k - 1; chunks reach the sink in order.  Returns the length of
 * the prefix the sink accepted.
 */
static uint64_t dma_d2h(gf_ctx *c, uint64_t dev, uint64_t bytes, const gfh::sink_fn &sink, bool parallel)
{
    (void)parallel;                       /* chunks are always handed over in order */
    DmaLane &L = c->dma[tl_dma_lane % GF_DMA_LANES];
    std::lock_guard<std::mutex> g(L.mu);
    const uint64_t nchunk = (bytes + GF_DMA_CHUNK - 1) / GF_DMA_CHUNK;
    uint64_t pend[2] = {UINT64_MAX, UINT64_MAX};   /* chunk held by each staging buffer */
    uint64_t delivered = 0;
    bool failed = false;
    auto consume = [&](int k) {
        if (pend[k] == UINT64_MAX)
            return;
        const uint64_t ch = pend[k], off = ch * GF_DMA_CHUNK, n = std::min<uint64_t>(GF_DMA_CHUNK, bytes - off);
        if (!failed && cudaEventSynchronize(L.ev[k]) == cudaSuccess && sink(L.stage[k], n, off))
            delivered += n;
        else
            failed = true;
        pend[k] = UINT64_MAX;
    };
    for (uint64_t ch = 0; ch < nchunk && !failed; ch++) {
        const int k = (int)(ch & 1);
        consume(k);                       /* the buffer's previous chunk goes out first */
        const uint64_t off = ch * GF_DMA_CHUNK, n = std::min<uint64_t>(GF_DMA_CHUNK, bytes - off);
        if (cudaMemcpyAsync(L.stage[k], (const void *)(dev + off), n, cudaMemcpyDeviceToHost, L.stream) !=
                cudaSuccess ||
            cudaEventRecord(L.ev[k], L.stream) != cudaSuccess) {
            failed = true;
            break;
        }
        pend[k] = ch;
        consume(1 - k);                   /* the other buffer's chunk landed while this copy was issued */
    }
    consume(nchunk & 1 ? 0 : 1);          /* drain in chunk order: the older pending chunk first */
    consume(nchunk & 1 ? 1 : 0);
    cudaStreamSynchronize(L.stream);
    return delivered;
}

static uint64_t dma_h2d(gf_ctx *c, uint64_t dev, uint64_t bytes, const gfh::source_fn &src)
{
    DmaLane &L = c->dma[tl_dma_lane % GF_DMA_LANES];
    std::lock_guard<std::mutex> g(L.mu);
    uint64_t off = 0;
    int b = 0;
    bool inflight[2] = {false, false};
    while (off < bytes) {
        if (inflight[b]) {
            cudaEventSynchronize(L.ev[b]);
            inflight[b] = false;
        }
        const uint64_t want = std::min<uint64_t>(GF_DMA_CHUNK, bytes - off);
        const uint64_t got = src(L.stage[b], want);
        if (got) {
            if (cudaMemcpyAsync((void *)(dev + off), L.stage[b], got, cudaMemcpyHostToDevice, L.stream) !=
                    cudaSuccess ||
                cudaEventRecord(L.ev[b], L.stream) != cudaSuccess)
                break;
            inflight[b] = true;
            off += got;
        }
        if (got != want)
            break;
        b = 1 - b;
    }
    cudaStreamSynchronize(L.stream);
    return off;
}

/* ------------------------------------------------------------------ server threads */
static void server_main(gf_ctx *c, uint32_t tid, uint32_t nthr)
{
    tl_dma_lane = (int)(tid % GF_DMA_LANES);
    uint32_t idle = 0;
    while (!c->stop.load(std::memory_order_relaxed)) {
        int n = 0;
        for (Instance *in : c->inst)
            if (in->seg.active.load(std::memory_order_acquire))
                n += c->server.poll(in->seg, tid, nthr);
        if (n) {
            idle = 0;
            continue;
        }
        c->server.idle();                       /* mappings of this thread's finished writes */
        if (c->nactive.load(std::memory_order_acquire) == 0) {
            std::unique_lock<std::mutex> lk(c->act_mu);
            c->act_cv.wait_for(lk, std::chrono::milliseconds(5),
                               [&] { return c->stop.load() || c->nactive.load() > 0; });
        } else if (++idle > 4096) {
            std::this_thread::yield();
        }
    }
}

/* ------------------------------------------------------------------ init / finalize */
static int inst_alloc(gf_ctx *c, Instance *in)
{
    const gf_config &cf = c->cfg;
    GF_CK(cudaMalloc((void **)&in->d_state, sizeof(gf_state)));
    GF_CK(cudaMalloc(&in->d_partials, (size_t)c->nsm * GF_MAX_BLOCKS_PER_SM * 16));
    GF_CK(cudaMalloc(&in->d_fmt, (size_t)cf.fmt_cache * 8));
    GF_CK(cudaMalloc((void **)&in->d_argv, GF_ARGV_BYTES));
    /* heap metadata, sized for the largest quota (the whole pool); the heap
     * itself is the launch's quota inside the context's pool */
    GF_CK(cudaMalloc(&in->d_meta, (size_t)std::max<uint64_t>(c->max_slabs, 1) * 16));
    GF_CK(cudaMalloc(&in->d_heads, (size_t)GF_MAX_SM * GF_HEAP_NCLASS * GF_HEAP_LANES * 8));
    GF_CK(cudaMalloc(&in->d_cur, (size_t)GF_MAX_SM * GF_HEAP_NCLASS * 4));
    GF_CK(cudaMalloc(&in->d_ext, (size_t)GF_LARGE_EXT_MAX * 8));
    GF_CK(cudaMalloc(&in->d_lsize, (size_t)std::max<uint64_t>(c->max_pages, 1) * 4));
    GF_CK(cudaEventCreateWithFlags(&in->ev_done, cudaEventDisableTiming));
    if (cf.split_regions)
        GF_CK(cudaStreamCreateWithFlags(&in->region_stream, cudaStreamNonBlocking));
    in->seg.slot_bytes = cf.slot_bytes;
    in->seg.prog = (uint32_t)in->idx;
    if (cf.bulk_bytes) {
        if (cudaHostAlloc((void **)&in->bulk_host, cf.bulk_bytes, cudaHostAllocMapped | cudaHostAllocPortable) !=
            cudaSuccess)
            return GF_ENOMEM;
        void *bd = nullptr;
        GF_CK(cudaHostGetDevicePointer(&bd, in->bulk_host, 0));
        in->bulk_dev = (uint64_t)bd;
        in->seg.bulk = in->bulk_host;
        in->seg.bulk_bytes = cf.bulk_bytes;
    }
    return GF_OK;
}

static void inst_free(Instance *in)
{
    cudaFree(in->d_state);
    cudaFree(in->d_partials);
    cudaFree(in->d_fmt);
    cudaFree(in->d_argv);
    if (in->bulk_host)
        cudaFreeHost(in->bulk_host);
    cudaFree(in->d_meta);
    cudaFree(in->d_heads);
    cudaFree(in->d_cur);
    cudaFree(in->d_ext);
    cudaFree(in->d_lsize);
    if (in->ev_done)
        cudaEventDestroy(in->ev_done);
    if (in->region_stream)
        cudaStreamDestroy(in->region_stream);
}

extern "C" GF_API int gf_finalize(gf_ctx *c)
{
    if (!c)
        return GF_OK;
    for (Instance *in : c->inst)
        if (in->busy.load() && in->ev_done)
            cudaEventSynchronize(in->ev_done);
    c->stop = true;
    c->act_cv.notify_all();
    for (auto &t : c->threads)
        t.join();
    c->server.close_all();
    if (c->own_out && c->out) {
        c->server.set_stdout(nullptr);      /* the server keeps no pointer to the closed stream */
        if (c->aout)
            gfh::async_close(c->aout);
        else
            fclose(c->out);
        c->out = nullptr;
        c->aout = nullptr;
    }
    for (Instance *in : c->inst) {
        inst_free(in);
        delete in;
    }
    if (c->ring_host)
        cudaFreeHost(c->ring_host);
    if (c->heap_pool)
        cudaFree(c->heap_pool);
    if (c->intern_host)
        cudaFreeHost(c->intern_host);
    for (DmaLane &L : c->dma) {
        for (int k = 0; k < 2; k++) {
            if (L.stage[k])
                cudaFreeHost(L.stage[k]);
            if (L.ev[k])
                cudaEventDestroy(L.ev[k]);
        }
        if (L.stream)
            cudaStreamDestroy(L.stream);
    }
    if (c->own_stream)
        cudaStreamDestroy(c->own_stream);
    delete c;
    return GF_OK;
}

extern "C" GF_API int gf_init(const gf_config *cfg, gf_ctx **out)
{
    if (!out)
        return GF_EINVAL;
    *out = nullptr;
    gf_config cf;
    gf_config_default(&cf);
    if (cfg)
        cf = *cfg;
    if (!pow2(cf.ring_slots) || cf.slot_bytes < 1024 || cf.slot_bytes > 65536 || cf.slot_bytes % 64 ||
        !pow2(cf.fmt_cache) ||
        cf.max_programs < 1 || cf.max_programs > 1024 || cf.heap_small_pct > 100 || cf.timeout_ns <= 0)
        return GF_EINVAL;
    if (cf.server_threads && (!pow2(cf.server_threads) || cf.server_threads > cf.ring_slots))
        return GF_EINVAL;
    /* pools: whole slabs; a quota is rounded up to whole slabs, so the
     * default pool holds max_programs default quotas exactly */
    const uint64_t slab_b = 1ull << GF_SLAB_SHIFT;
    const uint64_t quota0 = (cf.heap_bytes + slab_b - 1) / slab_b * slab_b;
    const uint64_t ring_pool = cf.ring_pool_slots ? cf.ring_pool_slots : (uint64_t)cf.ring_slots * cf.max_programs;
    const uint64_t heap_pool =
        (cf.heap_pool_bytes ? (cf.heap_pool_bytes + slab_b - 1) / slab_b * slab_b : quota0 * cf.max_programs);
    if (ring_pool < cf.ring_slots || heap_pool < quota0 || ring_pool > (1ull << 24))
        return GF_EINVAL;
    if (cf.split_regions > 1 || (cf.split_regions && cf.server_threads == 0))
        return GF_EINVAL;                /* the split needs a server thread to launch regions */
    gf_ctx *c = new gf_ctx();
    c->cfg = cf;
    memset(&c->last, 0, sizeof c->last);
    int rc = GF_OK;
    auto fail = [&](int e) {
        gf_finalize(c);
        return e;
    };
    if (cf.device >= 0 && cudaSetDevice(cf.device) != cudaSuccess)
        return fail(GF_ECUDA);
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess)
        return fail(GF_ECUDA);
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->device);
    if (!coop)
        return fail(GF_ECUDA);
    size_t stack = 0;
    cudaDeviceGetLimit(&stack, cudaLimitStackSize);
    if (stack < 4096)
        cudaDeviceSetLimit(cudaLimitStackSize, 4096);
    /* heap pool: one device allocation, shared out as per-launch quotas in
     * whole slabs; per-instance metadata is sized for a quota of the whole pool */
    {
        const uint64_t slab = 1ull << GF_SLAB_SHIFT, page = 1ull << GF_PAGE_SHIFT;
        c->heap_pool_bytes = heap_pool;
        c->max_slabs = c->heap_pool_bytes / slab;
        c->max_pages = c->heap_pool_bytes / page;
        c->heap_ra.init(c->max_slabs);
        if (c->heap_pool_bytes && cudaMalloc((void **)&c->heap_pool, c->heap_pool_bytes) != cudaSuccess)
            return fail(GF_ENOMEM);
    }
    c->ring_ra.init(ring_pool);
    /* ring: pinned, device-mapped host memory */
    c->ring_bytes = (size_t)ring_pool * cf.slot_bytes;
    if (cudaHostAlloc((void **)&c->ring_host, c->ring_bytes, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess)
        return fail(GF_ENOMEM);
    memset(c->ring_host, 0, c->ring_bytes);
    void *rd = nullptr;
    if (cudaHostGetDevicePointer(&rd, c->ring_host, 0) != cudaSuccess)
        return fail(GF_ECUDA);
    c->ring_dev = (uint64_t)rd;
    if (cudaHostAlloc((void **)&c->intern_host, GF_INTERN_BYTES, cudaHostAllocMapped | cudaHostAllocPortable) !=
        cudaSuccess)
        return fail(GF_ENOMEM);
    void *idv = nullptr;
    cudaHostGetDevicePointer(&idv, c->intern_host, 0);
    c->intern_dev = (uint64_t)idv;
    for (DmaLane &L : c->dma) {
        for (int k = 0; k < 2; k++) {
            if (cudaHostAlloc(&L.stage[k], GF_DMA_CHUNK, cudaHostAllocPortable) != cudaSuccess)
                return fail(GF_ENOMEM);
            if (cudaEventCreateWithFlags(&L.ev[k], cudaEventDisableTiming) != cudaSuccess)
                return fail(GF_ECUDA);
        }
        if (cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking) != cudaSuccess)
            return fail(GF_ECUDA);
    }
    if (cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess)
        return fail(GF_ECUDA);
    for (uint32_t k = 0; k < cf.max_programs; k++) {
        Instance *in = new Instance();
        in->idx = (int)k;
        c->inst.push_back(in);
        if ((rc = inst_alloc(c, in)) != GF_OK)
            return fail(rc);
    }
    if (cf.stdout_path) {
        c->aout = gfh::async_open(cf.stdout_path);
        c->out = gfh::async_stream(c->aout);
        if (!c->out)
            return fail(GF_EINVAL);
        c->own_out = true;
    }
    c->server.set_stdout(c->out);
    c->server.set_dma([c](uint64_t d, uint64_t n, const gfh::sink_fn &s, bool par) { return dma_d2h(c, d, n, s, par); },
                      [c](uint64_t d, uint64_t n, const gfh::source_fn &s) { return dma_h2d(c, d, n, s); });
    /* kernel split: launch the running program's region kernel on its instance's
     * stream and answer with the grid; the device waits for its blocks */
    c->server.set_region([c](uint32_t idx) -> int64_t {
        if (idx >= c->inst.size())
            return -1;
        Instance *in = c->inst[idx];
        if (!in->region || !in->region_grid || !in->region_stream)
            return -1;
        gf_state *a_state = in->d_state;
        void *args[1] = {&a_state};
        const cudaError_t e = in->region(args, in->region_grid, GF_BLOCK_THREADS, in->region_stream);
        return e == cudaSuccess ? (int64_t)in->region_grid : -1;
    });
    c->server.set_intern([c](const std::string &s) -> uint64_t {
        if (c->intern_used + s.size() + 1 > GF_INTERN_BYTES)
            return 0;
        memcpy(c->intern_host + c->intern_used, s.c_str(), s.size() + 1);
        const uint64_t a = c->intern_dev + c->intern_used;
        c->intern_used += (s.size() + 16) & ~size_t(7);
        return a;
    });
    for (uint32_t t = 0; t < cf.server_threads; t++)
        c->threads.emplace_back(server_main, c, t, cf.server_threads);
    *out = c;
    return GF_OK;
}

extern "C" GF_API int gf_program_lookup(gf_ctx *c, const char *name, gf_program *out)
{
    if (!c || !name || !out)
        return GF_EINVAL;
    std::lock_guard<std::mutex> g(reg_mu());
    for (size_t k = 0; k < registry().size(); k++)
        if (registry()[k].name == name) {
            *out = (gf_program)k;
            return GF_OK;
        }
    return GF_ENOENT;
}

extern "C" GF_API int gf_rpc_register(gf_ctx *c, uint32_t opcode, gf_host_fn fn, void *user)
{
    if (!c || opcode < GF_OP_USER || !fn)
        return GF_EINVAL;
    return c->server.register_user(opcode, fn, user);
}

static int occupancy(gf_ctx *c, gf_program prog, uint32_t *per_sm)
{
    ProgEntry pe;
    {
        std::lock_guard<std::mutex> g(reg_mu());
        if (prog < 0 || (size_t)prog >= registry().size())
            return GF_ENOENT;
        pe = registry()[prog];
    }
    int occ = pe.occ(GF_BLOCK_THREADS);
    if (occ < 1)
        return GF_ECUDA;
    *per_sm = (uint32_t)std::min(occ, GF_MAX_BLOCKS_PER_SM);
    return GF_OK;
}

extern "C" GF_API int gf_grid_info(gf_ctx *c, gf_program prog, uint32_t *sms, uint32_t *per_sm)
{
    if (!c || !sms || !per_sm)
        return GF_EINVAL;
    *sms = (uint32_t)c->nsm;
    return occupancy(c, prog, per_sm);
}

/* ------------------------------------------------------------------ launch / wait */
static void release_staged(gf_handle *h, bool copy_back)
{
    for (Staged &s : h->staged) {
        if (copy_back && s.owned && (s.dir & GF_BUF_OUT))
            cudaMemcpyAsync(s.host, s.dev, s.bytes, cudaMemcpyDeviceToHost, h->stream);
    }
    cudaStreamSynchronize(h->stream);
    for (Staged &s : h->staged)
        if (s.owned)
            cudaFreeAsync(s.dev, h->stream);
    h->staged.clear();
}

static int inst_start(gf_ctx *c, Instance *in, cudaStream_t stream, uint32_t grid);

/* Admission: a free instance, a heap quota and a ring quota, all or none.
 * GF_EINVAL for a quota no pool can ever hold, GF_EBUSY when it does not fit
 * now.  The heap quota is [small slabs | large pages] like a whole arena. */
static int admit(gf_ctx *c, const gf_quota *q, Instance **out)
{
    const gf_config &cf = c->cfg;
    const uint64_t slab = 1ull << GF_SLAB_SHIFT, page = 1ull << GF_PAGE_SHIFT;
    const uint64_t hb = q && q->heap_bytes ? q->heap_bytes : cf.heap_bytes;
    const uint64_t rs = q && q->ring_slots ? q->ring_slots : cf.ring_slots;
    const uint64_t hu = (hb + slab - 1) / slab;
    if (!pow2(rs) || rs > c->ring_ra.total || rs < std::max<uint32_t>(1, cf.server_threads) ||
        hu > c->heap_ra.total)
        return GF_EINVAL;
    std::lock_guard<std::mutex> g(c->adm_mu);
    Instance *in = nullptr;
    for (Instance *x : c->inst)
        if (!x->busy.load()) {
            in = x;
            break;
        }
    if (!in)
        return GF_EBUSY;
    uint64_t ho = 0, ro = 0;
    if (hu && !c->heap_ra.alloc(hu, &ho))
        return GF_EBUSY;
    if (!c->ring_ra.alloc(rs, &ro)) {
        c->heap_ra.release(ho, hu);
        return GF_EBUSY;
    }
    in->busy = true;
    in->heap_first = ho;
    in->heap_units = hu;
    in->ring_first = ro;
    in->ring_n = rs;
    const uint64_t bytes = hu * slab;
    in->d_heap = hu ? c->heap_pool + ho * slab : nullptr;
    in->slab_bytes = (bytes * cf.heap_small_pct / 100) / slab * slab;
    in->large_bytes = (bytes - in->slab_bytes) / page * page;
    in->nslabs = (uint32_t)(in->slab_bytes / slab);
    in->npages = (uint32_t)(in->large_bytes / page);
    in->seg.slots = c->ring_host + ro * cf.slot_bytes;
    in->seg.nslots = (uint32_t)rs;
    *out = in;
    return GF_OK;
}

/* Stop serving the instance's ring segment and wait until no server thread
 * is inside it, so its slots can go to another program. */
static void seg_stop(gf_ctx *c, Instance *in)
{
    if (in->seg.active.exchange(false))
        c->nactive--;
    while (in->seg.pollers.load() != 0)
        std::this_thread::yield();
}

/* Give the instance and its quotas back (the program has ended or never started). */
static void inst_release(gf_ctx *c, Instance *in)
{
    std::lock_guard<std::mutex> g(c->adm_mu);
    c->heap_ra.release(in->heap_first, in->heap_units);
    c->ring_ra.release(in->ring_first, in->ring_n);
    in->heap_units = in->ring_n = 0;
    in->busy = false;
}

extern "C" GF_API int gf_launch(gf_ctx *c, gf_program prog, int argc, const char *const *argv, const gf_buf *bufs,
                                int nbufs, void *stream, uint32_t grid, gf_handle **out)
{
    return gf_launch_q(c, prog, argc, argv, bufs, nbufs, stream, grid, nullptr, out);
}

extern "C" GF_API int gf_launch_q(gf_ctx *c, gf_program prog, int argc, const char *const *argv, const gf_buf *bufs,
                                  int nbufs, void *stream, uint32_t grid, const gf_quota *quota, gf_handle **out)
{
    if (!c || !out || argc < 0 || nbufs < 0 || nbufs > GF_MAX_BUFS || (nbufs && !bufs) || (argc && !argv))
        return GF_EINVAL;
    *out = nullptr;
    ProgEntry pe;
    {
        std::lock_guard<std::mutex> g(reg_mu());
        if (prog < 0 || (size_t)prog >= registry().size())
            return GF_ENOENT;
        pe = registry()[prog];
    }
    uint32_t per_sm = 0;
    int rc = occupancy(c, prog, &per_sm);
    if (rc)
        return rc;
    const uint32_t full = per_sm * (uint32_t)c->nsm;
    if (!grid)
        grid = c->cfg.grid ? c->cfg.grid : std::max<uint32_t>(1, full / c->cfg.max_programs);
    if (grid > full || grid > (uint32_t)c->nsm * GF_MAX_BLOCKS_PER_SM)
        return GF_EINVAL;
    /* kernel split: the program kernel is one block (the initial thread's);
     * regions get the grid, less the block the program kernel holds */
    uint32_t region_grid = 0;
    if (c->cfg.split_regions) {
        region_grid = std::max<uint32_t>(1, grid >= full ? full - 1 : grid);
        grid = 1;
        /* load the region kernel now: with lazy loading its first launch
         * would otherwise wait for the running program kernel to finish */
        if (!pe.region || pe.region(nullptr, 0, 0, nullptr) != cudaSuccess)
            return GF_ECUDA;
    }
    /* argv block: pointer array then strings, all device addresses */
    size_t need = (size_t)(argc + 1) * 8;
    for (int k = 0; k < argc; k++)
        need += strlen(argv[k]) + 1;
    if (need > GF_ARGV_BYTES)
        return GF_EINVAL;
    /* admission: a free instance, its heap quota and its ring quota */
    Instance *in = nullptr;
    if ((rc = admit(c, quota, &in)) != GF_OK)
        return rc;
    gf_handle *h = new gf_handle();
    h->ctx = c;
    h->inst = in;
    h->stream = (cudaStream_t)(stream ? stream : (c->cfg.stream ? c->cfg.stream : c->own_stream));
    h->grid = grid;
    h->block = GF_BLOCK_THREADS;
    in->region = pe.region;
    in->region_grid = region_grid;
    auto bail = [&](int e) {
        release_staged(h, false);
        seg_stop(c, in);
        inst_release(c, in);
        delete h;
        return e;
    };
    in->h_argv.assign(need, 0);
    uint64_t *ptrs = (uint64_t *)in->h_argv.data();
    size_t off = (size_t)(argc + 1) * 8;
    for (int k = 0; k < argc; k++) {
        const size_t n = strlen(argv[k]) + 1;
        memcpy(in->h_argv.data() + off, argv[k], n);
        ptrs[k] = (uint64_t)in->d_argv + off;
        off += n;
    }
    ptrs[argc] = 0;
    if (cudaMemcpyAsync(in->d_argv, in->h_argv.data(), need, cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
        return bail(GF_ECUDA);
    /* mapped buffers */
    gf_state &s = in->h_init;
    memset(&s, 0, sizeof s);
    for (int k = 0; k < nbufs; k++) {
        cudaPointerAttributes at;
        void *dev = bufs[k].ptr;
        if (bufs[k].ptr && bufs[k].bytes) {
            if (cudaPointerGetAttributes(&at, bufs[k].ptr) != cudaSuccess)
                return bail(GF_EINVAL);
            if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) {
                if (cudaMallocAsync(&dev, bufs[k].bytes, h->stream) != cudaSuccess)
                    return bail(GF_ENOMEM);
                h->staged.push_back({bufs[k].ptr, dev, bufs[k].bytes, bufs[k].dir, true});
                if ((bufs[k].dir & GF_BUF_IN) &&
                    cudaMemcpyAsync(dev, bufs[k].ptr, bufs[k].bytes, cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
                    return bail(GF_ECUDA);
            }
        }
        s.buf_ptr[k] = (uint64_t)dev;
        s.buf_bytes[k] = bufs[k].bytes;
    }
    s.nbufs = (uint32_t)nbufs;
    if ((rc = inst_start(c, in, h->stream, grid)) != GF_OK)
        return bail(rc);
    int a_argc = argc;
    char **a_argv = (char **)in->d_argv;
    gf_state *a_state = in->d_state;
    void *args[3] = {&a_state, &a_argc, &a_argv};
    cudaError_t le = pe.launch(args, grid, GF_BLOCK_THREADS, h->stream);
    if (le != cudaSuccess || cudaEventRecord(in->ev_done, h->stream) != cudaSuccess) {
        fprintf(stderr, "gf: launch of %s failed: %s\n", pe.name.c_str(), cudaGetErrorString(le));
        return bail(GF_ECUDA);
    }
    *out = h;
    return GF_OK;
}

/* Fill the rest of in->h_init (buffers are already in it), copy it to the
 * device, reset the heap metadata, reset and activate the ring segment. */
static int inst_start(gf_ctx *c, Instance *in, cudaStream_t stream, uint32_t grid)
{
    gf_state &s = in->h_init;
    s.nblocks = grid;
    s.block_dim = GF_BLOCK_THREADS;
    s.nworkers = grid * GF_BLOCK_THREADS - 32;
    s.aggregate = c->cfg.aggregate;
    s.timeout_ns = c->cfg.timeout_ns;
    s.ring_slots = c->ring_dev + in->ring_first * c->cfg.slot_bytes;
    s.nslots = (uint32_t)in->ring_n;
    s.slot_bytes = c->cfg.slot_bytes;
    s.fmt_cache = (uint64_t)in->d_fmt;
    s.fmt_cache_cap = c->cfg.fmt_cache;
    s.prog_id = (uint32_t)in->idx;
    s.partials = (uint64_t)in->d_partials;
    s.bulk_dev = in->bulk_dev;
    s.bulk_bytes = in->bulk_host ? c->cfg.bulk_bytes : 0;
    s.split = c->cfg.split_regions ? 1u : 0u;
    gf_heap &H = s.heap;
    H.base = (uint64_t)in->d_heap;
    H.bytes = in->slab_bytes + in->large_bytes;
    H.slab_base = (uint64_t)in->d_heap;
    H.slab_bytes = in->slab_bytes;
    H.large_base = (uint64_t)in->d_heap + in->slab_bytes;
    H.large_bytes = in->large_bytes;
    H.slab_meta = (uint64_t)in->d_meta;
    H.free_heads = (uint64_t)in->d_heads;
    H.cur_slab = (uint64_t)in->d_cur;
    H.large_ext = (uint64_t)in->d_ext;
    H.large_size = (uint64_t)in->d_lsize;
    H.nslabs = in->nslabs;
    H.npages = in->npages;
    H.large_next = in->npages ? 1 : 0;
    in->h_ext0 = (uint64_t)0 | ((uint64_t)in->npages << 32);
    if (cudaMemcpyAsync(in->d_state, &s, sizeof s, cudaMemcpyHostToDevice, stream) != cudaSuccess ||
        cudaMemsetAsync(in->d_meta, 0, (size_t)std::max<uint32_t>(in->nslabs, 1) * 16, stream) != cudaSuccess ||
        cudaMemsetAsync(in->d_heads, 0, (size_t)GF_MAX_SM * GF_HEAP_NCLASS * GF_HEAP_LANES * 8, stream) != cudaSuccess ||
        cudaMemsetAsync(in->d_cur, 0, (size_t)GF_MAX_SM * GF_HEAP_NCLASS * 4, stream) != cudaSuccess ||
        cudaMemsetAsync(in->d_lsize, 0, (size_t)std::max<uint32_t>(in->npages, 1) * 4, stream) != cudaSuccess ||
        cudaMemsetAsync(in->d_fmt, 0, (size_t)c->cfg.fmt_cache * 8, stream) != cudaSuccess ||
        cudaMemcpyAsync(in->d_ext, &in->h_ext0, 8, cudaMemcpyHostToDevice, stream) != cudaSuccess)
        return GF_ECUDA;
    /* ring segment: every slot free for its first ticket */
    const uint32_t nthr = std::max<uint32_t>(1, c->cfg.server_threads);
    for (uint32_t k = 0; k < in->seg.nslots; k++) {
        gf_slot_hdr *hd = (gf_slot_hdr *)(in->seg.slots + (size_t)k * in->seg.slot_bytes);
        __atomic_store_n(&hd->seq, (uint64_t)k, __ATOMIC_RELEASE);
    }
    in->seg.reset(nthr);
    in->seg.active.store(true, std::memory_order_release);
    c->nactive++;
    c->act_cv.notify_all();
    return GF_OK;
}

/* Standalone kernels that use the device runtime's RPC or heap (synthetic
 * loops, the graph executor) borrow an instance: its state initialised with
 * no program and no buffers, its ring segment served.  Returns the device
 * state, or nullptr when every instance is taken. */
gf_state *gf_inst_acquire(gf_ctx *c, void *stream, uint32_t nblocks, int *idx)
{
    Instance *x = nullptr;
    if (admit(c, nullptr, &x) != GF_OK)
        return nullptr;
    memset(&x->h_init, 0, sizeof x->h_init);
    cudaStream_t s = (cudaStream_t)(stream ? stream : c->own_stream);
    if (inst_start(c, x, s, nblocks ? nblocks : 1) != GF_OK || cudaStreamSynchronize(s) != cudaSuccess) {
        seg_stop(c, x);
        inst_release(c, x);
        return nullptr;
    }
    *idx = x->idx;
    return x->d_state;
}

/* The caller has drained its stream: stop serving the segment, free the instance. */
void gf_inst_release(gf_ctx *c, int idx)
{
    Instance *in = c->inst[(size_t)idx];
    seg_stop(c, in);
    inst_release(c, in);
}

int gf_ctx_server_threads(gf_ctx *c) { return (int)c->cfg.server_threads; }
void *gf_inst_scratch(gf_ctx *c, int idx) { return c->inst[(size_t)idx]->d_partials; }
void gf_inst_heap(gf_ctx *c, int idx, void **base, uint64_t *bytes)
{
    Instance *in = c->inst[(size_t)idx];
    *base = in->d_heap;
    *bytes = in->slab_bytes + in->large_bytes;
}

extern "C" GF_API int gf_done(gf_handle *h)
{
    if (!h)
        return 1;
    return cudaEventQuery(h->inst->ev_done) == cudaErrorNotReady ? 0 : 1;
}

static double hist_pct(const uint64_t *hist, double q)
{
    uint64_t tot = 0;
    for (int k = 0; k < GF_LAT_BUCKETS; k++)
        tot += hist[k];
    if (!tot)
        return 0.0;
    const double want = q * (double)tot;
    uint64_t acc = 0;
    for (int k = 0; k < GF_LAT_BUCKETS; k++) {
        acc += hist[k];
        if ((double)acc >= want) {
            if (k < 8)
                return (double)k;
            const int e = k / 8, sub = k % 8;
            /* bucket covers [2^e (1 + sub/8), 2^e (1 + (sub+1)/8)): report its midpoint */
            return ldexp(1.0 + (sub + 0.5) / 8.0, e);
        }
    }
    return 0.0;
}

extern "C" GF_API int gf_wait(gf_handle *h, int *exit_code, int64_t timeout_ns)
{
    if (!h)
        return GF_EINVAL;
    gf_ctx *c = h->ctx;
    Instance *in = h->inst;
    const auto t0 = std::chrono::steady_clock::now();
    uint32_t spins = 0;
    for (;;) {
        cudaError_t q = cudaEventQuery(in->ev_done);
        if (q == cudaSuccess)
            break;
        if (q != cudaErrorNotReady) {
            fprintf(stderr, "gf: program failed: %s\n", cudaGetErrorString(q));
            seg_stop(c, in);
            release_staged(h, false);
            inst_release(c, in);
            delete h;
            return GF_ECUDA;
        }
        if (c->cfg.server_threads == 0) {
            if (!c->server.poll(in->seg, 0, 1))
                c->server.idle();
        } else if (++spins > 256)
            std::this_thread::sleep_for(std::chrono::microseconds(20));
        if (timeout_ns > 0 &&
            std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now() - t0).count() >
                timeout_ns)
            return GF_ETIMEDOUT;
    }
    seg_stop(c, in);
    int rc = GF_OK;
    if (cudaMemcpyAsync(&in->h_final, in->d_state, sizeof(gf_state), cudaMemcpyDeviceToHost, h->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
        rc = GF_ECUDA;
    release_staged(h, true);
    {
        std::lock_guard<std::mutex> g(c->stats_mu);
        gf_stats &st = c->last;
        const gf_state &f = in->h_final;
        memset(&st, 0, sizeof st);
        for (int k = 0; k < GF_NOPS && k < GF_NSTAT; k++) {
            st.rpc_calls[k] = f.st_calls[k];
            st.rpc_slots[k] = f.st_slots[k];
        }
        st.rpc_wait_ns = f.st_wait_ns;
        st.rpc_p50_ns = hist_pct(f.lat_hist, 0.50);
        st.rpc_p99_ns = hist_pct(f.lat_hist, 0.99);
        st.regions = f.st_regions;
        st.region_ns = f.st_region_ns;
        st.heap_alloc = f.heap.n_alloc;
        st.heap_free = f.heap.n_free;
        st.heap_fail = f.heap.n_fail;
        st.heap_bad_free = f.heap.n_bad_free;
        st.heap_live_bytes = f.heap.live_bytes;
        st.heap_high_water = f.heap.high_water;
        st.main_ns = f.t_main_end > f.t_main_start ? f.t_main_end - f.t_main_start : 0;
        st.host_slots = c->server.stats.slots;
        st.host_records = c->server.stats.records;
        st.host_ns = c->server.stats.ns;
        st.host_dma_bytes = c->server.stats.dma_bytes;
        st.grid = (int32_t)h->grid;
        st.block = (int32_t)h->block;
        st.error = f.error;
        st.exit_code = f.exit_code;
        st.heap_ns = f.st_heap_ns;
        st.copy_regions = f.st_copy_regions;
        st.copy_ns = f.st_copy_ns;
        st.host_ring_bytes = c->server.stats.ring_bytes;
        st.t_start_ns = f.t_main_start;
        st.t_end_ns = f.t_main_end;
        st.heap_quota = in->heap_units << GF_SLAB_SHIFT;
        st.ring_quota = in->ring_n;
        for (int k = 0; k < GF_NOPS && k < GF_NSTAT; k++)
            st.rpc_wait_op_ns[k] = f.st_wait_op_ns[k];
        st.rpc_client_ns = f.st_client_ns;
    }
    if (rc == GF_OK && in->h_final.error)
        rc = in->h_final.error;
    if (exit_code)
        *exit_code = in->h_final.exit_code;
    if (c->aout)
        gfh::async_drain(c->aout);           /* the program's text is in the file when it is done */
    else if (c->out)
        fflush(c->out);
    inst_release(c, in);
    delete h;
    return rc;
}

extern "C" GF_API int gf_run_main(gf_ctx *c, gf_program prog, int argc, const char *const *argv, const gf_buf *bufs,
                                  int nbufs, int *exit_code)
{
    gf_handle *h = nullptr;
    int rc = gf_launch(c, prog, argc, argv, bufs, nbufs, nullptr, 0, &h);
    if (rc)
        return rc;
    return gf_wait(h, exit_code, 0);
}

extern "C" GF_API int gf_rpc_serve(gf_ctx *c, const gf_serve_opts *o)
{
    if (!c)
        return GF_EINVAL;
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        if (o && o->stop && *o->stop)
            return GF_OK;
        bool any = false;
        for (Instance *in : c->inst)
            if (in->seg.active.load(std::memory_order_acquire)) {
                if (c->cfg.server_threads == 0 && !c->server.poll(in->seg, 0, 1))
                    c->server.idle();
                if (cudaEventQuery(in->ev_done) == cudaErrorNotReady)
                    any = true;   /* finished programs are collected by gf_wait */
            }
        if (!any)
            return GF_OK;
        if (o && o->timeout_ns > 0 &&
            std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now() - t0).count() >
                o->timeout_ns)
            return GF_ETIMEDOUT;
        if (c->cfg.server_threads)
            std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

extern "C" GF_API int gf_get_stats(gf_ctx *c, gf_stats *out)
{
    if (!c || !out)
        return GF_EINVAL;
    std::lock_guard<std::mutex> g(c->stats_mu);
    *out = c->last;
    return GF_OK;
}
