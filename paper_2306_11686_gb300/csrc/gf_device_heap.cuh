/*
 * Device heap: malloc/free served natively on the GPU (paper Sec. 3.4).
 *
 * The paper offers a generic allocator (two lists under one lock) and a
 * "balanced" allocator (N x M chunks picked by thread and team id, one lock
 * per chunk, watermark reclaim).  This heap keeps the balanced allocator's goal
 * -- concurrent allocation without a global lock or list walks -- with
 * structures that suit 152 SMs:
 *
 *  - small sizes (<= 64 KiB) round up to 13 power-of-two classes;
 *  - the small region is cut into 256 KiB slabs; a slab belongs to one class and
 *    to the SM that first took it (slab metadata gives any block's size, which
 *    is the allocation tracking the paper needs for pointer lookup, Sec. 3.2);
 *  - each (SM, class) pair has 32 lock-free LIFOs of freed blocks, one per
 *    lane index (Treiber stacks with a 32-bit ABA tag in the 64-bit head), and
 *    a current slab served by an atomic bump counter;
 *  - every lane pops and pushes its own block on the stack of its lane index,
 *    so a warp's 32 requests are 32 independent CASes issued together: no
 *    list is walked (a single stack per (SM, class) would need a warp's leader
 *    to follow 32 dependent next-links, about 16 us, before its one CAS); the
 *    first attempts run a fixed number of times with no early exit, so the
 *    lanes stay together through contention;
 *  - lanes whose stack is empty are served together by one bump of the
 *    current slab (the leader of the lanes that ask for the same class,
 *    __match_any_sync); with no fresh slab left they take blocks from the
 *    other stacks of their SM, then of the other SMs, before failing;
 *  - sizes above 64 KiB take 64 KiB pages first-fit from a sorted extent list
 *    under one device lock (rare; the paper notes large serial-part
 *    allocations come from the initial thread, Sec. 3.4); the last freed
 *    large block waits in a one-entry cache for a request of its size.
 *
 * Out of memory returns NULL.  Blocks are 16-byte aligned.  Freeing a pointer
 * that the heap did not hand out is counted in n_bad_free and ignored.
 */
#ifndef GF_DEVICE_HEAP_CUH
#define GF_DEVICE_HEAP_CUH

namespace gfd {

__device__ __forceinline__ uint32_t size_class(uint64_t n)
{
    if (n <= 16)
        return 0;
    return 64 - __clzll((unsigned long long)(n - 1)) - GF_HEAP_MIN_SHIFT;   /* ceil(log2 n) - 4 */
}

struct slab_meta {
    uint32_t cls1;     /* class + 1, 0 = unassigned */
    uint32_t owner;    /* SM whose free stack receives this slab's blocks */
    uint32_t bump;     /* blocks handed out by bump */
    uint32_t pad;
};

__device__ __forceinline__ slab_meta *metas(gf_heap *H) { return (slab_meta *)H->slab_meta; }
__device__ __forceinline__ unsigned long long *heads(gf_heap *H) { return (unsigned long long *)H->free_heads; }
__device__ __forceinline__ uint32_t *curs(gf_heap *H) { return (uint32_t *)H->cur_slab; }

__device__ __forceinline__ uint64_t node_addr(gf_heap *H, uint32_t node1) { return H->slab_base + ((uint64_t)(node1 - 1) << 4); }
__device__ __forceinline__ uint32_t node_of(gf_heap *H, uint64_t addr) { return (uint32_t)((addr - H->slab_base) >> 4) + 1; }

__device__ __forceinline__ unsigned long long *stack_of(gf_heap *H, uint32_t sm, uint32_t cls, uint32_t sub)
{
    return &heads(H)[((size_t)sm * GF_HEAP_NCLASS + cls) * GF_HEAP_LANES + sub];
}

/* pop: three attempts with a fixed trip count (no early exit), so the lanes of
 * a warp leave together; 0 if empty or still contended */
static __device__ __forceinline__ uint64_t heap_pop1(gf_heap *H, uint32_t sm, uint32_t cls, uint32_t sub)
{
    unsigned long long *head = stack_of(H, sm, cls, sub);
    const uint32_t max1 = (uint32_t)(H->slab_bytes >> 4);
    uint64_t got = 0;
    bool stop = false;
#pragma unroll
    for (int attempt = 0; attempt < 3; attempt++) {
        if (!stop) {
            const unsigned long long h = *(volatile unsigned long long *)head;
            const uint32_t cur = (uint32_t)h;
            if (cur == 0) {
                stop = true;
            } else {
                const uint32_t nxt = *(volatile uint32_t *)node_addr(H, cur);
                if (nxt <= max1 && atomicCAS(head, h, ((h >> 32) + 1ull) << 32 | nxt) == h) {
                    got = node_addr(H, cur);
                    stop = true;
                }
            }
        }
    }
    if (got)
        __threadfence();
    return got;
}

/* push: three attempts with a fixed trip count, then (rarely) a retry loop;
 * false after a contention bound no sane run reaches */
static __device__ __forceinline__ bool heap_push1(gf_heap *H, uint32_t sm, uint32_t cls, uint32_t sub, uint64_t a,
                                                   uint32_t node)
{
    unsigned long long *head = stack_of(H, sm, cls, sub);
    bool done = false;
#pragma unroll
    for (int attempt = 0; attempt < 3; attempt++) {
        if (!done) {
            const unsigned long long h = *(volatile unsigned long long *)head;
            *(volatile uint32_t *)a = (uint32_t)h;
            __threadfence();
            done = atomicCAS(head, h, ((h >> 32) + 1ull) << 32 | node) == h;
        }
    }
    for (int attempt = 0; attempt < (1 << 20) && !done; attempt++) {
        const unsigned long long h = *(volatile unsigned long long *)head;
        *(volatile uint32_t *)a = (uint32_t)h;
        __threadfence();
        done = atomicCAS(head, h, ((h >> 32) + 1ull) << 32 | node) == h;
    }
    return done;
}

/* a block of (cls) from any stack other than (sm, cls, own): the rest of this
 * SM's stacks first, then the other SMs' */
static __device__ uint64_t heap_steal1(gf_heap *H, uint32_t sm, uint32_t cls, uint32_t own)
{
    for (uint32_t o = 0; o < GF_MAX_SM; o++) {
        const uint32_t s = (sm + o) % GF_MAX_SM;
        for (uint32_t j = o ? 0 : 1; j < GF_HEAP_LANES; j++) {
            const uint32_t sub = (own + j) % GF_HEAP_LANES;
            if ((uint32_t)*(volatile unsigned long long *)stack_of(H, s, cls, sub) == 0)
                continue;
            const uint64_t p = heap_pop1(H, s, cls, sub);
            if (p)
                return p;
        }
    }
    return 0;
}

/* current-slab word of (sm, cls): slab + 1, 0 = none yet, or one of these */
#define GF_CUR_BUSY 0xffffffffu   /* a warp is installing a fresh slab */
#define GF_CUR_DRY 0xfffffffeu    /* no fresh slab was left */

/* bump up to k - *got blocks from slab s into out[...] (lanes of *m in order) */
__device__ __forceinline__ void bump_from(gf_heap *H, uint32_t s, uint32_t bs, uint32_t cap, uint32_t k, uint32_t *got,
                                          uint64_t *out, uint32_t *m)
{
    if (*(volatile uint32_t *)&metas(H)[s].bump >= cap)   /* full: no atomic (the counter stays small) */
        return;
    const uint32_t want = k - *got;
    const uint32_t old = atomicAdd(&metas(H)[s].bump, want);
    if (old >= cap)
        return;
    const uint32_t take = want < cap - old ? want : cap - old;
    for (uint32_t j = 0; j < take; j++) {
        const uint32_t l = __ffs(*m) - 1;
        *m &= *m - 1;
        out[l] = H->slab_base + ((uint64_t)s << GF_SLAB_SHIFT) + (uint64_t)(old + j) * bs;
    }
    *got += take;
}

/*
 * Bump-allocate up to k blocks of (sm, cls) into out[...] for the lanes of
 * mask (in lane order) from the SM's current slab; when it is full, one warp
 * at a time installs a fresh slab (the word goes BUSY meanwhile, so no two
 * warps each install one and orphan the other's remainder); with no fresh
 * slab left, from the other SMs' current slabs.  Returns the number served.
 */
static __device__ uint32_t heap_bump(gf_heap *H, uint32_t sm, uint32_t cls, uint32_t k, uint64_t *out, uint32_t mask,
                                     int64_t timeout_ns)
{
    const uint32_t bs = 16u << cls, cap = (1u << GF_SLAB_SHIFT) / bs;
    uint32_t *cur = &curs(H)[sm * GF_HEAP_NCLASS + cls];
    uint32_t got = 0;
    uint32_t m = mask;
    backoff bo(timeout_ns);
    bool dry = false;
    while (got < k) {
        const uint32_t s1 = *(volatile uint32_t *)cur;
        if (s1 == GF_CUR_BUSY) {
            if (!bo.wait())
                break;
            continue;
        }
        if (s1 == GF_CUR_DRY) {
            dry = true;
            break;
        }
        if (s1) {
            bump_from(H, s1 - 1, bs, cap, k, &got, out, &m);
            if (got == k)
                break;
        }
        /* the current slab is full (or there is none): install a fresh one */
        if (atomicCAS(cur, s1, GF_CUR_BUSY) != s1)
            continue;                   /* another warp changed it: use theirs */
        const uint32_t ns = atomicAdd(&H->next_slab, 1u);
        if (ns >= H->nslabs) {
            atomicExch(cur, GF_CUR_DRY);
            dry = true;
            break;
        }
        const uint32_t want = k - got < cap ? k - got : cap;
        slab_meta *mt = &metas(H)[ns];
        mt->cls1 = cls + 1;
        mt->owner = sm;
        mt->bump = want;
        for (uint32_t j = 0; j < want; j++) {
            const uint32_t l = __ffs(m) - 1;
            m &= m - 1;
            out[l] = H->slab_base + ((uint64_t)ns << GF_SLAB_SHIFT) + (uint64_t)j * bs;
        }
        got += want;
        __threadfence();
        atomicExch(cur, ns + 1);
    }
    if (dry) {
        /* no fresh slab left: bump from the other SMs' current slabs of this class */
        for (uint32_t o = 1; o < GF_MAX_SM && got < k; o++) {
            const uint32_t t1 = *(volatile uint32_t *)&curs(H)[((sm + o) % GF_MAX_SM) * GF_HEAP_NCLASS + cls];
            if (t1 == 0 || t1 >= GF_CUR_DRY)
                continue;
            bump_from(H, t1 - 1, bs, cap, k, &got, out, &m);
        }
    }
    return got;
}

/* ---------------------------------------------------------------- large path */
/* the large path's lock: an acquiring compare-and-swap takes it and a
 * releasing store gives it back, which order the extent table's reads and
 * writes inside it without full fences */
__device__ __forceinline__ uint32_t cas_acquire_gpu(uint32_t *p, uint32_t cmp, uint32_t val)
{
    uint32_t old;
    asm volatile("atom.acquire.gpu.global.cas.b32 %0, [%1], %2, %3;"
                 : "=r"(old) : "l"(p), "r"(cmp), "r"(val) : "memory");
    return old;
}
static __device__ bool large_lock(gf_heap *H, int64_t timeout_ns)
{
    backoff bo(timeout_ns);
    while (cas_acquire_gpu(&H->large_lock, 0u, 1u) != 0u)
        if (!bo.wait())
            return false;
    return true;
}
static __device__ void large_unlock(gf_heap *H)
{
    st_rel_gpu(&H->large_lock, 0u);
}

static __device__ void *large_alloc(gf_heap *H, uint64_t n, int64_t timeout_ns)
{
    const uint32_t need = (uint32_t)((n + (1ull << GF_PAGE_SHIFT) - 1) >> GF_PAGE_SHIFT);
    if (!large_lock(H, timeout_ns))
        return nullptr;
    volatile uint64_t *ext = (volatile uint64_t *)H->large_ext;   /* page | npages << 32 */
    volatile uint32_t *sz = (volatile uint32_t *)H->large_size;
    const uint32_t cnt = *(volatile uint32_t *)&H->large_next;
    void *r = nullptr;
    for (uint32_t k = 0; k < cnt; k++) {
        const uint64_t e = ext[k];
        const uint32_t pg = (uint32_t)e, np = (uint32_t)(e >> 32);
        if (np >= need) {
            if (np == need) {
                for (uint32_t q = k; q + 1 < cnt; q++)
                    ext[q] = ext[q + 1];
                *(volatile uint32_t *)&H->large_next = cnt - 1;
            } else {
                ext[k] = (uint64_t)(pg + need) | ((uint64_t)(np - need) << 32);
            }
            sz[pg] = need;
            r = (void *)(H->large_base + ((uint64_t)pg << GF_PAGE_SHIFT));
            break;
        }
    }
    large_unlock(H);
    return r;
}

/* pages [pg, pg + np) back into the sorted extent table, merged with the
 * free extents around them (each read from the table once: the lock holder
 * is the only writer, so the copies stay current) */
static __device__ bool large_insert(gf_heap *H, uint32_t pg, uint32_t np, int64_t timeout_ns)
{
    if (!large_lock(H, timeout_ns))
        return false;
    volatile uint64_t *ext = (volatile uint64_t *)H->large_ext;
    uint32_t cnt = *(volatile uint32_t *)&H->large_next;
    uint32_t k = 0;
    uint64_t prev = 0, cur = 0;
    for (; k < cnt; k++) {
        cur = ext[k];
        if ((uint32_t)cur >= pg)
            break;
        prev = cur;
    }
    const bool merge_prev = k > 0 && (uint32_t)prev + (uint32_t)(prev >> 32) == pg;
    const bool merge_next = k < cnt && pg + np == (uint32_t)cur;
    if (merge_prev && merge_next) {
        const uint32_t len = (uint32_t)(prev >> 32) + np + (uint32_t)(cur >> 32);
        ext[k - 1] = (uint64_t)(uint32_t)prev | ((uint64_t)len << 32);
        for (uint32_t q = k; q + 1 < cnt; q++)
            ext[q] = ext[q + 1];
        cnt--;
    } else if (merge_prev) {
        ext[k - 1] = (uint64_t)(uint32_t)prev | ((uint64_t)((uint32_t)(prev >> 32) + np) << 32);
    } else if (merge_next) {
        ext[k] = (uint64_t)pg | ((uint64_t)(np + (uint32_t)(cur >> 32)) << 32);
    } else if (cnt < GF_LARGE_EXT_MAX) {
        for (uint32_t q = cnt; q > k; q--)
            ext[q] = ext[q - 1];
        ext[k] = (uint64_t)pg | ((uint64_t)np << 32);
        cnt++;
    }   /* else: extent table full, the pages leak (counted as live) */
    *(volatile uint32_t *)&H->large_next = cnt;
    large_unlock(H);
    return true;
}

/*
 * The last freed large block waits in a one-entry cache (its page count in
 * the high word) instead of going back to the extent table: a program that
 * frees a block and then asks for one of the same size -- a scratch buffer
 * per iteration -- gets it back with one exchange, and the free is one
 * exchange too, neither taking the lock.  A request of another size, or one
 * the table cannot serve, first returns the cached block to the table, so
 * first fit still sees every free page merged.
 */
static __device__ void *large_malloc(gf_heap *H, uint64_t n, int64_t timeout_ns)
{
    const uint32_t need = (uint32_t)((n + (1ull << GF_PAGE_SHIFT) - 1) >> GF_PAGE_SHIFT);
    unsigned long long *cache = (unsigned long long *)&H->large_cache;
    unsigned long long c = atomicExch(cache, 0ull);
    if (c) {
        if ((uint32_t)(c >> 32) == need) {
            const uint32_t pg = (uint32_t)c;
            ((volatile uint32_t *)H->large_size)[pg] = need;
            return (void *)(H->large_base + ((uint64_t)pg << GF_PAGE_SHIFT));
        }
        large_insert(H, (uint32_t)c, (uint32_t)(c >> 32), timeout_ns);
    }
    void *p = large_alloc(H, n, timeout_ns);
    if (!p && (c = atomicExch(cache, 0ull)) != 0ull &&
        large_insert(H, (uint32_t)c, (uint32_t)(c >> 32), timeout_ns))
        p = large_alloc(H, n, timeout_ns);
    return p;
}

/* free of a large block: 0 pages if addr is not the start of a live one */
static __device__ uint32_t large_release(gf_heap *H, uint64_t addr, int64_t timeout_ns)
{
    const uint64_t off = addr - H->large_base;
    if (off & ((1ull << GF_PAGE_SHIFT) - 1))
        return 0;
    const uint32_t pg = (uint32_t)(off >> GF_PAGE_SHIFT);
    /* claim the block: of two frees of one pointer only one sees its size */
    const uint32_t np = atomicExch(&((uint32_t *)H->large_size)[pg], 0u);
    if (np == 0)
        return 0;
    const unsigned long long old =
        atomicExch((unsigned long long *)&H->large_cache, (unsigned long long)pg | ((unsigned long long)np << 32));
    if (old && !large_insert(H, (uint32_t)old, (uint32_t)(old >> 32), timeout_ns))
        set_error(GF_ETIMEDOUT);              /* the lock never came: those pages leak */
    return np;
}

} // namespace gfd

/* ====================================================================== malloc / free */
static __device__ __forceinline__ void *gf_malloc_body(size_t n)
{
    gf_state *S = gfd::s_st;
    gf_heap *H = &S->heap;
    if (n > GF_HEAP_MAX_SMALL) {
        const unsigned long long pb = ((unsigned long long)n + (1ull << GF_PAGE_SHIFT) - 1) &
                                      ~((1ull << GF_PAGE_SHIFT) - 1);   /* whole pages, as free counts them */
        /* counted before the allocation, so this atomic's round trip overlaps
         * the allocation's own (taken back if it fails; a concurrent failed
         * request can then show in another's high-water reading) */
        const unsigned long long live = atomicAdd((unsigned long long *)&H->live_bytes, pb) + pb;
        void *p = gfd::large_malloc(H, n, S->timeout_ns);
        atomicAdd((unsigned long long *)(p ? &H->n_alloc : &H->n_fail), 1ull);
        if (p)
            atomicMax((unsigned long long *)&H->high_water, live);
        else
            atomicAdd((unsigned long long *)&H->live_bytes, 0ull - pb);
        return p;
    }
    const uint32_t cls = gfd::size_class(n ? n : 1);
    const uint32_t lane = gfd::lane_id(), warp = threadIdx.x >> 5;
    const uint32_t active = __activemask();
    const uint32_t grp = __match_any_sync(active, cls);
    const uint32_t leader = __ffs(grp) - 1;
    const uint32_t sm = gfd::smid() % GF_MAX_SM;
    uint64_t *out = gfd::s_xfer[warp];
    /* every lane: its own stack */
    uint64_t p = gfd::heap_pop1(H, sm, cls, lane);
    /* the lanes left empty-handed: one bump of the current slab per class */
    const uint32_t gmiss = __ballot_sync(grp, p == 0) & grp;
    if (gmiss) {
        if (lane == leader) {
            const uint32_t got = gfd::heap_bump(H, sm, cls, __popc(gmiss), out, gmiss, S->timeout_ns);
            uint32_t r = gmiss;
            for (uint32_t j = 0; j < got; j++)
                r &= r - 1;
            for (; r; r &= r - 1)
                out[__ffs(r) - 1] = 0;
            __threadfence_block();
        }
        __syncwarp(grp);
        if (!p)
            p = out[lane];
        __syncwarp(grp);
        if (!p)                        /* no fresh slab: other stacks before failing */
            p = gfd::heap_steal1(H, sm, cls, lane);
    }
    const uint32_t ok = __ballot_sync(grp, p != 0) & grp;
    if (lane == leader) {
        const uint32_t got = __popc(ok), k = __popc(grp);
        const unsigned long long bs = 16ull << cls;
        atomicAdd((unsigned long long *)&H->n_alloc, (unsigned long long)got);
        if (got < k)
            atomicAdd((unsigned long long *)&H->n_fail, (unsigned long long)(k - got));
        const unsigned long long live = atomicAdd((unsigned long long *)&H->live_bytes, bs * got) + bs * got;
        atomicMax((unsigned long long *)&H->high_water, live);
    }
    __syncwarp(grp);                   /* the group leaves with its leader, so a following
                                        * warp-aggregated call (printf) finds it converged */
    return (void *)p;
}

static __device__ __forceinline__ void gf_free_body(void *p)
{
    if (!p)
        return;
    gf_state *S = gfd::s_st;
    gf_heap *H = &S->heap;
    const uint64_t a = (uint64_t)p;
    const uint32_t lane = gfd::lane_id();
    uint32_t key = 0xffffffffu - lane;          /* lanes off the slab path stay alone */
    uint32_t cls = 0, owner = 0;
    bool small = false;
    if (a >= H->slab_base && a < H->slab_base + H->slab_bytes) {
        const uint32_t s = (uint32_t)((a - H->slab_base) >> GF_SLAB_SHIFT);
        const uint32_t c1 = *(volatile uint32_t *)&gfd::metas(H)[s].cls1;
        if (c1 && ((a - H->slab_base) & ((16ull << (c1 - 1)) - 1)) == 0) {
            cls = c1 - 1;
            owner = *(volatile uint32_t *)&gfd::metas(H)[s].owner;
            key = owner * GF_HEAP_NCLASS + cls;
            small = true;
        }
    }
    const uint32_t active = __activemask();
    const uint32_t grp = __match_any_sync(active, key);
    if (!small) {
        if (a >= H->large_base && a < H->large_base + H->large_bytes) {
            const uint32_t np = gfd::large_release(H, a, S->timeout_ns);
            if (np) {
                const uint64_t bytes = (uint64_t)np << GF_PAGE_SHIFT;
                atomicAdd((unsigned long long *)&H->n_free, 1ull);
                atomicAdd((unsigned long long *)&H->live_bytes, (unsigned long long)(0ull - bytes));
                return;
            }
        }
        atomicAdd((unsigned long long *)&H->n_bad_free, 1ull);
        return;
    }
    /* every lane pushes its block on the stack of its lane index */
    const bool pushed = gfd::heap_push1(H, owner, cls, lane, a, gfd::node_of(H, a));
    if (!pushed)                       /* contention beyond reason: the block leaks */
        gfd::set_error(GF_ETIMEDOUT);
    const uint32_t done = __ballot_sync(grp, pushed) & grp;
    if (lane == __ffs(grp) - 1) {
        const unsigned long long bs = 16ull << cls;
        const unsigned long long nd = (unsigned long long)__popc(done);
        atomicAdd((unsigned long long *)&H->n_free, nd);
        atomicAdd((unsigned long long *)&H->live_bytes, 0ull - bs * nd);
    }
    __syncwarp(grp);                   /* leave together, as in gf_malloc */
}

/* malloc / free; the initial thread's time in them is counted (st_heap_ns),
 * so a program's serial heap cost shows apart from its regions and RPCs */
static __device__ __noinline__ void *gf_malloc(size_t n)
{
    const bool timed = gfd::is_initial_thread();
    const uint64_t t0 = timed ? gfd::now_ns() : 0;
    void *p = gf_malloc_body(n);
    if (timed)
        atomicAdd((unsigned long long *)&gfd::s_st->st_heap_ns, (unsigned long long)(gfd::now_ns() - t0));
    return p;
}

static __device__ __noinline__ void gf_free(void *p)
{
    const bool timed = gfd::is_initial_thread();
    const uint64_t t0 = timed ? gfd::now_ns() : 0;
    gf_free_body(p);
    if (timed)
        atomicAdd((unsigned long long *)&gfd::s_st->st_heap_ns, (unsigned long long)(gfd::now_ns() - t0));
}

/* size of the heap block holding p (0 if p is not a live heap block start) */
__device__ inline uint64_t gf_heap_block_size(const void *p)
{
    gf_heap *H = &gfd::s_st->heap;
    const uint64_t a = (uint64_t)p;
    if (a >= H->slab_base && a < H->slab_base + H->slab_bytes) {
        const uint32_t s = (uint32_t)((a - H->slab_base) >> GF_SLAB_SHIFT);
        const uint32_t c1 = *(volatile uint32_t *)&gfd::metas(H)[s].cls1;
        return c1 ? (16ull << (c1 - 1)) : 0;
    }
    if (a >= H->large_base && a < H->large_base + H->large_bytes)
        return (uint64_t)(*(volatile uint32_t *)&((uint32_t *)H->large_size)[(a - H->large_base) >> GF_PAGE_SHIFT])
               << GF_PAGE_SHIFT;
    return 0;
}

#endif
