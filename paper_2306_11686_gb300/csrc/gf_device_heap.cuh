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
 *  - each (SM, class) pair has a lock-free LIFO of freed blocks (Treiber stack
 *    with a 32-bit ABA tag in the 64-bit head) and a current slab served by an
 *    atomic bump counter;
 *  - a warp's lanes that ask for the same class are served by one leader
 *    (__match_any_sync): one CAS pops up to 32 blocks, one atomicAdd bumps up
 *    to 32; frees are chained per (owner SM, class) and pushed with one CAS;
 *  - sizes above 64 KiB take 64 KiB pages first-fit from a sorted extent list
 *    under one device lock (rare; the paper notes large serial-part
 *    allocations come from the initial thread, Sec. 3.4).
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

/* pop up to k blocks of (sm, cls); writes addresses to out[member lanes in mask order] */
static __device__ uint32_t heap_pop(gf_heap *H, uint32_t sm, uint32_t cls, uint32_t k, uint64_t *out, uint32_t mask)
{
    unsigned long long *head = &heads(H)[sm * GF_HEAP_NCLASS + cls];
    const uint32_t max1 = (uint32_t)(H->slab_bytes >> 4);
    for (int attempt = 0; attempt < 64; attempt++) {
        const unsigned long long h = *(volatile unsigned long long *)head;
        uint32_t cur = (uint32_t)h;
        if (cur == 0)
            return 0;
        uint32_t cnt = 0;
        uint32_t m = mask;
        bool ok = true;
        uint32_t after = 0;
        for (;;) {
            const uint32_t l = __ffs(m) - 1;
            m &= m - 1;
            out[l] = node_addr(H, cur);
            cnt++;
            const uint32_t nxt = *(volatile uint32_t *)node_addr(H, cur);
            if (nxt > max1) {          /* block reused under us: the CAS below must fail */
                ok = false;
                break;
            }
            if (cnt == k || nxt == 0) {
                after = nxt;
                break;
            }
            cur = nxt;
        }
        if (!ok)
            continue;
        const unsigned long long nh = ((h >> 32) + 1ull) << 32 | after;
        if (atomicCAS(head, h, nh) == h) {
            __threadfence();
            return cnt;
        }
    }
    return 0;
}

/* bump-allocate up to k fresh blocks for (sm, cls) into out[...] after the first `skip` members */
static __device__ uint32_t heap_bump(gf_heap *H, uint32_t sm, uint32_t cls, uint32_t k, uint64_t *out, uint32_t mask)
{
    const uint32_t bs = 16u << cls, cap = (1u << GF_SLAB_SHIFT) / bs;
    uint32_t *cur = &curs(H)[sm * GF_HEAP_NCLASS + cls];
    uint32_t got = 0;
    uint32_t m = mask;
    for (int attempt = 0; attempt < 40 && got < k; attempt++) {
        const uint32_t s1 = *(volatile uint32_t *)cur;
        if (s1) {
            const uint32_t s = s1 - 1;
            const uint32_t want = k - got;
            const uint32_t old = atomicAdd(&metas(H)[s].bump, want);
            if (old < cap) {
                const uint32_t take = want < cap - old ? want : cap - old;
                for (uint32_t j = 0; j < take; j++) {
                    const uint32_t l = __ffs(m) - 1;
                    m &= m - 1;
                    out[l] = H->slab_base + ((uint64_t)s << GF_SLAB_SHIFT) + (uint64_t)(old + j) * bs;
                }
                got += take;
                if (got == k)
                    break;
            }
        }
        /* current slab exhausted: take a fresh one and make it current */
        const uint32_t ns = atomicAdd(&H->next_slab, 1u);
        if (ns >= H->nslabs) {
            /* no fresh slab left: bump from other SMs' current slabs of this class */
            for (uint32_t o = 1; o < GF_MAX_SM && got < k; o++) {
                const uint32_t t1 = *(volatile uint32_t *)&curs(H)[((sm + o) % GF_MAX_SM) * GF_HEAP_NCLASS + cls];
                if (!t1)
                    continue;
                const uint32_t want = k - got;
                const uint32_t old = atomicAdd(&metas(H)[t1 - 1].bump, want);
                if (old >= cap)
                    continue;
                const uint32_t take = want < cap - old ? want : cap - old;
                for (uint32_t j = 0; j < take; j++) {
                    const uint32_t l = __ffs(m) - 1;
                    m &= m - 1;
                    out[l] = H->slab_base + ((uint64_t)(t1 - 1) << GF_SLAB_SHIFT) + (uint64_t)(old + j) * bs;
                }
                got += take;
            }
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
    return got;
}

/* ---------------------------------------------------------------- large path */
static __device__ bool large_lock(gf_heap *H, int64_t timeout_ns)
{
    backoff bo(timeout_ns);
    while (atomicCAS(&H->large_lock, 0u, 1u) != 0u)
        if (!bo.wait())
            return false;
    __threadfence();
    return true;
}
static __device__ void large_unlock(gf_heap *H)
{
    __threadfence();
    atomicExch(&H->large_lock, 0u);
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

static __device__ bool large_free(gf_heap *H, uint64_t addr, int64_t timeout_ns)
{
    const uint64_t off = addr - H->large_base;
    if (off & ((1ull << GF_PAGE_SHIFT) - 1))
        return false;
    const uint32_t pg = (uint32_t)(off >> GF_PAGE_SHIFT);
    if (!large_lock(H, timeout_ns))
        return false;
    volatile uint64_t *ext = (volatile uint64_t *)H->large_ext;
    volatile uint32_t *sz = (volatile uint32_t *)H->large_size;
    const uint32_t np = sz[pg];
    if (np == 0) {
        large_unlock(H);
        return false;
    }
    sz[pg] = 0;
    uint32_t cnt = *(volatile uint32_t *)&H->large_next;
    uint32_t k = 0;
    while (k < cnt && (uint32_t)ext[k] < pg)
        k++;
    uint32_t start = pg, len = np;
    const bool merge_prev = k > 0 && (uint32_t)ext[k - 1] + (uint32_t)(ext[k - 1] >> 32) == pg;
    const bool merge_next = k < cnt && pg + np == (uint32_t)ext[k];
    if (merge_prev && merge_next) {
        start = (uint32_t)ext[k - 1];
        len = (uint32_t)(ext[k - 1] >> 32) + np + (uint32_t)(ext[k] >> 32);
        ext[k - 1] = (uint64_t)start | ((uint64_t)len << 32);
        for (uint32_t q = k; q + 1 < cnt; q++)
            ext[q] = ext[q + 1];
        cnt--;
    } else if (merge_prev) {
        ext[k - 1] = (uint64_t)(uint32_t)ext[k - 1] | ((uint64_t)((uint32_t)(ext[k - 1] >> 32) + np) << 32);
    } else if (merge_next) {
        ext[k] = (uint64_t)pg | ((uint64_t)(np + (uint32_t)(ext[k] >> 32)) << 32);
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

} // namespace gfd

/* ====================================================================== malloc / free */
static __device__ __noinline__ void *gf_malloc(size_t n)
{
    gf_state *S = gfd::s_st;
    gf_heap *H = &S->heap;
    if (n > GF_HEAP_MAX_SMALL) {
        void *p = gfd::large_alloc(H, n, S->timeout_ns);
        atomicAdd((unsigned long long *)(p ? &H->n_alloc : &H->n_fail), 1ull);
        if (p) {
            const unsigned long long pb = ((unsigned long long)n + (1ull << GF_PAGE_SHIFT) - 1) &
                                          ~((1ull << GF_PAGE_SHIFT) - 1);   /* whole pages, as free counts them */
            const unsigned long long live = atomicAdd((unsigned long long *)&H->live_bytes, pb) + pb;
            atomicMax((unsigned long long *)&H->high_water, live);
        }
        return p;
    }
    const uint32_t cls = gfd::size_class(n ? n : 1);
    const uint32_t lane = gfd::lane_id(), warp = threadIdx.x >> 5;
    const uint32_t active = __activemask();
    const uint32_t grp = __match_any_sync(active, cls);
    const uint32_t leader = __ffs(grp) - 1;
    uint64_t *out = gfd::s_xfer[warp];
    if (lane == leader) {
        const uint32_t k = __popc(grp);
        const uint32_t sm = gfd::smid() % GF_MAX_SM;
        uint32_t got = gfd::heap_pop(H, sm, cls, k, out, grp);
        uint32_t rest = grp;
        for (uint32_t j = 0; j < got; j++)
            rest &= rest - 1;
        if (got < k)
            got += gfd::heap_bump(H, sm, cls, k - got, out, rest);
        if (got < k) {                 /* drain other SMs' free stacks before failing */
            for (uint32_t o = 1; o < GF_MAX_SM && got < k; o++) {
                uint32_t r2 = grp;
                for (uint32_t j = 0; j < got; j++)
                    r2 &= r2 - 1;
                got += gfd::heap_pop(H, (sm + o) % GF_MAX_SM, cls, k - got, out, r2);
            }
        }
        uint32_t r3 = grp;
        for (uint32_t j = 0; j < got; j++)
            r3 &= r3 - 1;
        for (; r3; r3 &= r3 - 1)
            out[__ffs(r3) - 1] = 0;
        const unsigned long long bs = 16ull << cls;
        atomicAdd((unsigned long long *)&H->n_alloc, (unsigned long long)got);
        if (got < k)
            atomicAdd((unsigned long long *)&H->n_fail, (unsigned long long)(k - got));
        const unsigned long long live = atomicAdd((unsigned long long *)&H->live_bytes, bs * got) + bs * got;
        atomicMax((unsigned long long *)&H->high_water, live);
        __threadfence_block();
    }
    __syncwarp(grp);
    void *p = (void *)gfd::s_xfer[warp][lane];
    __syncwarp(grp);
    return p;
}

static __device__ __noinline__ void gf_free(void *p)
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
            const uint32_t pg = (uint32_t)((a - H->large_base) >> GF_PAGE_SHIFT);
            const uint64_t bytes = (uint64_t)(*(volatile uint32_t *)&((uint32_t *)H->large_size)[pg]) << GF_PAGE_SHIFT;
            if (gfd::large_free(H, a, S->timeout_ns)) {
                atomicAdd((unsigned long long *)&H->n_free, 1ull);
                atomicAdd((unsigned long long *)&H->live_bytes, (unsigned long long)(0ull - bytes));
                return;
            }
        }
        atomicAdd((unsigned long long *)&H->n_bad_free, 1ull);
        return;
    }
    /* chain this group's blocks in lane order and push the chain with one CAS */
    const uint32_t node = gfd::node_of(H, a);
    const uint32_t higher = grp & ~((2u << lane) - 1u);
    const uint32_t next_lane = higher ? __ffs(higher) - 1 : lane;
    const uint32_t next_node = __shfl_sync(grp, node, next_lane);
    const uint32_t last_lane = 31 - __clz(grp);
    const uint32_t leader = __ffs(grp) - 1;
    const uint32_t first_node = __shfl_sync(grp, node, leader);
    if (higher)
        *(volatile uint32_t *)p = next_node;
    const uint32_t last_node = __shfl_sync(grp, node, last_lane);
    __threadfence();
    __syncwarp(grp);
    if (lane == leader) {
        const uint32_t n = __popc(grp);
        const unsigned long long bs = 16ull << cls;
        atomicAdd((unsigned long long *)&H->n_free, (unsigned long long)n);
        atomicAdd((unsigned long long *)&H->live_bytes, (unsigned long long)(0ull - bs * n));
        unsigned long long *head = &gfd::heads(H)[owner * GF_HEAP_NCLASS + cls];
        volatile uint32_t *lastp = (volatile uint32_t *)gfd::node_addr(H, last_node);
        bool pushed = false;
        for (int attempt = 0; attempt < (1 << 20) && !pushed; attempt++) {
            const unsigned long long h = *(volatile unsigned long long *)head;
            *lastp = (uint32_t)h;
            __threadfence();
            const unsigned long long nh = ((h >> 32) + 1ull) << 32 | first_node;
            pushed = atomicCAS(head, h, nh) == h;
        }
        if (!pushed)                          /* contention beyond reason: the blocks leak */
            gfd::set_error(GF_ETIMEDOUT);
    }
    __syncwarp(grp);
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
