/*
 * The paper's two device allocators (Sec. 3.4), rebuilt as comparators for
 * the runtime's slab heap.
 *
 * Balanced allocator (Sec. 3.4, Fig. 5): the arena is cut into N x M chunks;
 * a thread uses chunk (team mod M, thread mod N), so threads that never share
 * a chunk never contend; each chunk has its own lock.  The first of the N
 * chunks of every team slot is `ratio` times larger, since the initial thread
 * (thread 0) does the serial part's big allocations.  Entries are laid out
 * bottom-up with their metadata in band: a 16-byte header {size, prev
 * offset, in-use} before the user bytes.  Allocation bumps the chunk's
 * watermark ("top"); when the chunk is full it walks the entries for a free
 * one that fits.  Free marks the entry; if it is the top entry the watermark
 * drops to its start, and keeps dropping over entries below that were freed
 * earlier (chained reclaim).
 *
 * Generic allocator (Sec. 3.4): one lock; an allocation list and a free list
 * threaded through 16-byte headers; malloc takes the first free entry that
 * fits, else bumps the arena; free moves the entry to the free list.  Any
 * thread can use the whole heap, but every call is serialised.
 *
 * Both use the instance's heap arena and a small state area; all lock spins
 * are bounded and fail (NULL / ignored free) instead of hanging.
 */
#ifndef GF_PAPER_ALLOC_CUH
#define GF_PAPER_ALLOC_CUH

#include "gf_device.cuh"

namespace gfpa {

struct hdr {                     /* in-band entry header */
    uint32_t size;               /* user bytes (multiple of 16) */
    uint32_t prev;               /* offset of the previous entry's header + 1 (0 = bottom) */
    uint32_t used;
    uint32_t next;               /* generic allocator: list link (offset + 1) */
};

struct chunk_state {
    uint32_t lock, top;          /* watermark: offset of the first free byte of the chunk */
    uint32_t last;               /* offset + 1 of the top entry's header (0 = empty) */
    uint32_t pad;
};

struct balanced {
    unsigned char *arena;        /* N x M chunks */
    chunk_state *st;             /* N x M states */
    uint32_t N, M, chunk, ratio; /* chunk = bytes of an ordinary chunk */
    __device__ uint64_t slot_bytes() const { return (uint64_t)(ratio + N - 1) * chunk; }
    __device__ unsigned char *base(uint32_t n, uint32_t m) const
    {
        return arena + m * slot_bytes() + (n == 0 ? 0 : (uint64_t)(ratio + n - 1) * chunk);
    }
    __device__ uint32_t cap(uint32_t n) const { return n == 0 ? ratio * chunk : chunk; }
};

__device__ inline bool lock(uint32_t *l)
{
    for (int k = 0; k < (1 << 22); k++) {
        if (atomicCAS(l, 0u, 1u) == 0u) {
            __threadfence();
            return true;
        }
        __nanosleep(32);
    }
    return false;
}
__device__ inline void unlock(uint32_t *l)
{
    __threadfence();
    atomicExch(l, 0u);
}

__device__ inline void *balanced_malloc(const balanced &B, uint32_t tid, uint32_t team, uint64_t n)
{
    const uint32_t ni = tid % B.N, mi = team % B.M;
    chunk_state *cs = &B.st[mi * B.N + ni];
    unsigned char *base = B.base(ni, mi);
    const uint32_t need = (uint32_t)((n + 15) & ~15ull), cap = B.cap(ni);
    if (!lock(&cs->lock))
        return nullptr;
    void *r = nullptr;
    volatile chunk_state *v = cs;
    const uint32_t top = v->top;
    if ((uint64_t)top + 16 + need <= cap) {              /* bump the watermark */
        volatile hdr *h = (volatile hdr *)(base + top);
        h->size = need;
        h->prev = v->last;
        h->used = 1;
        v->last = top + 1;
        v->top = top + 16 + need;
        r = base + top + 16;
    } else {                                              /* full: walk down for a free entry that fits */
        uint32_t e = v->last;
        for (int guard = 0; e && guard < (1 << 20); guard++) {
            volatile hdr *h = (volatile hdr *)(base + e - 1);
            if (!h->used && h->size >= need) {
                h->used = 1;
                r = (void *)(base + e - 1 + 16);
                break;
            }
            e = h->prev;
        }
    }
    unlock(&cs->lock);
    return r;
}

__device__ inline void balanced_free(const balanced &B, uint32_t tid, uint32_t team, void *p)
{
    if (!p)
        return;
    const uint32_t ni = tid % B.N, mi = team % B.M;
    chunk_state *cs = &B.st[mi * B.N + ni];
    unsigned char *base = B.base(ni, mi);
    const uint32_t off = (uint32_t)((unsigned char *)p - base) - 16;
    if (!lock(&cs->lock))
        return;
    volatile chunk_state *v = cs;
    volatile hdr *h = (volatile hdr *)(base + off);
    h->used = 0;
    /* watermark reclaim: while the top entry is unused, drop the watermark below it */
    for (int guard = 0; v->last && guard < (1 << 20); guard++) {
        volatile hdr *t = (volatile hdr *)(base + v->last - 1);
        if (t->used)
            break;
        v->top = v->last - 1;
        v->last = t->prev;
    }
    unlock(&cs->lock);
}

struct generic {
    unsigned char *arena;
    uint64_t bytes;
    chunk_state *st;             /* st->lock, st->top (bump), st->last = free-list head (offset + 1) */
};

__device__ inline void *generic_malloc(const generic &G, uint64_t n)
{
    const uint32_t need = (uint32_t)((n + 15) & ~15ull);
    if (!lock(&G.st->lock))
        return nullptr;
    volatile chunk_state *v = G.st;
    void *r = nullptr;
    uint32_t prev = 0, e = v->last;
    for (int guard = 0; e && guard < (1 << 22); guard++) {       /* first fit on the free list */
        volatile hdr *h = (volatile hdr *)(G.arena + e - 1);
        if (h->size >= need) {
            if (prev)
                ((volatile hdr *)(G.arena + prev - 1))->next = h->next;
            else
                v->last = h->next;
            h->used = 1;
            r = (void *)(G.arena + e - 1 + 16);
            break;
        }
        prev = e;
        e = h->next;
    }
    if (!r && (uint64_t)v->top + 16 + need <= G.bytes) {
        volatile hdr *h = (volatile hdr *)(G.arena + v->top);
        h->size = need;
        h->used = 1;
        h->next = 0;
        r = (void *)(G.arena + v->top + 16);
        v->top = v->top + 16 + need;
    }
    unlock(&G.st->lock);
    return r;
}

__device__ inline void generic_free(const generic &G, void *p)
{
    if (!p)
        return;
    const uint32_t off = (uint32_t)((unsigned char *)p - G.arena) - 16;
    if (!lock(&G.st->lock))
        return;
    volatile hdr *h = (volatile hdr *)(G.arena + off);
    h->used = 0;
    h->next = G.st->last;
    ((volatile chunk_state *)G.st)->last = off + 1;
    unlock(&G.st->lock);
}

} // namespace gfpa

#endif
