/*
 * Device side of host RPC (paper Sec. 3.2, Fig. 4 and Sec. 5.2).
 *
 * A call site packs its arguments into a lane record: value arguments
 * (integers, doubles, opaque handles such as FILE*) as tagged 8-byte words,
 * reference arguments (strings, small objects with a read / write / readwrite
 * mode) as bytes in the record's tail, large objects as a device address that
 * the host moves by DMA.  The opcode names the host landing pad.
 *
 * Warp aggregation: the lanes of a warp that call the same opcode with the
 * same format and argument signature are grouped with __match_any_sync; their
 * leader claims ONE ring slot, every lane writes its record at its rank's
 * offset, the leader publishes the slot with a system-scope release store,
 * waits (bounded) for the host's release of the returns, and each lane reads
 * its own return value.  With aggregation off every lane takes its own slot,
 * which is the per-thread RPC of the paper.
 *
 * Format strings are shipped inside the slot the first time and cached on the
 * host by device address afterwards (the paper copies them on every call).
 * A format string must therefore not change while the context lives (string
 * literals are the intended use).
 *
 * Deferred calls: a printf-family call from the initial thread is published
 * without waiting for the host.  Its result comes back as a gf_call_result,
 * which waits when it is converted to int; a call whose result the program
 * never reads is collected (waited for, its slot given back) at the initial
 * thread's next RPC or when main returns.  At most one call is outstanding,
 * so the initial thread's calls still reach the host in program order, and
 * the serial part runs on (the next sweep, say) while the host formats the
 * text.  Calls from a region's threads complete before they return.
 *
 * After the first device-side error of a program (a ring or reply timeout),
 * every later call fails at once with that error instead of waiting out its
 * own timeout on a slot the host may still be writing into.
 */
#ifndef GF_DEVICE_RPC_CUH
#define GF_DEVICE_RPC_CUH

#define GF_INLINE_BLOB_MAX 2048u    /* larger objects move by DMA */

namespace gfd {

struct argpack {
    uint32_t n, tail;
    char tag[GF_MAX_ARGS];
    uint64_t word[GF_MAX_ARGS];
    const void *src[GF_MAX_ARGS];
    uint32_t len[GF_MAX_ARGS];
    __device__ argpack() : n(0), tail(0) {}
    __device__ void val(char t, uint64_t w)
    {
        if (n < GF_MAX_ARGS) {
            tag[n] = t;
            word[n] = w;
            src[n] = nullptr;
            len[n] = 0;
            n++;
        }
    }
    /* p = start of the underlying object, bytes = its size, off = the
     * argument pointer's offset inside it (paper Fig. 4c: addRefArg(ptr,
     * mode, size, offset)) */
    __device__ void blob(char t, const void *p, uint32_t bytes, uint32_t off = 0)
    {
        if (n < GF_MAX_ARGS) {
            tag[n] = t;
            word[n] = ((uint64_t)bytes << 32) | ((uint64_t)(off & 0xffffu) << 16) | tail;   /* bytes | off | tail */
            src[n] = p;
            len[n] = bytes;
            tail += (bytes + 7u) & ~7u;
            n++;
        }
    }
    __device__ uint32_t bytes() const { return 16u + ((n + 7u) & ~7u) + 8u * n + tail; }
    __device__ uint64_t signature(uint32_t op, uint64_t key) const
    {
        uint64_t h = 0xcbf29ce484222325ull ^ ((uint64_t)op << 48) ^ key;
        for (uint32_t k = 0; k < n; k++)
            h = (h ^ (uint8_t)tag[k]) * 0x100000001b3ull;
        return h;
    }
};

/* reference-argument wrappers (paper Fig. 4: addRefArg(ptr, mode, size, offset)) */
struct ref_r { const void *p; uint32_t bytes, off; };
struct ref_w { void *p; uint32_t bytes, off; };
struct ref_rw { void *p; uint32_t bytes, off; };
struct ref_val { uint64_t v; };                 /* a pointer passed as a plain value */
struct dma_ref { uint64_t addr; uint64_t bytes; };

__device__ inline void pack1(argpack &a, int v) { a.val(GF_T_I32, (uint64_t)(int64_t)v); }
__device__ inline void pack1(argpack &a, unsigned v) { a.val(GF_T_U32, (uint64_t)v); }
__device__ inline void pack1(argpack &a, long v) { a.val(GF_T_I64, (uint64_t)v); }
__device__ inline void pack1(argpack &a, long long v) { a.val(GF_T_I64, (uint64_t)v); }
__device__ inline void pack1(argpack &a, unsigned long v) { a.val(GF_T_U64, (uint64_t)v); }
__device__ inline void pack1(argpack &a, unsigned long long v) { a.val(GF_T_U64, (uint64_t)v); }
__device__ inline void pack1(argpack &a, double v) { a.val(GF_T_F64, (uint64_t)__double_as_longlong(v)); }
__device__ inline void pack1(argpack &a, float v) { pack1(a, (double)v); }
__device__ inline void pack1(argpack &a, char v) { pack1(a, (int)v); }
__device__ inline void pack1(argpack &a, short v) { pack1(a, (int)v); }
__device__ inline void pack1(argpack &a, bool v) { pack1(a, (int)v); }
__device__ inline void pack1(argpack &a, const char *s)
{
    if (!s) { a.val(GF_T_PTR, 0); return; }
    a.blob(GF_T_STR, s, gf_strlen(s) + 1u);
}
__device__ inline void pack1(argpack &a, char *s) { pack1(a, (const char *)s); }
__device__ inline void pack1(argpack &a, const void *p) { a.val(GF_T_PTR, (uint64_t)p); }
__device__ inline void pack1(argpack &a, void *p) { a.val(GF_T_PTR, (uint64_t)p); }
__device__ inline void pack1(argpack &a, ref_r r) { a.blob(GF_T_BLOB_R, r.p, r.bytes, r.off); }
__device__ inline void pack1(argpack &a, ref_w r) { a.blob(GF_T_BLOB_W, r.p, r.bytes, r.off); }
__device__ inline void pack1(argpack &a, ref_rw r) { a.blob(GF_T_BLOB_RW, r.p, r.bytes, r.off); }
__device__ inline void pack1(argpack &a, ref_val r) { a.val(GF_T_PTR, r.v); }
__device__ inline void pack1(argpack &a, dma_ref r)
{
    a.val(GF_T_DMA, r.addr);
    a.val(GF_T_U64, r.bytes);
}
__device__ inline void pack_all(argpack &) {}
template <class A0, class... A> __device__ inline void pack_all(argpack &a, A0 a0, A... rest)
{
    pack1(a, a0);
    pack_all(a, rest...);
}

/* copy `bytes` from any device-readable address into 8-byte-aligned mapped memory */
__device__ inline void copy_out(uint64_t *dst, const void *src, uint32_t bytes)
{
    const uint32_t nw = (bytes + 7u) >> 3;
    if (((uintptr_t)src & 7u) == 0) {
        const uint64_t *s = (const uint64_t *)src;
        for (uint32_t k = 0; k + 1 < nw || (k < nw && (bytes & 7u) == 0); k++)
            dst[k] = s[k];
        if (bytes & 7u) {
            const uint8_t *b = (const uint8_t *)src + 8u * (nw - 1);
            uint64_t w = 0;
            for (uint32_t j = 0; j < (bytes & 7u); j++)
                w |= (uint64_t)b[j] << (8 * j);
            dst[nw - 1] = w;
        }
    } else {
        const uint8_t *b = (const uint8_t *)src;
        for (uint32_t k = 0; k < nw; k++) {
            uint64_t w = 0;
            for (uint32_t j = 0; j < 8 && 8 * k + j < bytes; j++)
                w |= (uint64_t)b[8 * k + j] << (8 * j);
            dst[k] = w;
        }
    }
}

__device__ inline void copy_back(void *dst, const uint64_t *src, uint32_t bytes)
{
    uint8_t *d = (uint8_t *)dst;
    for (uint32_t k = 0; k < bytes; k += 8) {
        uint64_t w = ld_vol64(src + k / 8);
        for (uint32_t j = 0; j < 8 && k + j < bytes; j++)
            d[k + j] = (uint8_t)(w >> (8 * j));
    }
}

__device__ inline void write_rec(uint8_t *dst, const argpack &a, uint32_t lane, uint32_t gtid)
{
    uint64_t *w = (uint64_t *)dst;
    const uint32_t bytes = a.bytes();
    w[0] = (uint64_t)bytes | ((uint64_t)a.n << 32) | ((uint64_t)lane << 48);
    w[1] = (uint64_t)gtid;
    uint32_t k = 2;
    for (uint32_t t = 0; t < a.n; t += 8) {
        uint64_t tw = 0;
        for (uint32_t j = 0; j < 8 && t + j < a.n; j++)
            tw |= (uint64_t)(uint8_t)a.tag[t + j] << (8 * j);
        w[k++] = tw;
    }
    for (uint32_t t = 0; t < a.n; t++)
        w[k++] = a.word[t];
    for (uint32_t t = 0; t < a.n; t++)
        if (a.src[t] && a.tag[t] != GF_T_BLOB_W)
            copy_out(w + k + (uint32_t)(a.word[t] & 0xffffu) / 8, a.src[t], a.len[t]);
}

/* fmt cache: open addressing over device-address keys of shipped formats */
__device__ inline bool fmt_known(gf_state *S, uint64_t key)
{
    if (!key || !S->fmt_cache_cap)
        return false;
    const unsigned long long *tab = (const unsigned long long *)S->fmt_cache;
    uint32_t m = S->fmt_cache_cap - 1, h = (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> 40) & m;
    for (uint32_t p = 0; p < 16; p++) {
        unsigned long long v = *(volatile const unsigned long long *)&tab[(h + p) & m];
        if (v == key)
            return true;
        if (v == 0)
            return false;
    }
    return false;
}
__device__ inline void fmt_insert(gf_state *S, uint64_t key)
{
    if (!key || !S->fmt_cache_cap)
        return;
    unsigned long long *tab = (unsigned long long *)S->fmt_cache;
    uint32_t m = S->fmt_cache_cap - 1, h = (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> 40) & m;
    for (uint32_t p = 0; p < 16; p++) {
        unsigned long long old = atomicCAS(&tab[(h + p) & m], 0ull, (unsigned long long)key);
        if (old == 0 || old == key)
            return;
    }
}

__device__ __forceinline__ void st_relaxed_sys64(uint64_t *p, uint64_t v)
{
    asm volatile("st.relaxed.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

/*
 * The initial thread's outstanding deferred call (a printf-family call):
 * wait (bounded) until the host has answered it, give its slot back, and
 * return the nanoseconds waited.  With want_ret its result is kept for a
 * gf_call_result converted now (a round trip more, and the slot is given
 * back with a release so the read stays before it); from the thread's next
 * RPC the result is not read, and the give-back needs no ordering beyond
 * the acquire that saw the answer.  Initial thread only.
 */
/* names a buffered call in a gf_call_result (the rest is its sequence number) */
#define GF_CALL_BUFFERED (1ull << 63)

static __device__ __noinline__ uint64_t rpc_collect_deferred(gf_state *S, bool want_ret, uint32_t rank = 0)
{
    const unsigned long long t1 = s_pend_t1;
    if (!t1)
        return 0;
    const unsigned long long t = t1 - 1;
    const unsigned long long seq0 = s_pend_seq0;
    const uint32_t n = seq0 ? s_pend_n : 1u;
    s_pend_t1 = 0;
    /* the name the program holds for the record asked for: the ticket of a
     * lone call, the sequence number of a buffered one */
    const unsigned long long name = seq0 ? (GF_CALL_BUFFERED | (seq0 + rank)) : t1;
    uint8_t *slot = (uint8_t *)(S->ring_slots + (t % S->nslots) * (uint64_t)S->slot_bytes);
    gf_slot_hdr *h = (gf_slot_hdr *)slot;
    const uint64_t t0 = now_ns();
    backoff bo(S->timeout_ns);
    while (ld_acq_sys64(&h->seq) != t + 2)
        if (!bo.wait()) {
            set_error(GF_ETIMEDOUT);
            s_done_t1 = name;
            s_done_val = -1;
            return now_ns() - t0;
        }
    const uint64_t waited = now_ns() - t0;
    const uint32_t op = GF_OP_PRINTF;            /* the only deferred calls */
    atomicAdd((unsigned long long *)&S->st_wait_ns, (unsigned long long)waited);
    atomicAdd((unsigned long long *)&S->st_wait_op_ns[op], (unsigned long long)waited);
    atomicAdd((unsigned long long *)&S->st_calls[op], (unsigned long long)n);
    atomicAdd((unsigned long long *)&S->st_slots[op], 1ull);
    if (s_pend_key) {
        fmt_insert(S, s_pend_key);
        s_known_key = s_pend_key;
    }
    if (want_ret && rank < n) {
        s_done_val = (long long)ld_vol64((const uint64_t *)(slot + GF_SLOT_RET_OFF) + rank);
        s_done_t1 = name;
        st_rel_sys64(&h->seq, t + S->nslots);
    } else {
        s_done_t1 = 0;
        st_relaxed_sys64(&h->seq, t + S->nslots);
    }
    return waited;
}

/*
 * The initial thread's printf records wait in its block's shared memory and
 * go to the host together, up to 32 in one ring slot (the role of stdio's
 * buffer in the serial program): a call costs the packing of its record,
 * and one slot claim, credit check and publication serve the whole batch.
 * The batch is sent when it is full, before a record with another format,
 * before any other RPC of the initial thread (so its calls still reach the
 * host in program order), when a buffered call's result is read, and when
 * main returns.  Records of other threads are not ordered against it, as
 * for any two threads' calls.
 */
static __device__ __noinline__ void pb_flush(gf_state *S)
{
    const uint32_t n = s_pb_n;
    if (!n)
        return;
    s_pb_n = 0;
    const uint32_t bytes = s_pb_bytes, fbytes = s_pb_fbytes;
    s_pb_bytes = 0;
    if (s_pend_t1)                                  /* the previous slot is answered first */
        rpc_collect_deferred(S, false);
    if (*(volatile int32_t *)&S->error)
        return;                                     /* the program failed: the records are dropped */
    const unsigned long long t = atomicAdd(&S->rpc_ticket, 1ull);
    uint8_t *slot = (uint8_t *)(S->ring_slots + (t % S->nslots) * (uint64_t)S->slot_bytes);
    gf_slot_hdr *h = (gf_slot_hdr *)slot;
    const uint64_t t_issue = now_ns();
    backoff bo(S->timeout_ns);
    while (ld_acq_sys64(&h->seq) != t)
        if (!bo.wait()) {
            set_error(GF_ERING);
            return;
        }
    uint8_t *payload = slot + GF_SLOT_PAYLOAD_OFF;
    const uint32_t fmt_len = fbytes ? gf_strlen(s_pb_fmt) + 1u : 0u;
    if (fbytes)
        copy_out((uint64_t *)payload, s_pb_fmt, fmt_len);
    uint64_t *dst = (uint64_t *)(payload + fbytes);
    for (uint32_t w = 0; w < bytes / 8; w++)
        dst[w] = s_pb[w];
    h->opcode = GF_OP_PRINTF;
    h->nlanes = n;
    h->flags = fbytes ? GF_SF_FMT_INLINE : 0u;
    h->fmt_len = fmt_len;
    h->fmt_key = s_pb_key;
    h->prog = S->prog_id;
    h->t_issue = t_issue;
    h->payload_bytes = 0;
    h->t_publish = now_ns();
    st_rel_sys64(&h->seq, t + 1);                   /* orders this thread's record writes before it */
    s_pend_t1 = t + 1;
    s_pend_key = fbytes ? s_pb_key : 0ull;
    s_pend_seq0 = s_pb_seq - n;
    s_pend_n = n;
}

/* buffer one printf of the initial thread; false: it takes the unbuffered path */
static __device__ __noinline__ bool pb_printf(const char *fmt, const argpack &a, unsigned long long *name)
{
    gf_state *S = s_st;
    const uint64_t t_enter = now_ns();
    if (!fmt || *(volatile int32_t *)&S->error)
        return false;
    const uint64_t key = (uint64_t)fmt;
    const uint32_t my = a.bytes(), slot_cap = S->slot_bytes - GF_SLOT_PAYLOAD_OFF;
    if (s_pb_n && key != s_pb_key)
        pb_flush(S);
    for (int pass = 0; pass < 2; pass++) {
        if (!s_pb_n) {                              /* a new batch: does its format ship with it? */
            const bool ship = key != s_known_key && !fmt_known(S, key);
            if (!ship)
                s_known_key = key;
            s_pb_fbytes = ship ? (gf_strlen(fmt) + 1u + 7u) & ~7u : 0u;
            s_pb_key = key;
            s_pb_fmt = fmt;
        }
        const uint32_t room = slot_cap > s_pb_fbytes ? slot_cap - s_pb_fbytes : 0u;
        const uint32_t cap = room < 8u * GF_PBUF_WORDS ? room : 8u * GF_PBUF_WORDS;
        if (s_pb_bytes + my <= cap)
            break;
        if (!s_pb_n)
            return false;                           /* larger than the buffer: sent on its own */
        pb_flush(S);
    }
    write_rec((uint8_t *)s_pb + s_pb_bytes, a, s_pb_n, 0xffffffffu);
    s_pb_bytes += my;
    s_pb_n++;
    *name = GF_CALL_BUFFERED | s_pb_seq++;
    if (s_pb_n == 32)
        pb_flush(S);
    atomicAdd((unsigned long long *)&S->st_client_ns, (unsigned long long)(now_ns() - t_enter));
    return true;
}

/*
 * Issue one RPC from every calling lane; returns this lane's host result.
 * *status receives GF_OK, GF_ERING (no slot credit within the timeout),
 * GF_ETIMEDOUT (host did not answer), GF_EINVAL (record larger than a slot)
 * or the program's first error when one was already recorded.
 * defer_t1 (initial thread only): publish without waiting; *defer_t1
 * receives the ticket + 1 to collect later, and the return value is 0.
 */
static __device__ __noinline__ int64_t rpc_issue(uint32_t op, const char *fmt, const argpack &a, int *status,
                                                 unsigned long long *defer_t1 = nullptr)
{
    gf_state *S = s_st;
    const uint32_t lane = lane_id();
    const uint32_t active = __activemask();
    const bool initial = is_initial_thread();
    const uint64_t t_enter = initial ? now_ns() : 0;
    uint64_t t_waited = 0;                          /* this call's waits for the host */
    if (initial && s_pb_n)                          /* keep the initial thread's calls in order */
        pb_flush(S);
    if (initial && s_pend_t1)
        t_waited += rpc_collect_deferred(S, false);
    {
        /* fail fast after the first error; one reading for the whole group */
        const int err = __shfl_sync(active, *(volatile int32_t *)&S->error, __ffs(active) - 1);
        if (err) {
            if (status)
                *status = err;
            return -1;
        }
    }
    const uint64_t key = (uint64_t)fmt;
    const uint64_t sig = a.signature(op, key);
    const uint32_t grp = S->aggregate ? __match_any_sync(active, sig) : (1u << lane);
    const uint32_t my = a.bytes();
    const uint32_t gtid = is_initial_thread() ? 0xffffffffu : (uint32_t)gf_thread_num();
    const uint32_t slot_cap = S->slot_bytes - GF_SLOT_PAYLOAD_OFF;

    uint32_t remaining = grp;
    int64_t ret = -1;
    int st = GF_OK;
    while (remaining) {
        const bool in_round = (remaining >> lane) & 1u;
        /* format shipping is decided once per round by its leader */
        const uint32_t rl = __ffs(remaining) - 1;
        int ship = 0;
        uint32_t fmt_len = 0;
        if (lane == rl) {
            /* the initial thread remembers the last format it knows the host has */
            ship = (fmt && !(initial && key == s_known_key) && !fmt_known(S, key)) ? 1 : 0;
            if (initial && fmt && !ship)
                s_known_key = key;
            fmt_len = ship ? gf_strlen(fmt) + 1u : 0u;      /* read the format only to ship it */
        }
        ship = __shfl_sync(grp, ship, rl);
        fmt_len = __shfl_sync(grp, fmt_len, rl);
        const uint32_t fbytes = ship ? ((fmt_len + 7u) & ~7u) : 0u;
        const uint32_t cap = slot_cap > fbytes ? slot_cap - fbytes : 0u;
        /* exclusive prefix of record sizes over the lanes still waiting */
        const uint32_t v = in_round ? my : 0u;
        uint32_t off = 0;
        int same = 0;
        __match_all_sync(grp, v, &same);
        if (same) {
            off = v * __popc(remaining & lanemask_lt());
        } else {
            for (uint32_t m = grp; m; m &= m - 1) {
                const uint32_t l = __ffs(m) - 1;
                const uint32_t x = __shfl_sync(grp, v, l);
                if (l < lane)
                    off += x;
            }
        }
        uint32_t take = __ballot_sync(grp, in_round && off + my <= cap);
        bool oversized = false;
        if (!take) {               /* a single record larger than a slot: reject that lane */
            take = 1u << rl;
            oversized = true;
        }
        remaining &= ~take;
        const bool mine = (take >> lane) & 1u;
        if (oversized) {
            if (mine) {
                st = GF_EINVAL;
                ret = -1;
            }
            continue;
        }
        const uint32_t leader = __ffs(take) - 1;
        const uint32_t rank = __popc(take & lanemask_lt());
        const uint32_t nl = __popc(take);
        /* leader claims a ticket and waits for the slot's credit */
        unsigned long long t = 0;
        int cst = GF_OK;
        uint64_t t_issue = 0;
        if (lane == leader) {
            t_issue = now_ns();
            t = atomicAdd(&S->rpc_ticket, 1ull);
            uint64_t *seq = (uint64_t *)(S->ring_slots + (t % S->nslots) * (uint64_t)S->slot_bytes);
            backoff bo(S->timeout_ns);
            while (ld_acq_sys64(seq) != t)
                if (!bo.wait()) {
                    cst = GF_ERING;
                    break;
                }
        }
        t = __shfl_sync(grp, t, leader);
        cst = __shfl_sync(grp, cst, leader);
        if (cst != GF_OK) {
            if (mine) {
                st = cst;
                ret = -1;
            }
            if (lane == leader)
                set_error(cst);
            continue;
        }
        uint8_t *slot = (uint8_t *)(S->ring_slots + (t % S->nslots) * (uint64_t)S->slot_bytes);
        gf_slot_hdr *h = (gf_slot_hdr *)slot;
        uint8_t *payload = slot + GF_SLOT_PAYLOAD_OFF;
        if (mine)
            write_rec(payload + fbytes + off, a, lane, gtid);
        if (lane == leader) {
            if (ship)
                copy_out((uint64_t *)payload, fmt, fmt_len);
            h->opcode = op;
            h->nlanes = nl;
            h->flags = ship ? GF_SF_FMT_INLINE : 0u;
            h->fmt_len = ship ? fmt_len : 0u;
            h->fmt_key = key;
            h->prog = S->prog_id;
            h->t_issue = t_issue;
        }
        /* a lone lane's own record writes are ordered before its publishing
         * store by that store's release; a group's other lanes need the fence */
        if (nl > 1)
            __threadfence_system();
        __syncwarp(grp);
        int wst = GF_OK;
        if (defer_t1) {           /* the initial thread alone: publish and go on */
            h->payload_bytes = 0;
            h->t_publish = now_ns();
            st_rel_sys64(&h->seq, t + 1);
            s_pend_t1 = t + 1;
            s_pend_key = ship ? key : 0;
            s_pend_seq0 = 0;
            *defer_t1 = t + 1;
            ret = 0;
            continue;
        }
        if (lane == leader) {
            h->payload_bytes = 0;   /* the host walks records by their own sizes */
            h->t_publish = now_ns();
            st_rel_sys64(&h->seq, t + 1);
            backoff bo(S->timeout_ns);
            const uint64_t t0 = now_ns();
            while (ld_acq_sys64(&h->seq) != t + 2)
                if (!bo.wait()) {
                    wst = GF_ETIMEDOUT;
                    break;
                }
            const uint64_t waited = now_ns() - t0;
            t_waited += waited;
            atomicAdd((unsigned long long *)&S->st_wait_ns, (unsigned long long)waited);
            atomicAdd((unsigned long long *)&S->st_wait_op_ns[op < GF_NSTAT ? op : 0], (unsigned long long)waited);
            if (wst == GF_OK) {
                const uint64_t lat = now_ns() - t_issue;
                uint32_t bk = (uint32_t)lat;
                if (lat >= 8) {
                    const uint32_t e = 63 - __clzll((long long)lat);
                    bk = 8u * e + (uint32_t)((lat >> (e - 3)) & 7u);
                }
                if (bk >= GF_LAT_BUCKETS)
                    bk = GF_LAT_BUCKETS - 1;
                atomicAdd((unsigned long long *)&S->lat_hist[bk], (unsigned long long)nl);
                atomicAdd((unsigned long long *)&S->st_calls[op < GF_NSTAT ? op : 0], (unsigned long long)nl);
                atomicAdd((unsigned long long *)&S->st_slots[op < GF_NSTAT ? op : 0], 1ull);
            } else {
                set_error(wst);
            }
        }
        wst = __shfl_sync(grp, wst, leader);
        if (wst == GF_OK && mine) {
            ret = (int64_t)ld_vol64((const uint64_t *)(slot + GF_SLOT_RET_OFF) + rank);
            /* copy back written reference arguments (mode write / readwrite) */
            const uint64_t *rw = (const uint64_t *)(payload + fbytes + off);
            const uint32_t ntag = (a.n + 7u) & ~7u;
            const uint64_t *tail = rw + 2 + ntag / 8 + a.n;
            for (uint32_t k = 0; k < a.n; k++)
                if (a.tag[k] == GF_T_BLOB_W || a.tag[k] == GF_T_BLOB_RW)
                    copy_back((void *)a.src[k], tail + (uint32_t)(a.word[k] & 0xffffu) / 8, a.len[k]);
        } else if (mine) {
            st = wst;
            ret = -1;
        }
        __syncwarp(grp);
        if (lane == leader && wst == GF_OK) {
            if (ship) {
                fmt_insert(S, key);
                if (initial)
                    s_known_key = key;
            }
            st_rel_sys64(&h->seq, t + S->nslots);
        }
    }
    if (initial)
        atomicAdd((unsigned long long *)&S->st_client_ns, (unsigned long long)(now_ns() - t_enter - t_waited));
    if (status)
        *status = st;
    return ret;
}

template <class... A> __device__ inline int64_t rpc(uint32_t op, const char *fmt, int *status, A... args)
{
    argpack a;
    pack_all(a, args...);
    return rpc_issue(op, fmt, a, status);
}

/* the result of a deferred call (initial thread only), by its name: the
 * ticket + 1 of a lone call, or GF_CALL_BUFFERED | the sequence number of a
 * buffered one (sent now if it is still in the buffer) */
static __device__ __noinline__ int64_t deferred_value(unsigned long long t1)
{
    gf_state *S = s_st;
    if (t1 & GF_CALL_BUFFERED) {
        const unsigned long long seq = t1 & ~GF_CALL_BUFFERED;
        if (s_pb_n && seq >= s_pb_seq - s_pb_n)
            pb_flush(S);
        if (s_pend_t1 && s_pend_seq0 && seq >= s_pend_seq0 && seq < s_pend_seq0 + s_pend_n)
            rpc_collect_deferred(S, true, (uint32_t)(seq - s_pend_seq0));
    } else if (s_pend_t1 == t1 && !s_pend_seq0) {
        rpc_collect_deferred(S, true);
    }
    return s_done_t1 == t1 ? (int64_t)s_done_val : -1;
}
} // namespace gfd

/* Result of a printf-family call.  Converting it to int gives the call's
 * return value (sending the initial thread's buffered records and waiting
 * for the host if the call was buffered or deferred); a program that
 * ignores it never waits for the call.  Use it in the statement that made
 * the call: a deferred result converted after a later RPC of the initial
 * thread, or after its batch went to the host with later calls, reads -1. */
struct gf_call_result {
    int64_t v;
    unsigned long long t1;     /* ticket + 1 of a deferred call; 0: v is the result */
    __device__ operator int() const { return (int)(t1 ? gfd::deferred_value(t1) : v); }
};

namespace gfd {
template <class... A> __device__ inline gf_call_result rpc_deferrable(uint32_t op, const char *fmt, A... args)
{
    argpack a;
    pack_all(a, args...);
    if (is_initial_thread()) {
        unsigned long long t1 = 0;
        if (op == GF_OP_PRINTF && pb_printf(fmt, a, &t1))
            return gf_call_result{0, t1};
        const int64_t r = rpc_issue(op, fmt, a, nullptr, &t1);
        return gf_call_result{t1 ? 0 : r, t1};
    }
    return gf_call_result{rpc_issue(op, fmt, a, nullptr), 0ull};
}

/* the kernel split: the host launches this region as its own kernel and
 * answers with the kernel's grid (declared next to run_region) */
static __device__ int64_t split_launch(gf_state *S, int *status)
{
    return rpc(GF_OP_REGION, nullptr, status, (unsigned long long)S->prog_id);
}

/* Single-lane asynchronous call for the initial thread: post a slot now,
 * collect its return later, so the grid can work while the host does. */
static __device__ __noinline__ int rpc_post1(uint32_t op, const argpack &a, unsigned long long *tk)
{
    gf_state *S = s_st;
    if (a.bytes() > S->slot_bytes - GF_SLOT_PAYLOAD_OFF)
        return GF_EINVAL;
    if (s_pb_n)
        pb_flush(S);
    if (s_pend_t1)
        rpc_collect_deferred(S, false);
    if (*(volatile int32_t *)&S->error)
        return S->error;
    const unsigned long long t = atomicAdd(&S->rpc_ticket, 1ull);
    uint8_t *slot = (uint8_t *)(S->ring_slots + (t % S->nslots) * (uint64_t)S->slot_bytes);
    gf_slot_hdr *h = (gf_slot_hdr *)slot;
    backoff bo(S->timeout_ns);
    while (ld_acq_sys64(&h->seq) != t)
        if (!bo.wait()) {
            set_error(GF_ERING);
            return GF_ERING;
        }
    write_rec(slot + GF_SLOT_PAYLOAD_OFF, a, lane_id(), 0xffffffffu);
    h->opcode = op;
    h->nlanes = 1;
    h->flags = 0;
    h->fmt_len = 0;
    h->fmt_key = 0;
    h->payload_bytes = 0;
    h->prog = S->prog_id;
    h->t_issue = now_ns();
    __threadfence_system();
    h->t_publish = now_ns();
    st_rel_sys64(&h->seq, t + 1);
    *tk = t;
    return GF_OK;
}

static __device__ __noinline__ int64_t rpc_finish1(unsigned long long t, int *status)
{
    gf_state *S = s_st;
    uint8_t *slot = (uint8_t *)(S->ring_slots + (t % S->nslots) * (uint64_t)S->slot_bytes);
    gf_slot_hdr *h = (gf_slot_hdr *)slot;
    const uint64_t t0 = now_ns();
    backoff bo(S->timeout_ns);
    while (ld_acq_sys64(&h->seq) != t + 2)
        if (!bo.wait()) {
            set_error(GF_ETIMEDOUT);
            *status = GF_ETIMEDOUT;
            return -1;
        }
    const int64_t r = (int64_t)ld_vol64((const uint64_t *)(slot + GF_SLOT_RET_OFF));
    const uint32_t op = h->opcode;
    atomicAdd((unsigned long long *)&S->st_wait_ns, (unsigned long long)(now_ns() - t0));
    atomicAdd((unsigned long long *)&S->st_wait_op_ns[op < GF_NSTAT ? op : 0], (unsigned long long)(now_ns() - t0));
    atomicAdd((unsigned long long *)&S->st_calls[op < GF_NSTAT ? op : 0], 1ull);
    atomicAdd((unsigned long long *)&S->st_slots[op < GF_NSTAT ? op : 0], 1ull);
    st_rel_sys64(&h->seq, t + S->nslots);
    *status = GF_OK;
    return r;
}

/* dst[0 .. bytes) = src[...] by the whole grid: 16-byte vector copies when
 * both ends are 16-byte aligned, bytewise otherwise.  Initial thread only. */
static __device__ int copy_region_body(void *dst, const void *src, uint64_t bytes);

/* a grid-wide copy (initial thread), timed apart from the program's own regions */
static __device__ __noinline__ int copy_region(void *dst, const void *src, uint64_t bytes)
{
    const uint64_t t0 = now_ns();
    const int rc = copy_region_body(dst, src, bytes);
    s_st->st_copy_regions++;
    s_st->st_copy_ns += now_ns() - t0;
    return rc;
}

static __device__ int copy_region_body(void *dst, const void *src, uint64_t bytes)
{
    if ((((uintptr_t)dst | (uintptr_t)src) & 15u) == 0) {
        const uint64_t n16 = bytes >> 4;
        uint4 *d = (uint4 *)dst;
        const uint4 *s = (const uint4 *)src;
        const int rc = gf_parallel_for(0, (int64_t)n16, GF_SCHED_STATIC, 1, [=](int64_t i) { d[i] = s[i]; });
        for (uint64_t k = n16 << 4; k < bytes; k++)
            ((uint8_t *)dst)[k] = ((const uint8_t *)src)[k];
        return rc;
    }
    uint8_t *d = (uint8_t *)dst;
    const uint8_t *s = (const uint8_t *)src;
    return gf_parallel_for(0, (int64_t)bytes, GF_SCHED_STATIC, 1, [=](int64_t i) { d[i] = s[i]; });
}

/*
 * Large fwrite from the initial thread through the context's bulk arena
 * (pinned, device-mapped host memory, two halves): the grid copies chunk c
 * into one half while the host writes chunk c-1 from the other; chunk c is
 * posted only after chunk c-1 has been written, so the file sees the chunks
 * in order.  No host-side CUDA call is involved.
 */
static __device__ __noinline__ size_t fwrite_bulk(const void *buf, size_t size, size_t n, GF_FILE f)
{
    gf_state *S = s_st;
    const uint64_t bytes = (uint64_t)size * n, half = (S->bulk_bytes / 2) & ~(uint64_t)4095;
    uint8_t *arena = (uint8_t *)S->bulk_dev;
    uint64_t written = 0, prev_len = 0;
    unsigned long long tk = 0;
    bool pend = false, ok = true;
    int k = 0;
    for (uint64_t off = 0; off < bytes && ok; off += half, k ^= 1) {
        const uint64_t len = bytes - off < half ? bytes - off : half;
        if (copy_region(arena + (uint64_t)k * half, (const uint8_t *)buf + off, len) != GF_OK)
            ok = false;
        if (pend) {
            int st = GF_OK;
            const int64_t r = rpc_finish1(tk, &st);
            pend = false;
            if (st != GF_OK || r != (int64_t)prev_len)
                ok = false;
            else
                written += prev_len;
        }
        if (!ok)
            break;
        argpack a;
        pack_all(a, 1ull, (unsigned long long)len, (unsigned long long)f);
        a.val(GF_T_ARENA, (uint64_t)k * half);
        a.val(GF_T_U64, len);
        a.val(GF_T_U64, bytes - off);            /* the whole write still to come: the host maps it once */
        if (rpc_post1(GF_OP_FWRITE, a, &tk) != GF_OK)
            ok = false;
        else {
            pend = true;
            prev_len = len;
        }
    }
    if (pend) {
        int st = GF_OK;
        const int64_t r = rpc_finish1(tk, &st);
        if (st == GF_OK && r == (int64_t)prev_len)
            written += prev_len;
    }
    return (size_t)(written / size);
}

/* Large fread into device memory through the bulk arena: the host reads
 * chunk c+1 into one half while the grid copies chunk c out of the other. */
static __device__ __noinline__ size_t fread_bulk(void *buf, size_t size, size_t n, GF_FILE f)
{
    gf_state *S = s_st;
    const uint64_t bytes = (uint64_t)size * n, half = (S->bulk_bytes / 2) & ~(uint64_t)4095;
    uint8_t *arena = (uint8_t *)S->bulk_dev;
    auto post = [&](uint64_t off, int k, unsigned long long *tk) {
        const uint64_t len = bytes - off < half ? bytes - off : half;
        argpack a;
        pack_all(a, 1ull, (unsigned long long)len, (unsigned long long)f);
        a.val(GF_T_ARENA, (uint64_t)k * half);
        a.val(GF_T_U64, len);
        return rpc_post1(GF_OP_FREAD, a, tk);
    };
    uint64_t got = 0;
    unsigned long long tk = 0;
    if (!bytes || post(0, 0, &tk) != GF_OK)
        return 0;
    int k = 0;
    for (uint64_t off = 0; off < bytes; off += half, k ^= 1) {
        const uint64_t len = bytes - off < half ? bytes - off : half;
        int st = GF_OK;
        const int64_t r = rpc_finish1(tk, &st);
        if (st != GF_OK || r < 0)
            break;
        const bool more = (uint64_t)r == len && off + len < bytes;
        if (more && post(off + len, k ^ 1, &tk) != GF_OK)
            break;
        if (copy_region((uint8_t *)buf + off, arena + (uint64_t)k * half, (uint64_t)r) != GF_OK)
            break;
        got += (uint64_t)r;
        if (!more)
            break;
    }
    return (size_t)(got / size);
}

} // namespace gfd

/* ====================================================================== libc over RPC */
/* printf family: formatted on the host by the real libc, one landing pad per
 * argument-type signature (paper Fig. 4b), records grouped per warp. */
template <class... A> __device__ inline gf_call_result gf_printf(const char *fmt, A... args)
{
    return gfd::rpc_deferrable(GF_OP_PRINTF, fmt, (unsigned long long)GF_STDOUT_H, args...);
}
template <class... A> __device__ inline gf_call_result gf_fprintf(GF_FILE f, const char *fmt, A... args)
{
    return gfd::rpc_deferrable(GF_OP_PRINTF, fmt, (unsigned long long)f, args...);
}
__device__ inline GF_FILE gf_stdout() { return GF_STDOUT_H; }
__device__ inline GF_FILE gf_stderr() { return GF_STDERR_H; }

__device__ inline GF_FILE gf_fopen(const char *path, const char *mode)
{
    return (GF_FILE)gfd::rpc(GF_OP_FOPEN, nullptr, nullptr, path, mode);
}
__device__ inline int gf_fclose(GF_FILE f)
{
    return (int)gfd::rpc(GF_OP_FCLOSE, nullptr, nullptr, (unsigned long long)f);
}
__device__ inline int gf_fflush(GF_FILE f)
{
    return (int)gfd::rpc(GF_OP_FFLUSH, nullptr, nullptr, (unsigned long long)f);
}
/* fwrite: small objects travel inside the slot; large ones from the initial
 * thread go through the bulk arena (grid copy + host write, overlapped);
 * large ones from a region's thread are read by the host with a copy-engine
 * DMA straight from device memory. */
__device__ inline size_t gf_fwrite(const void *buf, size_t size, size_t n, GF_FILE f)
{
    const uint64_t bytes = (uint64_t)size * n;
    __threadfence_system();
    if (bytes <= GF_INLINE_BLOB_MAX)
        return (size_t)gfd::rpc(GF_OP_FWRITE, nullptr, nullptr, (unsigned long long)size,
                                (unsigned long long)n, (unsigned long long)f, gfd::ref_r{buf, (uint32_t)bytes});
    if (gfd::is_initial_thread() && gfd::s_st->bulk_bytes >= 8192 && size)
        return gfd::fwrite_bulk(buf, size, n, f);
    return (size_t)gfd::rpc(GF_OP_FWRITE, nullptr, nullptr, (unsigned long long)size, (unsigned long long)n,
                            (unsigned long long)f, gfd::dma_ref{(uint64_t)buf, bytes});
}
__device__ inline size_t gf_fread(void *buf, size_t size, size_t n, GF_FILE f)
{
    const uint64_t bytes = (uint64_t)size * n;
    if (bytes <= GF_INLINE_BLOB_MAX)
        return (size_t)gfd::rpc(GF_OP_FREAD, nullptr, nullptr, (unsigned long long)size,
                                (unsigned long long)n, (unsigned long long)f, gfd::ref_w{buf, (uint32_t)bytes});
    if (gfd::is_initial_thread() && gfd::s_st->bulk_bytes >= 8192 && size)
        return gfd::fread_bulk(buf, size, n, f);
    size_t r = (size_t)gfd::rpc(GF_OP_FREAD, nullptr, nullptr, (unsigned long long)size, (unsigned long long)n,
                                (unsigned long long)f, gfd::dma_ref{(uint64_t)buf, bytes});
    __threadfence();
    return r;
}
__device__ inline long long gf_clock()
{
    return (long long)gfd::rpc(GF_OP_CLOCK, nullptr, nullptr);
}
/* getenv: the host interns the value in device-readable mapped memory that
 * lives as long as the context; NULL when unset. */
__device__ inline const char *gf_getenv(const char *name)
{
    return (const char *)gfd::rpc(GF_OP_GETENV, nullptr, nullptr, name);
}
/* Generic RPC to a landing pad registered with gf_rpc_register (paper
 * Sec. 3.2, Fig. 4): `nargs` (<= GF_MAX_ARGS) arguments described by gf_arg
 * (gf_layout.h), integers sign- or zero-extended to 64 bits in `word`.
 * *ret (may be NULL) receives the landing pad's return value, -1 on failure.
 * Returns GF_OK, GF_EINVAL (bad tag, count or offset, or a record larger
 * than a ring slot), GF_ERING, GF_ETIMEDOUT, or the program's first error.
 * The lanes of a warp that call it with the same opcode and argument tags
 * share one ring slot. */
__device__ inline int gf_rpc(uint32_t opcode, const gf_arg *args, int nargs, int64_t *ret)
{
    if (ret)
        *ret = -1;
    if (nargs < 0 || nargs > GF_MAX_ARGS || (nargs > 0 && !args))
        return GF_EINVAL;
    gfd::argpack a;
    for (int k = 0; k < nargs; k++) {
        const gf_arg &g = args[k];
        switch (g.tag) {
        case GF_T_I32: case GF_T_U32: case GF_T_I64: case GF_T_U64: case GF_T_F64: case GF_T_PTR:
            a.val(g.tag, g.word);
            break;
        case GF_T_STR:
            if (g.ptr)
                a.blob(GF_T_STR, g.ptr, gf_strlen((const char *)g.ptr) + 1u);
            else
                a.val(GF_T_PTR, 0);
            break;
        case GF_T_BLOB_R: case GF_T_BLOB_W: case GF_T_BLOB_RW:
            if (!g.ptr || g.off >= 65536u || g.off > g.bytes)
                return GF_EINVAL;
            a.blob(g.tag, g.ptr, g.bytes, g.off);
            break;
        default:
            return GF_EINVAL;
        }
    }
    int st = GF_OK;
    const int64_t r = gfd::rpc_issue(opcode, nullptr, a, &st);
    if (ret)
        *ret = r;
    return st;
}
/* the same call with its arguments as a C++ parameter pack (values, strings,
 * gf_ref_read / gf_ref_write / gf_ref_readwrite, gf_ref_lookup) */
template <class... A> __device__ inline int64_t gf_rpc(uint32_t opcode, int *status, A... args)
{
    return gfd::rpc(opcode, nullptr, status, args...);
}
/* Reference arguments (paper Sec. 3.2, Fig. 4c): the whole underlying
 * object [obj, obj + bytes) travels to the host, and the host callee gets a
 * pointer at offset `off` into its copy.  read: copied to the host only;
 * write: copied back only; readwrite: both.  Inline objects are limited by
 * the slot size (and offsets to 64 KiB). */
__device__ inline gfd::ref_r gf_ref_read(const void *obj, uint32_t bytes, uint32_t off = 0)
{
    return gfd::ref_r{obj, bytes, off};
}
__device__ inline gfd::ref_w gf_ref_write(void *obj, uint32_t bytes, uint32_t off = 0)
{
    return gfd::ref_w{obj, bytes, off};
}
__device__ inline gfd::ref_rw gf_ref_readwrite(void *obj, uint32_t bytes, uint32_t off = 0)
{
    return gfd::ref_rw{obj, bytes, off};
}

/* Underlying object of a pointer that no analysis could pin down (the
 * paper's _FindObj, Sec. 3.2): the device heap's slab metadata and page
 * table give the enclosing block.  Returns false for memory the heap did not
 * hand out (the pointer then travels as a plain value, as in the paper). */
__device__ inline bool gf_find_obj(const void *p, uint64_t *base, uint64_t *size)
{
    gf_heap *H = &gfd::s_st->heap;
    const uint64_t a = (uint64_t)p;
    if (a >= H->slab_base && a < H->slab_base + H->slab_bytes) {
        const uint32_t s = (uint32_t)((a - H->slab_base) >> GF_SLAB_SHIFT);
        const uint32_t c1 = *(volatile uint32_t *)&((uint32_t *)H->slab_meta)[4 * s];
        if (!c1)
            return false;
        const uint64_t bs = 16ull << (c1 - 1);
        *base = H->slab_base + ((a - H->slab_base) / bs) * bs;
        *size = bs;
        return true;
    }
    if (a >= H->large_base && a < H->large_base + H->large_bytes) {
        const volatile uint32_t *sz = (const volatile uint32_t *)H->large_size;
        int64_t pg = (int64_t)((a - H->large_base) >> GF_PAGE_SHIFT);
        for (int64_t k = pg; k >= 0 && pg - k < 4096; k--)      /* bounded backward scan */
            if (sz[k]) {
                if ((uint64_t)(pg - k) < sz[k]) {
                    *base = H->large_base + ((uint64_t)k << GF_PAGE_SHIFT);
                    *size = (uint64_t)sz[k] << GF_PAGE_SHIFT;
                    return true;
                }
                return false;
            }
    }
    return false;
}

/* A reference argument whose object is found at run time (readwrite), or a
 * plain value when it is not a heap block or too large to travel inline. */
struct gf_ref_any {
    bool found;
    gfd::ref_rw r;
    uint64_t v;
};
__device__ inline gf_ref_any gf_ref_lookup(void *p)
{
    uint64_t base = 0, size = 0;
    gf_ref_any x;
    x.v = (uint64_t)p;
    x.found = gf_find_obj(p, &base, &size) && size <= GF_INLINE_BLOB_MAX;
    x.r = gfd::ref_rw{(void *)base, (uint32_t)size, (uint32_t)((uint64_t)p - base)};
    return x;
}
namespace gfd {
__device__ inline void pack1(argpack &a, gf_ref_any x)
{
    if (x.found)
        pack1(a, x.r);
    else
        a.val(GF_T_PTR, x.v);
}
} // namespace gfd

#endif
