/*
 * Memory layouts shared by the device runtime and the host server.
 *
 * Two regions cross the device/host boundary:
 *  - the RPC ring: an array of fixed-size slots in pinned, device-mapped host
 *    memory.  This replaces the paper's managed-memory RPC buffer and its
 *    "int flag set to 0" completion (Sec. 5.2, Fig. 7): every hand-off is one
 *    64-bit sequence word written with release and read with acquire semantics
 *    at system scope, so no page migration is involved;
 *  - the program state (gf_state): device memory owned by one running
 *    program, written by the host only before launch and read back after.
 *
 * Slot protocol for ticket t in slot s = t % nslots (seq starts at s):
 *   seq == t            slot free for ticket t (credit)
 *   seq == t + 1        device published a request       (device: st.release.sys)
 *   seq == t + 2        host wrote the returns            (host:   release store)
 *   seq == t + nslots   device consumed the returns; slot free for ticket t+nslots
 *
 * Plain C: no CUDA types.  Device pointers are stored as 64-bit integers.
 */
#ifndef GF_LAYOUT_H
#define GF_LAYOUT_H
#include <stdint.h>

#define GF_WARP 32

/* ------------------------------------------------------------------ ring */
#define GF_SLOT_HDR_BYTES 64u
#define GF_SLOT_RET_OFF 64u                       /* 32 x int64 per-lane returns */
#define GF_SLOT_PAYLOAD_OFF 320u                  /* fmt (optional) then lane records */

enum gf_opcode {
    GF_OP_NOP = 0,
    GF_OP_PRINTF = 1,     /* formatted write to a stream handle (stdout, stderr, FILE*)   */
    GF_OP_FOPEN = 2,      /* (path, mode) -> opaque FILE* handle                          */
    GF_OP_FWRITE = 3,     /* (buf, size, nmemb, FILE*) -> items written                   */
    GF_OP_FCLOSE = 4,     /* (FILE*) -> 0 / EOF                                           */
    GF_OP_CLOCK = 5,      /* () -> host clock()                                           */
    GF_OP_GETENV = 6,     /* (name) -> device-readable interned copy, 0 if unset          */
    GF_OP_FREAD = 7,      /* (buf, size, nmemb, FILE*) -> items read, bytes written back  */
    GF_OP_FFLUSH = 8,     /* (FILE*) -> 0 / EOF                                           */
    GF_OP_STRTOD = 9,     /* (str, int64 *used) -> bits of strtod(str), chars consumed    */
    GF_OP_REGION = 10,    /* (instance) -> grid of the region kernel the host launched     */
    GF_OP_USER = 256      /* first opcode for handlers registered with gf_rpc_register    */
};

/* slot header flags */
#define GF_SF_FMT_INLINE 1u    /* format string bytes precede the lane records */

typedef struct gf_slot_hdr {
    uint64_t seq;              /* protocol word (see above)                          */
    uint32_t opcode;
    uint32_t nlanes;           /* lane records in the payload                        */
    uint32_t flags;
    uint32_t fmt_len;          /* bytes of the inline format string incl. NUL        */
    uint64_t fmt_key;          /* device address of the format string (cache key)    */
    uint32_t payload_bytes;    /* bytes after GF_SLOT_PAYLOAD_OFF                    */
    uint32_t prog;             /* program instance (serving)                         */
    uint64_t t_issue;          /* device %globaltimer when the slot was claimed      */
    uint64_t t_publish;        /* device %globaltimer at publication                 */
    uint64_t t_host_ns;        /* host: ns spent in the landing pad for this slot    */
} gf_slot_hdr;

/*
 * Lane record (8-byte aligned, inside the payload):
 *   gf_rec_hdr | tags[nargs] padded to 8 | words[nargs] (8 B each) | tail blobs
 * Value arguments carry their bits in the word (the paper's value arguments,
 * Sec. 3.2: integers, floats, opaque handles such as FILE*).  Reference
 * arguments ('s' strings, 'b' byte blobs) carry (offset in tail | bytes << 32)
 * and their bytes in the tail; mode 'W'/'X' blobs are copied back to the device
 * object after the call (write / readwrite), 'D' blobs are moved by DMA.
 */
typedef struct gf_rec_hdr {
    uint32_t bytes;            /* whole record incl. header, multiple of 8           */
    uint16_t nargs;
    uint16_t lane;             /* issuing lane                                       */
    uint32_t gtid;             /* issuing thread's continuous id (or ~0 for main)    */
    uint32_t seq;              /* per-thread call sequence number (debug tracing)    */
} gf_rec_hdr;

/* argument tags */
#define GF_T_I32 'i'
#define GF_T_U32 'u'
#define GF_T_I64 'l'
#define GF_T_U64 'L'
#define GF_T_F64 'd'
#define GF_T_PTR 'p'           /* opaque pointer / handle, never dereferenced          */
#define GF_T_STR 's'           /* NUL-terminated string, bytes in the tail (read)      */
#define GF_T_BLOB_R 'b'        /* object bytes in tail, read only                       */
#define GF_T_BLOB_W 'w'        /* object written by the host, copied back               */
#define GF_T_BLOB_RW 'x'       /* object read and written                               */
#define GF_T_DMA 'D'           /* large object: word = device address, moved by DMA     */
#define GF_T_ARENA 'A'         /* large object staged in the bulk arena: word = offset  */

#define GF_MAX_ARGS 16

/* One argument of the array form of gf_rpc (paper Sec. 3.2, Fig. 4c: an
 * argument is a value, or a reference to an object with a mode, a size and
 * the pointer's offset inside the object).
 *   value arguments   tag GF_T_I32 / U32 / I64 / U64 / F64 / PTR: the bits in
 *                     `word` (a double as its IEEE bits); ptr, bytes, off unused;
 *   string            tag GF_T_STR: ptr = the NUL-terminated string;
 *   references        tag GF_T_BLOB_R / BLOB_W / BLOB_RW: ptr = start of the
 *                     underlying object, bytes = its size (it travels inside
 *                     the ring slot), off = the argument pointer's offset in
 *                     it (< 65536); write and readwrite objects are copied
 *                     back after the host call. */
typedef struct gf_arg {
    uint64_t word;
    const void *ptr;
    uint32_t bytes;
    uint32_t off;
    char tag;
    char pad[7];
} gf_arg;

/* standard stream handles (the device never sees host FILE* values for these) */
#define GF_STDOUT_H 1ull
#define GF_STDERR_H 2ull

/* ------------------------------------------------------------------ regions */
enum gf_sched_kind { GF_SCHED_STATIC = 0, GF_SCHED_DYNAMIC = 1 };
enum gf_red_op { GF_RED_NONE = 0, GF_RED_SUM = 1, GF_RED_MIN = 2, GF_RED_MAX = 3 };

#define GF_BODY_MAX 448u

typedef struct gf_region {
    uint64_t fn;               /* device trampoline (function pointer bits)          */
    int64_t b, e, chunk;
    int32_t sched, red;
    uint32_t loop_id, pad;
    unsigned char body[GF_BODY_MAX] __attribute__((aligned(16)));  /* captured loop body */
} gf_region;

/* ------------------------------------------------------------------ heap */
#define GF_HEAP_NCLASS 13       /* 16 B .. 64 KiB, powers of two                      */
#define GF_HEAP_MIN_SHIFT 4
#define GF_HEAP_MAX_SMALL (64u * 1024u)
#define GF_SLAB_SHIFT 18        /* 256 KiB slabs                                      */
#define GF_PAGE_SHIFT 16        /* 64 KiB pages for the large path                    */
#define GF_MAX_SM 256
#define GF_HEAP_LANES 32        /* free stacks per (SM, class): one per lane index    */
#define GF_LARGE_EXT_MAX 8192   /* free extents of the large path                     */

typedef struct gf_heap {
    uint64_t base;             /* device arena                                        */
    uint64_t bytes;
    uint64_t slab_base;        /* [slab_base, slab_base + slab_bytes): small classes  */
    uint64_t slab_bytes;
    uint64_t large_base;       /* [large_base, large_base + large_bytes): pages       */
    uint64_t large_bytes;
    uint64_t slab_meta;        /* device: per-slab {class, owner sm, bump} words      */
    uint64_t free_heads;       /* device: [GF_MAX_SM][NCLASS][LANES] tagged heads     */
    uint64_t cur_slab;         /* device: [GF_MAX_SM][NCLASS] current slab + 1        */
    uint64_t large_ext;        /* device: free extents {page, npages} sorted          */
    uint64_t large_size;       /* device: npages of the block starting at each page   */
    uint32_t nslabs, npages;
    uint32_t next_slab;        /* bump counter over fresh slabs                       */
    uint32_t large_lock;
    uint32_t large_next;       /* extents in use                                      */
    uint32_t pad;
    uint64_t live_bytes, high_water;
    uint64_t n_alloc, n_free, n_fail, n_bad_free;
    uint64_t large_cache;      /* the last freed large block {page, npages << 32}, 0 if none */
} gf_heap;

/* ------------------------------------------------------------------ program state */
#define GF_MAX_BUFS 16
#define GF_NSTAT 16
#define GF_LAT_BUCKETS 320      /* log-linear: 8 sub-buckets per octave, 40 octaves of ns */

typedef struct gf_state {
    uint32_t epoch;            uint32_t pad_e[31];     /* main -> workers: new region    */
    uint32_t done_blocks;      uint32_t pad_d[31];     /* workers -> main: blocks done   */
    uint32_t red_ticket;       uint32_t pad_r[31];     /* last-block detection           */
    uint32_t bar_count;        uint32_t pad_b[31];     /* grid barrier arrivals          */
    uint32_t bar_gen;          uint32_t pad_g[31];     /* grid barrier generation        */
    unsigned long long dyn_next; uint64_t pad_n[15];   /* dynamic schedule counter       */
    unsigned long long rpc_ticket; uint64_t pad_t[15]; /* ring ticket counter            */
    gf_region region;
    uint64_t red_result[2];
    uint32_t exit_flag;        /* main returned: the workers leave their loop            */
    uint32_t pad_x;
    /* configuration written by the host before launch */
    uint32_t nblocks, block_dim, nworkers, aggregate;
    int64_t timeout_ns;
    uint64_t ring_slots;       /* device address of the mapped slot array            */
    uint32_t nslots, slot_bytes;
    uint64_t fmt_cache;        /* device: open-addressed table of shipped fmt keys    */
    uint32_t fmt_cache_cap, prog_id;
    uint64_t partials;         /* device: nblocks x 16 B reduction partials          */
    uint64_t bulk_dev;         /* device address of the mapped bulk arena            */
    uint64_t bulk_bytes;
    uint64_t buf_ptr[GF_MAX_BUFS];
    uint64_t buf_bytes[GF_MAX_BUFS];
    uint32_t nbufs;
    uint32_t split;            /* 1: regions run as host-launched kernels (the paper's split) */
    /* results written by the device */
    int32_t exit_code, error, main_done;
    uint64_t st_calls[GF_NSTAT];  /* RPC calls per opcode (lane records)              */
    uint64_t st_slots[GF_NSTAT];  /* ring slots per opcode                            */
    uint64_t st_wait_ns;          /* device ns spent waiting for the host             */
    uint64_t st_wait_op_ns[GF_NSTAT]; /* the same, per opcode                          */
    uint64_t st_client_ns;        /* initial thread: ns inside RPC calls outside the waits */
    uint64_t st_regions;
    uint64_t st_region_ns;        /* initial thread: publish -> all blocks done       */
    uint64_t st_heap_ns;          /* initial thread: time inside gf_malloc / gf_free   */
    uint64_t st_copy_regions;     /* regions that copied through the bulk arena        */
    uint64_t st_copy_ns;          /* their time (also counted in st_region_ns)         */
    uint64_t t_main_start, t_main_end;
    uint64_t lat_hist[GF_LAT_BUCKETS];  /* RPC round trips (claim -> host done), lane records */
    uint32_t rand_words[40];      /* rand() state of the program (device libc)        */
    gf_heap heap;
} gf_state;

#endif
