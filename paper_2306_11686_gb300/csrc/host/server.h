/*
 * Host RPC server: the paper's single RPC thread next to the offload runtime
 * (Sec. 3.1, Fig. 2) and its generated landing pads (Sec. 3.2, Fig. 4b).
 *
 * The server owns no CUDA state: ring segments are plain memory (pinned and
 * device-mapped in production, ordinary memory when CPU threads stand in for
 * the device in tests), and device memory is reached only through the DMA and
 * intern callbacks.  Landing pads are keyed by opcode; printf-style calls are
 * formatted by the real libc one conversion at a time with the C type that
 * the conversion names, which is the per-signature non-variadic landing pad
 * of the paper built at run time from the argument tags.
 *
 * Ordering: a segment is scanned from its lowest unserved ticket; published
 * slots are served as found (out of ticket order when an earlier claimant is
 * slow), and a slot's "done" is released only after its output has reached
 * the stream, so one device thread's successive calls appear in program order.
 */
#ifndef GF_HOST_SERVER_H
#define GF_HOST_SERVER_H

#include <stdint.h>
#include <stdio.h>
#include <string.h>
#include <atomic>
#include <chrono>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../gf_layout.h"

namespace gfh {

/* Growable output text whose appends are inline (a slot's 32 records make
 * a hundred or more small appends). */
class OutBuf {
  public:
    size_t size() const { return n_; }
    bool empty() const { return n_ == 0; }
    const char *data() const { return p_.get(); }
    void clear() { n_ = 0; }
    void shrink(size_t n) { n_ = n < n_ ? n : n_; }
    /* at least k writable bytes at the end; commit() what was written */
    char *room(size_t k)
    {
        if (n_ + k > cap_)
            grow(n_ + k);
        return p_.get() + n_;
    }
    void commit(size_t k) { n_ += k; }
    void append(const char *s, size_t k)
    {
        if (k) {
            memcpy(room(k), s, k);
            n_ += k;
        }
    }

  private:
    void grow(size_t need)
    {
        size_t c = cap_ ? cap_ : 4096;
        while (c < need)
            c *= 2;
        std::unique_ptr<char[]> q(new char[c]);
        if (n_)
            memcpy(q.get(), p_.get(), n_);
        p_ = std::move(q);
        cap_ = c;
    }
    std::unique_ptr<char[]> p_;
    size_t n_ = 0, cap_ = 0;
};

/* A printf format cut once into literal runs and conversions, so the
 * records of a slot (up to 32 with one format) do not parse it again. */
struct FmtConv {
    uint32_t lit_off = 0, lit_len = 0;   /* the literal text before it, in FmtPlan::lits */
    char conv = 0;                        /* 0: the format ends after the literal        */
    char len[3] = {0, 0, 0};              /* length modifier                             */
    int prec = -1;                        /* -1: none given                              */
    bool plain = false;                   /* no flags, width or '*'                      */
    bool star_w = false, star_p = false;
    bool bad = false;                     /* conversion too long: the call fails here    */
    std::string spec;                     /* the whole conversion, for snprintf          */
};
struct FmtPlan {
    std::string lits;
    std::vector<FmtConv> convs;
};
FmtPlan compile_fmt(const char *fmt);

struct FmtEntry {
    std::string text;
    FmtPlan plan;
};

struct Segment {
    uint8_t *slots = nullptr;       /* host address of slot 0                        */
    uint32_t nslots = 0, slot_bytes = 0;
    uint32_t prog = 0;
    uint8_t *bulk = nullptr;        /* host address of the bulk arena (large fwrite/fread) */
    uint64_t bulk_bytes = 0;
    std::atomic<bool> active{false};
    /* server threads inside poll() for this segment; the runtime waits for
     * zero after clearing `active` before it hands the slots to another
     * program */
    std::atomic<int> pollers{0};
    /* scan state: each slot is served for its own next ticket, so a claimant
     * that never publishes blocks only its slot, not the ring */
    std::vector<uint64_t> expect;   /* next ticket each slot will carry               */
    std::vector<uint32_t> cursor;   /* per server thread: slot to start the next scan */
    std::vector<uint32_t> passes;   /* per server thread: scans so far                */
    std::vector<std::vector<uint32_t>> pending;   /* per server thread: claimed slots the scan
                                                     passed before their publication         */
    std::unordered_map<uint64_t, FmtEntry> fmt_cache;      /* fmt_key -> format (never overwritten) */
    std::mutex fmt_mu;
    /* per server thread: fmt_key -> the entry in fmt_cache, so a thread
     * takes the shared lock only for a format it has not seen */
    std::vector<std::unordered_map<uint64_t, const FmtEntry *>> fmt_local;
    void reset(uint32_t nthreads);
};

/* Streams a device range to `sink` chunk by chunk (fwrite DMA); `pos` is the
 * chunk's offset in the range.  With parallel = false chunks arrive in order
 * from one thread; with parallel = true they may arrive from several threads
 * at once and out of order (the sink writes at pos).  Returns the length of
 * the prefix the sink accepted; the sink returns false to stop. */
typedef std::function<bool(const void *chunk, uint64_t n, uint64_t pos)> sink_fn;
typedef std::function<uint64_t(uint64_t dev_src, uint64_t bytes, const sink_fn &sink, bool parallel)> d2h_fn;
/* Fills a device range from `source` chunk by chunk (fread DMA); the source
 * returns how many bytes it produced (fewer ends the transfer). */
typedef std::function<uint64_t(void *buf, uint64_t want)> source_fn;
typedef std::function<uint64_t(uint64_t dev_dst, uint64_t bytes, const source_fn &src)> h2d_fn;
/* returns a device-readable address of a stable copy of s (getenv interning) */
typedef std::function<uint64_t(const std::string &s)> intern_fn;
/* launches instance `idx`'s region kernel (kernel split); its grid, or < 0 */
typedef std::function<int64_t(uint32_t idx)> region_fn;
typedef int64_t (*user_fn)(void *user, uint32_t opcode, void *rec);

struct HostStats {
    std::atomic<uint64_t> slots{0}, records{0}, ns{0}, dma_bytes{0};
    std::atomic<uint64_t> ring_bytes{0};   /* slot bytes crossing the link: records in, returns out */
    std::atomic<uint64_t> per_op[GF_NSTAT];
    HostStats()
    {
        for (auto &x : per_op)
            x = 0;
    }
};

class CopyPool;

/* A stdio stream whose bytes a thread of its own writes to the file: a write
 * through the stream only queues the bytes (the stream is unbuffered, so
 * they are queued in call order), and the threads that print never wait for
 * the kernel's write of the file, which is serial per file.  async_drain
 * waits until everything queued is in the file (0, or -1 after a failed
 * write); async_close closes the stream, drains and frees. */
class AsyncFile;
AsyncFile *async_open(const char *path);      /* nullptr if the file cannot be opened */
FILE *async_stream(AsyncFile *a);
int async_drain(AsyncFile *a);
int async_close(AsyncFile *a);

class Server {
  public:
    Server();
    ~Server();
    void set_stdout(FILE *f);
    void set_dma(d2h_fn d2h, h2d_fn h2d);
    void set_intern(intern_fn f) { intern_ = f; }
    void set_region(region_fn f) { region_ = f; }
    int register_user(uint32_t opcode, user_fn fn, void *user);

    /* serve every published slot of `seg` that belongs to server thread `tid`
     * of `nthreads`; returns the number of slots served */
    int poll(Segment &seg, uint32_t tid, uint32_t nthreads);

    /* close FILE*s the programs left open (and release retired mappings) */
    void close_all();
    /* a server thread with nothing to serve calls this: it releases the
     * mappings of the large writes it served once it has been idle a while */
    void idle();
    HostStats stats;

    /* one landing pad: exposed for tests that decode a record by hand */
    int64_t call(uint32_t opcode, const char *fmt, const uint8_t *rec, Segment *seg = nullptr);

  private:
    int poll_active(Segment &seg, uint32_t tid, uint32_t nthreads);
    int64_t do_printf(const FmtPlan &plan, const uint8_t *rec, OutBuf &out, uint64_t *stream);
    /* A stream the device can name: stdout, stderr, or a FILE it opened.
     * Each has its own lock, which orders that stream's writes, reads,
     * flushes and close; different streams proceed in parallel. */
    struct Stream {
        explicit Stream(FILE *x) : f(x) {}
        FILE *f;
        std::mutex mu;
        bool closed = false;
        /* a large write in progress, arriving in chunks: the file range of
         * the whole write, sized and mapped at its first chunk */
        struct Bulk {
            uint8_t *m = nullptr;
            size_t mlen = 0;
            int64_t mstart = 0, next = 0, end = 0, orig = 0;
            int rfd = -1;
        } bulk;
    };
    /* the stream named h, or nullptr; a FILE the device opened is kept alive
     * through `hold` (stdout and stderr live as long as the server and are
     * returned without touching a shared count) */
    Stream *stream_of(uint64_t h, std::shared_ptr<Stream> &hold);
    bool stream_valid(uint64_t h);
    void emit(uint64_t stream, const char *s, size_t n);

    std::shared_ptr<Stream> out_s_, err_s_;
    std::mutex files_mu_;
    std::unordered_map<uint64_t, std::shared_ptr<Stream>> files_;
    std::mutex pool_mu_;                 /* one large write through the copy pool at a time */
    d2h_fn d2h_;
    h2d_fn h2d_;
    region_fn region_;
    intern_fn intern_;
    std::mutex intern_mu_;
    std::map<std::string, uint64_t> interned_;
    std::mutex user_mu_;
    std::map<uint32_t, std::pair<user_fn, void *>> user_;
    std::unique_ptr<CopyPool> pool_;   /* copy threads of large writes, started on first use */
    /* mappings of finished large writes, released later by idle() */
    struct Retired {
        void *m;
        size_t len;
        int fd;
        std::thread::id owner;       /* the server thread that served the write */
        std::chrono::steady_clock::time_point t;
    };
    std::mutex ret_mu_;
    std::vector<Retired> retired_;
    std::atomic<uint32_t> n_retired_{0};
    void release_retired();
    size_t big_fwrite(Stream *st, const void *src, size_t size, size_t nmemb, uint64_t rest);
    void bulk_settle(Stream *st);
    void bulk_retire(Stream *st);
};

/* record accessors (shared with tests) */
struct RecView {
    const uint8_t *base;
    uint32_t bytes, nargs;
    const uint8_t *tags;
    const uint64_t *words;
    const uint8_t *tail;
    explicit RecView(const uint8_t *r);
    uint8_t tag(uint32_t k) const { return tags[k]; }
    uint64_t word(uint32_t k) const { return words[k]; }
    /* reference arguments: word = object bytes << 32 | pointer offset << 16 | tail offset */
    const char *str(uint32_t k) const { return (const char *)(tail + (uint32_t)(words[k] & 0xffffu)); }
    uint32_t blob_len(uint32_t k) const { return (uint32_t)(words[k] >> 32); }
    uint32_t ptr_off(uint32_t k) const { return (uint32_t)((words[k] >> 16) & 0xffffu); }
    uint8_t *blob(uint32_t k) const { return (uint8_t *)(tail + (uint32_t)(words[k] & 0xffffu)); }
};

} // namespace gfh
#endif
