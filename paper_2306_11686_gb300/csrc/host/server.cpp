/* Host RPC server: slot scanning and the libc landing pads (see server.h). */
#include "server.h"
#include "fmt_fast.h"

#include <errno.h>
#include <fcntl.h>
#include <stdlib.h>
#include <string.h>
#include <sys/mman.h>
#include <sys/stat.h>
#include <time.h>
#include <unistd.h>

#include <algorithm>
#include <condition_variable>
#include <thread>
#include <chrono>
#include <vector>

namespace gfh {

static inline uint64_t acquire_load(const uint64_t *p) { return __atomic_load_n(p, __ATOMIC_ACQUIRE); }
static inline void release_store(uint64_t *p, uint64_t v) { __atomic_store_n(p, v, __ATOMIC_RELEASE); }
static inline uint64_t now_ns()
{
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

void Segment::reset(uint32_t nthreads)
{
    expect.resize(nslots);
    for (uint32_t s = 0; s < nslots; s++)
        expect[s] = s;                  /* slot s first carries ticket s */
    cursor.assign(nthreads, 0);
    for (uint32_t t = 0; t < nthreads; t++)
        cursor[t] = t;                  /* thread t serves slots t, t + nthreads, ... */
    passes.assign(nthreads, 0);
    pending.assign(nthreads, {});
    std::lock_guard<std::mutex> g(fmt_mu);
    fmt_cache.clear();
    fmt_local.assign(nthreads, {});
}

RecView::RecView(const uint8_t *r) : base(r)
{
    const gf_rec_hdr *h = (const gf_rec_hdr *)r;
    bytes = h->bytes;
    nargs = h->nargs;
    tags = r + sizeof(gf_rec_hdr);
    words = (const uint64_t *)(tags + ((nargs + 7u) & ~7u));
    tail = (const uint8_t *)(words + nargs);
}

/*
 * Copy threads kept for the server's life.  A large write hands every thread
 * one slice of the range and waits: creating and joining a dozen threads for
 * every 32 MiB chunk cost more than the copy itself.  One job at a time
 * (pool_mu_; large writes to different files take turns).
 */
class CopyPool {
  public:
    CopyPool()
    {
        /* page faults of distinct pages run in parallel; two cores are left
         * to the server thread and the host thread waiting on the program
         * (on a 16-core host a 128 MiB write took 1.91 ms with 14 copy
         * threads, 2.22-2.27 with 16, 1.95 with 12, 2.31 with 8) */
        const unsigned hw = std::thread::hardware_concurrency();
        const unsigned n = hw > 2 ? hw - 2 : 1;
        nthr_ = n < 4 ? 4 : n > 16 ? 16 : n;
        if (const char *e = getenv("GF_COPY_THREADS")) {  /* a fixed count, for measurement */
            const int v = atoi(e);
            if (v >= 1 && v <= 64)
                nthr_ = (unsigned)v;
        }
        for (unsigned t = 0; t < nthr_; t++)
            th_.emplace_back([this, t] { loop(t); });
    }
    ~CopyPool()
    {
        {
            std::lock_guard<std::mutex> g(mu_);
            stop_ = true;
        }
        cv_.notify_all();
        for (auto &t : th_)
            t.join();
    }
    void copy(unsigned char *dst, const unsigned char *src, uint64_t n)
    {
        std::unique_lock<std::mutex> lk(mu_);
        dst_ = dst;
        src_ = src;
        n_ = n;
        part_ = ((n + nthr_ - 1) / nthr_ + 4095) & ~4095ull;
        pending_ = nthr_;
        gen_++;
        cv_.notify_all();
        done_.wait(lk, [this] { return pending_ == 0; });
    }

  private:
    void loop(unsigned t)
    {
        uint64_t seen = 0;
        for (;;) {
            unsigned char *dst;
            const unsigned char *src;
            uint64_t lo, len = 0;
            {
                std::unique_lock<std::mutex> lk(mu_);
                cv_.wait(lk, [&] { return stop_ || gen_ != seen; });
                if (stop_)
                    return;
                seen = gen_;
                dst = dst_;
                src = src_;
                lo = (uint64_t)t * part_;
                if (lo < n_)
                    len = n_ - lo < part_ ? n_ - lo : part_;
            }
            if (len)
                memcpy(dst + lo, src + lo, len);
            std::lock_guard<std::mutex> g(mu_);
            if (--pending_ == 0)
                done_.notify_one();
        }
    }
    unsigned nthr_ = 0;
    std::vector<std::thread> th_;
    std::mutex mu_;
    std::condition_variable cv_, done_;
    bool stop_ = false;
    uint64_t gen_ = 0, n_ = 0, part_ = 0;
    unsigned pending_ = 0;
    unsigned char *dst_ = nullptr;
    const unsigned char *src_ = nullptr;
};

/*
 * fwrite of a large buffer.  A single write(2) to one file copies into the
 * page cache on one thread (the kernel serialises writers of a file), which
 * is the bottleneck for a 128 MiB write.  For a regular file not opened for
 * append, the target range is mapped instead and the pool's threads copy
 * into it (page faults of different pages proceed in parallel); the stdio
 * position is then moved past the data.  The bytes in the file are the same;
 * anything that is not a plain regular file, and small writes, use fwrite.
 *
 * A write the device sends in chunks (the halves of its bulk arena) says in
 * `rest` how many bytes remain including this chunk: when its chunks are
 * large, the file is sized and the whole range mapped once, at the first
 * chunk, and released after the last one, so the chunks cost no mapping,
 * sizing or unmapping of their own (chunks below 8 MiB go through stdio).
 * Anything else done to the stream in between, or its close, first settles
 * the mapping (bulk_settle), trimming the file to what was written when the
 * write stopped early.
 *
 * The mapping of a write that completed is not released before the reply
 * (bulk_retire): unmapping walks every page it covers (dirty state, reverse
 * map; 0.32 ms for 128 MiB on a Grace host), and the bytes are in the page
 * cache already.  The thread that served the write releases it once it has
 * been idle for GF_RETIRE_IDLE_US (idle()), so the unmap neither delays the
 * program's next call nor runs on another CPU: unmapped from another
 * thread, the file's pages cost the next open(O_TRUNC) of the file a third
 * more (0.64 against 0.48 ms for 128 MiB, measured on the same host).
 * Mappings left longer than GF_RETIRE_STALE_MS are released by any idle
 * server thread, more than GF_RETIRE_MAX at once by the writer itself, and
 * the rest by close_all.
 */
#define GF_RETIRE_IDLE_US 200
#define GF_RETIRE_STALE_MS 50
#define GF_RETIRE_MAX 16

static thread_local std::chrono::steady_clock::time_point tl_busy;   /* this thread last served a slot */

void Server::bulk_retire(Stream *st)
{
    Stream::Bulk &b = st->bulk;
    if (!b.m || b.next < b.end) {
        bulk_settle(st);
        return;
    }
    Retired r{b.m, b.mlen, b.rfd, std::this_thread::get_id(), std::chrono::steady_clock::now()};
    b = Stream::Bulk();
    Retired old{};
    {
        std::lock_guard<std::mutex> g(ret_mu_);
        retired_.push_back(r);
        if (retired_.size() > GF_RETIRE_MAX) {
            old = retired_.front();
            retired_.erase(retired_.begin());
        }
        n_retired_.store((uint32_t)retired_.size(), std::memory_order_release);
    }
    if (old.m) {
        munmap(old.m, old.len);
        close(old.fd);
    }
}

void Server::idle()
{
    if (!n_retired_.load(std::memory_order_acquire))
        return;
    const auto now = std::chrono::steady_clock::now();
    if (now - tl_busy < std::chrono::microseconds(GF_RETIRE_IDLE_US))
        return;
    std::vector<Retired> mine;
    {
        std::lock_guard<std::mutex> g(ret_mu_);
        const auto me = std::this_thread::get_id();
        for (size_t k = 0; k < retired_.size();) {
            const Retired &r = retired_[k];
            if (r.owner == me || now - r.t > std::chrono::milliseconds(GF_RETIRE_STALE_MS)) {
                mine.push_back(r);
                retired_.erase(retired_.begin() + (ptrdiff_t)k);
            } else {
                k++;
            }
        }
        n_retired_.store((uint32_t)retired_.size(), std::memory_order_release);
    }
    for (const Retired &r : mine) {
        munmap(r.m, r.len);
        close(r.fd);
    }
}

void Server::release_retired()
{
    std::vector<Retired> all;
    {
        std::lock_guard<std::mutex> g(ret_mu_);
        all.swap(retired_);
        n_retired_.store(0, std::memory_order_release);
    }
    for (const Retired &r : all) {
        munmap(r.m, r.len);
        close(r.fd);
    }
}

void Server::bulk_settle(Stream *st)
{
    Stream::Bulk &b = st->bulk;
    if (!b.m)
        return;
    munmap(b.m, b.mlen);
    if (b.next < b.end) {                        /* stopped early: drop the unwritten tail */
        const int64_t keep = b.next > b.orig ? b.next : b.orig;
        if (keep < b.end && ftruncate(b.rfd, (off_t)keep) != 0) {
            /* the file keeps its length; nothing else to undo */
        }
    }
    close(b.rfd);
    b = Stream::Bulk();
}

size_t Server::big_fwrite(Stream *st, const void *src, size_t size, size_t nmemb, uint64_t rest)
{
    FILE *f = st->f;
    Stream::Bulk &b = st->bulk;
    const uint64_t n = (uint64_t)size * nmemb;
    const uint64_t min_par = 8ull << 20;
    if (rest < n)
        rest = n;
    if (!b.m && n < min_par)                     /* small chunks: stdio (waking the pool costs more) */
        return fwrite(src, size, nmemb, f);
    if (fflush(f) != 0) {
        bulk_settle(st);
        return 0;
    }
    const off_t pos = ftello(f);
    if (b.m && (pos != (off_t)b.next || (int64_t)(pos + n) > b.end))
        bulk_settle(st);                         /* not the continuation of the mapped write */
    if (!b.m) {
        const int fd = fileno(f);
        struct stat sb;
        const int fl = fd >= 0 ? fcntl(fd, F_GETFL) : -1;
        const bool writable = fl >= 0 && ((fl & O_ACCMODE) == O_WRONLY || (fl & O_ACCMODE) == O_RDWR);
        if (fd < 0 || pos < 0 || !writable || (fl & O_APPEND) || fstat(fd, &sb) != 0 || !S_ISREG(sb.st_mode) ||
            lseek(fd, 0, SEEK_CUR) != pos)
            return fwrite(src, size, nmemb, f);
        /* a shared writable mapping needs a descriptor opened for reading too:
         * reopen the same file read-write through /proc (fall back if refused) */
        char path[64];
        snprintf(path, sizeof path, "/proc/self/fd/%d", fd);
        const int rfd = open(path, O_RDWR | O_CLOEXEC);
        if (rfd < 0)
            return fwrite(src, size, nmemb, f);
        const off_t end = pos + (off_t)rest;
        if (end > sb.st_size && ftruncate(rfd, end) != 0) {
            close(rfd);
            return fwrite(src, size, nmemb, f);
        }
        const long pg = sysconf(_SC_PAGESIZE);
        const off_t mstart = pos / pg * pg;
        const size_t mlen = (size_t)(end - mstart);
        void *m = mmap(nullptr, mlen, PROT_WRITE | PROT_READ, MAP_SHARED, rfd, mstart);
        if (m == MAP_FAILED) {
            const int bad = end > sb.st_size && ftruncate(rfd, sb.st_size) != 0;
            close(rfd);
            return bad ? 0 : fwrite(src, size, nmemb, f);
        }
        b.m = (uint8_t *)m;
        b.mlen = mlen;
        b.mstart = mstart;
        b.next = pos;
        b.end = end;
        b.orig = sb.st_size;
        b.rfd = rfd;
    }
    if (n < (1ull << 20)) {                      /* a short tail of a mapped write */
        memcpy(b.m + (pos - b.mstart), src, n);
    } else {
        std::lock_guard<std::mutex> g(pool_mu_);
        if (!pool_)
            pool_.reset(new CopyPool());
        pool_->copy(b.m + (pos - b.mstart), (const unsigned char *)src, n);
    }
    b.next = pos + (int64_t)n;
    if (b.next >= b.end)
        bulk_retire(st);
    if (fseeko(f, pos + (off_t)n, SEEK_SET) != 0)
        return 0;
    return nmemb;
}

/* Argument k of a lane record, for user landing pads (include/gf.h). */
extern "C" __attribute__((visibility("default"))) int gf_rec_arg(const void *rec, int k, uint8_t *tag, uint64_t *word,
                                                                   void **ptr, uint32_t *bytes, uint32_t *off)
{
    if (!rec)
        return -1;
    RecView r((const uint8_t *)rec);
    if (k < 0 || (uint32_t)k >= r.nargs)
        return -1;
    const uint8_t t = r.tag((uint32_t)k);
    if (tag)
        *tag = t;
    if (word)
        *word = r.word((uint32_t)k);
    const bool ref = t == GF_T_STR || t == GF_T_BLOB_R || t == GF_T_BLOB_W || t == GF_T_BLOB_RW;
    if (ptr)
        *ptr = ref ? (void *)(r.blob((uint32_t)k) + r.ptr_off((uint32_t)k)) : nullptr;
    if (bytes)
        *bytes = ref ? r.blob_len((uint32_t)k) : 8;
    if (off)
        *off = ref ? r.ptr_off((uint32_t)k) : 0;
    return 0;
}

class AsyncFile {
  public:
    explicit AsyncFile(int fd) : fd_(fd), th_([this] { loop(); }) {}
    ~AsyncFile()
    {
        {
            std::lock_guard<std::mutex> g(mu_);
            stop_ = true;
        }
        cv_.notify_all();
        th_.join();
        if (fd_ >= 0)
            ::close(fd_);
    }
    ssize_t put(const char *p, size_t n)
    {
        std::unique_lock<std::mutex> lk(mu_);
        /* bounded queue: a writer far behind holds the printing threads back */
        space_.wait(lk, [&] { return q_.size() < LIMIT || err_; });
        if (err_)
            return -1;
        q_.insert(q_.end(), p, p + n);
        queued_ += n;
        if (q_.size() >= CHUNK && !busy_)  /* wake the writer for whole chunks only */
            cv_.notify_one();
        return (ssize_t)n;
    }
    /* wait until the bytes queued before this call are in the file (bytes
     * other threads queue meanwhile are not waited for) */
    int drain()
    {
        std::unique_lock<std::mutex> lk(mu_);
        const uint64_t target = queued_;
        drain_++;
        cv_.notify_one();
        idle_.wait(lk, [&] { return written_ >= target || err_; });
        drain_--;
        return err_ ? -1 : 0;
    }
    FILE *f = nullptr;

  private:
    void loop()
    {
        std::vector<char> buf;
        for (;;) {
            {
                std::unique_lock<std::mutex> lk(mu_);
                /* large writes: wait for a chunk, a drain, or a short while */
                cv_.wait_for(lk, std::chrono::milliseconds(2),
                             [&] { return stop_ || drain_ || q_.size() >= CHUNK; });
                if (q_.empty()) {
                    if (stop_)
                        return;               /* stopping with nothing queued */
                    continue;
                }
                buf.swap(q_);
                busy_ = true;
            }
            space_.notify_all();
            size_t off = 0;
            bool bad = false;
            while (off < buf.size()) {
                const ssize_t w = ::write(fd_, buf.data() + off, buf.size() - off);
                if (w < 0 && errno == EINTR)
                    continue;
                if (w <= 0) {
                    bad = true;
                    break;
                }
                off += (size_t)w;
            }
            const uint64_t wrote = buf.size();
            buf.clear();
            {
                std::lock_guard<std::mutex> g(mu_);
                busy_ = false;
                written_ += wrote;
                if (bad)
                    err_ = true;
            }
            idle_.notify_all();
            space_.notify_all();
        }
    }
    static const size_t LIMIT = 64u << 20, CHUNK = 1u << 20;
    int drain_ = 0;
    uint64_t queued_ = 0, written_ = 0;   /* bytes queued and written since the open */
    int fd_;
    std::mutex mu_;
    std::condition_variable cv_, idle_, space_;
    std::vector<char> q_;
    bool stop_ = false, busy_ = false, err_ = false;
    std::thread th_;
};

static ssize_t async_write_fn(void *cookie, const char *p, size_t n) { return ((AsyncFile *)cookie)->put(p, n); }

AsyncFile *async_open(const char *path)
{
    const int fd = ::open(path, O_WRONLY | O_CREAT | O_TRUNC | O_CLOEXEC, 0666);
    if (fd < 0)
        return nullptr;
    AsyncFile *a = new AsyncFile(fd);
    cookie_io_functions_t io = {};
    io.write = async_write_fn;
    a->f = fopencookie(a, "w", io);
    if (!a->f) {
        delete a;
        return nullptr;
    }
    setvbuf(a->f, nullptr, _IONBF, 0);
    return a;
}

FILE *async_stream(AsyncFile *a) { return a ? a->f : nullptr; }

int async_drain(AsyncFile *a)
{
    if (!a)
        return -1;
    if (a->f)
        fflush(a->f);
    return a->drain();
}

int async_close(AsyncFile *a)
{
    if (!a)
        return -1;
    int rc = a->f ? fclose(a->f) : 0;         /* nothing is buffered in the stream itself */
    a->f = nullptr;
    if (a->drain() != 0)
        rc = -1;
    delete a;
    return rc;
}

Server::Server() : out_s_(std::make_shared<Stream>(stdout)), err_s_(std::make_shared<Stream>(stderr)) {}
Server::~Server() { close_all(); }

void Server::set_stdout(FILE *f) { out_s_ = std::make_shared<Stream>(f ? f : stdout); }
void Server::set_dma(d2h_fn d2h, h2d_fn h2d)
{
    d2h_ = d2h;
    h2d_ = h2d;
}
int Server::register_user(uint32_t opcode, user_fn fn, void *user)
{
    std::lock_guard<std::mutex> g(user_mu_);
    user_[opcode] = {fn, user};
    return 0;
}

void Server::close_all()
{
    std::unordered_map<uint64_t, std::shared_ptr<Stream>> open;
    {
        std::lock_guard<std::mutex> g(files_mu_);
        open.swap(files_);
    }
    for (auto &kv : open) {
        std::lock_guard<std::mutex> g(kv.second->mu);
        if (!kv.second->closed) {
            bulk_settle(kv.second.get());
            kv.second->closed = true;
            fclose(kv.second->f);
        }
    }
    release_retired();
    if (out_s_) {
        std::lock_guard<std::mutex> g(out_s_->mu);
        fflush(out_s_->f);
    }
}

Server::Stream *Server::stream_of(uint64_t h, std::shared_ptr<Stream> &hold)
{
    if (h == GF_STDOUT_H)
        return out_s_.get();
    if (h == GF_STDERR_H)
        return err_s_.get();
    std::lock_guard<std::mutex> g(files_mu_);
    auto it = files_.find(h);
    if (it == files_.end())
        return nullptr;
    hold = it->second;
    return hold.get();
}

bool Server::stream_valid(uint64_t h)
{
    if (h == GF_STDOUT_H || h == GF_STDERR_H)
        return true;
    std::lock_guard<std::mutex> g(files_mu_);
    return files_.count(h) != 0;
}

void Server::emit(uint64_t stream, const char *s, size_t n)
{
    if (!n)
        return;
    std::shared_ptr<Stream> hold;
    Stream *st = stream_of(stream, hold);
    if (!st)
        return;
    std::lock_guard<std::mutex> g(st->mu);
    if (!st->closed) {
        bulk_settle(st);
        fwrite(s, 1, n, st->f);
    }
}

/*
 * printf landing pad.  The format is cut once into literal runs and
 * conversions (compile_fmt); each record then appends the literals and, for
 * each conversion, snprintf with exactly that conversion and an argument of
 * the C type it names.  The output equals one printf call with the same
 * arguments, because printf's output is the concatenation of its literal
 * text and its conversions.  Plain conversions (no flags, width or '*') go
 * through gfh::fmt_fast (std::to_chars, the same characters) instead of
 * snprintf.
 */
FmtPlan compile_fmt(const char *fmt)
{
    FmtPlan pl;
    FmtConv c;
    c.lit_off = 0;
    for (const char *p = fmt; *p;) {
        if (*p != '%') {
            const char *q = strchr(p, '%');
            const size_t n = q ? (size_t)(q - p) : strlen(p);
            pl.lits.append(p, n);
            p += n;
            continue;
        }
        if (p[1] == '%') {
            pl.lits.push_back('%');
            p += 2;
            continue;
        }
        /* %[flags][width][.prec][length]conv */
        const char *s0 = p++;
        while (*p && strchr("-+ #0'", *p))
            p++;
        const bool flags = p != s0 + 1;
        bool width = false;
        if (*p == '*') {
            c.star_w = true;
            p++;
        } else
            while (*p >= '0' && *p <= '9') {
                width = true;
                p++;
            }
        if (*p == '.') {
            p++;
            if (*p == '*') {
                c.star_p = true;
                p++;
            } else {
                c.prec = 0;
                while (*p >= '0' && *p <= '9') {
                    c.prec = c.prec < 100000 ? c.prec * 10 + (*p - '0') : c.prec;
                    p++;
                }
            }
        }
        if (*p == 'h' || *p == 'l') {
            c.len[0] = *p++;
            if (*p == c.len[0])
                c.len[1] = *p++;
        } else if (*p == 'j' || *p == 'z' || *p == 't' || *p == 'L' || *p == 'q') {
            c.len[0] = *p++;
        }
        if (!*p)                        /* a conversion cut off by the end: output stops here */
            break;
        c.conv = *p++;
        c.lit_len = (uint32_t)pl.lits.size() - c.lit_off;
        c.spec.assign(s0, (size_t)(p - s0));
        c.bad = c.spec.size() >= 64;
        c.plain = !flags && !width && !c.star_w && !c.star_p;
        pl.convs.push_back(c);
        if (c.bad)
            return pl;
        c = FmtConv();
        c.lit_off = (uint32_t)pl.lits.size();
    }
    c.conv = 0;
    c.lit_len = (uint32_t)pl.lits.size() - c.lit_off;
    pl.convs.push_back(c);
    return pl;
}

int64_t Server::do_printf(const FmtPlan &pl, const uint8_t *recp, OutBuf &out, uint64_t *stream)
{
    RecView r(recp);
    if (r.nargs < 1)
        return -1;
    *stream = r.word(0);
    uint32_t ai = 1;
    const size_t start = out.size();
    char buf[512];
    const size_t FAST = 512;             /* room for any conversion fmt_fast takes */
    for (const FmtConv &c : pl.convs) {
        out.append(pl.lits.data() + c.lit_off, c.lit_len);
        if (!c.conv)
            break;
        if (c.bad)
            return -1;
        const char *spec = c.spec.c_str();
        const char conv = c.conv;
        const char *len = c.len;
        const bool star_w = c.star_w, star_p = c.star_p;
        int wv = 0, pv = 0;
        if (star_w) {
            if (ai >= r.nargs)
                break;
            wv = (int)(int64_t)r.word(ai++);
        }
        if (star_p) {
            if (ai >= r.nargs)
                break;
            pv = (int)(int64_t)r.word(ai++);
        }
        if (conv == 'n') {           /* no host-side write-back of %n */
            if (ai < r.nargs)
                ai++;
            continue;
        }
        if (ai >= r.nargs)
            break;
        const uint32_t k = ai++;
        const uint64_t w = r.word(k);
        int n = 0;
        if (c.plain && gfh::fmt_fast(conv, len, c.prec, w, r.tag(k) == GF_T_F64, out.room(FAST), FAST, &n)) {
            out.commit((size_t)n);
            continue;
        }
        char *dst = buf;
        std::string big;
#define GF_FMT(VAL)                                                                                 \
    do {                                                                                            \
        if (star_w && star_p)                                                                       \
            n = snprintf(dst, sizeof(buf), spec, wv, pv, VAL);                                      \
        else if (star_w || star_p)                                                                  \
            n = snprintf(dst, sizeof(buf), spec, star_w ? wv : pv, VAL);                            \
        else                                                                                        \
            n = snprintf(dst, sizeof(buf), spec, VAL);                                              \
        if (n >= (int)sizeof(buf)) {                                                                \
            big.resize((size_t)n + 1);                                                              \
            if (star_w && star_p)                                                                   \
                snprintf(&big[0], big.size(), spec, wv, pv, VAL);                                   \
            else if (star_w || star_p)                                                              \
                snprintf(&big[0], big.size(), spec, star_w ? wv : pv, VAL);                         \
            else                                                                                    \
                snprintf(&big[0], big.size(), spec, VAL);                                           \
            dst = &big[0];                                                                          \
        }                                                                                           \
    } while (0)
        switch (conv) {
        case 'd':
        case 'i':
            if (len[0] == 'l' && len[1] == 'l')
                GF_FMT((long long)w);
            else if (len[0] == 'l' || len[0] == 'j' || len[0] == 'z' || len[0] == 't' || len[0] == 'q')
                GF_FMT((long)w);
            else if (len[0] == 'h' && len[1] == 'h')
                GF_FMT((int)(signed char)w);
            else if (len[0] == 'h')
                GF_FMT((int)(short)w);
            else
                GF_FMT((int)w);
            break;
        case 'u':
        case 'o':
        case 'x':
        case 'X':
            if (len[0] == 'l' && len[1] == 'l')
                GF_FMT((unsigned long long)w);
            else if (len[0] == 'l' || len[0] == 'j' || len[0] == 'z' || len[0] == 't' || len[0] == 'q')
                GF_FMT((unsigned long)w);
            else if (len[0] == 'h' && len[1] == 'h')
                GF_FMT((unsigned)(unsigned char)w);
            else if (len[0] == 'h')
                GF_FMT((unsigned)(unsigned short)w);
            else
                GF_FMT((unsigned)w);
            break;
        case 'c':
            GF_FMT((int)w);
            break;
        case 'e':
        case 'E':
        case 'f':
        case 'F':
        case 'g':
        case 'G':
        case 'a':
        case 'A': {
            double d;
            memcpy(&d, &w, 8);
            if (r.tag(k) != GF_T_F64) /* an integer passed to a float conversion */
                d = (double)(int64_t)w;
            if (len[0] == 'L')
                GF_FMT((long double)d);
            else
                GF_FMT(d);
            break;
        }
        case 's': {
            const char *sv = r.tag(k) == GF_T_STR ? r.str(k) : (w == 0 ? "(null)" : "(?)");
            GF_FMT(sv);
            break;
        }
        case 'p':
            GF_FMT((void *)(uintptr_t)w);
            break;
        default:
            out.append(spec, c.spec.size());
            continue;
        }
#undef GF_FMT
        if (n > 0)
            out.append(dst, (size_t)n);
    }
    return (int64_t)(out.size() - start);
}

int64_t Server::call(uint32_t op, const char *fmt, const uint8_t *rec, Segment *seg)
{
    RecView r(rec);
    switch (op) {
    case GF_OP_PRINTF: {
        if (!fmt)
            return -1;
        OutBuf s;
        uint64_t stream = 0;
        int64_t n = do_printf(compile_fmt(fmt), rec, s, &stream);
        if (n >= 0) {
            if (!stream_valid(stream))
                return -1;
            emit(stream, s.data(), s.size());
        }
        return n;
    }
    case GF_OP_FOPEN: {
        if (r.nargs < 2 || r.tag(0) != GF_T_STR || r.tag(1) != GF_T_STR)
            return 0;
        FILE *f = fopen(r.str(0), r.str(1));
        if (!f)
            return 0;
        std::lock_guard<std::mutex> g(files_mu_);
        files_[(uint64_t)(uintptr_t)f] = std::make_shared<Stream>(f);
        return (int64_t)(uintptr_t)f;
    }
    case GF_OP_FCLOSE: {
        if (r.nargs < 1)
            return -1;
        const uint64_t h = r.word(0);
        std::shared_ptr<Stream> st;
        {
            std::lock_guard<std::mutex> g(files_mu_);
            auto it = files_.find(h);
            if (it == files_.end())
                return -1;
            st = it->second;
            files_.erase(it);
        }
        std::lock_guard<std::mutex> g(st->mu);   /* after the stream's pending writes */
        if (st->closed)
            return -1;
        bulk_settle(st.get());
        st->closed = true;
        return fclose(st->f);
    }
    case GF_OP_FFLUSH: {
        if (r.nargs < 1)
            return -1;
        std::shared_ptr<Stream> hold;
        Stream *st = stream_of(r.word(0), hold);
        if (!st)
            return -1;
        std::lock_guard<std::mutex> g(st->mu);
        if (st->closed)
            return -1;
        bulk_settle(st);
        return fflush(st->f);
    }
    case GF_OP_FWRITE:
    case GF_OP_FREAD: {
        /* (size, nmemb, FILE*, blob | DMA addr + bytes) */
        if (r.nargs < 4)
            return 0;
        const uint64_t size = r.word(0), nmemb = r.word(1);
        std::shared_ptr<Stream> hold;
        Stream *st = stream_of(r.word(2), hold);
        if (!st || size == 0)
            return 0;
        const uint64_t bytes = size * nmemb;
        if (op == GF_OP_FWRITE && r.tag(3) == GF_T_DMA) {
            /* device memory to the stream: the first chunk's copy runs
             * before the stream's lock is taken (other server threads may
             * write the same file meanwhile); from the first byte written
             * the lock is held to the end, so the fwrite stays whole */
            if (!d2h_)
                return 0;
            std::unique_lock<std::mutex> lk(st->mu, std::defer_lock);
            bool open = true;
            const uint64_t done = d2h_(
                r.word(3), bytes,
                [&](const void *c, uint64_t n, uint64_t) {
                    if (!lk.owns_lock()) {
                        lk.lock();
                        if (st->closed) {
                            open = false;
                            return false;
                        }
                        bulk_settle(st);
                    }
                    return fwrite(c, 1, n, st->f) == n;
                },
                false);
            stats.dma_bytes += done;
            return open ? (int64_t)(done / size) : 0;
        }
        if (op == GF_OP_FREAD && r.tag(3) == GF_T_DMA) {
            /* the stream to device memory: the lock is taken at the first
             * read, inside the DMA lane's own lock, the same order as fwrite
             * takes them (a lane is shared by server threads tid, tid + 8, ...) */
            if (!h2d_)
                return 0;
            std::unique_lock<std::mutex> lk(st->mu, std::defer_lock);
            bool open = true;
            const uint64_t done = h2d_(r.word(3), bytes, [&](void *c, uint64_t want) -> uint64_t {
                if (!lk.owns_lock()) {
                    lk.lock();
                    if (st->closed) {
                        open = false;
                        return 0;
                    }
                    bulk_settle(st);
                }
                return (uint64_t)fread(c, 1, want, st->f);
            });
            stats.dma_bytes += done;
            return open ? (int64_t)(done / size) : 0;
        }
        std::lock_guard<std::mutex> g(st->mu);   /* the whole transfer */
        if (st->closed)
            return 0;
        FILE *f = st->f;
        if (r.tag(3) == GF_T_ARENA) {
            /* staged in the bulk arena by the device grid (fwrite) or to be
             * copied out of it by the grid (fread) */
            const uint64_t off = r.word(3);
            const uint64_t len = r.nargs > 4 ? r.word(4) : 0;
            if (!seg || !seg->bulk || off + len > seg->bulk_bytes || len < bytes)
                return 0;
            /* bytes of the whole chunked write still to come, this chunk included */
            const uint64_t rest = r.nargs > 5 ? r.word(5) : bytes;
            if (op != GF_OP_FWRITE)
                bulk_settle(st);
            const size_t k = op == GF_OP_FWRITE ? big_fwrite(st, seg->bulk + off, size, nmemb, rest)
                                                : fread(seg->bulk + off, size, nmemb, f);
            stats.dma_bytes += k * size;
            return (int64_t)k;
        }
        bulk_settle(st);
        if (r.tag(3) != GF_T_DMA) {
            uint8_t *b = r.blob(3);
            if (r.blob_len(3) < bytes)
                return 0;
            return op == GF_OP_FWRITE ? (int64_t)fwrite(b, size, nmemb, f) : (int64_t)fread(b, size, nmemb, f);
        }
        return 0;                                /* an argument tag this call does not take */
    }
    case GF_OP_CLOCK:
        return (int64_t)clock();
    case GF_OP_REGION:
        /* the kernel split: launch the region, answer at once (the device
         * waits for the kernel's blocks; a server thread never blocks here) */
        if (!region_)
            return -1;
        return region_(seg ? seg->prog : (r.nargs ? (uint32_t)r.word(0) : 0u));
    case GF_OP_STRTOD: {
        /* the device's slow path: exact conversion by the host libc */
        if (r.nargs < 2 || r.tag(0) != GF_T_STR || r.tag(1) != GF_T_BLOB_W || r.blob_len(1) < 8)
            return 0;
        const char *s = r.str(0);
        char *end = nullptr;
        const double v = strtod(s, &end);
        const int64_t used = (int64_t)(end - s);
        memcpy(r.blob(1), &used, 8);
        int64_t bits;
        memcpy(&bits, &v, 8);
        return bits;
    }
    case GF_OP_GETENV: {
        if (r.nargs < 1 || r.tag(0) != GF_T_STR || !intern_)
            return 0;
        std::string name = r.str(0);
        std::lock_guard<std::mutex> g(intern_mu_);
        auto it = interned_.find(name);
        if (it != interned_.end())
            return (int64_t)it->second;
        const char *v = getenv(name.c_str());
        uint64_t a = v ? intern_(std::string(v)) : 0;
        interned_[name] = a;
        return (int64_t)a;
    }
    default: {
        std::pair<user_fn, void *> u{nullptr, nullptr};
        {
            std::lock_guard<std::mutex> g(user_mu_);
            auto it = user_.find(op);
            if (it != user_.end())
                u = it->second;
        }
        if (!u.first)
            return -1;
        return u.first(u.second, op, (void *)rec);
    }
    }
}

/* each server thread's text buffer, kept between passes so it is not
 * reallocated for every pass */
static OutBuf &tl_out()
{
    thread_local OutBuf b;
    return b;
}

int Server::poll(Segment &seg, uint32_t tid, uint32_t nthr)
{
    /* announce this poller before looking at `active`: whoever clears
     * `active` and then sees no pollers knows nobody reads the segment */
    seg.pollers.fetch_add(1, std::memory_order_seq_cst);
    const int n = seg.active.load(std::memory_order_seq_cst) ? poll_active(seg, tid, nthr) : 0;
    seg.pollers.fetch_sub(1, std::memory_order_release);
    if (n)
        tl_busy = std::chrono::steady_clock::now();
    return n;
}

int Server::poll_active(Segment &seg, uint32_t tid, uint32_t nthr)
{
    const uint32_t N = seg.nslots;
    int served = 0;
    uint32_t gap = 0;
    /* counters kept per call and added to the shared ones once at the end:
     * per-slot atomic adds from every server thread made the counters' cache
     * lines bounce between cores */
    uint64_t n_rec = 0, n_ns = 0, n_ring = 0, n_op[GF_NSTAT] = {};
    /* printf text of consecutive slots to one stream is written in one go;
     * those slots are released only after their text reached the stream, so
     * one device thread's calls still appear in program order */
    OutBuf &out = tl_out();
    out.clear();
    uint64_t out_stream = 0;
    uint64_t *held[16];
    uint64_t held_t[16];
    uint32_t nheld = 0;
    auto flush = [&]() {
        if (!out.empty())
            emit(out_stream, out.data(), out.size());
        out.clear();
        for (uint32_t k = 0; k < nheld; k++)
            release_store(held[k], held_t[k]);
        nheld = 0;
    };
    std::unordered_map<uint64_t, const FmtEntry *> *local =
        tid < seg.fmt_local.size() ? &seg.fmt_local[tid] : nullptr;
    /* Claims arrive in ticket order, so the next request is usually in the
     * slot after the last one served: start there and stop after a run of
     * quiet slots.  A slot passed while its claimant was still writing it
     * (its ticket below one served later) goes on this thread's pending
     * list; every 64th pass also scans all of this thread's slots. */
    /* serve slot s if it holds its expected ticket's published request */
    auto try_slot = [&](uint32_t s) -> bool {
        uint8_t *slot = seg.slots + (uint64_t)s * seg.slot_bytes;
        gf_slot_hdr *h = (gf_slot_hdr *)slot;
        const uint64_t t = seg.expect[s];
        const uint64_t q = acquire_load(&h->seq);
        if (q != t + 1)
            return false;
        const uint64_t t0 = now_ns();
        const uint32_t op = h->opcode, nl = h->nlanes;
        uint8_t *pay = slot + GF_SLOT_PAYLOAD_OFF;
        const FmtEntry *fe = nullptr;
        if (h->flags & GF_SF_FMT_INLINE) {
            const char *inl = (const char *)pay;
            {
                std::lock_guard<std::mutex> g(seg.fmt_mu);
                auto ins = seg.fmt_cache.try_emplace(h->fmt_key);
                if (ins.second) {          /* first sight: keep the text and its compiled form */
                    ins.first->second.text.assign(inl, strnlen(inl, h->fmt_len));
                    ins.first->second.plan = compile_fmt(ins.first->second.text.c_str());
                }
                fe = &ins.first->second;
            }
            if (local)
                (*local)[h->fmt_key] = fe;
            pay += (h->fmt_len + 7u) & ~7u;
        } else if (h->fmt_key) {
            if (local) {
                auto it = local->find(h->fmt_key);
                if (it != local->end())
                    fe = it->second;
            }
            if (!fe) {
                std::lock_guard<std::mutex> g(seg.fmt_mu);
                auto it = seg.fmt_cache.find(h->fmt_key);
                if (it != seg.fmt_cache.end()) {
                    fe = &it->second;
                    if (local)
                        (*local)[h->fmt_key] = fe;
                }
            }
            /* a key never shipped: printf answers -1 per lane (no format) */
        }
        int64_t *ret = (int64_t *)(slot + GF_SLOT_RET_OFF);
        const uint8_t *end = slot + seg.slot_bytes;
        bool hold = false;
        if (op == GF_OP_PRINTF) {
            /* all lanes of a slot share one format: format them into the
             * pending text of their stream */
            const size_t mark = out.size();
            uint64_t stream = 0;
            bool first = true, bad_stream = false;
            for (uint32_t l = 0; l < nl && l < 32; l++) {
                const gf_rec_hdr *rh = (const gf_rec_hdr *)pay;
                if (pay + sizeof(gf_rec_hdr) > end || rh->bytes < sizeof(gf_rec_hdr) || pay + rh->bytes > end) {
                    ret[l] = -1;
                    continue;
                }
                uint64_t st = 0;
                const size_t before = out.size();
                if (first) {
                    /* peek at the lane's stream before formatting into the buffer */
                    const RecView rv(pay);
                    st = rv.nargs ? rv.word(0) : 0;
                    if (st != out_stream)
                        flush();
                    out_stream = st;
                    stream = st;
                    first = false;
                }
                ret[l] = fe ? do_printf(fe->plan, pay, out, &st) : -1;
                if (st != stream) {                    /* lanes writing to different streams */
                    const std::string tail(out.data() + before, out.size() - before);
                    out.shrink(before);
                    flush();
                    out.append(tail.data(), tail.size());
                    out_stream = stream = st;
                }
                pay += rh->bytes;
            }
            if (!first && !stream_valid(stream)) {
                bad_stream = true;
                out.shrink(mark);
            }
            if (bad_stream)
                for (uint32_t l = 0; l < nl && l < 32; l++)
                    ret[l] = -1;
            hold = true;
        } else {
            flush();                                   /* earlier text first: other calls may touch the same files */
            for (uint32_t l = 0; l < nl && l < 32; l++) {
                const gf_rec_hdr *rh = (const gf_rec_hdr *)pay;
                if (pay + sizeof(gf_rec_hdr) > end || rh->bytes < sizeof(gf_rec_hdr) || pay + rh->bytes > end) {
                    ret[l] = -1;
                    continue;
                }
                ret[l] = call(op, fe ? fe->text.c_str() : nullptr, pay, &seg);
                pay += rh->bytes;
            }
        }
        const uint64_t dt = now_ns() - t0;
        h->t_host_ns = dt;
        served++;
        n_rec += nl;
        n_ns += dt;
        n_ring += (uint64_t)(pay - slot) + 8ull * nl;
        n_op[op < GF_NSTAT ? op : 0] += nl;
        seg.expect[s] = t + N;
        if (hold) {
            held[nheld] = &h->seq;
            held_t[nheld] = t + 2;
            if (++nheld == 16 || out.size() >= (16u << 10))
                flush();
        } else {
            release_store(&h->seq, t + 2);
        }
        return true;
    };
    /* slots whose ticket was claimed before a later one was served, but
     * which were still unpublished when the scan passed them: looked at
     * first, every pass, until served (a slow claimant costs one load per
     * pass instead of waiting for the full scan) */
    std::vector<uint32_t> &pend = seg.pending[tid];
    for (size_t i = 0; i < pend.size();) {
        if (try_slot(pend[i])) {
            pend[i] = pend.back();
            pend.pop_back();
        } else {
            i++;
        }
    }
    const bool full = (++seg.passes[tid] & 63u) == 0;
    uint32_t s = seg.cursor[tid];
    uint32_t quiet[64];
    uint32_t nq = 0;
    for (uint32_t k = 0; k < N; k += nthr, s = (s + nthr) % N) {
        if (!full && gap >= 64)
            break;
        if (!try_slot(s)) {
            gap++;
            if (nq < 64)
                quiet[nq++] = s;
            continue;
        }
        gap = 0;
        seg.cursor[tid] = (s + nthr) % N;
        /* the quiet slots just passed hold lower tickets than this one: their
         * claimants exist (tickets are handed out in order) */
        const uint64_t ts = seg.expect[s] - N;
        for (uint32_t j = 0; j < nq; j++)
            if (seg.expect[quiet[j]] < ts && pend.size() < 256 &&
                std::find(pend.begin(), pend.end(), quiet[j]) == pend.end())
                pend.push_back(quiet[j]);
        nq = 0;
    }
    flush();
    if (served) {
        stats.slots += (uint64_t)served;
        stats.records += n_rec;
        stats.ns += n_ns;
        stats.ring_bytes += n_ring;
        for (int k = 0; k < GF_NSTAT; k++)
            if (n_op[k])
                stats.per_op[k] += n_op[k];
    }
    return served;
}

} // namespace gfh
