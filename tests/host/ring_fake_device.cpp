/*
 * Host-only test of the RPC ring protocol and the host server: CPU threads
 * stand in for device warps.  They claim tickets, wait for slot credit, write
 * lane records in the device's layout, publish with a release store, wait for
 * the host's release of the returns and hand the slot back, exactly as the
 * device client does with st.release.sys / ld.acquire.sys.
 *
 *   ring_fake_device <scenario> <out_path>
 *
 * Scenarios (each prints "OK" and exits 0, or prints the failure and exits 1):
 *   basic      16 producers x 2000 calls over 8 slots (credit exhaustion, wrap)
 *   aggregate  producers write 1..32 records per slot (warp aggregation)
 *   ooo        a producer holds a claimed slot unpublished while others pass it
 *   dead       a producer dies after claiming a slot: others finish or time out
 *              (bounded), nobody hangs
 *   stall      the server pauses: producers report a timeout, then recover
 *   threads    4 server threads, per-producer order still holds
 *   fmtcache   the format ships once; later slots carry only its key
 *   bulkfile   large fwrites from the bulk arena between small inline ones
 *   bulkchunks large fwrites in chunks mapped once, and writes cut short
 *   closerace  fclose while other producers write and flush the same file
 *   retire     mappings of finished large writes while no server thread goes
 *              idle: at most 16 are kept, stale ones are released by any idle
 *              thread, closing the server releases the rest
 */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <map>
#include <string>
#include <thread>
#include <vector>

#include "gf.h"
#include "host/server.h"

using clk = std::chrono::steady_clock;

struct Ring {
    std::vector<uint8_t> mem;
    uint32_t nslots, slot_bytes;
    std::atomic<uint64_t> ticket{0};
    gfh::Segment seg;
    Ring(uint32_t n, uint32_t sb) : mem((size_t)n * sb, 0), nslots(n), slot_bytes(sb)
    {
        for (uint32_t k = 0; k < n; k++)
            hdr(k)->seq = k;
        seg.slots = mem.data();
        seg.nslots = n;
        seg.slot_bytes = sb;
    }
    gf_slot_hdr *hdr(uint64_t t) { return (gf_slot_hdr *)(mem.data() + (t % nslots) * (uint64_t)slot_bytes); }
};

static uint64_t acq(const uint64_t *p) { return __atomic_load_n(p, __ATOMIC_ACQUIRE); }
static void rel(uint64_t *p, uint64_t v) { __atomic_store_n(p, v, __ATOMIC_RELEASE); }

/* one printf record: stream handle, then (int producer, int seq) in the device layout */
static uint32_t put_rec(uint8_t *dst, uint32_t lane, int a, int b)
{
    const uint32_t nargs = 3, bytes = 16 + 8 + 8 * nargs;
    uint64_t *w = (uint64_t *)dst;
    w[0] = (uint64_t)bytes | ((uint64_t)nargs << 32) | ((uint64_t)lane << 48);
    w[1] = 0;
    w[2] = (uint64_t)'L' | ((uint64_t)'i' << 8) | ((uint64_t)'i' << 16);
    w[3] = GF_STDOUT_H;
    w[4] = (uint64_t)(int64_t)a;
    w[5] = (uint64_t)(int64_t)b;
    return bytes;
}

/* a general lane record: value words and string / blob tails in the device layout */
struct Arg {
    char tag;
    uint64_t word;
    std::string bytes;     /* for 's' (with NUL) and 'b' */
};
static uint32_t put_args(uint8_t *dst, const std::vector<Arg> &args)
{
    const uint32_t n = (uint32_t)args.size();
    uint32_t tail = 0;
    std::vector<uint64_t> words(n);
    for (uint32_t k = 0; k < n; k++) {
        words[k] = args[k].word;
        if (args[k].tag == 's' || args[k].tag == 'b') {
            words[k] = ((uint64_t)args[k].bytes.size() << 32) | tail;
            tail += ((uint32_t)args[k].bytes.size() + 7u) & ~7u;
        }
    }
    const uint32_t bytes = 16 + ((n + 7u) & ~7u) + 8 * n + tail;
    memset(dst, 0, bytes);
    uint64_t *w = (uint64_t *)dst;
    w[0] = (uint64_t)bytes | ((uint64_t)n << 32);
    for (uint32_t k = 0; k < n; k++)
        dst[16 + k] = (uint8_t)args[k].tag;
    uint64_t *wd = (uint64_t *)(dst + 16 + ((n + 7u) & ~7u));
    uint8_t *tl = (uint8_t *)(wd + n);
    for (uint32_t k = 0; k < n; k++) {
        wd[k] = words[k];
        if (args[k].tag == 's' || args[k].tag == 'b')
            memcpy(tl + (words[k] & 0xffff), args[k].bytes.data(), args[k].bytes.size());
    }
    return bytes;
}

/* one synchronous single-lane call of opcode op */
static int64_t call1(Ring &R, uint32_t op, const std::vector<Arg> &args)
{
    const uint64_t t = R.ticket.fetch_add(1);
    gf_slot_hdr *h = R.hdr(t);
    while (acq(&h->seq) != t)
        std::this_thread::yield();
    put_args((uint8_t *)h + GF_SLOT_PAYLOAD_OFF, args);
    h->opcode = op;
    h->nlanes = 1;
    h->flags = 0;
    h->fmt_len = 0;
    h->fmt_key = 0;
    rel(&h->seq, t + 1);
    while (acq(&h->seq) != t + 2)
        std::this_thread::yield();
    const int64_t r = *(int64_t *)((uint8_t *)h + GF_SLOT_RET_OFF);
    rel(&h->seq, t + R.nslots);
    return r;
}

static const char *FMT = "p %d s %d\n";
static const uint64_t FMT_KEY = 0x1000;

/* returns 0 ok, GF_ERING, GF_ETIMEDOUT; rets[] receive the lane returns */
static int call(Ring &R, int producer, const std::vector<int> &seqs, std::vector<int64_t> &rets, bool ship_fmt,
                double timeout_s, int hold_ms = 0, bool die = false)
{
    const uint64_t t = R.ticket.fetch_add(1);
    gf_slot_hdr *h = R.hdr(t);
    auto t0 = clk::now();
    while (acq(&h->seq) != t) {
        if (std::chrono::duration<double>(clk::now() - t0).count() > timeout_s)
            return GF_ERING;
        std::this_thread::yield();
    }
    uint8_t *pay = (uint8_t *)h + GF_SLOT_PAYLOAD_OFF;
    uint32_t fb = 0;
    if (ship_fmt) {
        memcpy(pay, FMT, strlen(FMT) + 1);
        fb = (uint32_t)((strlen(FMT) + 1 + 7) & ~7u);
    }
    uint32_t off = fb;
    for (size_t l = 0; l < seqs.size(); l++)
        off += put_rec(pay + off, (uint32_t)l, producer, seqs[l]);
    h->opcode = GF_OP_PRINTF;
    h->nlanes = (uint32_t)seqs.size();
    h->flags = ship_fmt ? GF_SF_FMT_INLINE : 0;
    h->fmt_len = ship_fmt ? (uint32_t)strlen(FMT) + 1 : 0;
    h->fmt_key = FMT_KEY;
    if (die)
        return 0;                                  /* claimed, never published */
    if (hold_ms)
        std::this_thread::sleep_for(std::chrono::milliseconds(hold_ms));
    rel(&h->seq, t + 1);
    t0 = clk::now();
    while (acq(&h->seq) != t + 2) {
        if (std::chrono::duration<double>(clk::now() - t0).count() > timeout_s)
            return GF_ETIMEDOUT;
        std::this_thread::yield();
    }
    rets.assign(seqs.size(), 0);
    int64_t *ret = (int64_t *)((uint8_t *)h + GF_SLOT_RET_OFF);
    for (size_t l = 0; l < seqs.size(); l++)
        rets[l] = ret[l];
    rel(&h->seq, t + R.nslots);
    return 0;
}

struct ServerRun {
    gfh::Server srv;
    std::vector<std::thread> th;
    std::atomic<bool> stop{false}, pause{false}, no_idle{false};
    void start(Ring &R, int n)
    {
        R.seg.reset((uint32_t)n);
        R.seg.active = true;
        for (int k = 0; k < n; k++)
            th.emplace_back([this, &R, k, n] {
                while (!stop) {
                    if (pause) {
                        std::this_thread::sleep_for(std::chrono::milliseconds(1));
                        continue;
                    }
                    if (!srv.poll(R.seg, (uint32_t)k, (uint32_t)n)) {
                        if (!no_idle)
                            srv.idle();    /* as the runtime's server threads do */
                        std::this_thread::yield();
                    }
                }
            });
    }
    void join()
    {
        stop = true;
        for (auto &t : th)
            t.join();
        srv.close_all();
        srv.set_stdout(nullptr);   /* the caller closes its stream next: the server keeps no pointer to it */
    }
};

static int fail(const char *m)
{
    printf("FAIL %s\n", m);
    return 1;
}

/* parse the output: every line "p P s S" once, and S increasing per P */
static int check_output(const char *path, int producers, int calls, const std::vector<int> &skip = {})
{
    FILE *f = fopen(path, "r");
    if (!f)
        return fail("no output");
    std::map<int, int> last;
    std::map<int, int> count;
    int p, s;
    while (fscanf(f, "p %d s %d\n", &p, &s) == 2) {
        if (last.count(p) && s <= last[p]) {
            fclose(f);
            return fail("per-producer order");
        }
        last[p] = s;
        count[p]++;
    }
    fclose(f);
    for (int q = 0; q < producers; q++) {
        if (std::find(skip.begin(), skip.end(), q) != skip.end())
            continue;
        if (count[q] != calls) {
            printf("producer %d: %d lines, want %d\n", q, count[q], calls);
            return fail("line count");
        }
    }
    return 0;
}

int main(int argc, char **argv)
{
    if (argc < 3)
        return 2;
    const std::string sc = argv[1];
    FILE *out = fopen(argv[2], "w");
    int nthreads = sc == "threads" || sc == "closerace" ? 4 : 1;
    Ring R(sc == "basic" || sc == "dead" ? 8 : 64, 4096);
    ServerRun S;
    S.srv.set_stdout(out);
    S.start(R, nthreads);
    int rc = 0;
    std::atomic<int> errors{0};

    if (sc == "basic" || sc == "threads" || sc == "fmtcache") {
        const int P = 16, C = sc == "fmtcache" ? 50 : 2000;
        std::atomic<int> shipped{0};
        std::vector<std::thread> ps;
        for (int p = 0; p < P; p++)
            ps.emplace_back([&, p] {
                std::vector<int64_t> r;
                for (int s = 0; s < C; s++) {
                    const bool ship = sc != "fmtcache" || (p == 0 && s == 0);
                    if (sc == "fmtcache" && !(p == 0 && s == 0))
                        while (shipped.load() == 0)
                            std::this_thread::yield();
                    int e = call(R, p, {s}, r, ship, 20.0);
                    if (e || r[0] != (int64_t)strlen("p  s \n") + (int64_t)std::to_string(p).size() +
                                          (int64_t)std::to_string(s).size())
                        errors++;
                    if (p == 0 && s == 0)
                        shipped = 1;
                }
            });
        for (auto &t : ps)
            t.join();
        S.join();
        fclose(out);
        if (errors)
            return fail("call errors");
        rc = check_output(argv[2], P, C);
    } else if (sc == "aggregate") {
        const int P = 8, C = 200;
        std::vector<std::thread> ps;
        for (int p = 0; p < P; p++)
            ps.emplace_back([&, p] {
                std::vector<int64_t> r;
                int s = 0;
                for (int k = 0; s < C; k++) {
                    const int lanes = std::min(C - s, 1 + (k * 7 + p) % 32);
                    std::vector<int> seqs;
                    for (int l = 0; l < lanes; l++)
                        seqs.push_back(s + l);
                    if (call(R, p, seqs, r, true, 20.0))
                        errors++;
                    for (int l = 0; l < lanes; l++)
                        if (r[l] <= 0)
                            errors++;
                    s += lanes;
                }
            });
        for (auto &t : ps)
            t.join();
        S.join();
        fclose(out);
        if (errors)
            return fail("call errors");
        rc = check_output(argv[2], P, C);
    } else if (sc == "ooo") {
        std::vector<int64_t> r0;
        std::atomic<bool> slow_published{false};
        std::thread slow([&] {
            /* claims ticket 0 and holds it unpublished for 2 s */
            if (call(R, 99, {0}, r0, true, 20.0, 2000))
                errors++;
            slow_published = true;
        });
        while (R.ticket.load() == 0)
            std::this_thread::yield();
        std::vector<int64_t> r;
        for (int s = 0; s < 60; s++)          /* fewer than the 64 slots: no lap onto the held slot */
            if (call(R, 1, {s}, r, true, 20.0))
                errors++;
        const bool overtook = !slow_published.load();
        slow.join();
        S.join();
        fclose(out);
        if (errors)
            return fail("call errors");
        if (!overtook)
            return fail("later slots waited behind an unpublished one");
        rc = check_output(argv[2], 0, 0);
    } else if (sc == "dead") {
        std::vector<int64_t> r;
        call(R, 7, {0}, r, true, 1.0, 0, /*die=*/true);   /* slot 0 is claimed forever */
        int ok = 0, ering = 0;
        auto t0 = clk::now();
        for (int s = 0; s < 40; s++) {
            int e = call(R, 1, {s}, r, true, 0.2);
            if (e == 0)
                ok++;
            else if (e == GF_ERING)
                ering++;
            else
                errors++;
        }
        const double dt = std::chrono::duration<double>(clk::now() - t0).count();
        S.join();
        fclose(out);
        if (errors)
            return fail("unexpected error kind");
        if (ok < 30 || ering < 1)
            return fail("expected most calls served and the dead slot's laps to time out");
        if (dt > 10.0)
            return fail("waits not bounded");
    } else if (sc == "stall") {
        std::vector<int64_t> r;
        if (call(R, 1, {0}, r, true, 5.0))
            return fail("first call");
        S.pause = true;
        int e = call(R, 1, {1}, r, true, 0.1);
        if (e != GF_ETIMEDOUT)
            return fail("no timeout while the server stalls");
        S.pause = false;
        /* the stalled slot is served late; later calls succeed */
        std::this_thread::sleep_for(std::chrono::milliseconds(50));
        for (int s = 2; s < 10; s++)
            if (call(R, 1, {s}, r, true, 5.0))
                return fail("no recovery");
        S.join();
        fclose(out);
    } else if (sc == "bulkfile") {
        /* two large fwrites from the bulk arena (the copy pool filling a shared
         * mapping for regular files, plain fwrite for append mode) between
         * small inline ones */
        const uint64_t len = (40ull << 20) + 3;
        std::vector<uint8_t> arena(len);
        for (uint64_t k = 0; k < len; k++)
            arena[k] = (uint8_t)((k * 2654435761ull) >> 13);
        R.seg.bulk = arena.data();
        R.seg.bulk_bytes = len;
        const std::string path = std::string(argv[2]) + ".bin";
        for (const char *mode : {"wb", "w+b", "ab"}) {
            if (!strcmp(mode, "ab")) {
                FILE *pre = fopen(path.c_str(), "wb");
                fwrite("PRE", 1, 3, pre);
                fclose(pre);
            }
            const int64_t fh = call1(R, GF_OP_FOPEN, {{'s', 0, path + '\0'}, {'s', 0, std::string(mode) + '\0'}});
            if (!fh)
                return fail("fopen");
            if (call1(R, GF_OP_FWRITE, {{'L', 1, ""}, {'L', 4, ""}, {'L', (uint64_t)fh, ""}, {'b', 0, "HEAD"}}) != 4)
                return fail("inline fwrite");
            for (int rep = 0; rep < 2; rep++)   /* twice: the copy pool's second job, the position after the first */
                if (call1(R, GF_OP_FWRITE, {{'L', 1, ""}, {'L', len, ""}, {'L', (uint64_t)fh, ""}, {'A', 0, ""},
                                            {'L', len, ""}}) != (int64_t)len)
                    return fail("arena fwrite");
            if (call1(R, GF_OP_FWRITE, {{'L', 1, ""}, {'L', 4, ""}, {'L', (uint64_t)fh, ""}, {'b', 0, "TAIL"}}) != 4)
                return fail("inline fwrite after");
            if (call1(R, GF_OP_FCLOSE, {{'L', (uint64_t)fh, ""}}) != 0)
                return fail("fclose");
            FILE *in = fopen(path.c_str(), "rb");
            std::vector<uint8_t> got(2 * len + 64);
            const size_t k = fread(got.data(), 1, got.size(), in);
            fclose(in);
            const size_t pre = !strcmp(mode, "ab") ? 3 : 0;
            if (k != pre + 4 + 2 * len + 4 || memcmp(got.data() + pre, "HEAD", 4) ||
                memcmp(got.data() + pre + 4, arena.data(), len) ||
                memcmp(got.data() + pre + 4 + len, arena.data(), len) ||
                memcmp(got.data() + pre + 4 + 2 * len, "TAIL", 4))
                return fail(mode);
        }
        remove(path.c_str());
        S.join();
        fclose(out);
    } else if (sc == "closerace") {
        /* a file closed while other producers keep writing to it and
         * flushing it through other server threads: every call returns (a
         * write after the close fails), nothing crashes, and the file holds
         * whole records only */
        const std::string path = std::string(argv[2]) + ".race";
        for (int round = 0; round < 20; round++) {
            const int64_t fh = call1(R, GF_OP_FOPEN, {{'s', 0, path + '\0'}, {'s', 0, std::string("wb") + '\0'}});
            if (!fh)
                return fail("fopen");
            std::atomic<bool> closed{false};
            std::atomic<int> bad{0};
            std::vector<std::thread> ps;
            for (int p = 0; p < 3; p++)
                ps.emplace_back([&, p] {
                    for (int k = 0; k < 200; k++) {
                        const int64_t w = call1(R, GF_OP_FWRITE, {{'L', 1, ""}, {'L', 8, ""}, {'L', (uint64_t)fh, ""},
                                                                  {'b', 0, std::string("rec0123\n")}});
                        if (w != 8 && !closed.load())
                            bad++;
                        if (k % 50 == 0)
                            call1(R, GF_OP_FFLUSH, {{'L', (uint64_t)fh, ""}});
                    }
                    (void)p;
                });
            std::this_thread::sleep_for(std::chrono::microseconds(200 * (round % 5)));
            closed = true;
            const int64_t rc = call1(R, GF_OP_FCLOSE, {{'L', (uint64_t)fh, ""}});
            for (auto &t : ps)
                t.join();
            if (rc != 0 || bad)
                return fail("close race");
            if (call1(R, GF_OP_FWRITE, {{'L', 1, ""}, {'L', 8, ""}, {'L', (uint64_t)fh, ""},
                                        {'b', 0, std::string("late000\n")}}) != 0)
                return fail("write after close");
            FILE *in = fopen(path.c_str(), "rb");
            std::string got(1 << 16, '\0');
            got.resize(fread(&got[0], 1, got.size(), in));
            fclose(in);
            if (got.size() % 8)
                return fail("torn record");
            for (size_t o = 0; o < got.size(); o += 8)
                if (got.compare(o, 8, "rec0123\n"))
                    return fail("record content");
        }
        remove(path.c_str());
        S.join();
        fclose(out);
    } else if (sc == "retire") {
        S.no_idle = true;
        const uint64_t C = 8ull << 20;
        std::vector<uint8_t> arena(C, 0x5a);
        R.seg.bulk = arena.data();
        R.seg.bulk_bytes = C;
        const std::string base = std::string(argv[2]) + ".r";
        auto maps = [&]() {
            int n = 0;
            FILE *mp = fopen("/proc/self/maps", "r");
            char line[4096];
            while (mp && fgets(line, sizeof line, mp))
                if (strstr(line, base.c_str()))
                    n++;
            if (mp)
                fclose(mp);
            return n;
        };
        for (int k = 0; k < 20; k++) {
            const std::string path = base + std::to_string(k);
            const int64_t fh = call1(R, GF_OP_FOPEN, {{'s', 0, path + '\0'}, {'s', 0, std::string("wb") + '\0'}});
            if (!fh)
                return fail("fopen");
            if (call1(R, GF_OP_FWRITE, {{'L', 1, ""}, {'L', C, ""}, {'L', (uint64_t)fh, ""}, {'A', 0, ""},
                                        {'L', C, ""}, {'L', C, ""}}) != (int64_t)C)
                return fail("fwrite");
            if (call1(R, GF_OP_FCLOSE, {{'L', (uint64_t)fh, ""}}) != 0)
                return fail("fclose");
            if (maps() > 16)
                return fail("more than 16 finished writes still mapped");
        }
        if (maps() != 16)
            return fail("the 16 latest finished writes are not kept mapped");
        /* older than the stale limit, they are released by any thread that
         * calls idle(), here one that served nothing */
        std::this_thread::sleep_for(std::chrono::milliseconds(60));
        for (int k = 20; k < 22; k++) {              /* two fresh ones, which stay */
            const std::string path = base + std::to_string(k);
            const int64_t fh = call1(R, GF_OP_FOPEN, {{'s', 0, path + '\0'}, {'s', 0, std::string("wb") + '\0'}});
            if (!fh || call1(R, GF_OP_FWRITE, {{'L', 1, ""}, {'L', C, ""}, {'L', (uint64_t)fh, ""}, {'A', 0, ""},
                                               {'L', C, ""}, {'L', C, ""}}) != (int64_t)C ||
                call1(R, GF_OP_FCLOSE, {{'L', (uint64_t)fh, ""}}) != 0)
                return fail("fresh write");
        }
        S.srv.idle();
        if (maps() > 2)
            return fail("stale mappings not released by an idle thread");
        S.join();                                   /* close_all releases the rest */
        if (maps() != 0)
            return fail("mappings left after close_all");
        for (int k = 0; k < 22; k++) {
            const std::string path = base + std::to_string(k);
            FILE *in = fopen(path.c_str(), "rb");
            std::vector<uint8_t> got(C + 1);
            const size_t g = in ? fread(got.data(), 1, got.size(), in) : 0;
            if (in)
                fclose(in);
            remove(path.c_str());
            if (g != C || memcmp(got.data(), arena.data(), C))
                return fail("file content");
        }
        fclose(out);
    } else if (sc == "bulkchunks") {
        /* large writes sent in chunks that name the bytes still to come: the
         * file is mapped once per write; a write cut short (another call on
         * the stream, or fclose, before its last chunk) leaves no unwritten
         * tail in the file */
        const uint64_t C = (9ull << 20) + 24;
        std::vector<uint8_t> arena(C);
        R.seg.bulk = arena.data();
        R.seg.bulk_bytes = C;
        auto fill = [&](int tag) {
            for (uint64_t k = 0; k < C; k++)
                arena[k] = (uint8_t)(((k + 977 * (uint64_t)tag) * 2654435761ull) >> 13);
        };
        auto chunk = [&](int64_t fh, uint64_t rest) {
            return call1(R, GF_OP_FWRITE, {{'L', 1, ""}, {'L', C, ""}, {'L', (uint64_t)fh, ""}, {'A', 0, ""},
                                           {'L', C, ""}, {'L', rest, ""}}) == (int64_t)C;
        };
        const std::string path = std::string(argv[2]) + ".bin";
        for (const char *mode : {"wb", "w+b", "ab"}) {
            std::string want;
            if (!strcmp(mode, "ab")) {
                FILE *pre = fopen(path.c_str(), "wb");
                fwrite("PRE", 1, 3, pre);
                fclose(pre);
                want = "PRE";
            }
            const int64_t fh = call1(R, GF_OP_FOPEN, {{'s', 0, path + '\0'}, {'s', 0, std::string(mode) + '\0'}});
            if (!fh)
                return fail("fopen");
            auto inl = [&](const char *t) {
                want += t;
                return call1(R, GF_OP_FWRITE, {{'L', 1, ""}, {'L', 4, ""}, {'L', (uint64_t)fh, ""},
                                               {'b', 0, std::string(t, 4)}}) == 4;
            };
            if (!inl("HEAD"))
                return fail("inline fwrite");
            for (int c = 0; c < 3; c++) {               /* a whole write in three chunks */
                fill(c);
                want.append((const char *)arena.data(), C);
                if (!chunk(fh, (3 - c) * C))
                    return fail("chunk");
            }
            for (int c = 0; c < 2; c++) {               /* a write of three chunks cut after two */
                fill(10 + c);
                want.append((const char *)arena.data(), C);
                if (!chunk(fh, (3 - c) * C))
                    return fail("chunk of the cut write");
            }
            if (!inl("MID!") || !inl("TAIL"))
                return fail("inline fwrite after");
            fill(20);                                   /* cut again, then closed */
            want.append((const char *)arena.data(), C);
            if (!chunk(fh, 2 * C))
                return fail("chunk before fclose");
            if (call1(R, GF_OP_FCLOSE, {{'L', (uint64_t)fh, ""}}) != 0)
                return fail("fclose");
            FILE *in = fopen(path.c_str(), "rb");
            std::string got(want.size() + 64, '\0');
            const size_t k = fread(&got[0], 1, got.size(), in);
            fclose(in);
            got.resize(k);
            if (got != want) {
                printf("%s: %zu bytes, want %zu\n", mode, got.size(), want.size());
                return fail(mode);
            }
        }
        /* every mapping of the file is gone: the finished writes' ones are
         * released after their replies, by the serving thread once idle */
        bool mapped = true;
        for (int tries = 0; tries < 200 && mapped; tries++) {
            mapped = false;
            FILE *mp = fopen("/proc/self/maps", "r");
            char line[4096];
            while (mp && fgets(line, sizeof line, mp))
                if (strstr(line, path.c_str()))
                    mapped = true;
            if (mp)
                fclose(mp);
            if (mapped)
                std::this_thread::sleep_for(std::chrono::milliseconds(10));
        }
        if (mapped)
            return fail("the written file is still mapped");
        remove(path.c_str());
        S.join();
        fclose(out);
    } else {
        return fail("unknown scenario");
    }
    if (rc == 0)
        printf("OK %s\n", sc.c_str());
    return rc;
}
