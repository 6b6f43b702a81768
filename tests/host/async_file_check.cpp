/* The asynchronously written output file: four threads print numbered
 * lines through the one stream (each fwrite under a shared lock, as the
 * server's threads do), some of them large, with drains in between.  After
 * each drain the file must hold every line printed so far, whole, each
 * thread's lines in order; after close, all of them.  Then drains while
 * another thread keeps printing must each return within a second.
 * Prints "async checked N lines OK" or the first failure. */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "host/server.h"

static int check_file(const char *path, int threads, const std::vector<int> &want, bool exact)
{
    FILE *f = fopen(path, "r");
    if (!f)
        return printf("FAIL cannot read\n"), 1;
    std::vector<int> next(threads, 0);
    char line[70000];
    long lines = 0;
    while (fgets(line, sizeof line, f)) {
        int t, k;
        char pad[8];
        if (sscanf(line, "t%d k%d %7s", &t, &k, pad) < 2 || t < 0 || t >= threads || line[strlen(line) - 1] != '\n') {
            fclose(f);
            return printf("FAIL torn line %.40s\n", line), 1;
        }
        if (k != next[t]) {
            fclose(f);
            return printf("FAIL thread %d line %d, want %d\n", t, k, next[t]), 1;
        }
        next[t]++;
        lines++;
    }
    fclose(f);
    for (int t = 0; t < threads; t++)
        if (exact ? next[t] != want[t] : next[t] < want[t])
            return printf("FAIL thread %d: %d lines in the file, %d printed\n", t, next[t], want[t]), 1;
    return 0;
}

/* after the run under load: threads 0..T-1 whole and in order, plus the
 * markers and the noisy thread's lines, none torn */
static int check_markers_and_counts(const char *path, int threads, const std::vector<int> &want)
{
    FILE *f = fopen(path, "r");
    if (!f)
        return printf("FAIL cannot read\n"), 1;
    std::vector<int> next(threads + 1, 0);
    char line[70000];
    int markers = 0;
    while (fgets(line, sizeof line, f)) {
        if (!strcmp(line, "t0 marker\n")) {
            markers++;
            continue;
        }
        int t, k;
        if (sscanf(line, "t%d k%d", &t, &k) != 2 || t < 0 || t > threads || line[strlen(line) - 1] != '\n') {
            fclose(f);
            return printf("FAIL torn line %.40s\n", line), 1;
        }
        if (k != next[t]) {
            fclose(f);
            return printf("FAIL thread %d line %d, want %d\n", t, k, next[t]), 1;
        }
        next[t]++;
    }
    fclose(f);
    for (int t = 0; t < threads; t++)
        if (next[t] != want[t])
            return printf("FAIL thread %d: %d lines, want %d\n", t, next[t], want[t]), 1;
    if (markers != 20)
        return printf("FAIL %d markers\n", markers), 1;
    return 0;
}

int main(int argc, char **argv)
{
    if (argc < 2)
        return 2;
    const char *path = argv[1];
    gfh::AsyncFile *a = gfh::async_open(path);
    if (!a)
        return printf("FAIL open\n"), 1;
    FILE *f = gfh::async_stream(a);
    const int T = 4, ROUNDS = 5, PER = 20000;
    std::mutex mu;
    std::vector<int> printed(T, 0);
    for (int r = 0; r < ROUNDS; r++) {
        std::vector<std::thread> th;
        for (int t = 0; t < T; t++)
            th.emplace_back([&, t] {
                std::string big(65000, 'x');
                for (int k = 0; k < PER; k++) {
                    char b[80];
                    const int kk = printed[t] + k;
                    int n = snprintf(b, sizeof b, "t%d k%d %s\n", t, kk, kk % 997 == 0 ? "big" : "ok");
                    std::lock_guard<std::mutex> g(mu);
                    if (kk % 997 == 0) {         /* a long line in several writes */
                        fwrite(b, 1, (size_t)n - 1, f);
                        fputc(' ', f);
                        fwrite(big.data(), 1, big.size(), f);
                        fputc('\n', f);
                    } else {
                        fwrite(b, 1, (size_t)n, f);
                    }
                }
            });
        for (auto &x : th)
            x.join();
        for (int t = 0; t < T; t++)
            printed[t] += PER;
        if (gfh::async_drain(a) != 0)
            return printf("FAIL drain\n"), 1;
        if (check_file(path, T, printed, true))
            return 1;
    }
    /* a drain returns once the bytes queued before it are written, while
     * another thread keeps printing */
    {
        std::atomic<bool> stop{false};
        std::thread noisy([&] {
            int k = 0;
            while (!stop.load()) {
                char b[64];
                const int n = snprintf(b, sizeof b, "t%d k%d ok\n", T, k++);
                std::lock_guard<std::mutex> g(mu);
                fwrite(b, 1, (size_t)n, f);
            }
        });
        for (int r = 0; r < 20; r++) {
            {
                std::lock_guard<std::mutex> g(mu);
                fwrite("t0 marker\n", 1, 10, f);
            }
            const auto t0 = std::chrono::steady_clock::now();
            if (gfh::async_drain(a) != 0)
                return printf("FAIL drain under load\n"), 1;
            const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            if (dt > 1.0)
                return printf("FAIL drain under load took %.3f s\n", dt), 1;
            FILE *in = fopen(path, "r");
            fseek(in, 0, SEEK_END);
            const long sz = ftell(in);
            fclose(in);
            if (sz <= 0)
                return printf("FAIL empty file after drain\n"), 1;
        }
        stop = true;
        noisy.join();
    }
    if (gfh::async_close(a) != 0)
        return printf("FAIL close\n"), 1;
    if (check_markers_and_counts(path, T, printed))
        return 1;
    printf("async checked %d lines OK\n", T * ROUNDS * PER);
    return 0;
}
