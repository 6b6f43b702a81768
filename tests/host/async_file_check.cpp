/* The asynchronously written output file: four threads print numbered
 * lines through the one stream (each fwrite under a shared lock, as the
 * server's threads do), some of them large, with drains in between.  After
 * each drain the file must hold every line printed so far, whole, each
 * thread's lines in order; after close, all of them.
 * Prints "async checked N lines OK" or the first failure. */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

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
    if (gfh::async_close(a) != 0)
        return printf("FAIL close\n"), 1;
    if (check_file(path, T, printed, true))
        return 1;
    printf("async checked %d lines OK\n", T * ROUNDS * PER);
    return 0;
}
