/* The host printf landing pad, whole formats at a time: each format is cut
 * into literal runs and conversions once, and a record's output must equal
 * one snprintf call of the same format with the same arguments.  Covers
 * literal-only formats, "%%", flags, widths and precisions (given and '*'),
 * every length modifier, %n, strings, and formats whose conversions run
 * past the record's arguments or past the end of the format.
 * Prints "plan checked N mismatches M". */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cmath>
#include <random>
#include <string>
#include <vector>

#include "gf.h"
#include "host/server.h"

struct Arg {
    char tag;
    uint64_t word;
    std::string str;   /* tag 's': the bytes with their NUL */
};

/* a lane record in the device layout: header, tags, words, string tail */
static std::vector<uint8_t> record(const std::vector<Arg> &args)
{
    const uint32_t n = (uint32_t)args.size();
    uint32_t tail = 0;
    std::vector<uint64_t> words(n);
    for (uint32_t k = 0; k < n; k++) {
        words[k] = args[k].word;
        if (args[k].tag == 's') {
            words[k] = ((uint64_t)args[k].str.size() << 32) | tail;
            tail += ((uint32_t)args[k].str.size() + 7u) & ~7u;
        }
    }
    const uint32_t bytes = 16 + ((n + 7u) & ~7u) + 8 * n + tail;
    std::vector<uint8_t> r(bytes, 0);
    uint64_t *w = (uint64_t *)r.data();
    w[0] = (uint64_t)bytes | ((uint64_t)n << 32);
    for (uint32_t k = 0; k < n; k++)
        r[16 + k] = (uint8_t)args[k].tag;
    uint64_t *wd = (uint64_t *)(r.data() + 16 + ((n + 7u) & ~7u));
    uint8_t *tl = (uint8_t *)(wd + n);
    for (uint32_t k = 0; k < n; k++) {
        wd[k] = words[k];
        if (args[k].tag == 's')
            memcpy(tl + (words[k] & 0xffff), args[k].str.data(), args[k].str.size());
    }
    return r;
}

static uint64_t dbits(double d)
{
    uint64_t b;
    memcpy(&b, &d, 8);
    return b;
}

int main(int argc, char **argv)
{
    if (argc < 2)
        return 2;
    const char *path = argv[1];
    std::mt19937_64 rng(11);
    int checked = 0, bad = 0;
    auto check = [&](const char *fmt, const std::vector<Arg> &args, const std::string &want) {
        FILE *f = fopen(path, "w+");
        gfh::Server srv;
        srv.set_stdout(f);
        std::vector<Arg> all = {{'L', GF_STDOUT_H, ""}};
        all.insert(all.end(), args.begin(), args.end());
        const std::vector<uint8_t> rec = record(all);
        const int64_t n = srv.call(GF_OP_PRINTF, fmt, rec.data());
        srv.set_stdout(nullptr);          /* f is closed below, before the server goes */
        fflush(f);
        rewind(f);
        std::string got;
        char buf[4096];
        size_t k;
        while ((k = fread(buf, 1, sizeof buf, f)) > 0)
            got.append(buf, k);
        fclose(f);
        checked++;
        if (got != want || n != (int64_t)want.size()) {
            bad++;
            if (bad <= 20)
                printf("MISMATCH fmt \"%s\": got \"%s\" (%lld) want \"%s\"\n", fmt, got.c_str(), (long long)n,
                       want.c_str());
        }
    };
    char w[8192];
    /* literal text, %% and conversions at the edges of the format */
    check("", {}, "");
    check("plain text\n", {}, "plain text\n");
    check("100%% done %%\n", {}, "100% done %\n");
    snprintf(w, sizeof w, "%d%%%d", 3, 4);
    check("%d%%%d", {{'i', 3, ""}, {'i', 4, ""}}, w);
    snprintf(w, sizeof w, "%d", -7);
    check("%d", {{'i', (uint64_t)-7, ""}}, w);
    check("tail %d and %d\n", {{'i', 5, ""}}, "tail 5 and ");             /* arguments run out */
    check("cut %", {}, "cut ");                                            /* conversion cut off by the end */
    check("cut %-08.", {{'i', 1, ""}}, "cut ");
    snprintf(w, sizeof w, "%s|%5s|%-5s|%.2s", "ab", "cd", "ef", "ghij");
    check("%s|%5s|%-5s|%.2s", {{'s', 0, "ab"}, {'s', 0, "cd"}, {'s', 0, "ef"}, {'s', 0, "ghij"}}, w);
    /* %n writes nothing back and takes its argument */
    snprintf(w, sizeof w, "a%db", 9);
    check("a%n%db", {{'p', 0, ""}, {'i', 9, ""}}, w);
    /* '*' width and precision */
    snprintf(w, sizeof w, "[%*d|%.*f|%*.*e]", 6, 42, 3, 2.5, 12, 2, 1234.5);
    check("[%*d|%.*f|%*.*e]", {{'i', 6, ""}, {'i', 42, ""}, {'i', 3, ""}, {'d', dbits(2.5), ""}, {'i', 12, ""},
                               {'i', 2, ""}, {'d', dbits(1234.5), ""}}, w);
    /* every conversion with flags, widths and precisions, random values */
    const char *ifmts[] = {"%d", "%5d", "%-5d|", "%05d", "%+d", "% d", "%'d", "%hd", "%hhd", "%ld", "%lld", "%zd",
                           "%jd", "%td", "%qd", "%u", "%lu", "%llu", "%hu", "%hhu", "%x", "%#x", "%08lx", "%X",
                           "%#llo", "%o", "%c", "%.3d", "%10.4d", "%i"};
    const char *ffmts[] = {"%f", "%.0f", "%.3f", "%10.2f", "%-10.2f|", "%+.1f", "%e", "%.0e", "%.6e", "%E",
                           "%.17e", "%g", "%.3g", "%.17g", "%#g", "%G", "%a", "%A", "%.2a", "%lf", "%le", "%lg",
                           "%Lf", "%Le", "%.25g", "%015.3f", "% .4e"};
    std::uniform_int_distribution<int> ex(-330, 310);
    for (int it = 0; it < 400; it++) {
        for (const char *f : ifmts) {
            const uint64_t v = rng();
            const std::string fm = std::string("<") + f + ">\n";
            /* the C type the conversion and its length modifier name */
            const char *l = f + 1 + strspn(f + 1, "-+ #0'123456789.");
            const char conv = f[strlen(f) - (f[strlen(f) - 1] == '|' ? 2 : 1)];
            const bool sgn = conv == 'd' || conv == 'i';
            std::string g = fm;
            if (l[0] == 'q')
                g.replace(g.find('q'), 1, "ll");
            int wn;
            if (conv == 'c')
                wn = snprintf(w, sizeof w, g.c_str(), (int)v);
            else if ((l[0] == 'l' && l[1] == 'l') || l[0] == 'q')
                wn = sgn ? snprintf(w, sizeof w, g.c_str(), (long long)v) : snprintf(w, sizeof w, g.c_str(), (unsigned long long)v);
            else if (l[0] == 'l' || l[0] == 'j' || l[0] == 'z' || l[0] == 't')
                wn = sgn ? snprintf(w, sizeof w, g.c_str(), (long)v) : snprintf(w, sizeof w, g.c_str(), (unsigned long)v);
            else if (l[0] == 'h' && l[1] == 'h')
                wn = sgn ? snprintf(w, sizeof w, g.c_str(), (int)(signed char)v)
                    : snprintf(w, sizeof w, g.c_str(), (unsigned)(unsigned char)v);
            else if (l[0] == 'h')
                wn = sgn ? snprintf(w, sizeof w, g.c_str(), (int)(short)v)
                    : snprintf(w, sizeof w, g.c_str(), (unsigned)(unsigned short)v);
            else
                wn = sgn ? snprintf(w, sizeof w, g.c_str(), (int)v) : snprintf(w, sizeof w, g.c_str(), (unsigned)v);
            check(fm.c_str(), {{'l', v, ""}}, std::string(w, (size_t)wn));  /* %c may write a NUL */
        }
        for (const char *f : ffmts) {
            const double d = std::ldexp((double)(rng() >> 11) / 9007199254740992.0, ex(rng)) *
                             ((rng() & 1) ? -1.0 : 1.0);
            std::string fm = std::string("x=") + f + ";\n";
            if (strchr(f, 'L'))
                snprintf(w, sizeof w, fm.c_str(), (long double)d);
            else
                snprintf(w, sizeof w, fm.c_str(), d);
            check(fm.c_str(), {{'d', dbits(d), ""}}, w);
        }
    }
    printf("plan checked %d mismatches %d\n", checked, bad);
    return bad ? 1 : 0;
}
