/* Host build of gf_strtod_fast compared with the C library's strtod on every
 * line of the input file: where the fast path answers, the value bits and the
 * end pointer must be the library's.  Prints "handled H of N, mismatches M". */
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include "gf_strtod_fast.h"

int main(int argc, char **argv)
{
    if (argc < 2)
        return 2;
    FILE *f = fopen(argv[1], "r");
    if (!f)
        return 2;
    char line[512];
    long n = 0, handled = 0, bad = 0;
    while (fgets(line, sizeof line, f)) {
        line[strcspn(line, "\n")] = 0;
        n++;
        double got;
        const char *end;
        if (!gf_strtod_fast(line, &got, &end))
            continue;
        handled++;
        char *lend;
        const double want = strtod(line, &lend);
        if (memcmp(&got, &want, 8) != 0 || end != lend) {
            if (bad < 10)
                printf("mismatch \"%s\": %.17g (end %ld) vs %.17g (end %ld)\n", line, got, (long)(end - line), want,
                       (long)(lend - line));
            bad++;
        }
    }
    fclose(f);
    printf("handled %ld of %ld, mismatches %ld\n", handled, n, bad);
    return 0;
}
