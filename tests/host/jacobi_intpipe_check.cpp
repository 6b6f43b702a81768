/* Host build of the Jacobi sweep's arithmetic as the device program composes
 * it: the index split by gf_udiv32, the boundary test on max(i-1, j-1, k-1),
 * the first int_adds neighbour adds by gf_dadd_int and the rest by IEEE adds
 * in the serial order, the division by gf_div6_int and |un - u| by
 * gf_fabs_int.  It prints and writes what the serial program prints and
 * writes, so the two can be compared byte for byte.
 *
 *   jacobi_intpipe_check n sweeps int_adds in.bin out.bin */
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>
#include "gf_intpipe.cuh"

int main(int argc, char **argv)
{
    if (argc != 6)
        return 2;
    const uint32_t nn = (uint32_t)atol(argv[1]);
    const int sweeps = atoi(argv[2]), int_adds = atoi(argv[3]);
    const uint64_t cells = (uint64_t)nn * nn * nn;
    std::vector<double> u(cells), un(cells);
    FILE *f = fopen(argv[4], "rb");
    if (!f || fread(u.data(), 8, cells, f) != cells)
        return 2;
    fclose(f);
    const uint32_t sk = nn * nn;
    const gf_udiv32 dn = gf_udiv32::make(nn);
    for (int s = 1; s <= sweeps; s++) {
        double res = 0.0;
        for (uint32_t c = 0; c < cells; c++) {
            const uint32_t jk = dn.div(c), im1 = c - 1u - jk * nn;
            const uint32_t k = dn.div(jk), jm1 = jk - 1u - k * nn;
            uint32_t m = im1 > jm1 ? im1 : jm1;
            m = m > k - 1u ? m : k - 1u;
            if (m >= nn - 2u) {
                un[c] = 0.0;
                continue;
            }
            const double nb[6] = {u[c - 1], u[c + 1], u[c - nn], u[c + nn], u[c - sk], u[c + sk]};
            double v = nb[0];
            for (int q = 1; q < 6; q++) {
                if (q <= int_adds) {
                    v = gf_dadd_int(v, nb[q]);
                } else {
                    volatile double t = v + nb[q];
                    v = t;
                }
            }
            v = gf_div6_int(v);
            un[c] = v;
            volatile double diff = v - u[c];
            const double d = gf_fabs_int(diff);
            if (d > res)
                res = d;
        }
        printf("%d %.17g\n", s, res);
        u.swap(un);
    }
    f = fopen(argv[5], "wb");
    if (!f || fwrite(u.data(), 8, cells, f) != cells)
        return 3;
    fclose(f);
    return 0;
}
