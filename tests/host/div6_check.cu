/* Host-side check of gf_div6_int (the integer-pipe division by 6) against
 * the CPU's IEEE division: random bit patterns, every binade, mantissas
 * around the k-switch (3 * 2^51) and the binade ends, and special values. */
#include <cstdio>
#include <cstring>
#include <cstdint>
#include <random>
#include "gf_intpipe.cuh"
int main() {
  std::mt19937_64 g(1); long bad = 0, n = 0;
  auto chk = [&](double x){ double a = x / 6.0, b = gf_div6_int(x); uint64_t ua, ub; memcpy(&ua,&a,8); memcpy(&ub,&b,8);
     n++; if (ua != ub && !(a != a && b != b)) { if (bad < 10) printf("x=%a want %a got %a\n", x, a, b); bad++; } };
  for (long i = 0; i < 20000000; i++) { uint64_t u = g(); double x; memcpy(&x, &u, 8); chk(x); }
  for (int e = -1074; e < 1024; e++) for (int j = 0; j < 200; j++) { double m = 1.0 + (double)(g() >> 11) * 0x1p-53; chk(ldexp(m, e)); chk(-ldexp(m, e)); }
  // mantissa boundaries around 3*2^51, 2^52, 2^53-1 for several exponents
  for (int e = -1030; e < 1030; e += 7) for (long d = -3000; d <= 3000; d++) {
     for (uint64_t base : {3ull << 51, 1ull << 52, (1ull << 53) - 1}) { uint64_t m = base + d; if (m < (1ull<<52) || m >= (1ull<<53)) continue; chk(ldexp((double)m, e - 52)); } }
  for (double x : {0.0, -0.0, 6.0, 3.0, 1.0, 0x1p-1022, 0x1p-1020, 0x1.8p-1020, 0x1p-1021, 0x1.fffffffffffffp1023, 1e308, 5e-324}) chk(x);
  printf("checked %ld, mismatches %ld\n", n, bad);
}
