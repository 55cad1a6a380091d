// Host build of the library's integer-pipe binary64 multiply (csrc/swfp.cuh),
// compared bit for bit with the host's IEEE binary64 multiply (round to
// nearest even) on random operands over the whole exponent range, products
// with few significand bits (exact and tie cases), near-overflow and
// subnormal results, zeros, infinities and NaN.  Prints the mismatch count.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>
#define __device__
#define __forceinline__ inline
#define __noinline__
static inline long long __double_as_longlong(double x) { long long r; memcpy(&r, &x, 8); return r; }
static inline double __longlong_as_double(long long x) { double r; memcpy(&r, &x, 8); return r; }
static inline unsigned long long __umul64hi(unsigned long long a, unsigned long long b) {
  return (unsigned long long)(((unsigned __int128)a * b) >> 64);
}
static inline double __dmul_rn(double x, double y) { volatile double r = x * y; return r; }
#include "../paper_2212_08836_gb300/csrc/swfp.cuh"

static uint64_t bits(double x) { uint64_t r; memcpy(&r, &x, 8); return r; }
static double dbl(uint64_t b) { double r; memcpy(&r, &b, 8); return r; }

int main(int argc, char **argv) {
  long long n = argc > 1 ? atoll(argv[1]) : 4000000;
  std::mt19937_64 g(20240611);
  auto rnd = [&](int emin, int emax) {
    uint64_t m = g() & 0x000FFFFFFFFFFFFFull;
    int k = (int)(g() % 4);
    if (k == 0) m &= 0x000FFF0000000000ull;  // few significand bits: exact and tie products
    if (k == 1) m &= 0x000FFFFFFF000000ull;
    int e = emin + (int)(g() % (uint64_t)(emax - emin + 1));
    return dbl((g() & 0x8000000000000000ull) | ((uint64_t)e << 52) | m);
  };
  long long bad = 0;
  auto check = [&](double x, double y) {
    double p = pic::sw_dmul(x, y), r = x * y;
    if (bits(p) != bits(r) && !(std::isnan(p) && std::isnan(r))) {
      if (bad < 5) printf("mismatch %a * %a: %a vs %a\n", x, y, p, r);
      bad++;
    }
  };
  const double sp[] = {0.0, -0.0, 1.0, -1.5, 4.9e-324, -2.2250738585072009e-308,
                       2.2250738585072014e-308, 1e-310, 1.7976931348623157e308, INFINITY,
                       -INFINITY, NAN, 3.0e-200, 7.0e200};
  for (double x : sp)
    for (double y : sp) check(x, y);
  for (long long t = 0; t < n; ++t) {
    switch (t % 4) {
      case 0: check(rnd(1, 2046), rnd(1, 2046)); break;    // full range incl. overflow / underflow
      case 1: check(rnd(900, 1150), rnd(900, 1150)); break; // the mover's range
      case 2: check(rnd(1, 80), rnd(900, 1000)); break;     // subnormal results
      default: check(rnd(1500, 2046), rnd(1000, 1100)); break;  // near overflow
    }
  }
  printf("cases %lld mismatches %lld\n", n + (long long)(sizeof(sp) / sizeof(sp[0]) * sizeof(sp) / sizeof(sp[0])), bad);
  return bad ? 1 : 0;
}
