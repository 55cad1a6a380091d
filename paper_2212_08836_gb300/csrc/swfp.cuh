// Correctly rounded binary64 multiplication in 64-bit integer arithmetic
// (IEEE 754-2008, round to nearest, ties to even), written out from the
// definition: the exact 106-bit significand product, one normalisation step,
// then rounding on the guard bits with a sticky bit.  The result is
// bit-identical to the hardware multiply; operands or results outside the
// normal range (subnormals, infinities, NaN, overflow) take the hardware
// instruction; a zero operand gives the signed zero.
//
// Why: a GB300 SM retires 2 binary64 operations per cycle but 64 integer
// multiply-adds, and the FP64-form mover is bound by its FP64 pipe with the
// integer pipes mostly idle.  A product that does not feed an addition (an FMA
// keeps its add on the FP64 pipe) moves to the integer pipes this way.
#pragma once

namespace pic {

// the hardware multiply for the rare operands outside the fast range, out of
// line: an inlined fallback would be if-converted into a predicated FP64
// instruction that every call issues
static __device__ __noinline__ double sw_dmul_slow(double x, double y) { return __dmul_rn(x, y); }

__device__ __forceinline__ double sw_dmul(double x, double y) {
  const unsigned long long a = (unsigned long long)__double_as_longlong(x);
  const unsigned long long b = (unsigned long long)__double_as_longlong(y);
  const int ea = (int)((a >> 52) & 0x7ff), eb = (int)((b >> 52) & 0x7ff);
  int e = ea + eb - 1023;  // biased exponent of the product for a significand in [1, 2)
  if ((unsigned)(ea - 1) > 2045u || (unsigned)(eb - 1) > 2045u || (unsigned)(e - 1) > 2044u) {
    // a zero operand with a finite other one gives a zero of the product's sign
    if (((a << 1) == 0 && eb != 0x7ff) || ((b << 1) == 0 && ea != 0x7ff))
      return __longlong_as_double((long long)((a ^ b) & 0x8000000000000000ull));
    return sw_dmul_slow(x, y);
  }
  const unsigned long long M = 0x000FFFFFFFFFFFFFull, H = 0x0010000000000000ull;
  const unsigned long long ma = ((a & M) | H) << 11, mb = ((b & M) | H) << 11;
  // significand product = ph 2^64 + pl with ph in [2^62, 2^64)
  const unsigned long long ph = __umul64hi(ma, mb);
  const unsigned long long pl = ma * mb;
  const int top = (int)(ph >> 63);  // 1: the product is in [2, 4)
  const int s = 10 + top;
  unsigned long long m = ph >> s;   // the 53 significant bits
  const unsigned long long rem = ph & ((1ull << s) - 1), half = 1ull << (s - 1);
  e += top;
  m += (rem > half || (rem == half && (pl != 0 || (m & 1)))) ? 1ull : 0ull;
  // the significand's leading bit adds one to the exponent field, and a carry
  // out of the rounded significand one more (up to infinity on overflow)
  const unsigned long long r = ((unsigned long long)(e - 1) << 52) + m;
  return __longlong_as_double((long long)(r | ((a ^ b) & 0x8000000000000000ull)));
}

}  // namespace pic
