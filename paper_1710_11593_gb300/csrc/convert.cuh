// Conversions between double and float with integer operations.
//
// On this GPU every instruction that reads or writes a double -- arithmetic and also the
// F2F conversions double<->float -- issues at the FP64 rate (about 2 per SM per clock,
// against about 128 FP32 and 64 integer operations).  The mixed path moves data between
// the double fields of the interface and its float work arrays; doing that with the
// conversion instructions made those kernels FP64-bound.  These helpers rebuild the IEEE
// bit patterns instead.  Values outside the float normal range fall back to the hardware
// conversion (a rare, data-dependent branch), except that magnitudes below it round to
// signed zero.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ftoep {

// double -> float, round to nearest, ties to even.
__device__ __forceinline__ float d2f_fast(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;  // float biased exponent
  if (e <= 0) return __uint_as_float(sign);                // zero or below the float range
  if (e >= 255) return __double2float_rn(x);               // overflow, inf, nan
  const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);  // top 23 fraction bits
  const unsigned rest = lo & 0x1fffffffu;                  // 29 dropped bits
  unsigned r = ((unsigned)e << 23) | m;
  if (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) r += 1u;  // carry may bump the exponent
  return __uint_as_float(sign | r);
}

// float -> double (exact).
__device__ __forceinline__ double f2d_fast(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xffu;
  const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
  if (e == 0u) {
    if ((b & 0x7fffffu) == 0u) return __longlong_as_double((long long)sign);
    return (double)f;  // denormal
  }
  if (e == 255u) return (double)f;
  const unsigned long long ed = (unsigned long long)(e - 127u + 1023u);
  return __longlong_as_double((long long)(sign | (ed << 52) | ((unsigned long long)(b & 0x7fffffu) << 29)));
}

// double -> float pair hi + lo: hi keeps the top 24 significant bits (truncated), lo the
// next 29 rounded to 24; |x - hi - lo| <= 2^-47 |x|.
__device__ __forceinline__ void d2ff_fast(double x, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned h = (unsigned)(b >> 32), l = (unsigned)b;
  const unsigned sign = h & 0x80000000u;
  const int E = (int)((h >> 20) & 0x7ffu) - 1023;  // unbiased exponent
  const int e = E + 127;
  if (e <= 0) {
    hi = __uint_as_float(sign);
    lo = 0.0f;
    return;
  }
  if (e >= 255) {
    hi = __double2float_rn(x);
    lo = 0.0f;
    return;
  }
  hi = __uint_as_float(sign | ((unsigned)e << 23) | ((h & 0xfffffu) << 3) | (l >> 29));
  const unsigned rem = l & 0x1fffffffu;  // value rem * 2^(E - 52)
  if (rem == 0u) {
    lo = 0.0f;
    return;
  }
  const int pb = 31 - __clz((int)rem);  // leading bit position, 0..28
  const int el = E - 52 + pb + 127;     // biased exponent of lo
  if (el <= 0) {
    lo = 0.0f;
    return;
  }
  unsigned mant, rest = 0u, halfw = 0u;
  if (pb <= 23) {
    mant = (rem << (23 - pb)) & 0x7fffffu;
  } else {
    const int sh = pb - 23;
    mant = (rem >> sh) & 0x7fffffu;
    rest = rem & ((1u << sh) - 1u);
    halfw = 1u << (sh - 1);
  }
  unsigned r = ((unsigned)el << 23) | mant;
  if (rest > halfw || (rest == halfw && halfw != 0u && (mant & 1u))) r += 1u;
  lo = __uint_as_float(sign | r);
}

}  // namespace ftoep
