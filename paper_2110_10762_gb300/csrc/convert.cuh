// FP32 <-> FP64 conversions on the integer pipe.
#pragma once

#include <cuda_runtime.h>

namespace pr {

// On this GPU a float <-> double conversion instruction issues on the FP64
// pipe, at the DFMA rate (2 per SM and clock), so a pass that converts a few
// values per point is bound by conversions.  These two do the same conversions
// from the IEEE 754 binary32/binary64 encodings with integer operations; their
// results equal the hardware conversions bit for bit (round to nearest even
// for the narrowing; the widening is exact), NaN payloads aside.

// binary32 -> binary64: exponent rebiased by 1023 - 127 = 896, the 23-bit
// significand moved to the top of the 52-bit one; subnormals normalised.
__device__ __forceinline__ double widen_f32(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned s = b & 0x80000000u;
  const unsigned e = (b >> 23) & 0xffu;
  unsigned m = b & 0x7fffffu;
  unsigned E;
  if (e == 0xffu) {
    E = 0x7ffu;
  } else if (e != 0u) {
    E = e + 896u;
  } else if (m == 0u) {
    E = 0u;
  } else {
    const unsigned sh = (unsigned)__clz((int)m) - 8u;  // moves the leading one to bit 23
    m = (m << sh) & 0x7fffffu;
    E = 897u - sh;
  }
  return __hiloint2double((int)(s | (E << 20) | (m >> 3)), (int)(m << 29));
}

// binary64 -> binary32, round to nearest, ties to even: keep the top 23 of the
// 52 significand bits and round on the 29 dropped ones (a carry into the
// exponent field is the correct result, up to infinity); results below the
// binary32 normal range are formed as subnormals from the 53-bit significand.
__device__ __forceinline__ float narrow_f64_rn(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned s = (unsigned)(b >> 32) & 0x80000000u;
  const int E = (int)((b >> 52) & 0x7ffu);
  const unsigned long long M = b & 0xfffffffffffffull;
  if (E == 0x7ff) return __uint_as_float(s | 0x7f800000u | (M ? 0x400000u : 0u));
  const int e = E - 896;
  if (e >= 255) return __uint_as_float(s | 0x7f800000u);
  if (e >= 1) {
    unsigned v = ((unsigned)e << 23) | (unsigned)(M >> 29);
    const unsigned rem = (unsigned)(M & 0x1fffffffull);
    if (rem > 0x10000000u || (rem == 0x10000000u && (v & 1u))) ++v;
    return __uint_as_float(s | v);
  }
  // subnormal or zero: |d| = (2^52 + M) 2^(E - 1075) = q 2^-149 with q = (2^52 + M) 2^(E - 926)
  const int sh = 926 - E;  // >= 30
  if (E == 0 || sh > 54) return __uint_as_float(s);
  const unsigned long long full = (1ull << 52) | M;
  unsigned q = (unsigned)(full >> sh);
  const unsigned long long rem = full & ((1ull << sh) - 1ull);
  const unsigned long long half = 1ull << (sh - 1);
  if (rem > half || (rem == half && (q & 1u))) ++q;
  return __uint_as_float(s | q);
}

}  // namespace pr
