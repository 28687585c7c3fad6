// Error-free split of FP64 values into five BF16 slices (Ozaki, Ogita, Oishi
// & Rump, "Error-free transformations of matrix multiplication by using fast
// routines of matrix multiplication and its applications", 2012), with
// balanced base-256 digits.  For a group of values sharing a scale (a row of
// one K chunk), emax is the largest biased FP64 exponent in the group; each
// value is rounded to a 40-bit integer X = rint(|x| 2^(40 - e)) with
// 2^e > max |x|, X is written with five base-256 digits, the last four
// balanced into [-128, 127] (carry upward) and the first in [0, 256], and
// slice p (0-based) is sign(x) d_p 2^(emax - 1023 + 1 - 8 (p + 1)), exact in
// BF16 because |d_p| <= 256.  Slices whose scale leaves the FP32 normal range
// are zero.
#pragma once
#include <cuda_runtime.h>

namespace gpc {

constexpr int kSlices = 5;

// biased FP64 exponent of a value for the group maximum (0 for zero,
// denormal, Inf and NaN, which take no part in the scale)
__device__ __forceinline__ int slice_exponent(unsigned long long bits) {
  const int e = (int)((bits >> 52) & 0x7FF);
  return (e == 0x7FF) ? 0 : e;
}

__device__ __forceinline__ void split_value(unsigned long long bits, int emax, float (&v)[kSlices]) {
  const int e = (int)((bits >> 52) & 0x7FF);
  unsigned long long X = 0;
  if (e != 0 && e != 0x7FF && emax != 0) {
    const unsigned long long mant = (bits & ((1ull << 52) - 1)) | (1ull << 52);
    const int sh = 53 - 8 * kSlices + (emax - e);  // >= 13
    if (sh < 64) X = (mant + (1ull << (sh - 1))) >> sh;
  }
  const bool neg = (bits >> 63) != 0;
  int dig[kSlices];
#pragma unroll
  for (int pp = kSlices - 1; pp >= 1; --pp) {
    int t = (int)(X & 255u);
    X >>= 8;
    if (t >= 128) {
      t -= 256;
      X += 1;
    }
    dig[pp] = t;
  }
  dig[0] = (int)X;  // in [0, 256]
#pragma unroll
  for (int pp = 0; pp < kSlices; ++pp) {
    const int fexp = (emax - 1023 + 1) - 8 * (pp + 1) + 127;  // FP32 biased exponent of the scale
    float s = 0.0f;
    if (dig[pp] != 0 && fexp >= 1 && fexp <= 254) s = (float)dig[pp] * __int_as_float(fexp << 23);
    v[pp] = neg ? -s : s;
  }
}

}  // namespace gpc
