// Order-independent accumulation in 128-bit fixed point (deterministic mode).
//
// A contribution v is rounded once to the nearest multiple of 2^-64 and added
// to a two's-complement 128-bit integer (lo word unsigned, hi word signed)
// with integer atomics: integer addition is associative, so the sum does not
// depend on the order in which the contributions arrive, and repeated runs
// give bitwise identical results.  The carry out of the low word is taken
// from the value the low-word atomic returns, which is exact per addition.
// Range |sum| < 2^63, resolution 2^-64 (far below the FP64 rounding of any
// value the triples path produces).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace cc3 {

// round(v * 2^64) as a 128-bit two's-complement integer (hi:lo)
__device__ __forceinline__ void fx_from_double(double v, long long *hi, unsigned long long *lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int ex = (int)((b >> 52) & 0x7FF);
  unsigned long long mh = 0, ml = 0;  // magnitude
  if (ex != 0 && ex != 0x7FF) {
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
    const int sh = ex - 1075 + 64;  // v = m 2^(ex-1075), scaled by 2^64
    if (sh >= 64) {
      mh = sh - 64 < 10 ? (m << (sh - 64)) : 0x7FFFFFFFFFFFFFFFull;  // |v| < 2^63 assumed
    } else if (sh >= 0) {
      ml = m << sh;
      mh = sh > 11 ? (m >> (64 - sh)) : 0;
    } else if (sh > -64) {
      const int r = -sh;
      ml = (m >> r) + ((m >> (r - 1)) & 1ull);  // round half up on the magnitude
    } else if (sh == -64) {
      ml = m >> 63;  // 0 (m < 2^53)
    }
  }
  if (b >> 63) {  // negate
    ml = ~ml + 1ull;
    mh = ~mh + (ml == 0ull ? 1ull : 0ull);
  }
  *hi = (long long)mh;
  *lo = ml;
}

// slot[0] = lo word, slot[1] = hi word
__device__ __forceinline__ void fx_add(unsigned long long *slot, double v) {
  long long hi;
  unsigned long long lo;
  fx_from_double(v, &hi, &lo);
  if (lo == 0ull && hi == 0) return;
  const unsigned long long old = atomicAdd(slot, lo);
  const unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
  const unsigned long long h = (unsigned long long)hi + carry;
  if (h) atomicAdd(slot + 1, h);
}

}  // namespace cc3
