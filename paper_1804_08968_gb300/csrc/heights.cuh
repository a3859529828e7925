// Heights as order-preserving keys.
//
// The sweeps compare heights far more often than they do arithmetic on them.  On GB300 a
// double comparison runs on the narrow FP64 unit, so double heights are carried as 64-bit
// unsigned keys whose integer order is the numeric order (sign-magnitude flipped to two's
// complement order); comparisons and min/max become integer operations and the value is
// recovered exactly for the few places that compute (z -/+ w, the power predicates).
// Float heights stay floats (FP32 compares are full rate).  -0 is folded into +0; NaN never
// reaches the sweeps (the input is validated).
#pragma once
#include "warp_array.cuh"
#include <string.h>

namespace dexel {

DXI long long dbits(double x) {
#if defined(__CUDA_ARCH__)
  return __double_as_longlong(x);
#else
  long long b;
  memcpy(&b, &x, 8);
  return b;
#endif
}
DXI double bitsd(long long b) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double(b);
#else
  double x;
  memcpy(&x, &b, 8);
  return x;
#endif
}

typedef unsigned long long ukey;

DXI ukey dkey(double x) {
  long long b = dbits(x);
  if (b == (long long)0x8000000000000000ULL) b = 0;
  return (ukey)(b ^ ((b >> 63) | (long long)0x8000000000000000ULL));
}
DXI double dval(ukey k) {
  const long long s = (long long)k;
  return bitsd(s < 0 ? (long long)(k ^ 0x8000000000000000ULL) : (long long)~k);
}
constexpr ukey KEY_NINF = 0x000FFFFFFFFFFFFFULL;  // dkey(-inf)
constexpr ukey KEY_PINF = 0xFFF0000000000000ULL;  // dkey(+inf)

template <typename T>
struct H;

template <>
struct H<double> {
  typedef ukey K;
  DXI static K key(double x) { return dkey(x); }
  DXI static double val(K k) { return dval(k); }
  DXI static float valf(K k) { return (float)dval(k); }
  DXI static K ninf() { return KEY_NINF; }
  DXI static K pinf() { return KEY_PINF; }
};

template <>
struct H<float> {
  typedef float K;
  DXI static K key(float x) { return x == 0.0f ? 0.0f : x; }
  DXI static double val(K k) { return (double)k; }
  DXI static float valf(K k) { return k; }
  DXI static K ninf() { return -__builtin_huge_valf(); }
  DXI static K pinf() { return __builtin_huge_valf(); }
};

template <typename K>
DXI K kmax(K a, K b) { return a < b ? b : a; }
template <typename K>
DXI K kmin(K a, K b) { return b < a ? b : a; }

}  // namespace dexel
