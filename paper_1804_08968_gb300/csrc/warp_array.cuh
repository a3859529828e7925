// Warp-cooperative array primitives.
//
// The sweep kernels work "array at a time": one warp owns a work item and keeps its state
// in SoA arrays; every operation is a lane-strided loop over elements followed by a warp
// collective (scan, broadcast).  The same source also compiles as plain C++ with a single
// lane (nl == 1), which is how the step logic is unit-checked on a CPU during development.
#pragma once
#include <stdint.h>
#include <math.h>

#if defined(__CUDACC__)
#define DXI __host__ __device__ __forceinline__
#define DXN static __host__ __device__ __noinline__
#else
#define DXI inline
#define DXN static
#endif

#if !defined(__CUDACC__)
#include <algorithm>
#endif

namespace dexel {

#if !defined(__CUDACC__)
using std::max;
using std::min;
#endif

struct Lanes {
  int lane;  // this thread's lane (0..nl-1)
  int nl;    // lanes cooperating on the work item (32 on the GPU)
};

DXI void wsync() {
#if defined(__CUDA_ARCH__)
  __syncwarp();
#endif
}

DXI int w_incl_add(int v, int lane) {
#if defined(__CUDA_ARCH__)
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
#else
  (void)lane;
#endif
  return v;
}

DXI int w_bcast(int v, int src) {
#if defined(__CUDA_ARCH__)
  return __shfl_sync(0xffffffffu, v, src);
#else
  (void)src;
  return v;
#endif
}

DXI int w_max(int v) {
#if defined(__CUDA_ARCH__)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
#endif
  return v;
}

DXI int w_any(int p) {
#if defined(__CUDA_ARCH__)
  return __any_sync(0xffffffffu, p);
#else
  return p;
#endif
}

// Running maximum of an int across lanes (inclusive).
DXI int w_incl_max(int v, int lane) {
#if defined(__CUDA_ARCH__)
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v = max(v, u);
  }
#else
  (void)lane;
#endif
  return v;
}

DXI double w_incl_maxd(double v, int lane) {
#if defined(__CUDA_ARCH__)
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    double u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v = fmax(v, u);
  }
#else
  (void)lane;
#endif
  return v;
}

DXI double w_bcastd(double v, int src) {
#if defined(__CUDA_ARCH__)
  return __shfl_sync(0xffffffffu, v, src);
#else
  (void)src;
  return v;
#endif
}

// a[0..n) := exclusive prefix sums of a; returns the total (same value in every lane).
DXI int scan_excl(const Lanes& L, int* a, int n) {
  int carry = 0;
  for (int base = 0; base < n; base += L.nl) {
    const int t = base + L.lane;
    const int v = t < n ? a[t] : 0;
    const int inc = w_incl_add(v, L.lane);
    if (t < n) a[t] = carry + inc - v;
    carry += w_bcast(inc, L.nl - 1);
  }
  wsync();
  return carry;
}

// m[t] := max(idx[0..t-1]) over entries whose flag is set, -1 if none (exclusive).
// Used to find, for every element, the nearest earlier element with a property.
DXI void scan_last_flag(const Lanes& L, const int* flag, int* out, int n) {
  int carry = -1;
  for (int base = 0; base < n; base += L.nl) {
    const int t = base + L.lane;
    const int v = (t < n && flag[t]) ? t : -1;
    const int inc = w_incl_max(v, L.lane);
    // exclusive: shift the inclusive result by one lane
#if defined(__CUDA_ARCH__)
    int prev = __shfl_up_sync(0xffffffffu, inc, 1);
    if (L.lane == 0) prev = -1;
#else
    const int prev = -1;
#endif
    if (t < n) out[t] = prev > carry ? prev : carry;
    carry = max(carry, w_bcast(inc, L.nl - 1));
  }
  wsync();
}

// next[t] := min(idx[t+1..n)) over entries whose flag is set, n if none.
DXI void scan_next_flag(const Lanes& L, const int* flag, int* out, int n) {
  // walk chunks from the end; within a chunk take a suffix minimum
  int carry = n;
  const int nchunks = (n + L.nl - 1) / L.nl;
  for (int c = nchunks - 1; c >= 0; --c) {
    const int t = c * L.nl + L.lane;
    int v = (t < n && flag[t]) ? t : n;
    int suf = v;
#if defined(__CUDA_ARCH__)
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int u = __shfl_down_sync(0xffffffffu, suf, o);
      if (L.lane + o < 32) suf = min(suf, u);
    }
    int nxt = __shfl_down_sync(0xffffffffu, suf, 1);
    if (L.lane == 31) nxt = n;
#else
    const int nxt = n;
#endif
    if (t < n) out[t] = nxt < carry ? nxt : carry;
    carry = min(carry, w_bcast(suf, 0));
  }
  wsync();
}

// number of elements of the sorted array a[0..n) that are < x (lower bound)
template <typename T>
DXI int lower_bound(const T* a, int n, T x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < x)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// number of elements of the sorted array a[0..n) that are <= x (upper bound)
template <typename T>
DXI int upper_bound(const T* a, int n, T x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] <= x)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// Endpoints of a sorted list of closed pieces [a_p, b_p] read as one non-decreasing
// sequence a_0, b_0, a_1, b_1, ...
template <typename T>
DXI T endpoint(const T* a, const T* b, int e) {
  return (e & 1) ? b[e >> 1] : a[e >> 1];
}

// Number of endpoints of the piece list (a, b, n) that are < x (strict) or <= x.
template <typename T>
DXI int count_endpoints_lt(const T* a, const T* b, int n, T x) {
  int lo = 0, hi = 2 * n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (endpoint(a, b, mid) < x)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}
template <typename T>
DXI int count_endpoints_le(const T* a, const T* b, int n, T x) {
  int lo = 0, hi = 2 * n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (endpoint(a, b, mid) <= x)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

}  // namespace dexel
