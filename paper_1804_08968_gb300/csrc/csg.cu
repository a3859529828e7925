// Boolean operations of two dexel grids (CSG in dexel space, Sec. 2 "(3)": the rays of a
// column are combined on their own; the thick shell of Sec. 4 "3D Printing" is the difference
// of a dilation and an erosion).
//
// One thread a column merges the two sorted lists of disjoint segments in one pass, without
// arithmetic on the heights (the results' ends are input ends, so FP32 and FP64 results are
// exact):
//   union         the lists merged by start and folded: the next segment joins the run when
//                 it starts at or below the run's end (closed union; an isolated zero-length
//                 segment stays);
//   intersection  two pointers: [max(a, c), min(b, d)] of the current pair when it has
//                 positive length, then the pair member that ends first advances;
//   difference    each segment of A minus the open interiors of the B segments that overlap
//                 it; pieces of positive length are kept (the closure of A \ B).
// Results of one column are disjoint with positive gaps, as the inputs.  A counting launch
// sizes every column, a scan places them, and a writing launch stores them.
#include "launch.h"

namespace dexel {

template <typename T, bool WRITE>
struct BoolOut {
  T* z;
  long long n = 0;
  __device__ __forceinline__ void put(T a, T b) {
    if (WRITE) {
      z[2 * n] = a;
      z[2 * n + 1] = b;
    }
    ++n;
  }
};

template <typename T, bool WRITE>
__device__ long long bool_column(int op, const T* za, int a0, int a1, const T* zb, int b0, int b1,
                                 T* zo) {
  BoolOut<T, WRITE> o{zo};
  if (op == kBoolUnion) {
    int p = a0, q = b0;
    bool have = false;
    T ca = 0, cb = 0;
    while (p < a1 || q < b1) {
      // the next segment by start (A first on ties)
      const bool takeA = q >= b1 || (p < a1 && za[2 * p] <= zb[2 * q]);
      const T* s = takeA ? za + 2 * p : zb + 2 * q;
      const T a = s[0], b = s[1];
      if (takeA) ++p; else ++q;
      if (have && a <= cb) {
        cb = b > cb ? b : cb;
      } else {
        if (have) o.put(ca, cb);
        ca = a;
        cb = b;
        have = true;
      }
    }
    if (have) o.put(ca, cb);
  } else if (op == kBoolIntersect) {
    int p = a0, q = b0;
    while (p < a1 && q < b1) {
      const T a = za[2 * p], b = za[2 * p + 1], c = zb[2 * q], d = zb[2 * q + 1];
      const T lo = a > c ? a : c, hi = b < d ? b : d;
      if (lo < hi) o.put(lo, hi);
      if (b < d) ++p; else ++q;
    }
  } else {
    int q = b0;
    for (int p = a0; p < a1; ++p) {
      const T a = za[2 * p], b = za[2 * p + 1];
      // B segments that end at or below a cannot touch this or a later A segment
      while (q < b1 && zb[2 * q + 1] <= a) ++q;
      T cur = a;
      for (int r = q; r < b1; ++r) {
        const T c = zb[2 * r], d = zb[2 * r + 1];
        if (c >= b) break;          // starts at or beyond this segment's end
        if (!(c < d)) continue;     // a zero-length B segment has no interior
        if (cur < c) o.put(cur, c);
        cur = d > cur ? d : cur;
        if (cur >= b) break;
      }
      if (cur < b) o.put(cur, b);
    }
  }
  return o.n;
}

template <typename T>
__global__ void k_bool_count(int op, long long ncols, const int* oa, const T* za, const int* ob,
                             const T* zb, long long* cnt) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncols) return;
  cnt[c] = bool_column<T, false>(op, za, oa[c], oa[c + 1], zb, ob[c], ob[c + 1], nullptr);
}

template <typename T>
__global__ void k_bool_write(int op, long long ncols, const int* oa, const T* za, const int* ob,
                             const T* zb, const long long* pos, T* zo) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncols) return;
  bool_column<T, true>(op, za, oa[c], oa[c + 1], zb, ob[c], ob[c + 1], zo + 2 * pos[c]);
}

template <typename T>
cudaError_t launch_bool_count(int op, long long ncols, const int* oa, const T* za, const int* ob,
                              const T* zb, long long* cnt, cudaStream_t st) {
  if (ncols <= 0) return cudaSuccess;
  k_bool_count<T><<<(unsigned)((ncols + 255) / 256), 256, 0, st>>>(op, ncols, oa, za, ob, zb, cnt);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_bool_write(int op, long long ncols, const int* oa, const T* za, const int* ob,
                              const T* zb, const long long* pos, T* zo, cudaStream_t st) {
  if (ncols <= 0) return cudaSuccess;
  k_bool_write<T><<<(unsigned)((ncols + 255) / 256), 256, 0, st>>>(op, ncols, oa, za, ob, zb, pos, zo);
  return cudaGetLastError();
}

template cudaError_t launch_bool_count<float>(int, long long, const int*, const float*, const int*,
                                              const float*, long long*, cudaStream_t);
template cudaError_t launch_bool_count<double>(int, long long, const int*, const double*, const int*,
                                               const double*, long long*, cudaStream_t);
template cudaError_t launch_bool_write<float>(int, long long, const int*, const float*, const int*,
                                              const float*, const long long*, float*, cudaStream_t);
template cudaError_t launch_bool_write<double>(int, long long, const int*, const double*, const int*,
                                               const double*, const long long*, double*, cudaStream_t);

}  // namespace dexel
