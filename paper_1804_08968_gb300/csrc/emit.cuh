// Device pieces shared by the single-shape and the batched drivers: the output column
// finisher (erosion complement, rounding, re-merge), the multi-block exclusive scan and the
// packed float copy of S_mid.  Templates and static functions: every translation unit that
// includes this header gets its own copy.
#pragma once
#include "gather2.cuh"

namespace dexel {

// One output column: optional complement (erosion), rounding to T, and re-merge of pieces
// that touch after rounding.  Returns the count; writes pieces when out != nullptr.
template <typename T>
__device__ int finalize_column(const ukey* lk, const ukey* rk, int m, bool erode, T* out) {
  if (m < 0) m = 0;  // (a column a failed gather left marked: its call reports the failure)
  int cnt = 0;
  T ca = 0, cb = 0;
  bool have = false;
  auto push = [&](double a, double b) {
    const T ta = (T)a, tb = (T)b;
    if (erode && !(ta < tb)) return;
    if (have && ta <= cb) {
      if (tb > cb) cb = tb;
      return;
    }
    if (have) {
      if (out) { out[2 * cnt] = ca; out[2 * cnt + 1] = cb; }
      ++cnt;
    }
    ca = ta;
    cb = tb;
    have = true;
  };
  auto l = [&](int t) { return dval(lk[t]); };
  auto r = [&](int t) { return dval(rk[t]); };
  if (!erode) {
    for (int t = 0; t < m; ++t) push(l(t), r(t));
  } else if (m == 0) {
    push(-INFINITY, INFINITY);
  } else {
    if (l(0) > -INFINITY) push(-INFINITY, l(0));
    for (int t = 0; t + 1 < m; ++t) push(r(t), l(t + 1));
    if (r(m - 1) < INFINITY) push(r(m - 1), INFINITY);
  }
  if (have) {
    if (out) { out[2 * cnt] = ca; out[2 * cnt + 1] = cb; }
    ++cnt;
  }
  return cnt;
}

// exclusive scan of cnt[0..n) (int64) in three launches; writes pos (int64) and col_off
constexpr int kScanThreads = 256, kScanPer = 8, kScanTile = kScanThreads * kScanPer;

template <typename C>
__global__ void k_scan1(long long n, const C* cnt, long long* pos, long long* sums) {
  __shared__ long long sh[kScanThreads];
  const long long base = (long long)blockIdx.x * kScanTile + threadIdx.x * kScanPer;
  long long v[kScanPer];
  long long s = 0;
  for (int q = 0; q < kScanPer; ++q) {
    v[q] = base + q < n ? (long long)cnt[base + q] : 0;
    s += v[q];
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 1; o < kScanThreads; o <<= 1) {
    const long long u = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
    __syncthreads();
    sh[threadIdx.x] += u;
    __syncthreads();
  }
  long long run = sh[threadIdx.x] - s;
  for (int q = 0; q < kScanPer; ++q) {
    if (base + q < n) pos[base + q] = run;
    run += v[q];
  }
  if (threadIdx.x == kScanThreads - 1) sums[blockIdx.x] = sh[threadIdx.x];
}

// Line-contiguous float copy of S_mid for the gather: column q = i*ny + j gets the range
// c_start[q] = pos[q] + sums[q / kScanTile] (exclusive scan of the piece counts in q order), so
// that the pieces of any run of sources of a line are one contiguous range; ends as float
// approximations (keyf), dx as short.  Also records max |finite end| for the float filter.
template <typename Key>
__global__ void k_mid_pack(long long ncols, const long long* m_start, const int* m_cnt,
                           const Key* m_a, const Key* m_b, const short* m_l,
                           const long long* pos, const long long* sums, long long* c_start,
                           float* c_af, float* c_bf, short* c_dx, Counters* ctr,
                           long long m_cap = -1, long long c_cap = -1) {
  const int lane = threadIdx.x & 31;
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  float zm = 0.0f;
  for (long long q = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); q < ncols; q += nw) {
    const long long c = pos[q] + sums[q / kScanTile];
    if (lane == 0) c_start[q] = c;
    const long long ms = m_start[q];
    int n = m_cnt[q];
    if (m_cap >= 0 && (ms < 0 || n < 0 || ms + n > m_cap || c + n > c_cap)) {
      // (the capacities given: a column beyond S_mid or the copy is skipped, status set)
      if (lane == 0) set_status(&ctr->status, ST_OVERFLOW_ARENA);
      n = 0;
    }
    for (int p = lane; p < n; p += 32) {
      const float a = keyf(m_a[ms + p]), b = keyf(m_b[ms + p]);
      c_af[c + p] = a;
      c_bf[c + p] = b;
      c_dx[c + p] = m_l[ms + p];
      if (fabsf(a) < __builtin_huge_valf()) zm = fmaxf(zm, fabsf(a));
      if (fabsf(b) < __builtin_huge_valf()) zm = fmaxf(zm, fabsf(b));
    }
  }
  for (int o = 16; o > 0; o >>= 1) zm = fmaxf(zm, __shfl_xor_sync(0xffffffffu, zm, o));
  if (lane == 0 && zm > 0.0f) atomicMax(&ctr->zmax_bits, __float_as_uint(zm));
}

static __global__ void k_scan2(long long nb, long long* sums) {
  __shared__ long long sh[kScanThreads];
  long long carry = 0;
  for (long long b0 = 0; b0 < nb; b0 += kScanThreads) {
    const long long b = b0 + threadIdx.x;
    const long long v = b < nb ? sums[b] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < kScanThreads; o <<= 1) {
      const long long u = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
      __syncthreads();
      sh[threadIdx.x] += u;
      __syncthreads();
    }
    if (b < nb) sums[b] = carry + sh[threadIdx.x] - v;
    const long long tot = sh[kScanThreads - 1];
    __syncthreads();
    carry += tot;
  }
  if (threadIdx.x == 0) sums[nb] = carry;
}

}  // namespace dexel
