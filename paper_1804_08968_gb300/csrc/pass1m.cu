// Pass-1 kernel for short reaches, one lane a column merging its window's sources (the walk is
// in pass1m.cuh).
#include <algorithm>

#include "launch.h"
#include "pass1m.cuh"

namespace dexel {

// 4 blocks an SM (64 registers): latency-bound, more warps pay (k = 2: 0.35 -> 0.33 ms)
template <typename T, int NS>
__global__ void __launch_bounds__(256, 4) k_pass1m(P1Params<T> P) {
  if (*(volatile int*)&P.ctr->status & ST_BAD_CSR) return;  // (stream-ordered calls: no plan for a bad input)
  const int lane = threadIdx.x & 31;
  const Lanes L{lane, 32};
  const long long ncols = (long long)P.nx * P.ny;
  const long long stride = (long long)gridDim.x * blockDim.x;
  ArenaCursor cur{0, 0};
  for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < ncols;
       base += stride) {
    const long long c = base + lane;  // row-major: a warp takes consecutive columns of a row
    const bool act = c < ncols;
    const int i = act ? (int)(c % P.nx) : 0, j = act ? (int)(c / P.nx) : 0;
    const int n = merge_walk<T, NS, false>(P, i, j, act, nullptr, nullptr, nullptr);
    const int inc = w_incl_add(n, lane);
    const int tot = w_bcast(inc, 31);
    const long long s = arena_take(L, &P.ctr->arena_top[1], P.blk, cur, tot);
    const bool fits = s + tot <= P.m_cap;
    const long long o = s + inc - n;
    if (fits && n > 0) merge_walk<T, NS, true>(P, i, j, act, P.m_a + o, P.m_b + o, P.m_l + o);
    if (act) {
      const long long q = (long long)i * P.ny + j;
      P.m_start[q] = fits ? o : 0;
      P.m_cnt[q] = n;
    }
    if (lane == 0 && !fits) set_status(&P.ctr->status, ST_OVERFLOW_ARENA);
    const int mx = __reduce_max_sync(0xffffffffu, n);
    if (lane == 0) {
      cur.tally += tot;
      cur.tmax = mx > cur.tmax ? mx : cur.tmax;
    }
  }
  if (lane == 0 && cur.tally > 0) {
    add_total(&P.ctr->mid_total, cur.tally);
    note_max(&P.ctr->max_pieces, cur.tmax);
  }
}

template <typename T>
cudaError_t launch_pass1m(const P1Params<T>& P, int sms, cudaStream_t st) {
  if (P.K > kMergeMaxReach) return cudaErrorInvalidValue;
  const long long ncols = (long long)P.nx * P.ny;
  const int blocks = (int)std::max<long long>(1, std::min<long long>((long long)sms * 8, (ncols + 255) / 256));
  if (P.K <= 1)
    k_pass1m<T, 3><<<blocks, 256, 0, st>>>(P);
  else
    k_pass1m<T, 5><<<blocks, 256, 0, st>>>(P);
  return cudaGetLastError();
}

template cudaError_t launch_pass1m<float>(const P1Params<float>&, int, cudaStream_t);
template cudaError_t launch_pass1m<double>(const P1Params<double>&, int, cudaStream_t);

}  // namespace dexel
