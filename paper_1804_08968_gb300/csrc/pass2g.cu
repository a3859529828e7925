// Pass 2 as a gather over the window (gather2.cuh): k_pass2t (tiles of a line staged in
// shared memory, the main kernel) and k_pass2c (columns read from global memory with one
// bucket for the whole window, for the columns k_pass2t hands back).
#include "launch.h"
#include "pass2t.cuh"

namespace dexel {

// Balanced gather (cover_range): one warp per output column, the window's pieces split
// evenly over the lanes.  Per-warp shared memory: the window's piece offsets, the bucket (left
// and right keys), the union's flags and outputs.  A column whose bucket overflows is marked
// (count -1) for a second launch of the same kernel with a larger bucket (redo mode).

template <typename T>
__global__ void __launch_bounds__(256) k_pass2c(P2GParams<T> P) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwb = blockDim.x >> 5;
  const Lanes L{lane, 32};
  const int R = P.R, bcap = P.bcap;
  unsigned char* wb = smem + (long long)warp * pass2c_warp_bytes(R, bcap);
  int* srcoff = (int*)wb;
  ukey* bl = (ukey*)(wb + (((2LL * R + 2) * sizeof(int) + 15) & ~15LL));
  ukey* br = bl + bcap;
  ukey* ul = br + bcap;
  ukey* ur = ul + bcap;
  int* f0 = (int*)(ur + bcap);
  int* f1 = f0 + bcap;
  int* bcount = f1 + bcap;
  const float wmax2 = 2.0f * P.wtabf[0];
  const long long ncols = (long long)P.nx * P.ny;
  const long long nw = (long long)gridDim.x * nwb;
  ArenaCursor cur{0, 0};
  for (long long item = (long long)blockIdx.x * nwb + warp; item < ncols; item += nw) {
    const int i = (int)(item / P.ny), j = (int)(item % P.ny);
    const long long c = (long long)j * P.nx + i;
    if (P.redo && P.o_cnt[c] != -1) continue;
    PHASE_BEGIN();
    const long long qb = (long long)i * P.ny;
    const int s0 = max(0, j - R), s1 = min(P.ny - 1, j + R);
    const int ns = s1 - s0 + 1;
    int carry = 0;
    for (int base = 0; base < ns; base += 32) {
      const int t = base + lane;
      const int v = t < ns ? P.m_cnt[qb + s0 + t] : 0;
      const int inc = w_incl_add(v, lane);
      if (t < ns) srcoff[t] = carry + inc - v;
      carry += w_bcast(inc, 31);
    }
    if (lane == 0) { srcoff[ns] = carry; *bcount = 0; }
    wsync();
    PHASE(0);
    const int per = (carry + 31) >> 5;
    const int g0 = min(carry, lane * per), g1 = min(carry, g0 + per);
    cover_range<T>(P, qb, j, s0, ns, srcoff, g0, g1, wmax2, bl, br, bcount, bcap);
    wsync();
    PHASE(1);
    const int total = *bcount;
    PHASE_COUNT(8, total);
    PHASE_COUNT(9, carry);
    PHASE_COUNT(10, 1);
    if (total > bcap) {
      if (lane == 0) {
        P.o_cnt[c] = -1;
        note_max(&P.ctr->max_state, total);
        set_status(&P.ctr->status, ST_OVERFLOW_SLOT);
        atomicAdd(&P.ctr->redo_cols, 1);
      }
      wsync();
      continue;
    }
    const int n2 = pow2_at_least(total);
    for (int t = total + lane; t < n2; t += 32) { bl[t] = ~0ULL; br[t] = ~0ULL; }
    wsync();
    if (n2 > 1) warp_sort_pairs(L, bl, br, n2);
    PHASE(2);
    PHASE_COUNT(11, n2);
    const int no = total > 0 ? union_runs(L, bl, br, total, true, f0, f1, ul, ur, br, nullptr) : 0;
    const long long s = arena_take(L, &P.ctr->arena_top[3], P.blk, cur, no);
    const bool fits = s + no <= P.o_cap;
    if (!fits) {
      if (lane == 0) set_status(&P.ctr->status, ST_OVERFLOW_ARENA);
    } else {
      for (int q = lane; q < no; q += 32) { P.o_l[s + q] = ul[q]; P.o_r[s + q] = ur[q]; }
    }
    if (lane == 0) {
      P.o_start[c] = fits ? s : 0;
      P.o_cnt[c] = no;
      note_max(&P.ctr->max_out, no);
      add_total(&P.ctr->out_total, no);
    }
    wsync();
    PHASE(3);
  }
}

template <typename T>
cudaError_t launch_pass2c(const P2GParams<T>& P, int warps_per_block, int blocks, cudaStream_t st) {
  const size_t smem = (size_t)(warps_per_block * pass2c_warp_bytes(P.R, P.bcap));
  cudaError_t e = cudaFuncSetAttribute(k_pass2c<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_pass2c<T><<<blocks, warps_per_block * 32, smem, st>>>(P);
  return cudaGetLastError();
}

template cudaError_t launch_pass2c<float>(const P2GParams<float>&, int, int, cudaStream_t);
template cudaError_t launch_pass2c<double>(const P2GParams<double>&, int, int, cudaStream_t);

}  // namespace dexel

namespace dexel {

// Tiled balanced gather: a block takes tc consecutive output columns of one line, stages the
// pieces of their common window (float ends and dx) in shared memory with coalesced loads,
// and its warps take the tile's columns, each splitting its window's pieces evenly over the
// lanes (column_cover).  A tile whose window holds more pieces than the staging area is cut
// into the longest runs of columns whose windows fit; columns whose single window does not
// fit are covered a warp each, their joint window staged in chunks.  Columns whose union
// outgrows the bucket are marked (count -1) for the redo launch of k_pass2c.
template <typename T, int MINB>
__global__ void __launch_bounds__(512, MINB) k_pass2t(P2GParams<T> P, int tc, int ntab, int stage_cap, int Q, int M) {
  extern __shared__ __align__(16) unsigned char smem[];
  const P2TLayout Lo = p2t_layout(P.R, tc, ntab, stage_cap, blockDim.x >> 5, P.bcap);
  float* swt = (float*)(smem + Lo.swt);
  for (int q = threadIdx.x; q < ntab; q += blockDim.x) swt[q] = P.wtabf[q];
  const float* wt = ntab > 0 ? swt : P.wtabf;
  const long long ntiles = (long long)P.nx * ((P.ny + tc - 1) / tc);
  ArenaCursor cur{0, 0};
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
    pass2t_tile<T>(P, tile, tc, ntab, stage_cap, Q, M, smem, wt, cur);
}

// minb: blocks an SM the kernel is compiled for (2 caps its registers at 64)
template <typename T>
cudaError_t launch_pass2t(const P2GParams<T>& P, int warps_per_block, int tc, int ntab,
                          int stage_cap, int Q, int M, int minb, int blocks, cudaStream_t st) {
  const P2TLayout Lo = p2t_layout(P.R, tc, ntab, stage_cap, warps_per_block, P.bcap);
  auto kern = minb >= 2 ? k_pass2t<T, 2> : k_pass2t<T, 1>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Lo.total);
  if (e != cudaSuccess) return e;
  kern<<<blocks, warps_per_block * 32, (size_t)Lo.total, st>>>(P, tc, ntab, stage_cap, Q, M);
  return cudaGetLastError();
}

template cudaError_t launch_pass2t<float>(const P2GParams<float>&, int, int, int, int, int, int, int, int, cudaStream_t);
template cudaError_t launch_pass2t<double>(const P2GParams<double>&, int, int, int, int, int, int, int, int, cudaStream_t);

}  // namespace dexel
