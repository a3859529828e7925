// Pass 2 by levels: the kernels (the formulation and the per-item bodies are in pass2l.cuh).
#include <algorithm>

#include "launch.h"
#include "pass2l.cuh"

namespace dexel {

template <typename T, bool LTAB, bool EXACT>
__global__ void __launch_bounds__(256, 4) k_levels(LvlParams<T> A, int tab_floats) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const LvlLayout Lo = lvl_layout(blockDim.x >> 5, tab_floats, A.slots);
  unsigned* ws = (unsigned*)(smem + Lo.slots) + warp * 2 * A.slots * 32;
  float4* stg = (float4*)(smem + Lo.stage) + warp * kLvlStage;
  const float* tab = lvl_tables<LTAB>((float*)(smem + Lo.tab), A.P.R, A.L, A.G, A.NG, A.P.nmax,
                                      A.P.wtabf);
  __syncthreads();
  const float E = 9.5367432e-7f * (__uint_as_float(A.P.ctr->zmax_bits) + A.P.wtabf[0]);  // 2^-20
  const long long nitems = lvl_items(A.nsrc, A.L, A.yw);
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  ArenaCursor cur{0, 0};
  for (long long item = (long long)blockIdx.x * (blockDim.x >> 5) + warp; item < nitems; item += nw)
    levels_item<T, LTAB ? kTabBlock : kTabFlat, EXACT>(A, item, lane, ws, stg, E, (float*)tab, cur,
                                                       (long long)blockIdx.x * (blockDim.x >> 5) + warp);
}

// MINB blocks an SM: 4 (64 registers, some spilled) pays at short windows (k = 8: 0.47 ->
// 0.34 ms on the 512^2 workload), 3 (80 registers) at long ones (k = 32: 0.62 against 0.76)
template <typename T, int MINB>
__global__ void __launch_bounds__(256, MINB) k_lgather(LvlParams<T> A, int bcap, int redo) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char* wb = smem + (long long)warp * (bcap * (2 * sizeof(ukey) + 2 * sizeof(int)) + 16);
  const long long q1 = A.q0 + A.nsrc;  // the block's output columns in line order
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  if (*(volatile int*)&A.P.ctr->status & ST_LEVELS_OVER) return;  // the lists are incomplete
  if (redo && *(volatile int*)&A.P.ctr->redo_cols == 0) return;  // (a redo with nothing marked)
  ArenaCursor cur{0, 0};
  for (long long item = A.q0 + (long long)blockIdx.x * (blockDim.x >> 5) + warp; item < q1; item += nw)
    lgather_column<T>(A, item, bcap, redo, lane, wb, cur);
  if (lane == 0 && cur.tally > 0) {
    add_total(&A.P.ctr->out_total, cur.tally);
    note_max(&A.P.ctr->max_out, cur.tmax);
  }
}

// 6 blocks an SM (40 registers; the runs live in local memory): load-latency-bound
template <typename T>
__global__ void __launch_bounds__(256, 6) k_lgather_lanes(LvlParams<T> A) {
  const int lane = threadIdx.x & 31;
  const long long q1 = A.q0 + A.nsrc;  // the block's output columns in line order
  const long long stride = (long long)gridDim.x * blockDim.x;
  if (*(volatile int*)&A.P.ctr->status & ST_LEVELS_OVER) return;  // the lists are incomplete
  ArenaCursor cur{0, 0};
  for (long long base = A.q0 + (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < q1;
       base += stride)
    lgather_lane<T>(A, base + lane, base + lane < q1, lane, cur);
  if (lane == 0 && cur.tally > 0) {
    add_total(&A.P.ctr->out_total, cur.tally);
    note_max(&A.P.ctr->max_out, cur.tmax);
  }
}

template <typename T>
cudaError_t launch_lgather(const LvlParamsHost<T>& H, int bcap, int redo, cudaStream_t st, int sms);

template <typename T>
static LvlParams<T> lvl_params(const LvlParamsHost<T>& H) {
  LvlParams<T> A;
  A.P = H.P;
  A.l_p = H.l_p; A.l_cap = H.l_cap;
  A.W = 2 * H.P.R + 1;
  A.slots = H.slots > 0 && H.slots <= kLvlSlots ? H.slots : lvl_slots_for(H.P.R);
  A.spill = H.spill;
  A.spill_cap = H.spill ? H.spill_cap : 0;
  A.L = H.P.R + 1;
  if (A.L <= 32) {
    A.G = 32 / A.L;
    A.NG = 0;
  } else {
    A.G = 1;
    A.NG = (H.P.R + 31) / 32;
  }
  // a block of lines: the index is addressed with the global column index q, so its base
  // pointer is shifted by the block's first entry (q0 W); nlev bounds q W + u
  A.yw = H.yw >= 0 ? H.yw : H.P.R;
  A.q0 = H.q0;
  A.nsrc = H.nq > 0 ? H.nq : (long long)H.P.nx * H.P.ny;
  A.l_idx = H.l_idx - H.q0 * A.W;
  A.nlev = (H.q0 + A.nsrc) * A.W;
  A.m_cap = H.m_cap;
  A.c_cap = H.c_cap;
  return A;
}

// the grid of launch_levels: sms x 4 blocks of 8 warps
long long lvl_spill_bytes(int sms, int spill_cap) {
  return (long long)sms * 4 * 8 * 32 * 2 * spill_cap * (long long)sizeof(unsigned);
}

template <typename T>
cudaError_t launch_levels(const LvlParamsHost<T>& H, cudaStream_t st, int sms) {
  const LvlParams<T> A = lvl_params(H);
  // lists a warp skips (an overflow) then read as empty
  cudaError_t e = cudaMemsetAsync(H.l_idx, 0, sizeof(unsigned long long) * A.nsrc * A.W, st);
  if (e != cudaSuccess) return e;
  const long long lt = lvl_lane_tab(H.P.R);
  const bool ltab = lt <= kLvlLaneTab;
  const int tab_floats = ltab ? (int)lt : (H.P.nmax + 1 <= kLvlTable ? H.P.nmax + 1 : 0);
  const size_t sm1 = (size_t)lvl_layout(8, tab_floats, A.slots).total;
  auto kern = ltab ? (H.exact ? k_levels<T, true, true> : k_levels<T, true, false>)
                   : (H.exact ? k_levels<T, false, true> : k_levels<T, false, false>);
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
  if (e != cudaSuccess) return e;
  kern<<<sms * 4, 256, sm1, st>>>(A, tab_floats);
  return cudaGetLastError();
}

// the per-column gather with buckets of bcap intervals (redo: only the columns marked -1)
template <typename T>
cudaError_t launch_lgather(const LvlParamsHost<T>& H, int bcap, int redo, cudaStream_t st, int sms) {
  const LvlParams<T> A = lvl_params(H);
  const long long per_warp = lgather_smem(1, bcap);
  int warps = 8;
  while (warps > 1 && warps * per_warp > (110LL << 10)) warps >>= 1;
  const size_t sm2 = (size_t)lgather_smem(warps, bcap);
  if (sm2 > (220u << 10)) return cudaErrorInvalidValue;
  auto kern = H.P.R <= 12 ? k_lgather<T, 4> : k_lgather<T, 3>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
  if (e != cudaSuccess) return e;
  const int per_sm = (int)std::max<long long>(1, std::min<long long>(64 / warps, (220LL << 10) / (long long)sm2));
  kern<<<sms * per_sm, warps * 32, sm2, st>>>(A, bcap, redo);
  return cudaGetLastError();
}

// the per-column gather with one lane a column (short windows); marked columns are left for
// launch_lgather's redo
template <typename T>
cudaError_t launch_lgather_lanes(const LvlParamsHost<T>& H, cudaStream_t st, int sms) {
  const LvlParams<T> A = lvl_params(H);
  k_lgather_lanes<T><<<sms * 8, 256, 0, st>>>(A);
  return cudaGetLastError();
}

template cudaError_t launch_lgather_lanes<float>(const LvlParamsHost<float>&, cudaStream_t, int);
template cudaError_t launch_lgather_lanes<double>(const LvlParamsHost<double>&, cudaStream_t, int);
template cudaError_t launch_levels<float>(const LvlParamsHost<float>&, cudaStream_t, int);
template cudaError_t launch_levels<double>(const LvlParamsHost<double>&, cudaStream_t, int);
template cudaError_t launch_lgather<float>(const LvlParamsHost<float>&, int, int, cudaStream_t, int);
template cudaError_t launch_lgather<double>(const LvlParamsHost<double>&, int, int, cudaStream_t, int);

}  // namespace dexel
