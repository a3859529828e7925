// Pass 2 as a gather over the window (gather2.cuh).  A block takes a tile of consecutive
// output columns of one column line, stages the pieces of the tile's window (float
// approximations of the heights and dx) in shared memory with coalesced loads, and its warps
// compute one output column at a time.  A window too large for the staging area is read
// straight from global memory by the same code.
#include "launch.h"

namespace dexel {

long long pass2g_smem(int warps, int stcap, int bcap, int tile, int R, int stage_cap) {
  const long long win = (long long)tile + 2LL * R + 1;
  long long b = 0;
  b += (win + 1) * sizeof(int);                          // source offsets
  b += (long long)stage_cap * (2 * sizeof(float) + 1);  // staged pieces
  b = (b + 15) & ~15LL;
  b += warps * ((gather_warp_bytes(stcap, bcap) + 15) & ~15LL);
  return b;
}

template <typename T>
__global__ void __launch_bounds__(256) k_pass2g(P2GParams<T> P) {
  typedef typename H<T>::K Key;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const Lanes L{lane, 32};
  const int R = P.R, T_ = P.tile;
  const int win = T_ + 2 * R + 1;
  int* soff = (int*)smem;
  float* saf = (float*)(soff + win + 1);
  float* sbf = saf + P.stage_cap;
  unsigned char* sd8 = (unsigned char*)(sbf + P.stage_cap);
  unsigned char* wbase = smem + ((((long long)(win + 1) * sizeof(int) +
                                   (long long)P.stage_cap * (2 * sizeof(float) + 1)) + 15) & ~15LL);
  const GatherWarp G =
      gather_warp(wbase + (long long)warp * ((gather_warp_bytes(P.stcap, P.bcap) + 15) & ~15LL), P.stcap, P.bcap);
  const float wmax2 = 2.0f * P.wtabf[0];
  ArenaCursor cur{0, 0};
  if (P.redo) {
    // only the columns the register-stack kernel marked (count -1), read from global memory
    const long long ncols = (long long)P.nx * P.ny;
    const long long nw = (long long)gridDim.x * P.warps_per_block;
    for (long long c = (long long)blockIdx.x * P.warps_per_block + warp; c < ncols; c += nw) {
      if (P.o_cnt[c] != -1) continue;
      const int i = (int)(c % P.nx), j = (int)(c / P.nx);
      const long long qb = (long long)i * P.ny;
      auto src = [&](int jj) {
        Src<Key> S;
        const long long ms = P.m_start[qb + jj];
        S.a = P.m_a + ms; S.b = P.m_b + ms; S.dx = P.m_l + ms; S.np = P.m_cnt[qb + jj];
        S.af = nullptr; S.bf = nullptr; S.d8 = nullptr;
        return S;
      };
      gather_column<T>(L, P, i, j, G, P.stcap, P.bcap, wmax2, src, cur);
    }
    return;
  }
  const int tiles_per_line = (P.ny + T_ - 1) / T_;
  const long long ntiles = (long long)P.nx * tiles_per_line;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int i = (int)(tile / tiles_per_line);
    const int j0 = (int)(tile % tiles_per_line) * T_;
    const int j1 = min(P.ny, j0 + T_);
    const int s0 = max(0, j0 - R), s1 = min(P.ny, j1 + R);
    const int ns = s1 - s0;
    const long long qb = (long long)i * P.ny;
    // piece counts of the window's sources -> offsets (block-wide, one warp)
    if (warp == 0) {
      int carry = 0;
      for (int base = 0; base < ns; base += 32) {
        const int t = base + lane;
        const int v = t < ns ? P.m_cnt[qb + s0 + t] : 0;
        const int inc = w_incl_add(v, lane);
        if (t < ns) soff[t] = carry + inc - v;
        carry += w_bcast(inc, 31);
      }
      if (lane == 0) soff[ns] = carry;
    }
    __syncthreads();
    const int total = soff[ns];
    const bool staged = total <= P.stage_cap && R < 256;
    if (staged) {
      // warps take sources round-robin; lanes copy pieces (coalesced)
      for (int q = warp; q < ns; q += P.warps_per_block) {
        const long long ms = P.m_start[qb + s0 + q];
        const int n = soff[q + 1] - soff[q];
        const int o = soff[q];
        for (int p = lane; p < n; p += 32) {
          saf[o + p] = keyf(P.m_a[ms + p]);
          sbf[o + p] = keyf(P.m_b[ms + p]);
          sd8[o + p] = (unsigned char)P.m_l[ms + p];
        }
      }
    }
    __syncthreads();
    auto src = [&](int jj) {
      Src<Key> S;
      const long long q = qb + jj;
      const long long ms = P.m_start[q];
      S.a = P.m_a + ms;
      S.b = P.m_b + ms;
      S.dx = P.m_l + ms;
      S.np = P.m_cnt[q];
      if (staged) {
        const int o = soff[jj - s0];
        S.af = saf + o;
        S.bf = sbf + o;
        S.d8 = sd8 + o;
      } else {
        S.af = nullptr;
        S.bf = nullptr;
        S.d8 = nullptr;
      }
      return S;
    };
    for (int j = j0 + warp; j < j1; j += P.warps_per_block)
      gather_column<T>(L, P, i, j, G, P.stcap, P.bcap, wmax2, src, cur);
    __syncthreads();
  }
}

template <typename T>
cudaError_t launch_pass2g(const P2GParams<T>& P, int blocks, cudaStream_t st) {
  const size_t smem = (size_t)pass2g_smem(P.warps_per_block, P.stcap, P.bcap, P.tile, P.R, P.stage_cap);
  cudaError_t e = cudaFuncSetAttribute(k_pass2g<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_pass2g<T><<<blocks, P.warps_per_block * 32, smem, st>>>(P);
  return cudaGetLastError();
}

template cudaError_t launch_pass2g<float>(const P2GParams<float>&, int, cudaStream_t);
template cudaError_t launch_pass2g<double>(const P2GParams<double>&, int, cudaStream_t);

}  // namespace dexel

namespace dexel {

// Register-stack gather: a warp covers G consecutive output columns at once when the window
// is short (lane -> (column, dy)), otherwise one column with the lanes looping over dy.
// Each column collects its sources' intervals in a shared-memory bucket, which is then
// sorted and united by the whole warp.
long long pass2r_smem(int warps, int G, int bcap) {
  const long long per = (long long)G * bcap * 2 * sizeof(ukey) + 2LL * bcap * sizeof(ukey) +
                        2LL * bcap * sizeof(int) + 16LL * G + 16;
  return warps * ((per + 15) & ~15LL);
}

template <typename T>
__global__ void __launch_bounds__(128) k_pass2r(P2GParams<T> P, int G) {
  typedef typename H<T>::K Key;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const Lanes L{lane, 32};
  const int bcap = P.bcap;
  const long long per = (long long)G * bcap * 2 * sizeof(ukey) + 2LL * bcap * sizeof(ukey) +
                        2LL * bcap * sizeof(int) + 16LL * G + 16;
  unsigned char* wb = smem + (long long)warp * ((per + 15) & ~15LL);
  ukey* bkl = (ukey*)wb;                   // G buckets of bcap left keys
  ukey* bkr = bkl + (long long)G * bcap;   // ... right keys
  ukey* ul = bkr + (long long)G * bcap;
  ukey* ur = ul + bcap;
  int* f0 = (int*)(ur + bcap);
  int* f1 = f0 + bcap;
  int* cnt = f1 + bcap;                    // G counters
  const float wmaxf = P.wtabf[0];
  const int W = 2 * P.R + 1;
  const long long ncols = (long long)P.nx * P.ny;
  ArenaCursor cur{0, 0};
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long c0 = ((long long)blockIdx.x * (blockDim.x >> 5) + warp) * G; c0 < ncols; c0 += nwarps * G) {
    const int g_n = (int)min((long long)G, ncols - c0);
    if (lane < G) cnt[lane] = 0;
    wsync();
    bool ok = true;
    if (G > 1) {
      const int g = lane / W, d = lane % W;
      if (g < g_n) {
        const long long item = c0 + g;
        const int i = (int)(item / P.ny), j = (int)(item % P.ny);
        const int dy = d - P.R, jj = j + dy;
        if (jj >= 0 && jj < P.ny) {
          const long long q = (long long)i * P.ny + jj;
          const long long ms = P.m_start[q];
          Src<Key> S;
          S.a = P.m_a + ms; S.b = P.m_b + ms; S.dx = P.m_l + ms; S.np = P.m_cnt[q];
          S.af = nullptr; S.bf = nullptr; S.d8 = nullptr;
          ok = source_cover_reg<Key, true>(S, dy < 0 ? -dy : dy, P.reach, P.wtab, P.wtabf, wmaxf,
                                     bkl + (long long)g * bcap, bkr + (long long)g * bcap, cnt + g, bcap);
        }
      }
    } else {
      const int i = (int)(c0 / P.ny), j = (int)(c0 % P.ny);
      for (int dy = -P.R + lane; dy <= P.R && ok; dy += 32) {
        const int jj = j + dy;
        if (jj < 0 || jj >= P.ny) continue;
        const long long q = (long long)i * P.ny + jj;
        const long long ms = P.m_start[q];
        Src<Key> S;
        S.a = P.m_a + ms; S.b = P.m_b + ms; S.dx = P.m_l + ms; S.np = P.m_cnt[q];
        S.af = nullptr; S.bf = nullptr; S.d8 = nullptr;
        ok = source_cover_reg<Key, true>(S, dy < 0 ? -dy : dy, P.reach, P.wtab, P.wtabf, wmaxf, bkl, bkr,
                                   cnt, bcap);
      }
    }
    wsync();
    if (w_any(!ok)) {
      // too deep a stack or too many intervals: mark the columns for the fallback pass
      if (lane < g_n) {
        const long long item = c0 + lane;
        const int i = (int)(item / P.ny), j = (int)(item % P.ny);
        P.o_cnt[(long long)j * P.nx + i] = -1;
        note_max(&P.ctr->max_state, cnt[lane]);  // intervals the column needs (when counted)
      }
      if (lane == 0) {
        set_status(&P.ctr->status, ST_OVERFLOW_SLOT);
        atomicAdd(&P.ctr->redo_cols, g_n);
      }
      wsync();
      continue;
    }
    for (int g = 0; g < g_n; ++g) {
      const long long item = c0 + g;
      const int i = (int)(item / P.ny), j = (int)(item % P.ny);
      ukey* kl = bkl + (long long)g * bcap;
      ukey* kr = bkr + (long long)g * bcap;
      const int total = cnt[g];
      const int n2 = pow2_at_least(total);
      for (int t = total + lane; t < n2; t += 32) { kl[t] = ~0ULL; kr[t] = ~0ULL; }
      wsync();
      if (n2 > 1) warp_bitonic(L, kl, kr, n2);
      const int no = total > 0 ? union_runs(L, kl, kr, total, true, f0, f1, ul, ur, kr, nullptr) : 0;
      const long long s = arena_take(L, &P.ctr->arena_top[3], P.blk, cur, no);
      const bool fits = s + no <= P.o_cap;
      if (!fits) {
        if (lane == 0) set_status(&P.ctr->status, ST_OVERFLOW_ARENA);
      } else {
        for (int q = lane; q < no; q += 32) { P.o_l[s + q] = ul[q]; P.o_r[s + q] = ur[q]; }
      }
      if (lane == 0) {
        const long long c = (long long)j * P.nx + i;
        P.o_start[c] = fits ? s : 0;
        P.o_cnt[c] = no;
        note_max(&P.ctr->max_out, no);
        add_total(&P.ctr->out_total, no);
      }
      wsync();
    }
  }
}

template <typename T>
cudaError_t launch_pass2r(const P2GParams<T>& P, int G, int blocks, cudaStream_t st) {
  const size_t smem = (size_t)pass2r_smem(4, G, P.bcap);
  cudaError_t e = cudaFuncSetAttribute(k_pass2r<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_pass2r<T><<<blocks, 128, smem, st>>>(P, G);
  return cudaGetLastError();
}

template cudaError_t launch_pass2r<float>(const P2GParams<float>&, int, int, cudaStream_t);
template cudaError_t launch_pass2r<double>(const P2GParams<double>&, int, int, cudaStream_t);

}  // namespace dexel
