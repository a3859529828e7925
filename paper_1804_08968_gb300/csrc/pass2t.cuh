// Pass-2 tiled gather, the per-tile body shared by the single-shape and the batched kernels
// (see gather2.cuh for the formulation).
#pragma once
#include "gather2.cuh"

namespace dexel {

// Cover of output column j from the staged pieces [ga, gz) of its window (af/bf/dxs indexed
// by the window's piece index): the pieces are split evenly over the lanes, and in rounds
// every lane takes at most M pieces and appends at most Q intervals, after which the warp
// unites the bucket into its front (acc runs, carried in and out so that a window can be
// covered in several chunks).  Returns false when the union outgrows bcap - 32 Q runs.
template <typename T>
DXI bool column_cover(const P2GParams<T>& P, const Lanes& L, int j, int s0, const int* soff,
                      const long long* sbase, int qlo, int qhi, int ga, int gz, const float* af,
                      const float* bf, const short* dxs, const float* wt, float E, int Q, int M,
                      ukey* bl, ukey* br, int* f0, int* f1, int* bcount, int bcap, int& acc) {
  const int pc = gz - ga;
  int per = (pc + 31) >> 5;
  if (per > 1 && !(per & 1)) ++per;  // odd stride: no bank conflicts
  const int g0 = ga + min(pc, L.lane * per), g1 = ga + min(pc, L.lane * per + per);
  LaneWalk w;
  walk_init<T>(w, j, s0, soff, sbase, qlo, qhi, g0, g1);
  for (;;) {
    if (L.lane == 0) *bcount = acc;
    wsync();
    cover_round<T>(P, w, j, s0, soff, sbase, af, bf, dxs, wt, g1, E, Q, M, bl, br, bcount, bcap);
    wsync();
    const int n = *bcount;
    const bool fin = !w_any(!w.done);
    if (n > acc) {
      const int n2 = pow2_at_least(n);
      for (int t = n + L.lane; t < n2; t += 32) { bl[t] = ~0ULL; br[t] = ~0ULL; }
      wsync();
      if (n2 > 1) warp_bitonic(L, bl, br, n2);
      acc = union_count(L, bl, br, n, f0, f1);
      union_write_inplace(L, bl, br, n, f0, f1);
    }
    if (fin) return true;
    if (acc > bcap - 32 * Q) return false;
  }
}

// Writes the acc runs at the front of the bucket as output column (i, j), or marks the column
// (count -1) for the redo launch.
template <typename T>
DXI void column_out(const P2GParams<T>& P, const Lanes& L, int j, int i, bool ok, int acc,
                    const ukey* bl, const ukey* br, int bcap, ArenaCursor& cur) {
  const long long c = (long long)j * P.nx + i;
  if (!ok) {
    if (L.lane == 0) {
      P.o_cnt[c] = -1;
      note_max(&P.ctr->max_state, 2 * bcap);
      set_status(&P.ctr->status, ST_OVERFLOW_SLOT);
      atomicAdd(&P.ctr->redo_cols, 1);
    }
    wsync();
    return;
  }
  const long long s = arena_take(L, &P.ctr->arena_top[3], P.blk, cur, acc);
  const bool fits = s + acc <= P.o_cap;
  if (!fits) {
    if (L.lane == 0) set_status(&P.ctr->status, ST_OVERFLOW_ARENA);
  } else {
    for (int q = L.lane; q < acc; q += 32) { P.o_l[s + q] = bl[q]; P.o_r[s + q] = br[q]; }
  }
  if (L.lane == 0) {
    P.o_start[c] = fits ? s : 0;
    P.o_cnt[c] = acc;
    note_max(&P.ctr->max_out, acc);
    add_total(&P.ctr->out_total, acc);
  }
  wsync();
}

// One tile of k_pass2t: columns j0 .. j0 + tc - 1 of y line i (tile = i * tiles_per_line +
// j0 / tc).  smem holds the layout p2t_layout(R, tc, ntab, stage_cap, warps, bcap); the w
// table is at wt (staged or global).
template <typename T>
__device__ __forceinline__ void pass2t_tile(const P2GParams<T>& P, long long tile, int tc, int ntab, int stage_cap,
                     int Q, int M, unsigned char* smem, const float* wt, ArenaCursor& cur) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwb = blockDim.x >> 5;
  const Lanes L{lane, 32};
  const int R = P.R, bcap = P.bcap;
  const P2TLayout Lo = p2t_layout(R, tc, ntab, stage_cap, nwb, bcap);
  int* soff = (int*)(smem + Lo.soff);
  long long* sbase = (long long*)(smem + Lo.sbase);
  float* saf = (float*)(smem + Lo.saf);
  float* sbf = (float*)(smem + Lo.sbf);
  short* sdx = (short*)(smem + Lo.sdx);
  unsigned char* wb = smem + Lo.warps + (long long)warp * Lo.warp_bytes;
  ukey* bl = (ukey*)wb;
  ukey* br = bl + bcap;
  int* f0 = (int*)(br + bcap);
  int* f1 = f0 + bcap;
  int* bcount = f1 + bcap;
  const float E = 9.5367432e-7f * (__uint_as_float(P.ctr->zmax_bits) + P.wtabf[0]);  // 2^-20
  long long* sgb = sbase + tc + 2 * R + 1;  // the tile's first piece in the packed copy
  const int tpl = (P.ny + tc - 1) / tc;
  const int i = (int)(tile / tpl);
  const int j0 = (int)(tile % tpl) * tc;
  const int j1 = min(P.ny, j0 + tc);
  const int s0 = max(0, j0 - R), s1 = min(P.ny, j1 + R);
  const int ns = s1 - s0;
  const long long qb = (long long)i * P.ny;
  __syncthreads();  // the previous tile's readers are done
  PHASE_BEGIN();
  if (warp == 0) {
    int carry = 0;
    for (int base = 0; base < ns; base += 32) {
      const int t = base + lane;
      const int v = t < ns ? P.m_cnt[qb + s0 + t] : 0;
      const int inc = w_incl_add(v, lane);
      if (t < ns) {
        soff[t] = carry + inc - v;
        sbase[t] = P.m_start[qb + s0 + t] - (carry + inc - v);
      }
      carry += w_bcast(inc, 31);
    }
    if (lane == 0) {
      soff[ns] = carry;
      *sgb = P.c_start[qb + s0];
    }
  }
  __syncthreads();
  // runs of columns [ja, jb) whose window [ja - R, jb + R) fits the staging area; columns
  // whose single window does not fit are covered by the warps together, in chunks
  for (int ja = j0; ja < j1;) {
    const int qa = max(0, ja - R) - s0;
    int jb = j1;
    while (jb > ja + 1 && soff[min(P.ny, jb + R) - s0] - soff[qa] > stage_cap) --jb;
    const int qe = min(P.ny, jb + R) - s0;
    const int gofs = soff[qa];
    const int tot = soff[qe] - gofs;
    PHASE_COUNT(12, tot <= stage_cap ? 1 : 0);
    PHASE_COUNT(13, 1);
    if (tot <= stage_cap) {
      const long long src = *sgb + gofs;
      for (int g = threadIdx.x; g < tot; g += blockDim.x) {
        saf[g] = P.c_af[src + g];
        sbf[g] = P.c_bf[src + g];
        sdx[g] = P.c_dx[src + g];
      }
      __syncthreads();
      PHASE(0);
      for (int j = ja + warp; j < jb; j += nwb) {
        const int qlo = max(0, j - R) - s0, qhi = min(P.ny - 1, j + R) - s0;
        int acc = 0;
        const bool ok = column_cover<T>(P, L, j, s0, soff, sbase, qlo, qhi, soff[qlo],
                                        soff[qhi + 1], saf - gofs, sbf - gofs, sdx - gofs, wt,
                                        E, Q, M, bl, br, f0, f1, bcount, bcap, acc);
        PHASE(1);
        column_out<T>(P, L, j, i, ok, acc, bl, br, bcap, cur);
        PHASE(3);
      }
      __syncthreads();  // the run's staged pieces are no longer read
    } else {
      // a single column's window is larger than the staging area: the next nwb columns (one
      // a warp) are covered together, their joint window staged in chunks; each warp takes the
      // part of a chunk inside its column's window and carries its runs across chunks
      jb = min(j1, ja + nwb);
      const int j = ja + warp;
      const bool mine = j < jb;
      const int qlo = mine ? max(0, j - R) - s0 : 0, qhi = mine ? min(P.ny - 1, j + R) - s0 : 0;
      const int gb = mine ? soff[qlo] : 0, ge = mine ? soff[qhi + 1] : 0;
      const int ua = soff[qa], ue = soff[min(P.ny, jb + R) - s0];  // joint window
      int acc = 0;
      bool ok = true;
      for (int ga = ua; ga < ue; ga += stage_cap) {
        const int gz = min(ue, ga + stage_cap);
        const long long src = *sgb + ga;
        for (int g = threadIdx.x; g < gz - ga; g += blockDim.x) {
          saf[g] = P.c_af[src + g];
          sbf[g] = P.c_bf[src + g];
          sdx[g] = P.c_dx[src + g];
        }
        __syncthreads();
        const int ca = max(ga, gb), cz = min(gz, ge);
        if (mine && ok && ca < cz)
          ok = column_cover<T>(P, L, j, s0, soff, sbase, qlo, qhi, ca, cz, saf - ga, sbf - ga,
                               sdx - ga, wt, E, Q, M, bl, br, f0, f1, bcount, bcap, acc);
        __syncthreads();
      }
      if (mine) column_out<T>(P, L, j, i, ok, acc, bl, br, bcap, cur);
      PHASE(1);
    }
    ja = jb;
  }
}

}  // namespace dexel
