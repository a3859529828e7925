// Pass 2 in two steps: per-source level unions, then a per-column gather of those unions.
//
// Output column j of a y line receives from source column j' exactly the union of that
// source's capsule slices at level t = |j - j'| (Sec. 3.3: the part of the line covered by
// the source's seeds and rectangles at that offset).  This union depends on (j', t) only,
// and each (j', t) serves the two output columns j' - t and j' + t.  So:
//
//   k_levels   for every source column and every level t = 0 .. R, the union of its slices,
//              appended as a short list of exact intervals (float-filtered merges, exact
//              ends, as in gather2.cuh).  One lane a level: the lanes of a warp walk the same
//              pieces in height order (broadcast loads), each with its own radius
//              w(dx, t).  Short windows pack several sources into a warp (lane = (source,
//              level)); long ones split the levels into groups of 32 and give level 0 to
//              all 32 lanes, each a range of the pieces.
//   k_lgather  for every output column, the lists (j', |j - j'|) of its window gathered into
//              a bucket, sorted by left end and united exactly.
//
// Every (source, level) union is computed once instead of twice, by a walk without range
// splits or segment bookkeeping.  A list longer than its lane's buffer is walked a second
// time straight into place; a column whose lists outgrow the bucket is gathered again with a
// larger one.
#pragma once
#include "gather2.cuh"

namespace dexel {

// per-lane list buffer in shared memory (intervals)
constexpr int kLvlSlots = 8;
// w-table entries k_levels keeps in shared memory (n <= k^2: radii up to 64 spacings)
constexpr int kLvlTable = 4097;

template <typename T>
struct LvlParams {
  P2GParams<T> P;
  ukey* l_l;  // level-list arena: left keys
  ukey* l_r;  //                   right keys
  long long l_cap;
  long long* l_start;  // [q * L + t]: first interval of source q (line-2 index) at level t
  int* l_cnt;
  int L;     // levels a source: R + 1
  int G;     // sources a warp when L <= 32, else 1
  int NG;    // level groups of 32 (levels 1 .. R) when L > 32, else 0
  long long nsrc;  // source columns (nx * ny)
  long long nlev;  // entries of l_start / l_cnt
  long long m_cap, c_cap;  // entries of the S_mid arena and of its packed copy
};

// One lane's walk over source q's pieces [p0, p1) at level t (tt = t^2), uniting slices into
// one interval at a time; the first cap intervals are stored at bl / br; returns the count.
template <typename T>
DXI int level_walk(const P2GParams<T>& P, long long q, int p0, int p1, int tt, float E,
                   const float* wt, ukey* bl, ukey* br, int cap) {
  const long long cs = P.c_start[q];
  const long long ms = P.m_start[q];
  const short* dxp = P.c_dx + cs;
  const float* afp = P.c_af + cs;
  const float* bfp = P.c_bf + cs;
  int cnt = 0;
  bool have = false;
  float clf = 0.0f, crf = 0.0f;
  int gl = 0, gr = 0, nl = 0, nr = 0;
  auto emit = [&]() {
    if (cnt < cap) {
      bl[cnt] = dkey(keyd(P.m_a[ms + gl]) - P.wtab[nl]);
      br[cnt] = dkey(keyd(P.m_b[ms + gr]) + P.wtab[nr]);
    }
    ++cnt;
  };
  // the next piece is loaded while the current one is merged
  int dxn = 0;
  float afn = 0.0f, bfn = 0.0f;
  if (p0 < p1) { dxn = dxp[p0]; afn = afp[p0]; bfn = bfp[p0]; }
  for (int p = p0; p < p1; ++p) {
    const int dx = dxn;
    const float af = afn, bf = bfn;
    if (p + 1 < p1) { dxn = dxp[p + 1]; afn = afp[p + 1]; bfn = bfp[p + 1]; }
    const int n = dx * dx + tt;
    const bool in = n <= P.nmax;
    const float wf = wt[in ? n : 0];
    const float lf = af - wf;
    const float rf = bf + wf;
    const float dl = lf - clf, dr = rf - crf;
    const bool ov = lf <= crf - E && rf >= clf + E;  // certain overlap
    const bool decided = !(fabsf(dl) < E) && !(fabsf(dr) < E);
    const bool merge = in && have && ov && decided;
    if (in && have && !merge) emit();
    const bool fresh = in && !merge;
    const bool tl = fresh || (merge && dl < 0.0f);
    const bool tr = fresh || (merge && dr > 0.0f);
    clf = tl ? lf : clf;
    gl = tl ? p : gl;
    nl = tl ? n : nl;
    crf = tr ? rf : crf;
    gr = tr ? p : gr;
    nr = tr ? n : nr;
    have = have || in;
  }
  if (have) emit();
  return cnt;
}

// One work item of k_levels (see the file comment): item = a group of G sources (L <= 32)
// or (source, level group).  bl / br: the lane's buffer slots (br = bl + 32 slots).
template <typename T>
__device__ __forceinline__ void levels_item(const LvlParams<T>& A, long long item, int lane,
                                            ukey* bl, ukey* br, float E, const float* wt,
                                            ArenaCursor& cur) {
  const Lanes Ln{lane, 32};
  const P2GParams<T>& P = A.P;
  long long q;
  int t;
  bool act;
  if (A.NG == 0) {
    const int g = lane / A.L;
    q = item * A.G + g;
    t = lane % A.L;
    act = g < A.G && q < A.nsrc;
  } else {
    q = item / A.NG;
    t = 1 + (int)(item % A.NG) * 32 + lane;
    act = t < A.L;
  }
  int cnt = 0, np = 0;
  if (act) {
    np = P.m_cnt[q];
    if (np < 0 || P.m_start[q] < 0 || P.m_start[q] + np > A.m_cap || P.c_start[q] < 0 ||
        P.c_start[q] + np > A.c_cap || q * A.L + t >= A.nlev) {
      set_status(&P.ctr->status, ST_BOUNDS | ST_LEVELS_OVER);
      act = false;
    } else {
      cnt = level_walk<T>(P, q, 0, np, t * t, E, wt, bl, br, kLvlSlots);
    }
  }
  // the lanes' lists, contiguous in the level arena; a list longer than its buffer is
  // walked again straight into place
  {
    const int inc = w_incl_add(cnt, lane);
    const int tot = w_bcast(inc, 31);
    const long long s = arena_take(Ln, &P.ctr->arena_top[2], P.blk, cur, tot);
    if (s + tot > A.l_cap) {
      if (lane == 0) set_status(&P.ctr->status, ST_LEVELS_OVER);
      return;
    }
    const long long o = s + inc - cnt;
    if (cnt <= kLvlSlots) {
      for (int k = 0; k < cnt; ++k) { A.l_l[o + k] = bl[k]; A.l_r[o + k] = br[k]; }
    } else {
      level_walk<T>(P, q, 0, np, t * t, E, wt, A.l_l + o, A.l_r + o, cnt);
    }
    if (act) {
      A.l_start[q * A.L + t] = o;
      A.l_cnt[q * A.L + t] = cnt;
    }
  }
  // level 0 of a long window: all lanes, a range of the pieces each, one list
  if (A.NG != 0 && item % A.NG == 0) {
    const int np0 = P.m_cnt[q];
    if (np0 < 0 || P.m_start[q] < 0 || P.m_start[q] + np0 > A.m_cap || P.c_start[q] < 0 ||
        P.c_start[q] + np0 > A.c_cap) {
      if (lane == 0) set_status(&P.ctr->status, ST_BOUNDS | ST_LEVELS_OVER);
      return;
    }
    const int per = (np0 + 31) >> 5;
    const int p0 = min(np0, lane * per), p1 = min(np0, p0 + per);
    const int cnt0 = level_walk<T>(P, q, p0, p1, 0, E, wt, bl, br, kLvlSlots);
    const int inc = w_incl_add(cnt0, lane);
    const int tot = w_bcast(inc, 31);
    const long long s = arena_take(Ln, &P.ctr->arena_top[2], P.blk, cur, tot);
    if (s + tot > A.l_cap) {
      if (lane == 0) set_status(&P.ctr->status, ST_LEVELS_OVER);
      return;
    }
    const long long o = s + inc - cnt0;
    if (cnt0 <= kLvlSlots) {
      for (int k = 0; k < cnt0; ++k) { A.l_l[o + k] = bl[k]; A.l_r[o + k] = br[k]; }
    } else {
      level_walk<T>(P, q, p0, p1, 0, E, wt, A.l_l + o, A.l_r + o, cnt0);
    }
    if (lane == 0) {
      A.l_start[q * A.L] = s;
      A.l_cnt[q * A.L] = tot;
    }
  }
  wsync();
}

// One output column of k_lgather (item = i * ny + j); wb: the warp's bucket (bcap intervals
// with their union flags).
template <typename T>
__device__ __forceinline__ void lgather_column(const LvlParams<T>& A, long long item, int bcap,
                                               int redo, int lane, unsigned char* wb,
                                               ArenaCursor& cur) {
  const Lanes L{lane, 32};
  const P2GParams<T>& P = A.P;
  ukey* bl = (ukey*)wb;
  ukey* br = bl + bcap;
  int* f0 = (int*)(br + bcap);
  int* f1 = f0 + bcap;
  const int R = P.R;
  // output columns in line order (i, j): consecutive warps share the sources' lists
  const int i = (int)(item / P.ny), j = (int)(item % P.ny);
  const long long c = (long long)j * P.nx + i;
  if (redo && P.o_cnt[c] != -1) return;
  const int s0 = max(0, j - R), s1 = min(P.ny - 1, j + R);
  const long long qb = (long long)i * P.ny;
  int carry = 0;
  for (int base = s0; base <= s1; base += 32) {
    const int jj = base + lane;
    int n = 0;
    long long st = 0;
    if (jj <= s1) {
      const int t = jj > j ? jj - j : j - jj;
      const long long li = (qb + jj) * A.L + t;
      if (li < A.nlev) {
        n = A.l_cnt[li];
        st = A.l_start[li];
      }
      if (li >= A.nlev || n < 0 || st < 0 || st + n > A.l_cap) {
        set_status(&P.ctr->status, ST_BOUNDS | ST_LEVELS_OVER);
        n = 0;
      }
    }
    const int inc = w_incl_add(n, lane);
    const int o = carry + inc - n;
    for (int k = 0; k < n && o + k < bcap; ++k) { bl[o + k] = A.l_l[st + k]; br[o + k] = A.l_r[st + k]; }
    carry += w_bcast(inc, 31);
  }
  wsync();
  const int total = carry;
  if (total > bcap) {
    if (lane == 0) {
      P.o_cnt[c] = -1;
      note_max(&P.ctr->max_state, total);
      set_status(&P.ctr->status, ST_OVERFLOW_SLOT);
      atomicAdd(&P.ctr->redo_cols, 1);
    }
    wsync();
    return;
  }
  const int n2 = pow2_at_least(total);
  wsync();
  if (n2 > 1) {
    for (int t = total + lane; t < n2; t += 32) { bl[t] = ~0ULL; br[t] = ~0ULL; }
    wsync();
    warp_sort_pairs(L, bl, br, n2);
  }
  const int no = total > 0 ? union_count(L, bl, br, total, f0, f1) : 0;
  const long long s = arena_take(L, &P.ctr->arena_top[3], P.blk, cur, no);
  const bool fits = s + no <= P.o_cap;
  if (!fits) {
    if (lane == 0) set_status(&P.ctr->status, ST_OVERFLOW_ARENA);
  } else if (no > 0) {
    union_write(L, bl, br, total, f0, f1, P.o_l + s, P.o_r + s);
  }
  if (lane == 0) {
    P.o_start[c] = fits ? s : 0;
    P.o_cnt[c] = no;
    cur.tally += no;
    cur.tmax = no > cur.tmax ? no : cur.tmax;
  }
  wsync();
}

DXI long long lgather_smem(int warps, int bcap) {
  return (long long)warps * (bcap * (2 * sizeof(ukey) + 2 * sizeof(int)) + 16);
}

}  // namespace dexel
