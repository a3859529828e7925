// Pass 2 in two steps: per-source level unions, then a per-column gather of those unions.
//
// Output column j of a y line receives from source column j' exactly the union of that
// source's capsule slices at level t = |j - j'| (Sec. 3.3: the part of the line covered by
// the source's seeds and rectangles at that offset).  This union depends on (j', t) only,
// and each (j', t) serves the two output columns j' - t and j' + t.  So:
//
//   k_levels   for every source column and every level t = 0 .. R, the union of its slices,
//              appended as a short list of exact intervals (float-filtered merges, exact
//              ends, as in gather2.cuh).  One lane a level: short windows pack several
//              sources into a warp (lane = (source, level)); long ones give a warp one source
//              and 32 levels (the pieces staged in shared memory, broadcast reads), and level
//              0 one lane per source.  Each lane's radius comes from its own column of a
//              table indexed by |dx| (conflict-free shared-memory reads).  The walk records
//              only which pieces set the ends; the exact ends are computed afterwards by all
//              lanes together, so the double arithmetic stays out of the divergent loop.
//   k_lgather  for every output column, the lists (j', |j - j'|) of its window gathered into
//              a bucket and united exactly: by jumps (a run's right end raised by warp
//              reductions until it stops rising), or sorted when the runs are many.
//
// Every (source, level) union is computed once instead of twice, by a walk without range
// splits or segment bookkeeping.  A list longer than its lane's slots is walked a second
// time straight into place; a column whose lists outgrow the bucket is gathered again with a
// larger one.
#pragma once
#include "gather2.cuh"

#define DXD __device__ __forceinline__

namespace dexel {

// per-lane interval slots in shared memory (a slot: the pieces and |dx| of the two ends); a
// list longer than this is walked again straight into place
// list longer than this is walked again straight into place.  The count a launch uses
// (LvlParams::slots) follows the reach: longer windows give longer lists (measured: 2048^2
// k = 64, 16 slots 261 ms, 8 slots 220 ms; 4096^2 k = 128, 16 slots 1541 ms, 8 slots 2110 ms)
constexpr int kLvlSlots = 16;  // the most a launch uses
// Interval slots a lane by reach (a longer list spills to the lane's region in global memory):
// fewer slots leave more of the SM's shared memory to L1 (measured with 64 spilled intervals
// a lane: 2048^2 at k = 64, 4 slots 129 ms, 6 128, 8 138, 10 138; 4096^2 at k = 128, 6 slots
// 1415 ms, 8 1402, 10 1397, 12 1394, 16 1509)
DXI int lvl_slots_for(int R) { return R < 48 ? 8 : (R <= 64 ? 6 : 12); }
// without spill regions (the batched engine): a longer list is walked again, so more slots
// (measured at 2048^2 k = 64: 8 slots 218 ms, 10 200, 12 228, 16 258)
DXI int lvl_slots_nospill(int R) { return R < 48 ? 8 : (R <= 64 ? 10 : 16); }
// pieces a warp stages in shared memory at a time (a level group walks one source)
// pieces staged a chunk, and the unrolling of the walk over them (measured at 2048^2 k = 64:
// stage 128 237 ms against 200 at 64; unroll 1 209, 2 200, 4 195, 8 192, 16 196 ms)
#ifndef DEXEL_LVL_STAGE
#define DEXEL_LVL_STAGE 64
#endif
#ifndef DEXEL_LVL_UNROLL
#define DEXEL_LVL_UNROLL 8
#endif
constexpr int kLvlStage = DEXEL_LVL_STAGE;
constexpr int kLvlUnroll = DEXEL_LVL_UNROLL;
// w-table entries kept in shared memory when the per-lane tables do not fit (n <= k^2:
// radii up to 64 spacings)
constexpr int kLvlTable = 4097;
// shared memory for the per-lane tables (floats): (level groups) x (R + 1) x 32 lanes
constexpr int kLvlLaneTab = 12288;
// a level list's index entry: start << 24 | count (counts below 2^24)
constexpr unsigned long long kLvlIdxMaxCount = (1ULL << 24) - 1;
// piece index and |dx| packed in one word: index < 2^21, |dx| < 2^11
constexpr int kLvlDxBits = 11;
constexpr int kLvlMaxPieces = 1 << (32 - kLvlDxBits);

template <typename T>
struct LvlParams {
  P2GParams<T> P;
  ulonglong2* l_p;  // level-list arena: (left, right) keys of each interval, interleaved
  long long l_cap;
  // index of the lists by output column: entry u of output column q (line order) is the list
  // of source j - R + u at level |u - R| of the same line, packed as start << 24 | count
  // ((2R + 1) entries a column, contiguous: a column's gather reads them coalesced)
  unsigned long long* l_idx;
  int W;     // entries a column, 2R + 1
  int L;     // levels a source: R + 1
  int G;     // sources a warp when L <= 32, else 1
  int NG;    // level groups of 32 (levels 1 .. R) when L > 32, else 0
  int slots;       // per-lane interval slots of the level walks (at most kLvlSlots)
  // intervals a lane writes beyond its slots go to its spill region in global memory (spill:
  // 2 x spill_cap words a lane, lanes of a warp of the grid in order; null: none), so that
  // only a list longer than slots + spill_cap is walked again
  unsigned* spill;
  int spill_cap;
  int yw;          // reach of the output column's window along y (R; 0: the 2D slices, each
                   // column its own level-0 list)
  long long q0;    // first source column of the block (line order q = i * ny + j)
  long long nsrc;  // source columns of the block
  long long nlev;  // bound of the index q * W + u into l_idx
  long long m_cap, c_cap;  // entries of the S_mid arena and of its packed copy
};

// Work items of k_levels: L <= 32, groups of G = 32 / L sources (lane = (source, level));
// L > 32, first the level-0 items (32 sources, lane = source), then (source, level group).
// yw = 0 (the 2D slices): the level-0 items only, one lane a source, at every L.
DXI long long lvl_level0_items(long long nsrc, int L, int yw = -1) {
  return (L <= 32 && yw != 0) ? 0 : (nsrc + 31) / 32;
}
DXI long long lvl_items(long long nsrc, int L, int yw = -1) {
  if (yw == 0) return lvl_level0_items(nsrc, L, yw);
  if (L <= 32) return (nsrc + (32 / L) - 1) / (32 / L);
  return lvl_level0_items(nsrc, L) + nsrc * ((L - 1 + 31) / 32);
}

// entries of the per-lane tables: (level groups) x (R + 1) x 32, then the level-0 row (R + 1)
DXI long long lvl_lane_tab(int R) {
  const int L = R + 1;
  const int ng = L <= 32 ? 1 : (R + 31) / 32;
  return (long long)ng * L * 32 + L;
}

// shared memory of k_levels: per warp the slots (2 x kLvlSlots x 32 words) and the staged
// pieces (kLvlStage float4), then the table
struct LvlLayout {
  long long slots, stage, tab, total;
};
DXI LvlLayout lvl_layout(int warps, int tab_floats, int slots = kLvlSlots) {
  LvlLayout o;
  o.slots = 0;
  o.stage = (long long)warps * 2 * slots * 32 * sizeof(unsigned);
  o.tab = o.stage + (long long)warps * kLvlStage * 16;
  o.total = o.tab + (long long)tab_floats * sizeof(float);
  return o;
}

// The float radius of a piece at |dx| for one lane's level (negative: dx^2 + t^2 > k^2).
// STab: a table indexed by |dx| << sh (the per-lane tables: sh = 5, the lane's column;
// level 0: sh = 0).  FlatTab: w[dx^2 + t^2].
struct STab {
  const float* p;
  int sh;
  DXD float operator()(int adx) const { return p[adx << sh]; }
};
struct FlatTab {
  const float* w;
  int tt;
  int nmax;
  DXD float operator()(int adx) const {
    const int n = adx * adx + tt;
    return n <= nmax ? w[n] : -1.0f;
  }
};

// State of one lane's walk: the open interval (float ends) and the pieces that set its ends
// (piece index << kLvlDxBits | |dx|).
struct LvlRun {
  float clf, crf;
  unsigned pl, pr;
  bool have;
  int cnt;  // intervals closed so far
};
DXD LvlRun lvl_run() { return LvlRun{0.0f, 0.0f, 0u, 0u, false, 0}; }
DXD unsigned lvl_pack(int p, int adx) { return ((unsigned)p << kLvlDxBits) | (unsigned)adx; }

// One step of a level walk (Sec. 3.3: the slice [a - w, b + w] of piece p at this lane's
// level): merged into the open interval when the overlap is certain under the float error
// bound E, else the open interval is closed (emit) and the slice opens the next one.
template <typename Emit>
DXD void lvl_step(LvlRun& s, float af, float bf, unsigned pk, float wf, float E,
                  const Emit& emit) {
  const bool in = wf >= 0.0f;
  const float lf = af - wf;
  const float rf = bf + wf;
  const float dl = lf - s.clf, dr = rf - s.crf;
  const bool ov = lf <= s.crf - E && rf >= s.clf + E;  // certain overlap
  const bool decided = !(fabsf(dl) < E) && !(fabsf(dr) < E);
  const bool merge = in && s.have && ov && decided;
  if (in && s.have && !merge) {
    emit(s);
    ++s.cnt;
  }
  const bool fresh = in && !merge;
  const bool tl = fresh || (merge && dl < 0.0f);
  const bool tr = fresh || (merge && dr > 0.0f);
  s.clf = tl ? lf : s.clf;
  s.pl = tl ? pk : s.pl;
  s.crf = tr ? rf : s.crf;
  s.pr = tr ? pk : s.pr;
  s.have = s.have || in;
}
template <typename Emit>
DXD void lvl_close(LvlRun& s, const Emit& emit) {
  if (s.have) {
    emit(s);
    ++s.cnt;
  }
}

// emit into the lane's slots (the first cap intervals): slot k of lane x at ws[k * 32 + x],
// its right end kLvlSlots * 32 words further
struct PackEmit {
  unsigned* sl;  // ws + lane
  int slots;
  unsigned* sp;  // the lane's spill region (2 words an interval), or null
  int scap;      // its intervals
  DXD void operator()(const LvlRun& s) const {
    if (s.cnt < slots) {
      sl[s.cnt << 5] = s.pl;
      sl[(s.cnt << 5) + slots * 32] = s.pr;
    } else if (s.cnt - slots < scap) {
      sp[2 * (s.cnt - slots)] = s.pl;
      sp[2 * (s.cnt - slots) + 1] = s.pr;
    }
  }
};
// the spill region of lane `lane` of the grid's warp gw (null without one)
template <typename T>
DXD unsigned* lvl_spill(const LvlParams<T>& A, long long gw, int lane) {
  return A.spill ? A.spill + (gw * 32 + lane) * 2LL * A.spill_cap : nullptr;
}

// the exact ends: a - w(dx^2 + t^2) and b + w(dx^2 + t^2) in double
template <typename T>
DXD ukey lvl_left(const P2GParams<T>& P, long long ms, int p, int adx, int tt) {
  return dkey(keyd(P.m_a[ms + p]) - P.wtab[adx * adx + tt]);
}
template <typename T>
DXD ukey lvl_right(const P2GParams<T>& P, long long ms, int p, int adx, int tt) {
  return dkey(keyd(P.m_b[ms + p]) + P.wtab[adx * adx + tt]);
}

// emit exact ends straight into the level arena (a list longer than the slots)
template <typename T>
struct ExactEmit {
  const P2GParams<T>* P;
  long long ms;
  int tt;
  ulonglong2* o;
  DXD void operator()(const LvlRun& s) const {
    const unsigned m = (1u << kLvlDxBits) - 1;
    o[s.cnt] = make_ulonglong2(lvl_left<T>(*P, ms, (int)(s.pl >> kLvlDxBits), (int)(s.pl & m), tt),
                               lvl_right<T>(*P, ms, (int)(s.pr >> kLvlDxBits), (int)(s.pr & m), tt));
  }
};

// The pieces of one source as the walks read them: float ends and dx.  PackSrc: the packed
// float copy; ExactSrc: S_mid itself, each end rounded to float (by truncation, within the
// filter's error bound) as it is read.
struct PackSrc {
  const float* a;
  const float* b;
  const short* d;
  DXD float af(int p) const { return a[p]; }
  DXD float bf(int p) const { return b[p]; }
  DXD int dx(int p) const { return d[p]; }
};
template <typename Key>
struct ExactSrc {
  const Key* a;
  const Key* b;
  const short* d;
  DXD float af(int p) const { return keyf(a[p]); }
  DXD float bf(int p) const { return keyf(b[p]); }
  DXD int dx(int p) const { return d[p]; }
};

// A lane's walk over pieces [p0, p1) of one source (the next piece is loaded while the
// current one is merged).
template <typename T, typename W, typename Emit, typename Src>
DXD void walk_global(const P2GParams<T>& P, const Src& src, int p0, int p1, float E, const W& wl,
                     LvlRun& s, const Emit& emit) {
  int dxn = 0;
  float afn = 0.0f, bfn = 0.0f;
  if (p0 < p1) { dxn = src.dx(p0); afn = src.af(p0); bfn = src.bf(p0); }
  for (int p = p0; p < p1; ++p) {
    const int adx = min(dxn < 0 ? -dxn : dxn, P.R);  // labels lie in [-R, R]
    const float af = afn, bf = bfn;
    if (p + 1 < p1) { dxn = src.dx(p + 1); afn = src.af(p + 1); bfn = src.bf(p + 1); }
    lvl_step(s, af, bf, lvl_pack(p, adx), wl(adx), E, emit);
  }
  lvl_close(s, emit);
}

// The warp's walk over the np pieces of one source (all lanes, each its own level): the
// pieces pass through shared memory in chunks (coalesced loads, broadcast reads).  (Staging
// only the pieces that reach a level group's first level was measured slower: 269 -> 281 ms
// on the 2048^2 k = 64 workload.)
template <typename T, typename W, typename Emit, typename Src>
DXD void walk_staged(const P2GParams<T>& P, const Src& src, int np, int lane, float4* stg, float E,
                     const W& wl, LvlRun& s, const Emit& emit) {
  for (int base = 0; base < np; base += kLvlStage) {
    const int m = min(kLvlStage, np - base);
    wsync();
    for (int k = lane; k < m; k += 32) {
      const int dx = src.dx(base + k);
      const int adx = min(dx < 0 ? -dx : dx, P.R);  // labels lie in [-R, R]
      stg[k] = make_float4(src.af(base + k), src.bf(base + k), __int_as_float(adx),
                           __uint_as_float(lvl_pack(base + k, adx)));
    }
    wsync();
#pragma unroll kLvlUnroll
    for (int k = 0; k < m; ++k) {
      const float4 v = stg[k];
      lvl_step(s, v.x, v.y, __float_as_uint(v.w), wl(__float_as_int(v.z)), E, emit);
    }
  }
  lvl_close(s, emit);
  wsync();
}

// The lanes' lists (cnt each, in the slots; lane x's at level t of source q) into the level
// arena, contiguous per warp: the exact ends are computed by all lanes together, a list
// longer than the slots is walked again by its lane straight into place (redo).  Returns
// false when the arena is full (status set).
template <typename T, typename Redo>
DXD bool lvl_flush(const LvlParams<T>& A, int lane, const unsigned* ws, const unsigned* sp0,
                   int cnt, bool act, long long q, int t, long long ms, ArenaCursor& cur,
                   const Redo& redo) {
  // sp0: the spill region of the warp's lane 0 (null: none); a lane holds slots + scap
  const int scap = sp0 ? A.spill_cap : 0;
  const int held = A.slots + scap;
  const Lanes Ln{lane, 32};
  const P2GParams<T>& P = A.P;
  const int inc = w_incl_add(cnt, lane);
  const int tot = w_bcast(inc, 31);
  const long long s = arena_take(Ln, &P.ctr->arena_top[2], P.blk, cur, tot);
  if (s + tot > A.l_cap) {
    if (lane == 0) set_status(&P.ctr->status, ST_LEVELS_OVER);
    return false;
  }
  const int ex = inc - cnt;
  const int tt = t * t;
  wsync();
  for (int b = 0; b < tot; b += 32) {
    const int idx = b + lane;
    int own = 0;  // the lane whose list holds entry idx: lanes with inc <= idx
#pragma unroll
    for (int st = 16; st > 0; st >>= 1) {
      const int v = __shfl_sync(0xffffffffu, inc, own + st - 1);
      own += v <= idx ? st : 0;
    }
    const int exo = __shfl_sync(0xffffffffu, ex, own);
    const int cno = __shfl_sync(0xffffffffu, cnt, own);
    const int tto = __shfl_sync(0xffffffffu, tt, own);
    const long long mso = __shfl_sync(0xffffffffu, ms, own);
    if (idx < tot && cno <= held) {
      const int k = idx - exo;
      unsigned pl, pr;
      if (k < A.slots) {
        pl = ws[(k << 5) + own];
        pr = ws[(k << 5) + own + A.slots * 32];
      } else {  // (written by lane own before the warp synchronised)
        const unsigned* so = sp0 + (long long)own * 2 * scap + 2 * (k - A.slots);
        pl = so[0];
        pr = so[1];
      }
      const unsigned m = (1u << kLvlDxBits) - 1;
      A.l_p[s + idx] = make_ulonglong2(lvl_left<T>(P, mso, (int)(pl >> kLvlDxBits), (int)(pl & m), tto),
                                       lvl_right<T>(P, mso, (int)(pr >> kLvlDxBits), (int)(pr & m), tto));
    }
  }
  {
    const unsigned long_lists = __ballot_sync(0xffffffffu, cnt > held);
    if (long_lists && lane == 0) atomicAdd(&P.ctr->lvl_redo, (unsigned long long)__popc(long_lists));
  }
  if (cnt > held) redo(A.l_p + s + ex);
  if (act) {
    // the list serves output columns j +- t of its line: entry R - t of column j + t and entry
    // R + t of column j - t
    if (cnt > kLvlIdxMaxCount) set_status(&P.ctr->status, ST_LEVELS_OVER);  // beyond the packing
    const unsigned long long e = ((unsigned long long)(s + ex) << 24) | (unsigned long long)(cnt & kLvlIdxMaxCount);
    const int jj = (int)(q % P.ny);
    const long long qb = q - jj;
    if (jj + t < P.ny) A.l_idx[(qb + jj + t) * A.W + (P.R - t)] = e;
    if (t > 0 && jj - t >= 0) A.l_idx[(qb + jj - t) * A.W + (P.R + t)] = e;
  }
  wsync();
  return true;
}

// the bounds of source q's pieces (self-check against the arenas)
template <typename T, bool EXACT>
DXD bool lvl_src_ok(const LvlParams<T>& A, long long q, int np) {
  const P2GParams<T>& P = A.P;
  const bool m_ok = np >= 0 && np < kLvlMaxPieces && P.m_start[q] >= 0 && P.m_start[q] + np <= A.m_cap;
  if (EXACT) return m_ok;
  return m_ok && P.c_start[q] >= 0 && P.c_start[q] + np <= A.c_cap;
}

// the pieces of source q (m_start ms, packed copy at cs)
template <typename T, bool EXACT>
DXD auto lvl_src(const P2GParams<T>& P, long long ms, long long cs) {
  if constexpr (EXACT)
    return ExactSrc<typename H<T>::K>{P.m_a + ms, P.m_b + ms, P.m_l + ms};
  else
    return PackSrc{P.c_af + cs, P.c_bf + cs, P.c_dx + cs};
}

// Table modes of a level walk: the flat float table w[dx^2 + t^2] (global or shared), the
// block's per-lane tables (lvl_tables), or the warp's own per-lane table built per item
// ((R + 1) x 32 floats: lane x's radius at |dx| at tab[|dx| * 32 + x]).
constexpr int kTabFlat = 0, kTabBlock = 1, kTabWarp = 2;

// the warp's own table for this item: lane's level t (act false: no level)
DXD void lvl_warp_table(float* tab, int R, int nmax, const float* wtabf, int lane, int t,
                        bool act) {
  __syncwarp();  // the previous item no longer reads it
  for (int adx = 0; adx <= R; ++adx) {
    const int n = adx * adx + t * t;
    tab[(adx << 5) + lane] = act && n <= nmax ? wtabf[n] : -1.0f;
  }
  __syncwarp();
}

// One work item of k_levels.  TABM: the table mode; tab: the block's tables (kTabBlock), the
// flat table (kTabFlat) or the warp's table space (kTabWarp).  EXACT: the walks read S_mid
// itself (no packed copy).
template <typename T, int TABM, bool EXACT = false>
DXD void levels_item(const LvlParams<T>& A, long long item, int lane, unsigned* ws, float4* stg,
                     float E, float* tab, ArenaCursor& cur, long long gw = -1) {
  // gw: the warp's index in the grid (its spill regions; -1: none)
  unsigned* const sp0 = gw >= 0 ? lvl_spill(A, gw, 0) : nullptr;
  unsigned* const spl = sp0 ? sp0 + (long long)lane * 2 * A.spill_cap : nullptr;
  const int scap = sp0 ? A.spill_cap : 0;
  const P2GParams<T>& P = A.P;
  const int R1 = P.R + 1;
  const long long n0 = lvl_level0_items(A.nsrc, A.L, A.yw);
  const bool pairs = A.NG == 0 && A.yw != 0;  // lane = (source, level)
  if (pairs || item < n0) {
    // lane = (source, level): a walk of its own
    long long q;
    int t;
    bool act;
    if (pairs) {
      const int g = lane / A.L;
      q = item * A.G + g;
      t = lane % A.L;
      act = g < A.G && q < A.nsrc;
    } else {
      q = item * 32 + lane;
      t = 0;
      act = q < A.nsrc;
    }
    q += A.q0;
    int np = 0;
    long long ms = 0, cs = 0;
    if (act) {
      np = P.m_cnt[q];
      if (!lvl_src_ok<T, EXACT>(A, q, np) || q < A.q0 || q >= A.q0 + A.nsrc) {
        set_status(&P.ctr->status, ST_BOUNDS | ST_LEVELS_OVER);
        act = false;
        np = 0;
      } else {
        ms = P.m_start[q];
        cs = EXACT ? 0 : P.c_start[q];
      }
    }
    const auto src = lvl_src<T, EXACT>(P, ms, cs);
    LvlRun s = lvl_run();
    const PackEmit pe{ws + lane, A.slots, spl, scap};
    PHASE_BEGIN();
    if (TABM != kTabFlat) {
      STab wl;
      if (TABM == kTabWarp) {
        lvl_warp_table(tab, P.R, P.nmax, P.wtabf, lane, t, act);
        wl = STab{tab + lane, 5};
      } else {
        wl = pairs ? STab{tab + lane, 5} : STab{tab + (long long)max(A.NG, 1) * R1 * 32, 0};
      }
      walk_global<T>(P, src, 0, np, E, wl, s, pe);
      lvl_flush(A, lane, ws, sp0, s.cnt, act, q, t, ms, cur, [&](ulonglong2* ol) {
        LvlRun s2 = lvl_run();
        walk_global<T>(P, src, 0, np, E, wl, s2, ExactEmit<T>{&P, ms, t * t, ol});
      });
      PHASE(8);
    } else {
      const FlatTab wl{tab, t * t, P.nmax};
      walk_global<T>(P, src, 0, np, E, wl, s, pe);
      lvl_flush(A, lane, ws, sp0, s.cnt, act, q, t, ms, cur, [&](ulonglong2* ol) {
        LvlRun s2 = lvl_run();
        walk_global<T>(P, src, 0, np, E, wl, s2, ExactEmit<T>{&P, ms, t * t, ol});
      });
    }
    return;
  }
  // (source, level group): the warp walks one source, lane = level
  const long long it = item - n0;
  const long long q = A.q0 + it / A.NG;
  const int grp = (int)(it % A.NG);
  const int t = 1 + grp * 32 + lane;
  const bool act = t < A.L;
  const int np = P.m_cnt[q];
  if (!lvl_src_ok<T, EXACT>(A, q, np) || q < A.q0 || q >= A.q0 + A.nsrc) {
    if (lane == 0) set_status(&P.ctr->status, ST_BOUNDS | ST_LEVELS_OVER);
    return;
  }
  const long long ms = P.m_start[q], cs = EXACT ? 0 : P.c_start[q];
  const auto src = lvl_src<T, EXACT>(P, ms, cs);
  LvlRun s = lvl_run();
  const PackEmit pe{ws + lane, A.slots, spl, scap};
  if (TABM != kTabFlat) {
    PHASE_BEGIN();
    STab wl;
    if (TABM == kTabWarp) {
      lvl_warp_table(tab, P.R, P.nmax, P.wtabf, lane, t, act);
      wl = STab{tab + lane, 5};
    } else {
      wl = STab{tab + (long long)grp * R1 * 32 + lane, 5};
    }
    walk_staged<T>(P, src, np, lane, stg, E, wl, s, pe);
    PHASE(6);
#if defined(DEXEL_PHASES) && defined(__CUDA_ARCH__)
    const unsigned ph_cnt = __reduce_add_sync(0xffffffffu, (unsigned)s.cnt);  // (all lanes)
    PHASE_COUNT(12, ph_cnt);
#endif
    PHASE_COUNT(13, np);
    lvl_flush(A, lane, ws, sp0, s.cnt, act, q, t, ms, cur, [&](ulonglong2* ol) {
      LvlRun s2 = lvl_run();
      walk_global<T>(P, src, 0, np, E, wl, s2, ExactEmit<T>{&P, ms, t * t, ol});
    });
    PHASE(7);
  } else {
    const FlatTab wl{tab, t * t, P.nmax};
    walk_staged<T>(P, src, np, lane, stg, E, wl, s, pe);
    lvl_flush(A, lane, ws, sp0, s.cnt, act, q, t, ms, cur, [&](ulonglong2* ol) {
      LvlRun s2 = lvl_run();
      walk_global<T>(P, src, 0, np, E, wl, s2, ExactEmit<T>{&P, ms, t * t, ol});
    });
  }
}

// The tables of k_levels in shared memory.  LTAB: for every level group, |dx| and lane the
// lane's float radius (or -1), then the level-0 row w[dx^2]; else the flat float table when
// it fits (returns the table the walks read).
template <bool LTAB>
__device__ __forceinline__ const float* lvl_tables(float* tab, int R, int L, int G, int NG,
                                                   int nmax, const float* wtabf) {
  const int R1 = R + 1;
  if (LTAB) {
    const int ng = NG == 0 ? 1 : NG;
    const int ne = ng * R1 * 32;
    for (int e = threadIdx.x; e < ne + R1; e += blockDim.x) {
      float v;
      if (e < ne) {
        const int ln = e & 31, adx = (e >> 5) % R1, grp = (e >> 5) / R1;
        int t;
        bool ok;
        if (NG == 0) {
          ok = ln < G * L;
          t = ln % L;
        } else {
          t = 1 + grp * 32 + ln;
          ok = t < L;
        }
        const int n = adx * adx + t * t;
        v = ok && n <= nmax ? wtabf[n] : -1.0f;
      } else {
        const int adx = e - ne;
        v = wtabf[adx * adx];
      }
      tab[e] = v;
    }
    return tab;
  }
  if (nmax + 1 <= kLvlTable) {
    for (int n = threadIdx.x; n <= nmax; n += blockDim.x) tab[n] = wtabf[n];
    return tab;
  }
  return wtabf;
}

// Union of a column's bucket by jumps (the union of closed intervals, Sec. 3.3): a run starts
// at the least left end not yet covered, and its right end is raised to the largest right
// end among the intervals that start at or below it until it no longer rises (touching
// intervals join).  Each pass reads the bucket once and ends in warp reductions; run r is
// kept by lane r.  Returns the run count, or -1 after kJumpPasses passes or 32 runs (the
// caller then sorts the bucket).
constexpr int kJumpPasses = 24;

__device__ __forceinline__ ukey wmax_u64(ukey v) {
  const unsigned h = __reduce_max_sync(0xffffffffu, (unsigned)(v >> 32));
  const unsigned l = __reduce_max_sync(0xffffffffu, (unsigned)(v >> 32) == h ? (unsigned)v : 0u);
  return ((ukey)h << 32) | l;
}
__device__ __forceinline__ ukey wmin_u64(ukey v) {
  const unsigned h = __reduce_min_sync(0xffffffffu, (unsigned)(v >> 32));
  const unsigned l = __reduce_min_sync(0xffffffffu, (unsigned)(v >> 32) == h ? (unsigned)v : ~0u);
  return ((ukey)h << 32) | l;
}

// visit(f) calls f(l, pointer to r) for each interval this lane reads
template <typename Visit>
__device__ __forceinline__ int jump_union(const Visit& visit, int lane, ukey& run_l, ukey& run_r) {
  ukey mn = ~0ULL;
  visit([&](ukey l, const ukey*) { mn = l < mn ? l : mn; });
  ukey lo = wmin_u64(mn), hi = lo;
  int runs = 0;
  for (int pass = 0; pass < kJumpPasses; ++pass) {
    ukey mx = 0, nxt = ~0ULL;
    bool more = false;
    visit([&](ukey l, const ukey* rp) {
      if (l <= hi) {
        const ukey r = *rp;
        mx = r > mx ? r : mx;
      } else {
        nxt = l < nxt ? l : nxt;
        more = true;
      }
    });
    mx = wmax_u64(mx);
    if (mx > hi) {
      hi = mx;
      continue;
    }
    if (lane == runs) {
      run_l = lo;
      run_r = hi;
    }
    ++runs;
    if (!__any_sync(0xffffffffu, more)) return runs;
    if (runs == 32) return -1;
    lo = hi = wmin_u64(nxt);
  }
  return -1;
}

// buckets up to this size are sorted (one register a lane), larger ones united by jumps
constexpr int kJumpMin = 32;

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
  const int s0 = max(0, j - A.yw), s1 = min(P.ny - 1, j + A.yw);
  const long long qb = (long long)i * P.ny;
  // the window's lists into the bucket, 32 sources at a time; lists that do not fit wait, the
  // bucket is united into its runs (by jumps; the runs stay as its first entries) and they go
  // in after them
  int carry = 0;
  bool failed = false, collapsed = false;
  int need = 0;   // the window's entries before a collapse (sizes the next calls' bucket)
  int fneed = 0;  // a bucket that would have held the list that did not fit (the redo's)
  for (int base = s0; base <= s1 && !failed; base += 32) {
    const int jj = base + lane;
    int n = 0;
    long long st = 0;
    if (jj <= s1) {
      const long long li = (qb + j) * A.W + (jj - j + P.R);  // coalesced over the lanes
      if (li < A.nlev) {
        const unsigned long long e = A.l_idx[li];
        n = (int)(e & kLvlIdxMaxCount);
        st = (long long)(e >> 24);
      }
      if (li >= A.nlev || n < 0 || st < 0 || st + n > A.l_cap) {
        set_status(&P.ctr->status, ST_BOUNDS | ST_LEVELS_OVER);
        n = 0;
      }
    }
    bool pending = n > 0;
    while (__any_sync(0xffffffffu, pending)) {
      // the pending lists in lane order; those that fit after the bucket's entries go in
      const int inc = w_incl_add(pending ? n : 0, lane);
      bool fit = pending && carry + inc <= bcap;
      if (!__any_sync(0xffffffffu, fit)) {
        need = max(need, carry + w_bcast(inc, 31));
        int nr = -1;
        ukey rl = 0, rr = 0;
        if (carry > 0) {
          const int cur_n = carry;
          nr = jump_union(
              [&](auto f) {
                for (int t = lane; t < cur_n; t += 32) f(bl[t], br + t);
              },
              lane, rl, rr);
        }
        if (nr >= 0) {
          wsync();  // the bucket is read
          if (lane < nr) {
            bl[lane] = rl;
            br[lane] = rr;
          }
          wsync();
        } else if (carry > 0) {
          // more runs than the jumps keep (or a long chain): the bucket sorted and united in
          // place
          const int n2 = pow2_at_least(carry);
          for (int t = carry + lane; t < n2; t += 32) { bl[t] = ~0ULL; br[t] = ~0ULL; }
          wsync();
          warp_sort_pairs(L, bl, br, n2);
          nr = union_count(L, bl, br, carry, f0, f1);
          union_write_inplace(L, bl, br, carry, f0, f1);
        } else {  // one list longer than the bucket
          fneed = __reduce_max_sync(0xffffffffu, pending ? n : 0) + 32;
          failed = true;
          break;
        }
        carry = nr;
        collapsed = true;
        fit = pending && carry + inc <= bcap;
        if (!__any_sync(0xffffffffu, fit)) {  // a list longer than the bucket's room
          fneed = carry + __reduce_max_sync(0xffffffffu, pending ? n : 0);
          failed = true;
          break;
        }
      }
      if (fit) {
        const int o = carry + inc - n;
#pragma unroll 4
        for (int k = 0; k < n; ++k) {
          const ulonglong2 v = A.l_p[st + k];  // one 16-byte load an interval
          bl[o + k] = v.x;
          br[o + k] = v.y;
        }
      }
      carry += __reduce_max_sync(0xffffffffu, fit ? inc : 0);
      pending = pending && !fit;
    }
  }
  wsync();
  if (failed) {
    // more runs than a collapse keeps, or a list beyond the bucket: handed on (the redo takes
    // a bucket at least twice as large)
    if (lane == 0) {
      P.o_cnt[c] = -1;
      note_max(&P.ctr->max_state, max(fneed, 2 * bcap));
      set_status(&P.ctr->status, ST_OVERFLOW_SLOT);
      atomicAdd(&P.ctr->redo_cols, 1);
    }
    wsync();
    return;
  }
  if (collapsed && lane == 0) {  // the host sizes the next call's bucket by these
    atomicAdd(&P.ctr->over_cols, 1);
    note_max(&P.ctr->over_max, need);
  }
  const int total = carry;
  ukey run_l = 0, run_r = 0;
  int nj = -1;
  if (total > kJumpMin) {
    nj = jump_union(
        [&](auto f) {
          for (int t = lane; t < total; t += 32) f(bl[t], br + t);
        },
        lane, run_l, run_r);
  } else if (total == 0) {
    nj = 0;
  }
  // the runs found by jumps; else (a small bucket, many runs, a long chain of overlaps) the
  // bucket sorted and united
  if (nj >= 0) {
    const long long s = arena_take(L, &P.ctr->arena_top[3], P.blk, cur, nj);
    const bool fits = s + nj <= P.o_cap;
    if (!fits) {
      if (lane == 0) set_status(&P.ctr->status, ST_OVERFLOW_ARENA);
    } else if (lane < nj) {
      P.o_l[s + lane] = run_l;
      P.o_r[s + lane] = run_r;
    }
    if (lane == 0) {
      P.o_start[c] = fits ? s : 0;
      P.o_cnt[c] = nj;
      cur.tally += nj;
      cur.tmax = nj > cur.tmax ? nj : cur.tmax;
    }
    wsync();
    return;
  }
  const int n2 = pow2_at_least(total);
  if (n2 > 1) {
    for (int t = total + lane; t < n2; t += 32) { bl[t] = ~0ULL; br[t] = ~0ULL; }
    wsync();
    warp_sort_pairs(L, bl, br, n2);
  }
  const int no = union_count(L, bl, br, total, f0, f1);
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

// One output column a lane (short windows): the window's lists united by jumps straight from
// global memory, no bucket and no sort.  A column with more than kLaneRuns runs, or whose runs
// need more than kLanePasses passes, is marked (o_cnt = -1, with its interval count as the
// bucket it needs) for the warp-per-column gather.  Call with all 32 lanes; act false: a lane
// without a column.
constexpr int kLaneRuns = 32;   // a lane's runs (local memory)
constexpr int kLanePasses = 64;

template <typename T>
DXD void lgather_lane(const LvlParams<T>& A, long long item, bool act, int lane, ArenaCursor& cur) {
  const Lanes L{lane, 32};
  const P2GParams<T>& P = A.P;
  const int R = P.R;
  int i = 0, j = 0, s0 = 0, s1 = -1;
  long long c = 0, qb = 0;
  if (act) {
    i = (int)(item / P.ny);
    j = (int)(item % P.ny);
    c = (long long)j * P.nx + i;
    s0 = max(0, j - A.yw);
    s1 = min(P.ny - 1, j + A.yw);
    qb = (long long)i * P.ny;
  }
  // f(l, pointer to r) over the column's intervals
  auto visit = [&](auto f) {
    for (int jj = s0; jj <= s1; ++jj) {
      const long long li = (qb + j) * A.W + (jj - j + R);  // the column's entries, in order
      if (li >= A.nlev) continue;
      const unsigned long long e = A.l_idx[li];
      const int n = (int)(e & kLvlIdxMaxCount);
      const long long st = (long long)(e >> 24);
      if (n < 0 || st < 0 || st + n > A.l_cap) {
        set_status(&P.ctr->status, ST_BOUNDS | ST_LEVELS_OVER);
        continue;
      }
      for (int k = 0; k < n; ++k) f(A.l_p[st + k].x, &A.l_p[st + k].y);
    }
  };
  ukey rl[kLaneRuns], rr[kLaneRuns];
  int nr = 0, total = 0;
  bool ok = true;
  if (act) {
    ukey lo = ~0ULL;
    visit([&](ukey l, const ukey*) {
      lo = l < lo ? l : lo;
      ++total;
    });
    ukey hi = lo;
    bool more = total > 0;
    for (int pass = 0; more && pass < kLanePasses; ++pass) {
      ukey mx = 0, nxt = ~0ULL;
      bool later = false;
      visit([&](ukey l, const ukey* rp) {
        if (l <= hi) {
          const ukey r = *rp;
          mx = r > mx ? r : mx;
        } else {
          nxt = l < nxt ? l : nxt;
          later = true;
        }
      });
      if (mx > hi) {
        hi = mx;
        continue;
      }
      rl[nr] = lo;
      rr[nr] = hi;
      ++nr;
      more = later;
      if (more && nr == kLaneRuns) break;
      lo = hi = nxt;
    }
    ok = !more;
  }
  const bool mark = act && !ok;
  const int n = act && ok ? nr : 0;
  const int inc = w_incl_add(n, lane);
  const int tot = w_bcast(inc, 31);
  const long long s = arena_take(L, &P.ctr->arena_top[3], P.blk, cur, tot);
  const bool fits = s + tot <= P.o_cap;
  if (act) {
    if (mark) {
      P.o_cnt[c] = -1;
      note_max(&P.ctr->max_state, total);
      set_status(&P.ctr->status, ST_OVERFLOW_SLOT);
      atomicAdd(&P.ctr->redo_cols, 1);
    } else {
      const long long o = s + inc - n;
      if (fits) {
        for (int q = 0; q < n; ++q) { P.o_l[o + q] = rl[q]; P.o_r[o + q] = rr[q]; }
      }
      P.o_start[c] = fits ? o : 0;
      P.o_cnt[c] = n;
    }
  }
  if (lane == 0 && !fits) set_status(&P.ctr->status, ST_OVERFLOW_ARENA);
  const int mx = __reduce_max_sync(0xffffffffu, n);
  if (lane == 0) {
    cur.tally += tot;
    cur.tmax = mx > cur.tmax ? mx : cur.tmax;
  }
}

DXI long long lgather_smem(int warps, int bcap) {
  return (long long)warps * (bcap * (2 * sizeof(ukey) + 2 * sizeof(int)) + 16);
}

}  // namespace dexel
