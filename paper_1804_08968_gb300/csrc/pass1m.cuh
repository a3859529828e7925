// Pass 1 of the dexel offset (Sec. 3.3, the extrusion along x) for short reaches: one lane a
// column, merging its own window's sources.
//
// The partition and its per-height rule are those of pass1l.cuh (runs of equal nearest-source
// label and the points where a nearer source only touches).  For a reach R the window of a
// column holds 2R + 1 sources; a tile-wide sorted event list would give a lane mostly events
// of other lanes' windows (5 of 36 sources at R = 2).  Here a lane keeps the next event of
// each of its sources (in registers) and takes the lowest one at each step: a (2R + 1)-way
// merge of lists that are already sorted (a column's segments, or their complement's), so no
// sort, no shared memory and no barriers.  A first walk counts the pieces, a second writes
// them to the column's place in the S_mid arena.
#pragma once
#include "pass1l.cuh"

namespace dexel {

// The events of one source column in height order: its segments' ends, or (complement) the
// ends of the complement's closure, zero-length segments leaving no gap.
template <typename T>
struct SrcEvents {
  int g, g1;    // next segment, end
  int half;     // dilation: 0 = a of segment g next, 1 = b; erosion: 0 = -inf, 1 = a, 2 = b, 3 = +inf, 4 = done
  ukey key;     // the next event's key (~0 when done)
};

template <typename T>
DXD void src_next(const T* z, bool erode, SrcEvents<T>& e) {
  if (!erode) {
    if (e.half == 0) {
      e.key = event_key(z[2LL * e.g + 1]);
      e.half = 1;
    } else {
      ++e.g;
      e.half = 0;
      e.key = e.g < e.g1 ? event_key(z[2LL * e.g]) : ~0ULL;
    }
    return;
  }
  // erosion: after -inf or a b, the next non-degenerate segment's a (or +inf); after an a,
  // its b
  if (e.half == 1) {
    e.key = event_key(z[2LL * e.g + 1]);
    e.half = 2;
    ++e.g;
    return;
  }
  if (e.half == 0 || e.half == 2) {
    while (e.g < e.g1 && z[2LL * e.g] == z[2LL * e.g + 1]) ++e.g;  // zero length: no gap
    if (e.g < e.g1) {
      e.key = event_key(z[2LL * e.g]);
      e.half = 1;
    } else {
      e.key = KEY_PINF;
      e.half = 3;
    }
    return;
  }
  e.key = ~0ULL;
  e.half = 4;
}

template <typename T>
DXD void src_first(const T* z, bool erode, int g0, int g1, SrcEvents<T>& e) {
  e.g = g0;
  e.g1 = g1;
  if (!erode) {
    e.half = 0;
    e.key = g0 < g1 ? event_key(z[2LL * g0]) : ~0ULL;
  } else {
    e.half = 0;
    e.key = KEY_NINF;
  }
}

// One lane's merge walk for column i of row j (NS >= 2R + 1 slots; slot q: source i - R + q).
template <typename T, int NS, bool WRITE>
DXD int merge_walk(const P1Params<T>& P, int i, int j, bool act, typename H<T>::K* oa,
                   typename H<T>::K* ob, short* ol) {
  typedef typename H<T>::K Key;
  const int R = P.K;
  const long long rb = (long long)j * P.nx;
  SrcEvents<T> e[NS];
#pragma unroll
  for (int q = 0; q < NS; ++q) {
    const int s = i - R + q;
    if (act && q <= 2 * R && s >= 0 && s < P.nx) {
      src_first<T>(P.z, P.erode != 0, P.col_off[rb + s], P.col_off[rb + s + 1], e[q]);
    } else {
      e[q].key = ~0ULL;
      e[q].half = 4;
      e[q].g = e[q].g1 = 0;
    }
  }
  CMask<1> m;
  m.up[0] = 0;
  m.dn[0] = 0;
  m.cen = 0;
  int gmin = kNoLabel, Om = kNoLabel, cnt = 0;
  ukey run_a = 0, gkey = 0;
  bool have = false;
  auto close_group = [&](ukey v) {
    const int Ok = cnearest<1>(m);
    const bool pt = gmin < (Om < Ok ? Om : Ok);
    const bool ch = Ok != Om || pt;
    if (Om < kNoLabel && ch) {  // the run below v ends at v
      if (WRITE) {
        oa[cnt] = key_out<Key>(run_a);
        ob[cnt] = key_out<Key>(v);
        ol[cnt] = (short)Om;
      }
      ++cnt;
    }
    if (pt) {  // the point [v, v]
      if (WRITE) {
        oa[cnt] = key_out<Key>(v);
        ob[cnt] = key_out<Key>(v);
        ol[cnt] = (short)gmin;
      }
      ++cnt;
    }
    if (Ok < kNoLabel && ch) run_a = v;  // a run starts at v
    Om = Ok;
    gmin = kNoLabel;
  };
  for (;;) {
    // the lowest next event of the slots
    ukey key = e[0].key;
    int sel = 0;
#pragma unroll
    for (int q = 1; q < NS; ++q) {
      const bool lt = e[q].key < key;
      key = lt ? e[q].key : key;
      sel = lt ? q : sel;
    }
    if (key == ~0ULL) break;
    if (have && key != gkey) close_group(gkey);
    gkey = key;
    have = true;
    // toggle the source (slot sel is source i - R + sel, at distance |sel - R|)
    const int d = sel - R;
    const int ad = d < 0 ? -d : d;
    if (d == 0) {
      m.cen ^= 1;
    } else {
      const ukey bit = 1ULL << (ad - 1);
      if (d > 0) m.up[0] ^= bit;
      else m.dn[0] ^= bit;
    }
    gmin = ad < gmin ? ad : gmin;
#pragma unroll
    for (int q = 0; q < NS; ++q)
      if (q == sel) src_next<T>(P.z, P.erode != 0, e[q]);
  }
  if (have) close_group(gkey);
  return cnt;
}

}  // namespace dexel
