// Pass 2 of the dexel offset as a gather over the window (Sec. 3.3, GB300 formulation).
//
// After pass 1 every column (i, j') holds S_mid pieces (a, b, dx).  Along the y line i a
// piece reaches column j with the capsule slice [a - w, b + w], w = h sqrt(k^2 - n),
// n = dx^2 + (j - j')^2 <= k^2 -- its extruded rectangle (Fig. segments-separate, D-rect)
// united with the disks of its two endpoint seeds (D-disk).  For a fixed source column j'
// and level t = |j - j'| the union of its capsules is the part of the line covered by that
// column's seeds and rectangles: in power terms the sublevel set {z : min_e pi_e(z) <= 0}
// of that column's seeds, pi_e(z) = (z - z_e)^2 - w_e^2 (Eq. of power cells, App. B),
// together with its rectangles.  The covered set of output column j is the union of these
// per-source sets over the 2R + 1 sources of the window -- the paper's forward and backward
// half-space diagrams together (Sec. 3.2: Omega_i within the union of the two half cells).
//
// GB300 mapping: one warp per output column, no state carried from column to column.  The
// window's pieces are split evenly over the 32 lanes; a lane unites the slices of its range
// one at a time into an open interval and appends it to the column's bucket when the next
// slice cannot be merged for certain.  The bucket is sorted by left end (bitonic, shared
// memory) and united exactly; with the tiled kernel this happens in rounds, so that the
// bucket stays small.  Blocks take tiles of consecutive columns of a line and stage the
// tile's window (float ends, dx) in shared memory once for all its columns.
//
// Merge decisions are taken on float approximations with an error bound and are only an
// optimisation (an undecided pair is appended as two intervals); the appended ends are the
// exact doubles a - w and b + w, and the final union compares exact keys, so the result
// equals the all-double computation bit for bit.
#pragma once
#include "sweep2.cuh"

namespace dexel {

template <typename T>
struct P2GParams {
  typedef typename H<T>::K Key;
  int nx, ny;
  int R;
  double kk;
  const double* wtab;   // w[n] = h sqrt(k^2 - n)
  const float* wtabf;   // the same rounded to float
  const int* reach;     // reach[dx] = largest level t with dx^2 + t^2 <= k^2
  const Key* m_a; const Key* m_b; const short* m_l;
  const long long* m_start; const int* m_cnt;
  ukey* o_l; ukey* o_r; long long o_cap;
  long long* o_start;  // per output column, row-major c = j*nx + i
  int* o_cnt;
  long long blk;
  Counters* ctr;
  int bcap;  // bucket entries per output column (power of two)
  int redo;  // k_pass2c: only the columns whose count is -1
  int nmax;  // largest n = dx^2 + t^2 with n <= k^2
  // line-contiguous float copy of S_mid (k_mid_pack): pieces of column q = i*ny + j at
  // c_start[q] ..; float ends and dx
  const long long* c_start;
  const float* c_af;
  const float* c_bf;
  const short* c_dx;
};

// In-place bitonic sort of (key, val) pairs by key, n a power of two, one warp.
DXI void warp_bitonic(const Lanes& L, ukey* key, ukey* val, int n) {
  for (int k = 2; k <= n; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = L.lane; t < n; t += L.nl) {
        const int x = t ^ j;
        if (x > t) {
          const bool up = (t & k) == 0;
          const ukey kt = key[t], kx = key[x];
          if ((kt > kx) == up) {
            key[t] = kx; key[x] = kt;
            const ukey v = val[t]; val[t] = val[x]; val[x] = v;
          }
        }
      }
      wsync();
    }
  }
}

// Bitonic sort of (key, val) pairs by key held in registers: PER pairs a lane, element
// i = r * 32 + lane (so that the shared-memory loads and stores are conflict free); steps
// with partner distance >= 32 swap within a lane, shorter ones exchange by shuffles.
template <int PER>
__device__ __forceinline__ void reg_sort_pairs(ukey* key, ukey* val, int n2, int lane) {
#if defined(__CUDA_ARCH__)
  ukey k[PER], v[PER];
#pragma unroll
  for (int r = 0; r < PER; ++r) {
    const int i = r * 32 + lane;
    k[r] = i < n2 ? key[i] : ~0ULL;
    v[r] = i < n2 ? val[i] : ~0ULL;
  }
  const int n = 32 * PER;
  for (int kk = 2; kk <= n; kk <<= 1) {
#pragma unroll
    for (int jr = PER / 2; jr > 0; jr >>= 1) {  // distance jr * 32: within the lane
      if (jr * 32 > (kk >> 1)) continue;
#pragma unroll
      for (int r = 0; r < PER; ++r) {
        const int rp = r ^ jr;
        if (rp > r) {
          const bool up = ((r * 32 + lane) & kk) == 0;
          if ((k[r] > k[rp]) == up) {
            const ukey tk = k[r]; k[r] = k[rp]; k[rp] = tk;
            const ukey tv = v[r]; v[r] = v[rp]; v[rp] = tv;
          }
        }
      }
    }
    for (int jj = (kk >> 1) < 16 ? (kk >> 1) : 16; jj > 0; jj >>= 1) {  // across lanes
#pragma unroll
      for (int r = 0; r < PER; ++r) {
        const ukey ko = __shfl_xor_sync(0xffffffffu, k[r], jj);
        const ukey vo = __shfl_xor_sync(0xffffffffu, v[r], jj);
        const bool up = ((r * 32 + lane) & kk) == 0;
        const bool lower = (lane & jj) == 0;
        const bool take = lower ? ((k[r] > ko) == up) : ((ko > k[r]) == up);
        if (take) { k[r] = ko; v[r] = vo; }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < PER; ++r) {
    const int i = r * 32 + lane;
    if (i < n2) { key[i] = k[r]; val[i] = v[r]; }
  }
  __syncwarp();
#endif
}

// Sort of n2 (a power of two) pairs in shared memory by key: in registers up to 256, else
// the shared-memory network.
DXI void warp_sort_pairs(const Lanes& L, ukey* key, ukey* val, int n2) {
#if defined(__CUDA_ARCH__)
  if (n2 <= 32) reg_sort_pairs<1>(key, val, n2, L.lane);
  else if (n2 <= 64) reg_sort_pairs<2>(key, val, n2, L.lane);
  else if (n2 <= 128) reg_sort_pairs<4>(key, val, n2, L.lane);
  else if (n2 <= 256) reg_sort_pairs<8>(key, val, n2, L.lane);
  else warp_bitonic(L, key, val, n2);
#else
  warp_bitonic(L, key, val, n2);
#endif
}

DXI int pow2_at_least(int n) {
  int m = 1;
  while (m < n) m <<= 1;
  return m;
}

}  // namespace dexel

namespace dexel {

// Balanced cover of one output column (i, j): the pieces of the window's sources, taken in
// (source, height) order, are cut into 32 equal contiguous ranges, one per lane, so that the
// lanes' work does not depend on how the pieces spread over the sources.  A lane unites the
// capsule slices of its range one at a time into a single open interval and appends it to the
// column's bucket when the next slice cannot be merged for certain (float ends with the error
// bound e(x) = eps (|x| + |y| + 2 w_max)) or when its range passes to another source.  An
// undecided merge is left to the final exact union, so no double arithmetic is needed until
// the exact ends of an appended interval are formed.  Appended intervals may overlap; the
// caller sorts and unites them.
// Per-warp shared memory of the balanced gather kernel (window offsets, bucket, union).
DXI long long pass2c_warp_bytes(int R, int bcap) {
  const long long off = ((2LL * R + 2) * sizeof(int) + 15) & ~15LL;
  return off + 4LL * bcap * sizeof(ukey) + 2LL * bcap * sizeof(int) + 16;
}

struct CoverCur {
  float lf, rf;   // float approximations of the interval's ends
  int li, ri;     // pieces (within the source) of the exact ends
  int n_l, n_r;   // their squared offsets dx^2 + t^2
};

template <typename Key>
DXI void cover_emit(const Key* a, const Key* b, const double* wtab, const CoverCur& c,
                    ukey* bl, ukey* br, int* bcount, int bcap) {
  int pos;
#if defined(__CUDA_ARCH__)
  pos = atomicAdd(bcount, 1);
#else
  pos = (*bcount)++;
#endif
  if (pos < bcap) {
    bl[pos] = dkey(keyd(a[c.li]) - wtab[c.n_l]);
    br[pos] = dkey(keyd(b[c.ri]) + wtab[c.n_r]);
  }
}

// Merges the slice [lf, rf] (piece p, offset n) into the current interval when they overlap
// for certain and the float ends say for certain which end of the union comes from which.
DXI bool cover_merge(CoverCur& c, float lf, float rf, int p, int n, float wmax2) {
  const float eps = 2.5e-7f;
  const float INF = __builtin_huge_valf();
  bool merge;
  if (c.rf == INF || lf == -INF) merge = true;
  else merge = c.rf - lf > eps * (fabsf(lf) + fabsf(c.rf) + wmax2);
  if (!merge) return false;
  int lsel, rsel;  // 1: current, 2: new, 0: undecided
  if (c.lf == -INF) lsel = 1;
  else if (lf == -INF) lsel = 2;
  else {
    const float e = eps * (fabsf(lf) + fabsf(c.lf) + wmax2);
    lsel = lf - c.lf > e ? 1 : (c.lf - lf > e ? 2 : 0);
  }
  if (c.rf == INF) rsel = 1;
  else if (rf == INF) rsel = 2;
  else {
    const float e = eps * (fabsf(rf) + fabsf(c.rf) + wmax2);
    rsel = c.rf - rf > e ? 1 : (rf - c.rf > e ? 2 : 0);
  }
  if (!lsel || !rsel) return false;
  if (lsel == 2) { c.lf = lf; c.li = p; c.n_l = n; }
  if (rsel == 2) { c.rf = rf; c.ri = p; c.n_r = n; }
  return true;
}

// Covers the pieces g0 <= g < g1 of the window (sources s0 .. s0 + ns - 1 of line i, piece
// offsets srcoff[]), appending to the bucket.
template <typename T>
DXI void cover_range(const P2GParams<T>& P, long long qb, int j, int s0, int ns,
                     const int* srcoff, int g0, int g1, float wmax2, ukey* bl, ukey* br,
                     int* bcount, int bcap) {
  typedef typename H<T>::K Key;
  if (g0 >= g1) return;
  // source of the first piece: the last q with srcoff[q] <= g0
  int lo = 0, hi = ns - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (srcoff[mid] <= g0) lo = mid;
    else hi = mid - 1;
  }
  int q = lo;
  while (q < ns - 1 && srcoff[q + 1] <= g0) ++q;  // skip empty sources
  int g = g0;
  while (g < g1) {
    const int send = min(g1, srcoff[q + 1]);
    const int jj = s0 + q;
    const int t = jj > j ? jj - j : j - jj;
    const long long ms = P.m_start[qb + jj];
    const Key* a = P.m_a + ms;
    const Key* b = P.m_b + ms;
    const short* dxa = P.m_l + ms;
    bool have = false;
    CoverCur c{};
    for (int p = g - srcoff[q], pe = send - srcoff[q]; p < pe; ++p) {
      const int dx = dxa[p];
      const int n = dx * dx + t * t;
      if (n > P.nmax) continue;
      const float wf = P.wtabf[n];
      const float lf = keyf(a[p]) - wf;
      const float rf = keyf(b[p]) + wf;
      if (have && cover_merge(c, lf, rf, p, n, wmax2)) continue;
      if (have) cover_emit<Key>(a, b, P.wtab, c, bl, br, bcount, bcap);
      c.lf = lf; c.rf = rf; c.li = p; c.ri = p; c.n_l = n; c.n_r = n;
      have = true;
    }
    if (have) cover_emit<Key>(a, b, P.wtab, c, bl, br, bcount, bcap);
    g = send;
    ++q;
  }
}

// The same cover with the window's pieces staged in shared memory by the block (float
// approximations of the ends and dx; staged index g, pieces of source q at soff[q] ..
// soff[q + 1] - 1, exact keys at sbase[q] + g in global memory).  The lane's interval is
// carried across source boundaries, and odd sources are walked from the top, so that the
// top interval of one source meets the top pieces of the next one (and the bottom ones the
// bottom): the overlap test is therefore two-sided.
struct CoverCurG {
  float lf, rf;         // float approximations of the interval's ends
  long long kl, kr;     // global key indices of the pieces giving the exact ends
  int n_l, n_r;         // their squared offsets dx^2 + t^2
};

// Merge with a fixed bound E on the difference between a float end and the double it
// approximates, summed over the two ends compared: E = 2^-20 (max |z| + w_max) (each float
// end is within 2^-22 (|z| + w) of the double: key truncation 2^-23 |z|, rounding of w and of
// the difference 2^-24 each).  Infinite ends need no special case: inf - E = inf.
DXI bool cover_merge2(CoverCurG& c, float lf, float rf, long long kidx, int n, float E) {
  if (!(lf <= c.rf - E && rf >= c.lf + E)) return false;  // overlap not certain
  const bool l_new = lf <= c.lf - E, l_cur = lf >= c.lf + E;
  const bool r_new = rf >= c.rf + E, r_cur = rf <= c.rf - E;
  if (!(l_new || l_cur) || !(r_new || r_cur)) return false;  // an end undecided
  if (l_new) { c.lf = lf; c.kl = kidx; c.n_l = n; }
  if (r_new) { c.rf = rf; c.kr = kidx; c.n_r = n; }
  return true;
}

template <typename Key>
DXI void cover_emit2(const Key* ma, const Key* mb, const double* wtab, const CoverCurG& c,
                     ukey* bl, ukey* br, int* bcount, int bcap) {
  int pos;
#if defined(__CUDA_ARCH__)
  pos = atomicAdd(bcount, 1);
#else
  pos = (*bcount)++;
#endif
  if (pos < bcap) {
    bl[pos] = dkey(keyd(ma[c.kl]) - wtab[c.n_l]);
    br[pos] = dkey(keyd(mb[c.kr]) + wtab[c.n_r]);
  }
}

// Resumable walk of a lane over its range of staged pieces (see cover_staged): the current
// source q, its segment [lo, hi) of the range, the pieces taken so far in it (u) and the
// interval under construction.
struct LaneWalk {
  int q, lo, hi, u;
  int tt;          // squared level of source q
  bool down;       // source q is walked from the top
  bool have, done;
  long long kb;    // global key index of staged piece 0 of source q (sbase[q])
  CoverCurG c;
};

template <typename T>
DXI void walk_source(LaneWalk& w, int j, int s0, const int* soff, const long long* sbase, int g1) {
  const int jj = s0 + w.q;
  const int t = jj > j ? jj - j : j - jj;
  w.tt = t * t;
  w.down = (jj & 1) != 0;
  w.kb = sbase[w.q];
  w.hi = min(g1, soff[w.q + 1]);
  w.u = 0;
}

template <typename T>
DXI void walk_init(LaneWalk& w, int j, int s0, const int* soff, const long long* sbase,
                   int qlo, int qhi, int g0, int g1) {
  w.have = false;
  w.done = g0 >= g1;
  w.c = CoverCurG{};
  if (w.done) return;
  int lo = qlo, hi = qhi;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (soff[mid] <= g0) lo = mid;
    else hi = mid - 1;
  }
  w.q = lo;
  w.lo = g0;
  walk_source<T>(w, j, s0, soff, sbase, g1);
}

// One round of the lane's walk: takes at most M pieces, unites their slices into the current
// interval and appends at most Q intervals to the bucket (through the warp's shared counter);
// the state is kept for the next round.  The piece budget keeps the lanes of a round in step.
template <typename T>
DXI void cover_round(const P2GParams<T>& P, LaneWalk& w, int j, int s0, const int* soff,
                     const long long* sbase, const float* saf, const float* sbf,
                     const short* sdx, const float* wt, int g1, float E, int Q, int M,
                     ukey* bl, ukey* br, int* bcount, int bcap) {
  typedef typename H<T>::K Key;
  int emitted = 0;
  while (!w.done && emitted < Q && M > 0) {
    if (w.u == w.hi - w.lo) {  // segment done
      if (w.hi >= g1) {
        if (w.have) {
          cover_emit2<Key>(P.m_a, P.m_b, P.wtab, w.c, bl, br, bcount, bcap);
          ++emitted;
          w.have = false;
        }
        w.done = true;
        break;
      }
      ++w.q;
      w.lo = w.hi;
      walk_source<T>(w, j, s0, soff, sbase, g1);
      continue;
    }
    const int gg = w.down ? w.hi - 1 - w.u : w.lo + w.u;
    ++w.u;
    --M;
    // straight-line body (selects, no early exits) so that the lanes stay converged; only
    // the rare append branches
    const int dx = sdx[gg];
    const int n = dx * dx + w.tt;
    const bool v = n <= P.nmax;
    const float wf = wt[v ? n : 0];
    const float lf = saf[gg] - wf;
    const float rf = sbf[gg] + wf;
    const long long kidx = w.kb + gg;
    const bool ov = lf <= w.c.rf - E && rf >= w.c.lf + E;  // certain overlap
    const bool l_new = lf <= w.c.lf - E, l_cur = lf >= w.c.lf + E;
    const bool r_new = rf >= w.c.rf + E, r_cur = rf <= w.c.rf - E;
    const bool merge = v && w.have && ov && (l_new || l_cur) && (r_new || r_cur);
    if (v && w.have && !merge) {
      cover_emit2<Key>(P.m_a, P.m_b, P.wtab, w.c, bl, br, bcount, bcap);
      ++emitted;
    }
    const bool fresh = v && !merge;  // starts a new interval
    const bool tl = fresh || (merge && l_new);
    const bool tr = fresh || (merge && r_new);
    w.c.lf = tl ? lf : w.c.lf;
    w.c.kl = tl ? kidx : w.c.kl;
    w.c.n_l = tl ? n : w.c.n_l;
    w.c.rf = tr ? rf : w.c.rf;
    w.c.kr = tr ? kidx : w.c.kr;
    w.c.n_r = tr ? n : w.c.n_r;
    w.have = w.have || v;
  }
}

// Union of n intervals sorted by left key (closed: touching ones join), in two steps so that
// the runs can be written straight to their final place: union_count marks run starts
// (start[]), turns cr[] into running maxima and pos[] into run indices, and returns the run
// count; union_write stores the runs.
DXI int union_count(const Lanes& L, const ukey* cl, ukey* cr, int n, int* start, int* pos) {
  ukey carry = 0;
  for (int base = 0; base < n; base += L.nl) {
    const int t = base + L.lane;
    const ukey v = t < n ? cr[t] : 0;
    const ukey inc = w_incl_maxk(v, L.lane);
    const ukey prev = w_shift_up(inc, L.lane, 0);
    if (t < n) {
      const ukey ex = prev > carry ? prev : carry;
      const int st = (t == 0) || (cl[t] > ex);
      start[t] = st;
      pos[t] = st;
      cr[t] = ex > v ? ex : v;
    }
    const ukey last = w_bcastk(inc, L.nl - 1);
    carry = last > carry ? last : carry;
  }
  wsync();
  return scan_excl(L, pos, n);
}

DXI void union_write(const Lanes& L, const ukey* cl, const ukey* cr, int n, const int* start,
                     const int* pos, ukey* ol, ukey* orr) {
  for (int t = L.lane; t < n; t += L.nl) {
    const bool last = (t == n - 1) || start[t + 1];
    const int r = pos[t] - (start[t] ? 0 : 1);
    if (start[t]) ol[r] = cl[t];
    if (last) orr[r] = cr[t];
  }
}

// union_write into the front of the same arrays (run r <= element t): each chunk of 32 is
// read into registers before any lane writes.
DXI void union_write_inplace(const Lanes& L, ukey* cl, ukey* cr, int n, const int* start,
                             const int* pos) {
  for (int base = 0; base < n; base += L.nl) {
    const int t = base + L.lane;
    ukey l = 0, r = 0;
    int idx = -1;
    bool st = false, last = false;
    if (t < n) {
      l = cl[t];
      r = cr[t];
      st = start[t] != 0;
      last = (t == n - 1) || start[t + 1];
      idx = pos[t] - (st ? 0 : 1);
    }
    wsync();
    if (t < n) {
      if (st) cl[idx] = l;
      if (last) cr[idx] = r;
    }
    wsync();
  }
}

// Shared-memory layout of the tiled balanced kernel: the tile window's piece offsets, the
// w table, the staged pieces, and per warp a bucket with the union's flags.
struct P2TLayout {
  long long soff, sbase, swt, saf, sbf, sdx, warps, warp_bytes, total;
};

DXI long long align16(long long x) { return (x + 15) & ~15LL; }

DXI P2TLayout p2t_layout(int R, int tc, int ntab, int stage_cap, int nwarps, int bcap) {
  P2TLayout o;
  long long x = 0;
  o.soff = x; x = align16(x + (long long)(tc + 2 * R + 2) * sizeof(int));
  o.sbase = x; x = align16(x + (long long)(tc + 2 * R + 2) * sizeof(long long));
  o.swt = x; x = align16(x + (long long)ntab * sizeof(float));
  o.saf = x; x += (long long)stage_cap * sizeof(float);
  o.sbf = x; x += (long long)stage_cap * sizeof(float);
  o.sdx = x; x = align16(x + (long long)stage_cap * sizeof(short));
  o.warp_bytes = align16(2LL * bcap * sizeof(ukey) + 2LL * bcap * sizeof(int) + 16);
  o.warps = x; x += nwarps * o.warp_bytes;
  o.total = x;
  return o;
}

}  // namespace dexel
