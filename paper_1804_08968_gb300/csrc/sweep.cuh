// Per-line sweeps of the two-pass dexel offset (Sec. 3.3), one warp per work item.
//
// Pass 1 (x-extrusion, Sec. 3.3 "3D Dilation"): along a grid row, for every column i and
// height z, the distance dx(z) to the nearest column i' within reach K = floor(k) whose
// dexel contains z.  It is the forward and backward half-space sweep of Sec. 3.2 with
// DilateLine returning extruded seeds: the forward state F(i) keeps, for every z, the
// nearest column on the left; F(i) = S(i) labelled 0, plus F(i-1) minus S(i) with labels
// + 1 (pieces further than K drop out) -- a painter's merge.  The backward sweep does the
// same from the right; S_mid(i) is the pointwise minimum of the two labels ("closest
// parent", largest residual radius sqrt(r^2 - dx^2 h^2)).
//
// Pass 2 (y-dilation with per-piece radius, Sec. 3.3 "2D Power Diagram"): along a grid
// column line, a piece (a, b, dx) of S_mid at line position j' reaches position j with
// the interval [a - w, b + w], w = h sqrt(k^2 - n), n = dx^2 + (j - j')^2 <= k^2.  The
// capsule is split into the extruded rectangle [a, b] (alive while n <= k^2) and the two
// endpoint disks.  The rectangles are kept as a max-expiry envelope; the endpoint disks
// are points with power weight w^2 (Eq. of power cells, App. B) whose half-space power
// diagram along the sweep line is a lower envelope of equal-curvature parabolas, kept
// incrementally: seeds dominated by newer seeds are dropped for good (their disadvantage
// grows linearly with the sweep position), seeds dominated by older ones wait (the
// "not yet born" case of Fig. power-vertex).  Forward and backward results are united per
// column; a column's output is the union of its rectangles and disks.
#pragma once
#include "heights.cuh"

namespace dexel {

#define DEXEL_INF (__builtin_huge_val())

// ------------------------------------------------------------------------------------------
// status bits written by kernels
// ------------------------------------------------------------------------------------------
enum : int {
  ST_OVERFLOW_SLOT = 1,    // a per-warp state array would exceed its capacity
  ST_OVERFLOW_ARENA = 2,   // an output arena is full
  ST_BAD_CSR = 4,
  ST_TOO_MANY_OUT = 8,     // output does not fit int32 offsets
  ST_LEVELS_OVER = 16,     // a level list outgrew its buffer (pass 2 by levels)
  ST_BOUNDS = 32,          // a self-check found an index out of its array (access skipped)
};

constexpr int kWinBins = 32;
struct Counters {
  unsigned long long arena_top[4];  // bump pointers of the arenas
  unsigned long long work_next[2];  // persistent work queues
  int status;
  int max_pieces;     // max pieces of an S_mid column
  int max_out;        // max intervals of an output column
  int max_state;      // max live elements seen in a slot array (for resizing)
  int max_segs_in;    // max input segments per column
  int redo_cols;      // gather: output columns handed to the fallback kernel
  int p1_marked;      // pass-1 window kernel: tiles or columns marked for its redo launch
  unsigned long long mid_total;   // S_mid pieces written
  unsigned long long out_total;   // pass-2 intervals written
  unsigned long long bucket_sum;  // gather: intervals collected over all columns (sizing)
  unsigned zmax_bits;             // gather: bits of max |finite height| of S_mid (float >= 0)
  int over_cols;                  // level gather: columns whose lists outgrew the bucket
  int over_max;                   //   and the most intervals one of them collected
  int ring_spills;                // pass-1 window kernel: tiles walked twice (a lane's ring
                                  // region overflowed)
  unsigned long long lvl_redo;    // level walks: lists longer than a lane's slots (walked again)
  int sticky;                     // stream-ordered calls: status bits folded in before a
                                  // status word is cleared (their failures outlive the clear)
  unsigned long long win_hist[kWinBins];  // pass-1 window events by tile: bin b holds the
                                          // events of the tiles with 1024 b < E <= 1024 (b + 1)
                                          // (the last: E > 1024 (kWinBins - 1))
  unsigned long long phase[16];   // optional per-phase clock totals (DEXEL_PHASES builds)
};

// Optional phase timing of the sweeps (diagnostic builds with -DDEXEL_PHASES): lane 0 adds
// the clock cycles spent in each phase to Counters::phase.
#if defined(DEXEL_PHASES) && defined(__CUDA_ARCH__)
#define PHASE_BEGIN() long long ph_t0_ = clock64()
#define PHASE(k)                                                          \
  do {                                                                    \
    const long long ph_t1_ = clock64();                                   \
    if ((threadIdx.x & 31) == 0) atomicAdd(&P.ctr->phase[k], (unsigned long long)(ph_t1_ - ph_t0_)); \
    ph_t0_ = ph_t1_;                                                      \
  } while (0)
// (v is evaluated by lane 0 alone: no warp-collective operation may appear in it)
#define PHASE_COUNT(k, v) \
  do { if ((threadIdx.x & 31) == 0) atomicAdd(&P.ctr->phase[k], (unsigned long long)(v)); } while (0)
#else
#define PHASE_BEGIN() do {} while (0)
#define PHASE(k) do {} while (0)
#define PHASE_COUNT(k, v) do {} while (0)
#endif

struct ArenaCursor {
  long long cur, end;
  long long tally;  // entries written by this warp (lane 0), added to a counter at the end
  int tmax;         // the largest column of this warp (lane 0)
};

// Reserve n consecutive entries of an arena for one column (warp-uniform result).
DXI long long arena_take(const Lanes& L, unsigned long long* top, long long blk,
                         ArenaCursor& c, long long n) {
  if (c.cur + n > c.end) {
    const long long take = n > blk ? n : blk;
    long long s = 0;
#if defined(__CUDA_ARCH__)
    if (L.lane == 0) s = (long long)atomicAdd(top, (unsigned long long)take);
    s = __shfl_sync(0xffffffffu, s, 0);
#else
    (void)L;
    s = (long long)*top;
    *top += (unsigned long long)take;
#endif
    c.cur = s;
    c.end = s + take;
  }
  const long long r = c.cur;
  c.cur += n;
  return r;
}

DXI void set_status(int* st, int bit) {
#if defined(__CUDA_ARCH__)
  atomicOr(st, bit);
#else
  *st |= bit;
#endif
}
DXI void add_total(unsigned long long* p, long long v) {
#if defined(__CUDA_ARCH__)
  atomicAdd(p, (unsigned long long)v);
#else
  *p += (unsigned long long)v;
#endif
}
DXI void note_max(int* p, int v) {
#if defined(__CUDA_ARCH__)
  atomicMax(p, v);
#else
  if (v > *p) *p = v;
#endif
}

// ------------------------------------------------------------------------------------------
// generic merge of two sorted piece lists into maximal runs of positive-length elementary
// intervals with a combined value (min of labels for pass 1, max of expiries for pass 2).
// Zero-length pieces contribute nothing here (their two endpoints cancel in the parity).
// Scratch: X (T, 2(na+nb)), cA, cB, kind, lab, prev, next (int, 2(na+nb)).
// Output: oa, ob, ov (nout returned).  Runs of equal value that touch are coalesced.
// ------------------------------------------------------------------------------------------
template <typename T, bool TAKE_MIN>
DXN int merge_runs(const Lanes& L, const T* aa, const T* ab, const int* av, int na,
                   const T* ba, const T* bb, const int* bv, int nb, T* X, int* cA, int* cB,
                   int* kind, int* lab, int* prv, int* nxt, T* oa, T* ob, int* ov) {
  const int ea = 2 * na, eb = 2 * nb, m = ea + eb;
  if (m == 0) return 0;
  // merged endpoint sequence (A first on ties)
  for (int e = L.lane; e < ea; e += L.nl) {
    const T v = endpoint(aa, ab, e);
    const int before = count_endpoints_lt(ba, bb, nb, v);
    const int pos = e + before;
    X[pos] = v;
    cA[pos] = e + 1;
    cB[pos] = before;
  }
  for (int e = L.lane; e < eb; e += L.nl) {
    const T v = endpoint(ba, bb, e);
    const int before = count_endpoints_le(aa, ab, na, v);
    const int pos = e + before;
    X[pos] = v;
    cA[pos] = before;
    cB[pos] = e + 1;
  }
  wsync();
  const int ne = m - 1;  // elementary intervals (X[t], X[t+1])
  const int NONE = TAKE_MIN ? 0x7fffffff : (int)0x80000000;
  for (int t = L.lane; t < ne; t += L.nl) {
    int k = 0, v = NONE;
    if (X[t] < X[t + 1]) {
      const int ca = cA[t], cb = cB[t];
      bool cov = false;
      if (ca & 1) {
        v = av[(ca - 1) >> 1];
        cov = true;
      }
      if (cb & 1) {
        const int w = bv[(cb - 1) >> 1];
        v = cov ? (TAKE_MIN ? (w < v ? w : v) : (w > v ? w : v)) : w;
        cov = true;
      }
      k = cov ? 2 : 1;
    }
    kind[t] = k;
    lab[t] = v;
  }
  wsync();
  // nearest earlier non-transparent elementary interval
  for (int t = L.lane; t < ne; t += L.nl) cA[t] = kind[t] >= 1;
  wsync();
  scan_last_flag(L, cA, prv, ne);
  // run starts
  for (int t = L.lane; t < ne; t += L.nl) {
    int s = 0;
    if (kind[t] == 2) {
      const int p = prv[t];
      s = !(p >= 0 && kind[p] == 2 && lab[p] == lab[t]);
    }
    cB[t] = s;
  }
  wsync();
  // breaks: gaps or starts
  for (int t = L.lane; t < ne; t += L.nl) cA[t] = (kind[t] == 1) || cB[t];
  wsync();
  scan_next_flag(L, cA, nxt, ne);
  // positions of runs
  for (int t = L.lane; t < ne; t += L.nl) cA[t] = cB[t];
  wsync();
  const int nout = scan_excl(L, cA, ne);
  for (int t = L.lane; t < ne; t += L.nl) {
    if (cB[t]) {
      const int o = cA[t];
      const int u = nxt[t];
      oa[o] = X[t];
      ob[o] = X[u < ne ? u : ne];
      ov[o] = lab[t];
    }
  }
  wsync();
  return nout;
}

// ------------------------------------------------------------------------------------------
// PASS 1
// ------------------------------------------------------------------------------------------
template <typename T>
struct P1Params {
  typedef typename H<T>::K Key;
  int nx, ny;
  int K;          // reach in columns (largest integer with K^2 <= k^2)
  int erode;      // complement the input on load
  int chunk;      // columns per work item
  int nchunks;    // work items per row
  const int* col_off;
  const T* z;     // input pairs
  // arena 0: forward states (scratch), arena 1: S_mid pieces
  Key* f_a; Key* f_b; short* f_l; long long f_cap;
  Key* m_a; Key* m_b; short* m_l; long long m_cap;
  long long* m_start;   // S_mid index in line-2 order q = i*ny + j
  int* m_cnt;
  long long blk;
  Counters* ctr;
  // per-warp slot
  char* slots; long long slot_bytes;
  int capF, capS;  // capacities of state arrays and of one column's segments
  const int* rows;  // the sweep: only these rows (null: all rows)
  int nrows;
  // the window kernel's ring: per thread of the grid r_cap pieces (null: two walks)
  Key* r_a; Key* r_b; short* r_l; int r_cap;
  long long r_n;  // entries of each ring array (a group whose regions lie beyond walks twice)
  // the window kernel's dominance pruning of S_mid pieces: float half-widths w[n] and the
  // margin of the float test (null: keep every piece)
  const float* prune_w; float prune_E;
  // the window kernel's redo of columns whose windows did not fit: rows with such a column
  // are flagged in rowmark (when given); with redo set only those columns are computed
  int* rowmark; int redo;
  // the window kernel's block of output columns: i in [xa, xb) (xb = 0: the whole row)
  int xa, xb;
  // the window kernel's event buffers (1 or 2; 0 counts as 1)
  int nbuf;
  // the pruning margin computed on the device from the input's max |z| (zmax_bits after the
  // validation) when set: E = 2^-19 (max |z| + prune_kh), else prune_E as given
  const unsigned* prune_zmax;
  double prune_kh;
  // the window kernel's first launch when a redo launch with more room follows: a tile whose
  // window exceeds the room is marked whole for it (instead of split into narrower runs)
  int tile_redo;
  // local index of forward states for the current chunk: per warp, chunk entries
};

template <typename T>
struct P1Slot {
  T *fa, *fb, *ga, *gb, *ra, *rb, *sa, *sb, *ta, *tb, *X;
  int *fl, *gl, *rl, *tl, *c0, *c1, *c2, *c3, *c4, *c5;
  long long* fstart;
  int* fcnt;
};

// carve a slot; capacities: F states capF, segments capS, merge scratch 4*capF
template <typename T>
DXI long long p1_ce(int capF) { return 6LL * capF + 8; }

template <typename T>
DXI long long p1_slot_bytes(int capF, int capS, int chunk) {
  const long long ce = p1_ce<T>(capF);
  long long b = 0;
  b += 4LL * capF * sizeof(T);     // fa fb ta tb
  b += 4LL * ce * sizeof(T);       // ga gb ra rb
  b += 2LL * capS * sizeof(T);     // sa sb
  b += ce * sizeof(T);             // X
  b += 2LL * capF * sizeof(int);   // fl tl
  b += 2LL * ce * sizeof(int);     // gl rl
  b += 6LL * ce * sizeof(int);     // c0..c5
  b += (long long)chunk * (sizeof(long long) + sizeof(int));
  return (b + 1024 + 255) & ~255LL;
}

template <typename T>
DXI P1Slot<T> p1_slot(char* base, int capF, int capS, int chunk) {
  P1Slot<T> s;
  const long long ce = p1_ce<T>(capF);
  char* p = base;
  s.fstart = (long long*)p; p += (long long)chunk * sizeof(long long);
  T** tt[] = {&s.fa, &s.fb, &s.ta, &s.tb};
  for (T** q : tt) { *q = (T*)p; p += (long long)capF * sizeof(T); }
  T** te[] = {&s.ga, &s.gb, &s.ra, &s.rb, &s.X};
  for (T** q : te) { *q = (T*)p; p += ce * sizeof(T); }
  s.sa = (T*)p; p += (long long)capS * sizeof(T);
  s.sb = (T*)p; p += (long long)capS * sizeof(T);
  p = (char*)(((unsigned long long)p + 7) & ~7ULL);
  s.fl = (int*)p; p += (long long)capF * sizeof(int);
  s.tl = (int*)p; p += (long long)capF * sizeof(int);
  int** ie[] = {&s.gl, &s.rl, &s.c0, &s.c1, &s.c2, &s.c3, &s.c4, &s.c5};
  for (int** q : ie) { *q = (int*)p; p += ce * sizeof(int); }
  s.fcnt = (int*)p;
  return s;
}

// segments of input column c (complemented for erosion) into sa/sb as height keys
template <typename T>
DXI int load_segments(const Lanes& L, const P1Params<T>& P, int c, typename H<T>::K* sa,
                      typename H<T>::K* sb) {
  typedef H<T> HT;
  const int s0 = P.col_off[c], s1 = P.col_off[c + 1];
  const int cnt = s1 - s0;
  if (!P.erode) {
    for (int t = L.lane; t < cnt; t += L.nl) {
      sa[t] = HT::key(P.z[2 * (long long)(s0 + t)]);
      sb[t] = HT::key(P.z[2 * (long long)(s0 + t) + 1]);
    }
    wsync();
    return cnt;
  }
  // complement: (-inf, a0], [b0, a1], ..., [b_{n-1}, +inf)
  for (int t = L.lane; t <= cnt; t += L.nl) {
    sa[t] = t == 0 ? HT::ninf() : HT::key(P.z[2 * (long long)(s0 + t - 1) + 1]);
    sb[t] = t == cnt ? HT::pinf() : HT::key(P.z[2 * (long long)(s0 + t)]);
  }
  wsync();
  return cnt + 1;
}

// One painter step: G := S labelled 0  U  (F \ S) labelled +1 (labels > K dropped).
template <typename T>
DXN int painter_step(const Lanes& L, const P1Slot<T>& W, int nf, int ns, int K, int capF,
                     int* status) {
  const T *fa = W.fa, *fb = W.fb, *sa = W.sa, *sb = W.sb;
  const int* fl = W.fl;
  int* cnt = W.c0;
  // remnant counts
  for (int t = L.lane; t < nf; t += L.nl) {
    int c = 0;
    if (fl[t] + 1 <= K) {
      const T a = fa[t], b = fb[t];
      const int lo = lower_bound(sb, ns, a);
      const int hi = upper_bound(sa, ns, b) - 1;
      if (lo > hi) {
        c = 1;
      } else {
        c += a < sa[lo];
        for (int s = lo; s < hi; ++s) c += sb[s] < sa[s + 1];
        c += sb[hi] < b;
      }
    }
    cnt[t] = c;
  }
  wsync();
  const int nr = scan_excl(L, cnt, nf);
  if (nr + ns > capF) {
    if (L.lane == 0) set_status(status, ST_OVERFLOW_SLOT);
    return -1;
  }
  // remnants in z order
  for (int t = L.lane; t < nf; t += L.nl) {
    if (fl[t] + 1 > K) continue;
    int o = cnt[t];
    const T a = fa[t], b = fb[t];
    const int l = fl[t] + 1;
    const int lo = lower_bound(sb, ns, a);
    const int hi = upper_bound(sa, ns, b) - 1;
    if (lo > hi) {
      W.ra[o] = a; W.rb[o] = b; W.rl[o] = l;
      continue;
    }
    if (a < sa[lo]) { W.ra[o] = a; W.rb[o] = sa[lo]; W.rl[o] = l; ++o; }
    for (int s = lo; s < hi; ++s)
      if (sb[s] < sa[s + 1]) { W.ra[o] = sb[s]; W.rb[o] = sa[s + 1]; W.rl[o] = l; ++o; }
    if (sb[hi] < b) { W.ra[o] = sb[hi]; W.rb[o] = b; W.rl[o] = l; ++o; }
  }
  wsync();
  // merge remnants and S by (a, b), S first on ties
  for (int r = L.lane; r < nr; r += L.nl) {
    const T a = W.ra[r], b = W.rb[r];
    int lo = 0, hi = ns;  // count S with (sa < a) || (sa == a && sb <= b)
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (sa[mid] < a || (sa[mid] == a && sb[mid] <= b)) lo = mid + 1; else hi = mid;
    }
    const int pos = r + lo;
    W.ga[pos] = a; W.gb[pos] = b; W.gl[pos] = W.rl[r];
  }
  for (int s = L.lane; s < ns; s += L.nl) {
    const T a = sa[s], b = sb[s];
    int lo = 0, hi = nr;  // count R with (ra < a) || (ra == a && rb < b)
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (W.ra[mid] < a || (W.ra[mid] == a && W.rb[mid] < b)) lo = mid + 1; else hi = mid;
    }
    const int pos = s + lo;
    W.ga[pos] = a; W.gb[pos] = b; W.gl[pos] = 0;
  }
  wsync();
  return nr + ns;
}

template <typename T>
DXI void copy_state(const Lanes& L, T* da, T* db, int* dl, const T* sa, const T* sb,
                    const int* sl, int n) {
  for (int t = L.lane; t < n; t += L.nl) { da[t] = sa[t]; db[t] = sb[t]; dl[t] = sl[t]; }
  wsync();
}

// S_mid(i) = pointwise min label of F(i) and B(i).  Positive-length coverage comes from the
// elementary-interval merge.  A zero-length piece (a tangent sample of the input) is a point
// whose label can be below that of the pieces around it; it is kept only then, and the
// covering piece is split at the point so that the endpoints stay non-decreasing.
// F in (ta, tb, tl), B in (fa, fb, fl) of the slot.  Result in (ra, rb, rl).
template <typename T>
DXN int min_merge(const Lanes& L, const P1Slot<T>& W, int nF, int nB, int capF, int* status) {
  if (3LL * (nF + nB) > p1_ce<T>(capF) - 8) {
    if (L.lane == 0) set_status(status, ST_OVERFLOW_SLOT);
    return -1;
  }
  const int nr = merge_runs<T, true>(L, W.ta, W.tb, W.tl, nF, W.fa, W.fb, W.fl, nB, W.X, W.c0,
                                     W.c1, W.c2, W.c3, W.c4, W.c5, W.ra, W.rb, W.rl);
  int* zf = W.c1;
  int* zb = W.c2;
  for (int t = L.lane; t < nF; t += L.nl) zf[t] = W.ta[t] == W.tb[t];
  for (int t = L.lane; t < nB; t += L.nl) zb[t] = W.fa[t] == W.fb[t];
  wsync();
  const int nzf = scan_excl(L, zf, nF);
  const int nzb = scan_excl(L, zb, nB);
  const int nz = nzf + nzb;
  if (nz == 0) return nr;
  // zero pieces of F and B merged by height into (X, c3); F first on ties
  T* zx = W.X;
  int* zl = W.c3;
  T* zxb = W.ga;  // B's zero heights, temporarily
  for (int t = L.lane; t < nB; t += L.nl)
    if (W.fa[t] == W.fb[t]) zxb[zb[t]] = W.fa[t];
  // F's zero heights in gb temporarily
  T* zxf = W.gb;
  for (int t = L.lane; t < nF; t += L.nl)
    if (W.ta[t] == W.tb[t]) zxf[zf[t]] = W.ta[t];
  wsync();
  for (int t = L.lane; t < nF; t += L.nl)
    if (W.ta[t] == W.tb[t]) {
      const int pos = zf[t] + lower_bound(zxb, nzb, W.ta[t]);
      zx[pos] = W.ta[t]; zl[pos] = W.tl[t];
    }
  for (int t = L.lane; t < nB; t += L.nl)
    if (W.fa[t] == W.fb[t]) {
      const int pos = zb[t] + upper_bound(zxf, nzf, W.fa[t]);
      zx[pos] = W.fa[t]; zl[pos] = W.fl[t];
    }
  wsync();
  // keep a point when no other point at the same height has a smaller label (ties: the
  // last one) and every run containing it has a larger label
  int* keep = W.c4;
  for (int u = L.lane; u < nz; u += L.nl) {
    const T x = zx[u];
    bool k = true;
    if (u + 1 < nz && zx[u + 1] == x && zl[u + 1] <= zl[u]) k = false;
    if (u > 0 && zx[u - 1] == x && zl[u - 1] < zl[u]) k = false;
    if (k) {
      const int r = upper_bound(W.ra, nr, x) - 1;  // last run with a <= x
      for (int q = r; q >= 0 && q >= r - 1; --q)
        if (W.ra[q] <= x && x <= W.rb[q] && W.rl[q] <= zl[u]) k = false;
    }
    keep[u] = k;
  }
  wsync();
  int* kpos = W.c5;
  for (int u = L.lane; u < nz; u += L.nl) kpos[u] = keep[u];
  wsync();
  const int nk = scan_excl(L, kpos, nz);
  // kept points compacted into (gb as x, c2 as label)
  T* kx = W.gb;
  int* kl = W.c2;
  for (int u = L.lane; u < nz; u += L.nl)
    if (keep[u]) { kx[kpos[u]] = zx[u]; kl[kpos[u]] = zl[u]; }
  wsync();
  // split runs at kept points strictly inside them
  int* parts = W.c0;
  for (int r = L.lane; r < nr; r += L.nl) {
    const int lo = upper_bound(kx, nk, W.ra[r]);  // first point > a
    const int hi = lower_bound(kx, nk, W.rb[r]);  // first point >= b
    parts[r] = 1 + (hi > lo ? hi - lo : 0);
  }
  wsync();
  int* ppos = W.c1;
  for (int r = L.lane; r < nr; r += L.nl) ppos[r] = parts[r];
  wsync();
  const int np = scan_excl(L, ppos, nr);
  if (np + nk > p1_ce<T>(capF) - 8) {
    if (L.lane == 0) set_status(status, ST_OVERFLOW_SLOT);
    return -1;
  }
  // parts into (ga, X?) -- use ga / tb / c3 as (a, b, label); X (zx) no longer needed
  T* pa = W.ga;
  T* pb = W.X;
  int* pl = W.c3;
  for (int r = L.lane; r < nr; r += L.nl) {
    const int lo = upper_bound(kx, nk, W.ra[r]);
    const int hi = lower_bound(kx, nk, W.rb[r]);
    T a = W.ra[r];
    int o = ppos[r];
    for (int q = lo; q < hi; ++q) {
      pa[o] = a; pb[o] = kx[q]; pl[o] = W.rl[r]; ++o;
      a = kx[q];
    }
    pa[o] = a; pb[o] = W.rb[r]; pl[o] = W.rl[r];
  }
  wsync();
  // final order by (a, b): a point (x, x) precedes a part (a, b) iff x <= a
  for (int p = L.lane; p < np; p += L.nl) {
    const int pos = p + upper_bound(kx, nk, pa[p]);
    W.ra[pos] = pa[p]; W.rb[pos] = pb[p]; W.rl[pos] = pl[p];
  }
  for (int u = L.lane; u < nk; u += L.nl) {
    const int pos = u + lower_bound(pa, np, kx[u]);
    W.ra[pos] = kx[u]; W.rb[pos] = kx[u]; W.rl[pos] = kl[u];
  }
  wsync();
  return np + nk;
}

// Work item: row j, columns [c0, c1).  Writes S_mid(i, j) for i in [c0, c1).
template <typename T>
DXN void pass1_item(const Lanes& L, const P1Params<T>& P, const P1Slot<typename H<T>::K>& W,
                    int j, int c0, int c1, ArenaCursor& curF, ArenaCursor& curM) {
  int* status = &P.ctr->status;
  const int N = P.nx;
  const int K = P.K;
  // ---- forward sweep
  int nf = 0;
  const int i_begin = c0 - K > 0 ? c0 - K : 0;
  for (int i = i_begin; i < c1; ++i) {
    const int ns = load_segments(L, P, j * N + i, W.sa, W.sb);
    if (ns > P.capS) { if (L.lane == 0) set_status(status, ST_OVERFLOW_SLOT); return; }
    const int ng = painter_step(L, W, nf, ns, K, P.capF, status);
    if (ng < 0) return;
    copy_state(L, W.fa, W.fb, W.fl, W.ga, W.gb, W.gl, ng);
    nf = ng;
    if (i >= c0) {
      const long long s = arena_take(L, &P.ctr->arena_top[0], P.blk, curF, nf);
      const bool fits = s + nf <= P.f_cap;
      if (!fits) { if (L.lane == 0) set_status(status, ST_OVERFLOW_ARENA); }
      else {
        for (int t = L.lane; t < nf; t += L.nl) {
          P.f_a[s + t] = W.fa[t]; P.f_b[s + t] = W.fb[t]; P.f_l[s + t] = (short)W.fl[t];
        }
      }
      if (L.lane == 0) { W.fstart[i - c0] = fits ? s : -1; W.fcnt[i - c0] = nf; }
      wsync();
    }
  }
  // ---- backward sweep
  int nb = 0;
  long long item_total = 0;
  const int i_end = c1 - 1 + K < N - 1 ? c1 - 1 + K : N - 1;
  for (int i = i_end; i >= c0; --i) {
    const int ns = load_segments(L, P, j * N + i, W.sa, W.sb);
    if (ns > P.capS) { if (L.lane == 0) set_status(status, ST_OVERFLOW_SLOT); return; }
    const int ng = painter_step(L, W, nb, ns, K, P.capF, status);
    if (ng < 0) return;
    copy_state(L, W.fa, W.fb, W.fl, W.ga, W.gb, W.gl, ng);
    nb = ng;
    if (i < c1) {
      // F(i) back from the scratch arena into (ta, tb, tl)
      const long long fs = W.fstart[i - c0];
      const int nF = W.fcnt[i - c0];
      if (fs < 0) continue;  // overflow already flagged
      for (int t = L.lane; t < nF; t += L.nl) {
        W.ta[t] = P.f_a[fs + t]; W.tb[t] = P.f_b[fs + t]; W.tl[t] = P.f_l[fs + t];
      }
      wsync();
      const int nm = min_merge(L, W, nF, nb, P.capF, status);
      if (nm < 0) return;
      const long long s = arena_take(L, &P.ctr->arena_top[1], P.blk, curM, nm);
      const bool fits = s + nm <= P.m_cap;
      if (!fits) { if (L.lane == 0) set_status(status, ST_OVERFLOW_ARENA); }
      else {
        for (int t = L.lane; t < nm; t += L.nl) {
          P.m_a[s + t] = W.ra[t]; P.m_b[s + t] = W.rb[t]; P.m_l[s + t] = (short)W.rl[t];
        }
      }
      if (L.lane == 0) {
        const long long q = (long long)i * P.ny + j;
        P.m_start[q] = fits ? s : 0;
        P.m_cnt[q] = nm;
        note_max(&P.ctr->max_pieces, nm);
      }
      item_total += nm;
      wsync();
    }
  }
  if (L.lane == 0) add_total(&P.ctr->mid_total, item_total);
}

}  // namespace dexel
