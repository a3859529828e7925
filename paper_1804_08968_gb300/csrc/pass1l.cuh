// Pass 1 of the dexel offset (Sec. 3.3, the extrusion along x) with one lane per output
// column.
//
// The partition is the one of pass1g.cuh: between consecutive distinct endpoint heights the
// open interval carries the label O = min |i - i'| over the sources i' open there, and the
// height v itself the label P <= min(O_below, O_above); the pieces are the maximal runs of
// equal O (closed) and the points [v, v] with P below both neighbours.  Every source that
// contains v is open below it, open above it, or has an event at v, so P = min(O_below,
// O_above, g) with g the least |i - i'| over the sources with an event at v: a point exists
// exactly when g < min(O_below, O_above), and it does not matter in which order the events of
// one height are applied.
//
// GB300 mapping: a block takes 32 consecutive output columns of row j, one lane each.  The
// events of their window (32 + 2R source columns, contiguous in the row-major input) are
// staged in shared memory and sorted by height once.  The sorted events are cut at group
// boundaries into one chunk per warp; a warp walks its chunk for all 32 columns (broadcast
// reads, a warp-uniform loop: no divergence, no shuffles), each lane starting from the sources
// open at the chunk's start (the XOR of the earlier chunks' toggles) and keeping them as two
// bit masks centred on its column, so that the nearest open source is two find-first-set
// operations.  One walk writes each lane's pieces of its chunk to the lane's ring region and
// notes where its runs start; the counts then place every (column, chunk) in the S_mid arena
// and the warps copy the regions there (coalesced), a run that began in an earlier chunk taking
// its start from the last one noted.  Without a ring (or when a lane outgrows its region) a
// counting walk and a writing walk do the same.  A window with more events than fit is split
// into narrower runs of columns.
#pragma once
#include "pass1g.cuh"

#define DXD __device__ __forceinline__

namespace dexel {

// a height group of the walk is closed only when some lane saw an event within its label
#ifndef DEXEL_P1_LAZY
#define DEXEL_P1_LAZY 1
#endif

// words of the tile-relative source masks (32 + 2R + 1 <= 320 sources: R <= 128)
constexpr int kP1TileWords = 5;

// Event keys of the window kernel: the order-preserving 64-bit key of a double (double
// inputs), or the order-preserving 32-bit key of a float (float inputs: 6 bytes an event in
// shared memory instead of 10, a cheaper sort and 32-bit compares).  of: the key of a height;
// none: the sentinel that sorts last; ninf / pinf: the complement's unbounded ends; out: the
// S_mid key of an event key (exact); approx: a float approximation (the pruning test).
template <typename T>
struct EvK;
template <>
struct EvK<double> {
  typedef ukey type;
  DXD static ukey of(double x) { return dkey(x); }
  DXD static ukey none() { return ~0ULL; }
  DXD static ukey ninf() { return KEY_NINF; }
  DXD static ukey pinf() { return KEY_PINF; }
  DXD static ukey out(ukey k) { return k; }
  DXD static float approx(ukey k) { return keyf(k); }
};
template <>
struct EvK<float> {
  typedef unsigned type;
  DXD static unsigned of(float x) {
    const unsigned b = __float_as_uint(x == 0.0f ? 0.0f : x);  // -0 folded into +0
    return b ^ ((b >> 31) ? 0xFFFFFFFFu : 0x80000000u);
  }
  DXD static unsigned none() { return 0xFFFFFFFFu; }  // above the key of +inf (0xFF800000)
  DXD static unsigned ninf() { return 0x007FFFFFu; }  // the key of -inf
  DXD static unsigned pinf() { return 0xFF800000u; }  // the key of +inf
  DXD static float out(unsigned k) {
    return __uint_as_float((k >> 31) ? (k ^ 0x80000000u) : ~k);
  }
  DXD static float approx(unsigned k) { return out(k); }
};

// Shared memory of k_pass1l: sorted events (key, source), the window's event offsets, chunk
// bounds, chunk toggle masks, per (chunk, lane) counts, last run starts and open-run flags,
// the columns' offsets in the tile, tile base and ring-overflow flag.
struct P1LLayout {
  long long ek, ep, eoff, cb, cm, ccnt, cst, cco, cex, misc, wt, total;
};
DXI long long p1l_align(long long x) { return (x + 15) & ~15LL; }
// ksz: bytes of an event key (8 for double inputs, 4 for float); nbuf: event buffers of ecap
// events (2: the merge of the sources' runs has room for any window that fits one buffer)
DXI P1LLayout p1l_layout(int R, int ecap, int warps, int ksz = 8, int nbuf = 1) {
  P1LLayout o;
  long long x = 0;
  const long long room = (long long)ecap * (nbuf == 2 ? 2 : 1);
  o.ek = x; x = p1l_align(x + room * ksz);
  o.ep = x; x = p1l_align(x + room * sizeof(unsigned short));
  o.eoff = x; x = p1l_align(x + (long long)(32 + 2 * R + 2) * sizeof(int));
  o.cb = x; x = p1l_align(x + (long long)(warps + 1) * sizeof(int));
  o.cm = x; x = p1l_align(x + (long long)warps * kP1TileWords * sizeof(ukey));
  o.ccnt = x; x = p1l_align(x + (long long)warps * 32 * sizeof(int));
  o.cst = x; x = p1l_align(x + (long long)warps * 32 * ksz);
  o.cco = x; x = p1l_align(x + (long long)warps * 32 * sizeof(int));
  o.cex = x; x = p1l_align(x + 32 * sizeof(int));
  o.misc = x; x = p1l_align(x + 2 * sizeof(long long));
  o.wt = x; x = p1l_align(x + (long long)(R + 1) * sizeof(float));  // pruning: w(dx) at level 0
  o.total = x;
  return o;
}

// The open sources of one column as seen from it: bit d - 1 of `up` (`dn`) for the source d
// columns above (below) it, `cen` for the column itself; NH words each (R <= 64 NH).
template <int NH>
struct CMask {
  ukey up[NH], dn[NH];
  int cen;
};

// least distance of an open source (kNoLabel if none)
template <int NH>
DXD int cnearest(const CMask<NH>& m) {
  if (m.cen) return 0;
  int a = kNoLabel, b = kNoLabel;
#pragma unroll
  for (int q = NH - 1; q >= 0; --q) {
    if (m.up[q]) a = 64 * q + __ffsll((long long)m.up[q]);
    if (m.dn[q]) b = 64 * q + __ffsll((long long)m.dn[q]);
  }
  return a < b ? a : b;
}

// 64 bits of the multiword mask T starting at bit position p (zeros outside)
DXD ukey bits64(const ukey* T, int p) {
  const int w = p >> 6, off = p & 63;  // floor division (p may be negative)
  const ukey lo = (w >= 0 && w < kP1TileWords) ? T[w] : 0ULL;
  const ukey hi = (w + 1 >= 0 && w + 1 < kP1TileWords) ? T[w + 1] : 0ULL;
  return off ? (lo >> off) | (hi << (64 - off)) : lo;
}

// The column at tile position pc: its open sources from the tile-relative mask T (bit q:
// source s0 + q), within reach R.
template <int NH>
DXD CMask<NH> cmask_from(const ukey* T, int pc, int R) {
  CMask<NH> m;
  m.cen = (int)(bits64(T, pc) & 1ULL);
#pragma unroll
  for (int q = 0; q < NH; ++q) {
    const int keep = R - 64 * q;  // bits of this word within reach
    const ukey mk = keep >= 64 ? ~0ULL : (keep <= 0 ? 0ULL : ((1ULL << keep) - 1));
    m.up[q] = bits64(T, pc + 1 + 64 * q) & mk;
    // below: bit d - 1 is source pc - d, i.e. the 64 bits ending at pc - 1 - 64 q reversed
    m.dn[q] = __brevll(bits64(T, pc - 64 - 64 * q)) & mk;
  }
  return m;
}

// Dominance of S_mid pieces (Sec. 3.3: pass 2 unites, at every level t, the capsule slices
// [a - w, b + w] with w = h sqrt(k^2 - dx^2 - t^2)).  A piece q with a smaller label than
// piece p (dx_q < dx_p) has w_q(t) - w_p(t) non-decreasing in t, so if q's slice contains
// p's at level 0 it contains it at every level p reaches, and dropping p leaves every level's
// union unchanged.  The test runs on float approximations of a - w(0) and b + w(0) with a
// margin E above twice their error bound, so that it only drops pieces that are dominated
// exactly.  Each lane keeps its last kept piece in registers: a new piece that dominates it
// replaces it, a new piece it dominates is not emitted.
struct Prune {
  const float* w;  // float half-widths at level 0 by label: w[dx] = h sqrt(k^2 - dx^2) (null:
                   // no pruning)
  float E;         // margin of the float test
};
struct PTop {
  float lo, hi;  // the slice at level 0 (float)
  int l;         // its label
  bool have, fixed;  // a kept piece; fixed: its start lies before the chunk (never replaced)
};

// One lane's walk over the sorted events [c0, c1) (a chunk that starts at a group boundary)
// for the column at tile position pc.  m / Om: the open sources and the label just below the
// chunk; run_a: the start of the run open there.  WRITE: the first cap pieces go to oa, ob,
// ol.  last_start: the last run start in the chunk (~0 if none).  Returns the pieces.  The
// pruning decisions depend only on the events, so the counting and writing walks agree (a run
// open at the chunk's start is tested with the chunk's first height as its start: its slice
// is at least that large).
template <typename T, int NH, bool WRITE>
DXD int chunk_walk(const typename EvK<T>::type* ek, const unsigned short* ep, int c0, int c1,
                   int pc, int R, bool act, CMask<NH> m, int Om, typename EvK<T>::type run_a,
                   typename EvK<T>::type& last_start, typename H<T>::K* oa,
                   typename H<T>::K* ob, short* ol, int cap, const Prune& pr) {
  typedef typename EvK<T>::type EK;
  int gmin = kNoLabel;
  int cnt = 0;
  last_start = EvK<T>::none();
  if (c0 >= c1) return 0;
  EK gkey = ek[c0];
  bool carried = Om < kNoLabel;  // the first run closed began before the chunk
  PTop top{0.0f, 0.0f, 0, false, false};
  // float approximations of the current run's start (for a carried run: the chunk's first
  // height) and of the current height, converted once a group
  float run_af = pr.w ? EvK<T>::approx(gkey) : 0.0f;
  auto emit = [&](EK a, EK b, float af, float bf, int l, bool fixed) {
    if (pr.w) {
      const float w = pr.w[l];
      const float lo = af - w, hi = bf + w;
      if (top.have && !top.fixed && l < top.l && lo <= top.lo - pr.E && hi >= top.hi + pr.E) {
        --cnt;  // the new piece dominates the last kept one: it takes its place
      } else if (top.have && top.l < l && !fixed && top.lo <= lo - pr.E && top.hi >= hi + pr.E) {
        return;  // dominated by the last kept piece
      }
      top = PTop{lo, hi, l, true, fixed};
    }
    if (WRITE && cnt < cap) {
      oa[cnt] = EvK<T>::out(a);
      ob[cnt] = EvK<T>::out(b);
      ol[cnt] = (short)l;
    }
    ++cnt;
  };
  auto close_group = [&](EK v) {
    const int Ok = cnearest<NH>(m);
    const bool pt = gmin < (Om < Ok ? Om : Ok);
    const bool ch = Ok != Om || pt;
    const float vf = (pr.w && (ch || pt)) ? EvK<T>::approx(v) : 0.0f;
    if (Om < kNoLabel && ch) {  // the run below v ends at v
      emit(run_a, v, run_af, vf, Om, carried);
      carried = false;
    }
    if (pt) emit(v, v, vf, vf, gmin, false);  // the point [v, v]
    if (Ok < kNoLabel && ch) {  // a run starts at v
      run_a = v;
      run_af = vf;
      last_start = v;
      carried = false;
    }
    Om = Ok;
    gmin = kNoLabel;
  };
  // A height's events change nothing for a lane when all of them are farther than its label
  // below (a source beyond the nearest open one neither becomes nearest when it opens nor was
  // nearest when it closes, and gives no point piece): the height is closed only when some
  // lane saw an event within its label (warp-uniform vote; exact).
  bool dirty = false;
  for (int t = c0; t < c1; ++t) {
    const EK key = ek[t];
    const int src = ep[t];
    if (key != gkey) {  // warp-uniform: every lane reads the same event
#if DEXEL_P1_LAZY
      if (__any_sync(0xffffffffu, dirty)) close_group(gkey);
      dirty = false;
#else
      close_group(gkey);
#endif
      gkey = key;
    }
    const int d = src - pc;
    const int ad = d < 0 ? -d : d;
    if (act && ad <= R) {
      if (d == 0) {
        m.cen ^= 1;
      } else {
        const int b = ad - 1;
        const ukey bit = 1ULL << (b & 63);
#pragma unroll
        for (int q = 0; q < NH; ++q) {
          const ukey x = (b >> 6) == q ? bit : 0ULL;
          m.up[q] ^= d > 0 ? x : 0ULL;
          m.dn[q] ^= d < 0 ? x : 0ULL;
        }
      }
#if DEXEL_P1_LAZY
      if (ad <= Om) {
        dirty = true;
        gmin = ad < gmin ? ad : gmin;
      }
#else
      gmin = ad < gmin ? ad : gmin;
#endif
    }
  }
#if DEXEL_P1_LAZY
  if (__any_sync(0xffffffffu, dirty)) close_group(gkey);
#else
  close_group(gkey);
#endif
  return cnt;
}

// The warps of one tile group: W warps (1, 2, 4 or 8) synchronised by named barrier gid + 1
// (a single warp by __syncwarp).
struct TGroup {
  int W, gid, warp, gtid;  // warps, group index in the block, warp and thread within the group
  long long ring;          // the group's index in the grid (its ring region)
  DXD void sync() const {
    if (W == 1) {
      __syncwarp();
    } else {
      asm volatile("bar.sync %0, %1;" ::"r"(gid + 1), "r"(W * 32) : "memory");
    }
  }
};

// One tile of k_pass1l: columns i0 .. i0 + 31 of row j, the group's warps one chunk each.
// One level of the merge of the window's event runs: the events of source r (in height order)
// span [bo[r] - e0, bo[r + 1] - e0) of ks / ps; after the levels of widths 1, 2, 4, ... (runs
// of w sources merged in pairs into runs of 2w) the events are in height order.  The thread
// writes the outputs [o0, o1) of the level into kd / pd: for each pair of runs its output
// position is split into the two runs by a binary search along the merge path (ties: the
// lower run first), then the two runs are merged one output at a time.
template <typename EK>
DXD void p1l_merge_level(const EK* ks, const unsigned short* ps, EK* kd, unsigned short* pd,
                         const int* bo, int e0, int nr, int w, int o0, int o1) {
  auto bnd = [&](int r) { return bo[r < nr ? r : nr] - e0; };
  const int np = (nr + 2 * w - 1) / (2 * w);
  // the pair that holds output o0: the last whose start is at or below it
  int lo = 0, hi = np - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (bnd(2 * w * mid) <= o0) lo = mid; else hi = mid - 1;
  }
  int o = o0;
  for (int p = lo; o < o1 && p < np; ++p) {
    const int a0 = bnd(2 * w * p), a1 = bnd(2 * w * p + w), a2 = bnd(2 * w * p + 2 * w);
    if (o >= a2) continue;
    const int nL = a1 - a0, nR = a2 - a1, k = o - a0;
    // left events among the pair's first k outputs
    int i0 = k - nR > 0 ? k - nR : 0, i1 = k < nL ? k : nL;
    while (i0 < i1) {
      const int mid = (i0 + i1) >> 1;
      if (ks[a0 + mid] <= ks[a1 + k - 1 - mid]) i0 = mid + 1; else i1 = mid;
    }
    int i = i0, j = k - i0;
    const int oe = o1 < a2 ? o1 : a2;
    for (; o < oe; ++o) {
      const bool left = j >= nR || (i < nL && ks[a0 + i] <= ks[a1 + j]);
      const int src = left ? a0 + i : a1 + j;
      kd[o] = ks[src];
      pd[o] = ps[src];
      i += left ? 1 : 0;
      j += left ? 0 : 1;
    }
  }
}

template <typename T, int NH>
DXD void pass1l_tile(const P1Params<T>& P, long long tile, int ecap, unsigned char* smem,
                     const TGroup& G, ArenaCursor& cur) {
  const int lane = threadIdx.x & 31, warp = G.warp;
  const int W = G.W;
  const int gthreads = W * 32;
  typedef typename EvK<T>::type EK;
  const int nbuf = P.nbuf == 2 ? 2 : 1;
  const P1LLayout Lo = p1l_layout(P.K, ecap, W, (int)sizeof(EK), nbuf);
  const int room = nbuf * ecap;  // events of the buffers
  EK* ek = (EK*)(smem + Lo.ek);
  unsigned short* ep = (unsigned short*)(smem + Lo.ep);
  int* eoff = (int*)(smem + Lo.eoff);
  int* cb = (int*)(smem + Lo.cb);
  ukey* cm = (ukey*)(smem + Lo.cm);
  int* ccnt = (int*)(smem + Lo.ccnt);
  EK* cst = (EK*)(smem + Lo.cst);
  int* cco = (int*)(smem + Lo.cco);
  int* cex = (int*)(smem + Lo.cex);
  long long* misc = (long long*)(smem + Lo.misc);
  typedef typename H<T>::K Key;
  // the group's ring: W x 32 regions of r_cap pieces
  const long long rg0 = (long long)G.ring * W * 32 * P.r_cap;
  Key* rg_a = P.r_a ? P.r_a + rg0 : nullptr;
  Key* rg_b = P.r_b ? P.r_b + rg0 : nullptr;
  short* rg_l = P.r_l ? P.r_l + rg0 : nullptr;
  const Lanes L{lane, 32};
  const int R = P.K;
  const int xa = P.xb > 0 ? P.xa : 0, xb = P.xb > 0 ? P.xb : P.nx;
  const int tpr = (xb - xa + 31) >> 5;
  const int j = (int)(tile / tpr);
  const int i0 = xa + (int)(tile % tpr) * 32;
  const int i1 = min(xb, i0 + 32);
  const int s0 = max(0, i0 - R), s1 = min(P.nx, i1 + R);
  const int ns = s1 - s0;
  const long long rb = (long long)j * P.nx;
  if (P.redo && (P.rowmark == nullptr || P.rowmark[j] == 0)) return;  // nothing to redo here
  G.sync();  // the previous tile is done with the shared memory
  if (P.prune_w) {  // the pruning test's half-widths at level 0, by label
    float* wt = (float*)(smem + Lo.wt);
    for (int l = G.gtid; l <= R; l += W * 32) wt[l] = P.prune_w[l * l];
  }
  if (warp == 0) {  // event slots of the window's sources (exclusive prefix)
    int carry = 0;
    for (int base = 0; base < ns; base += 32) {
      const int q = base + lane;
      int v = 0;
      if (q < ns) {
        const int n = P.col_off[rb + s0 + q + 1] - P.col_off[rb + s0 + q];
        v = P.erode ? 2 * (n + 1) : 2 * n;
      }
      const int inc = w_incl_add(v, lane);
      if (q < ns) eoff[q] = carry + inc - v;
      carry += w_bcast(inc, 31);
    }
    if (lane == 0) eoff[ns] = carry;
  }
  G.sync();
  for (int ia = i0; ia < i1;) {
    // the widest run of columns from ia whose window's events fit (block-uniform); a redo
    // takes only the columns marked by the first launch
    int ib = i1;
    if (P.redo) {
      while (ia < i1 && P.m_start[(long long)ia * P.ny + j] != -1) ++ia;
      if (ia >= i1) break;
      ib = ia + 1;
      while (ib < i1 && P.m_start[(long long)ib * P.ny + j] == -1) ++ib;
    }
    const int qa = max(0, ia - R) - s0;
    if (P.tile_redo && !P.redo && eoff[min(P.nx, ib + R) - s0] - eoff[qa] > ecap) {
      // the whole tile to the redo launch, whose room holds its window (no narrower runs:
      // at wide reaches they would stage most of the window again)
      for (int i = ia + G.gtid; i < ib; i += gthreads) {
        P.m_start[(long long)i * P.ny + j] = -1;
        P.m_cnt[(long long)i * P.ny + j] = 0;
      }
      if (G.gtid == 0) {
        set_status(&P.ctr->status, ST_OVERFLOW_SLOT);
        if (P.rowmark) P.rowmark[j] = 1;
        atomicAdd(&P.ctr->p1_marked, 1);
      }
      break;
    }
    while (ib > ia + 1 && eoff[min(P.nx, ib + R) - s0] - eoff[qa] > ecap) ib = ia + ((ib - ia) >> 1);
    const int qe = min(P.nx, ib + R) - s0;
    const int e0 = eoff[qa];
    const int E = eoff[qe] - e0;
    if (E > ecap) {  // one column's window holds more events than fit: the sweep takes over
      if (G.gtid == 0) {
        set_status(&P.ctr->status, ST_OVERFLOW_SLOT);
        P.m_start[(long long)ia * P.ny + j] = -1;  // marks the column (count 0)
        atomicAdd(&P.ctr->p1_marked, 1);
        P.m_cnt[(long long)ia * P.ny + j] = 0;
        if (P.rowmark) P.rowmark[j] = 1;
      }
      ia = ib;
      continue;
    }
    const int n2 = pow2_at_least(E);  // (the sorting network's width; only E <= ecap events stored)
    PHASE_BEGIN();
    // stage the events, one thread per source (payload: the source's tile position)
    for (int q = qa + G.gtid; q < qe; q += gthreads) {
      const long long c = rb + s0 + q;
      const int g0 = P.col_off[c], g1 = P.col_off[c + 1];
      int o = eoff[q] - e0;
      const int oend = eoff[q + 1] - e0;
      const unsigned short src = (unsigned short)q;
      if (!P.erode) {
        for (int g = g0; g < g1; ++g) {
          ek[o] = EvK<T>::of(P.z[2LL * g]);
          ep[o++] = src;
          ek[o] = EvK<T>::of(P.z[2LL * g + 1]);
          ep[o++] = src;
        }
      } else {
        // closure of the complement: (-inf, a0], [b0, a1], ..., [b_last, +inf); zero-length
        // segments leave no gap
        EK lo = EvK<T>::ninf();
        for (int g = g0; g < g1; ++g) {
          const EK a = EvK<T>::of(P.z[2LL * g]), b = EvK<T>::of(P.z[2LL * g + 1]);
          if (a == b) continue;
          ek[o] = lo;
          ep[o++] = src;
          ek[o] = a;
          ep[o++] = src;
          lo = b;
        }
        ek[o] = lo;
        ep[o++] = src;
        ek[o] = EvK<T>::pinf();
        ep[o++] = src;
      }
      for (; o < oend; ++o) { ek[o] = EvK<T>::none(); ep[o] = 0xFFFFu; }
    }
    // the events in height order (the order within a height does not matter): merged from
    // the sources' runs when the buffers hold the window twice, else a bitonic sort in place
    const bool merge = 2 * E <= room;
    G.sync();
    PHASE(0);
    const EK* eks = ek;
    const unsigned short* eps = ep;
    int Er;
    if (merge) {
      EK* ka = ek;
      unsigned short* pa = ep;
      EK* kb = ek + (room >> 1);
      unsigned short* pb = ep + (room >> 1);
      const int nr = qe - qa;
      const int per = (E + gthreads - 1) / gthreads;
      const int o0 = min(E, G.gtid * per), o1 = min(E, o0 + per);
      for (int w = 1; w < nr; w <<= 1) {
        p1l_merge_level<EK>(ka, pa, kb, pb, eoff + qa, e0, nr, w, o0, o1);
        G.sync();
        EK* tk = ka; ka = kb; kb = tk;
        unsigned short* tp = pa; pa = pb; pb = tp;
      }
      eks = ka;
      eps = pa;
      Er = lower_bound(eks, E, EvK<T>::none());  // (a complement's padding sorts last)
    } else {
      // bitonic sort with every comparator ascending (each merge begins by comparing an
      // element with its mirror in the block): the positions from E to the network's width
      // n2 hold a virtual +inf that no comparator moves, so they are neither stored nor
      // touched (a room need not be a power of two)
      for (int k = 2; k <= n2; k <<= 1) {
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
          for (int p = G.gtid; p < (n2 >> 1); p += gthreads) {
            int t, x;
            if (jj == (k >> 1)) {  // the flip: t against its mirror in the block of k
              const int i = p & (jj - 1);
              t = (p >> (__ffs(jj) - 1)) * k + i;
              x = t - i + (k - 1 - i);
            } else {
              t = ((p & ~(jj - 1)) << 1) | (p & (jj - 1));
              x = t | jj;
            }
            if (x < E) {
              const EK kt = ek[t], kx = ek[x];
              if (kt > kx) {
                ek[t] = kx; ek[x] = kt;
                const unsigned short vt = ep[t]; ep[t] = ep[x]; ep[x] = vt;
              }
            }
          }
          G.sync();
        }
      }
      Er = lower_bound(ek, E, EvK<T>::none());  // real events (a complement's padding sorts last)
    }
    PHASE(1);
    // chunk bounds at group boundaries
    if (G.gtid == 0) ((int*)misc)[2] = 0;  // no ring region overflowed yet
    if (warp == 0 && lane <= W) {
      int b = (int)((long long)lane * Er / W);
      while (b > 0 && b < Er && eks[b] == eks[b - 1]) ++b;
      cb[lane] = b;
    }
    G.sync();
    const int c0 = cb[warp], c1 = cb[warp + 1];
    // the chunk's toggles as a tile-relative mask
    {
      ukey lm[kP1TileWords];
#pragma unroll
      for (int q = 0; q < kP1TileWords; ++q) lm[q] = 0;
      for (int t = c0 + lane; t < c1; t += 32) {
        const int src = eps[t];
        const ukey bit = 1ULL << (src & 63);
#pragma unroll
        for (int q = 0; q < kP1TileWords; ++q) lm[q] ^= (src >> 6) == q ? bit : 0ULL;
      }
#pragma unroll
      for (int q = 0; q < kP1TileWords; ++q) {
        const unsigned h = __reduce_xor_sync(0xffffffffu, (unsigned)(lm[q] >> 32));
        const unsigned l = __reduce_xor_sync(0xffffffffu, (unsigned)lm[q]);
        if (lane == 0) cm[warp * kP1TileWords + q] = ((ukey)h << 32) | l;
      }
    }
    G.sync();
    ukey Tm[kP1TileWords];  // sources open at the chunk's start
#pragma unroll
    for (int q = 0; q < kP1TileWords; ++q) Tm[q] = 0;
    for (int c = 0; c < warp; ++c) {
#pragma unroll
      for (int q = 0; q < kP1TileWords; ++q) Tm[q] ^= cm[c * kP1TileWords + q];
    }
    const int i = ia + lane;
    const bool act = i < ib;
    const int pc = i - s0;
    CMask<NH> m0 = cmask_from<NH>(Tm, pc, R);
    if (!act) {
      m0.cen = 0;
#pragma unroll
      for (int q = 0; q < NH; ++q) { m0.up[q] = 0; m0.dn[q] = 0; }
    }
    const int Om0 = cnearest<NH>(m0);
    EK last = EvK<T>::none();
    // one walk into the lane's ring region (the start of a run open at the chunk's start is
    // patched when the pieces are copied), or a counting walk without a ring
    // the group's ring regions must lie within the ring (else the two walks, no ring)
    const bool ring = P.r_a != nullptr && rg0 + (long long)W * 32 * P.r_cap <= P.r_n;
    const long long rbase = ring ? (long long)(warp * 32 + lane) * P.r_cap : 0;
    int n;
    const float pE = P.prune_zmax ? (float)(1.9073486328125e-6 * ((double)__uint_as_float(*P.prune_zmax) + P.prune_kh))
                                  : P.prune_E;  // (2^-19)
    const Prune pr{P.prune_w ? (const float*)(smem + Lo.wt) : nullptr, pE};
    if (ring)
      n = chunk_walk<T, NH, true>(eks, eps, c0, c1, pc, R, act, m0, Om0, (EK)0, last, rg_a + rbase,
                                  rg_b + rbase, rg_l + rbase, P.r_cap, pr);
    else
      n = chunk_walk<T, NH, false>(eks, eps, c0, c1, pc, R, act, m0, Om0, (EK)0, last, nullptr,
                                   nullptr, nullptr, 0, pr);
    ccnt[warp * 32 + lane] = n;
    cst[warp * 32 + lane] = last;
    cco[warp * 32 + lane] = Om0 < kNoLabel ? 1 : 0;
    if (ring && __any_sync(0xffffffffu, n > P.r_cap) && lane == 0) ((int*)misc)[2] = 1;
    PHASE(2);
    G.sync();
    PHASE(3);
    // the column's pieces before this chunk, its total, and the start of the run open at the
    // chunk's start
    int before = 0, tot_col = 0;
    EK run_a = (EK)0;
    for (int c = 0; c < W; ++c) {
      const int v = ccnt[c * 32 + lane];
      if (c < warp) {
        before += v;
        const EK st = cst[c * 32 + lane];
        if (st != EvK<T>::none()) run_a = st;
      }
      tot_col += v;
    }
    const int inc = w_incl_add(tot_col, lane);
    const int tot = w_bcast(inc, 31);
    if (warp == 0) {
      cex[lane] = inc - tot_col;
      const long long s = arena_take(L, &P.ctr->arena_top[1], P.blk, cur, tot);
      if (lane == 0) misc[0] = s;
      const int mx = __reduce_max_sync(0xffffffffu, tot_col);
      if (lane == 0) {
        cur.tally += tot;
        cur.tmax = mx > cur.tmax ? mx : cur.tmax;
      }
    }
    G.sync();
    const long long s = misc[0];
    const bool fits = s + tot <= P.m_cap;
    const bool spilled = ((const int*)misc)[2] != 0;
    if (ring && spilled && fits && G.gtid == 0) atomicAdd(&P.ctr->ring_spills, 1);  // walked twice
    if (fits && ring && !spilled) {
      // the ring regions into the arena: a warp a column, lanes over its pieces (coalesced)
      for (int x = warp; x < 32; x += W) {
        long long d = s + cex[x];
        EK carry = EvK<T>::none();
        for (int c = 0; c < W; ++c) {
          const int cn = ccnt[c * 32 + x];
          const long long sb = (long long)(c * 32 + x) * P.r_cap;
          const bool patch = cco[c * 32 + x] != 0 && carry != EvK<T>::none();
          for (int k = lane; k < cn; k += 32) {
            P.m_a[d + k] = (k == 0 && patch) ? EvK<T>::out(carry) : rg_a[sb + k];
            P.m_b[d + k] = rg_b[sb + k];
            P.m_l[d + k] = rg_l[sb + k];
          }
          d += cn;
          const EK st = cst[c * 32 + x];
          if (st != EvK<T>::none()) carry = st;
        }
      }
    } else if (fits) {
      // (warp-uniform: every lane walks, as the walk's votes need; a lane with no pieces in
      // this chunk writes none)
      const long long o = s + (inc - tot_col) + before;
      EK dummy;
      chunk_walk<T, NH, true>(eks, eps, c0, c1, pc, R, act, m0, Om0, run_a, dummy, P.m_a + o,
                              P.m_b + o, P.m_l + o, 1 << 30, pr);
    }
    if (warp == 0) {
      if (act) {
        const long long q = (long long)i * P.ny + j;
        P.m_start[q] = fits ? s + (inc - tot_col) : 0;
        P.m_cnt[q] = tot_col;
      }
      if (lane == 0 && !fits) set_status(&P.ctr->status, ST_OVERFLOW_ARENA);
    }
    PHASE(4);
    G.sync();
    PHASE(5);
    PHASE_COUNT(10, 1);
    PHASE_COUNT(11, Er);
    ia = ib;
  }
}

}  // namespace dexel
