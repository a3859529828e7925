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
// GB300 mapping: one warp per output column.  Every lane builds the covered sets of its
// sources (lane l takes dy = l - R, l - R + 32, ...) with a one-pass stack union over the
// source's pieces in height order -- a capsule of a later piece always ends above the left
// end of every earlier capsule, so a stack suffices.  The lanes' intervals are sorted by left
// end in shared memory (bitonic) and united.  There is no state carried from column to
// column, so no sequential sweep: the work is the window times the pieces, spread over 32
// lanes, with the sources of neighbouring output columns shared through L1.
//
// Decisions are taken on float approximations with a forward error bound; the double
// endpoints a - w and b + w are computed only when the float values cannot decide and for
// the final endpoints, so the result equals the all-double computation bit for bit.
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
  int stcap;      // stack entries per lane
  int bcap;       // intervals per output column (power of two)
  int tile;       // output columns per block tile
  int stage_cap;  // pieces the block can stage in shared memory
  int warps_per_block;
  int redo;  // k_pass2g: redo only the columns whose count is -1
};

// a stack entry of the per-source union: float approximations of the interval ends and the
// pieces (indices within the source) whose exact ends they approximate
struct PEnt {
  float lf, rf;
  unsigned short li, ri;
};

// one source column seen by the cover: float approximations (staged in shared memory or
// null) and the exact height keys in global memory
template <typename Key>
struct Src {
  const float* af;           // float approximations of the bottoms (or null: derive from a)
  const float* bf;           // ... of the tops
  const unsigned char* d8;   // dx (staged) or null
  const Key* a;              // exact bottoms
  const Key* b;              // exact tops
  const short* dx;           // exact dx
  int np;
};

template <typename Key>
DXI double src_lo(const Src<Key>& S, int p, int t, const double* wtab) {
  const int d = S.dx[p];
  return keyd(S.a[p]) - wtab[d * d + t * t];
}
template <typename Key>
DXI double src_hi(const Src<Key>& S, int p, int t, const double* wtab) {
  const int d = S.dx[p];
  return keyd(S.b[p]) + wtab[d * d + t * t];
}

// Union of the capsules of one source column's pieces at level t, appended as exact
// interval keys through the warp's shared counter.  The union runs in one pass over the
// pieces in height order: a capsule of a later piece ends above the left end of every earlier
// capsule, so it either starts a new interval or merges with the top ones of a stack.
// Comparisons use the float ends with the bound e(x) = eps (|x| + 2 w_max); the exact double
// ends decide when the floats cannot.  Returns false when the stack or the buffer would
// overflow.
template <typename Key>
DXI bool source_cover(const Src<Key>& S, int t, const int* reach, const double* wtab,
                      const float* wtabf, float wmax2, PEnt* st, int stcap, ukey* bl, ukey* br,
                      int* bcount, int bcap) {
  const float eps = 2.5e-7f;
  int top = -1;
  for (int p = 0; p < S.np; ++p) {
    const int dx = S.d8 ? (int)S.d8[p] : (int)S.dx[p];
    if (t > reach[dx]) continue;  // this piece no longer reaches level t
    const float wf = wtabf[dx * dx + t * t];
    const float af = S.af ? S.af[p] : keyf(S.a[p]);
    const float bf = S.bf ? S.bf[p] : keyf(S.b[p]);
    PEnt e;
    e.lf = af - wf;  // -inf stays -inf, +inf stays +inf
    e.rf = bf + wf;
    e.li = (unsigned short)p;
    e.ri = (unsigned short)p;
    while (top >= 0) {
      const PEnt s = st[top];
      const float ee = eps * (fabsf(e.lf) + fabsf(s.rf) + wmax2);
      bool overlap;
      if (e.lf == -__builtin_huge_valf() || s.rf == __builtin_huge_valf()) overlap = true;
      else if (e.lf - s.rf > ee) overlap = false;
      else if (s.rf - e.lf > ee) overlap = true;
      else overlap = src_lo(S, e.li, t, wtab) <= src_hi(S, s.ri, t, wtab);
      if (!overlap) break;
      // merged interval: left = min, right = max
      const float el = eps * (fabsf(e.lf) + fabsf(s.lf) + wmax2);
      bool left_from_s;
      if (s.lf == -__builtin_huge_valf()) left_from_s = true;
      else if (e.lf == -__builtin_huge_valf()) left_from_s = false;
      else if (e.lf - s.lf > el) left_from_s = true;
      else if (s.lf - e.lf > el) left_from_s = false;
      else left_from_s = src_lo(S, s.li, t, wtab) <= src_lo(S, e.li, t, wtab);
      if (left_from_s) { e.lf = s.lf; e.li = s.li; }
      const float er = eps * (fabsf(e.rf) + fabsf(s.rf) + wmax2);
      bool right_from_s;
      if (s.rf == __builtin_huge_valf()) right_from_s = true;
      else if (e.rf == __builtin_huge_valf()) right_from_s = false;
      else if (s.rf - e.rf > er) right_from_s = true;
      else if (e.rf - s.rf > er) right_from_s = false;
      else right_from_s = src_hi(S, s.ri, t, wtab) >= src_hi(S, e.ri, t, wtab);
      if (right_from_s) { e.rf = s.rf; e.ri = s.ri; }
      --top;
    }
    if (top + 1 >= stcap) return false;
    st[++top] = e;
  }
  if (top < 0) return true;
  int pos;
#if defined(__CUDA_ARCH__)
  pos = atomicAdd(bcount, top + 1);
#else
  pos = *bcount;
  *bcount += top + 1;
#endif
  if (pos + top + 1 > bcap) return false;
  for (int q = 0; q <= top; ++q) {
    bl[pos + q] = dkey(src_lo(S, st[q].li, t, wtab));
    br[pos + q] = dkey(src_hi(S, st[q].ri, t, wtab));
  }
  return true;
}

// The same union with the stack held in registers (kRegStack entries).  An interval whose
// right end lies more than w_max below the current bottom a can never be reached by a later
// capsule (their left ends are at least a - w_max) and is emitted at once; if the stack is
// still full the function gives up (false) and the caller falls back to the shared-memory
// version.
constexpr int kRegStack = 8;

// SHARED: the count is shared by several lanes (atomic); otherwise it is the lane's own.
template <typename Key, bool SHARED>
DXI void emit_interval(const Src<Key>& S, const PEnt& e, int t, const double* wtab, ukey* bl,
                       ukey* br, int* bcount, int bcap, bool& ok) {
  int pos;
#if defined(__CUDA_ARCH__)
  if (SHARED) pos = atomicAdd(bcount, 1);
  else pos = (*bcount)++;
#else
  pos = (*bcount)++;
#endif
  if (pos >= bcap) { ok = false; return; }
  bl[pos] = dkey(src_lo(S, e.li, t, wtab));
  br[pos] = dkey(src_hi(S, e.ri, t, wtab));
}

template <typename Key, bool SHARED>
DXI bool source_cover_reg(const Src<Key>& S, int t, const int* reach, const double* wtab,
                          const float* wtabf, float wmaxf, ukey* bl, ukey* br, int* bcount,
                          int bcap) {
  const float eps = 2.5e-7f;
  const float wmax2 = 2.0f * wmaxf;
  PEnt st[kRegStack];
  int depth = 0;
  bool ok = true;
  for (int p = 0; p < S.np; ++p) {
    const int dx = S.d8 ? (int)S.d8[p] : (int)S.dx[p];
    if (t > reach[dx]) continue;
    const float wf = wtabf[dx * dx + t * t];
    const float af = S.af ? S.af[p] : keyf(S.a[p]);
    const float bf = S.bf ? S.bf[p] : keyf(S.b[p]);
    PEnt e;
    e.lf = af - wf;
    e.rf = bf + wf;
    e.li = (unsigned short)p;
    e.ri = (unsigned short)p;
    while (depth > 0) {
      const PEnt s = st[0];
      const float ee = eps * (fabsf(e.lf) + fabsf(s.rf) + wmax2);
      bool overlap;
      if (e.lf == -__builtin_huge_valf() || s.rf == __builtin_huge_valf()) overlap = true;
      else if (e.lf - s.rf > ee) overlap = false;
      else if (s.rf - e.lf > ee) overlap = true;
      else overlap = src_lo(S, e.li, t, wtab) <= src_hi(S, s.ri, t, wtab);
      if (!overlap) break;
      const float el = eps * (fabsf(e.lf) + fabsf(s.lf) + wmax2);
      bool left_from_s;
      if (s.lf == -__builtin_huge_valf()) left_from_s = true;
      else if (e.lf == -__builtin_huge_valf()) left_from_s = false;
      else if (e.lf - s.lf > el) left_from_s = true;
      else if (s.lf - e.lf > el) left_from_s = false;
      else left_from_s = src_lo(S, s.li, t, wtab) <= src_lo(S, e.li, t, wtab);
      if (left_from_s) { e.lf = s.lf; e.li = s.li; }
      const float er = eps * (fabsf(e.rf) + fabsf(s.rf) + wmax2);
      bool right_from_s;
      if (s.rf == __builtin_huge_valf()) right_from_s = true;
      else if (e.rf == __builtin_huge_valf()) right_from_s = false;
      else if (s.rf - e.rf > er) right_from_s = true;
      else if (e.rf - s.rf > er) right_from_s = false;
      else right_from_s = src_hi(S, s.ri, t, wtab) >= src_hi(S, e.ri, t, wtab);
      if (right_from_s) { e.rf = s.rf; e.ri = s.ri; }
#pragma unroll
      for (int q = 0; q < kRegStack - 1; ++q) st[q] = st[q + 1];
      --depth;
    }
    if (depth == kRegStack) {
      // the bottom entry can be emitted if no later capsule can reach it
      const PEnt& bot = st[kRegStack - 1];
      const float reach_lo = af - wmaxf;
      if (!(bot.rf != __builtin_huge_valf() &&
            reach_lo - bot.rf > eps * (fabsf(reach_lo) + fabsf(bot.rf) + wmax2)))
        return false;
      emit_interval<Key, SHARED>(S, bot, t, wtab, bl, br, bcount, bcap, ok);
      --depth;
    }
#pragma unroll
    for (int q = kRegStack - 1; q > 0; --q) st[q] = st[q - 1];
    st[0] = e;
    ++depth;
  }
#pragma unroll
  for (int q = 0; q < kRegStack; ++q)
    if (q < depth) emit_interval<Key, SHARED>(S, st[q], t, wtab, bl, br, bcount, bcap, ok);
  return ok;
}

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

// Per-warp scratch of the gather: per-lane stacks, the interval buffer (left keys, right
// keys), union flags and outputs.
struct GatherWarp {
  PEnt* st;      // 32 * stcap
  ukey* bl;      // bcap
  ukey* br;      // bcap
  int* f0;       // bcap
  int* f1;       // bcap
  ukey* ul;      // bcap
  ukey* ur;      // bcap
  int* count;    // 1
};

DXI int pow2_at_least(int n) {
  int m = 1;
  while (m < n) m <<= 1;
  return m;
}

DXI long long gather_warp_bytes(int stcap, int bcap) {
  return 32LL * stcap * sizeof(PEnt) + 4LL * bcap * sizeof(ukey) + 2LL * bcap * sizeof(int) + 16;
}

DXI GatherWarp gather_warp(unsigned char* p, int stcap, int bcap) {
  GatherWarp g;
  g.bl = (ukey*)p; p += (long long)bcap * sizeof(ukey);
  g.br = (ukey*)p; p += (long long)bcap * sizeof(ukey);
  g.ul = (ukey*)p; p += (long long)bcap * sizeof(ukey);
  g.ur = (ukey*)p; p += (long long)bcap * sizeof(ukey);
  g.st = (PEnt*)p; p += 32LL * stcap * sizeof(PEnt);
  g.f0 = (int*)p; p += (long long)bcap * sizeof(int);
  g.f1 = (int*)p; p += (long long)bcap * sizeof(int);
  g.count = (int*)p;
  return g;
}

// One output column (i, j): the covers of the window's sources (lane l takes dy = l - R,
// l - R + 32, ...), a sort by left end, the union, and the write to the output arena.
// src(q) gives the view of source column j' = q.  bcap must be a power of two.
template <typename T, typename SrcFn>
DXN void gather_column(const Lanes& L, const P2GParams<T>& P, int i, int j, const GatherWarp& G,
                       int stcap, int bcap, float wmax2, SrcFn src, ArenaCursor& cur) {
  typedef typename H<T>::K Key;
  if (L.lane == 0) *G.count = 0;
  wsync();
  bool ok = true;
  for (int dy = -P.R + L.lane; dy <= P.R; dy += L.nl) {
    const int jj = j + dy;
    if (jj < 0 || jj >= P.ny) continue;
    const Src<Key> S = src(jj);
    ok = source_cover<Key>(S, dy < 0 ? -dy : dy, P.reach, P.wtab, P.wtabf, wmax2,
                           G.st + L.lane * stcap, stcap, G.bl, G.br, G.count, bcap);
    if (!ok) break;
  }
  wsync();
  if (w_any(!ok)) {
    if (L.lane == 0) { set_status(&P.ctr->status, ST_OVERFLOW_SLOT); note_max(&P.ctr->max_state, 2 * bcap); }
    return;
  }
  const int total = *G.count;
  const int n2 = pow2_at_least(total);
  for (int t = total + L.lane; t < n2; t += L.nl) { G.bl[t] = ~0ULL; G.br[t] = ~0ULL; }
  wsync();
  if (n2 > 1) warp_bitonic(L, G.bl, G.br, n2);
  const int no = total > 0 ? union_runs(L, G.bl, G.br, total, true, G.f0, G.f1, G.ul, G.ur, G.br, nullptr) : 0;
  const long long s = arena_take(L, &P.ctr->arena_top[3], P.blk, cur, no);
  const bool fits = s + no <= P.o_cap;
  if (!fits) {
    if (L.lane == 0) set_status(&P.ctr->status, ST_OVERFLOW_ARENA);
  } else {
    for (int q = L.lane; q < no; q += L.nl) { P.o_l[s + q] = G.ul[q]; P.o_r[s + q] = G.ur[q]; }
  }
  if (L.lane == 0) {
    const long long c = (long long)j * P.nx + i;
    P.o_start[c] = fits ? s : 0;
    P.o_cnt[c] = no;
    note_max(&P.ctr->max_out, no);
    add_total(&P.ctr->out_total, no);
  }
  wsync();
}

}  // namespace dexel
