// Pass 2 of the dexel offset: per column line, forward and backward sweeps over the S_mid
// pieces (Sec. 3.3 "2D Power Diagram", Fig. segments-separate, Fig. power-vertex).
//
// A piece (a, b, dx) of S_mid at line position j' reaches position j with the capsule slice
// [a - w, b + w], w = h sqrt(k^2 - n), n = dx^2 + (j - j')^2 <= k^2.  The capsule is the
// extruded rectangle [a, b] (alive while n <= k^2) plus the disks of its two endpoints.
//
// Rectangles: a max-expiry envelope over z (for every height, the furthest sweep position
// still reached), merged with the new column's pieces at every step.
//
// Endpoint disks: seeds e = (z_e, o_e, dx_e) with power pi_e(z) = (z - z_e)^2 - h^2 (k^2 - n_e)
// (Eq. of power cells, App. B).  Along the current line the covered set is
// {z : min_e pi_e(z) <= 0}; only the seeds of the lower envelope of the pi_e matter.  The
// envelope A is kept across steps; at every step the new column's seeds and the seeds due
// to wake up are merged in and parity rounds remove every seed dominated by its two
// neighbours (the three-seed power-vertex test of App. B, written without division).  For
// a removed seed s the domination margin V by its neighbours is linear in the sweep
// position (dV/du = 2 h^2 (Q (o_p - o_s) + P (o_n - o_s))): if dV/du >= 0 the seed stays
// dominated for the rest of the sweep and is discarded (in particular when both neighbours
// are newer -- older seeds only lose ground); otherwise it sleeps until the first position
// where V may turn negative and is tested again then (the "not yet born" seeds of
// Fig. power-vertex, which the paper handles with power-vertex events).  A sleeping seed's
// disk stays inside the union of the envelope's disks, so the envelope alone gives the
// covered set.
//
// Predicates are evaluated in float with a forward error bound and re-evaluated in double
// only when the float value is too close to zero to decide.  Heights are compared as
// order-preserving keys (heights.cuh); double arithmetic is left to the undecided
// predicates and the emitted endpoints z -/+ w.
#pragma once
#include "sweep.cuh"

namespace dexel {

template <typename T>
struct P2Params {
  typedef typename H<T>::K Key;
  int nx, ny;
  int R;           // reach in grid steps (largest integer with R^2 <= k^2)
  double kk;       // k^2
  double h2;       // h^2
  float h2f;
  int chunk, nchunks;
  const double* wtab;  // w[n] = h sqrt(k^2 - n), n = 0..floor(k^2)
  const int* reach;    // reach[dx] = largest dy with dx^2 + dy^2 <= k^2
  const Key* m_a; const Key* m_b; const short* m_l;
  const long long* m_start; const int* m_cnt;
  // arena 2: forward results (scratch), arena 3: final per-column intervals (height keys)
  ukey* f_l; ukey* f_r; long long f_cap;
  ukey* o_l; ukey* o_r; long long o_cap;
  long long* o_start;  // per output column, row-major c = j*nx + i
  int* o_cnt;
  long long blk;
  Counters* ctr;
  char* slots; long long slot_bytes;
  int capP;   // pieces of one S_mid column
  int capR;   // rectangle envelope
  int capA;   // envelope seeds (with the step's new and woken seeds)
  int capS;   // sleeping seeds
};

template <typename Key>
struct P2Slot {
  Key *pa, *pb; int* pd;                 // the column's pieces
  Key *ra, *rb, *qa, *qb; int *rt, *qt;  // rectangle envelope (state, next)
  Key *na, *nb; int* nt;                 // new rectangles
  Key *az, *bz; int *ao, *ad, *bo, *bd;  // envelope seeds (two buffers): height, order, dx
  Key* nz; int* nd;                      // new seeds of the column
  Key* wz; int *wo, *wd;                 // woken seeds
  Key* sz; int *so, *sd, *sw;            // sleeping seeds due soon: height, order, dx, wake-up
  Key* fz; int *fo, *fd, *fw;            // sleeping seeds due later (scanned every kFarEvery steps)
  ukey *el, *er, *gl, *gr, *hl, *hr, *xl, *xr;  // interval scratch
  Key* X;
  int *c0, *c1, *c2, *c3, *c4, *c5, *E;
  long long* fstart;
  int* fcnt;
};

DXI long long p2_ce(int capR, int capA, int capP, int capS) {
  long long m = 2LL * (capR + capP) + 8;
  const long long b = 2LL * capA + 2LL * capP + 8;
  const long long c = 2LL * (capR + capA) + 8;
  const long long d = (long long)capS + 8;
  m = m > b ? m : b;
  m = m > c ? m : c;
  m = m > d ? m : d;
  return m;
}

template <typename Key>
DXI long long p2_slot_bytes(int capP, int capR, int capA, int capS, int chunk) {
  const long long ce = p2_ce(capR, capA, capP, capS);
  long long b = 0;
  b += (long long)chunk * (sizeof(long long) + sizeof(int)) + 64;
  b += 8LL * ce * sizeof(ukey);
  b += 5LL * ce * sizeof(Key) + 9LL * ce * sizeof(int);
  b += 6LL * capP * sizeof(Key) + 4LL * capP * sizeof(int);
  b += 3LL * capA * sizeof(Key) + 6LL * capA * sizeof(int);
  b += 2LL * capS * sizeof(Key) + 6LL * capS * sizeof(int);
  return (b + 4096 + 255) & ~255LL;
}

template <typename Key>
DXI P2Slot<Key> p2_slot(char* base, int capP, int capR, int capA, int capS, int chunk) {
  P2Slot<Key> s;
  const long long ce = p2_ce(capR, capA, capP, capS);
  char* p = base;
  s.fstart = (long long*)p;
  p += (long long)chunk * sizeof(long long);
  p = (char*)(((unsigned long long)p + 15) & ~15ULL);
  ukey** uu[] = {&s.el, &s.er, &s.gl, &s.gr, &s.hl, &s.hr, &s.xl, &s.xr};
  for (ukey** q : uu) { *q = (ukey*)p; p += ce * sizeof(ukey); }
  Key** kp[] = {&s.pa, &s.pb, &s.na, &s.nb};
  for (Key** q : kp) { *q = (Key*)p; p += (long long)capP * sizeof(Key); }
  s.nz = (Key*)p; p += 2LL * capP * sizeof(Key);
  Key** kr[] = {&s.ra, &s.rb, &s.qa, &s.qb, &s.X};
  for (Key** q : kr) { *q = (Key*)p; p += ce * sizeof(Key); }
  Key** ka[] = {&s.az, &s.bz, &s.wz};
  for (Key** q : ka) { *q = (Key*)p; p += (long long)capA * sizeof(Key); }
  s.sz = (Key*)p; p += (long long)capS * sizeof(Key);
  s.fz = (Key*)p; p += (long long)capS * sizeof(Key);
  p = (char*)(((unsigned long long)p + 15) & ~15ULL);
  s.pd = (int*)p; p += (long long)capP * sizeof(int);
  s.nt = (int*)p; p += (long long)capP * sizeof(int);
  s.nd = (int*)p; p += 2LL * capP * sizeof(int);
  s.rt = (int*)p; p += ce * sizeof(int);
  s.qt = (int*)p; p += ce * sizeof(int);
  int** ia[] = {&s.ao, &s.ad, &s.bo, &s.bd, &s.wo, &s.wd};
  for (int** q : ia) { *q = (int*)p; p += (long long)capA * sizeof(int); }
  int** is[] = {&s.so, &s.sd, &s.sw, &s.fo, &s.fd, &s.fw};
  for (int** q : is) { *q = (int*)p; p += (long long)capS * sizeof(int); }
  int** ie[] = {&s.c0, &s.c1, &s.c2, &s.c3, &s.c4, &s.c5, &s.E};
  for (int** q : ie) { *q = (int*)p; p += ce * sizeof(int); }
  s.fcnt = (int*)p;
  return s;
}

// heights of a piece/seed key as an interval key (always the double encoding)
DXI ukey ikey(ukey k) { return k; }
DXI ukey ikey(float k) { return dkey((double)k); }

// float approximation of a height key by truncation (integer operations only for doubles);
// relative error below 2^-23, magnitudes below 2^-126 flush to 0
DXI float keyf(float k) { return k; }
DXI float keyf(ukey k) {
  const long long s = (long long)k;
  const unsigned long long b = s < 0 ? (k ^ 0x8000000000000000ULL) : ~k;  // double bits
  const unsigned sign = (unsigned)(b >> 63);
  const int e = (int)((b >> 52) & 0x7ff) - 1023 + 127;
  unsigned f;
  if (e <= 0)
    f = sign << 31;
  else if (e >= 255)
    f = (sign << 31) | 0x7f800000u;
  else
    f = (sign << 31) | ((unsigned)e << 23) | (unsigned)((b >> 29) & 0x7fffffULL);
#if defined(__CUDA_ARCH__)
  return __uint_as_float(f);
#else
  float x;
  memcpy(&x, &f, 4);
  return x;
#endif
}
DXI double keyd(float k) { return (double)k; }
DXI double keyd(ukey k) { return dval(k); }

constexpr int FATE_KEEP = -1;
constexpr int kFarEvery = 16;  // the far sleeper pool is scanned once per this many steps
constexpr int FATE_DROP = 0x7fffffff;

DXI int seed_n(int dx, int o, int u) { return dx * dx + (u - o) * (u - o); }

// seed s dominated by a seed t at the same height (n_t <= n_s): dominated while
// n_s - n_t >= 0, a margin that changes by 2 (o_t - o_s) per step
DXI int equal_fate(int ot, int nt, int os, int ns, int u) {
  if (ot >= os) return FATE_DROP;
  const long long V = (long long)ns - nt;
  const long long dec = 2LL * (os - ot);
  const long long w = (long long)u + V / dec + 1;
  return w < FATE_DROP ? (int)w : FATE_DROP - 1;
}

// Fate of seed s against its envelope neighbours p (below, -1 if none) and n (above) at
// sweep position u: FATE_KEEP, FATE_DROP, or the position at which to test it again.
template <typename Key>
DXI int seed_fate(const Key* z, const int* o, const int* d, int p, int s, int n, int u,
                  double h2, float h2f) {
  const Key zs = z[s];
  const int os = o[s];
  const int ns = seed_n(d[s], os, u);
  const bool eqp = p >= 0 && z[p] == zs;
  const bool eqn = n >= 0 && z[n] == zs;
  if (eqp || eqn) {
    int fate = FATE_KEEP;
    if (eqp) {
      const int np = seed_n(d[p], o[p], u);
      if (np <= ns) fate = equal_fate(o[p], np, os, ns, u);
    }
    if (eqn) {
      const int nn = seed_n(d[n], o[n], u);
      if (nn <= ns) {
        const int f = equal_fate(o[n], nn, os, ns, u);
        fate = fate == FATE_KEEP ? f : (f > fate ? f : fate);
      }
    }
    return fate;
  }
  if (p < 0 || n < 0) return FATE_KEEP;
  const int op = o[p], on = o[n];
  const int A = ns - seed_n(d[p], op, u);  // (W_p - W_s) / h^2
  const int B = ns - seed_n(d[n], on, u);  // (W_n - W_s) / h^2
  // float filter for V = h^2 (Q A + P B) - P Q (P + Q),  P = z_s - z_p, Q = z_n - z_s
  const float zpf = keyf(z[p]), zsf = keyf(zs), znf = keyf(z[n]);
  const float Pf = zsf - zpf, Qf = znf - zsf;
  const float uc = 1.1920929e-7f;  // 2^-23: key to float truncation
  const float ur = 5.9604645e-8f;  // 2^-24: float rounding
  const float eP = uc * (fabsf(zsf) + fabsf(zpf)) + ur * fabsf(Pf) + 1e-37f;
  const float eQ = uc * (fabsf(znf) + fabsf(zsf)) + ur * fabsf(Qf) + 1e-37f;
  const float fA = (float)A, fB = (float)B;
  const float PQ = Pf + Qf;
  const float T3 = Pf * Qf * PQ;
  const float Vf = h2f * (Qf * fA + Pf * fB) - T3;
  float E = h2f * (fabsf(fA) * eQ + fabsf(fB) * eP) + (Qf * PQ + Pf * Qf) * eP +
            (Pf * PQ + Pf * Qf) * eQ + 4.0f * (eP + eQ) * (eP + eQ) * (PQ + eP + eQ) +
            8.0f * ur * (h2f * (fabsf(Qf * fA) + fabsf(Pf * fB)) + fabsf(T3));
  E *= 2.0f;
  float Vlo;
  if (Vf > E) {
    Vlo = Vf - E;
  } else if (Vf < -E) {
    return FATE_KEEP;
  } else {
    const double zp = keyd(z[p]), zsd = keyd(zs), zn = keyd(z[n]);
    const double P = zsd - zp, Q = zn - zsd;
    const double V = h2 * (Q * (double)A + P * (double)B) - P * Q * (P + Q);
    if (!(V >= 0.0)) return FATE_KEEP;
    Vlo = 0.0f;
  }
  // dominated now; dV/du = 2 h^2 (Q a + P b)
  const int a = op - os, b = on - os;
  if (a >= 0 && b >= 0) return FATE_DROP;
  const float fa = (float)a, fb = (float)b;
  const float Gf = 2.0f * h2f * (Qf * fa + Pf * fb);
  const float EG = 2.0f * h2f * (fabsf(fa) * eQ + fabsf(fb) * eP) +
                   16.0f * ur * h2f * (fabsf(Qf * fa) + fabsf(Pf * fb)) + 1e-37f;
  if (Gf > 2.0f * EG) return FATE_DROP;
  if (Gf < -2.0f * EG) {
    const float steps = Vlo / (2.0f * EG - Gf) * 0.999f;
    const long long w = (long long)u + 1 + (long long)(steps < 1.0e9f ? steps : 1.0e9f);
    return w < FATE_DROP ? (int)w : FATE_DROP - 1;
  }
  return u + 1;
}

// ---------------------------------------------------------------------------------------
// sorted interval utilities on height keys
// ---------------------------------------------------------------------------------------
DXI ukey w_incl_maxk(ukey v, int lane) {
#if defined(__CUDA_ARCH__)
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const ukey w = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o && w > v) v = w;
  }
#else
  (void)lane;
#endif
  return v;
}
DXI ukey w_bcastk(ukey v, int src) {
#if defined(__CUDA_ARCH__)
  return __shfl_sync(0xffffffffu, v, src);
#else
  (void)src;
  return v;
#endif
}
DXI ukey w_shift_up(ukey v, int lane, ukey fill) {
#if defined(__CUDA_ARCH__)
  const ukey w = __shfl_up_sync(0xffffffffu, v, 1);
  return lane == 0 ? fill : w;
#else
  (void)v;
  (void)lane;
  return fill;
#endif
}

// C := merge of sorted interval lists A and B by left end (A first on ties)
DXN int merge_intervals(const Lanes& L, const ukey* al, const ukey* ar, int na, const ukey* bl,
                        const ukey* br, int nb, ukey* cl, ukey* cr) {
  for (int t = L.lane; t < na; t += L.nl) {
    const int pos = t + lower_bound(bl, nb, al[t]);
    cl[pos] = al[t];
    cr[pos] = ar[t];
  }
  for (int t = L.lane; t < nb; t += L.nl) {
    const int pos = t + upper_bound(al, na, bl[t]);
    cl[pos] = bl[t];
    cr[pos] = br[t];
  }
  wsync();
  return na + nb;
}

// Run-union of closed intervals (touching ones join).  With sorted = true the left ends are
// sorted; otherwise the list is an exact lower envelope in z order, whose disks never
// reach past a gap of the union, so every run is a contiguous range and its left end is
// the minimum over the run (smin scratch needed).
DXN int union_runs(const Lanes& L, const ukey* cl, const ukey* cr, int n, bool sorted,
                   int* start, int* pos, ukey* ul, ukey* ur, ukey* pmax, ukey* smin) {
  ukey carry = 0;
  for (int base = 0; base < n; base += L.nl) {
    const int t = base + L.lane;
    const ukey v = t < n ? cr[t] : 0;
    const ukey inc = w_incl_maxk(v, L.lane);
    const ukey prev = w_shift_up(inc, L.lane, 0);
    if (t < n) {
      const ukey ex = prev > carry ? prev : carry;
      start[t] = (t == 0) || (cl[t] > ex);
      pmax[t] = ex > v ? ex : v;
    }
    const ukey last = w_bcastk(inc, L.nl - 1);
    carry = last > carry ? last : carry;
  }
  wsync();
  if (!sorted) {
    ukey cmin = ~0ULL;
    for (int base = 0; base < n; base += L.nl) {
      const int t = base + L.lane;
      ukey v = t < n ? cl[t] : ~0ULL;
      int f = t < n ? start[t] : 0;
#if defined(__CUDA_ARCH__)
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const ukey w = __shfl_up_sync(0xffffffffu, v, o);
        const int g = __shfl_up_sync(0xffffffffu, f, o);
        if (L.lane >= o) {
          if (!f && w < v) v = w;
          f |= g;
        }
      }
#endif
      if (!f && cmin < v) v = cmin;
      if (t < n) smin[t] = v;
      cmin = w_bcastk(v, L.nl - 1);
    }
    wsync();
  }
  for (int t = L.lane; t < n; t += L.nl) pos[t] = start[t];
  wsync();
  const int nu = scan_excl(L, pos, n);
  for (int t = L.lane; t < n; t += L.nl) {
    const bool last = (t == n - 1) || start[t + 1];
    const int r = pos[t] - (start[t] ? 0 : 1);
    if (sorted) {
      if (start[t]) ul[r] = cl[t];
    } else if (last) {
      ul[r] = smin[t];
    }
    if (last) ur[r] = pmax[t];
  }
  wsync();
  return nu;
}

// Covered set of an exact lower envelope of disks D_t = [l_t, r_t] (z order), as sorted
// disjoint runs.  Seed t owns the cell between its bisectors with t-1 and t+1, so the covered
// set is the ordered union of C_t = D_t ∩ cell_t.  Whether a bisector clips D_t is decided by
// key comparisons alone: the bisector with t-1 lies above l_t iff l_t is strictly inside
// D_{t-1} (t-1 has the lower power there), and below r_t iff r_t is strictly inside D_{t+1}.
// A clipped side touches the neighbour's C; runs start at unclipped left ends and finish at
// unclipped right ends, so every run endpoint is an exact disk endpoint z -/+ w.  If the
// envelope is not exact (a near tie decided the other way) the runs could come out of
// order; that is detected and the disks are then sorted by left end and united directly.
DXN int envelope_runs(const Lanes& L, const ukey* dl, const ukey* dr, int n, int* start,
                      int* stop, int* pos, ukey* ul, ukey* ur, ukey* sl, ukey* sr) {
  for (int t = L.lane; t < n; t += L.nl) {
    const ukey lt = dl[t], rt = dr[t];
    const bool lT = t > 0 && dl[t - 1] < lt && lt < dr[t - 1];
    const bool rT = t + 1 < n && dl[t + 1] < rt && rt < dr[t + 1];
    bool ne;
    if (lT == rT)
      ne = true;
    else if (lT)
      ne = rt >= dr[t - 1];
    else
      ne = lt <= dl[t + 1];
    start[t] = ne && !lT;
    stop[t] = ne && !rT;
  }
  wsync();
  for (int t = L.lane; t < n; t += L.nl) pos[t] = start[t];
  wsync();
  const int nu = scan_excl(L, pos, n);
  for (int t = L.lane; t < n; t += L.nl) {
    if (start[t]) ul[pos[t]] = dl[t];
    if (stop[t]) ur[pos[t] + start[t] - 1] = dr[t];
  }
  wsync();
  int bad = 0;
  for (int r = L.lane; r < nu; r += L.nl) bad |= !(ul[r] <= ur[r]) || (r > 0 && !(ur[r - 1] < ul[r]));
  if (!w_any(bad)) return nu;
  // fallback: rank-sort the disks by left end, then a sorted union
  for (int t = L.lane; t < n; t += L.nl) {
    const ukey x = dl[t];
    int rk = 0;
    for (int v = 0; v < n; ++v) rk += dl[v] < x || (dl[v] == x && v < t);
    sl[rk] = x;
    sr[rk] = dr[t];
  }
  wsync();
  // (the running maximum may overwrite sr: each right end is read before it is replaced)
  return union_runs(L, sl, sr, n, true, start, pos, ul, ur, sr, nullptr);
}

// ---------------------------------------------------------------------------------------
// the work item: column line i, output positions [c0, c1)
// ---------------------------------------------------------------------------------------
template <typename T>
DXN void pass2_item(const Lanes& L, const P2Params<T>& P, const P2Slot<typename H<T>::K>& W,
                    int i, int c0, int c1, ArenaCursor& curF, ArenaCursor& curO) {
  typedef typename H<T>::K Key;
  int* status = &P.ctr->status;
  const int N = P.ny;
  const int R = P.R;
  const long long ce = p2_ce(P.capR, P.capA, P.capP, P.capS);
  long long item_total = 0;
  for (int dir = 1; dir >= -1; dir -= 2) {
    int nr = 0;   // rectangles
    int na = 0;   // envelope seeds
    int nsl = 0;  // sleeping seeds due soon
    int nfar = 0;  // sleeping seeds due later
    int next_far = 0;  // position of the next scan of the far pool
    Key* Az = W.az; int* Ao = W.ao; int* Ad = W.ad;  // envelope (current buffer)
    Key* Bz = W.bz; int* Bo = W.bo; int* Bd = W.bd;  // other buffer
    const int jb = dir > 0 ? (c0 - R > 0 ? c0 - R : 0) : (c1 - 1 + R < N - 1 ? c1 - 1 + R : N - 1);
    const int je = dir > 0 ? c1 : c0 - 1;
    for (int j = jb; j != je; j += dir) {
      const int u = dir > 0 ? j : N - 1 - j;  // sweep position: 0, 1, 2, ... in sweep order
      const bool emit = j >= c0 && j < c1;
      PHASE_BEGIN();
      // ---- load S_mid(i, j)
      const long long q = (long long)i * P.ny + j;
      const int np = P.m_cnt[q];
      const long long ms = P.m_start[q];
      if (np > P.capP) {
        if (L.lane == 0) { set_status(status, ST_OVERFLOW_SLOT); note_max(&P.ctr->max_state, np); }
        return;
      }
      for (int t = L.lane; t < np; t += L.nl) {
        W.pa[t] = P.m_a[ms + t];
        W.pb[t] = P.m_b[ms + t];
        W.pd[t] = P.m_l[ms + t];
      }
      wsync();

      PHASE(0);
      // ---- rectangles: expire, add the column's, max-expiry merge
      for (int t = L.lane; t < nr; t += L.nl) W.c0[t] = W.rt[t] >= u;
      wsync();
      for (int t = L.lane; t < nr; t += L.nl) W.c1[t] = W.c0[t];
      wsync();
      const int nq = scan_excl(L, W.c1, nr);
      for (int t = L.lane; t < nr; t += L.nl)
        if (W.c0[t]) { const int o = W.c1[t]; W.qa[o] = W.ra[t]; W.qb[o] = W.rb[t]; W.qt[o] = W.rt[t]; }
      for (int t = L.lane; t < np; t += L.nl) W.c2[t] = W.pa[t] < W.pb[t];
      wsync();
      for (int t = L.lane; t < np; t += L.nl) W.c3[t] = W.c2[t];
      wsync();
      const int nn = scan_excl(L, W.c3, np);
      for (int t = L.lane; t < np; t += L.nl)
        if (W.c2[t]) {
          const int o = W.c3[t];
          W.na[o] = W.pa[t]; W.nb[o] = W.pb[t]; W.nt[o] = u + P.reach[W.pd[t]];
        }
      wsync();
      if (2LL * (nq + nn) + 8 > ce) {
        if (L.lane == 0) { set_status(status, ST_OVERFLOW_SLOT); note_max(&P.ctr->max_state, nq + nn); }
        return;
      }
      nr = merge_runs<Key, false>(L, W.qa, W.qb, W.qt, nq, W.na, W.nb, W.nt, nn, W.X, W.c0, W.c1,
                                  W.c2, W.c3, W.c4, W.c5, W.ra, W.rb, W.rt);
      if (nr > P.capR) {
        if (L.lane == 0) { set_status(status, ST_OVERFLOW_SLOT); note_max(&P.ctr->max_state, nr); }
        return;
      }

      PHASE(1);
      // ---- far sleepers due within the next kFarEvery steps move to the near pool
      if (u >= next_far) {
        next_far = u + kFarEvery;
        int any = 0;
        for (int t = L.lane; t < nfar; t += L.nl) any |= W.fw[t] < next_far;
        if (w_any(any)) {
          for (int t = L.lane; t < nfar; t += L.nl) {
            const bool mv = W.fw[t] < next_far;
            W.c0[t] = !mv;
            W.c1[t] = mv;
          }
          wsync();
          for (int t = L.lane; t < nfar; t += L.nl) { W.c2[t] = W.c0[t]; W.c3[t] = W.c1[t]; }
          wsync();
          const int keep = scan_excl(L, W.c2, nfar);
          const int mv = scan_excl(L, W.c3, nfar);
          if (nsl + mv > P.capS) {
            if (L.lane == 0) { set_status(status, ST_OVERFLOW_SLOT); note_max(&P.ctr->max_state, nsl + mv); }
            return;
          }
          for (int t = L.lane; t < nfar; t += L.nl)
            if (W.c1[t]) {
              const int o = nsl + W.c3[t];
              W.sz[o] = W.fz[t]; W.so[o] = W.fo[t]; W.sd[o] = W.fd[t]; W.sw[o] = W.fw[t];
            }
          wsync();
          for (int base = 0; base < nfar; base += L.nl) {
            const int t = base + L.lane;
            Key z0 = Key();
            int o0 = 0, d0 = 0, w0 = 0, dst = -1;
            if (t < nfar && W.c0[t]) { z0 = W.fz[t]; o0 = W.fo[t]; d0 = W.fd[t]; w0 = W.fw[t]; dst = W.c2[t]; }
            wsync();
            if (dst >= 0) { W.fz[dst] = z0; W.fo[dst] = o0; W.fd[dst] = d0; W.fw[dst] = w0; }
            wsync();
          }
          nsl += mv;
          nfar = keep;
        }
      }

      // ---- sleeping seeds due now: wake the live ones, drop the dead ones
      int nw = 0;
      {
        int any = 0;
        for (int t = L.lane; t < nsl; t += L.nl) any |= W.sw[t] <= u;
        if (w_any(any)) {
          for (int t = L.lane; t < nsl; t += L.nl) {
            const bool due = W.sw[t] <= u;
            W.c0[t] = !due;
            W.c1[t] = due && (u - W.so[t] <= P.reach[W.sd[t]]);
          }
          wsync();
          for (int t = L.lane; t < nsl; t += L.nl) { W.c2[t] = W.c0[t]; W.c3[t] = W.c1[t]; }
          wsync();
          const int keep = scan_excl(L, W.c2, nsl);
          nw = scan_excl(L, W.c3, nsl);
          if (nw > P.capA) {
            if (L.lane == 0) { set_status(status, ST_OVERFLOW_SLOT); note_max(&P.ctr->max_state, nw); }
            return;
          }
          for (int t = L.lane; t < nsl; t += L.nl)
            if (W.c1[t]) { const int o = W.c3[t]; W.X[o] = W.sz[t]; W.c4[o] = W.so[t]; W.c5[o] = W.sd[t]; }
          wsync();
          // in-place stable compaction of the pool: every lane reads its element, then writes
          for (int base = 0; base < nsl; base += L.nl) {
            const int t = base + L.lane;
            Key z0 = Key();
            int o0 = 0, d0 = 0, w0 = 0, dst = -1;
            if (t < nsl && W.c0[t]) { z0 = W.sz[t]; o0 = W.so[t]; d0 = W.sd[t]; w0 = W.sw[t]; dst = W.c2[t]; }
            wsync();
            if (dst >= 0) { W.sz[dst] = z0; W.so[dst] = o0; W.sd[dst] = d0; W.sw[dst] = w0; }
            wsync();
          }
          nsl = keep;
          // woken seeds sorted by height (rank sort; usually a handful)
          for (int t = L.lane; t < nw; t += L.nl) {
            const Key x = W.X[t];
            int r = 0;
            for (int v = 0; v < nw; ++v) r += (W.X[v] < x) || (W.X[v] == x && v < t);
            W.wz[r] = x; W.wo[r] = W.c4[t]; W.wd[r] = W.c5[t];
          }
          wsync();
        }
      }

      PHASE(2);
      // ---- new seeds: piece endpoints (finite; top only if b > a); equal heights keep
      //      the smallest dx
      for (int t = L.lane; t < np; t += L.nl) {
        const Key a = W.pa[t], b = W.pb[t];
        const int ca = (a > H<T>::ninf() && a < H<T>::pinf()) ? 1 : 0;
        const int cb = (b > H<T>::ninf() && b < H<T>::pinf() && b != a) ? 1 : 0;
        W.c2[t] = ca + cb;
      }
      wsync();
      for (int t = L.lane; t < np; t += L.nl) W.c3[t] = W.c2[t];
      wsync();
      const int nc = scan_excl(L, W.c3, np);
      for (int t = L.lane; t < np; t += L.nl) {
        const Key a = W.pa[t], b = W.pb[t];
        int o = W.c3[t];
        const int dx = W.pd[t];
        if (a > H<T>::ninf() && a < H<T>::pinf()) { W.nz[o] = a; W.nd[o] = dx; ++o; }
        if (b > H<T>::ninf() && b < H<T>::pinf() && b != a) { W.nz[o] = b; W.nd[o] = dx; }
      }
      wsync();
      for (int t = L.lane; t < nc; t += L.nl) {
        bool keep = true;
        if (t + 1 < nc && W.nz[t + 1] == W.nz[t] && W.nd[t + 1] <= W.nd[t]) keep = false;
        if (t > 0 && W.nz[t - 1] == W.nz[t] && W.nd[t - 1] < W.nd[t]) keep = false;
        W.c0[t] = keep;
      }
      wsync();
      for (int t = L.lane; t < nc; t += L.nl) W.c1[t] = W.c0[t];
      wsync();
      const int nv = scan_excl(L, W.c1, nc);
      for (int t = L.lane; t < nc; t += L.nl)
        if (W.c0[t]) { W.X[W.c1[t]] = W.nz[t]; W.c2[W.c1[t]] = W.nd[t]; }
      wsync();

      PHASE(3);
      // ---- envelope of the previous step minus the dead, into B
      for (int t = L.lane; t < na; t += L.nl) W.c0[t] = u - Ao[t] <= P.reach[Ad[t]];
      wsync();
      for (int t = L.lane; t < na; t += L.nl) W.c1[t] = W.c0[t];
      wsync();
      const int nb = scan_excl(L, W.c1, na);
      for (int t = L.lane; t < na; t += L.nl)
        if (W.c0[t]) { const int o = W.c1[t]; Bz[o] = Az[t]; Bo[o] = Ao[t]; Bd[o] = Ad[t]; }
      wsync();
      na = nb + nv + nw;
      if (na > P.capA) {
        if (L.lane == 0) { set_status(status, ST_OVERFLOW_SLOT); note_max(&P.ctr->max_state, na); }
        return;
      }
      // three-way merge by height into A: previous envelope, then new, then woken on ties
      for (int t = L.lane; t < nb; t += L.nl) {
        const Key x = Bz[t];
        const int pos = t + lower_bound(W.X, nv, x) + lower_bound(W.wz, nw, x);
        Az[pos] = x; Ao[pos] = Bo[t]; Ad[pos] = Bd[t];
      }
      for (int t = L.lane; t < nv; t += L.nl) {
        const Key x = W.X[t];
        const int pos = t + upper_bound(Bz, nb, x) + lower_bound(W.wz, nw, x);
        Az[pos] = x; Ao[pos] = u; Ad[pos] = W.c2[t];
      }
      for (int t = L.lane; t < nw; t += L.nl) {
        const Key x = W.wz[t];
        const int pos = t + upper_bound(Bz, nb, x) + upper_bound(W.X, nv, x);
        Az[pos] = x; Ao[pos] = W.wo[t]; Ad[pos] = W.wd[t];
      }
      wsync();

      PHASE(4);
      // ---- lower envelope of the merged seeds: one monotone-stack pass (lane 0); a seed
      //      popped because the seed below it and the incoming one dominate it is discarded
      //      or put to sleep according to seed_fate
      PHASE_COUNT(10, na);
      PHASE_COUNT(11, nr);
      PHASE_COUNT(12, nsl);
      PHASE_COUNT(13, 1);
      if (L.lane == 0) {
        int* stk = W.c5;
        int top = -1;
        for (int t = 0; t < na; ++t) {
          bool pushed = true;
          while (top >= 0) {
            const int s = stk[top];
            if (Az[s] == Az[t]) {
              const int nS = seed_n(Ad[s], Ao[s], u), nT = seed_n(Ad[t], Ao[t], u);
              if (nS <= nT) {  // the incoming seed is dominated by the stack top
                W.c4[t] = equal_fate(Ao[s], nS, Ao[t], nT, u);
                pushed = false;
                break;
              }
              W.c4[s] = equal_fate(Ao[t], nT, Ao[s], nS, u);
              --top;
              continue;
            }
            if (top == 0) break;
            const int f = seed_fate<Key>(Az, Ao, Ad, stk[top - 1], s, t, u, P.h2, P.h2f);
            if (f == FATE_KEEP) break;
            W.c4[s] = f;
            --top;
          }
          if (pushed) {
            stk[++top] = t;
            W.c4[t] = FATE_KEEP;
          }
        }
      }
      wsync();
      {
        for (int t = L.lane; t < na; t += L.nl) {
          const int fate = W.c4[t];
          W.c0[t] = fate == FATE_KEEP;
          W.c1[t] = fate != FATE_KEEP && fate != FATE_DROP;
        }
        wsync();
        for (int t = L.lane; t < na; t += L.nl) { W.c2[t] = W.c0[t]; W.c3[t] = W.c1[t]; }
        wsync();
        // sleepers split by wake-up: before the next far scan -> near pool, else far pool
        for (int t = L.lane; t < na; t += L.nl) {
          int wk = W.c4[t];
          if (W.c1[t]) {
            const int dead = Ao[t] + P.reach[Ad[t]] + 1;  // first position where it is dead
            wk = wk < dead ? wk : dead;
            W.c4[t] = wk;
          }
          W.c5[t] = W.c1[t] && wk >= next_far;
          W.c1[t] = W.c1[t] && wk < next_far;
        }
        wsync();
        for (int t = L.lane; t < na; t += L.nl) W.c3[t] = W.c1[t];
        wsync();
        const int na2 = scan_excl(L, W.c2, na);
        const int ns2 = scan_excl(L, W.c3, na);
        int* fpos = W.E;
        for (int t = L.lane; t < na; t += L.nl) fpos[t] = W.c5[t];
        wsync();
        const int nf2 = scan_excl(L, fpos, na);
        if (nsl + ns2 > P.capS || nfar + nf2 > P.capS) {
          if (L.lane == 0) {
            set_status(status, ST_OVERFLOW_SLOT);
            note_max(&P.ctr->max_state, nsl + ns2 > nfar + nf2 ? nsl + ns2 : nfar + nf2);
          }
          return;
        }
        for (int t = L.lane; t < na; t += L.nl) {
          if (W.c0[t]) { const int o = W.c2[t]; Bz[o] = Az[t]; Bo[o] = Ao[t]; Bd[o] = Ad[t]; }
          if (W.c1[t]) {
            const int o = nsl + W.c3[t];
            W.sz[o] = Az[t]; W.so[o] = Ao[t]; W.sd[o] = Ad[t]; W.sw[o] = W.c4[t];
          }
          if (W.c5[t]) {
            const int o = nfar + fpos[t];
            W.fz[o] = Az[t]; W.fo[o] = Ao[t]; W.fd[o] = Ad[t]; W.fw[o] = W.c4[t];
          }
        }
        wsync();
        nsl += ns2;
        nfar += nf2;
        na = na2;
        Key* tz = Az; Az = Bz; Bz = tz;
        int* to = Ao; Ao = Bo; Bo = to;
        int* td = Ad; Ad = Bd; Bd = td;
      }
      PHASE_COUNT(14, na);
      if (L.lane == 0) {
        int m = nsl > na ? nsl : na;
        m = m > nfar ? m : nfar;
        note_max(&P.ctr->max_state, m > nr ? m : nr);
      }
      PHASE(5);
      if (!emit) continue;

      // ---- emission: rectangles (el, er) and envelope disks
      for (int t = L.lane; t < nr; t += L.nl) { W.el[t] = ikey(W.ra[t]); W.er[t] = ikey(W.rb[t]); }
      for (int t = L.lane; t < na; t += L.nl) {
        const double w = P.wtab[seed_n(Ad[t], Ao[t], u)];
        const double zz = keyd(Az[t]);
        W.xl[t] = dkey(zz - w);
        W.xr[t] = dkey(zz + w);
      }
      wsync();
      const int nd = envelope_runs(L, W.xl, W.xr, na, W.c0, W.c1, W.c2, W.hl, W.hr, W.gl, W.gr);
      PHASE(6);
      int nm = merge_intervals(L, W.el, W.er, nr, W.hl, W.hr, nd, W.gl, W.gr);
      const ukey* srcl = W.gl;
      const ukey* srcr = W.gr;
      if (dir < 0) {
        const long long fs = W.fstart[j - c0];
        const int nf = W.fcnt[j - c0];
        if (fs < 0) continue;
        for (int t = L.lane; t < nf; t += L.nl) { W.el[t] = P.f_l[fs + t]; W.er[t] = P.f_r[fs + t]; }
        wsync();
        nm = merge_intervals(L, W.gl, W.gr, nm, W.el, W.er, nf, W.xl, W.xr);
        srcl = W.xl;
        srcr = W.xr;
      }
      const int no = union_runs(L, srcl, srcr, nm, true, W.c0, W.c1, W.hl, W.hr,
                                dir < 0 ? W.gl : W.el, nullptr);
      PHASE(7);
      if (dir > 0) {
        const long long s = arena_take(L, &P.ctr->arena_top[2], P.blk, curF, no);
        const bool fits = s + no <= P.f_cap;
        if (!fits) { if (L.lane == 0) set_status(status, ST_OVERFLOW_ARENA); }
        else for (int t = L.lane; t < no; t += L.nl) { P.f_l[s + t] = W.hl[t]; P.f_r[s + t] = W.hr[t]; }
        if (L.lane == 0) { W.fstart[j - c0] = fits ? s : -1; W.fcnt[j - c0] = no; }
        wsync();
      } else {
        const long long s = arena_take(L, &P.ctr->arena_top[3], P.blk, curO, no);
        const bool fits = s + no <= P.o_cap;
        if (!fits) { if (L.lane == 0) set_status(status, ST_OVERFLOW_ARENA); }
        else for (int t = L.lane; t < no; t += L.nl) { P.o_l[s + t] = W.hl[t]; P.o_r[s + t] = W.hr[t]; }
        if (L.lane == 0) {
          const long long c = (long long)j * P.nx + i;
          P.o_start[c] = fits ? s : 0;
          P.o_cnt[c] = no;
          note_max(&P.ctr->max_out, no);
        }
        item_total += no;
        wsync();
      }
    }
  }
  if (L.lane == 0) add_total(&P.ctr->out_total, item_total);
}

}  // namespace dexel
