// Pass 2 of the dexel offset: per column line, forward and backward sweeps over the
// S_mid pieces with the rectangle envelope and the half-space power diagram of the
// endpoint seeds (Sec. 3.3 "2D Power Diagram", Fig. segments-separate, Fig. power-vertex).
#pragma once
#include "sweep.cuh"

namespace dexel {

// seed flags
enum : int { SEED_WAIT = 0, SEED_ENV = 1, SEED_GONE = -1 };

template <typename T>
DXI int seed_n(const int* sd, const int* sj, int t, int j) {
  const int dy = j - sj[t];
  return sd[t] + dy * dy;
}

// Is seed s dominated by its on-envelope neighbours p (below, or -1) and n (above, or -1)?
// *perm is set when the dominating seeds are all newer-or-equal in sweep order, so that
// the domination holds for the rest of the sweep.
template <typename T>
DXI bool seed_dominated(const T* z, const int* sj, const int* sd, int j, int dir, int p, int s,
                        int n, double h2, bool* perm) {
  const double zs = (double)z[s];
  const int ns = seed_n<T>(sd, sj, s, j);
  const int os = dir * sj[s];
  *perm = false;
  if (p >= 0 && n >= 0) {
    const double zp = (double)z[p], zn = (double)z[n];
    const int np = seed_n<T>(sd, sj, p, j), nn = seed_n<T>(sd, sj, n, j);
    if (zp == zs) {
      if (np <= ns) { *perm = dir * sj[p] >= os; return true; }
      return false;
    }
    if (zn == zs) {
      if (nn <= ns) { *perm = dir * sj[n] >= os; return true; }
      return false;
    }
    if (dominated3(zp, np, zs, ns, zn, nn, h2)) {
      *perm = dir * sj[p] >= os && dir * sj[n] >= os;
      return true;
    }
    return false;
  }
  const int q = p >= 0 ? p : n;
  if (q < 0) return false;
  if ((double)z[q] == zs && seed_n<T>(sd, sj, q, j) <= ns) {
    *perm = dir * sj[q] >= os;
    return true;
  }
  return false;
}

template <typename T>
DXN void pass2_item(const Lanes& L, const P2Params<T>& P, const P2Slot<T>& W, int i, int c0,
                    int c1, ArenaCursor& curF, ArenaCursor& curO) {
  int* status = &P.ctr->status;
  const int N = P.ny;
  const int K = P.K;
  const double kk = P.kk;
  long long item_total = 0;
  for (int dir = 1; dir >= -1; dir -= 2) {
    int nr = 0, ns = 0;
    const int jb = dir > 0 ? (c0 - K > 0 ? c0 - K : 0) : (c1 - 1 + K < N - 1 ? c1 - 1 + K : N - 1);
    const int je = dir > 0 ? c1 : c0 - 1;
    for (int j = jb; j != je; j += dir) {
      const int cur = dir * j;
      const bool emit = j >= c0 && j < c1;
      // ---- load S_mid(i, j)
      const long long q = (long long)i * P.ny + j;
      const int np = P.m_cnt[q];
      const long long ms = P.m_start[q];
      if (np > P.capP) { if (L.lane == 0) set_status(status, ST_OVERFLOW_SLOT); return; }
      for (int t = L.lane; t < np; t += L.nl) {
        W.pa[t] = P.m_a[ms + t];
        W.pb[t] = P.m_b[ms + t];
        const int dx = P.m_l[ms + t];
        W.pd[t] = dx;
      }
      wsync();
      // ---- rectangles: expire, new ones, max-expiry merge
      for (int t = L.lane; t < nr; t += L.nl) W.c0[t] = W.rt[t] >= cur;
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
          W.na[o] = W.pa[t]; W.nb[o] = W.pb[t]; W.nt[o] = cur + P.reach[W.pd[t]];
        }
      wsync();
      if (2 * (nq + nn) > p2_ce(P.capR, P.capD, P.capP)) {
        if (L.lane == 0) { set_status(status, ST_OVERFLOW_SLOT); note_max(&P.ctr->max_state, nq + nn); }
        return;
      }
      nr = merge_runs<T, false>(L, W.qa, W.qb, W.qt, nq, W.na, W.nb, W.nt, nn, W.X, W.c0, W.c1,
                                W.c2, W.c3, W.c4, W.c5, W.ra, W.rb, W.rt);
      if (nr > P.capR) {
        if (L.lane == 0) { set_status(status, ST_OVERFLOW_SLOT); note_max(&P.ctr->max_state, nr); }
        return;
      }

      // ---- seeds: drop dead or pruned ones
      for (int t = L.lane; t < ns; t += L.nl)
        W.c0[t] = W.so[t] != SEED_GONE && seed_n<T>(W.sd, W.sj, t, j) <= kk;
      wsync();
      for (int t = L.lane; t < ns; t += L.nl) W.c1[t] = W.c0[t];
      wsync();
      const int nu = scan_excl(L, W.c1, ns);
      for (int t = L.lane; t < ns; t += L.nl)
        if (W.c0[t]) {
          const int o = W.c1[t];
          W.uz[o] = W.sz[t]; W.uj[o] = W.sj[t]; W.ud[o] = W.sd[t]; W.uo[o] = W.so[t];
        }
      wsync();
      // new seeds: bottom and top endpoints of the pieces (finite, top only if b > a)
      for (int t = L.lane; t < np; t += L.nl) {
        const T a = W.pa[t], b = W.pb[t];
        const int ca = (a > (T)-DEXEL_INF && a < (T)DEXEL_INF) ? 1 : 0;
        const int cb = (b > (T)-DEXEL_INF && b < (T)DEXEL_INF && b != a) ? 1 : 0;
        W.c2[t] = ca + cb;
      }
      wsync();
      for (int t = L.lane; t < np; t += L.nl) W.c3[t] = W.c2[t];
      wsync();
      const int nc = scan_excl(L, W.c3, np);
      for (int t = L.lane; t < np; t += L.nl) {
        const T a = W.pa[t], b = W.pb[t];
        int o = W.c3[t];
        const int d2 = W.pd[t] * W.pd[t];
        if (a > (T)-DEXEL_INF && a < (T)DEXEL_INF) { W.nz[o] = a; W.nd[o] = d2; ++o; }
        if (b > (T)-DEXEL_INF && b < (T)DEXEL_INF && b != a) { W.nz[o] = b; W.nd[o] = d2; }
      }
      wsync();
      // equal heights within the column: keep the smallest dx (largest weight)
      for (int t = L.lane; t < nc; t += L.nl) {
        bool keep = true;
        if (t + 1 < nc && W.nz[t + 1] == W.nz[t] && W.nd[t + 1] <= W.nd[t]) keep = false;
        if (t > 0 && W.nz[t - 1] == W.nz[t] && W.nd[t - 1] < W.nd[t]) keep = false;
        W.c0[t] = keep;
      }
      wsync();
      for (int t = L.lane; t < nc; t += L.nl) W.c1[t] = W.c0[t];
      wsync();
      const int nw = scan_excl(L, W.c1, nc);
      // compact new seeds into (X as z, c2 as d2) to free nz/nd
      for (int t = L.lane; t < nc; t += L.nl)
        if (W.c0[t]) { W.X[W.c1[t]] = W.nz[t]; W.c2[W.c1[t]] = W.nd[t]; }
      wsync();
      if (nu + nw > P.capD) {
        if (L.lane == 0) { set_status(status, ST_OVERFLOW_SLOT); note_max(&P.ctr->max_state, nu + nw); }
        return;
      }
      // merge old (uz...) and new (X, c2) seeds by z, old first on ties -> (sz, sj, sd, so)
      for (int t = L.lane; t < nu; t += L.nl) {
        const int pos = t + lower_bound(W.X, nw, W.uz[t]);
        W.sz[pos] = W.uz[t]; W.sj[pos] = W.uj[t]; W.sd[pos] = W.ud[t]; W.so[pos] = W.uo[t];
      }
      for (int t = L.lane; t < nw; t += L.nl) {
        const int pos = t + upper_bound(W.uz, nu, W.X[t]);
        W.sz[pos] = W.X[t]; W.sj[pos] = j; W.sd[pos] = W.c2[t]; W.so[pos] = SEED_ENV;
      }
      ns = nu + nw;
      wsync();
      // waiting seeds: re-test against their on-envelope neighbours
      for (int t = L.lane; t < ns; t += L.nl) W.c0[t] = W.so[t] == SEED_ENV;
      wsync();
      scan_last_flag(L, W.c0, W.c1, ns);
      scan_next_flag(L, W.c0, W.c2, ns);
      for (int t = L.lane; t < ns; t += L.nl) {
        int f = W.so[t];
        if (f == SEED_WAIT) {
          const int p = W.c1[t];
          const int n = W.c2[t] < ns ? W.c2[t] : -1;
          bool perm = false;
          const bool dom = seed_dominated<T>(W.sz, W.sj, W.sd, j, dir, p, t, n, P.h2, &perm);
          f = dom ? (perm ? SEED_GONE : SEED_WAIT) : SEED_ENV;
        }
        W.c3[t] = f;
      }
      wsync();
      for (int t = L.lane; t < ns; t += L.nl) W.so[t] = W.c3[t];
      wsync();
      // envelope list E: indices of on-envelope seeds, then parity rounds
      for (int t = L.lane; t < ns; t += L.nl) W.c0[t] = W.so[t] == SEED_ENV;
      wsync();
      for (int t = L.lane; t < ns; t += L.nl) W.c1[t] = W.c0[t];
      wsync();
      int ne = scan_excl(L, W.c1, ns);
      for (int t = L.lane; t < ns; t += L.nl)
        if (W.c0[t]) W.E[W.c1[t]] = t;
      wsync();
      int quiet = 0;
      for (int round = 0; quiet < 2 && ne > 1; ++round) {
        const int parity = round & 1;
        int removed = 0;
        for (int qq = L.lane; qq < ne; qq += L.nl) {
          int r = 0;
          if ((qq & 1) == parity) {
            const int s = W.E[qq];
            const int p = qq > 0 ? W.E[qq - 1] : -1;
            const int n = qq + 1 < ne ? W.E[qq + 1] : -1;
            bool perm = false;
            if (seed_dominated<T>(W.sz, W.sj, W.sd, j, dir, p, s, n, P.h2, &perm)) {
              r = 1;
              W.so[s] = perm ? SEED_GONE : SEED_WAIT;
            }
          }
          W.c0[qq] = !r;
          removed |= r;
        }
        wsync();
        removed = w_any(removed);
        if (!removed) { ++quiet; continue; }
        quiet = 0;
        for (int qq = L.lane; qq < ne; qq += L.nl) W.c1[qq] = W.c0[qq];
        wsync();
        const int ne2 = scan_excl(L, W.c1, ne);
        for (int qq = L.lane; qq < ne; qq += L.nl)
          if (W.c0[qq]) W.c4[W.c1[qq]] = W.E[qq];
        wsync();
        for (int qq = L.lane; qq < ne2; qq += L.nl) W.E[qq] = W.c4[qq];
        wsync();
        ne = ne2;
      }
      if (L.lane == 0) note_max(&P.ctr->max_state, ns > nr ? ns : nr);
#ifdef DEXEL_TRACE
      if (i == DEXEL_TRACE) {
        printf("i=%d j=%d dir=%d np=%d nr=%d ns=%d ne=%d\n", i, j, dir, np, nr, ns, ne);
        for (int t = 0; t < np; ++t) printf("   piece %.6f %.6f dx=%d\n", (double)W.pa[t], (double)W.pb[t], W.pd[t]);
        for (int t = 0; t < nr; ++t) printf("   rect %.6f %.6f t=%d\n", (double)W.ra[t], (double)W.rb[t], W.rt[t]);
        for (int t = 0; t < ns; ++t) printf("   seed %.6f js=%d d2=%d flag=%d\n", (double)W.sz[t], W.sj[t], W.sd[t], W.so[t]);
        for (int t = 0; t < ne; ++t) printf("   env %d\n", W.E[t]);
      }
#endif
      if (!emit) continue;

      // ---- emission: rectangles (el, er) and envelope disks (hl, hr)
      for (int t = L.lane; t < nr; t += L.nl) { W.el[t] = (double)W.ra[t]; W.er[t] = (double)W.rb[t]; }
      for (int qq = L.lane; qq < ne; qq += L.nl) {
        const int s = W.E[qq];
        const double w = P.wtab[seed_n<T>(W.sd, W.sj, s, j)];
        const double zz = (double)W.sz[s];
        W.xl[qq] = zz - w;
        W.xr[qq] = zz + w;
      }
      wsync();
      const int nd = union_envelope(L, W.xl, W.xr, ne, W.c0, W.c1, W.hl, W.hr, W.gl, W.gr);
      int nm = merge_intervals(L, W.el, W.er, nr, W.hl, W.hr, nd, W.gl, W.gr);
      const double* srcl = W.gl;
      const double* srcr = W.gr;
      if (dir < 0) {
        // united with the forward result of this column
        const long long fs = W.fstart[j - c0];
        const int nf = W.fcnt[j - c0];
        if (fs < 0) continue;
        for (int t = L.lane; t < nf; t += L.nl) { W.el[t] = P.f_l[fs + t]; W.er[t] = P.f_r[fs + t]; }
        wsync();
        nm = merge_intervals(L, W.gl, W.gr, nm, W.el, W.er, nf, W.xl, W.xr);
        srcl = W.xl;
        srcr = W.xr;
      }
      const int no = union_sorted(L, srcl, srcr, nm, W.c0, W.c1, W.hl, W.hr,
                                  dir < 0 ? W.gl : W.el);
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
