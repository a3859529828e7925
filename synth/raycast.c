/*
 * Seeded-input generator: analytic ray casting of primitives into a CSR dexel grid.
 *
 * INPUT GENERATION ONLY.  It holds none of the offset method's arithmetic; it is the compiled
 * twin of synth/shapes.py's numpy ray caster (same operations in the same order, IEEE double,
 * no FMA contraction, so the two give bit-identical grids) and serves the tests and the
 * benchmark alike.
 *
 * The vertical ray of column (i, j) passes through ((i + 1/2) h, (j + 1/2) h).  Primitives
 * (world units over [0,1]^3), one row of 8 doubles each:
 *   kind 0  sphere  cx cy cz R
 *   kind 1  box     x0 x1 y0 y1 z0 z1
 *   kind 2  shell   cx cy cz R t       (hollow sphere, inner radius R - t)
 * Tangent rays (zero-length chords) are excluded by strict inequalities.  The intervals of a
 * column are sorted by (a, b) and joined when they touch or overlap (closed union).
 *
 * Two calls: rc_count fills the per-column segment counts, rc_fill writes the segments at the
 * caller's offsets.  Rows are split over threads.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  double a, b;
} ivl;

typedef struct {
  int n;
  double h;
  const double* prim; /* nprim x 8 */
  const int* kind;
  int nprim;
  const double* fp; /* footprints x0 x1 y0 y1 per primitive */
  int64_t* counts;  /* n*n (count pass) */
  const int64_t* off;
  double* z;        /* fill pass */
  int row0, row1;
  int fail, started;
} job_t;

static int cmp_ivl(const void* x, const void* y) {
  const ivl* p = (const ivl*)x;
  const ivl* q = (const ivl*)y;
  if (p->a < q->a) return -1;
  if (p->a > q->a) return 1;
  if (p->b < q->b) return -1;
  if (p->b > q->b) return 1;
  return 0;
}

static int push(ivl** v, int* n, int* cap, double a, double b) {
  if (*n == *cap) {
    int nc = *cap ? 2 * *cap : 64;
    ivl* nv = (ivl*)realloc(*v, (size_t)nc * sizeof(ivl));
    if (!nv) return -1;
    *v = nv;
    *cap = nc;
  }
  (*v)[*n].a = a;
  (*v)[*n].b = b;
  (*n)++;
  return 0;
}

/* chords of primitive p along the ray at (x, y) */
static int cast(const job_t* J, int p, double x, double y, ivl** v, int* n, int* cap) {
  const double* q = J->prim + 8 * (size_t)p;
  switch (J->kind[p]) {
    case 0: {
      const double dx = x - q[0], dy = y - q[1];
      const double d2 = dx * dx + dy * dy;
      const double R2 = q[3] * q[3];
      if (d2 < R2) {
        double t = R2 - d2;
        if (t < 0) t = 0;
        const double s = sqrt(t);
        if (push(v, n, cap, q[2] - s, q[2] + s)) return -1;
      }
      break;
    }
    case 1:
      if (x > q[0] && x < q[1] && y > q[2] && y < q[3])
        if (push(v, n, cap, q[4], q[5])) return -1;
      break;
    case 2: {
      const double dx = x - q[0], dy = y - q[1];
      const double d2 = dx * dx + dy * dy;
      const double R = q[3], Ri = q[3] - q[4];
      const double R2 = R * R, Ri2 = Ri * Ri;
      double to = R2 - d2, ti = Ri2 - d2;
      if (to < 0) to = 0;
      if (ti < 0) ti = 0;
      const double so = sqrt(to), si = sqrt(ti);
      const int outer = d2 < R2, inner = d2 < Ri2;
      if (outer && !inner) {
        if (push(v, n, cap, q[2] - so, q[2] + so)) return -1;
      } else if (outer && inner) {
        if (push(v, n, cap, q[2] - so, q[2] - si)) return -1;
        if (push(v, n, cap, q[2] + si, q[2] + so)) return -1;
      }
      break;
    }
  }
  return 0;
}

static void* work(void* arg) {
  job_t* J = (job_t*)arg;
  const int n = J->n;
  const double h = J->h;
  int* cand = (int*)malloc(sizeof(int) * (size_t)(J->nprim > 0 ? J->nprim : 1));
  ivl* v = NULL;
  int cap = 0;
  if (!cand) {
    J->fail = 1;
    return NULL;
  }
  for (int j = J->row0; j < J->row1; ++j) {
    const double y = ((double)j + 0.5) * h;
    /* primitives whose footprint reaches this row */
    int nc = 0;
    for (int p = 0; p < J->nprim; ++p) {
      const double* f = J->fp + 4 * (size_t)p;
      if (f[3] < y - h || f[2] > y + h) continue;
      cand[nc++] = p;
    }
    for (int i = 0; i < n; ++i) {
      const double x = ((double)i + 0.5) * h;
      int m = 0;
      for (int t = 0; t < nc; ++t) {
        const int p = cand[t];
        const double* f = J->fp + 4 * (size_t)p;
        if (f[1] < x - h || f[0] > x + h) continue;
        if (cast(J, p, x, y, &v, &m, &cap)) {
          J->fail = 1;
          goto done;
        }
      }
      int64_t out = 0;
      const int64_t c = (int64_t)j * n + i;
      double* dst = J->z ? J->z + 2 * J->off[c] : NULL;
      if (m > 0) {
        qsort(v, (size_t)m, sizeof(ivl), cmp_ivl);
        double ca = v[0].a, cb = v[0].b;
        for (int t = 1; t < m; ++t) {
          if (v[t].a <= cb) {
            if (v[t].b > cb) cb = v[t].b;
          } else {
            if (dst) {
              dst[2 * out] = ca;
              dst[2 * out + 1] = cb;
            }
            ++out;
            ca = v[t].a;
            cb = v[t].b;
          }
        }
        if (dst) {
          dst[2 * out] = ca;
          dst[2 * out + 1] = cb;
        }
        ++out;
      }
      if (J->counts) J->counts[c] = out;
    }
  }
done:
  free(cand);
  free(v);
  return NULL;
}

static int run(int n, const double* prim, const int* kind, int nprim, int64_t* counts,
               const int64_t* off, double* z, int threads) {
  if (n < 1 || nprim < 0 || threads < 1) return -1;
  double* fp = (double*)malloc(sizeof(double) * 4 * (size_t)(nprim > 0 ? nprim : 1));
  if (!fp) return -1;
  for (int p = 0; p < nprim; ++p) {
    const double* q = prim + 8 * (size_t)p;
    double* f = fp + 4 * (size_t)p;
    if (kind[p] == 1) {
      f[0] = q[0]; f[1] = q[1]; f[2] = q[2]; f[3] = q[3];
    } else {
      f[0] = q[0] - q[3]; f[1] = q[0] + q[3]; f[2] = q[1] - q[3]; f[3] = q[1] + q[3];
    }
  }
  if (threads > n) threads = n;
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)threads);
  job_t* jobs = (job_t*)calloc((size_t)threads, sizeof(job_t));
  if (!th || !jobs) {
    free(fp); free(th); free(jobs);
    return -1;
  }
  int rc = 0;
  for (int t = 0; t < threads; ++t) {
    job_t* J = &jobs[t];
    J->n = n;
    J->h = 1.0 / (double)n;
    J->prim = prim;
    J->kind = kind;
    J->nprim = nprim;
    J->fp = fp;
    J->counts = counts;
    J->off = off;
    J->z = z;
    J->row0 = (int)((int64_t)n * t / threads);
    J->row1 = (int)((int64_t)n * (t + 1) / threads);
    J->started = pthread_create(&th[t], NULL, work, J) == 0;
    if (!J->started) work(J);  /* no thread: this caller does the rows itself */
  }
  for (int t = 0; t < threads; ++t) {
    if (jobs[t].started) pthread_join(th[t], NULL);
    if (jobs[t].fail) rc = -1;
  }
  free(fp);
  free(th);
  free(jobs);
  return rc;
}

int rc_count(int n, const double* prim, const int* kind, int nprim, int64_t* counts, int threads) {
  return run(n, prim, kind, nprim, counts, NULL, NULL, threads);
}

int rc_fill(int n, const double* prim, const int* kind, int nprim, const int64_t* off, double* z,
            int threads) {
  return run(n, prim, kind, nprim, NULL, off, z, threads);
}
