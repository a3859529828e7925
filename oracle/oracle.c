/*
 * FP64 brute-force oracle for dexel dilation and erosion by a ball.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg may load this library.  It shares no code with the CUDA path.
 *
 * Grid: nx x ny columns, spacing h; column (i, j) is numbered c = j*nx + i and holds the
 * sorted, disjoint segments z[2*s], z[2*s+1] for s in [col_off[c], col_off[c+1]).
 *
 * Dilation (Sec. 3.1, Eq. of D_r: the points at distance <= r from the shape).  A point
 * (column c, height z) is within distance r = k h of a segment [a, b] of column c' iff
 * n h^2 + dist(z, [a, b])^2 <= r^2 with n = (i - i')^2 + (j - j')^2, i.e. iff n <= k^2 and
 * z lies in [a - w, b + w] with w = h sqrt(k^2 - n).  The dilated column is therefore the
 * closed union of those intervals over all in-grid columns c' with n <= k^2 -- the paper's
 * brute-force baseline of Sec. 4 ("Baseline Comparison"), written as a gather per output
 * column instead of a scatter per input segment.
 *
 * Erosion (Sec. 3.1, "Erosion": the complement of the dilation of the complement), written
 * directly rather than through complements, so that duality is a real test: z is kept in
 * column c iff for every in-grid column c' with n <= k^2 the interval [z - w, z + w] lies in
 * the shape of c'.  Because the segments of a column are disjoint with positive gaps, that
 * holds iff z is in some [a + w, b - w]; the result is the intersection over c' of those
 * unions.  Results of zero length are dropped (they are measure-zero artefacts of the
 * closed/open boundary).  Columns outside the grid do not take part.
 *
 * Everything is IEEE double; build with -ffp-contract=off so that h*sqrt(.) and the following
 * add are rounded separately.  Threads split the output columns.
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
  ivl* v;
  int64_t n, cap;
} ivec;

static int ivec_push(ivec* q, double a, double b) {
  if (q->n == q->cap) {
    int64_t nc = q->cap ? 2 * q->cap : 64;
    ivl* nv = (ivl*)realloc(q->v, (size_t)nc * sizeof(ivl));
    if (!nv) return -1;
    q->v = nv;
    q->cap = nc;
  }
  q->v[q->n].a = a;
  q->v[q->n].b = b;
  q->n++;
  return 0;
}

static int cmp_ivl(const void* x, const void* y) {
  const ivl* p = (const ivl*)x;
  const ivl* q = (const ivl*)y;
  if (p->a < q->a) return -1;
  if (p->a > q->a) return 1;
  if (p->b < q->b) return -1;
  if (p->b > q->b) return 1;
  return 0;
}

/* Sort, then fold closed intervals: the next one joins the current one when next.a <= cur.b. */
static void sort_merge(ivec* q) {
  if (q->n == 0) return;
  qsort(q->v, (size_t)q->n, sizeof(ivl), cmp_ivl);
  int64_t m = 0;
  for (int64_t t = 1; t < q->n; ++t) {
    if (q->v[t].a <= q->v[m].b) {
      if (q->v[t].b > q->v[m].b) q->v[m].b = q->v[t].b;
    } else {
      q->v[++m] = q->v[t];
    }
  }
  q->n = m + 1;
}

/* Largest integer R with R*R <= kk (as doubles): the reach of the ball in grid steps. */
static int64_t reach(double kk) {
  if (!(kk >= 0)) return -1;
  int64_t R = (int64_t)floor(sqrt(kk));
  while ((double)((R + 1) * (R + 1)) <= kk) ++R;
  while (R > 0 && (double)(R * R) > kk) --R;
  return R;
}

typedef struct {
  int32_t nx, ny;
  double h, k;
  const int64_t* col_off;
  const double* z;
  int erode;
  const int64_t* cols; /* output columns to compute; NULL = all, in order */
  int slices;          /* 1: every row is its own 2D image, offset by a disk (dj = 0 only) */
  int64_t ncols;
  ivec* res; /* one result vector per requested column */
  int64_t next;
  pthread_mutex_t lock;
  int failed;
} job;

static void dilate_column(const job* J, int64_t c, ivec* out) {
  const int32_t nx = J->nx, ny = J->ny;
  const int64_t i = c % nx, j = c / nx;
  const double kk = J->k * J->k;
  const int64_t R = reach(kk);
  const int64_t Rj = J->slices ? 0 : R;
  for (int64_t dj = -Rj; dj <= Rj; ++dj) {
    const int64_t jj = j + dj;
    if (jj < 0 || jj >= ny) continue;
    for (int64_t di = -R; di <= R; ++di) {
      const int64_t ii = i + di;
      if (ii < 0 || ii >= nx) continue;
      const int64_t n = di * di + dj * dj;
      if ((double)n > kk) continue;
      const double w = J->h * sqrt(kk - (double)n);
      const int64_t cc = jj * nx + ii;
      for (int64_t s = J->col_off[cc]; s < J->col_off[cc + 1]; ++s) {
        const double a = J->z[2 * s] - w;
        const double b = J->z[2 * s + 1] + w;
        if (ivec_push(out, a, b)) return;
      }
    }
  }
  sort_merge(out);
}

/* out := out  intersect  [list] (both sorted, disjoint); zero-length pieces dropped. */
static void intersect_into(ivec* out, const ivec* other, ivec* tmp) {
  tmp->n = 0;
  int64_t p = 0, q = 0;
  while (p < out->n && q < other->n) {
    const double lo = fmax(out->v[p].a, other->v[q].a);
    const double hi = fmin(out->v[p].b, other->v[q].b);
    if (lo < hi) ivec_push(tmp, lo, hi);
    if (out->v[p].b < other->v[q].b)
      ++p;
    else
      ++q;
  }
  ivec sw = *out;
  *out = *tmp;
  *tmp = sw;
}

static void erode_column(const job* J, int64_t c, ivec* out) {
  const int32_t nx = J->nx, ny = J->ny;
  const int64_t i = c % nx, j = c / nx;
  const double kk = J->k * J->k;
  const int64_t R = reach(kk);
  ivec part = {0}, tmp = {0};
  int first = 1;
  const int64_t Rj = J->slices ? 0 : R;
  for (int64_t dj = -Rj; dj <= Rj; ++dj) {
    const int64_t jj = j + dj;
    if (jj < 0 || jj >= ny) continue;
    for (int64_t di = -R; di <= R; ++di) {
      const int64_t ii = i + di;
      if (ii < 0 || ii >= nx) continue;
      const int64_t n = di * di + dj * dj;
      if ((double)n > kk) continue;
      const double w = J->h * sqrt(kk - (double)n);
      const int64_t cc = jj * nx + ii;
      part.n = 0;
      for (int64_t s = J->col_off[cc]; s < J->col_off[cc + 1]; ++s) {
        const double a = J->z[2 * s] + w;
        const double b = J->z[2 * s + 1] - w;
        if (a < b) ivec_push(&part, a, b);
      }
      if (first) {
        out->n = 0;
        for (int64_t t = 0; t < part.n; ++t) ivec_push(out, part.v[t].a, part.v[t].b);
        first = 0;
      } else {
        intersect_into(out, &part, &tmp);
      }
      if (out->n == 0) goto done;
    }
  }
done:
  free(part.v);
  free(tmp.v);
}

static void* worker(void* arg) {
  job* J = (job*)arg;
  for (;;) {
    pthread_mutex_lock(&J->lock);
    const int64_t t0 = J->next;
    J->next += 64;
    pthread_mutex_unlock(&J->lock);
    if (t0 >= J->ncols) break;
    const int64_t t1 = t0 + 64 < J->ncols ? t0 + 64 : J->ncols;
    for (int64_t t = t0; t < t1; ++t) {
      const int64_t c = J->cols ? J->cols[t] : t;
      if (J->erode)
        erode_column(J, c, &J->res[t]);
      else
        dilate_column(J, c, &J->res[t]);
    }
  }
  return NULL;
}

/*
 * Compute the dilation (erode == 0) or erosion (erode == 1) of the requested output columns.
 * cols == NULL computes all nx*ny columns in row-major order.  On success returns the total
 * number of output segments and stores malloc'd arrays in *out_off (ncols+1 int64) and
 * *out_z (2*total doubles); free both with oracle_free.  Returns -1 on bad arguments or
 * allocation failure.
 */
int64_t oracle_offset_any(int32_t nx, int32_t ny, double h, double k, const int64_t* col_off,
                          const double* z, int erode, int slices, const int64_t* cols,
                          int64_t ncols, int nthreads, int64_t** out_off, double** out_z);

int64_t oracle_offset(int32_t nx, int32_t ny, double h, double k, const int64_t* col_off,
                      const double* z, int erode, const int64_t* cols, int64_t ncols,
                      int nthreads, int64_t** out_off, double** out_z) {
  return oracle_offset_any(nx, ny, h, k, col_off, z, erode, 0, cols, ncols, nthreads, out_off,
                           out_z);
}

/*
 * The 2D offsets of Sec. 3.2 ("2D Offsets": a 2D shape given as parallel segments on a regular
 * grid, dilated by a disk), for every row of the grid at once: slices = 1 takes only the
 * columns of the output column's own row (dj = 0), so each row is offset by a disk of radius
 * k h in its (x, z) plane.  Otherwise as oracle_offset.
 */
int64_t oracle_offset_slices(int32_t nx, int32_t ny, double h, double k, const int64_t* col_off,
                             const double* z, int erode, const int64_t* cols, int64_t ncols,
                             int nthreads, int64_t** out_off, double** out_z) {
  return oracle_offset_any(nx, ny, h, k, col_off, z, erode, 1, cols, ncols, nthreads, out_off,
                           out_z);
}

int64_t oracle_offset_any(int32_t nx, int32_t ny, double h, double k, const int64_t* col_off,
                          const double* z, int erode, int slices, const int64_t* cols,
                          int64_t ncols, int nthreads, int64_t** out_off, double** out_z) {
  if (nx <= 0 || ny <= 0 || !(h > 0) || !(k >= 0) || !col_off || !out_off || !out_z) return -1;
  if (!cols) ncols = (int64_t)nx * ny;
  for (int64_t t = 0; cols && t < ncols; ++t)
    if (cols[t] < 0 || cols[t] >= (int64_t)nx * ny) return -1;
  job J;
  memset(&J, 0, sizeof J);
  J.nx = nx;
  J.ny = ny;
  J.h = h;
  J.k = k;
  J.col_off = col_off;
  J.z = z;
  J.erode = erode;
  J.slices = slices ? 1 : 0;
  J.cols = cols;
  J.ncols = ncols;
  J.res = (ivec*)calloc((size_t)(ncols > 0 ? ncols : 1), sizeof(ivec));
  if (!J.res) return -1;
  pthread_mutex_init(&J.lock, NULL);
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  pthread_t th[256];
  int started = 0;
  for (int t = 0; t < nthreads; ++t)
    if (pthread_create(&th[t], NULL, worker, &J) == 0) ++started;
  if (started == 0) worker(&J);
  for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
  pthread_mutex_destroy(&J.lock);

  int64_t total = 0;
  for (int64_t t = 0; t < ncols; ++t) total += J.res[t].n;
  int64_t* off = (int64_t*)malloc((size_t)(ncols + 1) * sizeof(int64_t));
  double* oz = (double*)malloc((size_t)(total > 0 ? 2 * total : 2) * sizeof(double));
  if (!off || !oz) {
    free(off);
    free(oz);
    for (int64_t t = 0; t < ncols; ++t) free(J.res[t].v);
    free(J.res);
    return -1;
  }
  off[0] = 0;
  for (int64_t t = 0; t < ncols; ++t) {
    for (int64_t s = 0; s < J.res[t].n; ++s) {
      oz[2 * (off[t] + s)] = J.res[t].v[s].a;
      oz[2 * (off[t] + s) + 1] = J.res[t].v[s].b;
    }
    off[t + 1] = off[t] + J.res[t].n;
    free(J.res[t].v);
  }
  free(J.res);
  *out_off = off;
  *out_z = oz;
  return total;
}

void oracle_free(void* p) { free(p); }

/*
 * Boolean operations of two dexel grids of the same size (CSG in dexel space, Sec. 2 "(3)":
 * carried out column by column on the rays; the thick shell of Sec. 4 "3D Printing" and the
 * teaser figure is the difference of a dilation and an erosion).
 *
 * Written from point membership, one column at a time: the breakpoints of a column are the
 * endpoints of both inputs, sorted; a breakpoint v is in A when some closed segment of A
 * holds it, an open elementary interval (v_t, v_t+1) is in A when its midpoint is.  The
 * result's membership is op(in A, in B) on the elementary intervals: A or B (union), A and
 * B (intersection), A and not B (difference).  The result is the closure of those open
 * intervals, consecutive ones joined; for the union a breakpoint held by A or B that joins no
 * interval is kept as a zero-length segment (a tangent sample); intersection and difference
 * keep no zero-length results (measure zero, as for erosion).
 *   op: 0 union, 1 intersection, 2 difference.
 */
static int in_column(const double* z, int64_t s0, int64_t s1, double x) {
  for (int64_t s = s0; s < s1; ++s)
    if (z[2 * s] <= x && x <= z[2 * s + 1]) return 1;
  return 0;
}

static int cmp_double(const void* x, const void* y) {
  const double a = *(const double*)x, b = *(const double*)y;
  return a < b ? -1 : (a > b ? 1 : 0);
}

static int bool_of(int op, int a, int b) {
  if (op == 0) return a || b;
  if (op == 1) return a && b;
  return a && !b;
}

static int boolean_column(int op, const double* za, int64_t a0, int64_t a1, const double* zb,
                          int64_t b0, int64_t b1, ivec* out) {
  const int64_t m = 2 * ((a1 - a0) + (b1 - b0));
  out->n = 0;
  if (m == 0) return 0;
  double* v = (double*)malloc((size_t)m * sizeof(double));
  if (!v) return -1;
  int64_t n = 0;
  for (int64_t s = a0; s < a1; ++s) { v[n++] = za[2 * s]; v[n++] = za[2 * s + 1]; }
  for (int64_t s = b0; s < b1; ++s) { v[n++] = zb[2 * s]; v[n++] = zb[2 * s + 1]; }
  qsort(v, (size_t)n, sizeof(double), cmp_double);
  int64_t u = 0;  /* distinct breakpoints */
  for (int64_t t = 0; t < n; ++t)
    if (u == 0 || v[t] != v[u - 1]) v[u++] = v[t];
  int open = 0;   /* a result interval is being built */
  double start = 0;
  for (int64_t t = 0; t < u; ++t) {
    /* the elementary interval after breakpoint t (none after the last) */
    int after = 0;
    if (t + 1 < u) {
      const double mid = 0.5 * (v[t] + v[t + 1]);
      after = bool_of(op, in_column(za, a0, a1, mid), in_column(zb, b0, b1, mid));
    }
    if (open && !after) {  /* the interval ends at v[t] */
      if (ivec_push(out, start, v[t])) { free(v); return -1; }
      open = 0;
    } else if (!open && after) {  /* an interval starts at v[t] */
      start = v[t];
      open = 1;
    } else if (!open && !after && op == 0) {
      /* a breakpoint that joins no interval: kept by the union when A or B holds it and the
         interval before it was out too */
      const int before = t > 0 && bool_of(op, in_column(za, a0, a1, 0.5 * (v[t - 1] + v[t])),
                                          in_column(zb, b0, b1, 0.5 * (v[t - 1] + v[t])));
      if (!before && bool_of(op, in_column(za, a0, a1, v[t]), in_column(zb, b0, b1, v[t])))
        if (ivec_push(out, v[t], v[t])) { free(v); return -1; }
    }
  }
  free(v);
  return 0;
}

/* Boolean op of grids A and B (same nx*ny columns); result as for oracle_offset. */
int64_t oracle_boolean(int op, int64_t ncols, const int64_t* off_a, const double* za,
                       const int64_t* off_b, const double* zb, int64_t** out_off, double** out_z) {
  if (op < 0 || op > 2 || ncols < 0 || !off_a || !off_b || !out_off || !out_z) return -1;
  ivec* res = (ivec*)calloc((size_t)(ncols > 0 ? ncols : 1), sizeof(ivec));
  if (!res) return -1;
  int64_t total = 0;
  for (int64_t c = 0; c < ncols; ++c) {
    if (boolean_column(op, za, off_a[c], off_a[c + 1], zb, off_b[c], off_b[c + 1], &res[c])) {
      for (int64_t t = 0; t <= c; ++t) free(res[t].v);
      free(res);
      return -1;
    }
    total += res[c].n;
  }
  int64_t* off = (int64_t*)malloc((size_t)(ncols + 1) * sizeof(int64_t));
  double* oz = (double*)malloc((size_t)(total > 0 ? 2 * total : 2) * sizeof(double));
  if (!off || !oz) {
    free(off);
    free(oz);
    for (int64_t t = 0; t < ncols; ++t) free(res[t].v);
    free(res);
    return -1;
  }
  off[0] = 0;
  for (int64_t c = 0; c < ncols; ++c) {
    for (int64_t s = 0; s < res[c].n; ++s) {
      oz[2 * (off[c] + s)] = res[c].v[s].a;
      oz[2 * (off[c] + s) + 1] = res[c].v[s].b;
    }
    off[c + 1] = off[c] + res[c].n;
    free(res[c].v);
  }
  free(res);
  *out_off = off;
  *out_z = oz;
  return total;
}

/*
 * Ray casting of analytic primitives into a dexel grid (Sec. 1: implicit shapes are turned
 * into ray representations directly, without meshing; Sec. 3.1 "Dexel Representation": the
 * segments where the vertical ray of each column is inside the solid).  Column (i, j) of an
 * nx x ny grid of spacing h casts the ray x = (i + 1/2) h, y = (j + 1/2) h.  Primitives, 8
 * doubles each after an int kind:
 *   0 sphere (cx cy cz R): chord cz -+ sqrt(R^2 - d^2) where d^2 = (x-cx)^2 + (y-cy)^2 < R^2;
 *   1 box (x0 x1 y0 y1 z0 z1): [z0, z1] where x0 < x < x1 and y0 < y < y1;
 *   2 shell (cx cy cz R t): the sphere of radius R minus the open sphere of radius R - t:
 *     one chord where the ray misses the inner sphere, else the two chords between them.
 * Tangent rays (zero-length chords) are excluded by the strict inequalities.  The chords of a
 * column are united (closed union, as everywhere else here).
 */
static void raycast_column(const int* kind, const double* prm, int nprim, double x, double y,
                           ivec* out) {
  out->n = 0;
  for (int p = 0; p < nprim; ++p) {
    const double* q = prm + 8 * (size_t)p;
    if (kind[p] == 1) {
      if (x > q[0] && x < q[1] && y > q[2] && y < q[3]) ivec_push(out, q[4], q[5]);
      continue;
    }
    const double d2 = (x - q[0]) * (x - q[0]) + (y - q[1]) * (y - q[1]);
    const double R = q[3];
    if (!(d2 < R * R)) continue;
    const double so = sqrt(R * R - d2);
    if (kind[p] == 0) {
      ivec_push(out, q[2] - so, q[2] + so);
    } else {
      const double Ri = R - q[4];
      if (d2 < Ri * Ri) {
        const double si = sqrt(Ri * Ri - d2);
        ivec_push(out, q[2] - so, q[2] - si);
        ivec_push(out, q[2] + si, q[2] + so);
      } else {
        ivec_push(out, q[2] - so, q[2] + so);
      }
    }
  }
  sort_merge(out);
}

/* Ray-cast nprim primitives on an nx x ny grid of spacing h; result as for oracle_offset. */
int64_t oracle_raycast(int32_t nx, int32_t ny, double h, const int* kind, const double* prm,
                       int nprim, int64_t** out_off, double** out_z) {
  if (nx <= 0 || ny <= 0 || !(h > 0) || nprim < 0 || !out_off || !out_z) return -1;
  const int64_t ncols = (int64_t)nx * ny;
  ivec* res = (ivec*)calloc((size_t)ncols, sizeof(ivec));
  if (!res) return -1;
  int64_t total = 0;
  for (int64_t c = 0; c < ncols; ++c) {
    const double x = ((double)(c % nx) + 0.5) * h, y = ((double)(c / nx) + 0.5) * h;
    raycast_column(kind, prm, nprim, x, y, &res[c]);
    total += res[c].n;
  }
  int64_t* off = (int64_t*)malloc((size_t)(ncols + 1) * sizeof(int64_t));
  double* oz = (double*)malloc((size_t)(total > 0 ? 2 * total : 2) * sizeof(double));
  if (!off || !oz) {
    free(off);
    free(oz);
    for (int64_t t = 0; t < ncols; ++t) free(res[t].v);
    free(res);
    return -1;
  }
  off[0] = 0;
  for (int64_t c = 0; c < ncols; ++c) {
    for (int64_t s = 0; s < res[c].n; ++s) {
      oz[2 * (off[c] + s)] = res[c].v[s].a;
      oz[2 * (off[c] + s) + 1] = res[c].v[s].b;
    }
    off[c + 1] = off[c] + res[c].n;
    free(res[c].v);
  }
  free(res);
  *out_off = off;
  *out_z = oz;
  return total;
}
