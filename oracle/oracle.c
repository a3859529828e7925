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
  for (int64_t dj = -R; dj <= R; ++dj) {
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
  for (int64_t dj = -R; dj <= R; ++dj) {
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
int64_t oracle_offset(int32_t nx, int32_t ny, double h, double k, const int64_t* col_off,
                      const double* z, int erode, const int64_t* cols, int64_t ncols,
                      int nthreads, int64_t** out_off, double** out_z) {
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
