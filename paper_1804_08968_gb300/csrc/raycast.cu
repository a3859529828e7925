// Ray casting of analytic primitives into a dexel grid (Sec. 1: implicit shapes are turned
// into ray representations directly, without meshing; Sec. 3.1 "Dexel Representation": the
// segments where the vertical ray of a column is inside the solid).
//
// Column (i, j) casts the ray x = (i + 1/2) h, y = (j + 1/2) h.  A sphere (cx, cy, cz, R) gives
// the chord cz -+ sqrt(R^2 - d^2) where d^2 = (x - cx)^2 + (y - cy)^2 < R^2; a box gives
// [z0, z1] where x0 < x < x1 and y0 < y < y1; a hollow sphere (outer R, inner R - t) gives the
// sphere's chord minus the inner one's open chord.  Tangent rays (zero-length chords) are
// excluded.  The chords of a column are sorted by (start, end) and united (closed union); in
// FP32 mode each end is then rounded to the nearest float and segments that touch after
// rounding are joined.
//
// GB300 mapping: a block takes 256 consecutive columns of the row-major grid; the primitives
// pass through shared memory in chunks, each thread tests its column against all of them
// (broadcast reads) and keeps its chords in a local array.  The arithmetic uses the
// round-to-nearest intrinsics one operation at a time, so no multiply-add is contracted.
// A counting launch sizes the columns, a scan places them, a writing launch stores them.
#include "../../include/dexel.h"
#include "launch.h"

namespace dexel {

constexpr int kRcChunk = 128;  // primitives staged in shared memory at a time
constexpr int kRayChords = 160;  // chords a column may hold before they are united

// A primitive seen from rays along axis `axis` (0: x, 1: y, 2: z): the coordinates cycled so
// that the ray runs along the third one, the grid over the other two in cyclic order (x rays:
// grid (y, z); y rays: grid (z, x)).
__device__ __forceinline__ dexel_prim view_of(dexel_prim q, int axis) {
  if (axis == 2) return q;
  dexel_prim r = q;
  if (q.kind == DEXEL_BOX) {
    // bounds (x0 x1 y0 y1 z0 z1) -> (u0 u1 v0 v1 w0 w1)
    const int u = axis == 0 ? 1 : 2, v = axis == 0 ? 2 : 0, w = axis;
    r.p[0] = q.p[2 * u]; r.p[1] = q.p[2 * u + 1];
    r.p[2] = q.p[2 * v]; r.p[3] = q.p[2 * v + 1];
    r.p[4] = q.p[2 * w]; r.p[5] = q.p[2 * w + 1];
  } else {
    const double c[3] = {q.p[0], q.p[1], q.p[2]};
    r.p[0] = c[axis == 0 ? 1 : 2];
    r.p[1] = c[axis == 0 ? 2 : 0];
    r.p[2] = c[axis];
  }
  return r;
}

template <typename T, bool WRITE>
__global__ void __launch_bounds__(256) k_raycast(const dexel_prim* prims, int nprim, int axis,
                                                 int nx, long long ncols, double h, long long* cnt,
                                                 const long long* pos, T* zo, Counters* ctr) {
  __shared__ dexel_prim sp[kRcChunk];
  __shared__ int sn;
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool act = c < ncols;
  const long long cc = act ? c : ncols - 1;
  const double x = __dmul_rn((double)(cc % nx) + 0.5, h);
  const double y = __dmul_rn((double)(cc / nx) + 0.5, h);
  // the block's columns lie in this box of ray positions (the culling below is conservative:
  // the chord tests decide)
  const long long c0 = (long long)blockIdx.x * blockDim.x;
  const long long c1 = min(ncols, c0 + (long long)blockDim.x) - 1;
  const long long j0 = c0 / nx, j1 = c1 / nx;
  const double bx0 = j0 == j1 ? ((double)(c0 % nx) + 0.5) * h : 0.5 * h;
  const double bx1 = j0 == j1 ? ((double)(c1 % nx) + 0.5) * h : ((double)(nx - 1) + 0.5) * h;
  const double by0 = ((double)j0 + 0.5) * h, by1 = ((double)j1 + 0.5) * h;
  double ca[kRayChords], cb[kRayChords];
  int m = 0;
  bool over = false;
  for (int p0 = 0; p0 < nprim; p0 += blockDim.x) {
    // the primitives of this chunk whose footprint reaches the block, staged in shared memory
    // (in chunks of kRcChunk; the order does not matter, the chords are sorted)
    bool mine = false;
    dexel_prim own{};
    if (p0 + (int)threadIdx.x < nprim) {
      own = view_of(prims[p0 + threadIdx.x], axis);
      double fx0, fx1, fy0, fy1;
      if (own.kind == DEXEL_BOX) {
        fx0 = own.p[0]; fx1 = own.p[1]; fy0 = own.p[2]; fy1 = own.p[3];
      } else {
        fx0 = own.p[0] - own.p[3]; fx1 = own.p[0] + own.p[3];
        fy0 = own.p[1] - own.p[3]; fy1 = own.p[1] + own.p[3];
      }
      const double e = 2.0 * h;  // generous: rounding of the bounds cannot exclude a hit
      mine = fx1 >= bx0 - e && fx0 <= bx1 + e && fy1 >= by0 - e && fy0 <= by1 + e;
    }
    for (int base = 0; base < (int)blockDim.x; base += kRcChunk) {
      // threads base .. base + kRcChunk - 1 append their primitive if it reaches the block
      __syncthreads();
      if (threadIdx.x == 0) sn = 0;
      __syncthreads();
      if (mine && (int)threadIdx.x >= base && (int)threadIdx.x < base + kRcChunk) {
        const int slot = atomicAdd(&sn, 1);
        sp[slot] = own;
      }
      __syncthreads();
      const int np = sn;
      for (int t = 0; t < np; ++t) {
      const dexel_prim& q = sp[t];
      double a0, b0, a1 = 0, b1 = 0;
      int k = 0;
      if (q.kind == DEXEL_BOX) {
        if (x > q.p[0] && x < q.p[1] && y > q.p[2] && y < q.p[3]) {
          a0 = q.p[4];
          b0 = q.p[5];
          k = 1;
        }
      } else {
        const double dx = __dsub_rn(x, q.p[0]), dy = __dsub_rn(y, q.p[1]);
        const double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
        const double R = q.p[3], R2 = __dmul_rn(R, R);
        if (d2 < R2) {
          const double so = __dsqrt_rn(__dsub_rn(R2, d2));
          const double cz = q.p[2];
          k = 1;
          a0 = __dsub_rn(cz, so);
          b0 = __dadd_rn(cz, so);
          if (q.kind == DEXEL_SHELL) {
            const double Ri = __dsub_rn(R, q.p[4]), Ri2 = __dmul_rn(Ri, Ri);
            if (d2 < Ri2) {
              const double si = __dsqrt_rn(__dsub_rn(Ri2, d2));
              b0 = __dsub_rn(cz, si);
              a1 = __dadd_rn(cz, si);
              b1 = __dadd_rn(cz, so);
              k = 2;
            }
          }
        }
      }
      for (int e = 0; e < k; ++e) {
        if (m < kRayChords) {
          ca[m] = e == 0 ? a0 : a1;
          cb[m] = e == 0 ? b0 : b1;
          ++m;
        } else {
          over = true;
        }
      }
      }
    }
  }
  if (!act) return;
  if (over) {
    set_status(&ctr->status, ST_OVERFLOW_SLOT);
    if (!WRITE) cnt[c] = 0;
    return;
  }
  // sort by (start, end): insertion sort (a column holds a few dozen chords at most)
  for (int s = 1; s < m; ++s) {
    const double va = ca[s], vb = cb[s];
    int t = s - 1;
    while (t >= 0 && (ca[t] > va || (ca[t] == va && cb[t] > vb))) {
      ca[t + 1] = ca[t];
      cb[t + 1] = cb[t];
      --t;
    }
    ca[t + 1] = va;
    cb[t + 1] = vb;
  }
  // closed union, then (FP32) the rounding with joins of segments that now touch
  long long n = 0;
  T* dst = WRITE ? zo + 2 * pos[c] : nullptr;
  bool have = false;
  T ra = 0, rb = 0;
  auto emit = [&](double a, double b) {
    const T ta = (T)a, tb = (T)b;  // round to nearest (exact for doubles)
    if (have && ta <= rb) {
      rb = tb > rb ? tb : rb;
      return;
    }
    if (have) {
      if (WRITE) { dst[2 * n] = ra; dst[2 * n + 1] = rb; }
      ++n;
    }
    ra = ta;
    rb = tb;
    have = true;
  };
  if (m > 0) {
    double ua = ca[0], ub = cb[0];
    for (int s = 1; s < m; ++s) {
      if (ca[s] <= ub) {
        ub = cb[s] > ub ? cb[s] : ub;
      } else {
        emit(ua, ub);
        ua = ca[s];
        ub = cb[s];
      }
    }
    emit(ua, ub);
  }
  if (have) {
    if (WRITE) { dst[2 * n] = ra; dst[2 * n + 1] = rb; }
    ++n;
  }
  if (!WRITE) cnt[c] = n;
}

template <typename T>
cudaError_t launch_raycast(const dexel_prim* prims, int nprim, int axis, int nx, long long ncols,
                           double h, long long* cnt, const long long* pos, T* zo, Counters* ctr,
                           bool write, cudaStream_t st) {
  if (ncols <= 0) return cudaSuccess;
  const unsigned g = (unsigned)((ncols + 255) / 256);
  if (write)
    k_raycast<T, true><<<g, 256, 0, st>>>(prims, nprim, axis, nx, ncols, h, cnt, pos, zo, ctr);
  else
    k_raycast<T, false><<<g, 256, 0, st>>>(prims, nprim, axis, nx, ncols, h, cnt, pos, zo, ctr);
  return cudaGetLastError();
}

template cudaError_t launch_raycast<float>(const dexel_prim*, int, int, int, long long, double,
                                           long long*, const long long*, float*, Counters*, bool,
                                           cudaStream_t);
template cudaError_t launch_raycast<double>(const dexel_prim*, int, int, int, long long, double,
                                            long long*, const long long*, double*, Counters*, bool,
                                            cudaStream_t);

}  // namespace dexel
