// Host side of libdexel: the C ABI declared in include/dexel.h, workspace planning, and the
// small kernels around the two sweeps (CSR validation, half-width table, output
// compaction with the erosion complement and the final rounding).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/dexel.h"
#include "launch.h"
#include "emit.cuh"

using namespace dexel;

// The counters a synchronous offset read at its host synchronisations, in order, and whether
// its path can be replayed without them (no fallback whose launches depend on host-read data).
struct Tape {
  std::vector<Counters> snaps;
  size_t pos = 0;
  bool replayable = true;
  // the context's learnt capacities the recorded attempt planned with (the replay plans with
  // them too, so that it needs the workspace the recorded call reported)
  long long needF = 0, needM = 0, needO = 0, needL = 0;
  int capA = 0, capR = 0, capS = 0, ccap = 0;
  bool noblock = false;
  size_t need = 0;  // the workspace the recorded call needed
};

struct dexel_ctx {
  int device = 0;
  int sm_count = 0;
  // library-owned scratch, used when the caller passes ws == NULL
  void* own = nullptr;
  size_t own_bytes = 0;
  // intermediate grid of closing / opening (and the dilation of a shell), and the erosion of
  // a shell
  void* mid = nullptr;
  size_t mid_bytes = 0;
  void* aux = nullptr;
  size_t aux_bytes = 0;
  size_t last_required = 0;
  long long launches = 0;
  // capacities learnt from earlier calls (grown on overflow)
  int capA = 1024, capR = 1024, capS = 4096;
  bool sweep1 = false;  // pass 1 as the per-row sweep instead of the window gather
  bool lane1 = true;    // pass 1 with one lane per column where the windows fit
  bool merge1 = true;   // short reaches: the per-lane merge instead
  int p1l_ecap = 0;     // its event room a tile (0: planned from the density)
  int lvl_slots = 0;    // interval slots a lane of the level walks (0: by reach)
  bool p1l_tile_redo = true;  // pass 1: tiles beyond the room go whole to the redo launch
  int lvl_spill_cap = 64;     // level walks: intervals a lane spills to global memory beyond its slots
  int p1l_block_cap = 2;      // pass 1's costed room: blocks an SM counted at most
  int p1l_nbuf = 0;     // its event buffers (0: two where they cost no block an SM)
  double p1l_ecap_mul = 0;  // its event room: this many times twice the mean window's events (0: by reach)
  int p1l_gw = 0;       // its warps a tile (0: by the reach)
  bool p1l_ring = true; // one walk into a ring (else a counting walk and a writing walk)
  bool p1l_ecap_max = false;  // event room for the densest window from the start (no redo)
  bool prune1 = true;   // dominance pruning of S_mid pieces in the window kernel
  // blocks of y lines: the bytes the block-scoped scratch (S_mid, its copy, level lists) may
  // take before an offset is split into blocks (0.45 of the device memory free when the
  // context is created, or DEXEL_BLOCK_MB); noblock: a fallback needed the whole grid
  double block_bytes = 48e9;
  bool noblock = false;
  int p1l_ring_cap = 0; // pieces a lane's ring region holds at most (0: up to p1l_ring_max)
  // (measured on the 2048^2 k = 64 workload: 128 pieces left 94 k tiles walked twice and pass
  // 1 at 345 ms, 256 pieces 72 tiles and 283 ms, 512 none and 282 ms)
  int p1l_ring_max = 256;
  long long batch_max_cols = 131072;  // larger shapes of a batch take the single-shape path
  // the level walks read S_mid itself (no packed copy) at reach >= 32: off by default
  // (measured: 0.04 ms a k = 32 offset faster on the 512^2 workload, 20 % slower at k = 64
  // on the 2048^2 one, where each source is staged three times)
  bool levels_exact = false;
  int lane_gather_max = 4;  // pass-2 gather with one lane a column up to this reach
  // largest bucket (intervals a column) the level gather grows to for later calls when many
  // columns had to unite their bucket part way (DEXEL_GATHER_BUCKET_MAX)
  int bucket_max = 512;  // (measured: 4096^2 k = 128, the gather 700 ms at 2048, 320 ms at 512)
  bool sweep2 = false;  // pass 2 as the per-line sweep instead of the window gather
  // gather: bucket entries per column, learnt per (radius, op): grown when many columns
  // needed the redo launch
  std::map<int, int> ccap;
  BatchEngine* batch = nullptr;  // batched offsets (created on first use)
  bool batch_autotune = true;
  long long needF = 0, needM = 0, needO = 0, needL = 0;  // arena entries
  bool levels = true;   // pass 2 by per-source level unions (else the tiled gather)
  int levels_status = 0;  // device status after the last level pass (diagnostics)
  Counters host_ctr{};
  // optional per-stage timing with CUDA events on the call's stream
  bool profiling = false;
  cudaEvent_t ev[18] = {};  // stage pairs 0-9, kernel pairs 10-17
  double stage_ms[5] = {0, 0, 0, 0, 0};
  double kernel_ms[4] = {0, 0, 0, 0};  // pass-1 kernel, k_levels, k_lgather, S_mid pack
  bool kernel_rec[4] = {false, false, false, false};
  long long stats[15] = {};
  unsigned long long phase[16] = {};
  // Stream-ordered calls (dexel_offset_enqueue): every synchronous offset records the
  // counters it read at its host synchronisations (its "tape"); a stream-ordered call of the
  // same grid size, radius and operation replays that tape instead of reading the device.
  std::map<std::string, Tape> tapes;
  Tape* replay = nullptr;        // the tape being replayed (a stream-ordered call), else null
  long long* replay_result = nullptr;  // its device result words [status, segments]
  // batched calls: the large shapes' stream-ordered offsets run on a side stream, their
  // result words in res_buf
  cudaStream_t side = nullptr;
  long long* res_buf = nullptr;
  size_t res_n = 0;
};

namespace {

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int reach_of(double kk) {
  if (!(kk >= 0)) return -1;
  long long R = (long long)std::floor(std::sqrt(kk));
  while ((double)((R + 1) * (R + 1)) <= kk) ++R;
  while (R > 0 && (double)(R * R) > kk) --R;
  return (int)R;
}

// ------------------------------------------------------------------------------------------
// small kernels
// ------------------------------------------------------------------------------------------
template <typename T>
__global__ void k_validate(int ncols, const int* off, const T* z, long long nseg, Counters* ctr) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float zm = 0.0f;  // max |z|: the scale of pass 2's float filter
  if (c < ncols) {
    const int s0 = off[c], s1 = off[c + 1];
    bool bad = false;
    if (c == 0 && s0 != 0) bad = true;
    if (c == ncols - 1 && (long long)s1 != nseg) bad = true;
    if (s1 < s0 || s0 < 0 || (long long)s1 > nseg) bad = true;
    if (!bad) {
      for (int s = s0; s < s1; ++s) {
        const T a = z[2LL * s], b = z[2LL * s + 1];
        if (!(a <= b)) { bad = true; break; }  // also catches NaN
        if (!(a > -(T)INFINITY) || !(b < (T)INFINITY)) { bad = true; break; }
        if (s + 1 < s1 && !(b < z[2LL * (s + 1)])) { bad = true; break; }
        zm = fmaxf(zm, fmaxf(fabsf((float)a), fabsf((float)b)));
      }
      atomicMax(&ctr->max_segs_in, s1 - s0);
    }
    if (bad) atomicOr(&ctr->status, ST_BAD_CSR);
  }
  const unsigned zb = __reduce_max_sync(0xffffffffu, __float_as_uint(zm));  // zm >= 0
  if ((threadIdx.x & 31) == 0 && zb > 0) atomicMax(&ctr->zmax_bits, zb);
}

// The events of every pass-1 tile window (32 output columns of a row and the K sources on
// either side; two events a segment, two more a column for a complement), summed by bins of
// 1024 events of the window's size: the planner sizes the tiles' event room by them.
__global__ void k_win_hist(int nx, int ny, int K, int erode, const int* off, Counters* ctr) {
  __shared__ unsigned long long hb[kWinBins];
  if (threadIdx.x < kWinBins) hb[threadIdx.x] = 0;
  __syncthreads();
  const int tpr = (nx + 31) >> 5;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < (long long)tpr * ny) {
    const int j = (int)(t / tpr), i0 = (int)(t % tpr) * 32;
    const int s0 = max(0, i0 - K), s1 = min(nx, i0 + 32 + K);
    const long long rb = (long long)j * nx;
    const long long E = 2LL * (off[rb + s1] - off[rb + s0]) + (erode ? 2LL * (s1 - s0) : 0);
    const long long bb = E <= 0 ? 0 : (E - 1) >> 10;
    const int b = bb < kWinBins - 1 ? (int)bb : kWinBins - 1;
    atomicAdd(&hb[b], (unsigned long long)E);
  }
  __syncthreads();
  if (threadIdx.x < kWinBins && hb[threadIdx.x]) atomicAdd(&ctr->win_hist[threadIdx.x], hb[threadIdx.x]);
}

// Stream-ordered calls: the status bits in `fatal` are kept in the sticky word (a failure the
// call cannot recover from on the device), then the status word is cleared if asked (before
// a redo launch that sets it again for what it could not finish).
__global__ void k_fold_status(Counters* ctr, int fatal, int clear) {
  ctr->sticky |= ctr->status & fatal;
  if (clear) ctr->status = 0;
}

// Stream-ordered calls: the result words [status, output segments] -- DEXEL_OK, or
// DEXEL_ERR_BAD_CSR, DEXEL_ERR_CAPACITY (output beyond capacity_seg or int32 offsets),
// DEXEL_ERR_NO_PLAN (the data needed more than the replayed plan: a synchronous call
// re-plans) -- from the sticky status and the total (the scan's last block sum).
__global__ void k_result(Counters* ctr, const long long* total, long long cap, long long* res) {
  const int f = ctr->sticky | ctr->status;
  const long long n = *total;
  long long st = DEXEL_OK;
  if (f & ST_BAD_CSR) st = DEXEL_ERR_BAD_CSR;
  else if (f & ~(ST_TOO_MANY_OUT)) st = DEXEL_ERR_NO_PLAN;
  else if ((f & ST_TOO_MANY_OUT) || n > cap) st = DEXEL_ERR_CAPACITY;
  res[0] = st;
  res[1] = n;
}

// rows of the grid with a column marked for the pass-1 sweep (line-2 index q = i * ny + j)
__global__ void k_mark_rows(long long ncols, int ny, const long long* m_start, int* rowflag) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < ncols && m_start[q] < 0) rowflag[q % ny] = 1;
}

__global__ void k_tables(double kk, double h, int nmax, int K, double* wtab, int* reach,
                         float* wtabf) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n <= nmax) {
    wtab[n] = h * sqrt(kk - (double)n);  // half-width h sqrt(k^2 - n)
    if (wtabf) wtabf[n] = (float)wtab[n];
  }
  if (n <= K) {
    // largest dy with n + dy^2 <= k^2 for n = dx^2
    const long long d2 = (long long)n * n;
    long long R = (long long)floor(sqrt(fmax(kk - (double)d2, 0.0)));
    while ((double)(d2 + (R + 1) * (R + 1)) <= kk) ++R;
    while (R > 0 && (double)(d2 + R * R) > kk) --R;
    reach[n] = (int)R;
  }
}

template <typename T>
__global__ void k_count(int ncols, const long long* ostart, const int* ocnt, const ukey* ol,
                        const ukey* orr, int erode, long long* cnt) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncols) return;
  const long long s = ostart[c];
  cnt[c] = finalize_column<T>(ol + s, orr + s, ocnt[c], erode != 0, nullptr);
}

template <typename T>
__global__ void k_write(int ncols, const long long* ostart, const int* ocnt, const ukey* ol,
                        const ukey* orr, int erode, const long long* pos, T* z,
                        const long long* gate = nullptr) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncols) return;
  if (gate && gate[0] != DEXEL_OK) return;  // (stream-ordered calls: nothing is written on failure)
  const long long s = ostart[c];
  finalize_column<T>(ol + s, orr + s, ocnt[c], erode != 0, z + 2 * pos[c]);
}

__global__ void k_scan3(long long n, long long* pos, const long long* sums, int* col_off,
                        Counters* ctr) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) {
    const long long p = pos[t] + sums[t / kScanTile];
    pos[t] = p;
    if (p > 0x7fffffffLL) atomicOr(&ctr->status, ST_TOO_MANY_OUT);
    col_off[t] = (int)p;
  }
  if (t == n) {
    const long long tot = sums[(n + kScanTile - 1) / kScanTile];
    if (tot > 0x7fffffffLL) atomicOr(&ctr->status, ST_TOO_MANY_OUT);
    col_off[n] = (int)tot;
  }
}

// ------------------------------------------------------------------------------------------
// workspace carving
// ------------------------------------------------------------------------------------------
struct Carver {
  char* base;
  size_t cap;
  size_t used = 0;
  bool ok = true;
  void* take(size_t bytes) {
    used = align_up(used, 256);
    void* p = base ? base + used : nullptr;
    used += bytes;
    if (used > cap) ok = false;
    return ok ? p : nullptr;
  }
};

struct Ws {
  void* base;
  size_t bytes;
  bool owned;
};

void mark(dexel_ctx* ctx, int e, cudaStream_t st) {
  if (!ctx->profiling) return;
  if (!ctx->ev[e]) cudaEventCreate(&ctx->ev[e]);
  cudaEventRecord(ctx->ev[e], st);
}

// a kernel's own event pair (10 + 2 q, 11 + 2 q)
void kmark(dexel_ctx* ctx, int q, bool end, cudaStream_t st) {
  if (!ctx->profiling) return;
  mark(ctx, 10 + 2 * q + (end ? 1 : 0), st);
  if (end) ctx->kernel_rec[q] = true;
}

// With profiling on, adds the device time of the pass-1 and pass-2 stages and of the kernels
// recorded since the last call (a block of the offset) to the call's totals.
void acc_block_times(dexel_ctx* ctx) {
  if (!ctx->profiling) return;
  for (int q = 1; q <= 2; ++q) {
    float ms = 0;
    if (ctx->ev[2 * q] && ctx->ev[2 * q + 1] && cudaEventSynchronize(ctx->ev[2 * q + 1]) == cudaSuccess &&
        cudaEventElapsedTime(&ms, ctx->ev[2 * q], ctx->ev[2 * q + 1]) == cudaSuccess)
      ctx->stage_ms[q] += ms;
  }
  for (int q = 0; q < 4; ++q) {
    float ms = 0;
    if (ctx->kernel_rec[q] && cudaEventSynchronize(ctx->ev[11 + 2 * q]) == cudaSuccess &&
        cudaEventElapsedTime(&ms, ctx->ev[10 + 2 * q], ctx->ev[11 + 2 * q]) == cudaSuccess)
      ctx->kernel_ms[q] += ms;
    ctx->kernel_rec[q] = false;
  }
  cudaGetLastError();
}

void reset_call(dexel_ctx* ctx) {
  ctx->launches = 0;
  for (int q = 0; q < 4; ++q) {
    ctx->kernel_ms[q] = 0;
    ctx->kernel_rec[q] = false;
  }
  for (unsigned long long& x : ctx->phase) x = 0;
  for (double& m : ctx->stage_ms) m = 0;
  for (long long& x : ctx->stats) x = 0;
}

thread_local char g_err_detail[192] = "";

dexel_status cuda_status(cudaError_t e, int line = 0) {
  if (e == cudaSuccess) return DEXEL_OK;
  snprintf(g_err_detail, sizeof(g_err_detail), "CUDA error %d (%s) at api.cu:%d", (int)e,
           cudaGetErrorName(e), line);
  return e == cudaErrorMemoryAllocation ? DEXEL_ERR_NOMEM : DEXEL_ERR_CUDA;
}

#define CK(call)                                                 \
  do {                                                           \
    cudaError_t e_ = (call);                                     \
    if (e_ != cudaSuccess) return cuda_status(e_, __LINE__);     \
  } while (0)

dexel_status ensure_owned(dexel_ctx* ctx, size_t bytes) {
  if (ctx->own_bytes >= bytes) return DEXEL_OK;
  if (ctx->own) {
    cudaFree(ctx->own);
    ctx->own = nullptr;
    ctx->own_bytes = 0;
  }
  size_t b = align_up(bytes + bytes / 4, 1 << 20);
  if (cudaMalloc(&ctx->own, b) != cudaSuccess) {
    cudaGetLastError();
    return DEXEL_ERR_NOMEM;
  }
  ctx->own_bytes = b;
  return DEXEL_OK;
}

// the offsets a tape serves: same element type, grid size, radius, operation and kind
std::string tape_key(const dexel_grid_in* in, double k, bool erode, bool slices, size_t tsize) {
  char b[128];
  snprintf(b, sizeof(b), "%zu/%d/%d/%.17g/%d/%d", tsize, in->nx, in->ny, k, erode ? 1 : 0,
           slices ? 1 : 0);
  return b;
}

template <typename T>
struct Offset {
  // one offset (dilation of S or of its complement) of a grid into the output CSR
  // slices: every row of the grid a 2D image, offset by a disk (Sec. 3.2): pass 1 as usual,
  // pass 2 takes only the column's own level-0 list
  static dexel_status run(dexel_ctx* ctx, const dexel_grid_in* in, double k, bool erode,
                          dexel_grid_out* out, void* ws, size_t ws_bytes, cudaStream_t st,
                          bool slices);
};

template <typename T>
dexel_status Offset<T>::run(dexel_ctx* ctx, const dexel_grid_in* in, double k, bool erode,
                            dexel_grid_out* out, void* ws_user, size_t ws_user_bytes,
                            cudaStream_t st, bool slices) {
  typedef typename H<T>::K Key;
  const int nx = in->nx, ny = in->ny;
  const long long ncols = (long long)nx * ny;
  const double kk = k * k;
  const int K = reach_of(kk);
  const int nmax = (int)std::floor(kk);
  const int sms = ctx->sm_count > 0 ? ctx->sm_count : 152;
  const int blocks = sms * 4;
  const int nwarps = blocks * kWarpsPerBlock;

  if (!ctx->replay) ctx->noblock = false;
  // Stream-ordered replay (ctx->replay): the counters come from the tape of an earlier
  // synchronous call of the same offset instead of the device, every redo launch is made
  // (a redo finds nothing to do when the first launch finished everything), the status bits
  // that would have sent the synchronous call elsewhere are folded into the sticky word, and
  // the result words report them.  A synchronous call records its tape.
  Tape* const rt = ctx->replay;
  const bool replay = rt != nullptr;
  Tape rec;
  if (replay && !ws_user) return DEXEL_ERR_INVALID_ARG;
  // the learnt capacities: the tape's while replaying (the context's own put back after)
  struct Saved {
    dexel_ctx* c;
    int key;
    long long nF, nM, nO, nL;
    int cA, cR, cS, cc;
    bool nb, on;
    ~Saved() {
      if (!on) return;
      c->needF = nF; c->needM = nM; c->needO = nO; c->needL = nL;
      c->capA = cA; c->capR = cR; c->capS = cS; c->noblock = nb;
      c->ccap[key] = cc;
    }
  } saved{ctx, 2 * K + (erode ? 1 : 0), ctx->needF, ctx->needM, ctx->needO, ctx->needL,
          ctx->capA, ctx->capR, ctx->capS, ctx->ccap[2 * K + (erode ? 1 : 0)], ctx->noblock, replay};
  if (replay) {
    ctx->needF = rt->needF; ctx->needM = rt->needM; ctx->needO = rt->needO; ctx->needL = rt->needL;
    ctx->capA = rt->capA; ctx->capR = rt->capR; ctx->capS = rt->capS; ctx->noblock = rt->noblock;
    ctx->ccap[2 * K + (erode ? 1 : 0)] = rt->ccap;
  }
  for (int attempt = 0; attempt < (replay ? 1 : 24); ++attempt) {
    rec.snaps.clear();
    rec.replayable = true;
    rec.needF = ctx->needF; rec.needM = ctx->needM; rec.needO = ctx->needO; rec.needL = ctx->needL;
    rec.capA = ctx->capA; rec.capR = ctx->capR; rec.capS = ctx->capS; rec.noblock = ctx->noblock;
    rec.ccap = ctx->ccap[2 * K + (erode ? 1 : 0)];
    // ---------------- plan
    // phase A: counters, tables, indices, validation
    void* pwtabf = nullptr;
    auto plan = [&](Carver& C, void** pctr, void** pwtab, void** preach, void** pmstart,
                    void** pmcnt, void** postart, void** pocnt, void** pcnt, void** ppos,
                    void** psums) {
      *pctr = C.take(sizeof(Counters));
      *pwtab = C.take(sizeof(double) * (nmax + 2));
      pwtabf = C.take(sizeof(float) * (nmax + 2));
      *preach = C.take(sizeof(int) * (K + 2));
      *pmstart = C.take(sizeof(long long) * ncols);
      *pmcnt = C.take(sizeof(int) * ncols);
      *postart = C.take(sizeof(long long) * ncols);
      *pocnt = C.take(sizeof(int) * ncols);
      *pcnt = C.take(sizeof(long long) * (ncols + 1));
      *ppos = C.take(sizeof(long long) * (ncols + 1));
      *psums = C.take(sizeof(long long) * ((ncols + kScanTile) / kScanTile + 2));
    };
    Carver probe{nullptr, (size_t)-1};
    void *pctr, *pwtab, *preach, *pmstart, *pmcnt, *postart, *pocnt, *pcnt, *ppos, *psums;
    plan(probe, &pctr, &pwtab, &preach, &pmstart, &pmcnt, &postart, &pocnt, &pcnt, &ppos, &psums);
    const size_t fixed = align_up(probe.used, 256);
    // input statistics first (needs only the fixed part)
    Ws W;
    if (ws_user) {
      W = {ws_user, ws_user_bytes, false};
      if (ws_user_bytes < fixed) {
        ctx->last_required = fixed;
        return DEXEL_ERR_CAPACITY;
      }
    } else {
      dexel_status s = ensure_owned(ctx, fixed + (64u << 20));
      if (s != DEXEL_OK) return s;
      W = {ctx->own, ctx->own_bytes, true};
    }
    Carver C{(char*)W.base, W.bytes};
    plan(C, &pctr, &pwtab, &preach, &pmstart, &pmcnt, &postart, &pocnt, &pcnt, &ppos, &psums);
    Counters* ctr = (Counters*)pctr;
    CK(cudaMemsetAsync(ctr, 0, sizeof(Counters), st));
    mark(ctx, 0, st);
    {
      const int thr = 256;
      k_validate<T><<<(unsigned)((ncols + thr - 1) / thr), thr, 0, st>>>(
          (int)ncols, in->col_off, (const T*)in->z, in->nseg, ctr);
      ++ctx->launches;
      k_tables<<<(std::max(nmax, K) + 1 + 255) / 256, 256, 0, st>>>(
          kk, in->h, nmax, K, (double*)pwtab, (int*)preach, (float*)pwtabf);
      ++ctx->launches;
      if (ctx->lane1 && K > kMergeMaxReach && K <= kLaneMaxReach1) {
        const long long ntl = (long long)ny * ((nx + 31) / 32);
        k_win_hist<<<(unsigned)((ntl + 255) / 256), 256, 0, st>>>(nx, ny, K, erode ? 1 : 0, in->col_off, ctr);
        ++ctx->launches;
      }
      CK(cudaGetLastError());
    }
    mark(ctx, 1, st);
    Counters hc;
    // the counters at a host synchronisation (recorded), or the tape's (replayed)
    auto rd = [&](Counters& h) -> dexel_status {
      if (replay) {
        if (rt->pos >= rt->snaps.size()) return DEXEL_ERR_NO_PLAN;
        h = rt->snaps[rt->pos++];
        return DEXEL_OK;
      }
      cudaError_t e = cudaMemcpyAsync(&h, ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return cuda_status(e, __LINE__);
      rec.snaps.push_back(h);
      return DEXEL_OK;
    };
    auto fold = [&](int fatal, bool clear) {
      k_fold_status<<<1, 1, 0, st>>>(ctr, fatal, clear ? 1 : 0);
      ++ctx->launches;
    };
#define RD(h)                               \
  do {                                      \
    const dexel_status rs_ = rd(h);         \
    if (rs_ != DEXEL_OK) return rs_;        \
  } while (0)
    RD(hc);
    if (hc.status & ST_BAD_CSR) return DEXEL_ERR_BAD_CSR;

    // ---------------- pass 1 plan
    const int capS = hc.max_segs_in + 2;
    long long capF_ll = 2LL * (K + 1) * capS + 8;
    const int capF = (int)std::min<long long>(capF_ll, 1 << 24);
    const int items1_target = nwarps * 2;
    int nch1 = std::max(1, std::min(nx, (items1_target + ny - 1) / ny));
    int chunk1 = (nx + nch1 - 1) / nch1;
    nch1 = (nx + chunk1 - 1) / chunk1;
    const long long sb1 = p1_slot_bytes<Key>(capF, capS, chunk1);
    // arena estimates (entries)
    const long long segs = std::max<long long>(in->nseg + ncols, 1024);
    long long eM = std::max<long long>(ctx->needM + ctx->needM / 8, segs * std::min(K + 2, 64));
    long long eF = std::max<long long>(ctx->needF + ctx->needF / 8, eM);
    long long eO = std::max<long long>(ctx->needO + ctx->needO / 8, segs * 2);
    long long eL = std::max<long long>(ctx->needL + ctx->needL / 8, 2 * ncols * (long long)(K + 1));
    // Blocks of whole y lines (x ranges [xa, xb)): pass 1 and pass 2 run block by block, so
    // that S_mid, its packed copy and the level lists exist for one block at a time (output
    // column (i, j) needs S_mid of line i only).  Only the lane kernel's path with the level
    // unions takes blocks; the estimates above are for the whole grid, a block gets its share
    // with a margin for uneven lines.
    const size_t pe = 2 * sizeof(Key) + 2;
    const double grid_bytes = (double)eM * pe + (double)eF * std::max<size_t>(pe, 16) +
                              (double)ncols * (2 * K + 1) * 8 + (double)eL * 16;
    const bool can_block = !ctx->sweep1 && !ctx->sweep2 && ctx->levels && ctx->lane1 &&
                           !ctx->noblock && K > kMergeMaxReach && K <= kLaneMaxReach1;
    int nb = 1, bw = nx;
    if (can_block && grid_bytes > (double)ctx->block_bytes) {
      nb = (int)std::ceil(grid_bytes / (double)ctx->block_bytes);
      bw = ((nx + nb - 1) / nb + 31) & ~31;
      if (bw >= nx) {
        bw = nx;
        nb = 1;
      } else {
        nb = (nx + bw - 1) / bw;
      }
    }
    const double bfrac = nb > 1 ? std::min(1.0, 1.3 * (double)bw / (double)nx) : 1.0;
    const long long eMb = nb > 1 ? (long long)(eM * bfrac) + 4096 : eM;
    const long long eFb = nb > 1 ? (long long)(eF * bfrac) + 4096 : eF;
    const long long eLb = nb > 1 ? (long long)(eL * bfrac) + 4096 : eL;
    const size_t bF = align_up((size_t)eFb * std::max<size_t>(pe, 16), 256);
    const size_t bM = align_up((size_t)eMb * pe, 256);
    const size_t bO = align_up((size_t)eO * 16, 256);
    // pass-2 slot estimate from the remembered capacities
    const long long sb2_est =
        p2_slot_bytes<Key>(std::max(capS * 4, 64), ctx->capR, ctx->capA, ctx->capS, 1024);
    const size_t slots_sw = std::max((size_t)sb1, (size_t)sb2_est) * nwarps;
    // the pass-2 level lists (one block's) use the same room as the sweeps' slots (never both
    // at once)
    const long long nlev = (long long)bw * ny * (2 * K + 1);  // index entries (8 B each)
    const size_t bL = K <= kGatherMaxReach ? align_up((size_t)nlev * 8 + 512, 256) + (size_t)eLb * 16 : 0;
    const size_t slots = std::max(slots_sw, bL);
    const size_t total = fixed + bF + bM + bO + slots + 4096;
    if (ws_user && total > ws_user_bytes) {
      ctx->last_required = total;
      return DEXEL_ERR_CAPACITY;
    }
    if (!ws_user) {
      dexel_status s = ensure_owned(ctx, total);
      if (s != DEXEL_OK) return s;
      if (ctx->own != W.base) {  // reallocated: the fixed part moved
        continue;
      }
    }
    char* aF = (char*)C.take(bF);
    char* aM = (char*)C.take(bM);
    char* aO = (char*)C.take(bO);
    const size_t slot_room = (W.bytes > C.used + 256) ? W.bytes - align_up(C.used, 256) - 256 : 0;
    char* pslots = (char*)C.take(slot_room);
    if (!C.ok || !aF || !aM || !aO || !pslots) {
      ctx->last_required = total;
      if (ws_user) return DEXEL_ERR_CAPACITY;
      continue;
    }

    // ---------------- pass 1
    P1Params<T> p1{};
    p1.nx = nx; p1.ny = ny; p1.K = K; p1.erode = erode ? 1 : 0;
    p1.chunk = chunk1; p1.nchunks = nch1;
    p1.col_off = in->col_off; p1.z = (const T*)in->z;
    const long long capF1 = (long long)(bF / (2 * sizeof(Key) + 2));
    p1.f_a = (Key*)aF; p1.f_b = (Key*)aF + capF1; p1.f_l = (short*)((Key*)aF + 2 * capF1);
    p1.f_cap = capF1;
    const long long capM = (long long)(bM / (2 * sizeof(Key) + 2));
    p1.m_a = (Key*)aM; p1.m_b = (Key*)aM + capM; p1.m_l = (short*)((Key*)aM + 2 * capM);
    p1.m_cap = capM;
    p1.m_start = (long long*)pmstart; p1.m_cnt = (int*)pmcnt;
    p1.blk = 256;
    p1.ctr = ctr;
    p1.slots = pslots; p1.slot_bytes = sb1;
    p1.capF = capF; p1.capS = capS;
    const int nw1 = (int)std::min<long long>(nwarps, (long long)(slot_room / sb1));
    if (nw1 < kWarpsPerBlock) {
      ctx->last_required = total + (size_t)sb1 * kWarpsPerBlock;
      if (ws_user) return DEXEL_ERR_CAPACITY;
      ensure_owned(ctx, ctx->last_required);
      continue;
    }
    // pass-2 columns start unmarked (a gather marks those it hands back with count -1)
    CK(cudaMemsetAsync(pocnt, 0, sizeof(int) * ncols, st));
    if (replay) {
      // (a pass 1 that stops on a malformed input leaves empty columns behind it)
      CK(cudaMemsetAsync(pmstart, 0, sizeof(long long) * ncols, st));
      CK(cudaMemsetAsync(pmcnt, 0, sizeof(int) * ncols, st));
    }
    bool again = false;  // an arena outgrew its estimate: plan again
    long long mid_sum = 0;  // S_mid pieces over the blocks
    for (int blk = 0; blk < nb; ++blk) {
    const int xa = blk * bw, xb = std::min(nx, xa + bw);
    const long long q0 = (long long)xa * ny, nq = (long long)(xb - xa) * ny;  // line order
    const double to_grid = (double)ncols / (double)nq;  // a block's needs scaled to the grid
    if (nb > 1) {
      // a block starts with empty arenas 0-2 (the pass-2 intervals of arena 3 accumulate)
      p1.xa = xa;
      p1.xb = xb;
      CK(cudaMemsetAsync(&ctr->arena_top[0], 0, 3 * sizeof(unsigned long long), st));
      CK(cudaMemsetAsync(&ctr->mid_total, 0, sizeof(ctr->mid_total), st));
    }
    mark(ctx, 2, st);
    bool sweep1 = ctx->sweep1 || K > (ctx->lane1 ? kLaneMaxReach1 : kGatherMaxReach1);
    if (!sweep1) {
      // gather: tiles of tc columns whose window's events (two per segment, two more per
      // column for a complement) fit ecap; a window beyond ecap hands the call to the sweep
      const double ev_col = 2.0 * (double)in->nseg / (double)std::max<long long>(ncols, 1) + (erode ? 2.0 : 0.0);
      // room for the densest single column's window, so that no row needs the sweep
      const double ev_win_max = (2.0 * K + 1) * 2.0 * (hc.max_segs_in + 1);
      // one lane per column: a tile of 32 columns, its window's events (32 + 2K columns) in
      // ecap events of shared memory, room for the densest single column's window
      const double ev_tile = (32.0 + 2.0 * K + 1) * ev_col * 2.0;
      if (ctx->merge1 && K <= kMergeMaxReach) {
        // short reaches: one lane a column, merging its own window's sources
        kmark(ctx, 0, false, st);
        CK(launch_pass1m<T>(p1, sms, st));
        kmark(ctx, 0, true, st);
        ++ctx->launches;
      } else if (ctx->lane1 && K <= kLaneMaxReach1) {
        // Event room of a tile.  A window beyond the room is, with a redo launch behind the
        // first (room ecapR, one group of 8 warps), marked whole for it; else split into
        // narrower runs of columns, which at wide reaches stage most of the window again.  A
        // window within half of the room is merged from its sources' runs in the other half.
        // The walks cost about the same warp cycles an event whatever the room, so the room
        // is the one with the least events / resident warps over both launches, from the
        // histogram of the tiles' window sizes (measured, 2048^2 k = 64 FP64: 8192 events at
        // two blocks an SM with the densest tiles redone against 16384 at one block an SM;
        // the rules in the else branch are the earlier ones, kept as switches).
        const int ecapR = 16384;  // the redo's event room (room for the densest window)
        const int ksz = sizeof(T) == 4 ? 4 : 8;  // the window kernel's event keys
        const int gw0 = ctx->p1l_gw > 0 ? ctx->p1l_gw : (K <= 12 ? 2 : (K <= 48 ? 4 : 8));
        // warps a tile (more as the windows grow: a tile's walk is split over its warps, its
        // sort shared; measured best on the 512^2 workload: 2 up to k = 8, 4 at k = 32), and
        // event buffers (a second one where it costs no block an SM)
        struct P1Plan { int gw, nbuf, warps_sm; };
        auto plan_for = [&](int room) {
          P1Plan pl{gw0, 1, 0};
          while (pl.gw < 8 && pass1l_smem(K, room, pl.gw, ksz) > (220LL << 10)) pl.gw <<= 1;
          auto per_sm = [&](int nb) { return std::min<long long>(3, (220LL << 10) / pass1l_smem(K, room, pl.gw, ksz, nb)); };
          pl.nbuf = per_sm(2) >= 1 && per_sm(2) == per_sm(1) ? 2 : 1;
          if (ctx->p1l_nbuf > 0) pl.nbuf = ctx->p1l_nbuf;
          if (pass1l_smem(K, room, pl.gw, ksz, pl.nbuf) > (220LL << 10)) pl.nbuf = 1;
          // (a third block an SM runs the 80-register plan, whose spills cost about what the
          // block gains: measured 136 against 122 ms at 2048^2 FP32, 461 against 434 ms at
          // 4096^2 k = 128 FP64; counted as two)
          pl.warps_sm = (int)std::min<long long>(ctx->p1l_block_cap, per_sm(pl.nbuf)) * 8;
          return pl;
        };
        const bool redo_fits = pass1l_smem(K, ecapR, 8, ksz) <= (220LL << 10);
        double all = 0;
        for (int b = 0; b < kWinBins; ++b) all += (double)hc.win_hist[b];
        auto beyond = [&](int room) {  // (a bin reaching above the room counts whole)
          double x = 0;
          for (int b = 0; b < kWinBins; ++b)
            if (1024LL * (b + 1) > room || b == kWinBins - 1) x += (double)hc.win_hist[b];
          return x;
        };
        int ecapL = 512;
        // (at reaches below 48 the mean rule: the 512^2 step at k <= 32 took 12.35 ms with it
        // against 12.66 with the costed room)
        const bool by_cost = ctx->p1l_ecap_mul <= 0 && !ctx->p1l_ecap_max && ctx->p1l_ecap <= 0 && K >= 48;
        if (by_cost) {
          const double wR = (double)std::max(1, plan_for(ecapR).warps_sm);
          // candidates: the powers of two, and the largest rooms that leave 1, 2 or 3 blocks
          // an SM (a room need not be a power of two)
          std::vector<int> rooms;
          for (int room = 512; room <= ecapR; room <<= 1) rooms.push_back(room);
          for (int nbk = 1; nbk <= 3; ++nbk) {
            int lo = 512, hi = ecapR;
            auto fits = [&](int room) { return pass1l_smem(K, room, gw0, ksz) * nbk <= (220LL << 10); };
            if (!fits(lo)) continue;
            while (hi - lo > 64) {
              const int mid = (lo + hi) / 2 & ~63;
              if (fits(mid)) lo = mid; else hi = mid;
            }
            rooms.push_back(fits(hi) ? hi : lo);
          }
          std::sort(rooms.begin(), rooms.end());
          double best = 0;
          bool first = true;
          for (int room : rooms) {
            const P1Plan pl = plan_for(room);
            if (pl.warps_sm <= 0) continue;
            const double out = beyond(room), in = all - out;
            // (windows beyond the largest room: narrower runs, about three times the events)
            const double cost = room < ecapR && redo_fits ? in / pl.warps_sm + out / wR
                                                          : (in + 3.0 * out) / pl.warps_sm;
            if (first || cost <= best * 1.0001) {  // (ties: the larger room)
              best = cost;
              ecapL = room;
              first = false;
            }
          }
        } else {
          // room for p1l_ecap_mul times twice the mean window (rule "mean"), for the densest
          // window (rule "max"), or as set
          const double mul = ctx->p1l_ecap_mul > 0 ? ctx->p1l_ecap_mul : 1.0;
          while (ecapL < 16384 && (ecapL < mul * ev_tile || (ctx->p1l_ecap_max && ecapL < ev_win_max))) ecapL <<= 1;
          if (ctx->p1l_ecap > 0) ecapL = ctx->p1l_ecap;
        }
        ctx->stats[13] = ecapL;
        const P1Plan pl1 = plan_for(ecapL);
        const int gw = pl1.gw, nbuf = pl1.nbuf;
        p1.nbuf = nbuf;
        const bool redo_ok = ecapL < ecapR && redo_fits;
        p1.tile_redo = redo_ok && ctx->p1l_tile_redo ? 1 : 0;
        // the ring of the one-walk variant in the (free) forward arena: up to 128 pieces a
        // thread of the grid
        {
          // threads of the larger of the two launches (the first, and the redo's)
          long long thr = (long long)pass1l_blocks(nx, ny, K, ecapL, gw, sms, ksz, nbuf) * 256;
          if (redo_ok)
            thr = std::max<long long>(thr, (long long)pass1l_blocks(nx, ny, K, ecapR, 8, sms, ksz) * 256);
          const long long esz = 2 * (long long)sizeof(Key) + 2;
          long long rc = std::min<long long>(ctx->p1l_ring_max, (long long)bF / (thr * esz)) & ~7LL;
          if (ctx->p1l_ring_cap > 0) rc = std::min<long long>(rc, ctx->p1l_ring_cap);
          if (rc >= 16 && ctx->p1l_ring) {
            const long long n = thr * rc;
            p1.r_a = (Key*)aF;
            p1.r_b = p1.r_a + n;
            p1.r_l = (short*)(p1.r_b + n);
            p1.r_cap = (int)rc;
            p1.r_n = n;
          }
        }
        if (ctx->prune1) {
          // dominance pruning of S_mid pieces: margin 2^-19 (max |z| + k h), over four times
          // the error bound of the float test (computed on the device from the validation's
          // max |z|)
          p1.prune_w = (const float*)pwtabf;
          p1.prune_zmax = &ctr->zmax_bits;
          p1.prune_kh = k * in->h;
        }
        int* rowmark = (int*)ppos;  // free until pass 2
        CK(cudaMemsetAsync(rowmark, 0, sizeof(int) * ny, st));
        p1.rowmark = rowmark;
        kmark(ctx, 0, false, st);
        CK(launch_pass1l<T>(p1, ecapL, gw, sms, st));
        ++ctx->launches;
        if (redo_ok) {
          // columns whose window did not fit: a second launch for them alone, with room for
          // the densest window (the first launch flagged their rows and marked them)
          RD(hc);
          if (replay || ((hc.status & ST_OVERFLOW_SLOT) && !(hc.status & ST_OVERFLOW_ARENA))) {
            if (replay)
              fold(~ST_OVERFLOW_SLOT, true);
            else
              CK(cudaMemsetAsync(&ctr->status, 0, sizeof(int), st));
            P1Params<T> pr = p1;
            pr.redo = 1;
            pr.nbuf = 1;  // (the densest windows: one buffer of ecapR events)
            CK(launch_pass1l<T>(pr, ecapR, 8, sms, st));
            ++ctx->launches;
            if (!replay) ++ctx->stats[8];  // a pass-1 redo launch
          }
        }
        kmark(ctx, 0, true, st);
      } else {
        // (a tile of about K/2 columns: a column's window then covers ~80 % of the tile's;
        // measured best of K/4 .. 2K on the 512^2 and 2048^2 workloads)
        int ecap = 2048, tc = 8;
        while (tc < 64 && tc < K / 2) tc <<= 1;
        while (tc > 8 && (tc + 2.0 * K + 1) * ev_col * 1.5 > 16384) tc >>= 1;
        while (ecap < 16384 && (tc + 2.0 * K + 1) * ev_col * 1.5 > ecap) ecap <<= 1;
        while (ecap < 16384 && ev_win_max > ecap) ecap <<= 1;
        int obuf = 256;
        while (obuf > 32 && pass1g_smem<T>(tc, K, ecap, obuf) > (220LL << 10)) obuf >>= 1;
        while (ecap > 1024 && pass1g_smem<T>(tc, K, ecap, obuf) > (220LL << 10)) ecap >>= 1;
        const long long sm1 = pass1g_smem<T>(tc, K, ecap, obuf);
        const int per_sm = (int)std::max<long long>(1, std::min<long long>(8, (220LL << 10) / sm1));
        const long long ntiles = (long long)ny * ((nx + tc - 1) / tc);
        const int b1 = (int)std::max<long long>(1, std::min<long long>((long long)sms * per_sm, ntiles));
        CK(launch_pass1g<T>(p1, tc, ecap, obuf, b1, st));
        ++ctx->launches;
        rec.replayable = false;  // (its own fallbacks)
      }
      RD(hc);
      if ((hc.status & ST_OVERFLOW_SLOT) && !(hc.status & ST_OVERFLOW_ARENA)) {
        rec.replayable = false;  // (the rows' list comes from the device)
        if (replay) return DEXEL_ERR_NO_PLAN;
        // columns whose window had more events than fit (marked m_start = -1): the sweep
        // redoes their rows
        int* rowflag = (int*)ppos;  // free until pass 2
        CK(cudaMemsetAsync(rowflag, 0, sizeof(int) * ny, st));
        k_mark_rows<<<(unsigned)((ncols + 255) / 256), 256, 0, st>>>(ncols, ny, p1.m_start, rowflag);
        std::vector<int> hf(ny);
        CK(cudaMemcpyAsync(hf.data(), rowflag, sizeof(int) * ny, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        std::vector<int> rows;
        for (int j = 0; j < ny; ++j)
          if (hf[j]) rows.push_back(j);
        CK(cudaMemcpyAsync(rowflag, rows.data(), sizeof(int) * rows.size(), cudaMemcpyHostToDevice, st));
        CK(cudaMemsetAsync(&ctr->status, 0, sizeof(int), st));
        P1Params<T> pr = p1;
        pr.rows = rowflag;
        pr.nrows = (int)rows.size();
        CK(launch_pass1<T>(pr, nw1 / kWarpsPerBlock, st));
        ++ctx->launches;
        RD(hc);
      }
    }
    if (sweep1) {
      rec.replayable = false;
      if (replay) return DEXEL_ERR_NO_PLAN;
      CK(launch_pass1<T>(p1, nw1 / kWarpsPerBlock, st));
      ++ctx->launches;
      RD(hc);
    }
    if (replay) fold(~0, false);  // (whatever pass 1 could not finish)
    mark(ctx, 3, st);
    ctx->stats[10] += hc.ring_spills;
    ctx->needF = std::max<long long>(ctx->needF, (long long)(hc.arena_top[0] * to_grid));
    ctx->needM = std::max<long long>(ctx->needM, (long long)(hc.arena_top[1] * to_grid));
    mid_sum += (long long)hc.mid_total;
    ctx->stats[6] = hc.status;
    ctx->stats[7] = attempt + 1;
    if (hc.status & (ST_OVERFLOW_SLOT | ST_OVERFLOW_ARENA)) {
      ctx->last_required = total + (size_t)(hc.arena_top[0] + hc.arena_top[1]) * 16;
      if (hc.status & ST_OVERFLOW_SLOT) return DEXEL_ERR_CAPACITY;  // bound exceeded: give up
      if (ws_user) return DEXEL_ERR_CAPACITY;
      again = true;
      break;
    }

    // ---------------- pass 2: window gather (default) or per-line sweep
    bool use_sweep = (ctx->sweep2 && !slices) || K > kGatherMaxReach;
    if (use_sweep && slices) return DEXEL_ERR_INVALID_ARG;  // beyond the slices' reach
    if (!use_sweep) {
      P2GParams<T> pg{};
      pg.nx = nx; pg.ny = ny; pg.R = K; pg.kk = kk; pg.nmax = nmax;
      pg.wtab = (const double*)pwtab; pg.wtabf = (const float*)pwtabf; pg.reach = (const int*)preach;
      pg.m_a = p1.m_a; pg.m_b = p1.m_b; pg.m_l = p1.m_l;
      pg.m_start = p1.m_start; pg.m_cnt = p1.m_cnt;
      const long long capO = (long long)(bO / 16);
      pg.o_l = (ukey*)aO; pg.o_r = (ukey*)aO + capO; pg.o_cap = capO;
      pg.o_start = (long long*)postart; pg.o_cnt = (int*)pocnt;
      pg.blk = 256;
      pg.ctr = ctr;
      // line-contiguous float copy of S_mid in the (now free) pass-1 forward arena: made here
      // unless the level walks read S_mid itself (DEXEL_LEVELS_EXACT=1, reach >= 32: each
      // piece is then rounded once as it is staged); the tiled gather always needs it
      const long long capC = (long long)(bF / 10);
      if ((long long)hc.mid_total > capC) return DEXEL_ERR_CAPACITY;  // not reached: bF >= 16 eM
      float* c_af = (float*)aF;
      float* c_bf = c_af + capC;
      short* c_dx = (short*)(c_bf + capC);
      bool packed = false;
      auto pack_lines = [&]() -> cudaError_t {
        kmark(ctx, 3, false, st);
        // the block's columns q0 .. q0 + nq - 1 (line order), packed from 0
        const long long nsb = (nq + kScanTile - 1) / kScanTile;
        k_scan1<int><<<(unsigned)nsb, kScanThreads, 0, st>>>(nq, (const int*)pmcnt + q0, (long long*)ppos,
                                                         (long long*)psums);
        k_scan2<<<1, kScanThreads, 0, st>>>(nsb, (long long*)psums);
        k_mid_pack<Key><<<sms * 8, 256, 0, st>>>(nq, p1.m_start + q0, p1.m_cnt + q0, p1.m_a, p1.m_b,
                                                 p1.m_l, (const long long*)ppos, (const long long*)psums,
                                                 (long long*)pcnt + q0, c_af, c_bf, c_dx, ctr,
                                                 p1.m_cap, capC);
        kmark(ctx, 3, true, st);
        ctx->launches += 3;
        pg.c_start = (const long long*)pcnt;
        pg.c_af = c_af; pg.c_bf = c_bf; pg.c_dx = c_dx;
        packed = true;
        return cudaGetLastError();
      };
      const bool levels_exact = ctx->levels && K >= 32 && ctx->levels_exact;
      if (!levels_exact) CK(pack_lines());
      int& cc = ctx->ccap[2 * K + (erode ? 1 : 0)];
      if (cc < 128) cc = 128;
      pg.bcap = cc;
      // tiled kernel geometry: the first of (warps a block, blocks an SM) = (16, 2) (the
      // kernel compiled for 64 registers, for short windows), (16, 1), (8, 1), (4, 1) whose
      // shared memory leaves room to stage the window of a tile of >= 16 columns (the
      // per-warp buckets compete with the staging area)
      {
        const int ntab = nmax + 1 <= 4096 ? nmax + 1 : 0;
        const double avg = (double)hc.mid_total / (double)std::max<long long>(nq, 1);
        int tw = 16, tc = 0, per_sm = 2, stage_cap = 0;
        const int cand[4][2] = {{16, 2}, {16, 1}, {8, 1}, {4, 1}};
        for (const auto& cd : cand) {
          if (cd[1] == 2 && K > 12) continue;
          tw = cd[0];
          per_sm = cd[1];
          const long long budget = per_sm == 2 ? (108LL << 10) : (220LL << 10);
          const P2TLayout base = p2t_layout(K, 128, ntab, 0, tw, pg.bcap);
          const long long room = budget - base.total - 64;
          stage_cap = room > 0 ? (int)std::min<long long>(room / 10, 1 << 22) : 0;
          for (tc = 128; tc >= 16; tc >>= 1)
            if ((tc + 2.0 * K + 1) * avg * 1.25 <= stage_cap) break;
          if (tc >= 16) break;
        }
        if (tc < 16) tc = 16;
        if (stage_cap < 256) return DEXEL_ERR_CAPACITY;  // not reached for K <= kGatherMaxReach
        const int ntiles_cap = nx * ((ny + tc - 1) / tc);
        const int tblocks = std::max(1, std::min(sms * per_sm, ntiles_cap));
        mark(ctx, 4, st);  // the stage covers the pass-2 kernels only (not the copy above)
        bool done = false;
        if ((ctx->levels || slices) && slot_room >= bL && bL > 0) {
          // per-source level unions in the sweeps' slot room, then the per-column gather
          LvlParamsHost<T> H;
          H.P = pg;
          H.l_idx = (unsigned long long*)pslots;
          const size_t ib = align_up((size_t)nlev * 8 + 512, 256);
          // the walks' spill regions at the end of the room, when it has them to spare
          const int scap = ctx->lvl_spill_cap;
          const size_t sb = scap > 0 ? align_up((size_t)lvl_spill_bytes(sms, scap), 256) : 0;
          const bool spill = sb > 0 && slot_room > ib + 2 * sb + 256;
          const size_t so = spill ? (slot_room - sb) / 256 * 256 : slot_room;  // spill offset
          H.l_cap = (long long)((so - ib) / 16);
          H.l_p = (ulonglong2*)(pslots + ib);
          if (spill) {
            H.spill = (unsigned*)(pslots + so);  // [so, so + sb) within the room
            H.spill_cap = scap;
          }
          int& lb = ctx->ccap[2 * K + (erode ? 1 : 0)];
          if (lb < 256) lb = 256;
          H.bcap = lb;
          H.m_cap = p1.m_cap;
          H.c_cap = capC;
          H.exact = !packed;
          H.q0 = q0;
          H.nq = nq;
          H.yw = slices ? 0 : -1;
          H.slots = ctx->lvl_slots;
          kmark(ctx, 1, false, st);
          CK(launch_levels<T>(H, st, sms));
          kmark(ctx, 1, true, st);
          kmark(ctx, 2, false, st);
          if (K <= ctx->lane_gather_max)
            CK(launch_lgather_lanes<T>(H, st, sms));
          else
            CK(launch_lgather<T>(H, H.bcap, 0, st, sms));
          kmark(ctx, 2, true, st);
          ctx->launches += 2;
          RD(hc);
          ctx->needL = std::max<long long>(ctx->needL, (long long)(hc.arena_top[2] * to_grid));
          ctx->stats[11] = std::max<long long>(ctx->stats[11], hc.over_cols);
          ctx->stats[12] = std::max<long long>(ctx->stats[12], H.bcap);
          ctx->stats[14] += (long long)hc.lvl_redo;
          ctx->levels_status = hc.status;
          if (hc.over_cols * 64LL > ncols && !replay) {
            // many columns outgrew the bucket (united straight from the lists, slower): a
            // bucket for their need in the next calls of this reach and operation
            int b = lb;
            while (b < hc.over_max && b < ctx->bucket_max) b <<= 1;
            lb = b;
          }
          if ((hc.status & ST_LEVELS_OVER) && (nb > 1 || slices)) {
            // the level arena outgrew its share: plan again with its need (the tiled gather
            // would take the whole grid)
            ctx->needL = std::max<long long>(ctx->needL, (long long)(hc.arena_top[2] * to_grid * 1.25));
            ctx->last_required = total + (size_t)hc.arena_top[2] * 16;
            if (ws_user) return DEXEL_ERR_CAPACITY;
            again = true;
            break;
          }
          if (hc.status & ST_LEVELS_OVER) {
            // a list beyond its buffer or the arena: the tiled gather redoes pass 2
            rec.replayable = false;
            if (replay) return DEXEL_ERR_NO_PLAN;
            CK(cudaMemsetAsync(&ctr->status, 0, sizeof(int), st));
            CK(cudaMemsetAsync(&ctr->arena_top[3], 0, sizeof(unsigned long long), st));
            CK(cudaMemsetAsync(&ctr->out_total, 0, sizeof(unsigned long long), st));
            CK(cudaMemsetAsync(&ctr->max_state, 0, sizeof(int), st));
            CK(cudaMemsetAsync(&ctr->redo_cols, 0, sizeof(int), st));
          } else {
            done = true;
            const bool redo_rec = (hc.status & ST_OVERFLOW_SLOT) && !(hc.status & ST_OVERFLOW_ARENA);
            if (replay) {
              // (the lists' failures are final; columns the gather handed back get their redo)
              fold(~ST_OVERFLOW_SLOT, true);
            }
            if (redo_rec || replay) {
              // columns whose lists outgrew the bucket: the gather again, those columns only,
              // with a bucket for their need (8192 entries at most: columns beyond it are
              // left for the window gather below)
              int b = 2 * H.bcap;
              while (b < hc.max_state && b < 8192) b <<= 1;
              if (replay) b = std::max(b, 2048);  // (the data may need more than the tape's)
              if (hc.redo_cols * 64LL > ncols && !replay) lb = std::min(2 * lb, ctx->bucket_max);  // next calls
              if (!replay) CK(cudaMemsetAsync(&ctr->status, 0, sizeof(int), st));
              CK(launch_lgather<T>(H, b, 1, st, sms));
              ++ctx->launches;
              if (redo_rec) RD(hc);
            }
          }
        }
        if (!done && slices) return DEXEL_ERR_CAPACITY;  // the level path's room (not reached)
        if (!done && nb > 1) {
          // the tiled gather takes the whole grid: plan again without blocks
          ctx->noblock = true;
          again = true;
          break;
        }
        if (!done) {
          rec.replayable = false;
          if (replay) return DEXEL_ERR_NO_PLAN;
          if (!packed) CK(pack_lines());  // the tiled gather stages line-contiguous sources
          CK(launch_pass2t<T>(pg, tw, tc, ntab, stage_cap, kRoundAppends, kRoundPieces, per_sm,
                              tblocks, st));
          ++ctx->launches;
        }
      }
      RD(hc);
      int redo = 0;
      if (slices && (hc.status & ST_OVERFLOW_SLOT) && !(hc.status & ST_OVERFLOW_ARENA))
        return DEXEL_ERR_CAPACITY;  // a column's own union beyond every bucket
      if ((hc.status & ST_OVERFLOW_SLOT) && !(hc.status & ST_OVERFLOW_ARENA)) {
        // columns whose union outgrew the bucket: k_pass2c with one bucket for the whole window
        redo = hc.redo_cols;
        int b = 4096;  // the whole window's appends in one bucket: as large as fits
        while (b > 4 * pg.bcap && pass2c_warp_bytes(K, b) > (200LL << 10)) b >>= 1;
        const long long wbytes = pass2c_warp_bytes(K, b);
        if (wbytes <= (200LL << 10)) {
          int w = 8;
          while (w > 1 && w * wbytes > (100LL << 10)) w >>= 1;
          const int per_sm = (int)std::max<long long>(1, std::min<long long>(64 / w, (220LL << 10) / (w * wbytes)));
          if (redo * 64LL > ncols && !replay) cc = std::min(2 * cc, 1024);  // next calls: a larger bucket
          P2GParams<T> pr = pg;
          pr.bcap = b;
          pr.redo = 1;
          if (replay)
            fold(~ST_OVERFLOW_SLOT, true);
          else
            CK(cudaMemsetAsync(&ctr->status, 0, sizeof(int), st));
          CK(launch_pass2c<T>(pr, w, sms * per_sm, st));
          ++ctx->launches;
          RD(hc);
        }
      }
      ctx->stats[5] = redo;
      mark(ctx, 5, st);
      ctx->needO = std::max<long long>(ctx->needO, (long long)hc.arena_top[3]);
      ctx->stats[6] = hc.status;
      ctx->stats[7] = attempt + 1;
      if (hc.status & ST_OVERFLOW_ARENA) {
        ctx->last_required = total + (size_t)hc.arena_top[3] * 16;
        if (ws_user) return DEXEL_ERR_CAPACITY;
        again = true;
        break;
      }
      if (hc.status & ST_OVERFLOW_SLOT) {
        // a column's union beyond any bucket: the per-line sweep does this call's pass 2
        CK(cudaMemsetAsync(&ctr->status, 0, sizeof(int), st));
        CK(cudaMemsetAsync(&ctr->arena_top[3], 0, sizeof(unsigned long long), st));
        CK(cudaMemsetAsync(&ctr->out_total, 0, sizeof(unsigned long long), st));
        CK(cudaMemsetAsync(&ctr->max_state, 0, sizeof(int), st));
        use_sweep = true;
      }
    }
    if (use_sweep) {
      rec.replayable = false;
      if (replay) return DEXEL_ERR_NO_PLAN;
    }
    if (use_sweep && nb > 1) {
      // the per-line sweep takes the whole grid: plan again without blocks
      ctx->noblock = true;
      again = true;
      break;
    }
    if (use_sweep) {
    const int capP = std::max(hc.max_pieces, 1) + 2;
    const int items2_target = nwarps * 2;
    int nch2 = std::max(1, std::min(ny, (items2_target + nx - 1) / nx));
    int chunk2 = (ny + nch2 - 1) / nch2;
    nch2 = (ny + chunk2 - 1) / chunk2;
    P2Params<T> p2{};
    p2.nx = nx; p2.ny = ny; p2.R = K; p2.kk = kk; p2.h2 = in->h * in->h;
    p2.h2f = (float)p2.h2;
    p2.chunk = chunk2; p2.nchunks = nch2;
    p2.wtab = (const double*)pwtab; p2.reach = (const int*)preach;
    p2.m_a = p1.m_a; p2.m_b = p1.m_b; p2.m_l = p1.m_l;
    p2.m_start = p1.m_start; p2.m_cnt = p1.m_cnt;
    const long long capF2 = (long long)(bF / 16);
    p2.f_l = (ukey*)aF; p2.f_r = (ukey*)aF + capF2; p2.f_cap = capF2;
    const long long capO = (long long)(bO / 16);
    p2.o_l = (ukey*)aO; p2.o_r = (ukey*)aO + capO; p2.o_cap = capO;
    p2.o_start = (long long*)postart; p2.o_cnt = (int*)pocnt;
    p2.blk = 256;
    p2.ctr = ctr;
    p2.capP = capP; p2.capR = ctx->capR; p2.capA = ctx->capA; p2.capS = ctx->capS;
    const long long sb2 = p2_slot_bytes<Key>(capP, p2.capR, p2.capA, p2.capS, chunk2);
    p2.slots = pslots; p2.slot_bytes = sb2;
    const int nw2 = (int)std::min<long long>(nwarps, (long long)(slot_room / sb2));
    if (nw2 < kWarpsPerBlock) {
      ctx->last_required = total + (size_t)sb2 * nwarps;
      if (ws_user) return DEXEL_ERR_CAPACITY;
      ensure_owned(ctx, ctx->last_required);
      again = true;
      break;
    }
    mark(ctx, 4, st);
    CK(launch_pass2<T>(p2, nw2 / kWarpsPerBlock, st));
    mark(ctx, 5, st);
    ++ctx->launches;
    RD(hc);
    ctx->needF = std::max<long long>(ctx->needF, (long long)hc.arena_top[2] * 16 / (long long)(2 * sizeof(Key) + 2) + 1);
    ctx->needO = std::max<long long>(ctx->needO, (long long)hc.arena_top[3]);
    ctx->stats[6] = hc.status;
    ctx->stats[7] = attempt + 1;
    if (hc.status & ST_OVERFLOW_SLOT) {
      // a per-warp state outgrew its arrays: grow them past the size that was needed
      const int need = std::max(hc.max_state, 1);
      ctx->capA = std::max(ctx->capA * 2, need + need / 2);
      ctx->capR = std::max(ctx->capR * 2, need + need / 2);
      ctx->capS = std::max(ctx->capS * 2, need + need / 2);
      ctx->last_required =
          total + (size_t)p2_slot_bytes<Key>(capP, ctx->capR, ctx->capA, ctx->capS, chunk2) * nwarps;
      if (ws_user) return DEXEL_ERR_CAPACITY;
      again = true;
      break;
    }
    if (hc.status & ST_OVERFLOW_ARENA) {
      ctx->last_required = total + (size_t)(hc.arena_top[2] + hc.arena_top[3]) * 16;
      if (ws_user) return DEXEL_ERR_CAPACITY;
      again = true;
      break;
    }
    }  // pass 2 variants

    if (!replay) acc_block_times(ctx);
    ctx->stats[9] = std::max<long long>(ctx->stats[9], nb);
    }  // blocks
    if (again && replay) return DEXEL_ERR_NO_PLAN;
    if (again) continue;

    // ---------------- compaction into the caller's CSR
    const int thr = 256;
    const unsigned gb = (unsigned)((ncols + thr - 1) / thr);
    mark(ctx, 6, st);
    const long long capOut = (long long)(bO / 16);
    const ukey* out_l = (const ukey*)aO;
    const ukey* out_r = (const ukey*)aO + capOut;
    k_count<T><<<gb, thr, 0, st>>>((int)ncols, (const long long*)postart, (const int*)pocnt,
                                   out_l, out_r, erode ? 1 : 0, (long long*)pcnt);
    const long long nsb = (ncols + kScanTile - 1) / kScanTile;
    k_scan1<long long><<<(unsigned)nsb, kScanThreads, 0, st>>>(ncols, (const long long*)pcnt, (long long*)ppos,
                                                  (long long*)psums);
    k_scan2<<<1, kScanThreads, 0, st>>>(nsb, (long long*)psums);
    k_scan3<<<(unsigned)((ncols + 1 + thr - 1) / thr), thr, 0, st>>>(
        ncols, (long long*)ppos, (const long long*)psums, out->col_off, ctr);
    ctx->launches += 4;
    CK(cudaGetLastError());
    mark(ctx, 7, st);
    if (replay) {
      // no host read: the result words, then the output written only if they say DEXEL_OK
      fold(~0, false);
      long long* res = ctx->replay_result;
      k_result<<<1, 1, 0, st>>>(ctr, (const long long*)psums + nsb, out->capacity_seg, res);
      k_write<T><<<gb, thr, 0, st>>>((int)ncols, (const long long*)postart, (const int*)pocnt,
                                     out_l, out_r, erode ? 1 : 0, (const long long*)ppos,
                                     (T*)out->z, res);
      ctx->launches += 3;
      CK(cudaGetLastError());
      mark(ctx, 9, st);
      out->nseg = -1;  // (in the result words)
      ctx->last_required = total;
      // (the tape's last entry is the synchronous call's read of the total)
      return rt->pos + 1 == rt->snaps.size() ? DEXEL_OK : DEXEL_ERR_NO_PLAN;
    }
    long long total_out = 0;
    CK(cudaMemcpyAsync(&total_out, (long long*)psums + nsb, sizeof(long long),
                       cudaMemcpyDeviceToHost, st));
    RD(hc);
    out->nseg = total_out;
    ctx->host_ctr = hc;
    if (hc.status & ST_TOO_MANY_OUT) return DEXEL_ERR_CAPACITY;
    if (total_out > out->capacity_seg) return DEXEL_ERR_CAPACITY;
    mark(ctx, 8, st);
    k_write<T><<<gb, thr, 0, st>>>((int)ncols, (const long long*)postart, (const int*)pocnt,
                                   out_l, out_r, erode ? 1 : 0, (const long long*)ppos,
                                   (T*)out->z);
    ++ctx->launches;
    CK(cudaGetLastError());
    mark(ctx, 9, st);
    CK(cudaStreamSynchronize(st));
    if (ctx->profiling) {
      for (int q = 0; q < 5; ++q) {
        if (q == 1 || q == 2) continue;  // added block by block
        float ms = 0;
        if (cudaEventElapsedTime(&ms, ctx->ev[2 * q], ctx->ev[2 * q + 1]) == cudaSuccess)
          ctx->stage_ms[q] += ms;
      }
      for (int q = 0; q < 4; ++q) {
        float ms = 0;
        if (ctx->kernel_rec[q] &&
            cudaEventElapsedTime(&ms, ctx->ev[10 + 2 * q], ctx->ev[11 + 2 * q]) == cudaSuccess)
          ctx->kernel_ms[q] += ms;
      }
    }
    for (int q = 0; q < 16; ++q) ctx->phase[q] += hc.phase[q];
    ctx->stats[0] += in->nseg;
    ctx->stats[1] += mid_sum;
    ctx->stats[2] += (long long)hc.out_total;
    ctx->stats[3] += total_out;
    ctx->stats[4] = std::max<long long>(ctx->stats[4], hc.max_pieces);
    ctx->stats[5] = std::max<long long>(ctx->stats[5], hc.max_state);
    ctx->last_required = total;
    rec.need = total;
    if (rec.replayable) ctx->tapes[tape_key(in, k, erode, slices, sizeof(T))] = std::move(rec);
    return DEXEL_OK;
  }
  return DEXEL_ERR_CAPACITY;
}
#undef RD

dexel_status check_in(const dexel_grid_in* in, double k) {
  if (!in || in->nx < 1 || in->ny < 1 || in->nx > 32768 || in->ny > 32768) return DEXEL_ERR_INVALID_ARG;
  if (!(in->h > 0) || !std::isfinite(in->h)) return DEXEL_ERR_INVALID_ARG;
  if (!(k >= 0) || !std::isfinite(k) || k > 4096) return DEXEL_ERR_INVALID_ARG;
  if (!in->col_off || in->nseg < 0 || (in->nseg > 0 && !in->z)) return DEXEL_ERR_INVALID_ARG;
  if ((long long)in->nx * in->ny > (1LL << 30)) return DEXEL_ERR_INVALID_ARG;
  return DEXEL_OK;
}

dexel_status offset(dexel_ctx* ctx, const dexel_grid_in* in, double k, bool erode, dexel_mode mode,
                    dexel_grid_out* out, void* ws, size_t ws_bytes, void* stream,
                    bool slices = false) {
  if (!ctx || !out || !out->col_off || (out->capacity_seg > 0 && !out->z) || out->capacity_seg < 0)
    return DEXEL_ERR_INVALID_ARG;
  dexel_status s = check_in(in, k);
  if (s != DEXEL_OK) return s;
  if (mode != DEXEL_FP64 && mode != DEXEL_FP32_PRED64) return DEXEL_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return DEXEL_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  if (mode == DEXEL_FP64) return Offset<double>::run(ctx, in, k, erode, out, ws, ws_bytes, st, slices);
  return Offset<float>::run(ctx, in, k, erode, out, ws, ws_bytes, st, slices);
}

// Boolean operation of two grids of the same size into the caller's CSR (csg.cu): both
// inputs validated, per-column counts, scan, then the segments.
template <typename T>
dexel_status boolean_run(dexel_ctx* ctx, int op, const dexel_grid_in* a, const dexel_grid_in* b,
                         dexel_grid_out* out, void* ws_user, size_t ws_bytes, cudaStream_t st) {
  const long long ncols = (long long)a->nx * a->ny;
  auto plan = [&](Carver& C, void** pctr, void** pcnt, void** ppos, void** psums) {
    *pctr = C.take(sizeof(Counters));
    *pcnt = C.take(sizeof(long long) * (ncols + 1));
    *ppos = C.take(sizeof(long long) * (ncols + 1));
    *psums = C.take(sizeof(long long) * ((ncols + kScanTile) / kScanTile + 2));
  };
  Carver probe{nullptr, (size_t)-1};
  void *pctr, *pcnt, *ppos, *psums;
  plan(probe, &pctr, &pcnt, &ppos, &psums);
  const size_t need = align_up(probe.used, 256) + 256;
  void* base = ws_user;
  size_t bytes = ws_bytes;
  if (ws_user) {
    if (ws_bytes < need) {
      ctx->last_required = need;
      return DEXEL_ERR_CAPACITY;
    }
  } else {
    dexel_status s = ensure_owned(ctx, need);
    if (s != DEXEL_OK) return s;
    base = ctx->own;
    bytes = ctx->own_bytes;
  }
  Carver C{(char*)base, bytes};
  plan(C, &pctr, &pcnt, &ppos, &psums);
  if (!C.ok) return DEXEL_ERR_CAPACITY;
  ctx->last_required = need;
  Counters* ctr = (Counters*)pctr;
  CK(cudaMemsetAsync(ctr, 0, sizeof(Counters), st));
  const unsigned g = (unsigned)((ncols + 255) / 256);
  k_validate<T><<<g, 256, 0, st>>>((int)ncols, a->col_off, (const T*)a->z, a->nseg, ctr);
  k_validate<T><<<g, 256, 0, st>>>((int)ncols, b->col_off, (const T*)b->z, b->nseg, ctr);
  CK(launch_bool_count<T>(op, ncols, a->col_off, (const T*)a->z, b->col_off, (const T*)b->z,
                          (long long*)pcnt, st));
  const long long nsb = (ncols + kScanTile - 1) / kScanTile;
  k_scan1<long long><<<(unsigned)nsb, kScanThreads, 0, st>>>(ncols, (const long long*)pcnt,
                                                            (long long*)ppos, (long long*)psums);
  k_scan2<<<1, kScanThreads, 0, st>>>(nsb, (long long*)psums);
  k_scan3<<<(unsigned)((ncols + 1 + 255) / 256), 256, 0, st>>>(ncols, (long long*)ppos,
                                                              (const long long*)psums, out->col_off, ctr);
  ctx->launches += 6;
  CK(cudaGetLastError());
  long long total = 0;
  Counters hc;
  CK(cudaMemcpyAsync(&total, (long long*)psums + nsb, sizeof(long long), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&hc, ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (hc.status & ST_BAD_CSR) return DEXEL_ERR_BAD_CSR;
  out->nseg = total;
  if ((hc.status & ST_TOO_MANY_OUT) || total > out->capacity_seg) return DEXEL_ERR_CAPACITY;
  CK(launch_bool_write<T>(op, ncols, a->col_off, (const T*)a->z, b->col_off, (const T*)b->z,
                          (const long long*)ppos, (T*)out->z, st));
  ++ctx->launches;
  CK(cudaStreamSynchronize(st));
  ctx->stats[0] += a->nseg + b->nseg;
  ctx->stats[3] += total;
  return DEXEL_OK;
}

dexel_status boolean_run_any(dexel_ctx* ctx, int op, const dexel_grid_in* a, const dexel_grid_in* b,
                             dexel_mode mode, dexel_grid_out* out, void* ws, size_t ws_bytes,
                             cudaStream_t st) {
  if (mode == DEXEL_FP64) return boolean_run<double>(ctx, op, a, b, out, ws, ws_bytes, st);
  return boolean_run<float>(ctx, op, a, b, out, ws, ws_bytes, st);
}

// A device buffer of the context, grown to `need` bytes.
dexel_status grow_buffer(void** p, size_t* bytes, size_t need) {
  if (*bytes >= need) return DEXEL_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *bytes = 0;
  if (cudaMalloc(p, need) != cudaSuccess) {
    cudaGetLastError();
    return DEXEL_ERR_NOMEM;
  }
  *bytes = need;
  return DEXEL_OK;
}

}  // namespace


// ------------------------------------------------------------------------------------------
// Allocation-free offset for small grids
//
// Some callers cannot allocate device memory at the moment they need an offset: a host
// application that owns every byte of the GPU through its own pool, a real-time loop that
// must not pay cudaMalloc's implicit synchronisation, or code running where allocation is
// forbidden.  dexel_offset_noalloc serves them: it runs the per-line sweep kernels of
// dexel_dilate / dexel_erode with all of their scratch (counters, tables, indices, arenas,
// per-warp sweep state) carved from one file-scope static device array.  Every GPU that loads
// the library holds that array until the process exits.  All calls on a device share it, so
// calls that overlap on the GPU (different streams or threads) race; the counters that must
// start at zero are cleared at the start of every call.
// ------------------------------------------------------------------------------------------
constexpr size_t kNoAllocBytes = (size_t)128 << 20;  // 128 MiB per device
constexpr long long kNoAllocMaxColumns = 256 * 256;
constexpr double kNoAllocMaxK = 32.0;
constexpr int kNoAllocWarps = 8;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {

// Device address of the static scratch in the current device's context.  In host code the
// array's name is only a host-side stand-in, so the address is asked of the runtime; it is
// asked on every call (a host-side table lookup), never cached, because a context torn down
// and created again (cudaDeviceReset) may load the module at another address.
dexel_status noalloc_scratch(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    return cuda_status(e == cudaSuccess ? cudaErrorInvalidSymbol : e, __LINE__);
  }
  *out = p;
  return DEXEL_OK;
}

template <typename T>
dexel_status noalloc_offset(const dexel_grid_in* in, double k, bool erode, dexel_grid_out* out,
                            cudaStream_t st) {
  typedef typename H<T>::K Key;
  void* base = nullptr;
  dexel_status s = noalloc_scratch(&base);
  if (s != DEXEL_OK) return s;
  // nseg = -1 until the output count is known: a DEXEL_ERR_CAPACITY returned before that
  // means the static scratch is too small, not the caller's output buffer
  out->nseg = -1;
  const int nx = in->nx, ny = in->ny;
  const long long ncols = (long long)nx * ny;
  const double kk = k * k;
  const int K = reach_of(kk);
  const int nmax = (int)std::floor(kk);
  Carver C{(char*)base, kNoAllocBytes};
  Counters* ctr = (Counters*)C.take(sizeof(Counters));
  double* wtab = (double*)C.take(sizeof(double) * (nmax + 2));
  int* reach = (int*)C.take(sizeof(int) * (K + 2));
  long long* mstart = (long long*)C.take(sizeof(long long) * ncols);
  int* mcnt = (int*)C.take(sizeof(int) * ncols);
  long long* ostart = (long long*)C.take(sizeof(long long) * ncols);
  int* ocnt = (int*)C.take(sizeof(int) * ncols);
  long long* cnt = (long long*)C.take(sizeof(long long) * (ncols + 1));
  long long* pos = (long long*)C.take(sizeof(long long) * (ncols + 1));
  long long* sums = (long long*)C.take(sizeof(long long) * ((ncols + kScanTile) / kScanTile + 2));
  if (!C.ok) return DEXEL_ERR_CAPACITY;
  CK(cudaMemsetAsync(ctr, 0, sizeof(Counters), st));
  const int thr = 256;
  k_validate<T><<<(unsigned)((ncols + thr - 1) / thr), thr, 0, st>>>((int)ncols, in->col_off,
                                                                    (const T*)in->z, in->nseg, ctr);
  k_tables<<<(std::max(nmax, K) + 1 + 255) / 256, 256, 0, st>>>(kk, in->h, nmax, K, wtab, reach,
                                                                nullptr);
  CK(cudaGetLastError());
  Counters hc;
  CK(cudaMemcpyAsync(&hc, ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (hc.status & ST_BAD_CSR) return DEXEL_ERR_BAD_CSR;

  // per-warp state for pass 1, then pass 2 (the same region), then the arenas
  const int capS = hc.max_segs_in + 2;
  const int capF = 2 * (K + 1) * capS + 8;
  const int chunk1 = nx, chunk2 = ny;  // one work item per line
  const size_t slot_region = (size_t)12 << 20;
  const long long sb1 = p1_slot_bytes<Key>(capF, capS, chunk1);
  if ((long long)slot_region < sb1 * kWarpsPerBlock) return DEXEL_ERR_CAPACITY;
  char* slots = (char*)C.take(slot_region);
  const size_t rest = C.cap > C.used + 4096 ? C.cap - align_up(C.used, 256) - 4096 : 0;
  // forward sweep states, S_mid, pass-2 intervals (measured on sphere unions at 256 x 256,
  // k = 32: about 25 MB of S_mid, as much of forward states, 3 MB of intervals)
  const size_t bF = align_up(rest / 100 * 38, 256), bM = align_up(rest / 100 * 46, 256);
  const size_t bO = align_up(rest / 100 * 14, 256);
  char* aF = (char*)C.take(bF);
  char* aM = (char*)C.take(bM);
  char* aO = (char*)C.take(bO);
  if (!C.ok || !slots || !aF || !aM || !aO) return DEXEL_ERR_CAPACITY;

  P1Params<T> p1{};
  p1.nx = nx; p1.ny = ny; p1.K = K; p1.erode = erode ? 1 : 0;
  p1.chunk = chunk1; p1.nchunks = 1;
  p1.col_off = in->col_off; p1.z = (const T*)in->z;
  const long long capF1 = (long long)(bF / (2 * sizeof(Key) + 2));
  p1.f_a = (Key*)aF; p1.f_b = (Key*)aF + capF1; p1.f_l = (short*)((Key*)aF + 2 * capF1);
  p1.f_cap = capF1;
  const long long capM = (long long)(bM / (2 * sizeof(Key) + 2));
  p1.m_a = (Key*)aM; p1.m_b = (Key*)aM + capM; p1.m_l = (short*)((Key*)aM + 2 * capM);
  p1.m_cap = capM;
  p1.m_start = mstart; p1.m_cnt = mcnt;
  p1.blk = 64;
  p1.ctr = ctr;
  p1.slots = slots; p1.slot_bytes = sb1;
  p1.capF = capF; p1.capS = capS;
  const int nw1 = (int)std::min<long long>(kNoAllocWarps, (long long)(slot_region / sb1));
  CK(launch_pass1<T>(p1, nw1 / kWarpsPerBlock, st));
  CK(cudaMemcpyAsync(&hc, ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (hc.status & (ST_OVERFLOW_SLOT | ST_OVERFLOW_ARENA)) return DEXEL_ERR_CAPACITY;

  P2Params<T> p2{};
  p2.nx = nx; p2.ny = ny; p2.R = K; p2.kk = kk; p2.h2 = in->h * in->h;
  p2.h2f = (float)p2.h2;
  p2.chunk = chunk2; p2.nchunks = 1;
  p2.wtab = wtab; p2.reach = reach;
  p2.m_a = p1.m_a; p2.m_b = p1.m_b; p2.m_l = p1.m_l;
  p2.m_start = mstart; p2.m_cnt = mcnt;
  const long long capF2 = (long long)(bF / 16);
  p2.f_l = (ukey*)aF; p2.f_r = (ukey*)aF + capF2; p2.f_cap = capF2;
  const long long capO = (long long)(bO / 16);
  p2.o_l = (ukey*)aO; p2.o_r = (ukey*)aO + capO; p2.o_cap = capO;
  p2.o_start = ostart; p2.o_cnt = ocnt;
  p2.blk = 64;
  p2.ctr = ctr;
  p2.capP = std::max(hc.max_pieces, 1) + 2;
  p2.capR = 1024; p2.capA = 1024; p2.capS = 4096;
  const long long sb2 = p2_slot_bytes<Key>(p2.capP, p2.capR, p2.capA, p2.capS, chunk2);
  if ((long long)slot_region < sb2 * kWarpsPerBlock) return DEXEL_ERR_CAPACITY;
  p2.slots = slots; p2.slot_bytes = sb2;
  const int nw2 = (int)std::min<long long>(kNoAllocWarps, (long long)(slot_region / sb2));
  CK(launch_pass2<T>(p2, nw2 / kWarpsPerBlock, st));
  CK(cudaMemcpyAsync(&hc, ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (hc.status & (ST_OVERFLOW_SLOT | ST_OVERFLOW_ARENA)) return DEXEL_ERR_CAPACITY;

  const unsigned gb = (unsigned)((ncols + thr - 1) / thr);
  k_count<T><<<gb, thr, 0, st>>>((int)ncols, ostart, ocnt, p2.o_l, p2.o_r, erode ? 1 : 0, cnt);
  const long long nb = (ncols + kScanTile - 1) / kScanTile;
  k_scan1<long long><<<(unsigned)nb, kScanThreads, 0, st>>>(ncols, cnt, pos, sums);
  k_scan2<<<1, kScanThreads, 0, st>>>(nb, sums);
  k_scan3<<<(unsigned)((ncols + 1 + thr - 1) / thr), thr, 0, st>>>(ncols, pos, sums, out->col_off, ctr);
  CK(cudaGetLastError());
  long long total_out = 0;
  CK(cudaMemcpyAsync(&total_out, sums + nb, sizeof(long long), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&hc, ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  out->nseg = total_out;
  if ((hc.status & ST_TOO_MANY_OUT) || total_out > out->capacity_seg) return DEXEL_ERR_CAPACITY;
  k_write<T><<<gb, thr, 0, st>>>((int)ncols, ostart, ocnt, p2.o_l, p2.o_r, erode ? 1 : 0, pos,
                                 (T*)out->z);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  return DEXEL_OK;
}

}  // namespace

extern "C" {

dexel_status dexel_ctx_create(dexel_ctx** ctx, int device) {
  if (!ctx) return DEXEL_ERR_INVALID_ARG;
  *ctx = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return DEXEL_ERR_CUDA;
  }
  dexel_ctx* c = new (std::nothrow) dexel_ctx();
  if (!c) return DEXEL_ERR_NOMEM;
  c->device = device;
  cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
  const char* mode = getenv("DEXEL_PASS2");
  c->sweep2 = mode && strcmp(mode, "sweep") == 0;
  if (mode && strcmp(mode, "tiled") == 0) c->levels = false;
  const char* mode1 = getenv("DEXEL_PASS1");
  c->sweep1 = mode1 && strcmp(mode1, "sweep") == 0;
  if (mode1 && strcmp(mode1, "gather") == 0) c->lane1 = false;
  if (mode1 && (strcmp(mode1, "gather") == 0 || strcmp(mode1, "lane") == 0)) c->merge1 = false;
  if (const char* e = getenv("DEXEL_PASS1_ECAP")) {
    const int v = atoi(e);
    if (v >= 256 && v <= 16384 && (v & (v - 1)) == 0) c->p1l_ecap = v;
  }
  if (const char* e = getenv("DEXEL_PASS1_RING")) c->p1l_ring = atoi(e) != 0;
  if (const char* e = getenv("DEXEL_PASS1_ECAP_RULE")) c->p1l_ecap_max = strcmp(e, "max") == 0;
  if (const char* e = getenv("DEXEL_PASS1_PRUNE")) c->prune1 = atoi(e) != 0;
  {
    size_t fr = 0, tot = 0;
    if (cudaSetDevice(device) == cudaSuccess && cudaMemGetInfo(&fr, &tot) == cudaSuccess)
      c->block_bytes = std::max(1e9, 0.45 * (double)fr);
    cudaGetLastError();
  }
  if (const char* e = getenv("DEXEL_BLOCK_MB")) {
    const double v = atof(e);
    if (v >= 1) c->block_bytes = v * 1e6;
  }
  if (const char* e = getenv("DEXEL_PASS1_RING_CAP")) {
    const int v = atoi(e);
    if (v >= 16 && v <= 1024) {
      c->p1l_ring_cap = v & ~7;
      c->p1l_ring_max = std::max(c->p1l_ring_max, c->p1l_ring_cap);
    }
  }
  if (const char* e = getenv("DEXEL_BATCH_MAX_COLS")) c->batch_max_cols = atoll(e);
  if (const char* e = getenv("DEXEL_LEVELS_EXACT")) c->levels_exact = atoi(e) != 0;
  if (const char* e = getenv("DEXEL_LANE_GATHER_MAX")) c->lane_gather_max = atoi(e);
  if (const char* e = getenv("DEXEL_GATHER_BUCKET_MAX")) {
    const int v = atoi(e);
    if (v >= 256 && v <= 8192 && (v & (v - 1)) == 0) c->bucket_max = v;
  }
  if (const char* e = getenv("DEXEL_PASS1_ECAP_MUL")) {
    const double v = atof(e);
    if (v >= 0.5 && v <= 64.0) c->p1l_ecap_mul = v;
  }
  if (const char* e = getenv("DEXEL_PASS1_TILE_REDO")) c->p1l_tile_redo = atoi(e) != 0;
  if (const char* e = getenv("DEXEL_PASS1_BLOCK_CAP")) {
    const int v = atoi(e);
    if (v >= 1 && v <= 3) c->p1l_block_cap = v;
  }
  if (const char* e = getenv("DEXEL_LEVEL_SPILL")) {
    const int v = atoi(e);
    if (v >= 0 && v <= 256) c->lvl_spill_cap = v;
  }
  if (const char* e = getenv("DEXEL_LEVEL_SLOTS")) {
    const int v = atoi(e);
    if (v >= 2 && v <= 16) c->lvl_slots = v;
  }
  if (const char* e = getenv("DEXEL_PASS1_NBUF")) {
    const int v = atoi(e);
    if (v == 1 || v == 2) c->p1l_nbuf = v;
  }
  if (const char* e = getenv("DEXEL_PASS1_GW")) {
    const int v = atoi(e);
    if (v == 1 || v == 2 || v == 4 || v == 8) c->p1l_gw = v;
  }
  *ctx = c;
  return DEXEL_OK;
}

void dexel_ctx_destroy(dexel_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->own) cudaFree(ctx->own);
  if (ctx->mid) cudaFree(ctx->mid);
  if (ctx->aux) cudaFree(ctx->aux);
  if (ctx->res_buf) cudaFree(ctx->res_buf);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  batch_engine_destroy(ctx->batch);
  for (cudaEvent_t e : ctx->ev)
    if (e) cudaEventDestroy(e);
  delete ctx;
}

size_t dexel_workspace_size(const dexel_grid_in* in, double k, dexel_mode mode) {
  if (check_in(in, k) != DEXEL_OK) return 0;
  const long long ncols = (long long)in->nx * in->ny;
  const int K = reach_of(k * k);
  const size_t es = mode == DEXEL_FP64 ? 8 : 4;
  const long long segs = std::max<long long>(in->nseg + ncols, 1024);
  const size_t fixed = (size_t)ncols * 48 + ((size_t)1 << 20);
  const size_t arenas = (size_t)segs * std::min(K + 2, 16) * (2 * (2 * es + 2) + 16) + segs * 32;
  return fixed + arenas + ((size_t)2 << 30);
}

size_t dexel_last_required(const dexel_ctx* ctx) { return ctx ? ctx->last_required : 0; }

int64_t dexel_last_launches(const dexel_ctx* ctx) { return ctx ? ctx->launches : 0; }

void dexel_set_profiling(dexel_ctx* ctx, int on) {
  if (ctx) ctx->profiling = on != 0;
}

int dexel_last_stage_ms(const dexel_ctx* ctx, double* ms, int max) {
  if (!ctx || !ms) return 0;
  int n = max < 5 ? max : 5;
  for (int q = 0; q < n; ++q) ms[q] = ctx->stage_ms[q];
  return n;
}

int dexel_last_kernel_ms(const dexel_ctx* ctx, double* ms, int max) {
  if (!ctx || !ms) return 0;
  int n = max < 4 ? max : 4;
  for (int q = 0; q < n; ++q) ms[q] = ctx->kernel_ms[q];
  return n;
}

int dexel_last_levels_status(const dexel_ctx* ctx) { return ctx ? ctx->levels_status : 0; }

int dexel_last_phases(const dexel_ctx* ctx, uint64_t* ph, int max) {
  if (!ctx || !ph) return 0;
  int n = max < 16 ? max : 16;
  for (int q = 0; q < n; ++q) ph[q] = ctx->phase[q];
  return n;
}

int dexel_last_stats(const dexel_ctx* ctx, int64_t* stats, int max) {
  if (!ctx || !stats) return 0;
  int n = max < 15 ? max : 15;
  for (int q = 0; q < n; ++q) stats[q] = ctx->stats[q];
  return n;
}

dexel_status dexel_validate(dexel_ctx* ctx, const dexel_grid_in* in, dexel_mode mode, void* ws,
                            size_t ws_bytes, void* stream) {
  if (!ctx) return DEXEL_ERR_INVALID_ARG;
  dexel_status s = check_in(in, 0.0);
  if (s != DEXEL_OK) return s;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return DEXEL_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  Counters* ctr = nullptr;
  if (ws) {
    if (ws_bytes < sizeof(Counters)) return DEXEL_ERR_CAPACITY;
    ctr = (Counters*)ws;
  } else {
    s = ensure_owned(ctx, 1 << 20);
    if (s != DEXEL_OK) return s;
    ctr = (Counters*)ctx->own;
  }
  const long long ncols = (long long)in->nx * in->ny;
  CK(cudaMemsetAsync(ctr, 0, sizeof(Counters), st));
  if (mode == DEXEL_FP64)
    k_validate<double><<<(unsigned)((ncols + 255) / 256), 256, 0, st>>>((int)ncols, in->col_off,
                                                                       (const double*)in->z, in->nseg, ctr);
  else
    k_validate<float><<<(unsigned)((ncols + 255) / 256), 256, 0, st>>>((int)ncols, in->col_off,
                                                                      (const float*)in->z, in->nseg, ctr);
  CK(cudaGetLastError());
  Counters hc;
  CK(cudaMemcpyAsync(&hc, ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return (hc.status & ST_BAD_CSR) ? DEXEL_ERR_BAD_CSR : DEXEL_OK;
}

dexel_status dexel_dilate(dexel_ctx* ctx, const dexel_grid_in* in, double k, dexel_mode mode,
                          dexel_grid_out* out, void* ws, size_t ws_bytes, void* stream) {
  if (ctx) reset_call(ctx);
  return offset(ctx, in, k, false, mode, out, ws, ws_bytes, stream);
}

dexel_status dexel_erode(dexel_ctx* ctx, const dexel_grid_in* in, double k, dexel_mode mode,
                         dexel_grid_out* out, void* ws, size_t ws_bytes, void* stream) {
  if (ctx) reset_call(ctx);
  return offset(ctx, in, k, true, mode, out, ws, ws_bytes, stream);
}

dexel_status dexel_offset_enqueue(dexel_ctx* ctx, const dexel_grid_in* in, double k, dexel_op op,
                                  dexel_mode mode, dexel_grid_out* out, void* ws,
                                  size_t ws_bytes, void* stream, int64_t* d_result) {
  if (!ctx || !d_result || !ws || (op != DEXEL_DILATE && op != DEXEL_ERODE))
    return DEXEL_ERR_INVALID_ARG;
  dexel_status s = check_in(in, k);
  if (s != DEXEL_OK) return s;
  if (mode != DEXEL_FP64 && mode != DEXEL_FP32_PRED64) return DEXEL_ERR_INVALID_ARG;
  const bool erode = op == DEXEL_ERODE;
  auto it = ctx->tapes.find(tape_key(in, k, erode, false, mode == DEXEL_FP64 ? sizeof(double) : sizeof(float)));
  if (it == ctx->tapes.end()) return DEXEL_ERR_NO_PLAN;
  reset_call(ctx);
  it->second.pos = 0;
  ctx->replay = &it->second;
  ctx->replay_result = (long long*)d_result;
  s = offset(ctx, in, k, erode, mode, out, ws, ws_bytes, stream);
  ctx->replay = nullptr;
  ctx->replay_result = nullptr;
  return s;
}

dexel_status dexel_morph(dexel_ctx* ctx, const dexel_grid_in* in, double k, dexel_op op,
                         dexel_mode mode, dexel_grid_out* out, void* ws, size_t ws_bytes,
                         void* stream) {
  if (!ctx || (op != DEXEL_CLOSE && op != DEXEL_OPEN)) return DEXEL_ERR_INVALID_ARG;
  reset_call(ctx);
  dexel_status s = check_in(in, k);
  if (s != DEXEL_OK) return s;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return DEXEL_ERR_CUDA;
  const long long ncols = (long long)in->nx * in->ny;
  const size_t es = mode == DEXEL_FP64 ? 8 : 4;
  // intermediate grid: offsets + endpoints, grown until the first stage fits
  long long cap = std::max<long long>(2 * in->nseg + ncols / 4, 1024);
  for (int attempt = 0; attempt < 4; ++attempt) {
    const size_t need = align_up((size_t)(ncols + 1) * 4, 256) + (size_t)cap * 2 * es;
    if (ctx->mid_bytes < need) {
      if (ctx->mid) cudaFree(ctx->mid);
      ctx->mid = nullptr;
      ctx->mid_bytes = 0;
      if (cudaMalloc(&ctx->mid, need) != cudaSuccess) { cudaGetLastError(); return DEXEL_ERR_NOMEM; }
      ctx->mid_bytes = need;
    }
    dexel_grid_out mid{(int32_t*)ctx->mid, (char*)ctx->mid + align_up((size_t)(ncols + 1) * 4, 256),
                       cap, 0};
    const bool first_erode = op == DEXEL_OPEN;
    s = offset(ctx, in, k, first_erode, mode, &mid, ws, ws_bytes, stream);
    if (s == DEXEL_ERR_CAPACITY && mid.nseg > cap) {
      cap = mid.nseg + 1024;
      reset_call(ctx);
      continue;
    }
    if (s != DEXEL_OK) return s;
    dexel_grid_in in2{in->nx, in->ny, in->h, mid.col_off, mid.z, mid.nseg};
    return offset(ctx, &in2, k, !first_erode, mode, out, ws, ws_bytes, stream);
  }
  return DEXEL_ERR_CAPACITY;
}

dexel_status dexel_offset_slices(dexel_ctx* ctx, const dexel_grid_in* in, double k, dexel_op op,
                                 dexel_mode mode, dexel_grid_out* out, void* ws, size_t ws_bytes,
                                 void* stream) {
  if (op != DEXEL_DILATE && op != DEXEL_ERODE) return DEXEL_ERR_INVALID_ARG;
  if (ctx) reset_call(ctx);
  return offset(ctx, in, k, op == DEXEL_ERODE, mode, out, ws, ws_bytes, stream, true);
}

dexel_status dexel_raycast(dexel_ctx* ctx, const dexel_prim* prims, int32_t nprim, int32_t nx,
                           int32_t ny, double h, dexel_mode mode, dexel_grid_out* out, void* ws,
                           size_t ws_bytes, void* stream) {
  return dexel_raycast_axis(ctx, prims, nprim, 2, nx, ny, h, mode, out, ws, ws_bytes, stream);
}

dexel_status dexel_raycast_axis(dexel_ctx* ctx, const dexel_prim* prims, int32_t nprim,
                                int32_t axis, int32_t nx, int32_t ny, double h, dexel_mode mode,
                                dexel_grid_out* out, void* ws, size_t ws_bytes, void* stream) {
  if (axis < 0 || axis > 2) return DEXEL_ERR_INVALID_ARG;
  if (!ctx || !out || !out->col_off || (out->capacity_seg > 0 && !out->z) || out->capacity_seg < 0)
    return DEXEL_ERR_INVALID_ARG;
  if (nx < 1 || ny < 1 || nx > 32768 || ny > 32768 || (long long)nx * ny > (1LL << 30))
    return DEXEL_ERR_INVALID_ARG;
  if (!(h > 0) || !std::isfinite(h) || nprim < 0 || (nprim > 0 && !prims)) return DEXEL_ERR_INVALID_ARG;
  if (mode != DEXEL_FP64 && mode != DEXEL_FP32_PRED64) return DEXEL_ERR_INVALID_ARG;
  reset_call(ctx);
  if (cudaSetDevice(ctx->device) != cudaSuccess) return DEXEL_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  const long long ncols = (long long)nx * ny;
  auto plan = [&](Carver& C, void** pctr, void** pcnt, void** ppos, void** psums) {
    *pctr = C.take(sizeof(Counters));
    *pcnt = C.take(sizeof(long long) * (ncols + 1));
    *ppos = C.take(sizeof(long long) * (ncols + 1));
    *psums = C.take(sizeof(long long) * ((ncols + kScanTile) / kScanTile + 2));
  };
  Carver probe{nullptr, (size_t)-1};
  void *pctr, *pcnt, *ppos, *psums;
  plan(probe, &pctr, &pcnt, &ppos, &psums);
  const size_t need = align_up(probe.used, 256) + 256;
  void* base = ws;
  size_t bytes = ws_bytes;
  ctx->last_required = need;
  if (ws) {
    if (ws_bytes < need) return DEXEL_ERR_CAPACITY;
  } else {
    dexel_status s = ensure_owned(ctx, need);
    if (s != DEXEL_OK) return s;
    base = ctx->own;
    bytes = ctx->own_bytes;
  }
  Carver C{(char*)base, bytes};
  plan(C, &pctr, &pcnt, &ppos, &psums);
  if (!C.ok) return DEXEL_ERR_CAPACITY;
  Counters* ctr = (Counters*)pctr;
  CK(cudaMemsetAsync(ctr, 0, sizeof(Counters), st));
  const bool f64 = mode == DEXEL_FP64;
  CK(f64 ? launch_raycast<double>(prims, nprim, axis, nx, ncols, h, (long long*)pcnt, nullptr,
                                  nullptr, ctr, false, st)
         : launch_raycast<float>(prims, nprim, axis, nx, ncols, h, (long long*)pcnt, nullptr,
                                 nullptr, ctr, false, st));
  const long long nsb = (ncols + kScanTile - 1) / kScanTile;
  k_scan1<long long><<<(unsigned)nsb, kScanThreads, 0, st>>>(ncols, (const long long*)pcnt,
                                                            (long long*)ppos, (long long*)psums);
  k_scan2<<<1, kScanThreads, 0, st>>>(nsb, (long long*)psums);
  k_scan3<<<(unsigned)((ncols + 1 + 255) / 256), 256, 0, st>>>(ncols, (long long*)ppos,
                                                              (const long long*)psums, out->col_off, ctr);
  ctx->launches += 4;
  CK(cudaGetLastError());
  long long total = 0;
  Counters hc;
  CK(cudaMemcpyAsync(&total, (long long*)psums + nsb, sizeof(long long), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&hc, ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (hc.status & ST_OVERFLOW_SLOT) {
    out->nseg = -1;  // a column beyond the chords a thread holds
    return DEXEL_ERR_CAPACITY;
  }
  out->nseg = total;
  if ((hc.status & ST_TOO_MANY_OUT) || total > out->capacity_seg) return DEXEL_ERR_CAPACITY;
  CK(f64 ? launch_raycast<double>(prims, nprim, axis, nx, ncols, h, nullptr, (const long long*)ppos,
                                  (double*)out->z, ctr, true, st)
         : launch_raycast<float>(prims, nprim, axis, nx, ncols, h, nullptr, (const long long*)ppos,
                                 (float*)out->z, ctr, true, st));
  ++ctx->launches;
  CK(cudaStreamSynchronize(st));
  ctx->stats[3] = total;
  return DEXEL_OK;
}

dexel_status dexel_offset_ldi(dexel_ctx* ctx, const dexel_grid_in* views, double k, dexel_op op,
                              dexel_mode mode, dexel_grid_out* outs, void* ws, size_t ws_bytes,
                              void* stream) {
  if (!ctx || !views || !outs) return DEXEL_ERR_INVALID_ARG;
  if (op < DEXEL_DILATE || op > DEXEL_OPEN) return DEXEL_ERR_INVALID_ARG;
  for (int v = 0; v < 3; ++v) {
    if (check_in(&views[v], k) != DEXEL_OK) return DEXEL_ERR_INVALID_ARG;
    if (!(views[v].h == views[0].h)) return DEXEL_ERR_INVALID_ARG;  // one spacing for the solid
  }
  long long launches = 0;
  long long st[11] = {};
  dexel_status first = DEXEL_OK;
  for (int v = 0; v < 3; ++v) {
    dexel_status s;
    if (op == DEXEL_DILATE || op == DEXEL_ERODE) {
      reset_call(ctx);
      s = offset(ctx, &views[v], k, op == DEXEL_ERODE, mode, &outs[v], ws, ws_bytes, stream);
    } else {
      s = dexel_morph(ctx, &views[v], k, op, mode, &outs[v], ws, ws_bytes, stream);
    }
    launches += ctx->launches;
    for (int q = 0; q < 11; ++q) st[q] += ctx->stats[q];
    if (s != DEXEL_OK && first == DEXEL_OK) first = s;
  }
  ctx->launches = launches;
  for (int q = 0; q < 11; ++q) ctx->stats[q] = st[q];
  return first;
}

dexel_status dexel_boolean(dexel_ctx* ctx, dexel_bool_op op, const dexel_grid_in* a,
                           const dexel_grid_in* b, dexel_mode mode, dexel_grid_out* out, void* ws,
                           size_t ws_bytes, void* stream) {
  if (!ctx || !out || !out->col_off || (out->capacity_seg > 0 && !out->z) || out->capacity_seg < 0)
    return DEXEL_ERR_INVALID_ARG;
  if (op != DEXEL_UNION && op != DEXEL_INTERSECT && op != DEXEL_DIFFERENCE) return DEXEL_ERR_INVALID_ARG;
  if (mode != DEXEL_FP64 && mode != DEXEL_FP32_PRED64) return DEXEL_ERR_INVALID_ARG;
  reset_call(ctx);
  if (check_in(a, 0.0) != DEXEL_OK || check_in(b, 0.0) != DEXEL_OK) return DEXEL_ERR_INVALID_ARG;
  if (a->nx != b->nx || a->ny != b->ny) return DEXEL_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return DEXEL_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  if (mode == DEXEL_FP64) return boolean_run<double>(ctx, (int)op, a, b, out, ws, ws_bytes, st);
  return boolean_run<float>(ctx, (int)op, a, b, out, ws, ws_bytes, st);
}

dexel_status dexel_shell(dexel_ctx* ctx, const dexel_grid_in* in, double k, dexel_mode mode,
                         dexel_grid_out* out, void* ws, size_t ws_bytes, void* stream) {
  if (!ctx || !out || !out->col_off || (out->capacity_seg > 0 && !out->z) || out->capacity_seg < 0)
    return DEXEL_ERR_INVALID_ARG;
  if (mode != DEXEL_FP64 && mode != DEXEL_FP32_PRED64) return DEXEL_ERR_INVALID_ARG;
  reset_call(ctx);
  dexel_status s = check_in(in, k);
  if (s != DEXEL_OK) return s;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return DEXEL_ERR_CUDA;
  const long long ncols = (long long)in->nx * in->ny;
  const size_t es = mode == DEXEL_FP64 ? 8 : 4;
  const size_t offb = align_up((size_t)(ncols + 1) * 4, 256);
  // the dilation and the erosion in two context buffers, each grown until its grid fits
  dexel_grid_out g[2];
  void** buf[2] = {&ctx->mid, &ctx->aux};
  size_t* len[2] = {&ctx->mid_bytes, &ctx->aux_bytes};
  for (int q = 0; q < 2; ++q) {
    long long cap = std::max<long long>(2 * in->nseg + ncols / 4, 1024);
    if (*len[q] > offb) cap = std::max<long long>(cap, (long long)((*len[q] - offb) / (2 * es)));
    for (int attempt = 0;; ++attempt) {
      s = grow_buffer(buf[q], len[q], offb + (size_t)cap * 2 * es);
      if (s != DEXEL_OK) return s;
      g[q] = dexel_grid_out{(int32_t*)*buf[q], (char*)*buf[q] + offb, cap, 0};
      s = offset(ctx, in, k, q == 1, mode, &g[q], ws, ws_bytes, stream);
      if (s == DEXEL_ERR_CAPACITY && g[q].nseg > cap && attempt < 3) {
        cap = g[q].nseg + 1024;
        continue;
      }
      if (s != DEXEL_OK) return s;
      break;
    }
  }
  const dexel_grid_in d{in->nx, in->ny, in->h, g[0].col_off, g[0].z, g[0].nseg};
  const dexel_grid_in e{in->nx, in->ny, in->h, g[1].col_off, g[1].z, g[1].nseg};
  return boolean_run_any(ctx, kBoolDifference, &d, &e, mode, out, ws, ws_bytes, (cudaStream_t)stream);
}

dexel_status dexel_offset_batched(dexel_ctx* ctx, int nshapes, const dexel_grid_in* ins,
                                  const double* k, const dexel_op* ops, dexel_mode mode,
                                  dexel_grid_out* outs, void* ws, size_t ws_bytes,
                                  int32_t* d_status, void* stream) {
  if (!ctx || nshapes < 0 || (nshapes > 0 && (!ins || !k || !ops || !outs))) return DEXEL_ERR_INVALID_ARG;
  if (mode != DEXEL_FP64 && mode != DEXEL_FP32_PRED64) return DEXEL_ERR_INVALID_ARG;
  for (int s = 0; s < nshapes; ++s) {
    if (check_in(&ins[s], k[s]) != DEXEL_OK) return DEXEL_ERR_INVALID_ARG;
    if (ops[s] < DEXEL_DILATE || ops[s] > DEXEL_OPEN) return DEXEL_ERR_INVALID_ARG;
    const dexel_grid_out& o = outs[s];
    if (!o.col_off || o.capacity_seg < 0 || (o.capacity_seg > 0 && !o.z)) return DEXEL_ERR_INVALID_ARG;
  }
  if (cudaSetDevice(ctx->device) != cudaSuccess) return DEXEL_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  if (!ctx->batch) {
    ctx->batch = batch_engine_create(ctx->device, ctx->sm_count);
    if (!ctx->batch) return DEXEL_ERR_NOMEM;
    batch_set_autotune(ctx->batch, ctx->batch_autotune ? 1 : 0);
  }
  const int fp32 = mode == DEXEL_FP32_PRED64 ? 1 : 0;
  long long launches = 0;
  // Shapes of more than batch_max_cols columns take the single-shape path (their own
  // kernel geometry; batching pays off for the many small shapes, whose launches it shares).
  // First offset of every other shape (the dilation of a closing, the erosion of an opening);
  // the result of a closing / opening goes to engine memory, the others straight to the caller.
  std::vector<int> inb;
  for (int s = 0; s < nshapes; ++s)
    if ((long long)ins[s].nx * ins[s].ny <= ctx->batch_max_cols) inb.push_back(s);
  std::vector<BatchItem> A(inb.size());
  for (size_t q = 0; q < inb.size(); ++q) {
    const int s = inb[q];
    const dexel_op op = ops[s];
    A[q] = BatchItem{ins[s].nx, ins[s].ny, ins[s].h, ins[s].col_off, ins[s].z, ins[s].nseg, k[s],
                     (op == DEXEL_ERODE || op == DEXEL_OPEN) ? 1 : 0, nullptr, nullptr, 0};
    if (op == DEXEL_DILATE || op == DEXEL_ERODE) {
      A[q].out_col_off = outs[s].col_off;
      A[q].out_z = outs[s].z;
      A[q].out_cap = outs[s].capacity_seg;
    }
  }
  std::vector<int> stA, stB;
  std::vector<long long> nA, nB;
  std::vector<int> fin(nshapes, 1);  // 1: the single-shape path
  std::vector<long long> fseg(nshapes, 0);
  // The shapes beyond the batch whose offset (a dilation or an erosion) has a recorded plan
  // on this context: stream-ordered (dexel_offset_enqueue) on a side stream, beside the
  // batch, into the library's workspace; their result words are read once after the batch.
  std::vector<int> queued;
  {
    size_t need = 0;
    std::vector<int> cand;
    for (int s = 0; s < nshapes; ++s) {
      if ((long long)ins[s].nx * ins[s].ny <= ctx->batch_max_cols) continue;
      if (ops[s] != DEXEL_DILATE && ops[s] != DEXEL_ERODE) continue;
      auto it = ctx->tapes.find(tape_key(&ins[s], k[s], ops[s] == DEXEL_ERODE, false,
                                         fp32 ? sizeof(float) : sizeof(double)));
      if (it == ctx->tapes.end()) continue;
      need = std::max(need, it->second.need);
      cand.push_back(s);
    }
    bool ok = !cand.empty() && ensure_owned(ctx, need) == DEXEL_OK;
    if (ok && !ctx->side) ok = cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking) == cudaSuccess;
    if (ok && ctx->res_n < 2 * cand.size()) {
      if (ctx->res_buf) cudaFree(ctx->res_buf);
      ctx->res_buf = nullptr;
      ctx->res_n = 0;
      ok = cudaMalloc(&ctx->res_buf, sizeof(long long) * 2 * cand.size()) == cudaSuccess;
      if (ok) ctx->res_n = 2 * cand.size();
    }
    cudaEvent_t ready = nullptr;
    ok = ok && cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaEventRecord(ready, st) == cudaSuccess && cudaStreamWaitEvent(ctx->side, ready, 0) == cudaSuccess;
    if (ready) cudaEventDestroy(ready);
    cudaGetLastError();
    if (ok) {
      for (size_t q = 0; q < cand.size(); ++q) {
        const int s = cand[q];
        const dexel_status r = dexel_offset_enqueue(ctx, &ins[s], k[s], ops[s], mode, &outs[s], ctx->own,
                                                    ctx->own_bytes, ctx->side,
                                                    (int64_t*)(ctx->res_buf + 2 * queued.size()));
        launches += ctx->launches;
        if (r == DEXEL_OK) {
          queued.push_back(s);
        } else if (r != DEXEL_ERR_NO_PLAN && r != DEXEL_ERR_CAPACITY) {
          return r;  // (a CUDA failure)
        }
      }
    }
  }
  if (!A.empty()) {
    int rc = batch_run(ctx->batch, fp32, A, st, stA, nA, &launches);
    if (rc != DEXEL_OK) return (dexel_status)rc;
    // second offset of closings / openings, from the engine-held first results
    std::vector<BatchItem> B;
    std::vector<int> which;
    for (size_t q = 0; q < inb.size(); ++q) {
      const int s = inb[q];
      if ((ops[s] == DEXEL_CLOSE || ops[s] == DEXEL_OPEN) && stA[q] == DEXEL_OK) {
        B.push_back(BatchItem{ins[s].nx, ins[s].ny, ins[s].h, A[q].out_col_off, A[q].out_z, nA[q],
                              k[s], ops[s] == DEXEL_CLOSE ? 1 : 0, outs[s].col_off, outs[s].z,
                              outs[s].capacity_seg});
        which.push_back(s);
      }
    }
    for (size_t q = 0; q < inb.size(); ++q) {
      fin[inb[q]] = stA[q];
      fseg[inb[q]] = nA[q];
    }
    if (!B.empty()) {
      rc = batch_run(ctx->batch, fp32, B, st, stB, nB, &launches);
      if (rc != DEXEL_OK) return (dexel_status)rc;
      for (size_t q = 0; q < which.size(); ++q) {
        fin[which[q]] = stB[q];
        fseg[which[q]] = nB[q];
      }
    }
  }
  if (!queued.empty()) {
    // the side stream's results (a shape the plan did not fit runs synchronously below)
    std::vector<long long> hr(2 * queued.size());
    if (cudaMemcpyAsync(hr.data(), ctx->res_buf, sizeof(long long) * hr.size(), cudaMemcpyDeviceToHost,
                        ctx->side) != cudaSuccess ||
        cudaStreamSynchronize(ctx->side) != cudaSuccess)
      return DEXEL_ERR_CUDA;
    for (size_t q = 0; q < queued.size(); ++q) {
      const int s = queued[q];
      if (hr[2 * q] == DEXEL_OK) {
        fin[s] = DEXEL_OK;
        fseg[s] = hr[2 * q + 1];
        outs[s].nseg = hr[2 * q + 1];
      }
    }
  }
  // shapes beyond the batch kernels' limits: the single-shape path
  long long singles = 0;
  for (int s = 0; s < nshapes; ++s) singles += fin[s] == 1;
  for (int s = 0; s < nshapes; ++s) {
    if (fin[s] != 1) continue;
    dexel_status r;
    switch (ops[s]) {
      case DEXEL_DILATE: r = dexel_dilate(ctx, &ins[s], k[s], mode, &outs[s], ws, ws_bytes, stream); break;
      case DEXEL_ERODE: r = dexel_erode(ctx, &ins[s], k[s], mode, &outs[s], ws, ws_bytes, stream); break;
      default: r = dexel_morph(ctx, &ins[s], k[s], ops[s], mode, &outs[s], ws, ws_bytes, stream); break;
    }
    launches += ctx->launches;
    fin[s] = r;
    fseg[s] = outs[s].nseg;
  }
  dexel_status first = DEXEL_OK;
  std::vector<int32_t> hst(nshapes > 0 ? nshapes : 1, 0);
  for (int s = 0; s < nshapes; ++s) {
    outs[s].nseg = fseg[s];
    hst[s] = (int32_t)fin[s];
    if (fin[s] != DEXEL_OK && first == DEXEL_OK) first = (dexel_status)fin[s];
  }
  ctx->launches = launches;
  ctx->stats[5] = singles;  // shapes that took the single-shape path
  if (d_status && nshapes > 0) {
    if (cudaMemcpyAsync(d_status, hst.data(), sizeof(int32_t) * nshapes, cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return DEXEL_ERR_CUDA;
  }
  return first;
}

void dexel_set_batch_autotune(dexel_ctx* ctx, int on) {
  if (!ctx) return;
  ctx->batch_autotune = on != 0;
  if (ctx->batch) batch_set_autotune(ctx->batch, on);
}

dexel_status dexel_offset_noalloc(const dexel_grid_in* in, double k, dexel_op op, dexel_mode mode,
                                  dexel_grid_out* out, void* stream) {
  if (!out || !out->col_off || (out->capacity_seg > 0 && !out->z) || out->capacity_seg < 0)
    return DEXEL_ERR_INVALID_ARG;
  if (op != DEXEL_DILATE && op != DEXEL_ERODE) return DEXEL_ERR_INVALID_ARG;
  if (mode != DEXEL_FP64 && mode != DEXEL_FP32_PRED64) return DEXEL_ERR_INVALID_ARG;
  const dexel_status s = check_in(in, k);
  if (s != DEXEL_OK) return s;
  out->nseg = -1;  // beyond the static scratch's limits (below): not an output-size problem
  if ((long long)in->nx * in->ny > kNoAllocMaxColumns || k > kNoAllocMaxK) return DEXEL_ERR_CAPACITY;
  cudaStream_t st = (cudaStream_t)stream;
  const bool erode = op == DEXEL_ERODE;
  if (mode == DEXEL_FP64) return noalloc_offset<double>(in, k, erode, out, st);
  return noalloc_offset<float>(in, k, erode, out, st);
}

const char* dexel_last_error_detail(void) { return g_err_detail; }

const char* dexel_status_string(dexel_status s) {
  switch (s) {
    case DEXEL_OK: return "ok";
    case DEXEL_ERR_INVALID_ARG: return "invalid argument";
    case DEXEL_ERR_BAD_CSR: return "malformed CSR dexel grid";
    case DEXEL_ERR_CAPACITY: return "output or workspace capacity too small";
    case DEXEL_ERR_CUDA: return "CUDA runtime error";
    case DEXEL_ERR_TIMEOUT: return "bounded device wait gave up";
    case DEXEL_ERR_NOMEM: return "out of memory";
    case DEXEL_ERR_NO_PLAN: return "no recorded plan fits this offset (call it synchronously)";
  }
  return "unknown status";
}

}  // extern "C"
