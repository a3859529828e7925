// Internal launch wrappers shared by the translation units of libdexel.
#pragma once
#include <cuda_runtime.h>

#include <vector>
#include "../../include/dexel.h"
#include "gather2.cuh"

namespace dexel {

constexpr int kWarpsPerBlock = 4;
// window gather (pass 2): largest reach it takes (beyond it the per-line sweep runs), and the
// per-round limits of a lane in k_pass2t (appended intervals, pieces taken)
constexpr int kGatherMaxReach = 1024;
// pass-1 gather: the open sources of a window are a mask of up to 256 bits, 2R + 1 <= 255
constexpr int kGatherMaxReach1 = 127;
// pass 1 with one lane per column: two 128-bit masks a side (R <= 128) and a tile-relative
// mask of 320 bits (32 + 2R + 1 <= 320)
constexpr int kLaneMaxReach1 = 128;
constexpr int kRoundAppends = 2;
constexpr int kRoundPieces = 32;

template <typename T>
cudaError_t launch_pass1(const P1Params<T>& P, int blocks, cudaStream_t st);
template <typename T>
cudaError_t launch_pass1g(const P1Params<T>& P, int tc, int ecap, int obuf, int blocks,
                          cudaStream_t st);
template <typename T>
long long pass1g_smem(int tc, int R, int ecap, int obuf);
// pass 1 with one lane per output column (pass1l.cu); ecap (a power of two) events a tile,
// gw (1, 2, 4, 8) warps a tile
template <typename T>
cudaError_t launch_pass1l(const P1Params<T>& P, int ecap, int gw, int sms, cudaStream_t st);
// ksz: bytes of an event key (8 for double inputs, 4 for float); nbuf: event buffers (2:
// room to merge the sources' runs of any window that fits one buffer)
long long pass1l_smem(int R, int ecap, int gw, int ksz = 8, int nbuf = 1);
// pass 1 for reaches up to kMergeMaxReach, one lane a column merging its window's sources
// (pass1m.cu); measured faster than the window kernel at reach 2 (0.35 against 0.57 ms on
// the 512^2 workload), much slower at reach 8 (each step advances one of 17 slots
// predicated over all of them)
constexpr int kMergeMaxReach = 2;
template <typename T>
cudaError_t launch_pass1m(const P1Params<T>& P, int sms, cudaStream_t st);
// blocks of 256 threads launch_pass1l starts (its ring, when given, holds r_cap pieces for
// each of their threads)
int pass1l_blocks(int nx, int ny, int R, int ecap, int gw, int sms, int ksz = 8, int nbuf = 1);
template <typename T>
cudaError_t launch_pass2(const P2Params<T>& P, int blocks, cudaStream_t st);
template <typename T>
cudaError_t launch_pass2t(const P2GParams<T>& P, int warps_per_block, int tc, int ntab,
                          int stage_cap, int Q, int M, int minb, int blocks, cudaStream_t st);
// Pass 2 by levels (pass2l.cu): per-source level unions into l_p, indexed by output
// column (l_idx: 2R + 1 packed entries a column, entry u the list of source j - R + u at level
// |u - R|), then the per-column gather with buckets of bcap intervals.
template <typename T>
struct LvlParamsHost {
  P2GParams<T> P;
  ulonglong2* l_p;  // (left, right) keys of the level lists' intervals
  long long l_cap;
  unsigned long long* l_idx;
  int bcap;
  long long m_cap, c_cap;  // entries of the S_mid arena and of its packed copy (self-checks)
  bool exact;  // k_levels reads S_mid itself (no packed copy; c_start unused)
  // a block of whole y lines: sources / output columns q0 .. q0 + nq - 1 in line order
  // (q = i * ny + j; nq = 0: the whole grid); l_idx holds the block's entries only
  long long q0 = 0, nq = 0;
  // reach of the output window along y (-1: R; 0: the 2D slices, a column's own level 0)
  int yw = -1;
  // interval slots a lane of the level walks (0: by reach; at most 16)
  int slots = 0;
  // spill regions of k_levels (lvl_spill_bytes of them; null: none): spill_cap intervals a
  // lane of every warp of its grid beyond the slots
  unsigned* spill = nullptr;
  int spill_cap = 0;
};
// bytes of k_levels' spill regions for spill_cap intervals a lane
long long lvl_spill_bytes(int sms, int spill_cap);
// k_levels (the per-source level lists); launch_lgather then unites them per column
template <typename T>
cudaError_t launch_levels(const LvlParamsHost<T>& H, cudaStream_t st, int sms);
template <typename T>
cudaError_t launch_lgather(const LvlParamsHost<T>& H, int bcap, int redo, cudaStream_t st, int sms);
// the same gather with one lane an output column (short windows; columns it cannot finish
// are marked for launch_lgather's redo)
template <typename T>
cudaError_t launch_lgather_lanes(const LvlParamsHost<T>& H, cudaStream_t st, int sms);
template <typename T>
cudaError_t launch_pass2c(const P2GParams<T>& P, int warps_per_block, int blocks, cudaStream_t st);

// Boolean operations of two grids (csg.cu): per-column counts, then the segments at the
// scanned positions
constexpr int kBoolUnion = 0, kBoolIntersect = 1, kBoolDifference = 2;
template <typename T>
cudaError_t launch_bool_count(int op, long long ncols, const int* oa, const T* za, const int* ob,
                              const T* zb, long long* cnt, cudaStream_t st);
template <typename T>
cudaError_t launch_bool_write(int op, long long ncols, const int* oa, const T* za, const int* ob,
                              const T* zb, const long long* pos, T* zo, cudaStream_t st);

// Ray casting of primitives into a grid (raycast.cu): a counting launch (write false: cnt[c]
// = segments of column c) or a writing launch at the scanned positions pos; a column with more
// chords than a thread holds sets ST_OVERFLOW_SLOT
template <typename T>
cudaError_t launch_raycast(const dexel_prim* prims, int nprim, int axis, int nx, long long ncols,
                           double h, long long* cnt, const long long* pos, T* zo, Counters* ctr,
                           bool write, cudaStream_t st);

// Batched offsets (batch.cu): one launch per stage over many shapes.  An item's status after
// batch_run: DEXEL_OK, DEXEL_ERR_BAD_CSR, DEXEL_ERR_CAPACITY (nseg holds the need), or 1 when
// the item needs the single-shape path (a window beyond the batch kernels' limits).  An item
// with out_z == nullptr gets its output in engine-owned memory (pointers set in the item,
// valid until the engine's next run).
struct BatchItem {
  int nx, ny;
  double h;
  const int* col_off;
  const void* z;
  long long nseg;
  double k;
  int erode;
  int* out_col_off;
  void* out_z;
  long long out_cap;
};
struct BatchEngine;
BatchEngine* batch_engine_create(int device, int sms);
void batch_engine_destroy(BatchEngine* e);
void batch_set_autotune(BatchEngine* e, int on);
int batch_run(BatchEngine* e, int fp32, std::vector<BatchItem>& items, cudaStream_t st,
              std::vector<int>& status, std::vector<long long>& nseg, long long* launches);

}  // namespace dexel
