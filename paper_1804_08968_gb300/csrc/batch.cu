// Batched offsets: many shapes, each with its own grid, radius and operation, computed with
// one launch per stage over a table of shapes (validation, tables, pass-1 gather, packing,
// pass-2 gather, output count, scan, output write).  Tiles of all shapes are numbered
// globally; a block (or a warp group) finds the shape of its tile by binary search over the
// tile bases and runs the same tile bodies as the single-shape kernels (pass1l.cuh,
// pass2l.cuh, pass2t.cuh).
//
// Once a batch of a given shape signature has run without growing its scratch, the launch
// sequence up to the output count is recorded as a CUDA graph and replayed by the next call
// with the same signature (the kernels read every per-shape pointer from the shape table, so
// only the table is uploaded again).  Pass-1 tiles are 32 columns, taken by groups of warps
// whose size follows the largest radius; pass-2 tiles are chosen per shape from its radius.
// Each rule has one scale; with autotuning on, the first call of a signature times the
// scales {1/2, 1, 2} x the default for each pass and keeps the fastest.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "../../include/dexel.h"
#include "emit.cuh"
#include "launch.h"
#include "pass1l.cuh"
#include "pass2l.cuh"
#include "pass2t.cuh"

namespace dexel {

constexpr int BS_BAD = 1, BS_REDO = 2, BS_CAP = 4, BS_SWEEP = 8;  // per-shape status bits

template <typename T>
struct BShape {
  P1Params<T> p1;   // pass 1 (m_start / m_cnt point at the shape's columns)
  P2GParams<T> p2;  // pass 2 (o_start / o_cnt / c_start likewise, tables at the shape's)
  LvlParams<T> lv;  // pass 2 by levels (p2 plus the shape's level lists)
  long long col_base, ncols;
  int tc2, ntab2, nmax;
  double kk, h;
  int erode;
  int* out_col_off;
  T* out_z;
  long long out_cap;
  long long nseg_in;
  unsigned zmax_bits;  // max |z| of the shape's input (float bits), for the pruning margin
};

// largest s in [0, ns) with base[s] <= x (base has ns + 1 entries)
__device__ __forceinline__ int find_base(const long long* base, int ns, long long x) {
  int lo = 0, hi = ns - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (base[mid] <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <typename T>
__global__ void k_b_validate(BShape<T>* S, const long long* colb, int ns, long long ncols,
                             int* sst) {
  const long long c0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long c = c0 < ncols ? c0 : ncols - 1;  // (every lane takes part in the reduction)
  const int s = find_base(colb, ns, c);
  float zm = 0.0f;  // max |z| of the column, reduced per shape below
  {
    const BShape<T>& B0 = S[s];
    const int s0 = B0.p1.col_off[c - colb[s]], s1 = B0.p1.col_off[c - colb[s] + 1];
    if (c0 < ncols && s0 >= 0 && s1 <= B0.nseg_in)
      for (int g = s0; g < s1; ++g) {
        const float a = fabsf((float)B0.p1.z[2LL * g]), b = fabsf((float)B0.p1.z[2LL * g + 1]);
        if (a < __builtin_huge_valf()) zm = fmaxf(zm, a);
        if (b < __builtin_huge_valf()) zm = fmaxf(zm, b);
      }
  }
  {
    // one atomic a warp when its columns are one shape's, else one a lane
    const int s_first = __shfl_sync(0xffffffffu, s, 0);
    if (__all_sync(0xffffffffu, s == s_first)) {
      const unsigned zb = __reduce_max_sync(0xffffffffu, __float_as_uint(zm));
      if ((threadIdx.x & 31) == 0 && zb > 0) atomicMax(&S[s].zmax_bits, zb);
    } else if (zm > 0.0f) {
      atomicMax(&S[s].zmax_bits, __float_as_uint(zm));
    }
  }
  if (c0 >= ncols) return;
  const BShape<T>& B = S[s];
  const long long cl = c - colb[s];
  B.p1.m_cnt[cl] = 0;
  B.p1.m_start[cl] = 0;
  B.p2.o_cnt[cl] = 0;
  B.p2.o_start[cl] = 0;
  const int* off = B.p1.col_off;
  const T* z = B.p1.z;
  const int s0 = off[cl], s1 = off[cl + 1];
  bool bad = false;
  if (cl == 0 && s0 != 0) bad = true;
  if (cl == B.ncols - 1 && (long long)s1 != B.nseg_in) bad = true;
  if (s1 < s0 || s0 < 0 || (long long)s1 > B.nseg_in) bad = true;
  if (!bad) {
    for (int g = s0; g < s1; ++g) {
      const T a = z[2LL * g], b = z[2LL * g + 1];
      if (!(a <= b)) { bad = true; break; }  // also catches NaN
      if (!(a > -(T)INFINITY) || !(b < (T)INFINITY)) { bad = true; break; }
      if (g + 1 < s1 && !(b < z[2LL * (g + 1)])) { bad = true; break; }
    }
  }
  if (bad) atomicOr(&sst[s], BS_BAD);
}

template <typename T>
__global__ void k_b_tables(const BShape<T>* S, const long long* tabb, int ns, long long ntab,
                           double* wtab, float* wtabf) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ntab) return;
  const int s = find_base(tabb, ns, e);
  const long long n = e - tabb[s];
  if (n <= S[s].nmax) {
    const double w = S[s].h * sqrt(S[s].kk - (double)n);  // half-width h sqrt(k^2 - n)
    wtab[e] = w;
    wtabf[e] = (float)w;
  }
}

// the pass-1 pruning margin of every shape: 2^-19 (max |z| + k h), over four times the error
// bound of the float dominance test (as for single shapes)
template <typename T>
__global__ void k_b_prune(BShape<T>* S, int ns) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ns || S[s].p1.prune_w == nullptr) return;
  const double zm = (double)__uint_as_float(S[s].zmax_bits);
  S[s].p1.prune_E = (float)(1.9073486328125e-6 * (zm + sqrt(S[s].kk) * S[s].h));  // 2^-19
}

// pass 1, one lane per output column: groups of gw warps, each a tile of 32 columns of one
// shape (the shapes of one mask width NH; the other launch takes the rest)
template <typename T, int NH>
__global__ void __launch_bounds__(256, 3) k_b_pass1(const BShape<T>* S, const long long* t1b,
                                                    int ns, long long ntiles, int ecap, int gw,
                                                    long long gstride, const int* sst) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5;
  const int groups = (blockDim.x >> 5) / gw;
  const TGroup G{gw, warp / gw, warp % gw, (int)threadIdx.x % (gw * 32), 0};  // no ring
  ArenaCursor cur{0, 0};
  for (long long gt = (long long)blockIdx.x * groups + G.gid; gt < ntiles;
       gt += (long long)gridDim.x * groups) {
    const int s = find_base(t1b, ns, gt);
    if ((sst[s] & BS_BAD) || (S[s].p1.K <= 64 ? 1 : 2) != NH) continue;  // another launch's class
    unsigned char* gsm = smem + (long long)G.gid * gstride;  // the largest shape's layout
    pass1l_tile<T, NH>(S[s].p1, gt - t1b[s], ecap, gsm, G, cur);
  }
  if (G.gtid == 0 && cur.tally > 0) {
    add_total(&S[0].p1.ctr->mid_total, cur.tally);
    note_max(&S[0].p1.ctr->max_pieces, cur.tmax);
  }
}

template <typename T, int MINB>
__global__ void __launch_bounds__(512, MINB) k_b_pass2(const BShape<T>* S, const long long* t2b,
                                                       int ns, long long ntiles, int stage_cap,
                                                       int Q, int M, const int* sst) {
  extern __shared__ __align__(16) unsigned char smem[];
  ArenaCursor cur{0, 0};
  for (long long gt = blockIdx.x; gt < ntiles; gt += gridDim.x) {
    const int s = find_base(t2b, ns, gt);
    if (sst[s] & BS_BAD) continue;
    const P2GParams<T> P = S[s].p2;
    const int tc = S[s].tc2, ntab = S[s].ntab2;
    const P2TLayout Lo = p2t_layout(P.R, tc, ntab, stage_cap, blockDim.x >> 5, P.bcap);
    float* swt = (float*)(smem + Lo.swt);
    __syncthreads();  // the previous tile no longer reads the table
    for (int q = threadIdx.x; q < ntab; q += blockDim.x) swt[q] = P.wtabf[q];
    pass2t_tile<T>(P, gt - t2b[s], tc, ntab, stage_cap, Q, M, smem, ntab > 0 ? swt : P.wtabf, cur);
  }
}

// TABM: kTabWarp (each warp builds its lanes' radius table per item, tstride floats a warp
// after the level layout) or kTabFlat (the shape's flat table in global memory)
template <typename T, int TABM>
__global__ void __launch_bounds__(256) k_b_levels(const BShape<T>* __restrict__ S,
                                                  const long long* lvb, int ns, long long nitems,
                                                  int tstride, const int* sst) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const LvlLayout Lo = lvl_layout(blockDim.x >> 5, 0);
  unsigned* ws = (unsigned*)(smem + Lo.slots) + warp * 2 * kLvlSlots * 32;  // room for any shape's
  float4* stg = (float4*)(smem + Lo.stage) + warp * kLvlStage;
  float* wt = (float*)(smem + Lo.total) + (long long)warp * tstride;
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  ArenaCursor cur{0, 0};
  for (long long gi = (long long)blockIdx.x * (blockDim.x >> 5) + warp; gi < nitems; gi += nw) {
    const int s = find_base(lvb, ns, gi);
    if (sst[s] & BS_BAD) continue;
    const LvlParams<T> A = S[s].lv;
    const float E = 9.5367432e-7f * (__uint_as_float(A.P.ctr->zmax_bits) + A.P.wtabf[0]);
    levels_item<T, TABM>(A, gi - lvb[s], lane, ws, stg, E,
                         TABM == kTabWarp ? wt : (float*)A.P.wtabf, cur,
                         (long long)blockIdx.x * (blockDim.x >> 5) + warp);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_b_lgather(const BShape<T>* S, const long long* colb,
                                                   int ns, long long ncols, int bcap,
                                                   const int* sst, const Counters* ctr) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char* wb = smem + (long long)warp * (bcap * (2 * sizeof(ukey) + 2 * sizeof(int)) + 16);
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  if (*(const volatile int*)&ctr->status & ST_LEVELS_OVER) return;  // the lists are incomplete
  ArenaCursor cur{0, 0};
  for (long long gi = (long long)blockIdx.x * (blockDim.x >> 5) + warp; gi < ncols; gi += nw) {
    const int s = find_base(colb, ns, gi);
    if (sst[s] & BS_BAD) continue;
    const LvlParams<T> A = S[s].lv;
    lgather_column<T>(A, gi - colb[s], bcap, 0, lane, wb, cur);
  }  if (lane == 0 && cur.tally > 0) {
    add_total(&S[0].p2.ctr->out_total, cur.tally);
    note_max(&S[0].p2.ctr->max_out, cur.tmax);
  }
}

// the columns marked -1 by k_b_lgather, with a larger bucket
template <typename T>
__global__ void __launch_bounds__(256) k_b_lgather_redo(const BShape<T>* S, const long long* colb,
                                                        int ns, long long ncols, int bcap,
                                                        const int* sst) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char* wb = smem + (long long)warp * (bcap * (2 * sizeof(ukey) + 2 * sizeof(int)) + 16);
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  ArenaCursor cur{0, 0};
  for (long long gi = (long long)blockIdx.x * (blockDim.x >> 5) + warp; gi < ncols; gi += nw) {
    const int s = find_base(colb, ns, gi);
    if (sst[s] & BS_BAD) continue;
    const LvlParams<T> A = S[s].lv;
    lgather_column<T>(A, gi - colb[s], bcap, 1, lane, wb, cur);
  }  if (lane == 0 && cur.tally > 0) {
    add_total(&S[0].p2.ctr->out_total, cur.tally);
    note_max(&S[0].p2.ctr->max_out, cur.tmax);
  }
}

template <typename T>
__global__ void k_b_count(const BShape<T>* S, const long long* colb, int ns, long long ncols,
                          long long* cnt, int* sst) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncols) return;
  const int s = find_base(colb, ns, c);
  const BShape<T>& B = S[s];
  const long long cl = c - colb[s];
  const int nx = B.p1.nx, ny = B.p1.ny;
  const long long i = cl % nx, j = cl / nx;
  long long v = 0;
  if (B.p1.m_start[i * ny + j] < 0) atomicOr(&sst[s], BS_SWEEP);
  const int oc = B.p2.o_cnt[cl];
  if (oc < 0) atomicOr(&sst[s], BS_REDO);
  else if (!(sst[s] & BS_BAD))
    v = finalize_column<T>(B.p2.o_l + B.p2.o_start[cl], B.p2.o_r + B.p2.o_start[cl], oc,
                           B.erode != 0, nullptr);
  cnt[c] = v;
}

// prefix of the scanned counts at x (x == ncols: the total)
__device__ __forceinline__ long long scanned(const long long* pos, const long long* sums,
                                             long long ncols, long long x) {
  return x < ncols ? pos[x] + sums[x / kScanTile] : sums[(ncols + kScanTile - 1) / kScanTile];
}

template <typename T>
__global__ void k_b_totals(const BShape<T>* S, const long long* colb, int ns, long long ncols,
                           const long long* pos, const long long* sums, long long* totals,
                           int* sst) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ns) return;
  const long long tot = scanned(pos, sums, ncols, colb[s + 1]) - scanned(pos, sums, ncols, colb[s]);
  totals[s] = tot;
  if (S[s].out_z && (tot > S[s].out_cap || tot > 0x7fffffffLL)) atomicOr(&sst[s], BS_CAP);
}

template <typename T>
__global__ void k_b_write(const BShape<T>* S, const long long* colb, int ns, long long ncols,
                          const long long* pos, const long long* sums, const long long* totals,
                          const int* sst) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncols) return;
  const int s = find_base(colb, ns, c);
  if (sst[s] & (BS_BAD | BS_REDO | BS_SWEEP | BS_CAP)) return;
  const BShape<T>& B = S[s];
  const long long cl = c - colb[s];
  const long long p = scanned(pos, sums, ncols, c) - scanned(pos, sums, ncols, colb[s]);
  B.out_col_off[cl] = (int)p;
  if (cl == B.ncols - 1) B.out_col_off[B.ncols] = (int)totals[s];
  finalize_column<T>(B.p2.o_l + B.p2.o_start[cl], B.p2.o_r + B.p2.o_start[cl], B.p2.o_cnt[cl],
                     B.erode != 0, B.out_z + 2 * p);
}

// ------------------------------------------------------------------------------------------
// host engine
// ------------------------------------------------------------------------------------------

struct BatchEngine {
  int device = 0, sms = 152;
  bool autotune = true;
  bool prune = true;  // dominance pruning of S_mid pieces in pass 1
  cudaStream_t cap_stream = nullptr;  // private stream for graph capture
  void* ws = nullptr;
  size_t ws_bytes = 0;
  void* host = nullptr;  // pinned upload buffer
  size_t host_bytes = 0;
  void* mid = nullptr;  // internal outputs
  size_t mid_bytes = 0;
  unsigned* spill = nullptr;  // the level walks' spill regions (every warp of k_b_levels' grid)
  long long needM = 0, needO = 0, needL = 0;  // arena entries learnt
  std::map<std::vector<long long>, bool> no_levels;  // signatures whose level lists overflowed
  // recorded launch sequences by signature (shapes, scratch, tile scales)
  std::map<std::vector<long long>, cudaGraphExec_t> graphs;
  std::map<std::vector<long long>, bool> graph_writes;  // the graph ends with the output write
  std::map<std::vector<long long>, std::vector<long long>> last_tot;  // totals of the last call
  // autotuned tile scales per signature (x 1/2: 0 = half, 1 = default, 2 = double)
  std::map<std::vector<long long>, std::pair<int, int>> scales;
};

// intervals a lane of the batched level walks spills beyond its slots
constexpr int kBatchSpill = 64;

BatchEngine* batch_engine_create(int device, int sms) {
  BatchEngine* e = new (std::nothrow) BatchEngine;
  if (!e) return nullptr;
  e->device = device;
  e->sms = sms > 0 ? sms : 152;
  // the level walks' spill regions (the grid of k_b_levels: sms x 4 blocks of 8 warps); without
  // them a long list is walked again
  if (cudaMalloc(&e->spill, (size_t)lvl_spill_bytes(e->sms, kBatchSpill)) != cudaSuccess) {
    cudaGetLastError();
    e->spill = nullptr;
  }
  return e;
}

void batch_engine_destroy(BatchEngine* e) {
  if (!e) return;
  for (auto& g : e->graphs) cudaGraphExecDestroy(g.second);
  if (e->cap_stream) cudaStreamDestroy(e->cap_stream);
  if (e->ws) cudaFree(e->ws);
  if (e->mid) cudaFree(e->mid);
  if (e->spill) cudaFree(e->spill);
  if (e->host) cudaFreeHost(e->host);
  delete e;
}

void batch_set_autotune(BatchEngine* e, int on) {
  if (e) e->autotune = on != 0;
}

namespace {

inline size_t bal(size_t x) { return (x + 255) / 256 * 256; }

int reach_of_kk(double kk) {
  long long R = (long long)std::floor(std::sqrt(kk));
  while ((double)((R + 1) * (R + 1)) <= kk) ++R;
  while (R > 0 && (double)(R * R) > kk) --R;
  return (int)R;
}

// tile rule of pass 2: about 2K + 16 columns, scaled by 2^(scale - 1) (the pass-1 scale
// scales the warps a pass-1 tile instead)
int tile2(int K, int scale) {
  int tc = 16;
  const int want = std::max(16, (2 * K + 16) << scale >> 1);
  while (tc < 128 && tc < want) tc <<= 1;
  return tc;
}

struct Plan {
  size_t total = 0;
  size_t o_ctr, o_shapes, o_bases, o_sst, o_tot, o_colll, o_colint, o_cnt, o_pos, o_sums, o_cst,
      o_tab, o_tabf, o_M, o_F, o_O, o_lst, o_lcnt, o_L;
  long long capM = 0, capO = 0, capF = 0, capL = 0;
};

}  // namespace

template <typename T>
static int batch_run_t(BatchEngine* E, std::vector<BatchItem>& items, cudaStream_t st,
                       std::vector<int>& status, std::vector<long long>& nseg, long long* launches,
                       int depth) {
  typedef typename H<T>::K Key;
  const int ns = (int)items.size();
  status.assign(ns, DEXEL_OK);
  nseg.assign(ns, 0);
  if (ns == 0) return DEXEL_OK;
  if (cudaSetDevice(E->device) != cudaSuccess) return DEXEL_ERR_CUDA;
#define BK(x) do { if ((x) != cudaSuccess) return DEXEL_ERR_CUDA; } while (0)
  // ---- per-shape geometry
  std::vector<int> K(ns), nmax(ns);
  std::vector<long long> colb(ns + 1, 0), tabb(ns + 1, 0), t1b(ns + 1, 0), t2b(ns + 1, 0);
  std::vector<long long> lvb(ns + 1, 0), nlb(ns + 1, 0);  // level items, level-list entries
  std::vector<long long> sig;
  sig.push_back(ns);
  sig.push_back(sizeof(T));
  long long nseg_all = 0, estM = 0, estO = 0;
  int maxK = 0;
  for (int s = 0; s < ns; ++s) {
    const BatchItem& it = items[s];
    const double kk = it.k * it.k;
    K[s] = reach_of_kk(kk);
    nmax[s] = (int)std::floor(kk);
    maxK = std::max(maxK, K[s]);
    const long long nc = (long long)it.nx * it.ny;
    colb[s + 1] = colb[s] + nc;
    {
      const int L = K[s] + 1;
      const long long items = lvl_items(nc, L);
      lvb[s + 1] = lvb[s] + items;
      nlb[s + 1] = nlb[s] + nc * (2LL * K[s] + 1);  // index entries by output column
    }
    tabb[s + 1] = tabb[s] + nmax[s] + 2;
    nseg_all += it.nseg;
    estM += (it.nseg + nc) * std::min(K[s] + 2, 64);
    estO += 2 * (it.nseg + nc);
    sig.push_back(it.nx);
    sig.push_back(it.ny);
    sig.push_back((long long)std::llround(kk * 1024.0));
    sig.push_back(it.erode);
  }
  if (maxK > kGatherMaxReach1) {
    // beyond the pass-1 gather: every shape takes the single-shape path
    for (int s = 0; s < ns; ++s) status[s] = 1;
    return DEXEL_OK;
  }
  const long long ncols = colb[ns], ntab = tabb[ns];
  auto sc_it = E->scales.find(sig);
  int sc1 = 1, sc2 = 1;
  if (sc_it != E->scales.end()) { sc1 = sc_it->second.first; sc2 = sc_it->second.second; }
  std::vector<int> tc2(ns);
  auto tiles = [&](int a1, int a2) {
    for (int s = 0; s < ns; ++s) {
      tc2[s] = tile2(K[s], a2);
      t1b[s + 1] = t1b[s] + (long long)items[s].ny * ((items[s].nx + 31) / 32);
      t2b[s + 1] = t2b[s] + (long long)items[s].nx * ((items[s].ny + tc2[s] - 1) / tc2[s]);
    }
  };
  tiles(sc1, sc2);
  // kernel geometry: pass-1 events and pass-2 staging sized for the largest shape parameters.
  // Pass 1: a tile's window events (twice the mean density of its shape, at least 1024; a
  // shape with a denser window takes the single-shape path), warps a tile by the largest
  // reach, scaled by the pass-1 scale
  int ecap = 1024;
  for (int s = 0; s < ns; ++s) {
    const long long nc = (long long)items[s].nx * items[s].ny;
    const double ev_col = 2.0 * (double)items[s].nseg / (double)std::max<long long>(nc, 1) + 2.0;
    const double ev_tile = (32.0 + 2.0 * K[s] + 1) * ev_col * 2.0;
    while (ecap < 16384 && ecap < ev_tile) ecap <<= 1;
  }
  int gw1 = std::min(8, std::max(1, ((maxK <= 12 ? 2 : (maxK <= 48 ? 4 : 8)) << sc1) >> 1));
  long long sm1 = 0;
  for (;;) {  // fewer tile groups a block when their shared memory does not fit
    sm1 = 0;
    for (int s = 0; s < ns; ++s) sm1 = std::max(sm1, pass1l_smem(K[s], ecap, gw1));
    if (sm1 <= (220LL << 10) || gw1 == 8) break;
    gw1 <<= 1;
  }
  const int bcap = 128, wpb2 = 16;
  long long base2 = 0;
  for (int s = 0; s < ns; ++s) {
    const int nt = nmax[s] + 1 <= 4096 ? nmax[s] + 1 : 0;
    base2 = std::max(base2, p2t_layout(K[s], 128, nt, 0, wpb2, bcap).total);
  }
  const int minb = maxK <= 12 ? 2 : 1;
  bool has_nh[2] = {false, false};  // pass-1 centred mask widths present (1, 2 words)
  for (int s = 0; s < ns; ++s) has_nh[K[s] <= 64 ? 0 : 1] = true;
  const long long budget2 = minb == 2 ? (108LL << 10) : (220LL << 10);
  const int stage_cap = (int)std::max<long long>(512, (budget2 - base2 - 64) / 10);
  long long sm2 = 0;
  for (int s = 0; s < ns; ++s) {
    const int nt = nmax[s] + 1 <= 4096 ? nmax[s] + 1 : 0;
    sm2 = std::max(sm2, p2t_layout(K[s], 128, nt, stage_cap, wpb2, bcap).total);
  }
  if (sm2 > (227LL << 10) || sm1 > (227LL << 10)) {
    for (int s = 0; s < ns; ++s) status[s] = 1;
    return DEXEL_OK;
  }

  // outputs the engine provides (the first offset of a closing / opening), fixed before the
  // attempts (an attempt may point them into the engine's buffer)
  std::vector<char> internal(ns, 0);
  bool have_internal = false;
  for (int s = 0; s < ns; ++s) {
    internal[s] = items[s].out_z == nullptr;
    have_internal = have_internal || internal[s];
  }
  for (int attempt = 0; attempt < 8; ++attempt) {
    // ---- workspace plan
    Plan pl;
    size_t x = 0;
    auto take = [&](size_t bytes) { const size_t o = x; x = bal(x + bytes); return o; };
    pl.o_ctr = take(sizeof(Counters));
    pl.o_shapes = take(sizeof(BShape<T>) * ns);
    pl.o_bases = take(sizeof(long long) * 5 * (ns + 1));
    pl.o_sst = take(sizeof(int) * ns);
    pl.o_tot = take(sizeof(long long) * ns);
    pl.o_colll = take(sizeof(long long) * 2 * ncols);  // m_start, o_start
    pl.o_colint = take(sizeof(int) * 2 * ncols);       // m_cnt, o_cnt
    pl.o_cnt = take(sizeof(long long) * (ncols + 1));
    pl.o_pos = take(sizeof(long long) * (ncols + 1));
    pl.o_sums = take(sizeof(long long) * ((ncols + kScanTile) / kScanTile + 2));
    pl.o_cst = take(sizeof(long long) * (ncols + 1));
    pl.o_tab = take(sizeof(double) * ntab);
    pl.o_tabf = take(sizeof(float) * ntab);
    pl.capM = std::max<long long>(std::max(E->needM + E->needM / 8, estM), 1024);
    pl.capO = std::max<long long>(std::max(E->needO + E->needO / 8, estO), 1024);
    pl.capF = pl.capM;
    pl.o_M = take((size_t)pl.capM * (2 * sizeof(Key) + 2));
    pl.o_F = take((size_t)pl.capF * 10);
    pl.o_O = take((size_t)pl.capO * 16);
    const bool levels = !E->no_levels.count(sig);
    const long long nlev_all = nlb[ns];
    // level-list intervals: about two a (source, level) pair, half the index entries
    pl.capL = levels ? std::max<long long>(std::max(E->needL + E->needL / 8, nlev_all), 1024) : 0;
    pl.o_lst = take(levels ? sizeof(unsigned long long) * nlev_all : 0);
    pl.o_lcnt = take(0);
    pl.o_L = take((size_t)pl.capL * 16);
    pl.total = x + 256;
    if (pl.total > E->ws_bytes) {
      if (E->ws) cudaFree(E->ws);
      E->ws = nullptr;
      E->ws_bytes = 0;
      for (auto& g : E->graphs) cudaGraphExecDestroy(g.second);  // they point into the old scratch
      E->graphs.clear();
      const size_t want = pl.total + pl.total / 4;
      if (cudaMalloc(&E->ws, want) != cudaSuccess) return DEXEL_ERR_NOMEM;
      E->ws_bytes = want;
    }
    char* W = (char*)E->ws;
    Counters* ctr = (Counters*)(W + pl.o_ctr);
    BShape<T>* dS = (BShape<T>*)(W + pl.o_shapes);
    long long* dB = (long long*)(W + pl.o_bases);
    long long *d_colb = dB, *d_tabb = dB + (ns + 1), *d_t1b = dB + 2 * (ns + 1), *d_t2b = dB + 3 * (ns + 1);
    long long* d_lvb = dB + 4 * (ns + 1);
    int* d_sst = (int*)(W + pl.o_sst);
    long long* d_tot = (long long*)(W + pl.o_tot);
    long long* m_start = (long long*)(W + pl.o_colll);
    long long* o_start = m_start + ncols;
    int* m_cnt = (int*)(W + pl.o_colint);
    int* o_cnt = m_cnt + ncols;
    long long* cnt = (long long*)(W + pl.o_cnt);
    long long* pos = (long long*)(W + pl.o_pos);
    long long* sums = (long long*)(W + pl.o_sums);
    long long* cst = (long long*)(W + pl.o_cst);
    double* wtab = (double*)(W + pl.o_tab);
    float* wtabf = (float*)(W + pl.o_tabf);
    Key* m_a = (Key*)(W + pl.o_M);
    Key* m_b = m_a + pl.capM;
    short* m_l = (short*)(m_b + pl.capM);
    float* c_af = (float*)(W + pl.o_F);
    float* c_bf = c_af + pl.capF;
    short* c_dx = (short*)(c_bf + pl.capF);
    ukey* o_l = (ukey*)(W + pl.o_O);
    ukey* o_r = o_l + pl.capO;
    unsigned long long* l_idx = (unsigned long long*)(W + pl.o_lst);
    ulonglong2* l_p = (ulonglong2*)(W + pl.o_L);

    // ---- shape table
    std::vector<BShape<T>> hs(ns);
    for (int s = 0; s < ns; ++s) {
      const BatchItem& it = items[s];
      BShape<T>& B = hs[s];
      memset(&B, 0, sizeof(B));
      B.col_base = colb[s];
      B.ncols = colb[s + 1] - colb[s];
      B.tc2 = tc2[s];
      B.nmax = nmax[s];
      B.ntab2 = nmax[s] + 1 <= 4096 ? nmax[s] + 1 : 0;
      B.kk = it.k * it.k;
      B.h = it.h;
      B.erode = it.erode;
      B.out_col_off = it.out_col_off;
      B.out_z = (T*)it.out_z;
      B.out_cap = it.out_cap;
      B.nseg_in = it.nseg;
      P1Params<T>& p = B.p1;
      p.nx = it.nx; p.ny = it.ny; p.K = K[s]; p.erode = it.erode;
      p.col_off = it.col_off; p.z = (const T*)it.z;
      p.m_a = m_a; p.m_b = m_b; p.m_l = m_l; p.m_cap = pl.capM;
      p.m_start = m_start + colb[s]; p.m_cnt = m_cnt + colb[s];
      p.blk = 256;
      p.ctr = ctr;
      p.prune_w = E->prune ? wtabf + tabb[s] : nullptr;  // margin set on the device (k_b_prune)
      P2GParams<T>& q = B.p2;
      q.nx = it.nx; q.ny = it.ny; q.R = K[s]; q.kk = B.kk; q.nmax = nmax[s];
      q.wtab = wtab + tabb[s]; q.wtabf = wtabf + tabb[s]; q.reach = nullptr;
      q.m_a = m_a; q.m_b = m_b; q.m_l = m_l;
      q.m_start = m_start + colb[s]; q.m_cnt = m_cnt + colb[s];
      q.o_l = o_l; q.o_r = o_r; q.o_cap = pl.capO;
      q.o_start = o_start + colb[s]; q.o_cnt = o_cnt + colb[s];
      q.blk = 256;
      q.ctr = ctr;
      q.bcap = bcap;
      q.c_start = cst + colb[s]; q.c_af = c_af; q.c_bf = c_bf; q.c_dx = c_dx;
      LvlParams<T>& v = B.lv;
      v.P = q;
      v.l_p = l_p; v.l_cap = pl.capL;
      v.l_idx = l_idx + nlb[s];
      v.W = 2 * K[s] + 1;
      v.slots = E->spill ? lvl_slots_for(K[s]) : lvl_slots_nospill(K[s]);
      v.spill = E->spill;
      v.spill_cap = E->spill ? kBatchSpill : 0;
      v.L = K[s] + 1;
      v.G = v.L <= 32 ? 32 / v.L : 1;
      v.NG = v.L <= 32 ? 0 : (K[s] + 31) / 32;
      v.q0 = 0;
      v.yw = K[s];
      v.nsrc = colb[s + 1] - colb[s];
      v.nlev = nlb[s + 1] - nlb[s];
      v.m_cap = pl.capM;
      v.c_cap = pl.capF;
    }
    // internal outputs (first offset of a closing / opening) sized from the last call of this
    // signature, so that the device checks their capacity and the output write can be part of
    // the recorded sequence (a shape that outgrows its room is written again below)
    bool pre_assigned = false;
    // room in the engine's buffer for every internal output (tot: segments each; margin: room
    // to grow)
    auto assign_mid = [&](const std::vector<long long>& tot, bool margin) -> int {
      size_t need = 0;
      std::vector<long long> cap(ns, 0);
      for (int s = 0; s < ns; ++s) {
        if (!internal[s]) continue;
        cap[s] = std::max<long long>(margin ? tot[s] + tot[s] / 4 + 1024 : tot[s], 1);
        need += bal(sizeof(int) * (colb[s + 1] - colb[s] + 1)) + bal(sizeof(T) * 2 * cap[s]);
      }
      if (need > E->mid_bytes) {
        if (E->mid) cudaFree(E->mid);
        E->mid = nullptr;
        E->mid_bytes = 0;
        if (cudaMalloc(&E->mid, need + need / 4) != cudaSuccess) return DEXEL_ERR_NOMEM;
        E->mid_bytes = need + need / 4;
      }
      size_t o = 0;
      for (int s = 0; s < ns; ++s) {
        if (!internal[s]) continue;
        items[s].out_col_off = (int*)((char*)E->mid + o);
        o += bal(sizeof(int) * (colb[s + 1] - colb[s] + 1));
        items[s].out_z = (char*)E->mid + o;
        items[s].out_cap = cap[s];
        o += bal(sizeof(T) * 2 * cap[s]);
        hs[s].out_col_off = items[s].out_col_off;
        hs[s].out_z = (T*)items[s].out_z;
        hs[s].out_cap = items[s].out_cap;
      }
      return DEXEL_OK;
    };
    if (have_internal) {
      auto lt = E->last_tot.find(sig);
      if (lt != E->last_tot.end() && (int)lt->second.size() == ns) {
        const int rc = assign_mid(lt->second, true);
        if (rc != DEXEL_OK) return rc;
        pre_assigned = true;
      }
    }
    const bool write_in_seq = !have_internal || pre_assigned;
    const size_t up_bytes = sizeof(BShape<T>) * ns + sizeof(long long) * 5 * (ns + 1);
    if (up_bytes > E->host_bytes) {
      if (E->host) cudaFreeHost(E->host);
      E->host = nullptr;
      E->host_bytes = 0;
      if (cudaMallocHost(&E->host, up_bytes) != cudaSuccess) return DEXEL_ERR_NOMEM;
      E->host_bytes = up_bytes;
    }
    // the previous call's upload must be done before the buffer is rewritten
    BK(cudaStreamSynchronize(st));
    memcpy(E->host, hs.data(), sizeof(BShape<T>) * ns);
    long long* hb = (long long*)((char*)E->host + sizeof(BShape<T>) * ns);
    for (int s = 0; s <= ns; ++s) {
      hb[s] = colb[s];
      hb[(ns + 1) + s] = tabb[s];
      hb[2 * (ns + 1) + s] = t1b[s];
      hb[3 * (ns + 1) + s] = t2b[s];
      hb[4 * (ns + 1) + s] = lvb[s];
    }
    BK(cudaMemcpyAsync(dS, E->host, sizeof(BShape<T>) * ns, cudaMemcpyHostToDevice, st));
    BK(cudaMemcpyAsync(dB, hb, sizeof(long long) * 5 * (ns + 1), cudaMemcpyHostToDevice, st));

    // level kernels' geometry
    // per-warp radius tables when the largest reach allows ((R + 1) x 32 floats a warp)
    const bool warp_tab = (long long)(maxK + 1) * 32 * 4 * 8 <= (64LL << 10);
    const int tstride = warp_tab ? (maxK + 1) * 32 : 0;
    const size_t smL = (size_t)lvl_layout(8, 0).total + (size_t)8 * tstride * sizeof(float);
    const int bcapG = 256;
    const size_t smG = (size_t)lgather_smem(8, bcapG);
    const int perG = (int)std::max<long long>(1, std::min<long long>(8, (220LL << 10) / (long long)smG));
    BK(cudaFuncSetAttribute(k_b_levels<T, kTabWarp>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smL));
    BK(cudaFuncSetAttribute(k_b_levels<T, kTabFlat>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smL));
    BK(cudaFuncSetAttribute(k_b_lgather<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smG));
    // ---- the launch sequence (recorded as a graph for a repeated signature)
    const long long nt1 = t1b[ns], nt2 = t2b[ns];
    const int thr = 256;
    auto seq = [&](cudaStream_t s_, long long* nl) -> cudaError_t {
      cudaError_t e;
      if ((e = cudaMemsetAsync(ctr, 0, sizeof(Counters), s_)) != cudaSuccess) return e;
      if ((e = cudaMemsetAsync(d_sst, 0, sizeof(int) * ns, s_)) != cudaSuccess) return e;
      if (ncols > 0)
        k_b_validate<T><<<(unsigned)((ncols + thr - 1) / thr), thr, 0, s_>>>(dS, d_colb, ns, ncols, d_sst);
      if (ntab > 0)
        k_b_tables<T><<<(unsigned)((ntab + thr - 1) / thr), thr, 0, s_>>>(dS, d_tabb, ns, ntab, wtab, wtabf);
      k_b_prune<T><<<(ns + 127) / 128, 128, 0, s_>>>(dS, ns);
      const int per1 = (int)std::max<long long>(1, std::min<long long>(3, (220LL << 10) / sm1));
      const long long want1 = (nt1 + (8 / gw1) - 1) / (8 / gw1);
      const unsigned b1 = (unsigned)std::max<long long>(1, std::min<long long>((long long)E->sms * per1, want1));
      if (nt1 > 0) {
        // one launch per mask width, each taking the shapes of its class
        const long long gstride = sm1 / (8 / gw1);
        if (has_nh[0])
          k_b_pass1<T, 1><<<b1, 256, (size_t)sm1, s_>>>(dS, d_t1b, ns, nt1, ecap, gw1, gstride, d_sst);
        if (has_nh[1])
          k_b_pass1<T, 2><<<b1, 256, (size_t)sm1, s_>>>(dS, d_t1b, ns, nt1, ecap, gw1, gstride, d_sst);
      }
      const long long nb = (ncols + kScanTile - 1) / kScanTile;
      if (ncols > 0) {
        k_scan1<int><<<(unsigned)nb, kScanThreads, 0, s_>>>(ncols, m_cnt, pos, sums);
        k_scan2<<<1, kScanThreads, 0, s_>>>(nb, sums);
        k_mid_pack<Key><<<E->sms * 8, 256, 0, s_>>>(ncols, m_start, m_cnt, m_a, m_b, m_l, pos, sums,
                                                   cst, c_af, c_bf, c_dx, ctr);
      }
      const unsigned b2 = (unsigned)std::max<long long>(1, std::min<long long>((long long)E->sms * minb, nt2));
      if (levels && ncols > 0) {
        if ((e = cudaMemsetAsync(l_idx, 0, sizeof(unsigned long long) * nlev_all, s_)) != cudaSuccess) return e;
        if (warp_tab)
          k_b_levels<T, kTabWarp><<<E->sms * 4, 256, smL, s_>>>(dS, d_lvb, ns, lvb[ns], tstride, d_sst);
        else
          k_b_levels<T, kTabFlat><<<E->sms * 4, 256, smL, s_>>>(dS, d_lvb, ns, lvb[ns], 0, d_sst);
        k_b_lgather<T><<<E->sms * perG, 256, smG, s_>>>(dS, d_colb, ns, ncols, bcapG, d_sst, ctr);
      } else if (nt2 > 0) {
        if (minb == 2)
          k_b_pass2<T, 2><<<b2, wpb2 * 32, (size_t)sm2, s_>>>(dS, d_t2b, ns, nt2, stage_cap,
                                                             kRoundAppends, kRoundPieces, d_sst);
        else
          k_b_pass2<T, 1><<<b2, wpb2 * 32, (size_t)sm2, s_>>>(dS, d_t2b, ns, nt2, stage_cap,
                                                             kRoundAppends, kRoundPieces, d_sst);
      }
      if (ncols > 0) {
        k_b_count<T><<<(unsigned)((ncols + thr - 1) / thr), thr, 0, s_>>>(dS, d_colb, ns, ncols, cnt, d_sst);
        k_scan1<long long><<<(unsigned)nb, kScanThreads, 0, s_>>>(ncols, cnt, pos, sums);
        k_scan2<<<1, kScanThreads, 0, s_>>>(nb, sums);
      }
      k_b_totals<T><<<(ns + 127) / 128, 128, 0, s_>>>(dS, d_colb, ns, ncols, pos, sums, d_tot, d_sst);
      if (nl) *nl += 13;
      if (write_in_seq && ncols > 0) {
        // every output has its room: the write ends the sequence (shapes over capacity, or
        // handed to a redo or the single-shape path, are skipped by it)
        k_b_write<T><<<(unsigned)((ncols + thr - 1) / thr), thr, 0, s_>>>(dS, d_colb, ns, ncols, pos,
                                                                          sums, d_tot, d_sst);
        if (nl) ++*nl;
      }
      return cudaGetLastError();
    };
    BK(cudaFuncSetAttribute(k_b_pass1<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1));
    BK(cudaFuncSetAttribute(k_b_pass1<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1));
    BK(cudaFuncSetAttribute(k_b_pass2<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2));
    BK(cudaFuncSetAttribute(k_b_pass2<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2));
    std::vector<long long> fullsig = sig;
    fullsig.push_back((long long)(size_t)E->ws);
    fullsig.push_back(pl.capM);
    fullsig.push_back(pl.capO);
    fullsig.push_back(sc1);
    fullsig.push_back(sc2);
    fullsig.push_back(levels ? 1 : 0);
    fullsig.push_back(write_in_seq ? 1 : 0);
    auto gi = E->graphs.find(fullsig);
    const bool replay = gi != E->graphs.end();
    if (replay) {
      BK(cudaGraphLaunch(gi->second, st));
      if (launches) *launches += 13 + (write_in_seq ? 1 : 0);
    } else {
      BK(seq(st, launches));
    }
    bool rewrite = false;  // the write must run (again) after the sequence
    Counters hc;
    std::vector<int> hsst(ns);
    std::vector<long long> htot(ns);
    BK(cudaMemcpyAsync(&hc, ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
    BK(cudaMemcpyAsync(hsst.data(), d_sst, sizeof(int) * ns, cudaMemcpyDeviceToHost, st));
    BK(cudaMemcpyAsync(htot.data(), d_tot, sizeof(long long) * ns, cudaMemcpyDeviceToHost, st));
    BK(cudaStreamSynchronize(st));
    E->needM = std::max<long long>(E->needM, (long long)hc.arena_top[1]);
    E->needO = std::max<long long>(E->needO, (long long)hc.arena_top[3]);
    if (levels) E->needL = std::max<long long>(E->needL, (long long)hc.arena_top[2]);
    if (hc.status & ST_OVERFLOW_ARENA) continue;  // grown plan, uncaptured rerun
    if (hc.status & ST_LEVELS_OVER) {
      // level lists beyond their arena (grown next time) or a self-check: this signature
      // reruns with the tiled gather
      if (hc.arena_top[2] <= (unsigned long long)pl.capL) E->no_levels[sig] = true;
      continue;
    }

    if (levels && (hc.status & ST_OVERFLOW_SLOT)) {
      // columns whose lists outgrew the bucket: gathered again with a bucket for their need
      int b = 2 * bcapG;
      while (b < hc.max_state && b < 8192) b <<= 1;
      if (b >= hc.max_state) {
        int warps = 8;
        while (warps > 1 && warps * lgather_smem(1, b) > (110LL << 10)) warps >>= 1;
        const size_t smR = (size_t)lgather_smem(warps, b);
        BK(cudaFuncSetAttribute(k_b_lgather_redo<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smR));
        k_b_lgather_redo<T><<<E->sms * 2, warps * 32, smR, st>>>(dS, d_colb, ns, ncols, b, d_sst);
        BK(cudaGetLastError());
        // count again (the first count saw the redone columns as marked)
        for (int q = 0; q < ns; ++q) hsst[q] &= ~BS_REDO;
        BK(cudaMemcpyAsync(d_sst, hsst.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, st));
        const long long nb = (ncols + kScanTile - 1) / kScanTile;
        k_b_count<T><<<(unsigned)((ncols + thr - 1) / thr), thr, 0, st>>>(dS, d_colb, ns, ncols, cnt, d_sst);
        k_scan1<long long><<<(unsigned)nb, kScanThreads, 0, st>>>(ncols, cnt, pos, sums);
        k_scan2<<<1, kScanThreads, 0, st>>>(nb, sums);
        k_b_totals<T><<<(ns + 127) / 128, 128, 0, st>>>(dS, d_colb, ns, ncols, pos, sums, d_tot, d_sst);
        BK(cudaGetLastError());
        if (launches) *launches += 5;
        rewrite = true;
        BK(cudaMemcpyAsync(&hc, ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
        BK(cudaMemcpyAsync(hsst.data(), d_sst, sizeof(int) * ns, cudaMemcpyDeviceToHost, st));
        BK(cudaMemcpyAsync(htot.data(), d_tot, sizeof(long long) * ns, cudaMemcpyDeviceToHost, st));
        BK(cudaStreamSynchronize(st));
        if (hc.status & ST_OVERFLOW_ARENA) continue;
      }
    }
    // autotuning of the tile scales: the first call of a signature times both passes at the
    // three scales (a rerun of the whole sequence per candidate) and keeps the fastest
    if (E->autotune && sc_it == E->scales.end() && depth == 0) {
      cudaEvent_t a, b;
      BK(cudaEventCreate(&a));
      BK(cudaEventCreate(&b));
      float best = 1e30f;
      int b1s = 1, b2s = 1;
      for (int c1 = 0; c1 < 3; ++c1) {
        for (int c2 = 0; c2 < 3; ++c2) {
          if (c1 != 1 && c2 != 1) continue;  // one pass varied at a time
          tiles(c1, c2);
          E->scales[sig] = {c1, c2};
          std::vector<int> st2;
          std::vector<long long> ns2;
          BK(cudaEventRecord(a, st));
          const int rc = batch_run_t<T>(E, items, st, st2, ns2, nullptr, 1);
          BK(cudaEventRecord(b, st));
          BK(cudaEventSynchronize(b));
          float ms = 0;
          BK(cudaEventElapsedTime(&ms, a, b));
          if (rc == DEXEL_OK && ms < best) { best = ms; b1s = c1; b2s = c2; }
        }
      }
      cudaEventDestroy(a);
      cudaEventDestroy(b);
      E->scales[sig] = {b1s, b2s};
      return batch_run_t<T>(E, items, st, status, nseg, launches, 1);
    }

    // internal outputs without room yet (first call of a signature) or beyond the room of the
    // last call's totals: space from the engine, then the write
    if (have_internal) {
      bool regrow = !pre_assigned;
      for (int s = 0; s < ns; ++s)
        if (internal[s] && (hsst[s] & BS_CAP)) regrow = true;
      if (regrow) {
        BK(cudaStreamSynchronize(st));
        const int rc = assign_mid(htot, false);
        if (rc != DEXEL_OK) return rc;
        for (int s = 0; s < ns; ++s)
          if (internal[s]) hsst[s] &= ~BS_CAP;
        memcpy(E->host, hs.data(), sizeof(BShape<T>) * ns);
        BK(cudaMemcpyAsync(dS, E->host, sizeof(BShape<T>) * ns, cudaMemcpyHostToDevice, st));
        BK(cudaMemcpyAsync(d_sst, hsst.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, st));
        rewrite = true;
      }
    }
    if ((rewrite || !write_in_seq) && ncols > 0) {
      k_b_write<T><<<(unsigned)((ncols + thr - 1) / thr), thr, 0, st>>>(dS, d_colb, ns, ncols, pos,
                                                                        sums, d_tot, d_sst);
      if (launches) ++*launches;
      BK(cudaGetLastError());
    }
    E->last_tot[sig] = htot;
    // record the sequence for the next call with this signature (recording does not run it)
    if (!replay) {
      if (!E->cap_stream) BK(cudaStreamCreateWithFlags(&E->cap_stream, cudaStreamNonBlocking));
      if (E->graphs.size() >= 16) {  // bounded cache
        for (auto& g : E->graphs) cudaGraphExecDestroy(g.second);
        E->graphs.clear();
      }
      cudaGraph_t g = nullptr;
      BK(cudaStreamBeginCapture(E->cap_stream, cudaStreamCaptureModeThreadLocal));
      const cudaError_t ce = seq(E->cap_stream, nullptr);
      const cudaError_t ee = cudaStreamEndCapture(E->cap_stream, &g);
      if (ce == cudaSuccess && ee == cudaSuccess && g) {
        cudaGraphExec_t ex = nullptr;
        if (cudaGraphInstantiate(&ex, g, 0) == cudaSuccess) E->graphs[fullsig] = ex;
      }
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
    }
    for (int s = 0; s < ns; ++s) {
      nseg[s] = htot[s];
      if (hsst[s] & BS_BAD) status[s] = DEXEL_ERR_BAD_CSR;
      else if (hsst[s] & (BS_REDO | BS_SWEEP)) status[s] = 1;  // the single-shape path
      else if (hsst[s] & BS_CAP) status[s] = DEXEL_ERR_CAPACITY;
    }
    return DEXEL_OK;
  }
#undef BK
  for (int s = 0; s < ns; ++s) status[s] = 1;
  return DEXEL_OK;
}

int batch_run(BatchEngine* E, int fp32, std::vector<BatchItem>& items, cudaStream_t st,
              std::vector<int>& status, std::vector<long long>& nseg, long long* launches) {
  if (!E) return DEXEL_ERR_INVALID_ARG;
  return fp32 ? batch_run_t<float>(E, items, st, status, nseg, launches, 0)
              : batch_run_t<double>(E, items, st, status, nseg, launches, 0);
}

}  // namespace dexel
