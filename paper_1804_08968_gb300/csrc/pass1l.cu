// Pass-1 kernel with one lane per output column (the formulation and the per-tile body are
// in pass1l.cuh).
#include <algorithm>

#include "launch.h"
#include "pass1l.cuh"

namespace dexel {

constexpr int kP1LWarps = 8;

// the block's warps in groups of gw (1, 2, 4, 8), each group its own tiles and shared memory;
// MINB: blocks an SM the registers are planned for (3: 80 registers a thread, with some
// spilled; 2: up to 128, none spilled), taken from the blocks the shared memory leaves room for
template <typename T, int NH, int MINB>
__global__ void __launch_bounds__(256, MINB) k_pass1l(P1Params<T> P, int ecap, int gw) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5;
  const int groups = (blockDim.x >> 5) / gw;
  const TGroup G{gw, warp / gw, warp % gw, (int)threadIdx.x % (gw * 32),
                 (long long)blockIdx.x * groups + warp / gw};
  unsigned char* gsm =
      smem + (long long)G.gid * p1l_layout(P.K, ecap, gw, (int)sizeof(typename EvK<T>::type), P.nbuf).total;
  if (*(volatile int*)&P.ctr->status & ST_BAD_CSR) return;  // (stream-ordered calls: no plan for a bad input)
  if (P.redo && *(volatile int*)&P.ctr->p1_marked == 0) return;  // (a redo with nothing marked)
  const int xw = P.xb > 0 ? P.xb - P.xa : P.nx;  // the block of columns
  const long long ntiles = (long long)P.ny * ((xw + 31) >> 5);
  ArenaCursor cur{0, 0};
  for (long long tile = (long long)blockIdx.x * groups + G.gid; tile < ntiles;
       tile += (long long)gridDim.x * groups)
    pass1l_tile<T, NH>(P, tile, ecap, gsm, G, cur);
  if (G.gtid == 0 && cur.tally > 0) {
    add_total(&P.ctr->mid_total, cur.tally);
    note_max(&P.ctr->max_pieces, cur.tmax);
  }
}

long long pass1l_smem(int R, int ecap, int gw, int ksz, int nbuf) {
  return p1l_layout(R, ecap, gw, ksz, nbuf).total * (kP1LWarps / gw);
}

int pass1l_blocks(int nx, int ny, int R, int ecap, int gw, int sms, int ksz, int nbuf) {
  const long long smem = pass1l_smem(R, ecap, gw, ksz, nbuf);
  const long long ntiles = (long long)ny * ((nx + 31) >> 5);
  const int groups = kP1LWarps / gw;
  const int per_sm = (int)std::max<long long>(1, std::min<long long>(3, (220LL << 10) / smem));
  const long long want = (ntiles + groups - 1) / groups;
  return (int)std::max<long long>(1, std::min<long long>((long long)sms * per_sm, want));
}

template <typename T>
cudaError_t launch_pass1l(const P1Params<T>& P, int ecap, int gw, int sms, cudaStream_t st) {
  if (gw != 1 && gw != 2 && gw != 4 && gw != 8) return cudaErrorInvalidValue;
  const int ksz = (int)sizeof(typename EvK<T>::type);
  const size_t smem = (size_t)pass1l_smem(P.K, ecap, gw, ksz, P.nbuf);
  if (smem > (220u << 10) || P.K > kLaneMaxReach1) return cudaErrorInvalidValue;
  const bool three = (220LL << 10) / (long long)smem >= 3;  // three blocks an SM fit
  auto kern = P.K <= 64 ? (three ? k_pass1l<T, 1, 3> : k_pass1l<T, 1, 2>)
                        : (three ? k_pass1l<T, 2, 3> : k_pass1l<T, 2, 2>);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // the grid the ring (when given) was sized for: pass1l_blocks threads x r_cap pieces
  const int blocks = pass1l_blocks(P.nx, P.ny, P.K, ecap, gw, sms, ksz, P.nbuf);  // (sized for whole rows)
  kern<<<blocks, kP1LWarps * 32, smem, st>>>(P, ecap, gw);
  return cudaGetLastError();
}

template cudaError_t launch_pass1l<float>(const P1Params<float>&, int, int, int, cudaStream_t);
template cudaError_t launch_pass1l<double>(const P1Params<double>&, int, int, int, cudaStream_t);

}  // namespace dexel
