// Pass-1 window gather kernel (the formulation and the per-tile body are in pass1g.cuh).
#include "launch.h"
#include "pass1g.cuh"

namespace dexel {

template <typename T, int NW>
__global__ void __launch_bounds__(256) k_pass1g(P1Params<T> P, int tc, int ecap, int obuf) {
  extern __shared__ __align__(16) unsigned char smem[];
  const long long ntiles = (long long)P.ny * ((P.nx + tc - 1) / tc);
  ArenaCursor cur{0, 0};
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
    pass1g_tile<T, NW>(P, tile, tc, ecap, obuf, smem, cur);
  if ((threadIdx.x & 31) == 0 && cur.tally > 0) {
    add_total(&P.ctr->mid_total, cur.tally);
    note_max(&P.ctr->max_pieces, cur.tmax);
  }
}

template <typename T>
cudaError_t launch_pass1g(const P1Params<T>& P, int tc, int ecap, int obuf, int blocks,
                          cudaStream_t st) {
  const size_t smem = (size_t)pass1g_smem<T>(tc, P.K, ecap, obuf);
  const int nw = mask_words(P.K);
  auto kern = nw == 1 ? k_pass1g<T, 1> : (nw == 2 ? k_pass1g<T, 2> : k_pass1g<T, 4>);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<blocks, 256, smem, st>>>(P, tc, ecap, obuf);
  return cudaGetLastError();
}

template <typename T>
long long pass1g_smem(int tc, int R, int ecap, int obuf) {
  long long a, b;
  return p1g_layout<T>(tc, R, ecap, obuf, 8, &a, &b);
}

template cudaError_t launch_pass1g<float>(const P1Params<float>&, int, int, int, int, cudaStream_t);
template cudaError_t launch_pass1g<double>(const P1Params<double>&, int, int, int, int, cudaStream_t);
template long long pass1g_smem<float>(int, int, int, int);
template long long pass1g_smem<double>(int, int, int, int);

}  // namespace dexel
