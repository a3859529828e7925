// Pass 1 kernel: persistent warps take (row, chunk) work items from a queue and run the
// forward/backward extrusion sweeps of sweep.cuh (Sec. 3.3 "3D Dilation").
#include "launch.h"

namespace dexel {

template <typename T>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_pass1(P1Params<T> P) {
  const Lanes L{(int)(threadIdx.x & 31), 32};
  const long long gw = (long long)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  typedef typename H<T>::K Key;
  const P1Slot<Key> W = p1_slot<Key>(P.slots + gw * P.slot_bytes, P.capF, P.capS, P.chunk);
  ArenaCursor cf{0, 0}, cm{0, 0};
  const int nitems = (P.rows ? P.nrows : P.ny) * P.nchunks;
  for (;;) {
    int item = 0;
    if (L.lane == 0) item = (int)atomicAdd(&P.ctr->work_next[0], 1ULL);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= nitems) break;
    const int j = P.rows ? P.rows[item / P.nchunks] : item / P.nchunks;
    const int c = item % P.nchunks;
    const int c0 = c * P.chunk;
    const int c1 = min(P.nx, c0 + P.chunk);
    if (c0 >= c1) continue;
    pass1_item<T>(L, P, W, j, c0, c1, cf, cm);
  }
}

template <typename T>
cudaError_t launch_pass1(const P1Params<T>& P, int blocks, cudaStream_t st) {
  k_pass1<T><<<blocks, kWarpsPerBlock * 32, 0, st>>>(P);
  return cudaGetLastError();
}

template cudaError_t launch_pass1<float>(const P1Params<float>&, int, cudaStream_t);
template cudaError_t launch_pass1<double>(const P1Params<double>&, int, cudaStream_t);

}  // namespace dexel
