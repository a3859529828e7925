// Pass 2 kernel: persistent warps take (column line, chunk) work items and run the
// forward/backward rectangle + power-diagram sweeps of sweep2.cuh (Sec. 3.3).
#include "launch.h"

namespace dexel {

template <typename T>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_pass2(P2Params<T> P) {
  const Lanes L{(int)(threadIdx.x & 31), 32};
  const long long gw = (long long)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  typedef typename H<T>::K Key;
  const P2Slot<Key> W =
      p2_slot<Key>(P.slots + gw * P.slot_bytes, P.capP, P.capR, P.capA, P.capS, P.chunk);
  ArenaCursor cf{0, 0}, co{0, 0};
  const int nitems = P.nx * P.nchunks;
  for (;;) {
    int item = 0;
    if (L.lane == 0) item = (int)atomicAdd(&P.ctr->work_next[1], 1ULL);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= nitems) break;
    const int i = item / P.nchunks;
    const int c = item % P.nchunks;
    const int c0 = c * P.chunk;
    const int c1 = min(P.ny, c0 + P.chunk);
    if (c0 >= c1) continue;
    pass2_item<T>(L, P, W, i, c0, c1, cf, co);
  }
}

template <typename T>
cudaError_t launch_pass2(const P2Params<T>& P, int blocks, cudaStream_t st) {
  k_pass2<T><<<blocks, kWarpsPerBlock * 32, 0, st>>>(P);
  return cudaGetLastError();
}

template cudaError_t launch_pass2<float>(const P2Params<float>&, int, cudaStream_t);
template cudaError_t launch_pass2<double>(const P2Params<double>&, int, cudaStream_t);

}  // namespace dexel
