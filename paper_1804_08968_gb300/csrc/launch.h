// Internal launch wrappers shared by the translation units of libdexel.
#pragma once
#include <cuda_runtime.h>
#include "gather2.cuh"

namespace dexel {

constexpr int kWarpsPerBlock = 4;

template <typename T>
cudaError_t launch_pass1(const P1Params<T>& P, int blocks, cudaStream_t st);
template <typename T>
cudaError_t launch_pass2(const P2Params<T>& P, int blocks, cudaStream_t st);
template <typename T>
cudaError_t launch_pass2g(const P2GParams<T>& P, int blocks, cudaStream_t st);
long long pass2g_smem(int warps, int stcap, int bcap, int tile, int R, int stage_cap);
template <typename T>
cudaError_t launch_pass2r(const P2GParams<T>& P, int G, int blocks, cudaStream_t st);
long long pass2r_smem(int warps, int G, int bcap);


}  // namespace dexel
