// Internal launch wrappers shared by the translation units of libdexel.
#pragma once
#include <cuda_runtime.h>
#include "sweep2.cuh"

namespace dexel {

constexpr int kWarpsPerBlock = 4;

template <typename T>
cudaError_t launch_pass1(const P1Params<T>& P, int blocks, cudaStream_t st);
template <typename T>
cudaError_t launch_pass2(const P2Params<T>& P, int blocks, cudaStream_t st);

}  // namespace dexel
