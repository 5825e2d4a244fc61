// reduce.cuh - fixed-order block reduction used by the moment kernels (bitwise reproducible).
#pragma once
#include <cuda_runtime.h>

namespace twa {

// Tree reduction of NP doubles over a 256-thread block into part[blockIdx.x * NP + j].
template <int NP>
__device__ __forceinline__ void block_reduce_store(double (&v)[NP], double* part) {
    __shared__ double red[NP][256];
#pragma unroll
    for (int j = 0; j < NP; ++j) red[j][threadIdx.x] = v[j];
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
#pragma unroll
            for (int j = 0; j < NP; ++j) red[j][threadIdx.x] += red[j][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int j = 0; j < NP; ++j) part[(long long)blockIdx.x * NP + j] = red[j][0];
    }
}

}  // namespace twa
