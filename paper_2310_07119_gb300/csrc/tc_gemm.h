// tc_gemm.h - tensor-core (tcgen05, TF32) GEMM of tall-skinny FP32 matrices (internal header).
#pragma once
#include <cuda_runtime.h>

namespace twa {

constexpr int TC_ERR_TIMEOUT_BIT = 4;  // error word bit: a bounded wait of the tensor-core GEMM gave up

// Shapes the kernel takes: K a multiple of 32 up to 128 (whole 128-byte swizzle rows of FP32), the
// padded column count Np a multiple of 16 in [16, 256], and two 128-row A tiles plus the Np-row B tile
// within 227 KB of shared memory (Np <= 192 at K = 128).
bool tc_gemm_supported(long long K, int Np);

// C[p][j] (+)= sum_k A[p][k] Bt[j][k] for p < P, j < N: A row-major with row stride lda floats, Bt
// [Np][K] row-major (rows N..Np-1 zero), C row stride ldc floats.  TF32 products, FP32 sums.  A and
// Bt 16-byte aligned, lda * 4 a multiple of 16.  Asynchronous on st; a wait that runs out sets
// TC_ERR_TIMEOUT_BIT in *err (device int).  Returns 0, or -1 (shape), -2 (no tensor-map encoder),
// -3 (launch).
int tc_gemm(const float* A, long long P, long long K, long long lda, const float* Bt, int N, int Np, float* C,
            long long ldc, int accumulate, int* err, double wait_s, cudaStream_t st);

}  // namespace twa
