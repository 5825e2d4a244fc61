// observable.h - run-time compiled stream averages (internal interface of observable.cu).
#pragma once
#include <cuda_runtime.h>

#include <string>

namespace twa {

struct ObsProgram;

// Compiles f = f_re + i f_im for the current device, evaluated in FP64 (sums in FP64) or, with
// fp32, in FP32 (sums over the streams as float pairs).  Returns 0, -1 (the expression is rejected
// or does not compile; msg holds the reason or the compiler log) or -3 (NVRTC or CUDA unavailable).
int obs_compile(const char* f_re, const char* f_im, bool fp32, ObsProgram** out, std::string* msg);
void obs_free(ObsProgram* p);

// One averaging pass over an instance (slot 0 classical, slots 1.. sampled; values scaled by
// `scale` before f), then total = w * (sum over cells of per_cell).  per_cell and f_cl may be null
// (2 * cells doubles each otherwise); part holds 2 * max_blocks doubles; total 2 doubles.
int obs_launch(const ObsProgram* p, bool f64, const void* psi, long long cells, int n_slots, int of_mean,
               double scale, const int* n3, double* per_cell, double* f_cl, double* part, int max_blocks, double w,
               double* total, cudaStream_t st, std::string* msg);

}  // namespace twa
