// batch.h - persistent batch launch over the 2D split-step passes (internal header).
#pragma once
#include <cuda_runtime.h>

#include "passes.cuh"

namespace twa {

constexpr int BATCH_THREADS = 256;       // threads of every CTA of the persistent launch (two per SM)

// One (step, pass, instance) entry of the work list.  Its items are tickets first .. first +
// fields * items - 1; item r covers tiles [c * per_item, min((c + 1) * per_item, tiles)) of field
// f = r / items, c = r % items (a few tiles per ticket keep the per-item bookkeeping small).  An item
// of field f waits until counters[ctr + f] (tiles of that pair finished so far in this launch)
// reaches target.
struct BatchPass {
    long long first;
    int kind;      // batch_kind(N, pass)
    int tiles;     // tiles per field
    int per_item;  // tiles per item
    int items;     // items per field
    int fields;    // pairs of the instance
    int args;      // index of the PassArgs of this pass
    int ctr;       // first counter of the instance (one per pair)
    int target;    // tiles of the pair's earlier passes in this launch
};

// Item kind of pass `pass` (0: x rows kick + drift, 1: y columns drift + density + FFT, 2: x rows
// FFT + Poisson + iFFT, 3: y columns iFFT) on lines of length n; -1 if the persistent kernel has no
// variant for n (lengths 256 to 2048).
int batch_kind(int n, int pass);
// Lines per tile at length n (BATCH_THREADS / threads per line).
int batch_lines(int n);
// Launch the persistent kernel (one CTA per resident slot, at most n_items CTAs).  counters, *ticket
// and *abort_flag must be zero.  budget: the longest wait in clock64 cycles.
int launch_batch(const BatchPass* passes, int n_passes, const PassArgs* args, unsigned* counters,
                 unsigned long long* ticket, long long n_items, int* err_word, int* abort_flag, long long budget,
                 const int* kinds, int n_kinds, cudaStream_t st);

}  // namespace twa
