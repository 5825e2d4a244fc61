// batch.cu - one persistent launch over the split steps of every instance of a 2D batch.
//
// The realizations of the stream ensemble evolve independently (Sec. III.A), and a batch may hold
// instances of different grid sizes.  Instead of one launch per pass and instance, a persistent
// kernel walks a work list: for each KDK step, each of the four passes of the 2D pipeline
// (x rows: kick + drift_x; y columns: drift_y + packed density + FFT_y; x rows: FFT_x, Poisson,
// iFFT_x; y columns: iFFT_y), each instance, each pair of slots and each tile of lines.  Items are
// handed out in that order by an atomic ticket; an item of a pair may start once every tile of the
// pair's earlier passes is done, which a per-pair counter of finished tiles records.  So the passes
// of different pairs and instances overlap instead of draining the GPU at every pass boundary.
//
// Every item's dependencies carry smaller tickets, and a CTA takes a ticket only while it runs, so
// the oldest unfinished item can always proceed: the launch needs no co-residency guarantee.  Waits
// are bounded: a CTA that has waited longer than the handle's limit (clock64 cycles) sets
// TWA_ETIMEOUT in the device error word and an abort flag that makes every other CTA stop taking
// work and leave its own wait; the batch's fields are then undefined, the GPU stays usable.
#include <cuda_runtime.h>

#include "batch.h"
#include "passes.cuh"

namespace twa {
namespace {

constexpr int kThreads = BATCH_THREADS;

template <int N>
__host__ __device__ constexpr int lines_of() { return kThreads / Plan<N>::T; }

// Dynamic shared memory of one variant, as the stand-alone pass kernels size it.
template <int N, bool STR, int OP>
constexpr size_t smem_of() {
    return (size_t)TileSmem<N, lines_of<N>(), STR, OP, false>::total * sizeof(float2);
}

// One variant per (length, pass of the 2D pipeline), each compiled as a function of its own so its
// registers are allocated for it alone (inlined into one switch they spilled).
template <int N, int Q>
__device__ __noinline__ void run_variant(const PassArgs& a, int tile, int f, float2* smem) {
    constexpr int L = lines_of<N>();
    if constexpr (Q == 0) line_tile<N, L, false, OP_KICK_DRIFT>(a, tile, f, smem);
    else if constexpr (Q == 1) line_tile<N, L, true, OP_DRIFT_RHO>(a, tile, f, smem);
    else if constexpr (Q == 2) line_tile<N, L, false, OP_FWD_MUL_INV>(a, tile, f, smem);
    else line_tile<N, L, true, OP_INV>(a, tile, f, smem);
}

template <int N>
__device__ __forceinline__ void run_pass_n(int q, const PassArgs& a, int tile, int f, float2* smem) {
    switch (q) {
        case 0: run_variant<N, 0>(a, tile, f, smem); break;
        case 1: run_variant<N, 1>(a, tile, f, smem); break;
        case 2: run_variant<N, 2>(a, tile, f, smem); break;
        default: run_variant<N, 3>(a, tile, f, smem); break;
    }
}

// The item kinds: (length index) * 4 + (pass of the 2D pipeline).
__device__ __forceinline__ void run_kind(int kind, const PassArgs& a, int tile, int f, float2* smem) {
    switch (kind >> 2) {
        case 0: run_pass_n<256>(kind & 3, a, tile, f, smem); break;
        case 1: run_pass_n<512>(kind & 3, a, tile, f, smem); break;
        case 2: run_pass_n<1024>(kind & 3, a, tile, f, smem); break;
        default: run_pass_n<2048>(kind & 3, a, tile, f, smem); break;
    }
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Thread 0: wait until *c >= target, the abort flag is raised, or `budget` cycles have passed.
// Returns 1 when the dependency is met.
__device__ int wait_counter(const unsigned* c, unsigned target, const int* abort_flag, long long budget) {
    if (ld_acquire(c) >= target) return 1;
    const long long t0 = clock64();
    for (;;) {
        __nanosleep(200);
        if (ld_acquire(c) >= target) return 1;
        if (ld_relaxed(abort_flag)) return 0;
        if (clock64() - t0 > budget) return -1;
    }
}

__global__ void __launch_bounds__(kThreads, 2)
k_batch(const BatchPass* __restrict__ passes, int n_passes, const PassArgs* __restrict__ args,
        unsigned* counters, unsigned long long* ticket, long long n_items, int* err_word, int* abort_flag,
        long long budget) {
    extern __shared__ __align__(16) float2 smem[];
    __shared__ long long s_item;
    __shared__ int s_ok;
    // the item's pass arguments, read by every thread many times: kept in shared memory
    __shared__ __align__(16) PassArgs s_args;
    for (;;) {
        if (threadIdx.x == 0) {
            const long long it = (long long)atomicAdd(ticket, 1ull);
            s_item = (it < n_items && !ld_relaxed(abort_flag)) ? it : -1;
        }
        __syncthreads();
        const long long it = s_item;
        if (it < 0) return;
        // the pass entry holding this ticket (entries are sorted by their first ticket)
        int lo = 0, hi = n_passes - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (passes[mid].first <= it) lo = mid;
            else hi = mid - 1;
        }
        const BatchPass& P = passes[lo];
        const long long r = it - P.first;
        const int f = (int)(r / P.items), c = (int)(r % P.items);
        const int t0 = c * P.per_item, t1 = min(t0 + P.per_item, P.tiles);
        unsigned* ctr = counters + P.ctr + f;
        if (threadIdx.x == 0) {
            const int w = wait_counter(ctr, (unsigned)P.target, abort_flag, budget);
            if (w < 0) {
                atomicOr(err_word, TWA_ERR_TIMEOUT_BIT);
                atomicExch(abort_flag, 1);
            }
            s_ok = w > 0;
        }
        if (threadIdx.x < (int)(sizeof(PassArgs) / 4))
            reinterpret_cast<int*>(&s_args)[threadIdx.x] = reinterpret_cast<const int*>(args + P.args)[threadIdx.x];
        __syncthreads();
        if (!s_ok) return;
        for (int tile = t0; tile < t1; ++tile) {
            run_kind(P.kind, s_args, tile, f, smem);
            __syncthreads();  // the exchange buffers are free for the next tile
        }
        // every thread's stores of these tiles are issued before the counter moves
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(ctr, (unsigned)(t1 - t0));
        }
    }
}

size_t kind_smem(int kind) {
    const int q = kind & 3;
    switch (kind >> 2) {
#define TWA_SM(I, N)                                                                      \
    case I:                                                                                \
        return q == 0 ? smem_of<N, false, OP_KICK_DRIFT>() : q == 1 ? smem_of<N, true, OP_DRIFT_RHO>() \
               : q == 2 ? smem_of<N, false, OP_FWD_MUL_INV>() : smem_of<N, true, OP_INV>();
        TWA_SM(0, 256)
        TWA_SM(1, 512)
        TWA_SM(2, 1024)
        TWA_SM(3, 2048)
#undef TWA_SM
        default: return 0;
    }
}

}  // namespace

int batch_kind(int n, int pass) {
    int idx;
    switch (n) {
        case 256: idx = 0; break;
        case 512: idx = 1; break;
        case 1024: idx = 2; break;
        case 2048: idx = 3; break;
        default: return -1;
    }
    return pass < 0 || pass > 3 ? -1 : idx * 4 + pass;
}

int batch_lines(int n) { return kThreads / plan_threads_per_line(n); }

int launch_batch(const BatchPass* passes, int n_passes, const PassArgs* args, unsigned* counters,
                 unsigned long long* ticket, long long n_items, int* err_word, int* abort_flag, long long budget,
                 const int* kinds, int n_kinds, cudaStream_t st) {
    size_t smem = 0;
    for (int i = 0; i < n_kinds; ++i) smem = kind_smem(kinds[i]) > smem ? kind_smem(kinds[i]) : smem;
    static size_t smem_set = 0;
    static int ctas = 0;
    if (smem > smem_set || ctas == 0) {
        if (cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return -3;
        smem_set = smem > smem_set ? smem : smem_set;
        int per_sm = 0, sms = 0, dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch, kThreads, smem_set);
        ctas = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
    }
    const long long g = n_items < ctas ? n_items : ctas;
    if (g <= 0) return 0;
    k_batch<<<(unsigned)g, kThreads, smem_set, st>>>(passes, n_passes, args, counters, ticket, n_items, err_word,
                                                      abort_flag, budget);
    return 0;
}

}  // namespace twa
