// tc_gemm.cu - C[P][N] (+)= A[P][K] B[N][K]^T on the fifth-generation tensor cores: TF32 operands read
// from shared memory, FP32 accumulation in tensor memory (tcgen05), tiles moved by TMA.
//
// Used by the surrogate for the contractions along the contiguous axis of its truncated DFT: the
// forward transform of a real field (A = rows of n cells, B = the (re, im) rows of the 2m retained
// DFT rows, C = interleaved complex coefficients) and the real part of the adjoint (A = rows of 2m
// complex coefficients as 4m reals, B = (Re M, -Im M) columns, C = n cells).  Both are tall-skinny
// GEMMs (P up to ~10^7 rows, N and K <= 128) bound by the streaming of A, so one CTA per SM walks row
// tiles with a double-buffered TMA pipeline while the tensor core and the epilogue work on the
// previous tile.
//
// Per CTA (128 threads): thread 0 issues the TMA copies and the MMAs; all four warps read the
// accumulator out of tensor memory (warp w owns rows 32w..32w+31 of the 128-row tile) and store it.
// Operands sit in shared memory in the 128-byte swizzled K-major layout TMA writes: a tile of R rows
// and K = 32 a floats is a atoms of R x 128 bytes; each MMA consumes K = 8 (32 bytes) of one atom.
// Every wait is bounded (clock64): on time-out the CTA records an error bit, waits (bounded) for its
// copies in flight, releases its tensor memory and returns.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "tc_gemm.h"
#include "tma.cuh"

namespace twa {
namespace {

constexpr int BM = 128;           // rows per tile (MMA M)
constexpr int ATOM_F = 32;        // floats per 128-byte swizzle row
constexpr int THREADS = 128;


// Shared-memory matrix descriptor: 128-byte swizzle, K-major, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);     // start address (16-byte units)
    d |= (uint64_t)1u << 16;                      // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024u >> 4) << 32;            // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1u << 46;                      // descriptor version
    d |= (uint64_t)2u << 61;                      // layout: 128-byte swizzle
    return d;
}

// Instruction descriptor of kind::tf32: F32 accumulator, TF32 A and B, both K-major, N x M = n x 128.
__device__ __forceinline__ uint32_t idesc_tf32(int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// 16 consecutive accumulator columns of this thread's row.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&r)[16]) {
    uint32_t u[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
        "[%16];"
        : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]), "=r"(u[8]),
          "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) r[i] = __uint_as_float(u[i]);
}

__global__ void __launch_bounds__(THREADS, 1)
k_tc_gemm(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, float* __restrict__ C,
          long long P, int N, int Kp, int Np, long long ldc, int accumulate, int ncols, int* err, long long budget) {
    extern __shared__ __align__(1024) uint8_t sraw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(sraw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t bar_a[2], bar_b, bar_mma;
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;
    const int natoms = Kp / ATOM_F;
    const uint32_t a_bytes = (uint32_t)natoms * BM * 128, b_bytes = (uint32_t)natoms * Np * 128;
    uint8_t* sA[2] = {sm, sm + a_bytes};
    uint8_t* sB = sm + 2 * a_bytes;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long ntiles = (P + BM - 1) / BM;

    if (threadIdx.x == 0) {
        s_fail = 0;
        mbar_init(smem_u32(&bar_a[0]), 1);
        mbar_init(smem_u32(&bar_a[1]), 1);
        mbar_init(smem_u32(&bar_b), 1);
        mbar_init(smem_u32(&bar_mma), 1);
        mbar_init_fence();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = idesc_tf32(Np);

    auto load_a = [&](long long tile, int buf) {
        mbar_expect_tx(smem_u32(&bar_a[buf]), a_bytes);
        for (int k = 0; k < natoms; ++k)
            tma_load_2d(smem_u32(sA[buf] + (size_t)k * BM * 128), &ta, k * ATOM_F, (int)(tile * BM), smem_u32(&bar_a[buf]));
    };
    if (threadIdx.x == 0) {
        mbar_expect_tx(smem_u32(&bar_b), b_bytes);
        for (int k = 0; k < natoms; ++k) tma_load_2d(smem_u32(sB + (size_t)k * Np * 128), &tb, k * ATOM_F, 0, smem_u32(&bar_b));
        if ((long long)blockIdx.x < ntiles) load_a(blockIdx.x, 0);
    }
    int issued = 0, used = 0;  // A tiles copied / consumed by this CTA (thread 0's count)
    bool b_done = false;
    if (threadIdx.x == 0 && (long long)blockIdx.x < ntiles) issued = 1;

    int i = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
        const int buf = i & 1;
        if (threadIdx.x == 0) {
            const long long next = tile + gridDim.x;
            // the other buffer was read by the previous tile's MMAs, complete before its epilogue
            if (next < ntiles) {
                load_a(next, buf ^ 1);
                ++issued;
            }
            bool ok = true;
            if (i == 0) ok = b_done = mbar_wait(smem_u32(&bar_b), 0, budget);
            ok = ok && mbar_wait(smem_u32(&bar_a[buf]), (uint32_t)((i >> 1) & 1), budget);
            if (ok) {
                ++used;
                fence_after();
                const uint32_t a0 = smem_u32(sA[buf]), b0 = smem_u32(sB);
                for (int s = 0; s < Kp / 8; ++s) {
                    const uint32_t koff = (uint32_t)(s % 4) * 32u;  // K = 8 TF32 values = 32 bytes
                    const uint64_t ad = sw128_desc(a0 + (uint32_t)(s / 4) * BM * 128 + koff);
                    const uint64_t bd = sw128_desc(b0 + (uint32_t)(s / 4) * (uint32_t)Np * 128 + koff);
                    mma_tf32(tmem, ad, bd, idesc, s > 0 ? 1u : 0u);
                }
                mma_commit(smem_u32(&bar_mma));
            } else {
                s_fail = 1;
            }
        }
        __syncthreads();
        if (s_fail) break;
        if (!mbar_wait(smem_u32(&bar_mma), (uint32_t)(i & 1), budget)) {
            atomicOr(&s_fail, 1);
        }
        __syncthreads();
        if (s_fail) break;
        fence_after();
        // epilogue: row r of the tile -> TMEM lane r; warp w reads lanes 32w..32w+31
        const long long row = tile * BM + warp * 32 + lane;
        float* crow = C + row * ldc;
        const bool vec = (N % 16) == 0 && (ldc % 4) == 0 && ((reinterpret_cast<uintptr_t>(C) & 15u) == 0);
        for (int c0 = 0; c0 < Np; c0 += 16) {
            float r[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
            if (row < P) {
                if (vec) {
                    float4* c4 = reinterpret_cast<float4*>(crow + c0);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        float4 o = make_float4(r[4 * j], r[4 * j + 1], r[4 * j + 2], r[4 * j + 3]);
                        if (accumulate) {
                            const float4 p = c4[j];
                            o = make_float4(o.x + p.x, o.y + p.y, o.z + p.z, o.w + p.w);
                        }
                        c4[j] = o;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (c0 + j < N) crow[c0 + j] = accumulate ? crow[c0 + j] + r[j] : r[j];
                }
            }
        }
        fence_before();
        __syncthreads();
    }
    if (s_fail && threadIdx.x == 0) {
        atomicOr(err, TC_ERR_TIMEOUT_BIT);
        // copies still in flight land in this CTA's shared memory: wait for them (bounded) before leaving
        for (int u = used; u < issued; ++u) mbar_wait(smem_u32(&bar_a[u & 1]), (uint32_t)((u >> 1) & 1), budget);
        if (!b_done) mbar_wait(smem_u32(&bar_b), 0, budget);
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// 2D FP32 tensor map: rows of `inner` floats `stride_f` floats apart, boxes of 32 floats x box_rows.
bool make_map(CUtensorMap* m, const float* base, long long inner, long long rows, long long stride_f, int box_rows) {
    EncodeTiledFn fn = encode_tiled_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)stride_f * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)ATOM_F, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool tc_gemm_supported(long long K, int Np) {
    if (!(K > 0 && K % ATOM_F == 0 && K <= 128 && Np >= 16 && Np <= 256 && Np % 16 == 0)) return false;
    // two A tiles and the B tile in shared memory (plus the 1024-byte alignment slack)
    return (K / ATOM_F) * 128 * (2 * BM + Np) + 1024 <= 227 * 1024;
}

int tc_gemm(const float* A, long long P, long long K, long long lda, const float* Bt, int N, int Np, float* C,
            long long ldc, int accumulate, int* err, double wait_s, cudaStream_t st) {
    if (!tc_gemm_supported(K, Np) || N > Np || P <= 0) return -1;
    if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(Bt)) & 15u) return -1;
    if ((lda * (long long)sizeof(float)) % 16) return -1;
    CUtensorMap ta, tb;
    if (!make_map(&ta, A, K, P, lda, BM) || !make_map(&tb, Bt, K, Np, K, Np)) return -2;
    const int natoms = (int)(K / ATOM_F);
    const size_t smem = (size_t)natoms * 128 * (2 * BM + Np) + 1024;
    static size_t smem_set = 0;
    static int sms = 0;
    if (smem > smem_set) {
        if (cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return -3;
        smem_set = smem;
    }
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    int ncols = 32;
    while (ncols < Np) ncols <<= 1;
    // the peak SM clock, queried once: the attribute query costs hundreds of microseconds per call
    static int khz = 0;
    if (!khz) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
        if (khz <= 0) khz = 2000000;
    }
    const long long budget = (long long)(wait_s * (double)khz * 1e3);
    const long long ntiles = (P + BM - 1) / BM;
    const int grid = (int)(ntiles < sms ? ntiles : sms);
    k_tc_gemm<<<grid, THREADS, smem, st>>>(ta, tb, C, P, N, (int)K, Np, ldc, accumulate, ncols, err, budget);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace twa
