// pipe.cuh - persistent, software-pipelined variant of the line passes.
//
// A CTA walks a sequence of items (tile of LINES lines, field) with stride gridDim.x.  Each item
// needs one to three tile loads (e.g. Poisson line, stream 2p, stream 2p+1); the loads of all items
// form one sequence, and the next tile is copied from global into one of two shared-memory stages
// with cp.async (16-byte copies, no registers held) while the current one is transformed.  Once a
// thread has read its values out of a stage, that stage is reused as the FFT exchange buffer, so the
// pipeline costs no extra shared memory beyond the second stage.  Results go straight from
// registers to global memory.  Only full tiles are handled (the host checks that LINES divides the
// line count); the per-thread arrays that live across the loads of one item sit in the stash.
//
// TMA variant (column passes): the tile is copied by the Tensor Memory Accelerator instead of the
// threads' 16-byte copies.  The field is viewed as a dense 4D tensor {line start q, position j, outer
// index, field} of 8-byte elements, and a tile (LINES consecutive line starts x N positions) is up
// to eight boxes of LINES x 256 elements, issued by one thread and completed on the stage's
// mbarrier.  The strided gathers (one 8 * LINES-byte segment per position) then cost the load/store
// units nothing; the threads read the tile from shared memory in the same layout as the copies.
// Row passes take the same path with one bulk copy (cp.async.bulk) per contiguous row into the
// padded stage rows.
// Every wait is bounded: on time-out the CTA sets TWA_ERR_TIMEOUT_BIT in the error word, lets its
// copies in flight land (bounded) and returns.
#pragma once
#include "passes.cuh"
#include "tma.cuh"

namespace twa {

__device__ __forceinline__ void cp16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int K>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(K) : "memory");
}

__host__ __device__ constexpr bool pipe_op(int op) {
    return op == OP_DRIFT || op == OP_DRIFT_RHO || op == OP_KICK_DRIFT_VINV || op == OP_KICK_DRIFT ||
           op == OP_FWD || op == OP_INV || op == OP_FWD_MUL_INV;
}
__host__ __device__ constexpr int pipe_loads(int op) {
    return (op == OP_KICK_DRIFT_VINV || op == OP_KICK_DRIFT) ? 3 : (op == OP_DRIFT_RHO ? 2 : 1);
}
__host__ __device__ constexpr bool pipe_stash(int op) { return pipe_loads(op) > 1; }
// stash floats per thread: the first stream's density (drift_rho) or the pair's two potentials (kicks)
__host__ __device__ constexpr int pipe_stash_floats(int op, int rmax) {
    return !pipe_stash(op) ? 0 : (op == OP_DRIFT_RHO ? rmax : 2 * rmax);
}
// elements (float2) of one stage: the raw tile, or the padded exchange lines if larger
template <int N, int LINES, bool STRIDED>
__host__ __device__ constexpr int pipe_stage_elems() {
    constexpr int T = Plan<N>::T;
    constexpr int ex = LINES * (STRIDED ? line_stride(N, LINES) : line_stride_rows(N, T));
    constexpr int raw = STRIDED ? LINES * N : LINES * line_stride_rows(N, T);
    return ((ex > raw ? ex : raw) + 1) / 2 * 2;
}
// stage elements rounded for the TMA variant (each stage starts on 128 bytes)
template <int N, int LINES, bool STRIDED, bool TMA>
__host__ __device__ constexpr int pipe_stage_elems_al() {
    constexpr int se = pipe_stage_elems<N, LINES, STRIDED>();
    return TMA ? (se + 15) / 16 * 16 : se;
}
// dynamic shared memory of a variant: two stages, the stash, and (TMA) 128 bytes of alignment slack
template <int N, int LINES, bool STRIDED, int OP, bool TMA>
__host__ __device__ constexpr size_t pipe_smem_bytes() {
    return (2 * (size_t)pipe_stage_elems_al<N, LINES, STRIDED, TMA>() +
            (size_t)LINES * Plan<N>::T * pipe_stash_floats(OP, Plan<N>::RMAX) / 2) * sizeof(float2) + (TMA ? 128 : 0);
}
// tensor maps of the TMA variant: the batch's fields and the pass's field buffer
struct PipeMaps {
    CUtensorMap psi;
    CUtensorMap buf;
};

template <int N, int LINES, bool STRIDED, int OP, bool TMA>
__global__ void __launch_bounds__(LINES * Plan<N>::T, min_ctas(LINES * Plan<N>::T))
k_pipe(const PassArgs a, int tiles, int n_items, const __grid_constant__ PipeMaps maps) {
    using P = Plan<N>;
    constexpr int T = P::T, RMAX = P::RMAX, NTH = LINES * T;
    constexpr int LS = STRIDED ? line_stride(N, LINES) : line_stride_rows(N, T);
    constexpr int RS = line_stride_rows(N, T);      // row stride of a contiguous raw tile
    constexpr bool WARP = !STRIDED && (T <= 32);
    constexpr unsigned MASK = (NTH >= 32) ? 0xffffffffu : ((1u << NTH) - 1u);
    constexpr int SE = pipe_stage_elems_al<N, LINES, STRIDED, TMA>();
    constexpr int LPI = pipe_loads(OP);
    constexpr int CHUNKS = LINES * N / 2;           // 16-byte copies per tile
    constexpr int BOXR = N < 256 ? N : 256;         // positions per TMA box
    constexpr uint32_t TILE_BYTES = (uint32_t)LINES * N * sizeof(float2);
    static_assert(!TMA || STRIDED || RS % 2 == 0, "bulk row copies need 16-byte aligned shared rows");
    extern __shared__ __align__(16) float2 psm_raw[];
    __shared__ __align__(8) uint64_t bars[2];
    float2* psm = psm_raw;
    if constexpr (TMA) psm = psm_raw + (((128u - (smem_u32(psm_raw) & 127u)) & 127u) >> 3);
    float2* stage0 = psm;
    float2* stage1 = psm + SE;
    float* stf = reinterpret_cast<float*>(psm + 2 * SE) + threadIdx.x;  // per-thread stash, stf[i * NTH]
    const int tid = threadIdx.x;
    const int l = STRIDED ? (tid % LINES) : (tid / T);
    const int t = STRIDED ? (tid / LINES) : (tid % T);
    const float4* __restrict__ tw = a.tw;
    const int S = STRIDED ? a.S : 1;
    const int tq = STRIDED ? a.Qn / LINES : 1;
    const int G = gridDim.x;
    const int my_items = (n_items - (int)blockIdx.x + G - 1) / G;
    const int Q = my_items * LPI;

    // first element of line 0 of a tile, and of this thread's line
    auto tile_base = [&](int tile) -> int {
        if constexpr (STRIDED) return (tile % tq) * LINES + (tile / tq) * (int)a.OS;
        else return tile * LINES * N;
    };
    // field feeding load `sub` of item (pair or slot index f); nullptr when the slot does not exist
    auto source = [&](int f, int sub) -> const float2* {
        if constexpr (OP == OP_DRIFT) return a.psi + (long long)f * a.cells;
        else if constexpr (OP == OP_FWD || OP == OP_INV || OP == OP_FWD_MUL_INV) return a.buf + (long long)f * a.cells;
        else if constexpr (OP == OP_DRIFT_RHO) {
            const int slot = 2 * f + sub;
            return slot < a.n_slots ? a.psi + (long long)slot * a.cells : nullptr;
        } else {
            if (sub == 0) return a.buf + (long long)f * a.cells;
            const int slot = 2 * f + sub - 1;
            return slot < a.n_slots ? a.psi + (long long)slot * a.cells : nullptr;
        }
    };
    auto issue = [&](int q) {
        const int it = (int)blockIdx.x + (q / LPI) * G;
        const int f = it / tiles, tile = it % tiles;
        const float2* src = source(f, q % LPI);
        float2* dst = (q & 1) ? stage1 : stage0;
        if (src) {
            const float2* s0 = src + tile_base(tile);
            for (int c = tid; c < CHUNKS; c += NTH) {
                if constexpr (STRIDED) {
                    const int j = c / (LINES / 2), cp = (c % (LINES / 2)) * 2;
                    cp16(dst + j * LINES + cp, s0 + (long long)j * S + cp);
                } else {
                    const int r = c / (N / 2), off = (c % (N / 2)) * 2;
                    cp16(dst + r * RS + off, s0 + r * N + off);
                }
            }
        }
        cp_commit();
    };
    // TMA: one thread copies the tile of load q into its stage; a missing slot only arrives
    auto issue_tma = [&](int q) {
        const int it = (int)blockIdx.x + (q / LPI) * G;
        const int f = it / tiles, tile = it % tiles, sub = q % LPI;
        const uint32_t bar = smem_u32(&bars[q & 1]);
        const CUtensorMap* m = nullptr;
        int fi = 0;
        if constexpr (OP == OP_DRIFT) {
            m = &maps.psi;
            fi = f;
        } else if constexpr (OP == OP_FWD || OP == OP_INV || OP == OP_FWD_MUL_INV) {
            m = &maps.buf;
            fi = f;
        } else if constexpr (OP == OP_DRIFT_RHO) {
            fi = 2 * f + sub;
            if (fi < a.n_slots) m = &maps.psi;
        } else {
            if (sub == 0) {
                m = &maps.buf;
                fi = f;
            } else {
                fi = 2 * f + sub - 1;
                if (fi < a.n_slots) m = &maps.psi;
            }
        }
        if constexpr (!STRIDED) {
            // row tiles: LINES contiguous rows, one bulk copy each into the padded stage rows
            const float2* src = source(f, sub);
            if (src) {
                const uint32_t dst = smem_u32((q & 1) ? stage1 : stage0);
                const float2* s0 = src + tile_base(tile);
                mbar_expect_tx(bar, TILE_BYTES + a.stall_tx);
#pragma unroll 1
                for (int r = 0; r < LINES; ++r)
                    bulk_load(dst + (uint32_t)(r * RS * sizeof(float2)), s0 + (long long)r * N,
                              (uint32_t)(N * sizeof(float2)), bar);
            } else {
                mbar_arrive(bar);
            }
        } else if (m) {
            const uint32_t dst = smem_u32((q & 1) ? stage1 : stage0);
            const int q0 = (tile % tq) * LINES, outer = tile / tq;
            mbar_expect_tx(bar, TILE_BYTES + a.stall_tx);
#pragma unroll
            for (int b = 0; b < N / BOXR; ++b)
                tma_load_4d(dst + (uint32_t)(b * BOXR * LINES * sizeof(float2)), m, q0, b * BOXR, outer, fi, bar);
        } else {
            mbar_arrive(bar);
        }
    };

    if constexpr (TMA) {
        if (tid == 0) {
            mbar_init(smem_u32(&bars[0]), 1);
            mbar_init(smem_u32(&bars[1]), 1);
            mbar_init_fence();
        }
        __syncthreads();
        if (Q > 0 && tid == 0) issue_tma(0);
    } else {
        if (Q > 0) issue(0);
    }
#pragma unroll 1
    for (int q = 0; q < Q; ++q) {
        if constexpr (TMA) {
            if (q + 1 < Q && tid == 0) issue_tma(q + 1);
            const bool ok = mbar_wait(smem_u32(&bars[q & 1]), (uint32_t)((q >> 1) & 1), a.wait);
            if (__syncthreads_or(!ok)) {
                if (tid == 0) {
                    atomicOr(a.err, TWA_ERR_TIMEOUT_BIT);
                    // the copies in flight land before the CTA's shared memory is released
                    mbar_wait(smem_u32(&bars[q & 1]), (uint32_t)((q >> 1) & 1), a.wait);
                    if (q + 1 < Q)
                        mbar_wait(smem_u32(&bars[(q + 1) & 1]), (uint32_t)(((q + 1) >> 1) & 1), a.wait);
                }
                __syncthreads();
                return;
            }
        } else {
            if (q + 1 < Q) {
                issue(q + 1);
                cp_wait<1>();
            } else {
                cp_wait<0>();
            }
            __syncthreads();
        }
        const int it = (int)blockIdx.x + (q / LPI) * G;
        const int sub = q % LPI;
        const int f = it / tiles, tile = it % tiles;
        const int base = tile_base(tile) + (STRIDED ? l : l * N);
        float2* stg = (q & 1) ? stage1 : stage0;
        float2* sm = stg + l * LS;
        float2 v[RMAX];
        auto ld = [&](bool spec) {
#pragma unroll
            for (int i = 0; i < RMAX; ++i) {
                const int p = spec ? pos_spec<N>(t, i) : pos_nat<N>(t, i);
                v[i] = STRIDED ? stg[p * LINES + l] : stg[l * RS + p];
            }
            if constexpr (WARP) __syncwarp(MASK);
            else __syncthreads();
        };
        auto st_nat = [&](float2* F) {
#pragma unroll
            for (int i = 0; i < RMAX; ++i) F[base + pos_nat<N>(t, i) * S] = v[i];
        };
        auto st_spec = [&](float2* F) {
#pragma unroll
            for (int i = 0; i < RMAX; ++i) F[base + pos_spec<N>(t, i) * S] = v[i];
        };
        auto drift = [&]() {
            fft_line<N, false, WARP, MASK>(v, t, sm, tw);
#pragma unroll
            for (int i = 0; i < RMAX; ++i) {
                const int k = pos_spec<N>(t, i);
                const float4 p = __ldg(&a.ph[k]);
                v[i] = cmul_c(v[i], make_float2(p.x, p.y), make_float2(p.z, p.w));
            }
            fft_line<N, true, WARP, MASK>(v, t, sm, tw);
        };
        if constexpr (OP == OP_DRIFT) {
            ld(false);
            drift();
            st_nat(a.psi + (long long)f * a.cells);
        } else if constexpr (OP == OP_FWD) {
            ld(false);
            fft_line<N, false, WARP, MASK>(v, t, sm, tw);
            if (a.post != 1.0f) {
#pragma unroll
                for (int i = 0; i < RMAX; ++i) v[i] = make_float2(v[i].x * a.post, v[i].y * a.post);
            }
            st_spec(a.buf + (long long)f * a.cells);
        } else if constexpr (OP == OP_INV) {
            ld(true);
            fft_line<N, true, WARP, MASK>(v, t, sm, tw);
            st_nat(a.buf + (long long)f * a.cells);
        } else if constexpr (OP == OP_FWD_MUL_INV) {
            ld(false);
            fft_line<N, false, WARP, MASK>(v, t, sm, tw);
            const int mx = (1 << a.lx) - 1, my = (1 << (a.lxy - a.lx)) - 1;
            const float k2f = __ldg(&a.k2x[base & mx]) + __ldg(&a.k2y[(base >> a.lx) & my]) + __ldg(&a.k2z[base >> a.lxy]);
#pragma unroll
            for (int i = 0; i < RMAX; ++i) {
                const float k2 = k2f + __ldg(&a.k2a[pos_spec<N>(t, i)]);
                const float m = inv_k2(k2);
                v[i] = make_float2(v[i].x * m, v[i].y * m);
            }
            fft_line<N, true, WARP, MASK>(v, t, sm, tw);
            st_nat(a.buf + (long long)f * a.cells);
        } else if constexpr (OP == OP_DRIFT_RHO) {
            const int slot = 2 * f + sub;
            if (slot < a.n_slots) {
                ld(false);
                drift();
                st_nat(a.psi + (long long)slot * a.cells);
            } else {
#pragma unroll
                for (int i = 0; i < RMAX; ++i) v[i] = make_float2(0.f, 0.f);
            }
            if (sub == 0) {
#pragma unroll
                for (int i = 0; i < RMAX; ++i) stf[i * NTH] = fmaf(v[i].x, v[i].x, v[i].y * v[i].y);
            } else {
#pragma unroll
                for (int i = 0; i < RMAX; ++i)
                    v[i] = make_float2(stf[i * NTH], fmaf(v[i].x, v[i].x, v[i].y * v[i].y));
                fft_line<N, false, WARP, MASK>(v, t, sm, tw);
                st_spec(a.buf + (long long)f * a.cells);
            }
        } else {  // OP_KICK_DRIFT_VINV, OP_KICK_DRIFT
            if (sub == 0) {
                if constexpr (OP == OP_KICK_DRIFT_VINV) {
                    ld(true);
                    fft_line<N, true, WARP, MASK>(v, t, sm, tw);
                } else {
                    ld(false);
                }
                float* stv = reinterpret_cast<float*>(psm + 2 * SE) + threadIdx.x;
#pragma unroll
                for (int i = 0; i < RMAX; ++i) {
                    stv[i * NTH] = v[i].x;
                    stv[(RMAX + i) * NTH] = v[i].y;
                }
            } else {
                const int slot = 2 * f + sub - 1;
                if (slot < a.n_slots) {
                    ld(false);
                    const float* sv = reinterpret_cast<const float*>(psm + 2 * SE) + threadIdx.x + (sub - 1) * RMAX * NTH;
                    kick_all(v, a.kick, a.kick_lo, [&](int i) { return sv[i * NTH]; });
                    drift();
                    st_nat(a.psi + (long long)slot * a.cells);
                }
            }
        }
        // this item's shared-memory accesses precede the next TMA copy into its stage
        if constexpr (TMA) fence_proxy_async_smem();
        __syncthreads();
    }
}

template <int N>
int launch_pipe(const LaunchCfg& c, const PassArgs& a, int tiles, int n_items, cudaStream_t st, bool prepare_only);
template <int N>
bool has_pipe_variant(int op, bool strided, int lines);
template <int N>
bool has_pipe_tma_variant(int op, bool strided, int lines);

}  // namespace twa
