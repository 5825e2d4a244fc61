// passes.cuh - fused FP32 line passes of the batched split step (Sec. III.B.2).
//
// A pass transforms every line of a field along one axis.  A CTA owns LINES lines: for the x axis
// (contiguous, "row" passes) LINES consecutive rows, for y and z (strided, "column" passes) LINES
// lines whose starting cells are consecutive in memory, so that a warp reads 32 consecutive
// complex values per access.  The pointwise work of the method is fused into the passes:
//   kick      psi <- psi exp(-i kick V)            (U^V, kick = a dt / hbar, a = 1/2 or 1)
//   drift     FFT -> exp(-i hbar k_a^2 dt / 2) / N_a -> iFFT along the axis (U^T factorizes by axis)
//   density   rho = |psi|^2 of two streams packed as one complex line c = rho_0 + i rho_1, so one
//             complex transform serves two real Poisson solves
//   Poisson   W_k = rho_k / k^2, W_0 = 0, applied between the last forward and the first inverse
//             transform; the potential of lap V = C (rho - mean rho) (Eq. mft_normed) is V = -C W / cells,
//             and that scale is folded into the kick factor (kick = -a dt C / (hbar cells), carried as a
//             float hi + lo pair so its rounding does not bias every step by the same amount)
// Fields of the batch are processed in pairs of slots (2p, 2p+1) that share one packed Poisson
// line in `buf`; a missing partner (odd slot count) contributes zero density.
#pragma once
#include "fft_engine.cuh"

namespace twa {

enum Op : int {
    OP_DRIFT = 0,        // one field of psi: fwd, kinetic phase, inv
    OP_KICK_DRIFT,       // pair, V real in buf: kick both slots, drift both
    OP_KICK_DRIFT_VINV,  // pair, buf spectral along this axis: inverse -> V, kick, drift
    OP_DRIFT_RHO,        // pair: drift both slots, packed density -> forward -> buf (spectral)
    OP_RHO_FWD,          // pair: packed density of psi -> forward -> buf
    OP_FWD,              // one field of buf: forward (natural -> spectral layout)
    OP_FWD_MUL_INV,      // one field of buf: forward, Poisson multiplier, inverse
    OP_INV,              // one field of buf: inverse (spectral -> natural layout)
    OP_KICK_VINV,        // pair, buf spectral: inverse -> V, kick both slots (no drift)
    OP_KICK_FWD_OUT,     // pair, V real in buf: kick both slots, forward into out (moments)
    OP_STEPS_1D,         // pair, 1D field = one line: nsteps whole steps on chip
    OP_MUL_INV,          // one field of buf (spectral): Poisson multiplier, inverse
    OP_COUNT
};

struct PassArgs {
    float2* psi;            // slot 0 of the instance
    float2* buf;            // packed Poisson buffer (one field per pair) or a field buffer
    float2* out;            // destination of OP_KICK_FWD_OUT (one field per slot)
    const float4* tw;       // exp(-2 pi i m / N), m < N, as (hi.re, hi.im, lo.re, lo.im)
    const float4* ph;       // exp(-i hbar k^2 dt / 2) / N along this axis, FFT order: (hi.re, hi.im,
                            // lo.re, lo.im), lo = the remainder (exact value - hi) rounded to float
    const float* k2x;       // k^2 tables per axis (FFT order; length 1 and 0 for unused axes)
    const float* k2y;
    const float* k2z;
    const float* k2a;       // k^2 table of the pass's own axis (FFT order)
    float kick, kick_lo;    // -a dt C / (hbar cells) for the (first) kick, as hi + lo
    float kick2, kick2_lo;  // same with a = 1 for later kicks (OP_STEPS_1D)
    int S;                  // stride of the axis (elements)
    int Qn;                 // strided: starting cells per outer index; contiguous: unused
    long long OS;           // strided: outer stride
    long long cells;
    int n_slots;
    int n_pairs;
    int lx, lxy;            // log2 nx, log2 (nx ny)
    int nsteps;             // OP_STEPS_1D
    float post;             // OP_FWD: factor applied before the store (1, or 1/N to undo an inverse)
    const float4* ph2;      // plane passes: kinetic phase along y (hi, lo)
    int* err;               // device error word (bit TWA_ERR_TIMEOUT_BIT: a bounded wait gave up)
    long long wait;         // longest device-side wait, in clock64 cycles
    unsigned stall_tx;      // fault injection (tests): bytes a TMA tile pass expects beyond its copies
};

constexpr int TWA_ERR_TIMEOUT_BIT = 2;  // device error word: a bounded wait gave up

// Asks L2 to fetch a byte range ahead of its use (a hint: nothing waits on it, no data returns).
// The range must lie inside one allocation, start on 16 bytes and span a multiple of 16 bytes.
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "r"(bytes)
                 : "memory");
}
// The same for the cache sector holding one address, as an ordinary per-thread instruction.
__device__ __forceinline__ void prefetch_l2_sector(const void* p) { asm volatile("prefetch.L2 [%0];" ::"l"(p)); }

// z * exp(-i theta).  For |theta| <= 1/4 (every kick of the measured workloads) sin and cos are
// their Taylor polynomials through theta^7 and theta^8 (truncation below 1e-11, so the result is
// correctly rounded to float up to the rounding of the evaluation); otherwise theta is reduced to
// [-pi, pi] by a two-constant (Cody-Waite) split of 2 pi and sincosf is used.
__device__ __forceinline__ float2 kick_small(float2 z, float theta) {
    const float t2 = theta * theta;
    const float s = theta * fmaf(t2, fmaf(t2, fmaf(t2, -1.9841269841e-4f, 8.3333333333e-3f), -1.6666666667e-1f), 1.0f);
    const float c = fmaf(t2, fmaf(t2, fmaf(t2, fmaf(t2, 2.4801587302e-5f, -1.3888888889e-3f), 4.1666666667e-2f), -0.5f), 1.0f);
    return make_float2(fmaf(z.x, c, z.y * s), fmaf(z.y, c, -z.x * s));
}
__device__ __forceinline__ float2 kick_phase(float2 z, float theta) {
    float s, c;
    if (fabsf(theta) <= 0.25f) {
        return kick_small(z, theta);
    } else {
        const float n = rintf(theta * 0.15915494309189535f);
        float r = fmaf(-n, 6.28125f, theta);
        r = fmaf(-n, 0.0019353071795862327f, r);
        sincosf(r, &s, &c);
    }
    return make_float2(fmaf(z.x, c, z.y * s), fmaf(z.y, c, -z.x * s));
}

// Poisson multiplier 1/k^2 (0 for the k = 0 mode) without the quotient path of an IEEE division,
// whose per-value check and branch made the Poisson pass 20 % slower: the reciprocal approximation
// r0 = rcp.approx(k^2) (relative error e) refined by one Newton-Raphson step for 1/x,
// r1 = r0 + r0 (1 - k^2 r0) = (1 - e^2) / k^2 before its final rounding, so r1 is within 1 ulp of
// 1/k^2 and correctly rounded unless 1/k^2 lies within ~e^2 of a rounding boundary.  For any grid
// both k^2 >= (2 pi / L)^2 and 1/k^2 are normal floats, so flushing subnormals changes nothing.
__device__ __forceinline__ float inv_k2(float k2) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(k2));
    r = fmaf(r, fmaf(-k2, r, 1.0f), r);
    return k2 > 0.f ? r : 0.f;
}

// z * exp(-i (k_hi + k_lo) W): the kick with its scale carried in two floats.
__device__ __forceinline__ float2 kick_w(float2 z, float k_hi, float k_lo, float W) {
    return kick_phase(z, fmaf(k_hi, W, k_lo * W));
}

// The kick of a thread's R values, W_i = W(i), with one branch per thread instead of one per value:
// the Taylor form for all when every |theta_i| <= 1/4, else kick_phase for all.
template <int R, class G>
__device__ __forceinline__ void kick_all(float2 (&v)[R], float k_hi, float k_lo, G W_of) {
    float th[R];
    float m = 0.f;
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const float W = W_of(i);
        th[i] = fmaf(k_hi, W, k_lo * W);
        m = fmaxf(m, fabsf(th[i]));
    }
    if (m <= 0.25f) {
#pragma unroll
        for (int i = 0; i < R; ++i) v[i] = kick_small(v[i], th[i]);
    } else {
#pragma unroll
        for (int i = 0; i < R; ++i) v[i] = kick_phase(v[i], th[i]);
    }
}

// At least 512 resident threads (16 warps) per SM so that one CTA's loads overlap another's
// transforms; this caps the registers per thread at 128.
constexpr int min_ctas(int threads) { return threads >= 512 ? 1 : (512 / threads < 32 ? 512 / threads : 32); }

// Ops that keep a per-thread array across the two streams of a pair park it in a thread-private
// shared-memory stash (2 RMAX floats per thread, after the exchange lines) instead of registers.
// The heavy pair passes (four or five transforms per CTA) of lengths 16..256 copy the twiddle table
// and this axis' kinetic phases into shared memory once per CTA: the per-value table reads then skip
// the L1 tag stage, which the streamed field accesses keep busy.  Lighter passes keep L1-cached
// reads (the copy and its barrier would cost them more than it saves).
template <int N, int OP>
__host__ __device__ constexpr bool tables_in_smem() {
    return N >= 16 && N <= 256 && (OP == OP_KICK_DRIFT_VINV || OP == OP_DRIFT_RHO || OP == OP_KICK_DRIFT);
}
template <int N, int OP>
__host__ __device__ constexpr int smem_table_float4() { return tables_in_smem<N, OP>() ? tw_entries<N>() + N : 0; }

__host__ __device__ constexpr bool op_stash(int op) {
    return op == OP_DRIFT_RHO || op == OP_RHO_FWD || op == OP_KICK_DRIFT_VINV || op == OP_KICK_VINV ||
           op == OP_KICK_DRIFT || op == OP_KICK_FWD_OUT;
}

// Ops with a two-field variant (DUAL): both fields of a pair (slots 2f, 2f+1) are transformed by the
// same threads at once, so every twiddle and kinetic-phase table read serves two fields; the drift
// then runs over pairs instead of slots.
__host__ __device__ constexpr bool op_dual(int op) {
    return op == OP_DRIFT || op == OP_KICK_DRIFT || op == OP_KICK_DRIFT_VINV || op == OP_DRIFT_RHO;
}

// Shared-memory layout of a tile (offsets in float2): the exchange lines, the per-thread stash, the
// staged tables (16-byte aligned) and, for DUAL, a second set of exchange lines.
template <int N, int LINES, bool STRIDED, int OP, bool DUAL>
struct TileSmem {
    static constexpr int T = Plan<N>::T, RMAX = Plan<N>::RMAX, NTH = LINES * T;
    static constexpr int LS = STRIDED ? line_stride(N, LINES) : line_stride_rows(N, T);
    static constexpr bool TS = tables_in_smem<N, OP>() || (DUAL && N >= 16 && N <= 256);
    static constexpr int stash = LINES * LS;
    static constexpr int tables = (stash + (op_stash(OP) ? RMAX * NTH : 0) + 1) / 2 * 2;
    static constexpr int ex2 = tables + (TS ? 2 * (tw_entries<N>() + N) : 0);
    static constexpr int total = ex2 + (DUAL ? LINES * LS : 0);
};

// One tile of a line pass: LINES lines of field f (tile index bx along the field), run by the
// LINES * T threads of the CTA with dynamic shared memory smem.  Kernel body of k_line, and the
// work item of the persistent batch kernel.
template <int N, int LINES, bool STRIDED, int OP, bool DUAL = false>
__device__ __forceinline__ void line_tile(const PassArgs& a, int bx, int f, float2* smem) {
    using P = Plan<N>;
    using SM = TileSmem<N, LINES, STRIDED, OP, DUAL>;
    static_assert(!DUAL || op_dual(OP), "no two-field variant of this op");
    constexpr int T = P::T, RMAX = P::RMAX, LS = SM::LS;
    constexpr bool WARP = !STRIDED && (T <= 32);
    constexpr unsigned MASK = (LINES * T >= 32) ? 0xffffffffu : ((1u << (LINES * T)) - 1u);
    const int tid = threadIdx.x;
    const int l = STRIDED ? (tid % LINES) : (tid / T);
    const int t = STRIDED ? (tid / LINES) : (tid % T);
    float2* sm = smem + l * LS;
    float2* sm2 = smem + SM::ex2 + l * LS;  // second exchange line (DUAL)
    constexpr int NTH = LINES * T;
    const float4* tw = a.tw;
    const float4* ph = a.ph;
    constexpr bool TS = SM::TS;
    if constexpr (TS) {
        constexpr int E = tw_entries<N>();
        float4* st = reinterpret_cast<float4*>(smem + SM::tables);
        for (int i = tid; i < E; i += NTH) st[i] = __ldg(&a.tw[i]);
        for (int i = tid; i < N; i += NTH) st[E + i] = __ldg(&a.ph[i]);
        __syncthreads();
        tw = st;
        ph = st + E;
    }

    // Line of this thread (element offset of its first cell inside a field; a field has fewer
    // than 2^31 cells); lines past the end of the field (partial tiles of small grids) run on a
    // clamped valid line and store nothing, so every thread reaches every barrier.
    int base;
    bool act;
    if constexpr (STRIDED) {
        const int tq = (a.Qn + LINES - 1) / LINES;
        const int q = (int)(bx % tq) * LINES + l;
        act = q < a.Qn;
        base = (act ? q : a.Qn - 1) + (int)(bx / tq) * (int)a.OS;
    } else {
        const int rows = (int)(a.cells / N);
        const int row = (int)bx * LINES + l;
        act = row < rows;
        base = (act ? row : rows - 1) * N;
    }
    const int S = STRIDED ? a.S : 1;
    float2 v[RMAX];

    // The pair passes ask L2 for the stream lines they read after another field (the potential, or
    // the first stream) right after that field's loads are issued: the hint queues behind those
    // loads, and the stream's DRAM latency then overlaps the first field's transforms.
    auto prefetch_lines = [&](const float2* F) {
        if constexpr (STRIDED) {
            const int tq = (a.Qn + LINES - 1) / LINES;
            const int q0 = (int)(bx % tq) * LINES;
            const unsigned bytes = (unsigned)min(LINES, a.Qn - q0) * 8u;
            const float2* b0 = F + q0 + (long long)(bx / tq) * a.OS;
            // one short segment per position: plain per-thread prefetches, one per 32-byte sector
            for (int j = tid; j < N; j += NTH) {
                const char* p = reinterpret_cast<const char*>(b0 + (long long)j * S);
                for (unsigned o = 0; o < bytes; o += 32u) prefetch_l2_sector(p + o);
            }
        } else {
            const int r0 = (int)bx * LINES;
            const unsigned bytes = (unsigned)min(LINES, (int)(a.cells / N) - r0) * N * 8u;
            const char* b0 = reinterpret_cast<const char*>(F + (long long)r0 * N);
            if (((reinterpret_cast<uintptr_t>(b0) | bytes) & 15u) == 0)
                for (unsigned o = (unsigned)tid * 4096u; o < bytes; o += NTH * 4096u)
                    prefetch_l2(b0 + o, min(4096u, bytes - o));
        }
    };
    auto prefetch_pair = [&](bool first) {
        if (first) prefetch_lines(a.psi + (long long)(2 * f) * a.cells);
        if (2 * f + 1 < a.n_slots) prefetch_lines(a.psi + (long long)(2 * f + 1) * a.cells);
    };

    // field data is read once per pass: load it through L2 only (ld.global.cg), so the twiddle,
    // phase and k^2 tables keep the L1 cache
    auto load_nat = [&](float2 (&w)[RMAX], const float2* F) {
#pragma unroll
        for (int i = 0; i < RMAX; ++i) w[i] = __ldcg(&F[base + pos_nat<N>(t, i) * S]);
    };
    auto store_nat = [&](const float2 (&w)[RMAX], float2* F) {
        if (!act) return;
#pragma unroll
        for (int i = 0; i < RMAX; ++i) F[base + pos_nat<N>(t, i) * S] = w[i];
    };
    auto load_spec = [&](float2 (&w)[RMAX], const float2* F) {
#pragma unroll
        for (int i = 0; i < RMAX; ++i) w[i] = __ldcg(&F[base + pos_spec<N>(t, i) * S]);
    };
    auto store_spec = [&](const float2 (&w)[RMAX], float2* F) {
        if (!act) return;
#pragma unroll
        for (int i = 0; i < RMAX; ++i) F[base + pos_spec<N>(t, i) * S] = w[i];
    };
    // multiply by the kinetic phase carried as hi + lo, so its rounding does not repeat every step
    auto phase = [&](float2 (&w)[RMAX]) {
#pragma unroll
        for (int i = 0; i < RMAX; ++i) {
            const int k = pos_spec<N>(t, i);
            const float4 p = TS ? ph[k] : __ldg(&ph[k]);
            w[i] = cmul_c(w[i], make_float2(p.x, p.y), make_float2(p.z, p.w));
        }
    };
    // 1/k^2 (0 at k = 0): the k^2 of the two other axes is fixed along the line (read once at the
    // line's first cell, where this axis' wavenumber is 0); this axis' k^2 is read per slot
    auto poisson = [&](float2 (&w)[RMAX]) {
        const int mx = (1 << a.lx) - 1, my = (1 << (a.lxy - a.lx)) - 1;
        const float k2f = __ldg(&a.k2x[base & mx]) + __ldg(&a.k2y[(base >> a.lx) & my]) + __ldg(&a.k2z[base >> a.lxy]);
#pragma unroll
        for (int i = 0; i < RMAX; ++i) {
            const float k2 = k2f + __ldg(&a.k2a[pos_spec<N>(t, i)]);
            const float m = inv_k2(k2);
            w[i] = make_float2(w[i].x * m, w[i].y * m);
        }
    };
    auto drift = [&](float2 (&w)[RMAX]) {
        fft_line<N, false, WARP, MASK, TS>(w, t, sm, tw);
        phase(w);
        fft_line<N, true, WARP, MASK, TS>(w, t, sm, tw);
    };
    // both fields of a pair at once: one table read per twiddle and phase for the two
    auto drift2 = [&](float2 (&w)[RMAX], float2 (&x)[RMAX]) {
        fft_line2<N, false, WARP, MASK, TS>(w, x, t, sm, sm2, tw);
#pragma unroll
        for (int i = 0; i < RMAX; ++i) {
            const int k = pos_spec<N>(t, i);
            const float4 p = TS ? ph[k] : __ldg(&ph[k]);
            w[i] = cmul_c(w[i], make_float2(p.x, p.y), make_float2(p.z, p.w));
            x[i] = cmul_c(x[i], make_float2(p.x, p.y), make_float2(p.z, p.w));
        }
        fft_line2<N, true, WARP, MASK, TS>(w, x, t, sm, sm2, tw);
    };

    if constexpr (DUAL) {
        // field f is the pair (2f, 2f+1); a missing second slot is transformed as zeros and not stored
        float2* F0 = a.psi + (long long)(2 * f) * a.cells;
        float2* F1 = F0 + a.cells;
        const bool has1 = 2 * f + 1 < a.n_slots;
        float2 u[RMAX];
        float* stv = reinterpret_cast<float*>(smem + SM::stash) + tid;
        if constexpr (OP == OP_KICK_DRIFT_VINV || OP == OP_KICK_DRIFT) {
            // the pair's potentials (inverse-transformed from the spectral Poisson line, or read real)
            // parked in the stash as two float planes
            const bool kick = OP == OP_KICK_DRIFT_VINV || a.kick != 0.f;
            if (kick) {
                if constexpr (OP == OP_KICK_DRIFT_VINV) {
                    load_spec(v, a.buf + (long long)f * a.cells);
                } else {
                    load_nat(v, a.buf + (long long)f * a.cells);
                }
            }
            prefetch_pair(kick);
            if (kick) {
                if constexpr (OP == OP_KICK_DRIFT_VINV) fft_line<N, true, WARP, MASK, TS>(v, t, sm, tw);
#pragma unroll
                for (int i = 0; i < RMAX; ++i) {
                    stv[i * NTH] = v[i].x;
                    stv[(RMAX + i) * NTH] = v[i].y;
                }
            }
            load_nat(v, F0);
            if (has1) load_nat(u, F1);
            else {
#pragma unroll
                for (int i = 0; i < RMAX; ++i) u[i] = make_float2(0.f, 0.f);
            }
            if (kick) {
                kick_all(v, a.kick, a.kick_lo, [&](int i) { return stv[i * NTH]; });
                kick_all(u, a.kick, a.kick_lo, [&](int i) { return stv[(RMAX + i) * NTH]; });
            }
            drift2(v, u);
            store_nat(v, F0);
            if (has1) store_nat(u, F1);
        } else {  // OP_DRIFT (over pairs), OP_DRIFT_RHO
            load_nat(v, F0);
            if (has1) load_nat(u, F1);
            else {
#pragma unroll
                for (int i = 0; i < RMAX; ++i) u[i] = make_float2(0.f, 0.f);
            }
            drift2(v, u);
            store_nat(v, F0);
            if (has1) store_nat(u, F1);
            if constexpr (OP == OP_DRIFT_RHO) {
#pragma unroll
                for (int i = 0; i < RMAX; ++i)
                    v[i] = make_float2(fmaf(v[i].x, v[i].x, v[i].y * v[i].y), fmaf(u[i].x, u[i].x, u[i].y * u[i].y));
                fft_line<N, false, WARP, MASK, TS>(v, t, sm, tw);
                store_spec(v, a.buf + (long long)f * a.cells);
            }
        }
    } else if constexpr (OP == OP_DRIFT) {
        float2* F = a.psi + (long long)f * a.cells;
        load_nat(v, F);
        drift(v);
        store_nat(v, F);
    } else if constexpr (OP == OP_KICK_DRIFT || OP == OP_KICK_FWD_OUT) {
        // the pair's real potentials are read once and parked in the stash as two float planes
        float* stv = reinterpret_cast<float*>(smem + LINES * LS) + tid;
        const bool kick = a.kick != 0.f;
        if (kick) load_nat(v, a.buf + (long long)f * a.cells);
        prefetch_pair(kick);
        if (kick) {
#pragma unroll
            for (int i = 0; i < RMAX; ++i) {
                stv[i * NTH] = v[i].x;
                stv[(RMAX + i) * NTH] = v[i].y;
            }
        }
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            const int slot = 2 * f + h;
            if (slot >= a.n_slots) break;
            float2* F = a.psi + (long long)slot * a.cells;
            load_nat(v, F);
            if (kick) {
                const float* sv = stv + h * RMAX * NTH;
                kick_all(v, a.kick, a.kick_lo, [&](int i) { return sv[i * NTH]; });
            }
            if constexpr (OP == OP_KICK_DRIFT) {
                drift(v);
                store_nat(v, F);
            } else {
                fft_line<N, false, WARP, MASK, TS>(v, t, sm, tw);
                store_spec(v, a.out + (long long)slot * a.cells);
            }
        }
    } else if constexpr (OP == OP_KICK_DRIFT_VINV || OP == OP_KICK_VINV) {
        // inverse transform of the pair's Poisson line, parked in the stash for both streams
        load_spec(v, a.buf + (long long)f * a.cells);
        prefetch_pair(true);
        fft_line<N, true, WARP, MASK, TS>(v, t, sm, tw);
        // the two streams' potentials as separate float planes (each stream reads only its own)
        float* stv = reinterpret_cast<float*>(smem + LINES * LS) + tid;
#pragma unroll
        for (int i = 0; i < RMAX; ++i) {
            stv[i * NTH] = v[i].x;
            stv[(RMAX + i) * NTH] = v[i].y;
        }
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            const int slot = 2 * f + h;
            if (slot >= a.n_slots) break;
            float2* F = a.psi + (long long)slot * a.cells;
            load_nat(v, F);
            const float* sv = stv + h * RMAX * NTH;
            kick_all(v, a.kick, a.kick_lo, [&](int i) { return sv[i * NTH]; });
            if constexpr (OP == OP_KICK_DRIFT_VINV) drift(v);
            store_nat(v, F);
        }
    } else if constexpr (OP == OP_DRIFT_RHO || OP == OP_RHO_FWD) {
        // density of slot 2f parked in the stash while slot 2f+1 is processed, then packed as
        // rho_0 + i rho_1 in v and transformed (one loop body: no hoisting of the second stream)
        float* sr = reinterpret_cast<float*>(smem + LINES * LS) + tid;  // density of slot 2f
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            const int slot = 2 * f + h;
            if (slot < a.n_slots) {
                float2* F = a.psi + (long long)slot * a.cells;
                load_nat(v, F);
                if (h == 0) prefetch_pair(false);
                if constexpr (OP == OP_DRIFT_RHO) {
                    drift(v);
                    store_nat(v, F);
                }
            } else {
#pragma unroll
                for (int i = 0; i < RMAX; ++i) v[i] = make_float2(0.f, 0.f);
            }
            if (h == 0) {
#pragma unroll
                for (int i = 0; i < RMAX; ++i) sr[i * NTH] = fmaf(v[i].x, v[i].x, v[i].y * v[i].y);
            } else {
#pragma unroll
                for (int i = 0; i < RMAX; ++i) v[i] = make_float2(sr[i * NTH], fmaf(v[i].x, v[i].x, v[i].y * v[i].y));
            }
        }
        fft_line<N, false, WARP, MASK, TS>(v, t, sm, tw);
        store_spec(v, a.buf + (long long)f * a.cells);
    } else if constexpr (OP == OP_FWD) {
        float2* F = a.buf + (long long)f * a.cells;
        load_nat(v, F);
        fft_line<N, false, WARP, MASK, TS>(v, t, sm, tw);
        if (a.post != 1.0f) {
#pragma unroll
            for (int i = 0; i < RMAX; ++i) v[i] = make_float2(v[i].x * a.post, v[i].y * a.post);
        }
        store_spec(v, F);
    } else if constexpr (OP == OP_FWD_MUL_INV) {
        float2* F = a.buf + (long long)f * a.cells;
        load_nat(v, F);
        fft_line<N, false, WARP, MASK, TS>(v, t, sm, tw);
        poisson(v);
        fft_line<N, true, WARP, MASK, TS>(v, t, sm, tw);
        store_nat(v, F);
    } else if constexpr (OP == OP_MUL_INV) {
        float2* F = a.buf + (long long)f * a.cells;
        load_spec(v, F);
        poisson(v);
        fft_line<N, true, WARP, MASK, TS>(v, t, sm, tw);
        store_nat(v, F);
    } else if constexpr (OP == OP_INV) {
        float2* F = a.buf + (long long)f * a.cells;
        load_spec(v, F);
        fft_line<N, true, WARP, MASK, TS>(v, t, sm, tw);
        store_nat(v, F);
    } else if constexpr (OP == OP_STEPS_1D) {
        // base is the line offset inside the field; here each line slot of the CTA is one pair.
        const int p = (int)bx * LINES + l;
        const bool active = p < a.n_pairs;
        const int pe = active ? p : a.n_pairs - 1;
        const bool has1 = 2 * pe + 1 < a.n_slots;
        float2* F0 = a.psi + (long long)(2 * pe) * a.cells;
        float2* F1 = a.psi + (long long)(2 * pe + 1) * a.cells;
        float2* VC = a.buf + (long long)pe * a.cells;
        float2 u1[RMAX], w[RMAX];
#pragma unroll
        for (int i = 0; i < RMAX; ++i) {
            const int e = pos_nat<N>(t, i);
            v[i] = F0[e];
            u1[i] = has1 ? F1[e] : make_float2(0.f, 0.f);
            w[i] = VC[e];
        }
#pragma unroll 1
        for (int st = 0; st < a.nsteps; ++st) {
            const float kk = (st == 0) ? a.kick : a.kick2;
            const float kl = (st == 0) ? a.kick_lo : a.kick2_lo;
            kick_all(v, kk, kl, [&](int i) { return w[i].x; });
            kick_all(u1, kk, kl, [&](int i) { return w[i].y; });
            drift(v);
            drift(u1);
#pragma unroll
            for (int i = 0; i < RMAX; ++i)
                w[i] = make_float2(fmaf(v[i].x, v[i].x, v[i].y * v[i].y), fmaf(u1[i].x, u1[i].x, u1[i].y * u1[i].y));
            fft_line<N, false, WARP, MASK, TS>(w, t, sm, tw);
#pragma unroll
            for (int i = 0; i < RMAX; ++i) {
                const float k2 = __ldg(&a.k2x[pos_spec<N>(t, i)]);
                const float m = inv_k2(k2);
                w[i] = make_float2(w[i].x * m, w[i].y * m);
            }
            fft_line<N, true, WARP, MASK, TS>(w, t, sm, tw);
        }
        if (active) {
#pragma unroll
            for (int i = 0; i < RMAX; ++i) {
                const int e = pos_nat<N>(t, i);
                F0[e] = v[i];
                if (has1) F1[e] = u1[i];
                VC[e] = w[i];
            }
        }
    }
}

template <int N, int LINES, bool STRIDED, int OP, bool DUAL = false>
__global__ void __launch_bounds__(LINES * Plan<N>::T, (OP == OP_STEPS_1D) ? 1 : min_ctas(LINES * Plan<N>::T))
k_line(const PassArgs a) {
    extern __shared__ float2 smem[];
    line_tile<N, LINES, STRIDED, OP, DUAL>(a, (int)blockIdx.x, (int)blockIdx.y, smem);
}

// ---------------------------------------------------------------------------------------------
// xy-plane passes of 3D fields (nx = ny = N): one CTA owns one z-plane of one pair of slots.  The
// rows are transformed first and written back to the field; after a CTA barrier the columns are
// read back with L2-only loads (the plane was just written, so it is L2-resident and DRAM sees one
// read and one write of it) and transformed.  This fuses the x and y passes without holding a plane
// in shared memory.
//   PL_KICK_DRIFT : per slot of the pair: kick with the real Poisson field, drift_x (rows), drift_y
//   PL_POISSON    : Poisson field plane at fixed k_z: FFT_x (rows), FFT_y, 1/k^2, iFFT_y (columns),
//                   iFFT_x (rows)
enum PlaneOp : int { PL_KICK_DRIFT = 0, PL_POISSON = 1, PL_COUNT };

template <int N, int L, int POP>
__global__ void __launch_bounds__(L * Plan<N>::T, min_ctas(L * Plan<N>::T))
k_plane(const PassArgs a) {
    using P = Plan<N>;
    constexpr int T = P::T, RMAX = P::RMAX;
    constexpr int LSR = line_stride_rows(N, T), LSC = line_stride(N, L);
    constexpr bool WARP = (T <= 32);
    constexpr unsigned MASK = (L * T >= 32) ? 0xffffffffu : ((1u << (L * T)) - 1u);
    extern __shared__ float2 smem[];
    const int tid = threadIdx.x;
    const int lr = tid / T, tr = tid % T;        // row mapping: lanes walk along a row
    const int lc = tid % L, tc = tid / L;        // column mapping: lanes walk across columns
    const float4* __restrict__ tw = a.tw;
    const int plane = (int)blockIdx.x * N * N;
    const int f = blockIdx.y;
    float2 v[RMAX];

    auto phase = [&](float2 (&w)[RMAX], const float4* ph, int t) {
#pragma unroll
        for (int i = 0; i < RMAX; ++i) {
            const int k = pos_spec<N>(t, i);
            const float4 p = __ldg(&ph[k]);
            w[i] = cmul_c(w[i], make_float2(p.x, p.y), make_float2(p.z, p.w));
        }
    };
    // columns run along y: k_x (the column) and k_z (the plane) are fixed, k_y is read per slot
    auto poisson = [&](float2 (&w)[RMAX], int col) {
        const float k2f = __ldg(&a.k2x[col]) + __ldg(&a.k2z[blockIdx.x]);
#pragma unroll
        for (int i = 0; i < RMAX; ++i) {
            const float k2 = k2f + __ldg(&a.k2y[pos_spec<N>(tc, i)]);
            const float m = inv_k2(k2);
            w[i] = make_float2(w[i].x * m, w[i].y * m);
        }
    };

    if constexpr (POP == PL_KICK_DRIFT) {
        const float2* Wp = a.buf + (long long)f * a.cells + plane;
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            const int slot = 2 * f + h;
            if (slot >= a.n_slots) break;
            float2* F = a.psi + (long long)slot * a.cells + plane;
            float2* smr = smem + lr * LSR;
#pragma unroll 1
            for (int r0 = 0; r0 < N; r0 += L) {
                const int row = (r0 + lr) * N;
                // all loads first (the field, then this stream's potential component), then the kicks
                const float* Wh = reinterpret_cast<const float*>(Wp) + h;
                float w[RMAX];
#pragma unroll
                for (int i = 0; i < RMAX; ++i) v[i] = __ldcg(&F[row + pos_nat<N>(tr, i)]);
#pragma unroll
                for (int i = 0; i < RMAX; ++i) w[i] = __ldcg(&Wh[2 * (row + pos_nat<N>(tr, i))]);
                kick_all(v, a.kick, a.kick_lo, [&](int i) { return w[i]; });
                fft_line<N, false, WARP, MASK>(v, tr, smr, tw);
                phase(v, a.ph, tr);
                fft_line<N, true, WARP, MASK>(v, tr, smr, tw);
#pragma unroll
                for (int i = 0; i < RMAX; ++i) F[row + pos_nat<N>(tr, i)] = v[i];
            }
            __syncthreads();
            float2* smc = smem + lc * LSC;
#pragma unroll 1
            for (int c0 = 0; c0 < N; c0 += L) {
                const int col = c0 + lc;
#pragma unroll
                for (int i = 0; i < RMAX; ++i) v[i] = __ldcg(&F[col + pos_nat<N>(tc, i) * N]);
                fft_line<N, false, false>(v, tc, smc, tw);
                phase(v, a.ph2, tc);
                fft_line<N, true, false>(v, tc, smc, tw);
#pragma unroll
                for (int i = 0; i < RMAX; ++i) F[col + pos_nat<N>(tc, i) * N] = v[i];
            }
            __syncthreads();
        }
    } else {
        float2* Wp = a.buf + (long long)f * a.cells + plane;
        float2* smr = smem + lr * LSR;
        float2* smc = smem + lc * LSC;
#pragma unroll 1
        for (int r0 = 0; r0 < N; r0 += L) {
            const int row = (r0 + lr) * N;
#pragma unroll
            for (int i = 0; i < RMAX; ++i) v[i] = __ldcg(&Wp[row + pos_nat<N>(tr, i)]);
            fft_line<N, false, WARP, MASK>(v, tr, smr, tw);
#pragma unroll
            for (int i = 0; i < RMAX; ++i) Wp[row + pos_spec<N>(tr, i)] = v[i];
        }
        __syncthreads();
#pragma unroll 1
        for (int c0 = 0; c0 < N; c0 += L) {
            const int col = c0 + lc;
#pragma unroll
            for (int i = 0; i < RMAX; ++i) v[i] = __ldcg(&Wp[col + pos_nat<N>(tc, i) * N]);
            fft_line<N, false, false>(v, tc, smc, tw);
            poisson(v, col);
            fft_line<N, true, false>(v, tc, smc, tw);
#pragma unroll
            for (int i = 0; i < RMAX; ++i) Wp[col + pos_nat<N>(tc, i) * N] = v[i];
        }
        __syncthreads();
#pragma unroll 1
        for (int r0 = 0; r0 < N; r0 += L) {
            const int row = (r0 + lr) * N;
#pragma unroll
            for (int i = 0; i < RMAX; ++i) v[i] = __ldcg(&Wp[row + pos_spec<N>(tr, i)]);
            fft_line<N, true, WARP, MASK>(v, tr, smr, tw);
#pragma unroll
            for (int i = 0; i < RMAX; ++i) Wp[row + pos_nat<N>(tr, i)] = v[i];
        }
    }
}

template <int N>
int launch_plane(int pop, int lines, dim3 grid, const PassArgs& a, cudaStream_t st, bool prepare_only);
template <int N>
bool has_plane_variant(int pop, int lines);

// Host-side launcher of one pass (defined per N in passes_n*.cu).
struct LaunchCfg {
    int op;
    bool strided;
    int lines;
    dim3 grid;
    bool dual = false;  // two-field variant (both slots of a pair per thread; drift over pairs)
    bool tma = false;   // pipelined column pass with TMA tile copies
    const void* maps = nullptr;  // its tensor maps (PipeMaps, pipe.cuh)
};
template <int N>
int launch_line(const LaunchCfg& c, const PassArgs& a, cudaStream_t st, bool prepare_only);
template <int N>
bool has_variant(int op, bool strided, int lines);
template <int N>
bool has_dual_variant(int op, bool strided, int lines);
int plan_threads_per_line(int n);

}  // namespace twa
