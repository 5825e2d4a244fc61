// run1d.cuh - a whole 1D run (steps and moment sums of every output) in one launch.
//
// A 1D field is one line, so each stream stays in the registers of the T threads of its line for
// the whole run (Sec. III.B.2's split step: kick, drift by FFT / kinetic phase / iFFT, density,
// Poisson solve by FFT / 1/k^2 / iFFT, all on chip).  At every output the pair's synchronized fields (the pending
// half kick applied to copies) contribute their per-cell sums |psi|^2, Re psi, Im psi, and the
// classical slot its |psi_cl|^2, to a partial-sum buffer indexed by (output, pair); one finishing
// kernel then adds the pairs in pair order and forms the scalars of every output (Eq. E[op],
// Eq. Q).  The run begins on a synchronized batch (its Poisson field is computed on chip) and ends
// with the closing half kick, so the batch is synchronized again.
#pragma once
#include "passes.cuh"

namespace twa {

struct Run1DArgs {
    PassArgs a;       // psi, tw, ph, k2x, cells = N, n_slots, n_pairs; kick: half, kick2: full
    int n_out;        // outputs after the initial one
    int out_every;    // KDK steps per output
    double* part;     // [(n_out + 1) * n_pairs][3][N]: per-pair sums |psi|^2, Re psi, Im psi
    double* part_cl;  // [(n_out + 1)][N]: |psi_cl|^2
    double* part_bad; // [(n_out + 1) * n_pairs]: non-finite values met
};

// Each stream of a pair is a line of its own: the pair's two lines are neighbours in the CTA (lines
// 2q and 2q + 1), T threads each, so the two fields' transforms run side by side (in one warp for
// T <= 16) instead of one after the other, and each thread holds one field and the pair's packed
// potential.  Both lines form the packed density (each takes the partner's |psi|^2 at the same
// positions, by a shuffle or through shared memory) and transform it, so each has the potential
// without a second exchange; the arithmetic of every field is that of the per-interval passes.
template <int N, int LINES>
__global__ void __launch_bounds__(LINES * Plan<N>::T, 1)
k_run1d(const Run1DArgs r) {
    static_assert(LINES % 2 == 0, "two lines per pair");
    using P = Plan<N>;
    constexpr int T = P::T, RMAX = P::RMAX;
    constexpr int LS = line_stride_rows(N, T);
    constexpr bool WARP = T <= 32;
    constexpr bool SHFL = 2 * T <= 32;  // the pair's two lines share a warp
    constexpr unsigned MASK = (LINES * T >= 32) ? 0xffffffffu : ((1u << (LINES * T)) - 1u);
    extern __shared__ float2 smem[];
    const PassArgs& a = r.a;
    const int tid = threadIdx.x, l = tid / T, t = tid % T;
    float2* sm = smem + l * LS;
    const float4* tw = a.tw;
    const int fld = l & 1;                                  // field of the pair on this line
    const int p = ((int)blockIdx.x * LINES + l) >> 1;
    const bool active = p < a.n_pairs;
    const int pe = active ? p : a.n_pairs - 1;
    const int slot = 2 * pe + fld;
    const bool has = slot < a.n_slots;                      // the last pair of an odd slot count has one field
    float2* F = a.psi + (long long)slot * N;                // dereferenced only when has
    float2 v[RMAX], w[RMAX];
#pragma unroll
    for (int i = 0; i < RMAX; ++i) v[i] = has ? F[pos_nat<N>(t, i)] : make_float2(0.f, 0.f);

    // y = the partner line's x at this thread's positions (every thread of the CTA takes part)
    auto swap_f = [&](const float (&x)[RMAX], float (&y)[RMAX]) {
        if constexpr (SHFL) {
#pragma unroll
            for (int i = 0; i < RMAX; ++i) y[i] = __shfl_xor_sync(MASK, x[i], T);
        } else {
            float* mine = reinterpret_cast<float*>(sm);
            const float* other = reinterpret_cast<const float*>(smem + (l ^ 1) * LS);
            __syncthreads();  // the line regions are free of the last transform's exchange
#pragma unroll
            for (int i = 0; i < RMAX; ++i) mine[i * T + t] = x[i];
            __syncthreads();
#pragma unroll
            for (int i = 0; i < RMAX; ++i) y[i] = other[i * T + t];
            __syncthreads();  // before the next transform reuses the regions
        }
    };
    auto drift = [&]() {
        fft_line<N, false, WARP, MASK>(v, t, sm, tw);
#pragma unroll
        for (int i = 0; i < RMAX; ++i) {
            const float4 ph = __ldg(&a.ph[pos_spec<N>(t, i)]);
            v[i] = cmul_c(v[i], make_float2(ph.x, ph.y), make_float2(ph.z, ph.w));
        }
        fft_line<N, true, WARP, MASK>(v, t, sm, tw);
    };
    // packed potential of the pair: W = iFFT(FFT(|psi_0|^2 + i |psi_1|^2) / k^2), on both lines
    auto poisson = [&]() {
        float d[RMAX], e[RMAX];
#pragma unroll
        for (int i = 0; i < RMAX; ++i) d[i] = fmaf(v[i].x, v[i].x, v[i].y * v[i].y);
        swap_f(d, e);
#pragma unroll
        for (int i = 0; i < RMAX; ++i) w[i] = fld ? make_float2(e[i], d[i]) : make_float2(d[i], e[i]);
        fft_line<N, false, WARP, MASK>(w, t, sm, tw);
#pragma unroll
        for (int i = 0; i < RMAX; ++i) {
            const float m = inv_k2(__ldg(&a.k2x[pos_spec<N>(t, i)]));
            w[i] = make_float2(w[i].x * m, w[i].y * m);
        }
        fft_line<N, true, WARP, MASK>(w, t, sm, tw);
    };
    auto pot = [&](int i) { return fld ? w[i].y : w[i].x; };
    // per-cell sums of the pair at output o (the line of field 0 stores them); the pending half kick
    // (hk != 0) applied to copies
    auto moments = [&](int o, float hk, float hk_lo) {
        float2 z[RMAX];
        float x[RMAX], y[RMAX];
        int bad = 0;
        const bool quantum = has && slot > 0;  // slot 0 is the classical field
#pragma unroll
        for (int i = 0; i < RMAX; ++i) {
            // |psi|^2 does not depend on the pending kick (a phase): densities from the field, the
            // mean field from the kicked copy
            z[i] = hk != 0.f ? kick_w(v[i], hk, hk_lo, pot(i)) : v[i];
            bad += (has && (!isfinite(v[i].x) || !isfinite(v[i].y))) ? 1 : 0;
            x[i] = quantum ? fmaf(v[i].x, v[i].x, v[i].y * v[i].y) : 0.f;
            if (active && slot == 0)
                r.part_cl[(long long)o * N + pos_nat<N>(t, i)] = (double)v[i].x * v[i].x + (double)v[i].y * v[i].y;
        }
        // the pair's sums in FP64 (the partner's float values, converted exactly)
        double* pp = r.part + ((long long)o * a.n_pairs + pe) * 3 * N;
        const bool store = active && fld == 0;
        swap_f(x, y);
        if (store) {
#pragma unroll
            for (int i = 0; i < RMAX; ++i) pp[pos_nat<N>(t, i)] = (double)x[i] + (double)y[i];
        }
#pragma unroll
        for (int i = 0; i < RMAX; ++i) x[i] = quantum ? z[i].x : 0.f;
        swap_f(x, y);
        if (store) {
#pragma unroll
            for (int i = 0; i < RMAX; ++i) pp[N + pos_nat<N>(t, i)] = (double)x[i] + (double)y[i];
        }
#pragma unroll
        for (int i = 0; i < RMAX; ++i) x[i] = quantum ? z[i].y : 0.f;
        swap_f(x, y);
        if (store) {
#pragma unroll
            for (int i = 0; i < RMAX; ++i) pp[2 * N + pos_nat<N>(t, i)] = (double)x[i] + (double)y[i];
        }
        // non-finite counts of the pair: a shuffle sum over each line, then over the two lines when
        // they share a warp; otherwise integer-valued atomic adds (exact, order-free)
        if constexpr (T <= 32) {
#pragma unroll
            for (int o2 = T / 2; o2 > 0; o2 >>= 1) bad += __shfl_down_sync(MASK, bad, o2, T);
        }
        if constexpr (SHFL) {
            bad += __shfl_xor_sync(MASK, bad, T);
            if (store && t == 0) r.part_bad[(long long)o * a.n_pairs + p] = (double)bad;
        } else if (T <= 32) {
            if (active && t == 0 && bad) atomicAdd(&r.part_bad[(long long)o * a.n_pairs + p], (double)bad);
        } else if (active && bad) {
            atomicAdd(&r.part_bad[(long long)o * a.n_pairs + p], (double)bad);
        }
    };
    if constexpr (!SHFL) {
        // the bad-count slots of this launch start at zero (atomic adds)
        for (int o = 0; o <= r.n_out; ++o)
            if (active && fld == 0 && t == 0) r.part_bad[(long long)o * a.n_pairs + p] = 0.0;
        __syncthreads();
    }
    poisson();
    moments(0, 0.f, 0.f);
#pragma unroll 1
    for (int o = 1; o <= r.n_out; ++o) {
#pragma unroll 1
        for (int s = 0; s < r.out_every; ++s) {
            const bool first = o == 1 && s == 0;
            kick_all(v, first ? a.kick : a.kick2, first ? a.kick_lo : a.kick2_lo, pot);
            drift();
            poisson();
        }
        moments(o, a.kick, a.kick_lo);
    }
    // closing half kick: the batch ends synchronized
    kick_all(v, a.kick, a.kick_lo, pot);
    if (active && has) {
#pragma unroll
        for (int i = 0; i < RMAX; ++i) F[pos_nat<N>(t, i)] = v[i];
    }
}

template <int N>
int launch_run1d(const Run1DArgs& r, cudaStream_t st);

}  // namespace twa
