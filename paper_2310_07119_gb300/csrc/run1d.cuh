// run1d.cuh - a whole 1D run (steps and moment sums of every output) in one launch.
//
// A 1D field is one line, so a pair of streams stays in the registers of T threads for the whole
// run (Sec. III.B.2's split step: kick, drift by FFT / kinetic phase / iFFT, density, Poisson solve
// by FFT / 1/k^2 / iFFT, all on chip).  At every output the pair's synchronized fields (the pending
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

template <int N, int LINES>
__global__ void __launch_bounds__(LINES * Plan<N>::T, 1)
k_run1d(const Run1DArgs r) {
    using P = Plan<N>;
    constexpr int T = P::T, RMAX = P::RMAX;
    constexpr int LS = line_stride_rows(N, T);
    constexpr bool WARP = T <= 32;
    constexpr unsigned MASK = (LINES * T >= 32) ? 0xffffffffu : ((1u << (LINES * T)) - 1u);
    extern __shared__ float2 smem[];
    const PassArgs& a = r.a;
    const int tid = threadIdx.x, l = tid / T, t = tid % T;
    float2* sm = smem + l * LS;
    const float4* tw = a.tw;
    const int p = (int)blockIdx.x * LINES + l;
    const bool active = p < a.n_pairs;
    const int pe = active ? p : a.n_pairs - 1;
    const bool has1 = 2 * pe + 1 < a.n_slots;
    float2* F0 = a.psi + (long long)(2 * pe) * N;
    float2* F1 = a.psi + (long long)(2 * pe + 1) * N;
    float2 v[RMAX], u[RMAX], w[RMAX];
#pragma unroll
    for (int i = 0; i < RMAX; ++i) {
        const int e = pos_nat<N>(t, i);
        v[i] = F0[e];
        u[i] = has1 ? F1[e] : make_float2(0.f, 0.f);
    }
    // (the two fields' transforms one after the other: interleaving them ran out of registers and
    // measured slower, 1.27e9 against 1.48e9 cell-updates/s on the 256-cell workload)
    auto drift = [&](float2 (&x)[RMAX]) {
        fft_line<N, false, WARP, MASK>(x, t, sm, tw);
#pragma unroll
        for (int i = 0; i < RMAX; ++i) {
            const float4 ph = __ldg(&a.ph[pos_spec<N>(t, i)]);
            x[i] = cmul_c(x[i], make_float2(ph.x, ph.y), make_float2(ph.z, ph.w));
        }
        fft_line<N, true, WARP, MASK>(x, t, sm, tw);
    };
    // packed potential of the pair: W = iFFT(FFT(|v|^2 + i |u|^2) / k^2)
    auto poisson = [&]() {
#pragma unroll
        for (int i = 0; i < RMAX; ++i)
            w[i] = make_float2(fmaf(v[i].x, v[i].x, v[i].y * v[i].y), fmaf(u[i].x, u[i].x, u[i].y * u[i].y));
        fft_line<N, false, WARP, MASK>(w, t, sm, tw);
#pragma unroll
        for (int i = 0; i < RMAX; ++i) {
            const float m = inv_k2(__ldg(&a.k2x[pos_spec<N>(t, i)]));
            w[i] = make_float2(w[i].x * m, w[i].y * m);
        }
        fft_line<N, true, WARP, MASK>(w, t, sm, tw);
    };
    // per-cell sums of the pair at output o; the pending half kick (hk != 0) applied to copies
    auto moments = [&](int o, float hk, float hk_lo) {
        double* pp = r.part + ((long long)o * a.n_pairs + pe) * 3 * N;
        int bad = 0;
#pragma unroll
        for (int i = 0; i < RMAX; ++i) {
            if (!active) break;
            const int e = pos_nat<N>(t, i);
            // |psi|^2 does not depend on the pending kick (a phase): densities from the fields,
            // the mean field from the kicked copies
            const float2 z0 = hk != 0.f ? kick_w(v[i], hk, hk_lo, w[i].x) : v[i];
            const float2 z1 = hk != 0.f ? kick_w(u[i], hk, hk_lo, w[i].y) : u[i];
            double m2 = 0.0, pr = 0.0, pi = 0.0;
            bad += (!isfinite(v[i].x) || !isfinite(v[i].y)) ? 1 : 0;
            if (p > 0) {
                m2 += (double)fmaf(v[i].x, v[i].x, v[i].y * v[i].y);
                pr += (double)z0.x;
                pi += (double)z0.y;
            } else {
                r.part_cl[(long long)o * N + e] = (double)v[i].x * v[i].x + (double)v[i].y * v[i].y;
            }
            if (has1) {
                bad += (!isfinite(u[i].x) || !isfinite(u[i].y)) ? 1 : 0;
                m2 += (double)fmaf(u[i].x, u[i].x, u[i].y * u[i].y);
                pr += (double)z1.x;
                pi += (double)z1.y;
            }
            pp[e] = m2;
            pp[N + e] = pr;
            pp[2 * N + e] = pi;
        }
        // non-finite counts of the T threads of the line: a shuffle sum when the line sits in one warp,
        // integer-valued atomic adds (exact, order-free) when it spans several
        // (every lane takes part in the shuffles; lines past the last pair carry 0 and store nothing)
        if constexpr (T <= 32) {
#pragma unroll
            for (int o2 = T / 2; o2 > 0; o2 >>= 1) bad += __shfl_down_sync(MASK, bad, o2, T);
            if (active && t == 0) r.part_bad[(long long)o * a.n_pairs + p] = (double)bad;
        } else if (active && bad) {
            atomicAdd(&r.part_bad[(long long)o * a.n_pairs + p], (double)bad);
        }
    };
    poisson();
    if constexpr (T > 32) {
        // the bad-count slots of this launch start at zero (atomic adds)
        for (int o = 0; o <= r.n_out; ++o)
            if (active && t == 0) r.part_bad[(long long)o * a.n_pairs + p] = 0.0;
        __syncthreads();
    }
    moments(0, 0.f, 0.f);
#pragma unroll 1
    for (int o = 1; o <= r.n_out; ++o) {
#pragma unroll 1
        for (int s = 0; s < r.out_every; ++s) {
            const bool first = o == 1 && s == 0;
            const float kk = first ? a.kick : a.kick2, kl = first ? a.kick_lo : a.kick2_lo;
            kick_all(v, kk, kl, [&](int i) { return w[i].x; });
            kick_all(u, kk, kl, [&](int i) { return w[i].y; });
            drift(v);
            drift(u);
            poisson();
        }
        moments(o, a.kick, a.kick_lo);
    }
    // closing half kick: the batch ends synchronized
    kick_all(v, a.kick, a.kick_lo, [&](int i) { return w[i].x; });
    kick_all(u, a.kick, a.kick_lo, [&](int i) { return w[i].y; });
    if (active) {
#pragma unroll
        for (int i = 0; i < RMAX; ++i) {
            const int e = pos_nat<N>(t, i);
            F0[e] = v[i];
            if (has1) F1[e] = u[i];
        }
    }
}

template <int N>
int launch_run1d(const Run1DArgs& r, cudaStream_t st);

}  // namespace twa
