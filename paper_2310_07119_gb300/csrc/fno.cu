// fno.cu - Fourier-neural-operator surrogate of the TWA correction spectrum: forward, backward,
// AdamW, with BF16 weights (FP32 master copy) and FP32 accumulation.
//
// Network (features on the grid of Fourier modes of an n^3 field, layout [B][C][n][n][n]):
//   h_0 = P x + p;  z_l = Re A^H (R_l . A h_l) + W_l h_l + b_l;  h_{l+1} = gelu(z_l) (l < L-1);
//   y = Q h_L + q.
// A is the unitary 3D DFT restricted to the frequencies |m_a| < modes on each axis, applied as three
// axis transforms with (2 modes) x n complex matrices; A^H is its adjoint.  R_l holds one complex
// W x W matrix per retained mode.  All reductions (weight gradients, the loss) run in a fixed
// order, so training is bitwise reproducible.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "reduce.cuh"
#include "tc_gemm.h"
#include "twa.h"

void twa_set_global_error(const std::string& msg);

namespace {

constexpr int kThreads = 256;
constexpr int kPwBlocks = 152 * 2;  // CTAs of the pointwise weight-gradient stage 1 (and its partials)

int blocks_for(long long n) {
    const long long b = (n + kThreads - 1) / kThreads;
    return (int)(b < 152LL * 64 ? b : 152LL * 64);
}

__device__ __forceinline__ float bf(const __nv_bfloat16* w, long long i) { return __bfloat162float(w[i]); }

// Y[b][o][k] = sum_c W[o][c] X[b][c][k] + bias[o] (+ Y if accumulate); TRANS reads W as [c][o].
template <bool TRANS>
__global__ void k_pointwise(const float* __restrict__ X, const __nv_bfloat16* __restrict__ Wt,
                            const float* __restrict__ bias, float* __restrict__ Y, int B, int cin, int cout,
                            long long K, int accumulate) {
    extern __shared__ float wsm[];
    for (int i = threadIdx.x; i < cin * cout; i += blockDim.x) wsm[i] = __bfloat162float(Wt[i]);
    __syncthreads();
    const long long total = (long long)B * K;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long b = t / K, k = t - b * K;
        float x[64];
#pragma unroll 4
        for (int c = 0; c < cin; ++c) x[c] = X[(b * cin + c) * K + k];
        for (int o = 0; o < cout; ++o) {
            float acc = bias ? bias[o] : 0.f;
            for (int c = 0; c < cin; ++c) acc = fmaf(TRANS ? wsm[c * cout + o] : wsm[o * cin + c], x[c], acc);
            float* y = &Y[(b * cout + o) * K + k];
            *y = accumulate ? *y + acc : acc;
        }
    }
}

// Stage 1 of dW[o][c] = sum_{b,k} dY[b][o][k] X[b][c][k] and db[o] = sum dY: block (o, chunk) sums a
// fixed chunk of positions; stage 2 adds the chunks in order.
__global__ void k_pointwise_wgrad_part(const float* __restrict__ dY, const float* __restrict__ X, int B, int cin,
                                       int cout, long long K, int nchunk, float* __restrict__ part) {
    const int o = blockIdx.x, ch = blockIdx.y;
    const long long total = (long long)B * K;
    const long long per = (total + nchunk - 1) / nchunk;
    const long long lo = ch * per, hi = (lo + per < total) ? lo + per : total;
    float acc[65];
    for (int c = 0; c <= cin; ++c) acc[c] = 0.f;
    for (long long t = lo + threadIdx.x; t < hi; t += blockDim.x) {
        const long long b = t / K, k = t - b * K;
        const float g = dY[(b * cout + o) * K + k];
        for (int c = 0; c < cin; ++c) acc[c] = fmaf(g, X[(b * cin + c) * K + k], acc[c]);
        acc[cin] += g;
    }
    __shared__ float red[kThreads];
    for (int c = 0; c <= cin; ++c) {
        red[threadIdx.x] = acc[c];
        __syncthreads();
        for (int s = kThreads / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[((long long)o * nchunk + ch) * (cin + 1) + c] = red[0];
        __syncthreads();
    }
}

__global__ void k_pointwise_wgrad_sum(const float* __restrict__ part, int cin, int cout, int nchunk,
                                      float* __restrict__ dW, float* __restrict__ db) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cout * (cin + 1)) return;
    const int o = i / (cin + 1), c = i % (cin + 1);
    float s = 0.f;
    for (int ch = 0; ch < nchunk; ++ch) s += part[((long long)o * nchunk + ch) * (cin + 1) + c];
    if (c < cin) dW[o * cin + c] += s;
    else db[o] += s;
}

// out[p][i][q] = sum_j M[i][j] in[p][j][q] (complex M, nout x nin); in may be real; out may keep the
// real part only (then optionally added to out).
__global__ void k_axis(const float2* __restrict__ in_c, const float* __restrict__ in_r, const float2* __restrict__ M,
                       float2* __restrict__ out_c, float* __restrict__ out_r, long long P, int nin, int nout,
                       long long Q, int accumulate) {
    const long long total = P * nout * Q;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long q = t % Q;
        const long long r = t / Q;
        const int i = (int)(r % nout);
        const long long p = r / nout;
        float ar = 0.f, ai = 0.f;
        for (int j = 0; j < nin; ++j) {
            const float2 m = M[i * nin + j];
            const long long src = (p * nin + j) * Q + q;
            if (in_r) {
                const float x = in_r[src];
                ar = fmaf(m.x, x, ar);
                ai = fmaf(m.y, x, ai);
            } else {
                const float2 x = in_c[src];
                ar = fmaf(m.x, x.x, fmaf(-m.y, x.y, ar));
                ai = fmaf(m.x, x.y, fmaf(m.y, x.x, ai));
            }
        }
        if (out_r) out_r[t] = accumulate ? out_r[t] + ar : ar;
        else out_c[t] = make_float2(ar, ai);
    }
}

// Ymix[b][o][m] = sum_c R[m][o][c] S[b][c][m]  (R complex, BF16 re/im); ADJ: dS[b][c][m] = sum_o conj(R[m][o][c]) G[b][o][m]
template <bool ADJ>
__global__ void k_mix(const float2* __restrict__ S, const __nv_bfloat16* __restrict__ R, float2* __restrict__ Y, int B,
                      int W, long long Mm) {
    const long long total = (long long)B * W * Mm;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long m = t % Mm;
        const long long r = t / Mm;
        const int o = (int)(r % W);
        const long long b = r / W;
        float ar = 0.f, ai = 0.f;
        for (int c = 0; c < W; ++c) {
            const long long ri = ADJ ? ((m * W + c) * W + o) * 2 : ((m * W + o) * W + c) * 2;
            const float rr = bf(R, ri), rim = ADJ ? -bf(R, ri + 1) : bf(R, ri + 1);
            const float2 x = S[(b * W + c) * Mm + m];
            ar = fmaf(rr, x.x, fmaf(-rim, x.y, ar));
            ai = fmaf(rr, x.y, fmaf(rim, x.x, ai));
        }
        Y[t] = make_float2(ar, ai);
    }
}

// dR[m][o][c] += sum_b G[b][o][m] conj(S[b][c][m])   (re/im interleaved in the flat gradient)
__global__ void k_mix_wgrad(const float2* __restrict__ G, const float2* __restrict__ S, float* __restrict__ dR, int B,
                            int W, long long Mm) {
    const long long total = Mm * W * W;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(t % W);
        const long long r = t / W;
        const int o = (int)(r % W);
        const long long m = r / W;
        float ar = 0.f, ai = 0.f;
        for (int b = 0; b < B; ++b) {
            const float2 g = G[((long long)b * W + o) * Mm + m];
            const float2 s = S[((long long)b * W + c) * Mm + m];
            ar = fmaf(g.x, s.x, fmaf(g.y, s.y, ar));
            ai = fmaf(g.y, s.x, fmaf(-g.x, s.y, ai));
        }
        dR[2 * t] += ar;
        dR[2 * t + 1] += ai;
    }
}

// ---------------------------------------------------------------------------------------------
// Restructured contractions (same sums, same order per output; fewer passes over the inputs).

// out[p][i][q] = sum_j M[i][j] in[p][j][q] (as k_axis): one thread per (p, q) and group of up to AG
// outputs i, so every input value is read once per group; M is staged in shared memory and read
// by the whole warp at the same address.
constexpr int AG = 16;
__global__ void k_axis_g(const float2* __restrict__ in_c, const float* __restrict__ in_r, const float2* __restrict__ M,
                         float2* __restrict__ out_c, float* __restrict__ out_r, long long P, int nin, int nout, long long Q,
                         int accumulate) {
    extern __shared__ float2 Ms[];
    for (int i = threadIdx.x; i < nin * nout; i += blockDim.x) Ms[i] = M[i];
    __syncthreads();
    const int ng = (nout + AG - 1) / AG;
    const long long total = P * ng * Q;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long q = t % Q;
        const long long r = t / Q;
        const int g = (int)(r % ng);
        const long long p = r / ng;
        const int i0 = g * AG;
        float ar[AG], ai[AG];
#pragma unroll
        for (int u = 0; u < AG; ++u) ar[u] = ai[u] = 0.f;
        for (int j = 0; j < nin; ++j) {
            const long long src = (p * nin + j) * Q + q;
            if (in_r) {
                const float x = in_r[src];
#pragma unroll
                for (int u = 0; u < AG; ++u) {
                    const float2 m = Ms[min(i0 + u, nout - 1) * nin + j];
                    ar[u] = fmaf(m.x, x, ar[u]);
                    ai[u] = fmaf(m.y, x, ai[u]);
                }
            } else {
                const float2 x = in_c[src];
#pragma unroll
                for (int u = 0; u < AG; ++u) {
                    const float2 m = Ms[min(i0 + u, nout - 1) * nin + j];
                    ar[u] = fmaf(m.x, x.x, fmaf(-m.y, x.y, ar[u]));
                    ai[u] = fmaf(m.x, x.y, fmaf(m.y, x.x, ai[u]));
                }
            }
        }
#pragma unroll
        for (int u = 0; u < AG; ++u) {
            const int i = i0 + u;
            if (i >= nout) break;
            const long long dst = (p * nout + i) * Q + q;
            if (out_r) out_r[dst] = accumulate ? out_r[dst] + ar[u] : ar[u];
            else out_c[dst] = make_float2(ar[u], ai[u]);
        }
    }
}

// k_mix with a CTA per block of MB modes: the modes' R matrices (W x W complex BF16) and the inputs
// of every batch element for them are staged in shared memory, so R is read from memory once per
// call instead of once per batch element.  Thread (x, mm): x = output channel (o, or c for ADJ).
template <bool ADJ>
__global__ void k_mix_g(const float2* __restrict__ S, const __nv_bfloat16* __restrict__ R, float2* __restrict__ Y, int B,
                        int W, long long Mm, int MB) {
    extern __shared__ float2 sm[];
    float2* Rs = sm;                              // [MB][W][W]
    float2* Ss = sm + (size_t)MB * W * W;         // [B][W][MB]
    const int x = threadIdx.x % W, mm = threadIdx.x / W;
    for (long long m0 = (long long)blockIdx.x * MB; m0 < Mm; m0 += (long long)gridDim.x * MB) {
        const int nm = (int)min((long long)MB, Mm - m0);
        __syncthreads();
        for (int i = threadIdx.x; i < nm * W * W; i += blockDim.x) {
            const long long ri = (m0 * W * W + i) * 2;
            Rs[i] = make_float2(bf(R, ri), bf(R, ri + 1));
        }
        for (int i = threadIdx.x; i < B * W * MB; i += blockDim.x) {
            const int k = i % MB, bc = i / MB;
            Ss[i] = (k < nm) ? S[(long long)bc * Mm + m0 + k] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        if (mm < nm) {
            for (int b = 0; b < B; ++b) {
                float ar = 0.f, ai = 0.f;
                for (int c = 0; c < W; ++c) {
                    const float2 r = ADJ ? Rs[((size_t)mm * W + c) * W + x] : Rs[((size_t)mm * W + x) * W + c];
                    const float rim = ADJ ? -r.y : r.y;
                    const float2 v = Ss[((size_t)b * W + c) * MB + mm];
                    ar = fmaf(r.x, v.x, fmaf(-rim, v.y, ar));
                    ai = fmaf(r.x, v.y, fmaf(rim, v.x, ai));
                }
                Y[((long long)b * W + x) * Mm + m0 + mm] = make_float2(ar, ai);
            }
        }
    }
}

// k_mix_wgrad with a CTA per block of MB modes: G and S of those modes staged in shared memory, one
// thread per (o, c) pair of a mode, writes consecutive in c.
__global__ void k_mix_wgrad_g(const float2* __restrict__ G, const float2* __restrict__ S, float* __restrict__ dR, int B,
                              int W, long long Mm, int MB) {
    extern __shared__ float2 sm[];
    float2* Gs = sm;                         // [B][W][MB]
    float2* Ss = sm + (size_t)B * W * MB;    // [B][W][MB]
    for (long long m0 = (long long)blockIdx.x * MB; m0 < Mm; m0 += (long long)gridDim.x * MB) {
        const int nm = (int)min((long long)MB, Mm - m0);
        __syncthreads();
        for (int i = threadIdx.x; i < B * W * MB; i += blockDim.x) {
            const int k = i % MB, bc = i / MB;
            const bool in = k < nm;
            Gs[i] = in ? G[(long long)bc * Mm + m0 + k] : make_float2(0.f, 0.f);
            Ss[i] = in ? S[(long long)bc * Mm + m0 + k] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < nm * W * W; i += blockDim.x) {
            const int c = i % W, o = (i / W) % W, mm = i / (W * W);
            float ar = 0.f, ai = 0.f;
            for (int b = 0; b < B; ++b) {
                const float2 g = Gs[((size_t)b * W + o) * MB + mm];
                const float2 v = Ss[((size_t)b * W + c) * MB + mm];
                ar = fmaf(g.x, v.x, fmaf(g.y, v.y, ar));
                ai = fmaf(g.y, v.x, fmaf(-g.x, v.y, ai));
            }
            const long long t = (m0 + mm) * W * W + (long long)o * W + c;
            dR[2 * t] += ar;
            dR[2 * t + 1] += ai;
        }
    }
}

// Stage 1 of the pointwise weight gradient with a CTA per chunk of positions: dY and X of CH
// positions staged in shared memory, each thread accumulating a few of the cout x (cin + 1) sums
// over its CTA's chunks; part[(o * nblk + blk) * (cin + 1) + c] (stage 2 as before).
constexpr int PW_CH = 64, PW_LD = PW_CH + 1;  // positions per chunk; padded row (distinct banks per channel)
__global__ void k_pointwise_wgrad_g(const float* __restrict__ dY, const float* __restrict__ X, int B, int cin, int cout,
                                    long long K, float* __restrict__ part) {
    extern __shared__ float sm2[];
    float* Ys = sm2;                         // [cout][PW_LD]
    float* Xs = sm2 + (size_t)cout * PW_LD;  // [cin][PW_LD]
    const int nout = cout * (cin + 1);
    constexpr int MAXO = 8;
    float acc[MAXO];
#pragma unroll
    for (int u = 0; u < MAXO; ++u) acc[u] = 0.f;
    const long long kchunks = (K + PW_CH - 1) / PW_CH, total = (long long)B * kchunks;
    for (long long ch = blockIdx.x; ch < total; ch += gridDim.x) {
        const long long b = ch / kchunks, k0 = (ch % kchunks) * PW_CH;
        const int nk = (int)min((long long)PW_CH, K - k0);
        __syncthreads();
        for (int i = threadIdx.x; i < cout * PW_CH; i += blockDim.x) {
            const int o = i / PW_CH, k = i % PW_CH;
            Ys[o * PW_LD + k] = k < nk ? dY[(b * cout + o) * K + k0 + k] : 0.f;
        }
        for (int i = threadIdx.x; i < cin * PW_CH; i += blockDim.x) {
            const int c = i / PW_CH, k = i % PW_CH;
            Xs[c * PW_LD + k] = k < nk ? X[(b * cin + c) * K + k0 + k] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < MAXO; ++u) {
            const int j = threadIdx.x + u * blockDim.x;
            if (j >= nout) break;
            const int o = j / (cin + 1), c = j % (cin + 1);
            const float* yr = Ys + (size_t)o * PW_LD;
            float a = acc[u];
            if (c < cin) {
                const float* xr = Xs + (size_t)c * PW_LD;
                for (int k = 0; k < PW_CH; ++k) a = fmaf(yr[k], xr[k], a);
            } else {
                for (int k = 0; k < PW_CH; ++k) a += yr[k];
            }
            acc[u] = a;
        }
    }
#pragma unroll
    for (int u = 0; u < MAXO; ++u) {
        const int j = threadIdx.x + u * blockDim.x;
        if (j >= nout) break;
        const int o = j / (cin + 1), c = j % (cin + 1);
        part[((long long)o * gridDim.x + blockIdx.x) * (cin + 1) + c] = acc[u];
    }
}

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_g(float z) {
    return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

__global__ void k_gelu(const float* __restrict__ z, float* __restrict__ h, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        h[i] = gelu_f(z[i]);
}
__global__ void k_gelu_bwd(const float* __restrict__ dh, const float* __restrict__ z, float* __restrict__ dz, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dz[i] = dh[i] * gelu_g(z[i]);
}

// MSE: per-block partial sums of (y - t)^2 and dy = 2 (y - t) / n; then a fixed-order final sum.
__global__ void k_mse_part(const float* __restrict__ y, const float* __restrict__ t, long long n, float* __restrict__ dy,
                           double* __restrict__ part) {
    double acc[1] = {0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float d = y[i] - t[i];
        acc[0] += (double)d * d;
        if (dy) dy[i] = 2.f * d / (float)n;
    }
    twa::block_reduce_store<1>(acc, part);
}
__global__ void k_mse_final(const double* __restrict__ part, int nb, long long n, float* __restrict__ loss) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += part[b];
        *loss = (float)(s / (double)n);
    }
}

__global__ void k_adamw(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                        __nv_bfloat16* __restrict__ th16, long long n, float lr, float b1, float b2, float eps, float wd,
                        float c1, float c2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float upd = (mi / c1) / (sqrtf(vi / c2) + eps) + wd * th[i];
        const float t = th[i] - lr * upd;
        th[i] = t;
        th16[i] = __float2bfloat16(t);
    }
}

__global__ void k_to_bf16(const float* __restrict__ a, __nv_bfloat16* __restrict__ b, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = __float2bfloat16(a[i]);
}

}  // namespace

// ---------------------------------------------------------------------------------------------
struct twa_fno {
    twa_fno_config cfg{};
    long long n_params = 0;
    // offsets into the flat parameter vector
    long long oP = 0, op = 0, oQ = 0, oq = 0;
    std::vector<long long> oR, oW, ob;
    float* th = nullptr;            // FP32 master
    __nv_bfloat16* th16 = nullptr;  // BF16 copy used by the kernels
    float* grad = nullptr;
    float* am = nullptr;
    float* av = nullptr;
    long long step = 0;
    float2* Mf[3] = {nullptr, nullptr, nullptr};  // forward truncated DFT per axis (2m x n)
    float2* Mi[3] = {nullptr, nullptr, nullptr};  // adjoint (n x 2m)
    // the x-axis (contiguous) contractions as real GEMMs on the tensor cores (tc_gemm.cu):
    // Bf [npf][n]: rows (Re, Im) of the 2m DFT rows; Ba [npa][4m]: per cell the (Re, -Im) of its adjoint row
    float* Bf = nullptr;
    float* Ba = nullptr;
    int npf = 0, npa = 0;
    bool tc_fwd = false, tc_adj = false, tc_on = true;
    int* d_err = nullptr;
    // activations for the largest batch seen
    int cap_b = 0;
    std::vector<float*> h, z;
    std::vector<float2*> s;
    float2* t1 = nullptr;
    float2* t2 = nullptr;
    float2* mixed = nullptr;
    float* dh = nullptr;
    float* dz = nullptr;
    float* dh2 = nullptr;
    float* part = nullptr;
    double* lpart = nullptr;
    const float* x_in = nullptr;
    int last_b = 0;
    std::vector<void*> allocs;
    std::string err;
};

namespace {

int ffail(twa_fno* f, int code, const std::string& m) {
    if (f) f->err = m;
    twa_set_global_error(m);
    return code;
}

#define FC(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) return ffail(f, TWA_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <class T>
int falloc(twa_fno* f, T** p, size_t n) {
    if (cudaMalloc((void**)p, (n ? n : 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return ffail(f, TWA_ENOMEM, "twa_fno: cudaMalloc failed");
    }
    f->allocs.push_back(*p);
    return 0;
}

long long kcells(const twa_fno* f) { return (long long)f->cfg.grid * f->cfg.grid * f->cfg.grid; }
long long kmodes(const twa_fno* f) {
    const long long m2 = 2LL * f->cfg.modes;
    return m2 * m2 * m2;
}

int ensure_batch(twa_fno* f, int B) {
    if (B <= f->cap_b) return 0;
    for (float* p : f->h) cudaFree(p);
    for (float* p : f->z) cudaFree(p);
    for (float2* p : f->s) cudaFree(p);
    for (void* p : {(void*)f->t1, (void*)f->t2, (void*)f->mixed, (void*)f->dh, (void*)f->dz, (void*)f->dh2})
        if (p) cudaFree(p);
    std::vector<void*> keep;
    for (void* p : f->allocs) {
        bool act = false;
        for (float* q : f->h) act |= (p == q);
        for (float* q : f->z) act |= (p == q);
        for (float2* q : f->s) act |= (p == (void*)q);
        for (void* q : {(void*)f->t1, (void*)f->t2, (void*)f->mixed, (void*)f->dh, (void*)f->dz, (void*)f->dh2})
            act |= (p == q && q);
        if (!act) keep.push_back(p);
    }
    f->allocs = keep;
    const int L = f->cfg.layers, W = f->cfg.width, n = f->cfg.grid, m2 = 2 * f->cfg.modes;
    const long long K = kcells(f), Mm = kmodes(f);
    f->h.assign(L + 1, nullptr);
    f->z.assign(L, nullptr);
    f->s.assign(L, nullptr);
    for (int l = 0; l <= L; ++l)
        if (int rc = falloc(f, &f->h[l], (size_t)B * W * K)) return rc;
    for (int l = 0; l < L; ++l) {
        if (int rc = falloc(f, &f->z[l], (size_t)B * W * K)) return rc;
        if (int rc = falloc(f, &f->s[l], (size_t)B * W * Mm)) return rc;
    }
    const size_t tsz = (size_t)B * W * n * n * (size_t)(m2 > n ? m2 : n);
    if (int rc = falloc(f, &f->t1, tsz)) return rc;
    if (int rc = falloc(f, &f->t2, tsz)) return rc;
    if (int rc = falloc(f, &f->mixed, (size_t)B * W * Mm)) return rc;
    if (int rc = falloc(f, &f->dh, (size_t)B * W * K)) return rc;
    if (int rc = falloc(f, &f->dz, (size_t)B * W * K)) return rc;
    if (int rc = falloc(f, &f->dh2, (size_t)B * W * K)) return rc;
    f->cap_b = B;
    return 0;
}

// Axis contraction: the grouped kernel when M fits in shared memory, else the per-output one.
void axis_launch(const twa_fno* f, int blocks, int threads, int smem0, cudaStream_t st, const float2* in_c,
                 const float* in_r, const float2* M, float2* out_c, float* out_r, long long P, int nin, int nout,
                 long long Q, int accumulate) {
    (void)f;
    (void)smem0;
    const size_t sm = (size_t)nin * nout * sizeof(float2);
    if (sm <= 48 * 1024) {
        const long long work = P * ((nout + AG - 1) / AG) * Q;
        k_axis_g<<<blocks_for(work), threads, sm, st>>>(in_c, in_r, M, out_c, out_r, P, nin, nout, Q, accumulate);
    } else {
        k_axis<<<blocks, threads, 0, st>>>(in_c, in_r, M, out_c, out_r, P, nin, nout, Q, accumulate);
    }
}

// Modes per CTA of the mixing kernels (W threads per mode) and their shared memory.
int mix_modes(int W) { return kThreads / W > 0 ? kThreads / W : 1; }

template <bool ADJ>
void mix_launch(const float2* S, const __nv_bfloat16* R, float2* Y, int B, int W, long long Mm, cudaStream_t st) {
    const int MB = mix_modes(W);
    const size_t sm = ((size_t)MB * W * W + (size_t)B * W * MB) * sizeof(float2);
    if (W <= kThreads && sm <= 100 * 1024) {
        static size_t set = 0;
        if (sm > set) {
            cudaFuncSetAttribute(k_mix_g<ADJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            set = sm;
        }
        const long long nb = (Mm + MB - 1) / MB;
        k_mix_g<ADJ><<<(int)(nb < 152LL * 8 ? nb : 152LL * 8), MB * W, sm, st>>>(S, R, Y, B, W, Mm, MB);
    } else {
        k_mix<ADJ><<<blocks_for((long long)B * W * Mm), kThreads, 0, st>>>(S, R, Y, B, W, Mm);
    }
}

void mix_wgrad_launch(const float2* G, const float2* S, float* dR, int B, int W, long long Mm, cudaStream_t st) {
    const int MB = mix_modes(W);
    const size_t sm = (size_t)2 * B * W * MB * sizeof(float2);
    if (sm <= 100 * 1024) {
        static size_t set = 0;
        if (sm > set) {
            cudaFuncSetAttribute(k_mix_wgrad_g, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            set = sm;
        }
        const long long nb = (Mm + MB - 1) / MB;
        k_mix_wgrad_g<<<(int)(nb < 152LL * 8 ? nb : 152LL * 8), kThreads, sm, st>>>(G, S, dR, B, W, Mm, MB);
    } else {
        k_mix_wgrad<<<blocks_for(Mm * W * W), kThreads, 0, st>>>(G, S, dR, B, W, Mm);
    }
}

// A (truncated forward DFT) of a real [B*W][n][n][n] field into complex [B*W][2m][2m][2m].
void dft_fwd(twa_fno* f, const float* in, float2* out, long long BW, cudaStream_t st) {
    const int n = f->cfg.grid, m2 = 2 * f->cfg.modes;
    // x axis (last): (BW*n*n, n, 1) -> (BW*n*n, 2m, 1); on the tensor cores when the shape allows
    if (!(f->tc_on && f->tc_fwd &&
          twa::tc_gemm(in, BW * n * n, n, n, f->Bf, 2 * m2, f->npf, reinterpret_cast<float*>(f->t1), 2 * m2, 0, f->d_err,
                  2.0, st) == 0))
        axis_launch(f, blocks_for(BW * n * n * m2), kThreads, 0, st, nullptr, in, f->Mf[2], f->t1, nullptr, BW * n * n, n, m2, 1,
                                                                  0);
    // y axis: (BW*n, n, 2m) -> (BW*n, 2m, 2m)
    axis_launch(f, blocks_for(BW * n * m2 * m2), kThreads, 0, st, f->t1, nullptr, f->Mf[1], f->t2, nullptr, BW * n, n, m2, m2, 0);
    // z axis: (BW, n, 4m^2) -> (BW, 2m, 4m^2)
    axis_launch(f, blocks_for(BW * m2 * m2 * m2), kThreads, 0, st, f->t2, nullptr, f->Mf[0], out, nullptr, BW, n, m2,
                                                               (long long)m2 * m2, 0);
}

// Re A^H of complex [BW][2m][2m][2m] into a real [BW][n][n][n] field (overwrite or add).
void dft_adj(twa_fno* f, const float2* in, float* out, long long BW, int accumulate, cudaStream_t st) {
    const int n = f->cfg.grid, m2 = 2 * f->cfg.modes;
    axis_launch(f, blocks_for(BW * n * m2 * m2), kThreads, 0, st, in, nullptr, f->Mi[0], f->t1, nullptr, BW, m2, n,
                                                              (long long)m2 * m2, 0);
    axis_launch(f, blocks_for(BW * n * n * m2), kThreads, 0, st, f->t1, nullptr, f->Mi[1], f->t2, nullptr, BW * n, m2, n, m2, 0);
    if (!(f->tc_on && f->tc_adj &&
          twa::tc_gemm(reinterpret_cast<const float*>(f->t2), BW * n * n, 2 * m2, 2 * m2, f->Ba, n, f->npa, out, n, accumulate,
                  f->d_err, 2.0, st) == 0))
        axis_launch(f, blocks_for(BW * n * n * n), kThreads, 0, st, f->t2, nullptr, f->Mi[2], nullptr, out, BW * n * n, m2, n,
                                                                1, accumulate);
}

void pointwise(const float* X, const __nv_bfloat16* W, const float* b, float* Y, int B, int cin, int cout, long long K,
               int acc, bool trans, cudaStream_t st) {
    const size_t sm = (size_t)cin * cout * sizeof(float);
    if (trans)
        k_pointwise<true><<<blocks_for((long long)B * K), kThreads, sm, st>>>(X, W, b, Y, B, cin, cout, K, acc);
    else
        k_pointwise<false><<<blocks_for((long long)B * K), kThreads, sm, st>>>(X, W, b, Y, B, cin, cout, K, acc);
}

void pointwise_wgrad(twa_fno* f, const float* dY, const float* X, int B, int cin, int cout, long long K, float* dW,
                     float* db, cudaStream_t st) {
    if ((long long)cout * (cin + 1) <= 8LL * kThreads) {
        const int nblk = kPwBlocks;
        const size_t sm = (size_t)(cin + cout) * PW_LD * sizeof(float);
        k_pointwise_wgrad_g<<<nblk, kThreads, sm, st>>>(dY, X, B, cin, cout, K, f->part);
        k_pointwise_wgrad_sum<<<(cout * (cin + 1) + 127) / 128, 128, 0, st>>>(f->part, cin, cout, nblk, dW, db);
        return;
    }
    const int nchunk = 64;
    k_pointwise_wgrad_part<<<dim3(cout, nchunk), kThreads, 0, st>>>(dY, X, B, cin, cout, K, nchunk, f->part);
    k_pointwise_wgrad_sum<<<(cout * (cin + 1) + 127) / 128, 128, 0, st>>>(f->part, cin, cout, nchunk, dW, db);
}

}  // namespace

extern "C" {

int twa_fno_create(twa_fno** out, const twa_fno_config* cfg, uint64_t seed) {
    twa_fno* f = nullptr;
    if (!out || !cfg) return ffail(nullptr, TWA_EINVAL, "twa_fno_create: null argument");
    *out = nullptr;
    const twa_fno_config c = *cfg;
    if (c.grid < 4 || c.grid > 128 || c.width < 1 || c.width > 64 || c.modes < 1 || 2 * c.modes > c.grid ||
        c.layers < 1 || c.c_in < 1 || c.c_in > 64 || c.c_out < 1 || c.c_out > 64 ||
        2LL * (2 * c.modes) * (2 * c.modes) * (2 * c.modes) > (long long)c.grid * c.grid * c.grid)
        return ffail(nullptr, TWA_EINVAL,
                     "twa_fno_create: sizes out of range (grid <= 128; width, c_in, c_out <= 64; 2 (2 modes)^3 <= grid^3)");
    f = new twa_fno();
    f->cfg = c;
    const int W = c.width, L = c.layers;
    const long long Mm = kmodes(f);
    long long o = 0;
    f->oP = o; o += (long long)W * c.c_in;
    f->op = o; o += W;
    for (int l = 0; l < L; ++l) {
        f->oR.push_back(o); o += Mm * W * W * 2;
        f->oW.push_back(o); o += (long long)W * W;
        f->ob.push_back(o); o += W;
    }
    f->oQ = o; o += (long long)c.c_out * W;
    f->oq = o; o += c.c_out;
    f->n_params = o;
    auto bail = [&](int rc) {
        twa_fno_destroy(f);
        return rc;
    };
    int rc;
    if ((rc = falloc(f, &f->th, o)) || (rc = falloc(f, &f->th16, o)) || (rc = falloc(f, &f->grad, o)) ||
        (rc = falloc(f, &f->am, o)) || (rc = falloc(f, &f->av, o)))
        return bail(rc);
    const int maxc = (W > c.c_in ? W : c.c_in) > c.c_out ? (W > c.c_in ? W : c.c_in) : c.c_out;
    if ((rc = falloc(f, &f->part, (size_t)maxc * (kPwBlocks > 64 ? kPwBlocks : 64) * (maxc + 1))) ||
        (rc = falloc(f, &f->lpart, (size_t)152 * 64)))
        return bail(rc);
    // truncated unitary DFT matrices (FP64 on the host), kept frequencies {0..m-1} U {n-m..n-1}
    const int n = c.grid, m2 = 2 * c.modes;
    std::vector<float2> mf((size_t)m2 * n), mi((size_t)n * m2);
    for (int i = 0; i < m2; ++i) {
        const int k = (i < c.modes) ? i : n - m2 + i;
        for (int j = 0; j < n; ++j) {
            const double a = -2.0 * M_PI * (double)k * (double)j / (double)n, s = 1.0 / std::sqrt((double)n);
            mf[(size_t)i * n + j] = make_float2((float)(std::cos(a) * s), (float)(std::sin(a) * s));
            mi[(size_t)j * m2 + i] = make_float2((float)(std::cos(a) * s), (float)(-std::sin(a) * s));
        }
    }
    for (int a = 0; a < 3; ++a) {
        if ((rc = falloc(f, &f->Mf[a], mf.size())) || (rc = falloc(f, &f->Mi[a], mi.size()))) return bail(rc);
        cudaMemcpy(f->Mf[a], mf.data(), mf.size() * sizeof(float2), cudaMemcpyHostToDevice);
        cudaMemcpy(f->Mi[a], mi.data(), mi.size() * sizeof(float2), cudaMemcpyHostToDevice);
    }
    // real forms of the x-axis matrices for the tensor-core GEMMs (rows past 2 m2 / n stay zero)
    f->npf = (2 * m2 + 15) / 16 * 16;
    f->npa = (n + 15) / 16 * 16;
    f->tc_fwd = twa::tc_gemm_supported(n, f->npf);
    f->tc_adj = twa::tc_gemm_supported(2 * m2, f->npa);
    if ((rc = falloc(f, &f->d_err, 1))) return bail(rc);
    cudaMemset(f->d_err, 0, sizeof(int));
    if (f->tc_fwd) {
        std::vector<float> bf((size_t)f->npf * n, 0.f);
        for (int i = 0; i < m2; ++i)
            for (int j = 0; j < n; ++j) {
                bf[(size_t)(2 * i) * n + j] = mf[(size_t)i * n + j].x;
                bf[(size_t)(2 * i + 1) * n + j] = mf[(size_t)i * n + j].y;
            }
        if ((rc = falloc(f, &f->Bf, bf.size()))) return bail(rc);
        cudaMemcpy(f->Bf, bf.data(), bf.size() * sizeof(float), cudaMemcpyHostToDevice);
    }
    if (f->tc_adj) {
        std::vector<float> ba((size_t)f->npa * 2 * m2, 0.f);
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < m2; ++i) {
                ba[(size_t)j * 2 * m2 + 2 * i] = mi[(size_t)j * m2 + i].x;
                ba[(size_t)j * 2 * m2 + 2 * i + 1] = -mi[(size_t)j * m2 + i].y;
            }
        if ((rc = falloc(f, &f->Ba, ba.size()))) return bail(rc);
        cudaMemcpy(f->Ba, ba.data(), ba.size() * sizeof(float), cudaMemcpyHostToDevice);
    }
    // initial weights: uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) for pointwise maps, scale 1/(W^2) for R,
    // zero biases, from a fixed linear-congruential stream of the seed (host side)
    std::vector<float> h0((size_t)o, 0.f);
    uint64_t st = seed * 6364136223846793005ULL + 1442695040888963407ULL;
    auto uni = [&]() {
        st = st * 6364136223846793005ULL + 1442695040888963407ULL;
        return ((double)(st >> 11) / 9007199254740992.0) * 2.0 - 1.0;
    };
    for (long long i = 0; i < (long long)W * c.c_in; ++i) h0[f->oP + i] = (float)(uni() / std::sqrt((double)c.c_in));
    for (int l = 0; l < L; ++l) {
        for (long long i = 0; i < Mm * W * W * 2; ++i) h0[f->oR[l] + i] = (float)(uni() / ((double)W * W));
        for (long long i = 0; i < (long long)W * W; ++i) h0[f->oW[l] + i] = (float)(uni() / std::sqrt((double)W));
    }
    for (long long i = 0; i < (long long)c.c_out * W; ++i) h0[f->oQ + i] = (float)(uni() / std::sqrt((double)W));
    cudaMemcpy(f->th, h0.data(), o * sizeof(float), cudaMemcpyHostToDevice);
    k_to_bf16<<<blocks_for(o), kThreads>>>(f->th, f->th16, o);
    cudaMemset(f->am, 0, o * sizeof(float));
    cudaMemset(f->av, 0, o * sizeof(float));
    cudaMemset(f->grad, 0, o * sizeof(float));
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        return bail(ffail(f, TWA_ECUDA, "twa_fno_create: setup failed"));
    }
    *out = f;
    return TWA_OK;
}

int twa_fno_destroy(twa_fno* f) {
    if (!f) return TWA_OK;
    for (void* p : f->allocs) cudaFree(p);
    delete f;
    return TWA_OK;
}

long long twa_fno_num_params(const twa_fno* f) { return f ? f->n_params : 0; }

int twa_fno_set_params(twa_fno* f, const float* src, void* stream) {
    if (!f || !src) return ffail(f, TWA_EINVAL, "twa_fno_set_params: null argument");
    cudaStream_t st = (cudaStream_t)stream;
    FC(cudaMemcpyAsync(f->th, src, f->n_params * sizeof(float), cudaMemcpyDeviceToDevice, st));
    k_to_bf16<<<blocks_for(f->n_params), kThreads, 0, st>>>(f->th, f->th16, f->n_params);
    FC(cudaMemsetAsync(f->am, 0, f->n_params * sizeof(float), st));
    FC(cudaMemsetAsync(f->av, 0, f->n_params * sizeof(float), st));
    f->step = 0;
    FC(cudaGetLastError());
    return TWA_OK;
}

int twa_fno_get_params(twa_fno* f, float* dst, int which, void* stream) {
    if (!f || !dst) return ffail(f, TWA_EINVAL, "twa_fno_get_params: null argument");
    const float* src = which == 1 ? f->grad : f->th;
    FC(cudaMemcpyAsync(dst, src, f->n_params * sizeof(float), cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return TWA_OK;
}

int twa_fno_forward(twa_fno* f, const float* x, int B, float* y, void* stream) {
    if (!f || !x || !y || B < 1) return ffail(f, TWA_EINVAL, "twa_fno_forward: bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    if (int rc = ensure_batch(f, B)) return rc;
    const int W = f->cfg.width, L = f->cfg.layers;
    const long long K = kcells(f), Mm = kmodes(f), BW = (long long)B * W;
    const __nv_bfloat16* P = f->th16;
    pointwise(x, P + f->oP, f->th + f->op, f->h[0], B, f->cfg.c_in, W, K, 0, false, st);
    for (int l = 0; l < L; ++l) {
        dft_fwd(f, f->h[l], f->s[l], BW, st);
        mix_launch<false>(f->s[l], P + f->oR[l], f->mixed, B, W, Mm, st);
        dft_adj(f, f->mixed, f->z[l], BW, 0, st);
        pointwise(f->h[l], P + f->oW[l], f->th + f->ob[l], f->z[l], B, W, W, K, 1, false, st);
        if (l < L - 1)
            k_gelu<<<blocks_for(BW * K), kThreads, 0, st>>>(f->z[l], f->h[l + 1], BW * K);
        else
            FC(cudaMemcpyAsync(f->h[l + 1], f->z[l], BW * K * sizeof(float), cudaMemcpyDeviceToDevice, st));
    }
    pointwise(f->h[L], P + f->oQ, f->th + f->oq, y, B, W, f->cfg.c_out, K, 0, false, st);
    f->x_in = x;
    f->last_b = B;
    FC(cudaGetLastError());
    return TWA_OK;
}

int twa_fno_backward(twa_fno* f, const float* dy, int B, float* dx, void* stream) {
    if (!f || !dy || B != f->last_b || !f->x_in) return ffail(f, TWA_EINVAL, "twa_fno_backward: call after twa_fno_forward with the same batch");
    cudaStream_t st = (cudaStream_t)stream;
    const int W = f->cfg.width, L = f->cfg.layers;
    const long long K = kcells(f), Mm = kmodes(f), BW = (long long)B * W;
    const __nv_bfloat16* P = f->th16;
    float* g = f->grad;
    pointwise_wgrad(f, dy, f->h[L], B, W, f->cfg.c_out, K, g + f->oQ, g + f->oq, st);
    pointwise(dy, P + f->oQ, nullptr, f->dh, B, f->cfg.c_out, W, K, 0, true, st);
    for (int l = L - 1; l >= 0; --l) {
        float* dzl = f->dz;
        if (l < L - 1)
            k_gelu_bwd<<<blocks_for(BW * K), kThreads, 0, st>>>(f->dh, f->z[l], dzl, BW * K);
        else
            FC(cudaMemcpyAsync(dzl, f->dh, BW * K * sizeof(float), cudaMemcpyDeviceToDevice, st));
        pointwise_wgrad(f, dzl, f->h[l], B, W, W, K, g + f->oW[l], g + f->ob[l], st);
        pointwise(dzl, P + f->oW[l], nullptr, f->dh2, B, W, W, K, 0, true, st);
        // spectral branch: dmixed = A dz, dR += dmixed conj(s), ds = R^H dmixed, dh += Re A^H ds
        dft_fwd(f, dzl, f->mixed, BW, st);
        mix_wgrad_launch(f->mixed, f->s[l], g + f->oR[l], B, W, Mm, st);
        mix_launch<true>(f->mixed, P + f->oR[l], reinterpret_cast<float2*>(f->dz), B, W, Mm, st);
        // f->dz now holds ds (complex, B*W*Mm <= B*W*K floats / 2 since Mm <= K / 8)
        dft_adj(f, reinterpret_cast<float2*>(f->dz), f->dh2, BW, 1, st);
        std::swap(f->dh, f->dh2);
    }
    pointwise_wgrad(f, f->dh, f->x_in, B, f->cfg.c_in, W, K, g + f->oP, g + f->op, st);
    if (dx) pointwise(f->dh, P + f->oP, nullptr, dx, B, W, f->cfg.c_in, K, 0, true, st);
    FC(cudaGetLastError());
    return TWA_OK;
}

int twa_fno_zero_grad(twa_fno* f, void* stream) {
    if (!f) return ffail(nullptr, TWA_EINVAL, "null model");
    FC(cudaMemsetAsync(f->grad, 0, f->n_params * sizeof(float), (cudaStream_t)stream));
    return TWA_OK;
}

int twa_fno_adamw(twa_fno* f, float lr, float beta1, float beta2, float eps, float weight_decay, void* stream) {
    if (!f) return ffail(nullptr, TWA_EINVAL, "null model");
    f->step += 1;
    const float c1 = 1.f - (float)std::pow((double)beta1, (double)f->step);
    const float c2 = 1.f - (float)std::pow((double)beta2, (double)f->step);
    k_adamw<<<blocks_for(f->n_params), kThreads, 0, (cudaStream_t)stream>>>(f->th, f->grad, f->am, f->av, f->th16,
                                                                          f->n_params, lr, beta1, beta2, eps,
                                                                          weight_decay, c1, c2);
    FC(cudaGetLastError());
    return TWA_OK;
}

int twa_fno_mse(twa_fno* f, const float* y, const float* t, long long n, float* loss, float* dy, void* stream) {
    if (!f || !y || !t || !loss || n < 1) return ffail(f, TWA_EINVAL, "twa_fno_mse: bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    const int nb = 152 * 4;
    k_mse_part<<<nb, 256, 0, st>>>(y, t, n, dy, f->lpart);
    k_mse_final<<<1, 32, 0, st>>>(f->lpart, nb, n, loss);
    FC(cudaGetLastError());
    return TWA_OK;
}

const char* twa_fno_last_error(const twa_fno* f) { return f ? f->err.c_str() : ""; }

int twa_fno_set_tensor_cores(twa_fno* f, int on) {
    if (!f) return ffail(nullptr, TWA_EINVAL, "twa_fno_set_tensor_cores: null handle");
    f->tc_on = on != 0;
    return TWA_OK;
}

int twa_fno_tensor_core_shapes(const twa_fno* f) {
    if (!f) return 0;
    return (f->tc_fwd ? 1 : 0) | (f->tc_adj ? 2 : 0);
}

int twa_fno_sync_status(twa_fno* f, void* stream) {
    if (!f) return ffail(nullptr, TWA_EINVAL, "twa_fno_sync_status: null handle");
    FC(cudaStreamSynchronize((cudaStream_t)stream));
    int w = 0;
    FC(cudaMemcpy(&w, f->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    FC(cudaMemset(f->d_err, 0, sizeof(int)));
    if (w & twa::TC_ERR_TIMEOUT_BIT) return ffail(f, TWA_ETIMEOUT, "a tensor-core GEMM wait gave up");
    return TWA_OK;
}

int twa_tc_gemm(const float* A, long long P, long long K, long long lda, const float* Bt, int N, int Np, float* C,
                long long ldc, int accumulate, int* err, void* stream) {
    if (!A || !Bt || !C || !err || P <= 0 || N <= 0 || N > Np || lda < K || ldc < N)
        return ffail(nullptr, TWA_EINVAL, "twa_tc_gemm: bad argument");
    const int rc = twa::tc_gemm(A, P, K, lda, Bt, N, Np, C, ldc, accumulate, err, 2.0, (cudaStream_t)stream);
    if (rc == -1)
        return ffail(nullptr, TWA_EINVAL,
                     "twa_tc_gemm: unsupported shape or alignment (K a multiple of 32 up to 128, Np a multiple of 16 "
                     "in [16, 256], 16-byte aligned A and Bt, lda * 4 a multiple of 16)");
    if (rc) return ffail(nullptr, TWA_ECUDA, "twa_tc_gemm: tensor map or launch failed");
    return TWA_OK;
}

}  // extern "C"

namespace {
// Features of one TWA snapshot on the mode grid (FFT index order), with nu = n_tot / grid^3 the mean
// occupation per mode:
//   x0 = log10(1 + n_cl) / 8,  x1 = (n_est - n_cl) / (n_cl + nu),  x2 = log10(n_tot) - 9,
//   x3 = |m| / (grid / 2);   target t = (n_ref - n_cl) / (n_cl + nu)  (the correction spectrum relative
// to the occupation, floored at the mean occupation).
__global__ void k_features(const double* __restrict__ ncl, const double* __restrict__ nest, const double* __restrict__ nref,
                           double lg_ntot, double nu, int n, float* __restrict__ x, float* __restrict__ t) {
    const long long K = (long long)n * n * n;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < K; k += (long long)gridDim.x * blockDim.x) {
        const double c = ncl[k];
        const double sc = 1.0 / ((c > 0.0 ? c : 0.0) + nu);
        const int ix = (int)(k % n), iy = (int)((k / n) % n), iz = (int)(k / ((long long)n * n));
        const double mx = ix < n / 2 ? ix : ix - n, my = iy < n / 2 ? iy : iy - n, mz = iz < n / 2 ? iz : iz - n;
        x[k] = (float)(log10(1.0 + (c > 0.0 ? c : 0.0)) / 8.0);
        x[K + k] = (float)((nest[k] - c) * sc);
        x[2 * K + k] = (float)(lg_ntot - 9.0);
        x[3 * K + k] = (float)(sqrt(mx * mx + my * my + mz * mz) / (0.5 * n));
        if (t) t[k] = (float)((nref[k] - c) * sc);
    }
}
}  // namespace

extern "C" int twa_fno_features(const double* nk_cl, const double* nk_est, const double* nk_ref, double n_tot, int grid,
                                float* x, float* t, void* stream) {
    if (!nk_cl || !nk_est || !x || grid < 2 || (t && !nk_ref) || !(n_tot > 0)) {
        twa_set_global_error("twa_fno_features: bad argument");
        return TWA_EINVAL;
    }
    const long long K = (long long)grid * grid * grid;
    k_features<<<blocks_for(K), kThreads, 0, (cudaStream_t)stream>>>(nk_cl, nk_est, nk_ref, std::log10(n_tot),
                                                                    n_tot / (double)K, grid, x, t);
    if (cudaGetLastError() != cudaSuccess) {
        twa_set_global_error("twa_fno_features: launch failed");
        return TWA_ECUDA;
    }
    return TWA_OK;
}

extern "C" {

}  // extern "C"
