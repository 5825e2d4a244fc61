// misc.cu - sampling, kick, ensemble-moment and reduction kernels.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_engine.cuh"
#include "kernels.h"
#include "passes.cuh"
#include "reduce.cuh"

namespace twa {

// ---------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of two 32x32->64 multiplies; the
// key is bumped by the Weyl constants before every round after the first.
__device__ __forceinline__ void philox4x32_10(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3,
                                              uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
}

template <class T2>
__device__ __forceinline__ T2 make_c(double x, double y);
template <>
__device__ __forceinline__ float2 make_c<float2>(double x, double y) { return make_float2((float)x, (float)y); }
template <>
__device__ __forceinline__ double2 make_c<double2>(double x, double y) { return make_double2(x, y); }

// Eq. sample: slot 0 <- psi_cl; slot s >= 1 <- psi_cl + sigma (zR + i zI), zR, zI from Box-Muller
// on the first two Philox words of counter (cell, s, instance, 0), key = seed; arithmetic in FP64.
template <class T2>
__global__ void k_sample(const double2* __restrict__ psi_cl, T2* __restrict__ psi, long long cells,
                         int n_slots, uint32_t k0, uint32_t k1, uint32_t inst, double sigma) {
    const long long total = cells * n_slots;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int slot = (int)(idx / cells);
        const long long g = idx - (long long)slot * cells;
        double2 z = psi_cl[g];
        if (slot > 0) {
            uint32_t c0 = (uint32_t)g, c1 = (uint32_t)slot, c2 = inst, c3 = 0;
            philox4x32_10(c0, c1, c2, c3, k0, k1);
            const double u0 = ((double)c0 + 0.5) * (1.0 / 4294967296.0);
            const double u1 = ((double)c1 + 0.5) * (1.0 / 4294967296.0);
            const double r = sqrt(-2.0 * log(u0));
            double s, c;
            sincospi(2.0 * u1, &s, &c);
            z.x += sigma * (r * c);
            z.y += sigma * (r * s);
        }
        psi[idx] = make_c<T2>(z.x, z.y);
    }
}

// psi_s <- psi_s exp(-i kick V_s) for every slot, V of pair p packed in buf[p] (re: slot 2p, im: 2p+1).
__global__ void k_kick_pairs(float2* __restrict__ psi, const float2* __restrict__ buf, long long cells,
                             int n_slots, float kick, float kick_lo) {
    const long long total = cells * n_slots;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int slot = (int)(idx / cells);
        const long long g = idx - (long long)slot * cells;
        const float2 c = buf[(long long)(slot >> 1) * cells + g];
        psi[idx] = kick_w(psi[idx], kick, kick_lo, (slot & 1) ? c.y : c.x);
    }
}

// Running sum of floats carried as an unevaluated pair hi + lo ("double-float"): each addition's
// rounding error is recovered exactly (Knuth's two-sum) and the pair is renormalized (Dekker's
// fast two-sum), so the sum keeps about 48 significant bits.  The moment kernels accumulate in
// this form because this part's FP64 rate is 1/64 of its FP32 rate: FP64 adds would make them
// compute-bound at several times their memory time.  Results are finished in FP64.
struct DF {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float a) {
        const float s = hi + a;
        const float bp = s - hi;
        float e = (hi - (s - bp)) + (a - bp);  // hi + a = s + e exactly
        e += lo;
        hi = s + e;
        lo = e - (hi - s);
    }
    // add a * a exactly (the product's rounding error recovered with an fma)
    __device__ __forceinline__ void add_sq(float a) {
        const float p = a * a;
        const float q = fmaf(a, a, -p);
        add(p);
        lo += q;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// FP64 counterpart of DF for the plain FP64 path.
struct DAcc {
    double v = 0.0;
    __device__ __forceinline__ void add(double a) { v += a; }
    __device__ __forceinline__ double value() const { return v; }
};
template <class T2> struct AccOf;
template <> struct AccOf<float2> { using type = DF; using real = float; };
template <> struct AccOf<double2> { using type = DAcc; using real = double; };

// Amplitude and phase moments (Eq. varA, Eq. varPhi) of a synchronized instance, one thread per
// cell, two passes over the streams (slots 1..n): the first sums psi, |psi| and |psi|^2, the
// second the squared deviations (A_s - <A>)^2 and dphi_s^2, dphi_s = arg(psi_s conj(<psi>)) (0
// reference where the mean field vanishes).  Per block: sum of <rho> Var(A) / <A> and of
// <rho> <dphi^2>, <rho> the Weyl-corrected mean density.
template <class T2>
__global__ void k_phase_moments(const T2* __restrict__ psi, long long cells, int n_slots, double weyl,
                                double* var_a, double* phi2, double* part) {
    using Acc = typename AccOf<T2>::type;
    using R = typename AccOf<T2>::real;
    const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double v[2] = {0.0, 0.0};
    if (g < cells) {
        const int ns = n_slots - 1;
        Acc sa, sa2, sx, sy;
        for (int s = 1; s < n_slots; ++s) {
            const T2 z = psi[(long long)s * cells + g];
            const R a2 = z.x * z.x + z.y * z.y;
            sa.add(sqrt(a2));
            sa2.add(a2);
            sx.add(z.x);
            sy.add(z.y);
        }
        const double am = sa.value() / ns, mx = sx.value() / ns, my = sy.value() / ns;
        const double mm = sqrt(mx * mx + my * my);
        const R ux = (R)(mm > 0.0 ? mx / mm : 1.0), uy = (R)(mm > 0.0 ? my / mm : 0.0);
        Acc da, dp;
        for (int s = 1; s < n_slots; ++s) {
            const T2 z = psi[(long long)s * cells + g];
            const R d = sqrt(z.x * z.x + z.y * z.y) - (R)am;
            da.add(d * d);
            const R ph = atan2(z.y * ux - z.x * uy, z.x * ux + z.y * uy);  // arg(z conj(u))
            dp.add(ph * ph);
        }
        const double va = da.value() / ns, p2 = dp.value() / ns;
        const double rho = sa2.value() / ns - weyl;
        if (var_a) var_a[g] = va;
        if (phi2) phi2[g] = p2;
        v[0] = am > 0.0 ? rho * va / am : 0.0;
        v[1] = rho * p2;
    }
    block_reduce_store<2>(v, part);
}

// Sum the block partials in block order: out = {sum dV part_0, sum dV part_1 / (pi^2 / 3)}.
__global__ void k_finish_phase(const double* __restrict__ part, int nb, double dV, double* out) {
    __shared__ double red[2][256];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nb; i += 256) {
        a += part[2 * i];
        b += part[2 * i + 1];
    }
    red[0][threadIdx.x] = a;
    red[1][threadIdx.x] = b;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            red[0][threadIdx.x] += red[0][threadIdx.x + s];
            red[1][threadIdx.x] += red[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = red[0][0] * dV;
        out[1] = red[1][0] * dV / (3.14159265358979323846 * 3.14159265358979323846 / 3.0);
    }
}

// Position-space moments (Eq. E[op], Eq. Q) of one instance, one thread per cell, streams summed
// in slot order (each |psi|^2 is formed in FP32, exact to its rounding, and summed in double-float).
// The pending half kick (kick != 0) is applied on the fly to the mean field; |psi|^2 does not
// depend on it.  Four pairs are loaded per iteration to keep loads in flight.
__global__ void k_moments_real(const float2* __restrict__ psi, const float2* __restrict__ buf,
                               long long cells, int n_slots, float kick, float kick_lo, double inv_ns, double weyl,
                               double* rho_mean, double* psi_mean, double* rho_cl, double* part) {
    const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double v[NP_REAL] = {0, 0, 0, 0, 0, 0};
    if (g < cells) {
        DF m2, pr, pi;
        int bad = 0;
        auto add = [&](float2 z, float2 zk) {
            bad += (!isfinite(z.x) || !isfinite(z.y)) ? 1 : 0;
            m2.add(fmaf(z.x, z.x, z.y * z.y));
            pr.add(zk.x);
            pi.add(zk.y);
        };
        // slot 1 pairs with slot 0 (pair 0); then pairs p = 1.. hold slots 2p, 2p+1
        {
            const float2 z = psi[cells + g];
            float2 zk = z;
            if (kick != 0.f) zk = kick_w(z, kick, kick_lo, buf[g].y);
            if (n_slots > 1) add(z, zk);
        }
        const int np = (n_slots + 1) / 2;
        int p = 1;
        for (; p + 3 < np; p += 4) {
            float2 z[8], c[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                z[2 * u] = psi[(long long)(2 * (p + u)) * cells + g];
                z[2 * u + 1] = (2 * (p + u) + 1 < n_slots) ? psi[(long long)(2 * (p + u) + 1) * cells + g] : make_float2(0.f, 0.f);
                c[u] = (kick != 0.f) ? buf[(long long)(p + u) * cells + g] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                add(z[2 * u], kick != 0.f ? kick_w(z[2 * u], kick, kick_lo, c[u].x) : z[2 * u]);
                if (2 * (p + u) + 1 < n_slots)
                    add(z[2 * u + 1], kick != 0.f ? kick_w(z[2 * u + 1], kick, kick_lo, c[u].y) : z[2 * u + 1]);
            }
        }
        for (; p < np; ++p) {
            const float2 c = (kick != 0.f) ? buf[(long long)p * cells + g] : make_float2(0.f, 0.f);
            const float2 z0 = psi[(long long)(2 * p) * cells + g];
            add(z0, kick != 0.f ? kick_w(z0, kick, kick_lo, c.x) : z0);
            if (2 * p + 1 < n_slots) {
                const float2 z1 = psi[(long long)(2 * p + 1) * cells + g];
                add(z1, kick != 0.f ? kick_w(z1, kick, kick_lo, c.y) : z1);
            }
        }
        const float2 z0 = psi[g];
        const double cl = (double)z0.x * z0.x + (double)z0.y * z0.y;
        const double m2d = m2.value() * inv_ns, prd = pr.value() * inv_ns, pid = pi.value() * inv_ns;
        const double rm = m2d - weyl;
        if (rho_mean) rho_mean[g] = rm;
        if (psi_mean) {
            psi_mean[2 * g] = prd;
            psi_mean[2 * g + 1] = pid;
        }
        if (rho_cl) rho_cl[g] = cl;
        if (!isfinite(z0.x) || !isfinite(z0.y)) bad += 1;
        v[0] = m2d - (prd * prd + pid * pid);
        v[1] = (rm - cl) * (rm - cl);
        v[2] = cl * cl;
        v[3] = m2d;
        v[4] = cl;
        v[5] = (double)bad;
    }
    block_reduce_store<NP_REAL>(v, part);
}

// Per-mode moments: a_k = sqrt(n dV / M) FFT(psi_s)_k (spec holds FFT(psi_s) for every slot);
// |FFT|^2 formed in FP32; the sums of |FFT|^2 and of its exact square kept in double-float, scaled
// in FP64; eight slots loaded per iteration.
__global__ void k_moments_modes(const float2* __restrict__ spec, long long cells, int n_slots, double anorm2,
                                double inv_ns, double* nk_mean, double* nk_var, double* nk_cl, double* part) {
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double v[NP_MODES] = {0, 0};
    if (k < cells) {
        DF a2s, a4s;
        int s = 1;
        for (; s + 7 < n_slots; s += 8) {
            float2 z[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) z[u] = spec[(long long)(s + u) * cells + k];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float q = fmaf(z[u].x, z[u].x, z[u].y * z[u].y);
                a2s.add(q);
                a4s.add_sq(q);
            }
        }
        for (; s < n_slots; ++s) {
            const float2 z = spec[(long long)s * cells + k];
            const float q = fmaf(z.x, z.x, z.y * z.y);
            a2s.add(q);
            a4s.add_sq(q);
        }
        const double m2 = anorm2 * a2s.value() * inv_ns, m4 = anorm2 * anorm2 * a4s.value() * inv_ns;
        const double nk = m2 - 0.5;
        if (nk_mean) nk_mean[k] = nk;
        if (nk_var) nk_var[k] = m4 - m2 - nk * nk;
        if (nk_cl) {
            const float2 z = spec[k];
            nk_cl[k] = anorm2 * ((double)z.x * z.x + (double)z.y * z.y);
        }
        v[0] = nk;
    }
    block_reduce_store<NP_MODES>(v, part);
}

// Largest |re| or |im| over n complex values (the packed potentials of a batch), folded into *vmax
// as float bits: for non-negative floats the unsigned order of the bits is their numeric order.
// Non-finite values are skipped (the moments flag them).
__global__ void k_max_abs(const float2* __restrict__ buf, long long n, unsigned* vmax) {
    float m = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float2 v = __ldcg(&buf[i]);
        const float a = fmaxf(fabsf(v.x), fabsf(v.y));
        if (a <= 3.0e38f) m = fmaxf(m, a);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ float wm[32];
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, wm[w]);
        atomicMax(vmax, __float_as_uint(m));
    }
}

// Test particles (Sec. III.D, Eq. cl_int), one per slot: block s moves the particle of slot s,
// prt[6 s + (0..2)] = r, prt[6 s + 3 + (0..2)] = p.  The force -grad V = (C / cells) grad W uses W, the
// slot's real component of the packed Poisson field (real space): its spectral derivative along
// each axis at the 2^dim grid points around r is a periodic convolution of the axis line with the
// derivative kernel ker_a (one warp per corner and axis, FP64 sums), then interpolated multilinearly
// to r.  p += force kick_dt, then r += p drift_dt, wrapped into [0, L).
__global__ void k_particles(const float2* __restrict__ W, long long cells, int nx, int ny, int nz, int dim, double L,
                            const double* __restrict__ kx, const double* __restrict__ ky,
                            const double* __restrict__ kz, double fscale, double kick_dt, double drift_dt,
                            double* prt) {
    const int s = blockIdx.x;
    const float* Wc = reinterpret_cast<const float*>(W + (long long)(s >> 1) * cells) + (s & 1);
    double* q = prt + 6 * s;
    const int n[3] = {nx, ny, nz};
    const long long stride[3] = {1, nx, (long long)nx * ny};
    __shared__ double D[8][3];
    __shared__ int i0[3];
    __shared__ double fr[3];
    if (threadIdx.x < dim) {
        const int a = threadIdx.x;
        const double sc = q[a] / (L / n[a]);
        const double fl = floor(sc);
        long long i = (long long)fl % n[a];
        if (i < 0) i += n[a];
        i0[a] = (int)i;
        fr[a] = sc - fl;
    }
    __syncthreads();
    const int nc = 1 << dim;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int pr = warp; pr < nc * dim; pr += nw) {
        const int c = pr / dim, a = pr % dim;
        int j[3] = {0, 0, 0};
        for (int b = 0; b < dim; ++b) j[b] = (i0[b] + ((c >> b) & 1)) % n[b];
        const long long base = j[0] + (long long)nx * (j[1] + (long long)ny * j[2]) - (long long)j[a] * stride[a];
        const double* ker = a == 0 ? kx : (a == 1 ? ky : kz);
        double acc = 0.0;
        for (int m = lane; m < n[a]; m += 32) {
            int d = j[a] - m;
            if (d < 0) d += n[a];
            acc += ker[d] * (double)Wc[2 * (base + (long long)m * stride[a])];
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) D[c][a] = acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int a = 0; a < dim; ++a) {
            double g = 0.0;
            for (int c = 0; c < nc; ++c) {
                double w = 1.0;
                for (int b = 0; b < dim; ++b) w *= ((c >> b) & 1) ? fr[b] : 1.0 - fr[b];
                g += w * D[c][a];
            }
            const double p = q[3 + a] + fscale * g * kick_dt;
            double r = fmod(q[a] + p * drift_dt, L);
            if (r < 0.0) r += L;
            q[3 + a] = p;
            q[a] = r;
        }
    }
}

// Sum the per-block partials in block order and form the TWA_NSCALARS scalars of one instance.
__global__ void k_finish_scalars(const double* __restrict__ part_r, int nb_r, const double* __restrict__ part_m,
                                 int nb_m, double dV, double q_offset, double* scalars, int* err_word) {
    __shared__ double red[NP_REAL + NP_MODES][256];
    double v[NP_REAL + NP_MODES];
#pragma unroll
    for (int j = 0; j < NP_REAL + NP_MODES; ++j) v[j] = 0.0;
    for (int b = threadIdx.x; b < nb_r; b += 256)
        for (int j = 0; j < NP_REAL; ++j) v[j] += part_r[(long long)b * NP_REAL + j];
    for (int b = threadIdx.x; b < nb_m; b += 256)
        for (int j = 0; j < NP_MODES; ++j) v[NP_REAL + j] += part_m[(long long)b * NP_MODES + j];
    for (int j = 0; j < NP_REAL + NP_MODES; ++j) red[j][threadIdx.x] = v[j];
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int j = 0; j < NP_REAL + NP_MODES; ++j) red[j][threadIdx.x] += red[j][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double q = red[0][0] * dV - q_offset;
        const double d2 = sqrt(red[1][0]), c2 = sqrt(red[2][0]);
        scalars[0] = q;
        scalars[1] = d2 / c2;
        scalars[2] = red[3][0] * dV;
        scalars[3] = red[4][0] * dV;
        scalars[4] = red[5][0];
        scalars[5] = (nb_m > 0) ? red[NP_REAL][0] : 0.0;
        scalars[6] = d2;
        scalars[7] = c2;
        if (red[5][0] > 0.0 && err_word) atomicOr(err_word, 1);
    }
}

// Scalars of every output of a whole 1D run (block o = output o): per cell the pair partials of
// the run kernel added in pair order, then the cell sums of k_finish_scalars in a fixed tree order.
// Sum_k <n_k> follows from the streams' mass by Parseval's identity for the unitary DFT:
// sum_k mean|a_k|^2 = n_tot sum_g dV mean|psi_g|^2 (only written when modes are on, as elsewhere).
__global__ void k_finish_run1d(const double* __restrict__ part, const double* __restrict__ part_cl,
                               const double* __restrict__ part_bad, int n_pairs, int N, double inv_ns, double weyl,
                               double dV, double q_offset, double n_tot_modes, double* series, int row0, int inst,
                               int n_inst, int* err_word) {
    const int o = blockIdx.x;
    double v[NP_REAL] = {0, 0, 0, 0, 0, 0};
    for (int g = threadIdx.x; g < N; g += blockDim.x) {
        double m2 = 0.0, pr = 0.0, pi = 0.0;
        for (int p = 0; p < n_pairs; ++p) {
            const double* pp = part + ((long long)o * n_pairs + p) * 3 * N;
            m2 += pp[g];
            pr += pp[N + g];
            pi += pp[2 * N + g];
        }
        m2 *= inv_ns;
        pr *= inv_ns;
        pi *= inv_ns;
        const double cl = part_cl[(long long)o * N + g], rm = m2 - weyl;
        v[0] += m2 - (pr * pr + pi * pi);
        v[1] += (rm - cl) * (rm - cl);
        v[2] += cl * cl;
        v[3] += m2;
        v[4] += cl;
    }
    for (int p = threadIdx.x; p < n_pairs; p += blockDim.x) v[5] += part_bad[(long long)o * n_pairs + p];
    __shared__ double red[NP_REAL][256];
    for (int j = 0; j < NP_REAL; ++j) red[j][threadIdx.x] = v[j];
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int j = 0; j < NP_REAL; ++j) red[j][threadIdx.x] += red[j][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double* sc = series + ((long long)(row0 + o) * n_inst + inst) * 8;
        const double d2 = sqrt(red[1][0]), c2 = sqrt(red[2][0]);
        sc[0] = red[0][0] * dV - q_offset;
        sc[1] = d2 / c2;
        sc[2] = red[3][0] * dV;
        sc[3] = red[4][0] * dV;
        sc[4] = red[5][0];
        sc[5] = n_tot_modes > 0.0 ? n_tot_modes * sc[2] - 0.5 * N : 0.0;
        sc[6] = d2;
        sc[7] = c2;
        if (red[5][0] > 0.0 && err_word) atomicOr(err_word, 1);
    }
}

// Copy the current output's scalars into series[counter] and advance the device counter (keeps a
// captured graph identical across replays).
__global__ void k_store_series(const double* __restrict__ cur, double* series, int* counter, int n) {
    const int o = *counter;
    for (int j = threadIdx.x; j < n; j += blockDim.x) series[(long long)o * n + j] = cur[j];
    __syncthreads();
    if (threadIdx.x == 0) *counter = o + 1;
}

// ---------------------------------------------------------------------------------------------
// Host launchers.
int launch_sample_f32(const double2* psi_cl, float2* psi, long long cells, int n_slots, uint64_t seed,
                      int inst, double sigma, cudaStream_t st) {
    const long long total = cells * n_slots;
    const int blocks = (int)((total + 255) / 256 < 152 * 32 ? (total + 255) / 256 : 152 * 32);
    k_sample<float2><<<blocks, 256, 0, st>>>(psi_cl, psi, cells, n_slots, (uint32_t)seed,
                                             (uint32_t)(seed >> 32), (uint32_t)inst, sigma);
    return 0;
}
int launch_sample_f64(const double2* psi_cl, double2* psi, long long cells, int n_slots, uint64_t seed,
                      int inst, double sigma, cudaStream_t st) {
    const long long total = cells * n_slots;
    const int blocks = (int)((total + 255) / 256 < 152 * 32 ? (total + 255) / 256 : 152 * 32);
    k_sample<double2><<<blocks, 256, 0, st>>>(psi_cl, psi, cells, n_slots, (uint32_t)seed,
                                              (uint32_t)(seed >> 32), (uint32_t)inst, sigma);
    return 0;
}
int launch_kick_pairs(float2* psi, const float2* buf, long long cells, int n_slots, float kick, float kick_lo,
                      cudaStream_t st) {
    const long long total = cells * n_slots;
    const int blocks = (int)((total + 255) / 256 < 152 * 16 ? (total + 255) / 256 : 152 * 16);
    k_kick_pairs<<<blocks, 256, 0, st>>>(psi, buf, cells, n_slots, kick, kick_lo);
    return 0;
}
int moments_blocks(long long cells) { return (int)((cells + 255) / 256); }
int launch_moments_real(const float2* psi, const float2* buf, long long cells, int n_slots, float kick,
                        float kick_lo, double inv_ns, double weyl, double* rho_mean, double* psi_mean, double* rho_cl,
                        double* part, cudaStream_t st) {
    k_moments_real<<<moments_blocks(cells), 256, 0, st>>>(psi, buf, cells, n_slots, kick, kick_lo, inv_ns, weyl,
                                                          rho_mean, psi_mean, rho_cl, part);
    return 0;
}
int launch_moments_modes(const float2* spec, long long cells, int n_slots, double anorm2, double inv_ns,
                         double* nk_mean, double* nk_var, double* nk_cl, double* part, cudaStream_t st) {
    k_moments_modes<<<moments_blocks(cells), 256, 0, st>>>(spec, cells, n_slots, anorm2, inv_ns, nk_mean,
                                                           nk_var, nk_cl, part);
    return 0;
}
template <class T2>
int launch_phase_moments_t(const T2* psi, long long cells, int n_slots, double weyl, double dV, double* var_a,
                           double* phi2, double* part, double* out, cudaStream_t st) {
    const int nb = moments_blocks(cells);
    k_phase_moments<T2><<<nb, 256, 0, st>>>(psi, cells, n_slots, weyl, var_a, phi2, part);
    k_finish_phase<<<1, 256, 0, st>>>(part, nb, dV, out);
    return 0;
}
int launch_phase_moments(const float2* psi, long long cells, int n_slots, double weyl, double dV, double* var_a,
                         double* phi2, double* part, double* out, cudaStream_t st) {
    return launch_phase_moments_t(psi, cells, n_slots, weyl, dV, var_a, phi2, part, out, st);
}
int launch_phase_moments_f64(const double2* psi, long long cells, int n_slots, double weyl, double dV,
                             double* var_a, double* phi2, double* part, double* out, cudaStream_t st) {
    return launch_phase_moments_t(psi, cells, n_slots, weyl, dV, var_a, phi2, part, out, st);
}
int launch_finish_scalars(const double* part_r, int nb_r, const double* part_m, int nb_m, double dV,
                          double q_offset, double* scalars, int* err_word, cudaStream_t st) {
    k_finish_scalars<<<1, 256, 0, st>>>(part_r, nb_r, part_m, nb_m, dV, q_offset, scalars, err_word);
    return 0;
}
__global__ void k_poisson_multiplier(const float* __restrict__ k2, float* __restrict__ m, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        m[i] = inv_k2(k2[i]);
}
int launch_poisson_multiplier(const float* k2, float* m, long long n, cudaStream_t st) {
    if (n <= 0) return 0;
    const long long b = (n + 255) / 256;
    k_poisson_multiplier<<<(int)(b < 152 * 8 ? b : 152 * 8), 256, 0, st>>>(k2, m, n);
    return 0;
}
int launch_max_abs(const float2* buf, long long n, unsigned* vmax, cudaStream_t st) {
    const long long b = (n + 255) / 256;
    k_max_abs<<<(int)(b < 152 * 8 ? (b > 0 ? b : 1) : 152 * 8), 256, 0, st>>>(buf, n, vmax);
    return 0;
}
int launch_particles(const float2* W, long long cells, const int* n, int dim, double L, const double* const* ker,
                     double fscale, double kick_dt, double drift_dt, int n_slots, double* prt, cudaStream_t st) {
    k_particles<<<n_slots, 128, 0, st>>>(W, cells, n[0], n[1], n[2], dim, L, ker[0], ker[1], ker[2], fscale, kick_dt,
                                         drift_dt, prt);
    return 0;
}
int launch_finish_run1d(const double* part, const double* part_cl, const double* part_bad, int n_pairs, int N,
                        int n_outputs, double inv_ns, double weyl, double dV, double q_offset, double n_tot_modes,
                        double* series, int row0, int inst, int n_inst, int* err_word, cudaStream_t st) {
    k_finish_run1d<<<n_outputs, 256, 0, st>>>(part, part_cl, part_bad, n_pairs, N, inv_ns, weyl, dV, q_offset,
                                              n_tot_modes, series, row0, inst, n_inst, err_word);
    return 0;
}
int launch_store_series(const double* cur, double* series, int* counter, int n, cudaStream_t st) {
    k_store_series<<<1, 128, 0, st>>>(cur, series, counter, n);
    return 0;
}

}  // namespace twa
