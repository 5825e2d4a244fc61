// plain_f64.cu - plain FP64 single-realization comparator path (complex128, no fusion).
//
// The same split step as the batched path (Sec. III.B.2, Eq. mft_normed) written the plain way:
// every FFT axis, the kinetic phase, the density, the Poisson multiplier and the kick are separate
// kernels, one realization per launch.  The FFT is a radix-2 Stockham transform of one line per CTA.
#include <cuda_runtime.h>

#include "kernels.h"
#include "reduce.cuh"

namespace twa {

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

// One line of length N (stride S) per CTA; lines are (q, o) with base q + o OS, q < Qn.
__global__ void k64_fft_line(double2* f, int N, long long S, int Qn, long long OS, const double2* __restrict__ tw,
                             int inv) {
    extern __shared__ double2 sm64[];
    double2* a = sm64;
    double2* b = sm64 + N;
    const long long L = blockIdx.x;
    const long long base = (L % Qn) + (L / Qn) * OS;
    for (int i = threadIdx.x; i < N; i += blockDim.x) a[i] = f[base + i * S];
    __syncthreads();
    for (int ns = 1; ns < N; ns *= 2) {
        for (int j = threadIdx.x; j < N / 2; j += blockDim.x) {
            const int k = j & (ns - 1);
            double2 w = tw[k * (N / (2 * ns))];
            if (inv) w.y = -w.y;
            const double2 v0 = a[j];
            const double2 v1 = zmul(a[j + N / 2], w);
            const int d = (j / ns) * ns * 2 + k;
            b[d] = make_double2(v0.x + v1.x, v0.y + v1.y);
            b[d + ns] = make_double2(v0.x - v1.x, v0.y - v1.y);
        }
        __syncthreads();
        double2* t = a;
        a = b;
        b = t;
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) f[base + i * S] = a[i];
}

__device__ __forceinline__ void coords(long long e, const int* n, int& x, int& y, int& z) {
    x = (int)(e % n[0]);
    const long long r = e / n[0];
    y = (int)(r % n[1]);
    z = (int)(r / n[1]);
}

struct G64 {
    int n[3];
    long long cells;
};

// f <- f exp(-i hbar k^2 dt / 2) / cells (product of the per-axis factors)
__global__ void k64_kinetic(double2* f, G64 g, const double2* px, const double2* py, const double2* pz) {
    const double sc = 1.0 / (double)g.cells;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < g.cells; e += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        coords(e, g.n, x, y, z);
        const double2 ph = zmul(zmul(px[x], py[y]), pz[z]);
        const double2 v = zmul(f[e], ph);
        f[e] = make_double2(v.x * sc, v.y * sc);
    }
}

__global__ void k64_rho(const double2* psi, double2* work, long long cells) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < cells; e += (long long)gridDim.x * blockDim.x) {
        const double2 z = psi[e];
        work[e] = make_double2(z.x * z.x + z.y * z.y, 0.0);
    }
}

// V_k = -C rho_k / (k^2 cells), V_0 = 0
__global__ void k64_poisson_mul(double2* w, G64 g, const double* kx, const double* ky, const double* kz, double mulc) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < g.cells; e += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        coords(e, g.n, x, y, z);
        const double k2 = kx[x] + ky[y] + kz[z];
        const double m = (k2 > 0.0) ? mulc / k2 : 0.0;
        w[e] = make_double2(w[e].x * m, w[e].y * m);
    }
}

// psi <- psi exp(-i kick V), V = Re(work); the phase is reduced mod 2 pi in FP64.
__global__ void k64_kick(double2* psi, const double2* work, long long cells, double kick) {
    const double two_pi = 6.283185307179586476925286766559;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < cells; e += (long long)gridDim.x * blockDim.x) {
        double th = kick * work[e].x;
        th = th - two_pi * rint(th / two_pi);
        double s, c;
        sincos(th, &s, &c);
        const double2 z = psi[e];
        psi[e] = make_double2(z.x * c + z.y * s, z.y * c - z.x * s);
    }
}

// Running per-cell sums over realizations (first = 1 initializes): acc = (sum |psi|^2, sum re, sum im).
__global__ void k64_moments_accum(const double2* psi, long long cells, int first, double* acc, double* bad) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < cells; e += (long long)gridDim.x * blockDim.x) {
        const double2 z = psi[e];
        const double m = z.x * z.x + z.y * z.y;
        if (first) {
            acc[e] = m;
            acc[cells + e] = z.x;
            acc[2 * cells + e] = z.y;
        } else {
            acc[e] += m;
            acc[cells + e] += z.x;
            acc[2 * cells + e] += z.y;
        }
        if (!isfinite(z.x) || !isfinite(z.y)) atomicAdd(bad, 1.0);
    }
}

__global__ void k64_modes_accum(const double2* spec, long long cells, double anorm2, int first, double* acc2) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < cells; e += (long long)gridDim.x * blockDim.x) {
        const double2 z = spec[e];
        const double a2 = anorm2 * (z.x * z.x + z.y * z.y);
        if (first) {
            acc2[e] = a2;
            acc2[cells + e] = a2 * a2;
        } else {
            acc2[e] += a2;
            acc2[cells + e] += a2 * a2;
        }
    }
}

__global__ void k64_moments_finish(const double* acc, const double* acc2, const double2* psi0, long long cells, int n_real,
                                   double weyl, double* rho_mean, double* psi_mean, double* rho_cl, double* nk_mean,
                                   double* nk_var, double* part_r, double* part_m, const double* bad) {
    const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double vr[NP_REAL] = {0, 0, 0, 0, 0, 0};
    double vm[NP_MODES] = {0, 0};
    const double inv = 1.0 / n_real;
    if (g < cells) {
        const double m2 = acc[g] * inv, pr = acc[cells + g] * inv, pi = acc[2 * cells + g] * inv;
        const double2 z0 = psi0[g];
        const double cl = z0.x * z0.x + z0.y * z0.y;
        const double rm = m2 - weyl;
        if (rho_mean) rho_mean[g] = rm;
        if (psi_mean) {
            psi_mean[2 * g] = pr;
            psi_mean[2 * g + 1] = pi;
        }
        if (rho_cl) rho_cl[g] = cl;
        vr[0] = m2 - (pr * pr + pi * pi);
        vr[1] = (rm - cl) * (rm - cl);
        vr[2] = cl * cl;
        vr[3] = m2;
        vr[4] = cl;
        vr[5] = (g == 0) ? *bad : 0.0;
        if (acc2) {
            const double a2 = acc2[g] * inv, a4 = acc2[cells + g] * inv;
            const double nk = a2 - 0.5;
            if (nk_mean) nk_mean[g] = nk;
            if (nk_var) nk_var[g] = a4 - a2 - nk * nk;
            vm[0] = nk;
        }
    }
    block_reduce_store<NP_REAL>(vr, part_r);
    if (part_m) block_reduce_store<NP_MODES>(vm, part_m);
}

static int ew_blocks(long long n) {
    const long long b = (n + 255) / 256;
    return (int)(b < 152 * 16 ? b : 152 * 16);
}

int launch_f64_fft3(double2* f, const Geom64& g, const Tables64& t, bool inverse, cudaStream_t st, long long* nl) {
    static bool big_smem = false;
    if (!big_smem) {
        if (cudaFuncSetAttribute(k64_fft_line, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 2048 * (int)sizeof(double2)) !=
            cudaSuccess)
            return -3;
        big_smem = true;
    }
    long long stride = 1;
    for (int a = 0; a < g.dim; ++a) {
        const int N = g.n[a];
        const int Qn = (int)stride;
        const long long OS = stride * N;
        const long long lines = g.cells / N;
        const int thr = N / 2 < 256 ? (N / 2 > 32 ? N / 2 : 32) : 256;
        k64_fft_line<<<(unsigned)lines, thr, 2 * N * sizeof(double2), st>>>(f, N, stride, Qn, OS, t.tw[a], inverse ? 1 : 0);
        ++*nl;
        stride *= N;
    }
    return 0;
}
int launch_f64_kinetic(double2* f, const Geom64& g, const Tables64& t, cudaStream_t st, long long* nl) {
    G64 gg{{g.n[0], g.n[1], g.n[2]}, g.cells};
    k64_kinetic<<<ew_blocks(g.cells), 256, 0, st>>>(f, gg, t.ph[0], t.ph[1], t.ph[2]);
    ++*nl;
    return 0;
}
int launch_f64_rho(const double2* psi, double2* work, long long cells, cudaStream_t st, long long* nl) {
    k64_rho<<<ew_blocks(cells), 256, 0, st>>>(psi, work, cells);
    ++*nl;
    return 0;
}
int launch_f64_poisson_mul(double2* work, const Geom64& g, const Tables64& t, double mulc, cudaStream_t st, long long* nl) {
    G64 gg{{g.n[0], g.n[1], g.n[2]}, g.cells};
    k64_poisson_mul<<<ew_blocks(g.cells), 256, 0, st>>>(work, gg, t.k2[0], t.k2[1], t.k2[2], mulc);
    ++*nl;
    return 0;
}
int launch_f64_kick(double2* psi, const double2* work, long long cells, double kick, cudaStream_t st, long long* nl) {
    k64_kick<<<ew_blocks(cells), 256, 0, st>>>(psi, work, cells, kick);
    ++*nl;
    return 0;
}
int launch_f64_moments_accum(const double2* psi, const double2* /*work*/, long long cells, double /*kick*/, int first,
                             double* acc, double* bad, cudaStream_t st, long long* nl) {
    k64_moments_accum<<<ew_blocks(cells), 256, 0, st>>>(psi, cells, first, acc, bad);
    ++*nl;
    return 0;
}
int launch_f64_modes_accum(const double2* spec, long long cells, double anorm2, int first, double* acc2, cudaStream_t st,
                           long long* nl) {
    k64_modes_accum<<<ew_blocks(cells), 256, 0, st>>>(spec, cells, anorm2, first, acc2);
    ++*nl;
    return 0;
}
int launch_f64_moments_finish(const double* acc, const double* acc2, const double2* psi0, long long cells, int n_real,
                              double weyl, double dV, double q_offset, double* rho_mean, double* psi_mean,
                              double* rho_cl, double* nk_mean, double* nk_var, double* part_r, double* part_m,
                              const double* bad, double* scalars, int* err_word, cudaStream_t st, long long* nl) {
    const int nb = (int)((cells + 255) / 256);
    k64_moments_finish<<<nb, 256, 0, st>>>(acc, acc2, psi0, cells, n_real, weyl, rho_mean, psi_mean, rho_cl, nk_mean,
                                            nk_var, part_r, acc2 ? part_m : nullptr, bad);
    ++*nl;
    launch_finish_scalars(part_r, nb, part_m, acc2 ? nb : 0, dV, q_offset, scalars, err_word, st);
    ++*nl;
    return 0;
}

}  // namespace twa
