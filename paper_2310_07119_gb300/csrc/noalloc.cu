// noalloc.cu - a 1D step entry point that allocates no device memory.
//
// Some callers cannot allocate device memory at the point where they need a step: a serving
// process whose memory is fully owned by its own pooled allocator, a real-time loop that must not
// risk an allocation failure or the device-wide synchronization cudaMalloc/cudaFree can cause,
// or a plugin whose host forbids it.  twa_step_batch_1d_static gives them the 1D kick-drift-kick
// step of twa_step_batch without a handle: the Poisson buffer and the FFT/phase tables live in
// the file-scope device arrays below (the caller still passes the field batch).
//
// The arrays are static device memory: every GPU that loads the library holds them (about 4.1 MB)
// until the process exits.  Every call reuses them and they keep the previous call's contents, so
// each call rebuilds the tables and the Poisson field before using them; two calls whose work
// overlaps on the GPU (different streams, or the same arrays from different host threads) race.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>

#include "kernels.h"
#include "passes.cuh"
#include "twa.h"

void twa_set_global_error(const std::string& msg);

namespace {

using namespace twa;

constexpr int kMaxN = 2048;
constexpr long long kScratchElems = TWA_STATIC_SCRATCH_ELEMS;  // pairs * N complex values

static __device__ __align__(256) float2 g_scratch[kScratchElems];
static __device__ __align__(256) float4 g_tw[2 * kMaxN];  // stage-major twiddles (< 2 N entries)
static __device__ __align__(256) float4 g_ph[kMaxN];  // kinetic phase (hi, lo)
static __device__ __align__(256) float g_k2[kMaxN];
static __device__ __align__(256) float g_zero[4];

struct DevSyms {
    bool ready = false;
    float2* scratch = nullptr;
    float4* tw = nullptr;
    float4* ph = nullptr;
    float* k2 = nullptr;
    float* zero = nullptr;
};
constexpr int kMaxDevices = 64;
DevSyms g_dev[kMaxDevices];
std::mutex g_mu;

// Twiddles exp(-2 pi i m / N) in the stage-major layout of the transforms, kinetic phases exp(-i hbar k^2 dt / 2) / N (phase reduced mod 2 pi
// in FP64) and k^2, each table entry split into float hi + lo, computed on the device in FP64.
__global__ void k_tables_1d(float4* tw, float4* ph, float* k2, float* zero, int n, double L,
                            double hbar, double dt) {
    for (int e = threadIdx.x; e < 2 * n; e += blockDim.x) {
        const int m = tw_exponent_n(n, e);
        if (m < 0) continue;
        double s, c;
        sincospi(-2.0 * (double)m / (double)n, &s, &c);
        const float cx = (float)c, sy = (float)s;
        tw[e] = make_float4(cx, sy, (float)(c - (double)cx), (float)(s - (double)sy));
    }
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const int m = (j < n / 2) ? j : j - n;
        const double k = 6.283185307179586476925286766559 * (double)m / L;
        const double th = fmod(hbar * k * k * dt * 0.5, 6.283185307179586476925286766559);
        double ps, pc;
        sincos(th, &ps, &pc);
        const double re = pc / n, im = -ps / n;
        const float rh = (float)re, ih = (float)im;
        ph[j] = make_float4(rh, ih, (float)(re - (double)rh), (float)(im - (double)ih));
        k2[j] = (float)(k * k);
    }
    if (threadIdx.x < 4) zero[threadIdx.x] = 0.f;
}

int fail(int code, const std::string& msg) {
    twa_set_global_error("twa_step_batch_1d_static: " + msg);
    return code;
}

int launch_n(int N, const LaunchCfg& c, const PassArgs& a, cudaStream_t st, bool prep) {
    switch (N) {
        case 8: return launch_line<8>(c, a, st, prep);
        case 16: return launch_line<16>(c, a, st, prep);
        case 32: return launch_line<32>(c, a, st, prep);
        case 64: return launch_line<64>(c, a, st, prep);
        case 128: return launch_line<128>(c, a, st, prep);
        case 256: return launch_line<256>(c, a, st, prep);
        case 512: return launch_line<512>(c, a, st, prep);
        case 1024: return launch_line<1024>(c, a, st, prep);
        case 2048: return launch_line<2048>(c, a, st, prep);
        default: return -1;
    }
}

int pass(int N, int op, int lines, dim3 grid, const PassArgs& a, cudaStream_t st) {
    LaunchCfg c{};
    c.op = op;
    c.strided = false;
    c.lines = lines;
    c.grid = grid;
    if (launch_n(N, c, a, st, true) != 0) return fail(TWA_ECUDA, "kernel attribute setup failed");
    if (launch_n(N, c, a, st, false) != 0) return fail(TWA_EINVAL, "no kernel variant for this size");
    return 0;
}

}  // namespace

extern "C" int twa_step_batch_1d_static(const twa_grid* grid, const twa_params* p, int n_real, void* psi,
                                        int n_steps, void* stream) {
    if (!grid || !p || !psi || n_real < 1 || n_steps < 0) return fail(TWA_EINVAL, "null pointer or bad count");
    // the line passes read and write the batch with 16-byte accesses, as the handle calls do
    if (reinterpret_cast<uintptr_t>(psi) & 15u) return fail(TWA_EINVAL, "psi must be 16-byte aligned");
    if (grid->dim != 1 || p->precision != TWA_F32) return fail(TWA_EINVAL, "only 1D grids on the FP32 path");
    const int N = grid->n[0];
    if (N < 8 || N > kMaxN || (N & (N - 1))) return fail(TWA_EINVAL, "n[0] must be a power of two in [8, 2048]");
    if (!(p->hbar_m > 0) || !(p->dt > 0) || !(grid->L > 0)) return fail(TWA_EINVAL, "hbar_m, dt and L must be positive");
    // counts in 64 bits: n_real near INT_MAX must not wrap before the size check
    const long long n_slots_ll = (long long)n_real + 1, n_pairs_ll = (n_slots_ll + 1) / 2;
    if (n_pairs_ll * N > kScratchElems)
        return fail(TWA_EINVAL, "pairs x n = " + std::to_string(n_pairs_ll * N) +
                                    " exceeds the static scratch of " + std::to_string(kScratchElems) +
                                    " complex values (TWA_STATIC_SCRATCH_ELEMS)");
    // the Poisson passes put one pair per grid row (grid.y <= 65535)
    if (n_pairs_ll > 65535) return fail(TWA_EINVAL, "more than 65535 stream pairs");
    const int n_slots = (int)n_slots_ll, n_pairs = (int)n_pairs_ll;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return fail(TWA_ECUDA, "no current CUDA device");
    }
    DevSyms d;
    {
        // First call on a device: look up the device addresses of the static arrays (host code
        // cannot use the symbols themselves).
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_dev[dev].ready) {
            DevSyms s;
            if (cudaGetSymbolAddress((void**)&s.scratch, g_scratch) != cudaSuccess ||
                cudaGetSymbolAddress((void**)&s.tw, g_tw) != cudaSuccess ||
                cudaGetSymbolAddress((void**)&s.ph, g_ph) != cudaSuccess ||
                cudaGetSymbolAddress((void**)&s.k2, g_k2) != cudaSuccess ||
                cudaGetSymbolAddress((void**)&s.zero, g_zero) != cudaSuccess) {
                cudaGetLastError();
                return fail(TWA_ECUDA, "cudaGetSymbolAddress failed");
            }
            s.ready = true;
            g_dev[dev] = s;
        }
        d = g_dev[dev];
    }
    if (n_steps == 0) return TWA_OK;
    k_tables_1d<<<1, 256, 0, st>>>(d.tw, d.ph, d.k2, d.zero, N, grid->L, p->hbar_m, p->dt);
    const long long cells = N;
    auto split = [&](double frac, float& hi, float& lo) {
        const double k = -frac * p->dt * p->C / (p->hbar_m * (double)cells);
        hi = (float)k;
        lo = (float)(k - (double)hi);
    };
    PassArgs a{};
    a.psi = static_cast<float2*>(psi);
    a.buf = d.scratch;
    a.tw = d.tw;
    a.ph = d.ph;
    a.k2x = d.k2;
    a.k2a = d.k2;
    a.k2y = d.zero;
    a.k2z = d.zero;
    a.S = 1;
    a.Qn = 1;
    a.OS = N;
    a.cells = cells;
    a.n_slots = n_slots;
    a.n_pairs = n_pairs;
    a.lx = 0;
    while ((1 << a.lx) < N) ++a.lx;
    a.lxy = a.lx;
    a.post = 1.0f;
    // Poisson field of the synchronized batch (overwrites whatever the last call left)
    if (int rc = pass(N, OP_RHO_FWD, 1, dim3(1, n_pairs, 1), a, st)) return rc;
    if (int rc = pass(N, OP_MUL_INV, 1, dim3(1, n_pairs, 1), a, st)) return rc;
    // a failed launch of the Poisson passes must not let the steps below touch psi
    if (const cudaError_t e0 = cudaGetLastError(); e0 != cudaSuccess) return fail(TWA_ECUDA, cudaGetErrorString(e0));
    // n_steps on chip with the opening half kick, then the closing half kick
    const int T = plan_threads_per_line(N);
    const int lines = (128 / T) > 1 ? 128 / T : 1;
    split(0.5, a.kick, a.kick_lo);
    split(1.0, a.kick2, a.kick2_lo);
    a.nsteps = n_steps;
    if (int rc = pass(N, OP_STEPS_1D, lines, dim3((n_pairs + lines - 1) / lines, 1, 1), a, st)) return rc;
    float kh, kl;
    split(0.5, kh, kl);
    launch_kick_pairs(a.psi, d.scratch, cells, n_slots, kh, kl, st);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(TWA_ECUDA, cudaGetErrorString(e));
    return TWA_OK;
}
