// observable.cu - run-time compiled stream averages of user functions (Appendix B: a synthesizer
// that evaluates arbitrary functions of the streams' fields and averages them across the streams,
// applied either to each stream before averaging or to the averaged field).
//
// The user gives f as two C expressions (real and imaginary part) in the variables re, im (the
// field value: double, or float in the FP32 mode), i (index of the cell or mode, x fastest), n
// (cells) and nx, ny, nz.  The
// expressions are pasted into a fixed kernel source, compiled with NVRTC for the current device and
// loaded as a CUDA library.  One kernel pass reads every slot of the instance once: per cell it sums
// f over the sampled streams in slot order (or sums the field and applies f to the mean), writes the
// per-cell result, applies f to the classical slot, and leaves per-block partial sums of the
// per-cell results that a one-thread kernel adds in block order, so the total is reproducible.
// NVRTC is opened with dlopen on first use: the library itself has no link-time dependency on it.
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvrtc.h>
#include <stdint.h>

#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

#include "observable.h"

namespace twa {
namespace {

const char* kSource = R"SRC(
#ifdef TWA_EVAL_FP32
// f in float; the sums over the streams as float pairs (Knuth's two-sum, the rounding errors summed)
typedef float twa_real;
struct twa_acc { float hi, lo; };
__device__ __forceinline__ void twa_acc_add(twa_acc& a, float b) {
    const float s = a.hi + b, bb = s - a.hi;
    a.lo += (a.hi - (s - bb)) + (b - bb);
    a.hi = s;
}
__device__ __forceinline__ double twa_acc_value(const twa_acc& a) { return (double)a.hi + (double)a.lo; }
#else
typedef double twa_real;
struct twa_acc { double hi, lo; };
__device__ __forceinline__ void twa_acc_add(twa_acc& a, double b) { a.hi += b; }
__device__ __forceinline__ double twa_acc_value(const twa_acc& a) { return a.hi; }
#endif
struct twa_c2 { twa_real x, y; };
__device__ __forceinline__ twa_c2 twa_f(twa_real re, twa_real im, long long i, long long n, int nx, int ny, int nz) {
    (void)re; (void)im; (void)i; (void)n; (void)nx; (void)ny; (void)nz;
    twa_c2 r;
    r.x = (twa_real)(TWA_F_RE);
    r.y = (twa_real)(TWA_F_IM);
    return r;
}
template <class T2>
__device__ __forceinline__ void twa_obs_body(const T2* __restrict__ psi, long long cells, int n_slots, int of_mean,
                                             double scale, int nx, int ny, int nz, double2* __restrict__ out,
                                             double2* __restrict__ cl, double* __restrict__ part) {
    __shared__ double sr[256], si[256];
    const double inv_ns = 1.0 / (double)(n_slots - 1);
    const twa_real sc = (twa_real)scale;
    double tr = 0.0, ti = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < cells;
         c += (long long)gridDim.x * blockDim.x) {
        twa_acc ar = {0, 0}, ai = {0, 0};
        double vr, vi;
        if (of_mean) {
            for (int s = 1; s < n_slots; ++s) {
                const T2 z = psi[(long long)s * cells + c];
                twa_acc_add(ar, (twa_real)z.x);
                twa_acc_add(ai, (twa_real)z.y);
            }
            const twa_c2 v = twa_f((twa_real)(twa_acc_value(ar) * inv_ns * scale),
                                   (twa_real)(twa_acc_value(ai) * inv_ns * scale), c, cells, nx, ny, nz);
            vr = (double)v.x;
            vi = (double)v.y;
        } else {
            for (int s = 1; s < n_slots; ++s) {
                const T2 z = psi[(long long)s * cells + c];
                const twa_c2 v = twa_f((twa_real)z.x * sc, (twa_real)z.y * sc, c, cells, nx, ny, nz);
                twa_acc_add(ar, v.x);
                twa_acc_add(ai, v.y);
            }
            vr = twa_acc_value(ar) * inv_ns;
            vi = twa_acc_value(ai) * inv_ns;
        }
        if (out) {
            out[c].x = vr;
            out[c].y = vi;
        }
        if (cl) {
            const T2 z = psi[c];
            const twa_c2 v = twa_f((twa_real)z.x * sc, (twa_real)z.y * sc, c, cells, nx, ny, nz);
            cl[c].x = (double)v.x;
            cl[c].y = (double)v.y;
        }
        tr += vr;
        ti += vi;
    }
    sr[threadIdx.x] = tr;
    si[threadIdx.x] = ti;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sr[threadIdx.x] += sr[threadIdx.x + w];
            si[threadIdx.x] += si[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = sr[0];
        part[2 * blockIdx.x + 1] = si[0];
    }
}
extern "C" __global__ void __launch_bounds__(256) twa_obs_f32(const float2* psi, long long cells, int n_slots,
        int of_mean, double scale, int nx, int ny, int nz, double2* out, double2* cl, double* part) {
    twa_obs_body<float2>(psi, cells, n_slots, of_mean, scale, nx, ny, nz, out, cl, part);
}
extern "C" __global__ void __launch_bounds__(256) twa_obs_f64(const double2* psi, long long cells, int n_slots,
        int of_mean, double scale, int nx, int ny, int nz, double2* out, double2* cl, double* part) {
    twa_obs_body<double2>(psi, cells, n_slots, of_mean, scale, nx, ny, nz, out, cl, part);
}
extern "C" __global__ void twa_obs_finish(const double* part, int nb, double w, double* total) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double r = 0.0, i = 0.0;
    for (int b = 0; b < nb; ++b) {
        r += part[2 * b];
        i += part[2 * b + 1];
    }
    total[0] = r * w;
    total[1] = i * w;
}
)SRC";

// NVRTC entry points, resolved with dlsym on first use.
struct Nvrtc {
    bool tried = false;
    void* so = nullptr;
    nvrtcResult (*create)(nvrtcProgram*, const char*, const char*, int, const char* const*, const char* const*) = nullptr;
    nvrtcResult (*compile)(nvrtcProgram, int, const char* const*) = nullptr;
    nvrtcResult (*log_size)(nvrtcProgram, size_t*) = nullptr;
    nvrtcResult (*log)(nvrtcProgram, char*) = nullptr;
    nvrtcResult (*cubin_size)(nvrtcProgram, size_t*) = nullptr;
    nvrtcResult (*cubin)(nvrtcProgram, char*) = nullptr;
    nvrtcResult (*destroy)(nvrtcProgram*) = nullptr;
};

Nvrtc& nvrtc() {
    static Nvrtc n;
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    if (n.tried) return n;
    n.tried = true;
    for (const char* name : {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13",
                             "/usr/local/cuda/lib64/libnvrtc.so"}) {
        n.so = dlopen(name, RTLD_NOW | RTLD_LOCAL);
        if (n.so) break;
    }
    if (!n.so) return n;
    n.create = reinterpret_cast<decltype(n.create)>(dlsym(n.so, "nvrtcCreateProgram"));
    n.compile = reinterpret_cast<decltype(n.compile)>(dlsym(n.so, "nvrtcCompileProgram"));
    n.log_size = reinterpret_cast<decltype(n.log_size)>(dlsym(n.so, "nvrtcGetProgramLogSize"));
    n.log = reinterpret_cast<decltype(n.log)>(dlsym(n.so, "nvrtcGetProgramLog"));
    n.cubin_size = reinterpret_cast<decltype(n.cubin_size)>(dlsym(n.so, "nvrtcGetCUBINSize"));
    n.cubin = reinterpret_cast<decltype(n.cubin)>(dlsym(n.so, "nvrtcGetCUBIN"));
    n.destroy = reinterpret_cast<decltype(n.destroy)>(dlsym(n.so, "nvrtcDestroyProgram"));
    if (!n.create || !n.compile || !n.log_size || !n.log || !n.cubin_size || !n.cubin || !n.destroy) n.so = nullptr;
    return n;
}

// The expressions are pasted into device code: keep them to arithmetic on the documented variables
// and math functions (no statements, blocks, subscripts, strings, preprocessor or pointer casts).
bool expression_ok(const std::string& e, std::string* why) {
    if (e.empty()) {
        *why = "empty expression";
        return false;
    }
    for (char ch : e) {
        const unsigned char u = (unsigned char)ch;
        if (u < 32 || u > 126 || std::string("[]{};#\"'\\`@$").find(ch) != std::string::npos) {
            *why = std::string("character not allowed in an expression: '") + ch + "'";
            return false;
        }
    }
    for (const char* bad : {"*)", "->", "asm", "__", "//", "/*"}) {
        if (e.find(bad) != std::string::npos) {
            *why = std::string("sequence not allowed in an expression: \"") + bad + "\"";
            return false;
        }
    }
    return true;
}

}  // namespace

struct ObsProgram {
    cudaLibrary_t lib = nullptr;
    cudaKernel_t k32 = nullptr, k64 = nullptr, kfin = nullptr;
};

int obs_compile(const char* f_re, const char* f_im, bool fp32, ObsProgram** out, std::string* msg) {
    *out = nullptr;
    const std::string re = f_re ? f_re : "", im = (f_im && *f_im) ? f_im : "0";
    std::string why;
    if (!expression_ok(re, &why) || !expression_ok(im, &why)) {
        *msg = "twa_observable_create: " + why;
        return -1;
    }
    Nvrtc& nv = nvrtc();
    if (!nv.so) {
        *msg = "twa_observable_create: NVRTC (libnvrtc.so) could not be opened";
        return -3;
    }
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev)) {
        cudaGetLastError();
        *msg = "twa_observable_create: no CUDA device";
        return -3;
    }
    const std::string src = std::string(fp32 ? "#define TWA_EVAL_FP32 1\n" : "") + "#define TWA_F_RE (" + re +
                            ")\n#define TWA_F_IM (" + im + ")\n" + kSource;
    const std::string arch = "--gpu-architecture=sm_" + std::to_string(major) + std::to_string(minor);
    const char* opts[] = {arch.c_str(), "--std=c++17", "--device-as-default-execution-space"};
    nvrtcProgram prog = nullptr;
    if (nv.create(&prog, src.c_str(), "twa_observable.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS) {
        *msg = "twa_observable_create: nvrtcCreateProgram failed";
        return -3;
    }
    const nvrtcResult rc = nv.compile(prog, 3, opts);
    if (rc != NVRTC_SUCCESS) {
        size_t n = 0;
        nv.log_size(prog, &n);
        std::string log(n, '\0');
        if (n) nv.log(prog, &log[0]);
        nv.destroy(&prog);
        *msg = "twa_observable_create: the expression does not compile:\n" + log;
        return -1;
    }
    size_t n = 0;
    nv.cubin_size(prog, &n);
    std::vector<char> cubin(n);
    nv.cubin(prog, cubin.data());
    nv.destroy(&prog);
    ObsProgram* p = new ObsProgram();
    cudaError_t e = cudaLibraryLoadData(&p->lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (e == cudaSuccess) e = cudaLibraryGetKernel(&p->k32, p->lib, "twa_obs_f32");
    if (e == cudaSuccess) e = cudaLibraryGetKernel(&p->k64, p->lib, "twa_obs_f64");
    if (e == cudaSuccess) e = cudaLibraryGetKernel(&p->kfin, p->lib, "twa_obs_finish");
    if (e != cudaSuccess) {
        *msg = std::string("twa_observable_create: loading the compiled kernels failed: ") + cudaGetErrorString(e);
        cudaGetLastError();
        obs_free(p);
        return -3;
    }
    *out = p;
    return 0;
}

void obs_free(ObsProgram* p) {
    if (!p) return;
    if (p->lib) cudaLibraryUnload(p->lib);
    delete p;
}

int obs_launch(const ObsProgram* p, bool f64, const void* psi, long long cells, int n_slots, int of_mean,
               double scale, const int* n3, double* per_cell, double* f_cl, double* part, int max_blocks, double w,
               double* total, cudaStream_t st, std::string* msg) {
    const long long want = (cells + 255) / 256;
    int nb = (int)(want < max_blocks ? want : max_blocks);
    if (nb < 1) nb = 1;
    int nx = n3[0], ny = n3[1], nz = n3[2];
    void* args[] = {const_cast<void**>(&psi), &cells, &n_slots, &of_mean, &scale, &nx, &ny, &nz,
                    &per_cell, &f_cl, &part};
    cudaError_t e = cudaLaunchKernel(reinterpret_cast<const void*>(f64 ? p->k64 : p->k32), dim3(nb), dim3(256), args, 0, st);
    if (e == cudaSuccess) {
        void* fargs[] = {&part, &nb, &w, &total};
        e = cudaLaunchKernel(reinterpret_cast<const void*>(p->kfin), dim3(1), dim3(32), fargs, 0, st);
    }
    if (e != cudaSuccess) {
        *msg = std::string("twa_observable_eval: launch failed: ") + cudaGetErrorString(e);
        cudaGetLastError();
        return -3;
    }
    return 0;
}

}  // namespace twa
