// api.cu - implementation of the C ABI in include/twa.h.
//
// Pipelines (per instance, FP32 path).  The state between steps is "drifted, kick pending": the
// kick of step s+1 is merged with the closing half kick of step s (Sec. III.B.2), and the pending
// half kick is applied on the fly by the moment kernels.
//   1D : one on-chip pass per launch runs many steps (whole field in registers).
//   2D : x rows  [kick + drift_x]  -> y cols [drift_y + packed density + FFT_y]
//        -> x rows [FFT_x, Poisson, iFFT_x] -> y cols [iFFT_y]                      (4 passes/step)
//   3D : x [iFFT_x of V + kick + drift_x] -> y [drift_y] -> z [drift_z + density + FFT_z]
//        -> x [FFT_x] -> y [FFT_y, Poisson, iFFT_y] -> z [iFFT_z]                   (6 passes/step)
//        V stays spectral along x between steps; its inverse is fused into the next kick.
//   3D, square xy planes (plane pipeline): [kick + drift_x + drift_y per z-plane] -> z [drift_z +
//        density + FFT_z] -> [FFT_xy, Poisson, iFFT_xy per plane] -> z [iFFT_z]    (4 passes/step)
//        The autotuner times both 3D pipelines and keeps the axis one on near-ties.
// Around these: adaptive steps (the Delta t rule read back before each output interval), test
// particles moved before every step, and the amplitude/phase moments on request.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <iterator>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <set>
#include <sstream>
#include <string>
#include <vector>

#include "kernels.h"
#include "observable.h"
#include "passes.cuh"
#include "batch.h"
#include "pipe.cuh"
#include "run1d.cuh"
#include "twa.h"

using namespace twa;

static_assert(OP_COUNT + PL_COUNT == TWA_PROF_NOPS, "profiler op table out of sync with the pass kinds");

namespace {

// 3D pipelines: MODE_3D axis passes (the Poisson field kept spectral along x between steps), MODE_3DP
// xy-plane passes for fields and Poisson field, MODE_3DH axis passes for the fields and the xy-plane
// Poisson pass (the Poisson field real between steps in both)
constexpr int MODE_1D = 0, MODE_2D = 1, MODE_3D = 2, MODE_3DP = 3, MODE_3DH = 4;
// Profiler ids of the xy-plane passes follow the line-pass ops.
constexpr int PROF_PLANE0 = OP_COUNT;
constexpr int PROF_NOPS = OP_COUNT + PL_COUNT;

struct Inst {
    int dim = 1;
    int n[3] = {1, 1, 1};
    int lg[3] = {0, 0, 0};
    long long cells = 0;
    double L = 1.0, dV = 1.0;
    int n_real = 0, n_slots = 0, n_pairs = 0;
    size_t off = 0;
    int mode = MODE_1D;
    // FP32 path
    float2* vc = nullptr;
    float2* spec = nullptr;
    float4* ph[3] = {nullptr, nullptr, nullptr};  // kinetic phase per axis, (hi, lo)
    float* k2[3] = {nullptr, nullptr, nullptr};
    double* part_r = nullptr;
    double* part_m = nullptr;
    double* run_part = nullptr;  // partial sums of whole 1D runs (k_run1d)
    size_t run_part_n = 0;
    std::map<int, int> lines;  // (axis * 64 + op) -> lines per CTA
    // test particles (FP32 path): state [n_slots][r 3, p 3] and the spectral derivative kernels
    double* prt = nullptr;
    double* dker[3] = {nullptr, nullptr, nullptr};
    // FP64 path
    double2* work64 = nullptr;
    double2* spec64 = nullptr;
    double* acc64 = nullptr;
    double* acc64m = nullptr;
    double* bad64 = nullptr;
    double2* tw64[3] = {nullptr, nullptr, nullptr};
    double2* ph64[3] = {nullptr, nullptr, nullptr};
    double* k264[3] = {nullptr, nullptr, nullptr};
};

std::string g_create_error;

}  // namespace

struct twa_handle {
    twa_params p{};
    std::vector<Inst> in;
    std::string err;
    int* d_err = nullptr;
    unsigned* d_vmax = nullptr;  // [n_inst] largest |W| per instance (float bits), adaptive steps
    int* d_counter = nullptr;
    double* d_cur = nullptr;  // [n_inst][TWA_NSCALARS] scalars of the current output
    std::map<int, float4*> tw32;
    std::set<long long> prepared;
    std::vector<void*> allocs;
    long long launches = 0;
    cudaStream_t cap = nullptr;
    cudaEvent_t ev_a = nullptr, ev_b = nullptr;
    cudaGraphExec_t gexec = nullptr;
    long long graph_launches = 0;
    // one stream and join event per instance, for the fork/join of multi-instance batches
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> side_ev;
    cudaEvent_t ev_fork = nullptr;
    const void* g_psi = nullptr;
    const void* g_series = nullptr;
    int g_out_every = -1;
    // run the instances of a multi-instance batch on parallel streams (see Fork)
    bool fork = false;
    // run the steps of all instances as one persistent launch over a work list (2D batches)
    bool persist = false;
    double wait_limit_s = 2.0;     // longest device-side wait (persistent launch, TMA tile pipelines)
    int clock_khz = 0;             // peak SM clock, converts the wait limit to clock64 cycles
    std::map<std::string, CUtensorMap> tmaps;  // tensor maps of the TMA column passes, by buffer and shape
    bool stall_next = false;       // fault injection: the next persistent launch waits forever
    bool stall_tma = false;        // fault injection: the next TMA tile pass expects bytes that never come
    unsigned* d_ctr = nullptr;     // per-pair tile counters of the persistent launch
    unsigned long long* d_tick = nullptr;  // [0] ticket, [1] abort flag (low word)
    struct BatchTable {
        twa::BatchPass* passes;
        twa::PassArgs* args;
        int n_passes;
        long long n_items;
        std::vector<int> kinds;
    };
    std::vector<std::pair<std::vector<double>, BatchTable>> btab;
    // pass profiler
    bool prof_on = false;
    struct ProfRec {
        int op;
        cudaEvent_t a, b;
        long long fields, cells;
    };
    std::vector<ProfRec> prof_pending;
    std::vector<cudaEvent_t> prof_pool;
    long long prof_launches[OP_COUNT + PL_COUNT] = {};
    double prof_ms[OP_COUNT + PL_COUNT] = {};
    long long prof_fields[OP_COUNT + PL_COUNT] = {};
    long long prof_cells[OP_COUNT + PL_COUNT] = {};
};

namespace {

// kick = -frac dt C / (hbar cells) in FP64, carried as float hi + lo (the stored Poisson field is
// W = iFFT(FFT(rho) / k^2), so V = -C W / cells and theta = kick W).
void split_kick(const twa_handle* h, const Inst& I, double frac, float& hi, float& lo) {
    const double k = -frac * h->p.dt * h->p.C / (h->p.hbar_m * (double)I.cells);
    hi = (float)k;
    lo = (float)(k - (double)hi);
}

int fail(twa_handle* h, int code, const std::string& msg) {
    if (h) h->err = msg;
    else g_create_error = msg;
    return code;
}

// Field buffers are read with 16-byte copies (cp.async in the pipelined passes, double2 loads of
// the classical field): their base addresses must be 16-byte aligned.  Instances and slots start
// on 64-byte multiples inside a batch (every axis has at least 8 cells), so the base decides.
bool misaligned(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) != 0; }

#define CU(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(h, TWA_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <class T>
int dalloc(twa_handle* h, T** ptr, size_t count) {
    void* p = nullptr;
    if (count == 0) count = 1;
    if (cudaMalloc(&p, count * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return fail(h, TWA_ENOMEM, "cudaMalloc of " + std::to_string(count * sizeof(T)) + " bytes failed");
    }
    h->allocs.push_back(p);
    *ptr = static_cast<T*>(p);
    return 0;
}

template <class T>
int upload(twa_handle* h, T** dst, const std::vector<T>& v) {
    int rc = dalloc(h, dst, v.size());
    if (rc) return rc;
    CU(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return 0;
}

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
int ilog2(int v) {
    int r = 0;
    while ((1 << r) < v) ++r;
    return r;
}

// Wavenumber of FFT index j on an axis of n cells and side L: 2 pi m / L, m in {0..n/2-1, -n/2..-1}.
double wavenumber(int j, int n, double L) {
    const int m = (j < n / 2) ? j : j - n;
    return 2.0 * M_PI * (double)m / L;
}

// exp(-i theta) with theta reduced mod 2 pi in FP64 first.
void phase_of(double theta, double& c, double& s) {
    const double r = std::fmod(theta, 2.0 * M_PI);
    c = std::cos(r);
    s = -std::sin(r);
}

int key_of(int axis, int op) { return axis * 64 + op; }

}  // namespace
struct twa_handle;
namespace {
void split_kick(const twa_handle* h, const Inst& I, double frac, float& hi, float& lo);

int default_lines(int N, bool strided, int op) {
    const int T = plan_threads_per_line(N);
    if (op == OP_STEPS_1D) return std::max(1, 128 / T);
    if (strided) return std::max(4, 256 / T);
    return std::max(1, 256 / T);
}

int dispatch(int N, const LaunchCfg& c, const PassArgs& a, cudaStream_t st, bool prep) {
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

constexpr int PIPE_FLAG = 1 << 16;  // "lines" values with this bit select the pipelined pass
constexpr int DUAL_FLAG = 1 << 17;  // ... and with this bit the two-field variant (both slots of a pair)
constexpr int TMA_FLAG = 1 << 18;   // ... and with PIPE_FLAG, the column pass whose tiles TMA copies

int dispatch_pipe(int N, const LaunchCfg& c, const PassArgs& a, int tiles, int n_items, cudaStream_t st, bool prep) {
    switch (N) {
        case 32: return launch_pipe<32>(c, a, tiles, n_items, st, prep);
        case 64: return launch_pipe<64>(c, a, tiles, n_items, st, prep);
        case 128: return launch_pipe<128>(c, a, tiles, n_items, st, prep);
        case 256: return launch_pipe<256>(c, a, tiles, n_items, st, prep);
        case 512: return launch_pipe<512>(c, a, tiles, n_items, st, prep);
        case 1024: return launch_pipe<1024>(c, a, tiles, n_items, st, prep);
        case 2048: return launch_pipe<2048>(c, a, tiles, n_items, st, prep);
        default: return -1;
    }
}

bool pipe_variant_ok(int N, int op, bool strided, int lines) {
    switch (N) {
        case 32: return has_pipe_variant<32>(op, strided, lines);
        case 64: return has_pipe_variant<64>(op, strided, lines);
        case 128: return has_pipe_variant<128>(op, strided, lines);
        case 256: return has_pipe_variant<256>(op, strided, lines);
        case 512: return has_pipe_variant<512>(op, strided, lines);
        case 1024: return has_pipe_variant<1024>(op, strided, lines);
        case 2048: return has_pipe_variant<2048>(op, strided, lines);
        default: return false;
    }
}

bool pipe_tma_variant_ok(int N, int op, bool strided, int lines) {
    switch (N) {
        case 32: return has_pipe_tma_variant<32>(op, strided, lines);
        case 64: return has_pipe_tma_variant<64>(op, strided, lines);
        case 128: return has_pipe_tma_variant<128>(op, strided, lines);
        case 256: return has_pipe_tma_variant<256>(op, strided, lines);
        case 512: return has_pipe_tma_variant<512>(op, strided, lines);
        case 1024: return has_pipe_tma_variant<1024>(op, strided, lines);
        case 2048: return has_pipe_tma_variant<2048>(op, strided, lines);
        default: return false;
    }
}

bool dual_variant_ok(int N, int op, bool strided, int lines) {
    switch (N) {
        case 8: return has_dual_variant<8>(op, strided, lines);
        case 16: return has_dual_variant<16>(op, strided, lines);
        case 32: return has_dual_variant<32>(op, strided, lines);
        case 64: return has_dual_variant<64>(op, strided, lines);
        case 128: return has_dual_variant<128>(op, strided, lines);
        case 256: return has_dual_variant<256>(op, strided, lines);
        case 512: return has_dual_variant<512>(op, strided, lines);
        case 1024: return has_dual_variant<1024>(op, strided, lines);
        case 2048: return has_dual_variant<2048>(op, strided, lines);
        default: return false;
    }
}

bool variant_ok(int N, int op, bool strided, int lines) {
    if ((lines & PIPE_FLAG) && (lines & DUAL_FLAG)) return false;
    if (lines & TMA_FLAG) {
        // TMA tiles of the pipelined kernel: column tiles by tensor map (a box row of LINES 8-byte
        // elements must span a multiple of 16 bytes), row tiles by one bulk copy per row
        const int l = lines & ~(PIPE_FLAG | TMA_FLAG);
        if (!(lines & PIPE_FLAG) || (lines & DUAL_FLAG)) return false;
        if (strided) return l % 2 == 0 && encode_tiled_fn() && pipe_tma_variant_ok(N, op, true, l);
        return pipe_tma_variant_ok(N, op, false, l);
    }
    if (lines & PIPE_FLAG) return pipe_variant_ok(N, op, strided, lines & ~PIPE_FLAG);
    if (lines & DUAL_FLAG) return dual_variant_ok(N, op, strided, lines & ~DUAL_FLAG);
    switch (N) {
        case 8: return has_variant<8>(op, strided, lines);
        case 16: return has_variant<16>(op, strided, lines);
        case 32: return has_variant<32>(op, strided, lines);
        case 64: return has_variant<64>(op, strided, lines);
        case 128: return has_variant<128>(op, strided, lines);
        case 256: return has_variant<256>(op, strided, lines);
        case 512: return has_variant<512>(op, strided, lines);
        case 1024: return has_variant<1024>(op, strided, lines);
        case 2048: return has_variant<2048>(op, strided, lines);
        default: return false;
    }
}

#define RC(x)                \
    do {                     \
        int rc_ = (x);       \
        if (rc_) return rc_; \
    } while (0)

int prof_events(twa_handle* h, cudaEvent_t* a, cudaEvent_t* b) {
    for (cudaEvent_t* e : {a, b}) {
        if (h->prof_pool.empty()) {
            cudaEvent_t n;
            CU(cudaEventCreate(&n));
            h->prof_pool.push_back(n);
        }
        *e = h->prof_pool.back();
        h->prof_pool.pop_back();
    }
    return 0;
}

// Arguments of a line pass along `axis` of instance I.
PassArgs make_args(twa_handle* h, Inst& I, float2* psi, int axis, double kick_frac, float2* buf, float2* out,
                   int nsteps = 0, float post = 1.0f) {
    const int N = I.n[axis];
    PassArgs a{};
    a.psi = psi;
    a.buf = buf;
    a.out = out;
    a.tw = h->tw32[N];
    a.ph = I.ph[axis];
    a.post = post;
    a.k2x = I.k2[0];
    a.k2y = I.k2[1];
    a.k2z = I.k2[2];
    a.k2a = I.k2[axis];
    split_kick(h, I, kick_frac, a.kick, a.kick_lo);
    split_kick(h, I, 1.0, a.kick2, a.kick2_lo);
    a.cells = I.cells;
    a.n_slots = I.n_slots;
    a.n_pairs = I.n_pairs;
    a.lx = I.lg[0];
    a.lxy = I.lg[0] + I.lg[1];
    a.nsteps = nsteps;
    long long stride = 1;
    for (int b = 0; b < axis; ++b) stride *= I.n[b];
    a.S = (int)stride;
    a.Qn = (int)stride;
    a.OS = stride * N;
    a.err = h->d_err;
    a.wait = (long long)(h->wait_limit_s * (double)h->clock_khz * 1e3);
    return a;
}

// Tensor map of `fields` fields of `cells` cells at base, for the TMA column passes along an axis of
// N cells whose line starts are `stride` apart: a dense 4D tensor {line start, position, outer,
// field} of 8-byte elements, boxes of `lines` line starts x min(N, 256) positions.
const CUtensorMap* column_map(twa_handle* h, const float2* base, long long cells, int N, long long stride, int fields,
                              int lines) {
    std::ostringstream k;
    k << (const void*)base << ":" << cells << ":" << N << ":" << stride << ":" << fields << ":" << lines;
    auto it = h->tmaps.find(k.str());
    if (it != h->tmaps.end()) return &it->second;
    EncodeTiledFn fn = encode_tiled_fn();
    if (!fn) return nullptr;
    const cuuint64_t dims[4] = {(cuuint64_t)stride, (cuuint64_t)N, (cuuint64_t)(cells / (stride * N)),
                                (cuuint64_t)fields};
    const cuuint64_t strides[3] = {(cuuint64_t)stride * 8, (cuuint64_t)stride * N * 8, (cuuint64_t)cells * 8};
    const cuuint32_t box[4] = {(cuuint32_t)lines, (cuuint32_t)std::min(N, 256), 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    CUtensorMap m;
    if (fn(&m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, const_cast<float2*>(base), dims, strides, box, estr,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return nullptr;
    if (h->tmaps.size() > 256) h->tmaps.clear();
    return &(h->tmaps[k.str()] = m);
}

// One line pass over `fields` fields (pairs or slots) of instance I.
int run_pass(twa_handle* h, Inst& I, float2* psi, int axis, int op, double kick_frac, float2* buf, float2* out, int fields,
             cudaStream_t st, int nsteps = 0, int force_lines = 0, float post = 1.0f) {
    const int N = I.n[axis];
    const bool strided = axis > 0;
    int lines = force_lines;
    if (!lines) {
        auto it = I.lines.find(key_of(axis, op));
        lines = (it != I.lines.end()) ? it->second : default_lines(N, strided, op);
    }
    const bool pipe = (lines & PIPE_FLAG) != 0;
    const bool dual = (lines & DUAL_FLAG) != 0;
    const bool tma = (lines & TMA_FLAG) != 0;
    if (!variant_ok(N, op, strided, lines))
        return fail(h, TWA_EINVAL, "no pass variant for N=" + std::to_string(N) + " op=" + std::to_string(op) +
                                       " lines=" + std::to_string(lines));
    lines &= ~(PIPE_FLAG | DUAL_FLAG | TMA_FLAG);
    // the two-field drift runs over pairs of slots
    const int slot_fields = fields;
    if (dual && op == OP_DRIFT) fields = (fields + 1) / 2;
    PassArgs a = make_args(h, I, psi, axis, kick_frac, buf, out, nsteps, post);
    if (tma && h->stall_tma) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(st, &cs);
        if (cs == cudaStreamCaptureStatusNone) {  // never baked into a graph
            a.stall_tx = 16;
            h->stall_tma = false;
        }
    }
    const long long stride = a.S;
    LaunchCfg c{};
    c.op = op;
    c.strided = strided;
    c.lines = lines;
    c.dual = dual;
    PipeMaps maps{};
    if (tma && strided) {
        // the batch's fields (psi) and the pass's field buffer, as far as the op reads them
        const bool reads_psi = op == OP_DRIFT || op == OP_DRIFT_RHO || op == OP_KICK_DRIFT || op == OP_KICK_DRIFT_VINV;
        const bool reads_buf = op == OP_FWD || op == OP_INV || op == OP_FWD_MUL_INV || op == OP_KICK_DRIFT ||
                               op == OP_KICK_DRIFT_VINV;
        if (reads_psi) {
            const CUtensorMap* m = column_map(h, psi, I.cells, N, stride, I.n_slots, lines);
            if (!m) return fail(h, TWA_ECUDA, "cuTensorMapEncodeTiled failed");
            maps.psi = *m;
        }
        if (reads_buf) {
            const CUtensorMap* m = column_map(h, buf, I.cells, N, stride, fields, lines);
            if (!m) return fail(h, TWA_ECUDA, "cuTensorMapEncodeTiled failed");
            maps.buf = *m;
        }
        c.maps = &maps;
    }
    c.tma = tma;
    if (op == OP_STEPS_1D) {
        c.grid = dim3((unsigned)((I.n_pairs + lines - 1) / lines), 1, 1);
    } else if (strided) {
        const long long tq = (stride + lines - 1) / lines;
        const long long outer = I.cells / (stride * N);
        c.grid = dim3((unsigned)(tq * outer), (unsigned)fields, 1);
    } else {
        const long long rows = I.cells / N;
        c.grid = dim3((unsigned)((rows + lines - 1) / lines), (unsigned)fields, 1);
    }
    int tiles = 0, n_items = 0;
    if (pipe) {
        const long long lines_per_field = strided ? (I.cells / N) : (I.cells / N);
        tiles = (int)(lines_per_field / lines);
        n_items = tiles * fields;
        if (lines_per_field % lines != 0 || (strided && stride % lines != 0))
            return fail(h, TWA_EINVAL, "pipelined pass needs full tiles");
    }
    const long long pk = ((long long)tma << 43) | ((long long)dual << 42) | ((long long)pipe << 41) | ((long long)N << 24) |
                         ((long long)op << 16) | ((long long)strided << 12) | lines;
    if (!h->prepared.count(pk)) {
        const int rc = pipe ? dispatch_pipe(N, c, a, tiles, n_items, st, true) : dispatch(N, c, a, st, true);
        if (rc != 0) return fail(h, TWA_ECUDA, "cudaFuncSetAttribute failed");
        h->prepared.insert(pk);
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (h->prof_on) {
        RC(prof_events(h, &e0, &e1));
        CU(cudaEventRecord(e0, st));
    }
    if ((pipe ? dispatch_pipe(N, c, a, tiles, n_items, st, false) : dispatch(N, c, a, st, false)) != 0)
        return fail(h, TWA_EINVAL, "pass dispatch failed");
    if (h->prof_on) {
        CU(cudaEventRecord(e1, st));
        const long long nf = (op == OP_STEPS_1D) ? (long long)I.n_pairs * nsteps : (long long)slot_fields;
        h->prof_pending.push_back({op, e0, e1, nf, I.cells});
    }
    ++h->launches;
    return 0;
}


int dispatch_plane(int N, int pop, int lines, dim3 grid, const PassArgs& a, cudaStream_t st, bool prep) {
    switch (N) {
        case 16: return launch_plane<16>(pop, lines, grid, a, st, prep);
        case 32: return launch_plane<32>(pop, lines, grid, a, st, prep);
        case 64: return launch_plane<64>(pop, lines, grid, a, st, prep);
        case 128: return launch_plane<128>(pop, lines, grid, a, st, prep);
        case 256: return launch_plane<256>(pop, lines, grid, a, st, prep);
        default: return -1;
    }
}

bool plane_variant_ok(int N, int pop, int lines) {
    switch (N) {
        case 16: return has_plane_variant<16>(pop, lines);
        case 32: return has_plane_variant<32>(pop, lines);
        case 64: return has_plane_variant<64>(pop, lines);
        case 128: return has_plane_variant<128>(pop, lines);
        case 256: return has_plane_variant<256>(pop, lines);
        default: return false;
    }
}

// One xy-plane pass over all z-planes of every pair of instance I (3D, nx = ny).
int run_plane(twa_handle* h, Inst& I, float2* psi, int pop, double kick_frac, cudaStream_t st, int force_lines = 0) {
    const int N = I.n[0];
    int lines = force_lines;
    if (!lines) {
        auto it = I.lines.find(key_of(3, pop));
        lines = (it != I.lines.end()) ? it->second : std::min(N, std::max(1, 256 / plan_threads_per_line(N)));
    }
    if (!plane_variant_ok(N, pop, lines))
        return fail(h, TWA_EINVAL, "no plane variant for N=" + std::to_string(N) + " lines=" + std::to_string(lines));
    PassArgs a{};
    a.psi = psi;
    a.buf = I.vc;
    a.tw = h->tw32[N];
    a.ph = I.ph[0];
    a.ph2 = I.ph[1];
    a.k2x = I.k2[0];
    a.k2y = I.k2[1];
    a.k2z = I.k2[2];
    split_kick(h, I, kick_frac, a.kick, a.kick_lo);
    a.cells = I.cells;
    a.n_slots = I.n_slots;
    a.n_pairs = I.n_pairs;
    a.lx = I.lg[0];
    a.lxy = I.lg[0] + I.lg[1];
    a.post = 1.0f;
    const dim3 grid((unsigned)I.n[2], (unsigned)I.n_pairs, 1);
    const long long pk = (1LL << 40) | ((long long)N << 24) | ((long long)pop << 16) | lines;
    if (!h->prepared.count(pk)) {
        if (dispatch_plane(N, pop, lines, grid, a, st, true) != 0) return fail(h, TWA_ECUDA, "cudaFuncSetAttribute failed");
        h->prepared.insert(pk);
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (h->prof_on) {
        RC(prof_events(h, &e0, &e1));
        CU(cudaEventRecord(e0, st));
    }
    if (dispatch_plane(N, pop, lines, grid, a, st, false) != 0) return fail(h, TWA_EINVAL, "plane dispatch failed");
    if (h->prof_on) {
        CU(cudaEventRecord(e1, st));
        h->prof_pending.push_back({PROF_PLANE0 + pop, e0, e1, (long long)I.n_pairs, I.cells});
    }
    ++h->launches;
    return 0;
}

float2* inst_psi(Inst& I, void* psi) { return static_cast<float2*>(psi) + I.off; }

// V of every field from its density (a synchronized batch, nothing pending).
int poisson_init(twa_handle* h, Inst& I, float2* psi, cudaStream_t st) {
    const int P = I.n_pairs;
    switch (I.mode) {
        case MODE_1D:
            RC(run_pass(h, I, psi, 0, OP_RHO_FWD, 0.0, I.vc, nullptr, P, st, 0, 1));
            RC(run_pass(h, I, psi, 0, OP_MUL_INV, 0.0, I.vc, nullptr, P, st, 0, 1));
            break;
        case MODE_2D:
            RC(run_pass(h, I, psi, 1, OP_RHO_FWD, 0.0, I.vc, nullptr, P, st));
            RC(run_pass(h, I, psi, 0, OP_FWD_MUL_INV, 0.0, I.vc, nullptr, P, st));
            RC(run_pass(h, I, psi, 1, OP_INV, 0.0, I.vc, nullptr, P, st));
            break;
        case MODE_3DP:
        case MODE_3DH:
            RC(run_pass(h, I, psi, 2, OP_RHO_FWD, 0.0, I.vc, nullptr, P, st));
            RC(run_plane(h, I, psi, PL_POISSON, 0.0, st));
            RC(run_pass(h, I, psi, 2, OP_INV, 0.0, I.vc, nullptr, P, st));
            break;
        default:
            RC(run_pass(h, I, psi, 2, OP_RHO_FWD, 0.0, I.vc, nullptr, P, st));
            RC(run_pass(h, I, psi, 0, OP_FWD, 0.0, I.vc, nullptr, P, st));
            RC(run_pass(h, I, psi, 1, OP_FWD_MUL_INV, 0.0, I.vc, nullptr, P, st));
            RC(run_pass(h, I, psi, 2, OP_INV, 0.0, I.vc, nullptr, P, st));
    }
    return 0;
}

// n steps; the first kick is the fraction a_first of a full kick (1/2 after a synchronized state).
// Move the instance's test particles in the potential of the current batch: kick by kick_frac dt,
// then drift by drift_frac dt.  Needs the Poisson field in real space: the axis pipeline keeps it
// spectral along x between steps, so it is transformed back and forth around the update.
int particles_step(twa_handle* h, Inst& I, float2* psi, double kick_frac, double drift_frac, cudaStream_t st) {
    const bool v_spec = I.mode == MODE_3D;
    if (v_spec) RC(run_pass(h, I, psi, 0, OP_INV, 0.0, I.vc, nullptr, I.n_pairs, st));
    const double* ker[3] = {I.dker[0], I.dker[1] ? I.dker[1] : I.dker[0], I.dker[2] ? I.dker[2] : I.dker[0]};
    launch_particles(I.vc, I.cells, I.n, I.dim, I.L, ker, h->p.C / (double)I.cells, kick_frac * h->p.dt,
                     drift_frac * h->p.dt, I.n_slots, I.prt, st);
    ++h->launches;
    if (v_spec) RC(run_pass(h, I, psi, 0, OP_FWD, 0.0, I.vc, nullptr, I.n_pairs, st, 0, 0, 1.0f / (float)I.n[0]));
    return 0;
}

int steps_f32(twa_handle* h, Inst& I, float2* psi, int n, double a_first, cudaStream_t st) {
    const int P = I.n_pairs;
    if (n <= 0) return 0;
    if (I.mode == MODE_1D) {
        if (!I.prt) return run_pass(h, I, psi, 0, OP_STEPS_1D, a_first, I.vc, nullptr, P, st, n);
        // with test particles the on-chip steps run one at a time, the particles moving in between
        for (int s = 0; s < n; ++s) {
            const double k = (s == 0) ? a_first : 1.0;
            RC(particles_step(h, I, psi, k, 1.0, st));
            RC(run_pass(h, I, psi, 0, OP_STEPS_1D, k, I.vc, nullptr, P, st, 1));
        }
        return 0;
    }
    for (int s = 0; s < n; ++s) {
        const double k = (s == 0) ? a_first : 1.0;
        if (I.prt) RC(particles_step(h, I, psi, k, 1.0, st));
        if (I.mode == MODE_3DP) {
            RC(run_plane(h, I, psi, PL_KICK_DRIFT, k, st));
            RC(run_pass(h, I, psi, 2, OP_DRIFT_RHO, 0.0, I.vc, nullptr, P, st));
            RC(run_plane(h, I, psi, PL_POISSON, 0.0, st));
            RC(run_pass(h, I, psi, 2, OP_INV, 0.0, I.vc, nullptr, P, st));
        } else if (I.mode == MODE_3DH) {
            // the fields by axis passes (kick with the real potential, then the x, y and z drifts),
            // the Poisson field by the xy-plane pass and the z inverse
            RC(run_pass(h, I, psi, 0, OP_KICK_DRIFT, k, I.vc, nullptr, P, st));
            RC(run_pass(h, I, psi, 1, OP_DRIFT, 0.0, I.vc, nullptr, I.n_slots, st));
            RC(run_pass(h, I, psi, 2, OP_DRIFT_RHO, 0.0, I.vc, nullptr, P, st));
            RC(run_plane(h, I, psi, PL_POISSON, 0.0, st));
            RC(run_pass(h, I, psi, 2, OP_INV, 0.0, I.vc, nullptr, P, st));
        } else if (I.mode == MODE_2D) {
            RC(run_pass(h, I, psi, 0, OP_KICK_DRIFT, k, I.vc, nullptr, P, st));
            RC(run_pass(h, I, psi, 1, OP_DRIFT_RHO, 0.0, I.vc, nullptr, P, st));
            RC(run_pass(h, I, psi, 0, OP_FWD_MUL_INV, 0.0, I.vc, nullptr, P, st));
            RC(run_pass(h, I, psi, 1, OP_INV, 0.0, I.vc, nullptr, P, st));
        } else {
            RC(run_pass(h, I, psi, 0, OP_KICK_DRIFT_VINV, k, I.vc, nullptr, P, st));
            RC(run_pass(h, I, psi, 1, OP_DRIFT, 0.0, I.vc, nullptr, I.n_slots, st));
            RC(run_pass(h, I, psi, 2, OP_DRIFT_RHO, 0.0, I.vc, nullptr, P, st));
            RC(run_pass(h, I, psi, 0, OP_FWD, 0.0, I.vc, nullptr, P, st));
            RC(run_pass(h, I, psi, 1, OP_FWD_MUL_INV, 0.0, I.vc, nullptr, P, st));
            RC(run_pass(h, I, psi, 2, OP_INV, 0.0, I.vc, nullptr, P, st));
        }
    }
    return 0;
}

int closing_kick(twa_handle* h, Inst& I, float2* psi, double frac, cudaStream_t st) {
    if (I.prt) RC(particles_step(h, I, psi, frac, 0.0, st));
    if (I.mode == MODE_3D) return run_pass(h, I, psi, 0, OP_KICK_VINV, frac, I.vc, nullptr, I.n_pairs, st);
    float k, kl;
    split_kick(h, I, frac, k, kl);
    launch_kick_pairs(psi, I.vc, I.cells, I.n_slots, k, kl, st);
    ++h->launches;
    return 0;
}

// Instances of a batch are independent.  With h->fork set, each instance's work goes to its own
// stream between a fork on st and a join back onto st (inside a capture this makes parallel graph
// branches), so small instances that cannot fill the GPU alone overlap.  Large instances run one
// after another: their concurrent passes compete for L1, shared memory and L2 (the 2D batch
// 512^2 x 128 + 1024^2 x 64 + 2048^2 x 16 runs 11 % slower forked).  twa_create sets fork for
// batches of small instances; twa_autotune times both.  The pass profiler keeps st.
struct Fork {
    twa_handle* h;
    cudaStream_t st;
    bool on;
    int open(size_t n) {
        on = n > 1 && !h->prof_on && h->fork;
        if (!on) return 0;
        while (h->side.size() < n) {
            cudaStream_t x;
            cudaEvent_t e;
            CU(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
            h->side.push_back(x);
            CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            h->side_ev.push_back(e);
        }
        if (!h->ev_fork) CU(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
        CU(cudaEventRecord(h->ev_fork, st));
        return 0;
    }
    // stream of instance i (waits for the fork)
    int stream(size_t i, cudaStream_t* out) {
        *out = st;
        if (!on) return 0;
        CU(cudaStreamWaitEvent(h->side[i], h->ev_fork, 0));
        *out = h->side[i];
        return 0;
    }
    int join(size_t i) {
        if (!on) return 0;
        CU(cudaEventRecord(h->side_ev[i], h->side[i]));
        CU(cudaStreamWaitEvent(st, h->side_ev[i], 0));
        return 0;
    }
};

// ---------------------------------------------------------------------------------------------
// Persistent batch launch (batch.cu): the steps of every instance of a 2D FP32 batch as one launch
// over a work list of (step, pass, instance, pair, tile) items.

// Every instance is 2D with both axis lengths in [256, 2048] and has no test particles.
bool batch_eligible(const twa_handle* h) {
    if (h->p.precision != TWA_F32 || h->in.empty()) return false;
    for (const auto& I : h->in)
        if (I.mode != MODE_2D || I.prt || batch_kind(I.n[0], 0) < 0 || batch_kind(I.n[1], 1) < 0) return false;
    return true;
}
bool use_batch(const twa_handle* h) { return h->persist && !h->prof_on && batch_eligible(h); }

// The work list of n steps (first kick a_first) of the batch psi, built once per (psi, n, a_first,
// dt) and kept: the list lives in device memory the launches read, so it is created before any
// stream capture and never rewritten while a launch may read it.
int batch_table(twa_handle* h, void* psi, int n, double a_first, cudaStream_t st, twa_handle::BatchTable** out) {
    const bool stall = h->stall_next;
    const std::vector<double> key = {(double)reinterpret_cast<uintptr_t>(psi), (double)n, a_first, h->p.dt};
    if (!stall)
        for (auto& e : h->btab)
            if (e.first == key) {
                *out = &e.second;
                return 0;
            }
    std::vector<BatchPass> P;
    std::vector<PassArgs> A;
    std::vector<int> kinds;
    std::vector<int> ctr_base, argi, tiles(h->in.size() * 4), tsum(h->in.size());
    int nctr = 0;
    for (size_t i = 0; i < h->in.size(); ++i) {
        Inst& I = h->in[i];
        float2* f = inst_psi(I, psi);
        ctr_base.push_back(nctr);
        nctr += I.n_pairs;
        argi.push_back((int)A.size());
        // pass arguments: x rows (first step's kick, later kicks), y columns, x rows, y columns
        A.push_back(make_args(h, I, f, 0, a_first, I.vc, nullptr));
        A.push_back(make_args(h, I, f, 0, 1.0, I.vc, nullptr));
        A.push_back(make_args(h, I, f, 1, 0.0, I.vc, nullptr));
        A.push_back(make_args(h, I, f, 0, 0.0, I.vc, nullptr));
        A.push_back(make_args(h, I, f, 1, 0.0, I.vc, nullptr));
        for (int q = 0; q < 4; ++q) {
            const int ax = q & 1, N = I.n[ax], L = batch_lines(N);
            const long long lines = I.cells / N;  // rows (x) or columns (y) of the field
            tiles[4 * i + q] = (int)((lines + L - 1) / L);
            tsum[i] += tiles[4 * i + q];
            const int k = batch_kind(N, q);
            if (std::find(kinds.begin(), kinds.end(), k) == kinds.end()) kinds.push_back(k);
        }
    }
    long long tick = 0;
    for (int st_ = 0; st_ < n; ++st_)
        for (int q = 0; q < 4; ++q)
            for (size_t i = 0; i < h->in.size(); ++i) {
                const Inst& I = h->in[i];
                int pre = st_ * tsum[i];
                for (int r = 0; r < q; ++r) pre += tiles[4 * i + r];
                BatchPass b{};
                b.first = tick;
                b.kind = batch_kind(I.n[q & 1], q);
                b.tiles = tiles[4 * i + q];
                // one tile per ticket: several tiles per ticket (up to 16) measured slower on the
                // uneven 2D mix (70.6 against 56.3 ms per 10 steps), longer items leaving CTAs idle
                b.per_item = 1;
                b.items = (b.tiles + b.per_item - 1) / b.per_item;
                b.fields = I.n_pairs;
                b.args = argi[i] + (q == 0 ? (st_ == 0 ? 0 : 1) : q + 1);
                b.ctr = ctr_base[i];
                b.target = pre;
                P.push_back(b);
                tick += (long long)b.items * b.fields;
            }
    if (stall && P.size() > h->in.size()) P[h->in.size()].target += 1;  // a tile that no item produces
    if (!h->d_ctr) RC(dalloc(h, &h->d_ctr, (size_t)nctr));
    if (!h->d_tick) RC(dalloc(h, &h->d_tick, 2));
    twa_handle::BatchTable T{};
    RC(dalloc(h, &T.passes, P.size()));
    RC(dalloc(h, &T.args, A.size()));
    CU(cudaMemcpyAsync(T.passes, P.data(), P.size() * sizeof(BatchPass), cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(T.args, A.data(), A.size() * sizeof(PassArgs), cudaMemcpyHostToDevice, st));
    T.n_passes = (int)P.size();
    T.n_items = tick;
    T.kinds = kinds;
    h->btab.push_back({stall ? std::vector<double>{-1.0} : key, T});
    *out = &h->btab.back().second;
    return 0;
}

// n KDK steps (first kick a_first) of every instance in one persistent launch.
int batch_steps(twa_handle* h, void* psi, int n, double a_first, cudaStream_t st) {
    if (n <= 0) return 0;
    twa_handle::BatchTable* T = nullptr;
    RC(batch_table(h, psi, n, a_first, st, &T));
    h->stall_next = false;
    size_t nctr = 0;
    for (const auto& I : h->in) nctr += (size_t)I.n_pairs;
    CU(cudaMemsetAsync(h->d_ctr, 0, nctr * sizeof(unsigned), st));
    CU(cudaMemsetAsync(h->d_tick, 0, 2 * sizeof(unsigned long long), st));
    const long long budget = (long long)(h->wait_limit_s * (double)h->clock_khz * 1e3);
    if (launch_batch(T->passes, T->n_passes, T->args, h->d_ctr, h->d_tick, T->n_items, h->d_err,
                     reinterpret_cast<int*>(h->d_tick + 1), budget, T->kinds.data(), (int)T->kinds.size(), st) != 0)
        return fail(h, TWA_ECUDA, "persistent batch launch: cudaFuncSetAttribute failed");
    ++h->launches;
    return 0;
}

// Moments with a pending kick (0 for a synchronized batch); scalars into `scalars` (device).
int moments_f32(twa_handle* h, Inst& I, float2* psi, double pend, const twa_moments_out* o, double* scalars,
                cudaStream_t st) {
    const bool v_spec = (I.mode == MODE_3D) && pend != 0.0;
    float pk, pkl;
    split_kick(h, I, pend, pk, pkl);
    if (v_spec) RC(run_pass(h, I, psi, 0, OP_INV, 0.0, I.vc, nullptr, I.n_pairs, st));
    const int nb = moments_blocks(I.cells);
    const double ns = (double)I.n_real;
    const double weyl = 1.0 / (2.0 * h->p.n_tot * I.dV);
    launch_moments_real(psi, I.vc, I.cells, I.n_slots, pk, pkl, 1.0 / ns, weyl, o ? o->rho_mean : nullptr,
                        o ? o->psi_mean : nullptr, o ? o->rho_cl : nullptr, I.part_r, st);
    ++h->launches;
    int nbm = 0;
    if (h->p.want_modes && I.spec) {
        RC(run_pass(h, I, psi, 0, OP_KICK_FWD_OUT, pend, I.vc, I.spec, I.n_pairs, st, 0, I.mode == MODE_1D ? 1 : 0));
        for (int ax = 1; ax < I.dim; ++ax) RC(run_pass(h, I, psi, ax, OP_FWD, 0.0, I.spec, nullptr, I.n_slots, st));
        launch_moments_modes(I.spec, I.cells, I.n_slots, h->p.n_tot * I.dV / (double)I.cells, 1.0 / ns,
                             o ? o->nk_mean : nullptr, o ? o->nk_var : nullptr, o ? o->nk_cl : nullptr, I.part_m, st);
        ++h->launches;
        nbm = nb;
    }
    launch_finish_scalars(I.part_r, nb, I.part_m, nbm, I.dV, (double)I.cells / (2.0 * h->p.n_tot), scalars, h->d_err, st);
    ++h->launches;
    // restore the x-spectral Poisson field: the unnormalized forward transform of the inverse
    // multiplies by N_x, which the post factor removes
    if (v_spec) RC(run_pass(h, I, psi, 0, OP_FWD, 0.0, I.vc, nullptr, I.n_pairs, st, 0, 0, 1.0f / (float)I.n[0]));
    return 0;
}

// ---------------------------------------------------------------------------------------------
// FP64 plain path.
Geom64 geom64(const Inst& I) {
    Geom64 g{};
    g.dim = I.dim;
    for (int a = 0; a < 3; ++a) g.n[a] = I.n[a];
    g.cells = I.cells;
    return g;
}
Tables64 tables64(const Inst& I) {
    Tables64 t{};
    for (int a = 0; a < 3; ++a) {
        t.tw[a] = I.tw64[a];
        t.ph[a] = I.ph64[a];
        t.k2[a] = I.k264[a];
    }
    return t;
}

int poisson_f64(twa_handle* h, Inst& I, double2* f, cudaStream_t st) {
    const Geom64 g = geom64(I);
    const Tables64 t = tables64(I);
    launch_f64_rho(f, I.work64, I.cells, st, &h->launches);
    launch_f64_fft3(I.work64, g, t, false, st, &h->launches);
    launch_f64_poisson_mul(I.work64, g, t, -h->p.C / (double)I.cells, st, &h->launches);
    launch_f64_fft3(I.work64, g, t, true, st, &h->launches);
    return 0;
}

int step_batch_f64(twa_handle* h, Inst& I, double2* psi, int n, cudaStream_t st) {
    const Geom64 g = geom64(I);
    const Tables64 t = tables64(I);
    const double kh = h->p.dt / (2.0 * h->p.hbar_m), kf = h->p.dt / h->p.hbar_m;
    for (int s = 0; s < I.n_slots; ++s) {
        double2* f = psi + (size_t)s * I.cells;
        RC(poisson_f64(h, I, f, st));
        launch_f64_kick(f, I.work64, I.cells, kh, st, &h->launches);
        for (int k = 0; k < n; ++k) {
            launch_f64_fft3(f, g, t, false, st, &h->launches);
            launch_f64_kinetic(f, g, t, st, &h->launches);
            launch_f64_fft3(f, g, t, true, st, &h->launches);
            RC(poisson_f64(h, I, f, st));
            launch_f64_kick(f, I.work64, I.cells, (k == n - 1) ? kh : kf, st, &h->launches);
        }
    }
    return 0;
}

int moments_f64(twa_handle* h, Inst& I, double2* psi, const twa_moments_out* o, double* scalars, cudaStream_t st) {
    const Geom64 g = geom64(I);
    const Tables64 t = tables64(I);
    CU(cudaMemsetAsync(I.bad64, 0, sizeof(double), st));
    const bool modes = h->p.want_modes && I.spec64;
    for (int s = 1; s < I.n_slots; ++s) {
        double2* f = psi + (size_t)s * I.cells;
        launch_f64_moments_accum(f, nullptr, I.cells, 0.0, s == 1, I.acc64, I.bad64, st, &h->launches);
        if (modes) {
            CU(cudaMemcpyAsync(I.spec64, f, I.cells * sizeof(double2), cudaMemcpyDeviceToDevice, st));
            launch_f64_fft3(I.spec64, g, t, false, st, &h->launches);
            launch_f64_modes_accum(I.spec64, I.cells, h->p.n_tot * I.dV / (double)I.cells, s == 1, I.acc64m, st,
                                   &h->launches);
        }
    }
    launch_f64_moments_finish(I.acc64, modes ? I.acc64m : nullptr, psi, I.cells, I.n_real,
                              1.0 / (2.0 * h->p.n_tot * I.dV), I.dV, (double)I.cells / (2.0 * h->p.n_tot),
                              o ? o->rho_mean : nullptr, o ? o->psi_mean : nullptr, o ? o->rho_cl : nullptr,
                              o ? o->nk_mean : nullptr, o ? o->nk_var : nullptr, I.part_r, I.part_m, I.bad64, scalars,
                              h->d_err, st, &h->launches);
    return 0;
}

// ---------------------------------------------------------------------------------------------
int build_tables(twa_handle* h, Inst& I) {
    const double hb = h->p.hbar_m, dt = h->p.dt;
    for (int a = 0; a < 3; ++a) {
        const int n = I.n[a];
        std::vector<float> k2f(n);
        std::vector<double> k2d(n);
        std::vector<float2> phf(n), phl(n);
        std::vector<double2> phd(n), twd(n);
        for (int j = 0; j < n; ++j) {
            const double k = (a < I.dim) ? wavenumber(j, n, I.L) : 0.0;
            k2d[j] = k * k;
            k2f[j] = (float)(k * k);
            double c, s;
            phase_of(hb * k * k * dt / 2.0, c, s);
            phd[j] = make_double2(c, s);
            phf[j] = make_float2((float)(c / n), (float)(s / n));
            phl[j] = make_float2((float)(c / n - (double)phf[j].x), (float)(s / n - (double)phf[j].y));
            const double ang = -2.0 * M_PI * (double)j / (double)n;
            twd[j] = make_double2(std::cos(ang), std::sin(ang));
        }
        if (h->p.precision == TWA_F32) {
            RC(upload(h, &I.k2[a], k2f));
            std::vector<float4> phc(n);
            for (int j = 0; j < n; ++j) phc[j] = make_float4(phf[j].x, phf[j].y, phl[j].x, phl[j].y);
            RC(upload(h, &I.ph[a], phc));
            if (a < I.dim && !h->tw32.count(n)) {
                // stage-major table of W_n^m (m from the plan's stage layout), hi + lo
                std::vector<float4> tw;
                for (int e = 0; tw_exponent_n(n, e) >= 0; ++e) {
                    const int m = tw_exponent_n(n, e);
                    const double c = twd[m].x, sv = twd[m].y;
                    const float hx = (float)c, hy = (float)sv;
                    tw.push_back(make_float4(hx, hy, (float)(c - (double)hx), (float)(sv - (double)hy)));
                }
                if (tw.empty()) tw.push_back(make_float4(1.f, 0.f, 0.f, 0.f));
                float4* d = nullptr;
                RC(upload(h, &d, tw));
                h->tw32[n] = d;
            }
        } else {
            RC(upload(h, &I.k264[a], k2d));
            RC(upload(h, &I.ph64[a], phd));
            RC(upload(h, &I.tw64[a], twd));
        }
    }
    return 0;
}

}  // namespace

namespace twa {
int plan_threads_per_line(int n) {
    switch (n) {
        case 8: return Plan<8>::T;
        case 16: return Plan<16>::T;
        case 32: return Plan<32>::T;
        case 64: return Plan<64>::T;
        case 128: return Plan<128>::T;
        case 256: return Plan<256>::T;
        case 512: return Plan<512>::T;
        case 1024: return Plan<1024>::T;
        case 2048: return Plan<2048>::T;
        default: return 1;
    }
}
}  // namespace twa

// =============================================================================================
extern "C" {

int twa_create(twa_handle** out, const twa_grid* grids, const twa_params* p, int n_inst, const int* n_real) {
    twa_handle* h = nullptr;
    if (!out || !grids || !p || !n_real || n_inst <= 0) return fail(nullptr, TWA_EINVAL, "twa_create: null argument");
    *out = nullptr;
    if (p->precision != TWA_F32 && p->precision != TWA_F64_PLAIN)
        return fail(nullptr, TWA_EINVAL, "twa_create: unknown precision");
    if (!(p->hbar_m > 0) || !(p->dt > 0) || !(p->n_tot > 0))
        return fail(nullptr, TWA_EINVAL, "twa_create: hbar_m, dt and n_tot must be positive");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(nullptr, TWA_ECUDA, "twa_create: no CUDA device");
    }
    h = new twa_handle();
    h->p = *p;
    size_t off = 0;
    for (int i = 0; i < n_inst; ++i) {
        Inst I;
        const twa_grid& g = grids[i];
        if (g.dim < 1 || g.dim > 3 || n_real[i] < 1 || !(g.L > 0)) {
            twa_destroy(h);
            return fail(nullptr, TWA_EINVAL, "twa_create: bad grid or realization count");
        }
        I.dim = g.dim;
        I.L = g.L;
        I.cells = 1;
        for (int a = 0; a < 3; ++a) {
            I.n[a] = (a < g.dim) ? g.n[a] : 1;
            if (a < g.dim && (!pow2(I.n[a]) || I.n[a] < 8 || I.n[a] > 2048)) {
                twa_destroy(h);
                return fail(nullptr, TWA_EINVAL, "twa_create: axis lengths must be powers of two in [8, 2048]");
            }
            I.lg[a] = ilog2(I.n[a]);
            I.cells *= I.n[a];
        }
        I.dV = 1.0;
        for (int a = 0; a < g.dim; ++a) I.dV *= g.L / I.n[a];
        I.n_real = n_real[i];
        I.n_slots = n_real[i] + 1;
        I.n_pairs = (I.n_slots + 1) / 2;
        I.off = off;
        off += (size_t)I.n_slots * I.cells;
        I.mode = (g.dim == 1) ? MODE_1D : (g.dim == 2 ? MODE_2D : MODE_3D);
        if (g.dim == 3 && I.n[0] == I.n[1] && I.n[0] >= 16 && I.n[0] <= 256) I.mode = MODE_3DP;
        h->in.push_back(I);
    }
    // fork batches whose instances are all small (at most 2^22 complex values each)
    h->fork = n_inst > 1;
    for (const auto& I : h->in) h->fork = h->fork && (long long)I.n_slots * I.cells <= (1LL << 22);
    int rc = 0;
    auto bail = [&](int code) {
        g_create_error = h->err;
        twa_destroy(h);
        return code;
    };
    if ((rc = dalloc(h, &h->d_err, 1))) return bail(rc);
    {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&h->clock_khz, cudaDevAttrClockRate, dev);
        if (h->clock_khz <= 0) h->clock_khz = 2000000;
    }
    if ((rc = dalloc(h, &h->d_vmax, (size_t)n_inst))) return bail(rc);
    if ((rc = dalloc(h, &h->d_counter, 1))) return bail(rc);
    if ((rc = dalloc(h, &h->d_cur, (size_t)n_inst * TWA_NSCALARS))) return bail(rc);
    cudaMemset(h->d_err, 0, sizeof(int));
    cudaMemset(h->d_counter, 0, sizeof(int));
    for (auto& I : h->in) {
        if ((rc = build_tables(h, I))) return bail(rc);
        const int nb = moments_blocks(I.cells);
        if ((rc = dalloc(h, &I.part_r, (size_t)nb * NP_REAL))) return bail(rc);
        if ((rc = dalloc(h, &I.part_m, (size_t)nb * NP_MODES))) return bail(rc);
        if (p->precision == TWA_F32) {
            if ((rc = dalloc(h, &I.vc, (size_t)I.n_pairs * I.cells))) return bail(rc);
            cudaMemset(I.vc, 0, (size_t)I.n_pairs * I.cells * sizeof(float2));
            if (p->want_modes && (rc = dalloc(h, &I.spec, (size_t)I.n_slots * I.cells))) return bail(rc);
        } else {
            if ((rc = dalloc(h, &I.work64, (size_t)I.cells))) return bail(rc);
            if ((rc = dalloc(h, &I.acc64, (size_t)3 * I.cells))) return bail(rc);
            if ((rc = dalloc(h, &I.bad64, 1))) return bail(rc);
            if (p->want_modes) {
                if ((rc = dalloc(h, &I.spec64, (size_t)I.cells))) return bail(rc);
                if ((rc = dalloc(h, &I.acc64m, (size_t)2 * I.cells))) return bail(rc);
            }
        }
    }
    if (cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_a, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_b, cudaEventDisableTiming) != cudaSuccess) {
        h->err = "stream/event creation failed";
        return bail(TWA_ECUDA);
    }
    if (cudaDeviceSynchronize() != cudaSuccess) {
        h->err = "device synchronize after setup failed";
        return bail(TWA_ECUDA);
    }
    *out = h;
    return TWA_OK;
}

int twa_destroy(twa_handle* h) {
    if (!h) return TWA_OK;
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    for (auto& r : h->prof_pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (cudaEvent_t e : h->prof_pool) cudaEventDestroy(e);
    if (h->cap) cudaStreamDestroy(h->cap);
    if (h->ev_a) cudaEventDestroy(h->ev_a);
    if (h->ev_b) cudaEventDestroy(h->ev_b);
    for (cudaStream_t x : h->side) cudaStreamDestroy(x);
    for (cudaEvent_t e : h->side_ev) cudaEventDestroy(e);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    for (void* p : h->allocs) cudaFree(p);
    delete h;
    return TWA_OK;
}

size_t twa_batch_elems(const twa_handle* h) {
    if (!h) return 0;
    size_t n = 0;
    for (const auto& I : h->in) n += (size_t)I.n_slots * I.cells;
    return n;
}

int twa_sample(twa_handle* h, const void* psi_cl, uint64_t seed, void* psi, void* stream) {
    if (!h) return fail(nullptr, TWA_EINVAL, "null handle");
    if (!psi_cl || !psi) return fail(h, TWA_EINVAL, "twa_sample: null buffer");
    if (misaligned(psi_cl) || misaligned(psi)) return fail(h, TWA_EINVAL, "twa_sample: buffers must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    h->launches = 0;
    size_t cl_off = 0;
    for (size_t i = 0; i < h->in.size(); ++i) {
        Inst& I = h->in[i];
        const double var_mode = h->p.noise_conv == 0 ? 0.5 : 1.0;
        const double sigma = std::sqrt(var_mode / (2.0 * h->p.n_tot * I.dV));
        const double2* cl = static_cast<const double2*>(psi_cl) + cl_off;
        if (h->p.precision == TWA_F32)
            launch_sample_f32(cl, static_cast<float2*>(psi) + I.off, I.cells, I.n_slots, seed, (int)i, sigma, st);
        else
            launch_sample_f64(cl, static_cast<double2*>(psi) + I.off, I.cells, I.n_slots, seed, (int)i, sigma, st);
        ++h->launches;
        cl_off += (size_t)I.cells;
    }
    CU(cudaGetLastError());
    return TWA_OK;
}

int twa_step_batch(twa_handle* h, void* psi, int n_steps, void* stream) {
    if (!h) return fail(nullptr, TWA_EINVAL, "null handle");
    if (!psi || n_steps < 0) return fail(h, TWA_EINVAL, "twa_step_batch: bad argument");
    if (misaligned(psi)) return fail(h, TWA_EINVAL, "twa_step_batch: psi must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    h->launches = 0;
    if (n_steps == 0) return TWA_OK;
    if (use_batch(h)) {
        for (auto& I : h->in) RC(poisson_init(h, I, inst_psi(I, psi), st));
        RC(batch_steps(h, psi, n_steps, 0.5, st));
        for (auto& I : h->in) RC(closing_kick(h, I, inst_psi(I, psi), 0.5, st));
        CU(cudaGetLastError());
        return TWA_OK;
    }
    Fork fk{h, st, false};
    RC(fk.open(h->in.size()));
    for (size_t i = 0; i < h->in.size(); ++i) {
        Inst& I = h->in[i];
        cudaStream_t s;
        RC(fk.stream(i, &s));
        if (h->p.precision == TWA_F32) {
            float2* f = inst_psi(I, psi);
            RC(poisson_init(h, I, f, s));
            RC(steps_f32(h, I, f, n_steps, 0.5, s));
            RC(closing_kick(h, I, f, 0.5, s));
        } else {
            RC(step_batch_f64(h, I, static_cast<double2*>(psi) + I.off, n_steps, s));
        }
        RC(fk.join(i));
    }
    CU(cudaGetLastError());
    return TWA_OK;
}

int twa_moments(twa_handle* h, int inst, const void* psi, const twa_moments_out* out, void* stream) {
    if (!h) return fail(nullptr, TWA_EINVAL, "null handle");
    if (!psi || !out || inst < 0 || inst >= (int)h->in.size()) return fail(h, TWA_EINVAL, "twa_moments: bad argument");
    if (misaligned(psi)) return fail(h, TWA_EINVAL, "twa_moments: psi must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    h->launches = 0;
    Inst& I = h->in[inst];
    double* sc = out->scalars ? out->scalars : h->d_cur + (size_t)inst * TWA_NSCALARS;
    if (h->p.precision == TWA_F32)
        RC(moments_f32(h, I, inst_psi(I, const_cast<void*>(psi)), 0.0, out, sc, st));
    else
        RC(moments_f64(h, I, static_cast<double2*>(const_cast<void*>(psi)) + I.off, out, sc, st));
    CU(cudaGetLastError());
    return TWA_OK;
}

}  // extern "C"

namespace {

// One output interval of the FP32 run for all instances: steps, moments (pending half kick), store.
int run_interval_f32(twa_handle* h, void* psi, int out_every, double a_first, double* series, cudaStream_t st) {
    if (use_batch(h)) {
        RC(batch_steps(h, psi, out_every, a_first, st));
        for (size_t i = 0; i < h->in.size(); ++i) {
            Inst& I = h->in[i];
            RC(moments_f32(h, I, inst_psi(I, psi), 0.5, nullptr, h->d_cur + i * TWA_NSCALARS, st));
        }
        launch_store_series(h->d_cur, series, h->d_counter, (int)h->in.size() * TWA_NSCALARS, st);
        ++h->launches;
        return 0;
    }
    Fork fk{h, st, false};
    RC(fk.open(h->in.size()));
    for (size_t i = 0; i < h->in.size(); ++i) {
        Inst& I = h->in[i];
        float2* f = inst_psi(I, psi);
        cudaStream_t s;
        RC(fk.stream(i, &s));
        RC(steps_f32(h, I, f, out_every, a_first, s));
        RC(moments_f32(h, I, f, 0.5, nullptr, h->d_cur + i * TWA_NSCALARS, s));
        RC(fk.join(i));
    }
    launch_store_series(h->d_cur, series, h->d_counter, (int)h->in.size() * TWA_NSCALARS, st);
    ++h->launches;
    return 0;
}

// Rewrite the FP32 kinetic-phase tables of every axis for the handle's current dt (as build_tables:
// phase reduced in FP64, stored as float hi + lo), in stream order.
int write_phase_tables(twa_handle* h, Inst& I, cudaStream_t st) {
    const double hb = h->p.hbar_m, dt = h->p.dt;
    for (int a = 0; a < 3; ++a) {
        const int n = I.n[a];
        std::vector<float4> phc(n);
        for (int j = 0; j < n; ++j) {
            const double k = (a < I.dim) ? wavenumber(j, n, I.L) : 0.0;
            double c, s;
            phase_of(hb * k * k * dt / 2.0, c, s);
            const float cx = (float)(c / n), sy = (float)(s / n);
            phc[j] = make_float4(cx, sy, (float)(c / n - (double)cx), (float)(s / n - (double)sy));
        }
        CU(cudaMemcpyAsync(I.ph[a], phc.data(), (size_t)n * sizeof(float4), cudaMemcpyHostToDevice, st));
    }
    return 0;
}

// Set the time step of every later kick and drift (a captured interval graph is dropped).
int set_dt(twa_handle* h, double dt, cudaStream_t st) {
    h->p.dt = dt;
    for (auto& I : h->in) RC(write_phase_tables(h, I, st));
    if (h->gexec) {
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
    }
    return 0;
}

// Time step of Sec. III.B.2 from the synchronized (kick pending) FP32 batch: per instance the
// largest |V| = |C| max|W| / cells over its streams and cells (W, the packed Poisson field, made
// real along x first where it is kept x-spectral), then
//   dt = 2 pi c_f min over instances of min[ hbar / max|V| ,  L dx_min / (pi hbar) ].
// Reads the maxima back: synchronizes the stream.
int adaptive_dt(twa_handle* h, void* psi, double c_f, cudaStream_t st, double* dt_out) {
    const size_t ni = h->in.size();
    CU(cudaMemsetAsync(h->d_vmax, 0, ni * sizeof(unsigned), st));
    for (size_t i = 0; i < ni; ++i) {
        Inst& I = h->in[i];
        float2* f = inst_psi(I, psi);
        const bool v_spec = I.mode == MODE_3D;
        if (v_spec) RC(run_pass(h, I, f, 0, OP_INV, 0.0, I.vc, nullptr, I.n_pairs, st));
        launch_max_abs(I.vc, (long long)I.n_pairs * I.cells, h->d_vmax + i, st);
        ++h->launches;
        if (v_spec) RC(run_pass(h, I, f, 0, OP_FWD, 0.0, I.vc, nullptr, I.n_pairs, st, 0, 0, 1.0f / (float)I.n[0]));
    }
    std::vector<unsigned> bits(ni);
    CU(cudaMemcpyAsync(bits.data(), h->d_vmax, ni * sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    double dt = INFINITY;
    const double hb = h->p.hbar_m;
    for (size_t i = 0; i < ni; ++i) {
        const Inst& I = h->in[i];
        float w;
        std::memcpy(&w, &bits[i], sizeof(float));
        const double vmax = std::fabs(h->p.C) * (double)w / (double)I.cells;
        double dx = INFINITY;
        for (int a = 0; a < I.dim; ++a) dx = std::min(dx, I.L / I.n[a]);
        const double kin = I.L * dx / (M_PI * hb);
        const double pot = vmax > 0.0 ? hb / vmax : INFINITY;
        dt = std::min(dt, std::min(pot, kin));
    }
    *dt_out = 2.0 * M_PI * c_f * dt;
    return 0;
}

// Whole 1D runs (run1d.cuh): every instance 1D, no test particles, the pass profiler off.
bool run1d_eligible(const twa_handle* h) {
    if (h->p.precision != TWA_F32 || h->prof_on) return false;
    for (const auto& I : h->in)
        if (I.mode != MODE_1D || I.prt) return false;
    return true;
}

int dispatch_run1d(int N, const Run1DArgs& r, cudaStream_t st) {
    switch (N) {
        case 8: return launch_run1d<8>(r, st);
        case 16: return launch_run1d<16>(r, st);
        case 32: return launch_run1d<32>(r, st);
        case 64: return launch_run1d<64>(r, st);
        case 128: return launch_run1d<128>(r, st);
        case 256: return launch_run1d<256>(r, st);
        case 512: return launch_run1d<512>(r, st);
        case 1024: return launch_run1d<1024>(r, st);
        case 2048: return launch_run1d<2048>(r, st);
        default: return -1;
    }
}

// n_out output intervals of out_every steps of every (1D) instance of a synchronized batch, with
// the scalars of outputs 0..n_out written to series: one on-chip launch per instance and chunk of
// outputs (the partial sums are kept under 256 MB per instance) plus one finishing launch.
int run1d_all(twa_handle* h, void* psi, int n_out, int out_every, double* series, cudaStream_t st) {
    const int ni = (int)h->in.size();
    for (int i = 0; i < ni; ++i) {
        Inst& I = h->in[i];
        const long long N = I.cells, P = I.n_pairs;
        const long long per_out = P * 3 * N + N + P;
        const long long cap = std::max(1LL, (256LL << 20) / (8 * per_out) - 1);
        const int chunk = (int)std::min<long long>(std::max(n_out, 1), cap);
        const size_t need = (size_t)(chunk + 1) * per_out;
        if (I.run_part_n < need) {
            RC(dalloc(h, &I.run_part, need));
            I.run_part_n = need;
        }
        double* part = I.run_part;
        double* part_cl = part + (size_t)(chunk + 1) * P * 3 * N;
        double* part_bad = part_cl + (size_t)(chunk + 1) * N;
        const double inv_ns = 1.0 / (double)I.n_real, weyl = 1.0 / (2.0 * h->p.n_tot * I.dV);
        const double q_off = (double)I.cells / (2.0 * h->p.n_tot), nm = h->p.want_modes ? h->p.n_tot : 0.0;
        int done = 0;
        do {
            const int k = std::min(chunk, n_out - done);
            Run1DArgs r{};
            r.a = make_args(h, I, inst_psi(I, psi), 0, 0.5, I.vc, nullptr);
            r.n_out = k;
            r.out_every = out_every;
            r.part = part;
            r.part_cl = part_cl;
            r.part_bad = part_bad;
            if (dispatch_run1d((int)N, r, st) != 0) return fail(h, TWA_ECUDA, "1D run: kernel attribute setup failed");
            ++h->launches;
            // the first chunk reports its initial output; later chunks start where the last one ended
            const int skip = done == 0 ? 0 : 1;
            launch_finish_run1d(part + skip * P * 3 * N, part_cl + skip * N, part_bad + skip * P, (int)P, (int)N,
                                k + 1 - skip, inv_ns, weyl, I.dV, q_off, nm, series, done + skip, i, ni, h->d_err, st);
            ++h->launches;
            done += k;
        } while (done < n_out);
    }
    return 0;
}

}  // namespace

extern "C" {

int twa_advance(twa_handle* h, void* psi_work, int n_steps, int out_every, double* series, void* stream) {
    if (!h) return fail(nullptr, TWA_EINVAL, "null handle");
    if (!psi_work || !series || out_every <= 0 || n_steps < 0 || n_steps % out_every)
        return fail(h, TWA_EINVAL, "twa_advance: bad argument (n_steps must be a multiple of out_every)");
    if (misaligned(psi_work)) return fail(h, TWA_EINVAL, "twa_advance: psi must be 16-byte aligned");
    cudaStream_t user = (cudaStream_t)stream;
    long long total = 0;
    h->launches = 0;
    const int n_out = n_steps / out_every;
    CU(cudaMemsetAsync(h->d_counter, 0, sizeof(int), user));
    if (h->p.precision == TWA_F64_PLAIN) {
        for (int o = 0; o <= n_out; ++o) {
            if (o > 0) {
                RC(twa_step_batch(h, psi_work, out_every, stream));
                total += h->launches;
            }
            h->launches = 0;
            for (size_t i = 0; i < h->in.size(); ++i) {
                Inst& I = h->in[i];
                RC(moments_f64(h, I, static_cast<double2*>(psi_work) + I.off, nullptr, h->d_cur + i * TWA_NSCALARS, user));
            }
            launch_store_series(h->d_cur, series, h->d_counter, (int)h->in.size() * TWA_NSCALARS, user);
            total += h->launches + 1;
        }
        h->launches = total;
        CU(cudaGetLastError());
        return TWA_OK;
    }
    if (run1d_eligible(h)) {
        RC(run1d_all(h, psi_work, n_out, out_every, series, user));
        CU(cudaGetLastError());
        return TWA_OK;
    }
    // FP32: eager prologue and first interval, then one captured graph per later interval.
    const double kh = 0.5, kf = 1.0;
    for (size_t i = 0; i < h->in.size(); ++i) {
        Inst& I = h->in[i];
        float2* f = inst_psi(I, psi_work);
        RC(poisson_init(h, I, f, user));
        RC(moments_f32(h, I, f, 0.0, nullptr, h->d_cur + i * TWA_NSCALARS, user));
    }
    launch_store_series(h->d_cur, series, h->d_counter, (int)h->in.size() * TWA_NSCALARS, user);
    ++h->launches;
    if (n_out >= 1) RC(run_interval_f32(h, psi_work, out_every, kh, series, user));
    total += h->launches;
    if (n_out >= 2 && h->prof_on) {
        for (int o = 2; o <= n_out; ++o) RC(run_interval_f32(h, psi_work, out_every, kf, series, user));
        total += h->launches;
    } else if (n_out >= 2) {
        const bool reuse = h->gexec && h->g_psi == psi_work && h->g_series == series && h->g_out_every == out_every;
        if (!reuse) {
            if (h->gexec) {
                cudaGraphExecDestroy(h->gexec);
                h->gexec = nullptr;
            }
            if (use_batch(h)) {
                // the persistent launch's work list is uploaded outside the capture
                twa_handle::BatchTable* T = nullptr;
                RC(batch_table(h, psi_work, out_every, kf, user, &T));
            }
            CU(cudaEventRecord(h->ev_a, user));
            CU(cudaStreamWaitEvent(h->cap, h->ev_a, 0));
            h->launches = 0;
            CU(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
            int rc = run_interval_f32(h, psi_work, out_every, kf, series, h->cap);
            cudaGraph_t g = nullptr;
            cudaError_t ce = cudaStreamEndCapture(h->cap, &g);
            if (rc) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            if (ce != cudaSuccess) return fail(h, TWA_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
            ce = cudaGraphInstantiate(&h->gexec, g, 0);
            cudaGraphDestroy(g);
            if (ce != cudaSuccess) return fail(h, TWA_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce));
            h->graph_launches = h->launches;
            h->g_psi = psi_work;
            h->g_series = series;
            h->g_out_every = out_every;
        } else {
            CU(cudaEventRecord(h->ev_a, user));
            CU(cudaStreamWaitEvent(h->cap, h->ev_a, 0));
        }
        for (int o = 2; o <= n_out; ++o) CU(cudaGraphLaunch(h->gexec, h->cap));
        total += h->graph_launches * (n_out - 1);
        CU(cudaEventRecord(h->ev_b, h->cap));
        CU(cudaStreamWaitEvent(user, h->ev_b, 0));
    }
    h->launches = 0;
    // the last step's closing half kick (with no step taken the batch is already synchronized)
    if (n_out >= 1)
        for (auto& I : h->in) RC(closing_kick(h, I, inst_psi(I, psi_work), kh, user));
    total += h->launches;
    h->launches = total;
    CU(cudaGetLastError());
    return TWA_OK;
}

int twa_particles_set(twa_handle* h, int inst, const double* rp, void* stream) {
    if (!h) return fail(nullptr, TWA_EINVAL, "null handle");
    if (!rp || inst < 0 || inst >= (int)h->in.size()) return fail(h, TWA_EINVAL, "twa_particles_set: bad argument");
    if (h->p.precision != TWA_F32) return fail(h, TWA_EINVAL, "twa_particles_set: FP32 path only");
    Inst& I = h->in[inst];
    if (!I.prt) {
        RC(dalloc(h, &I.prt, (size_t)I.n_slots * 6));
        // derivative kernel of each axis: d(m) = (1/n) sum_k i k exp(i k m dx), Nyquist mode excluded
        for (int a = 0; a < I.dim; ++a) {
            const int n = I.n[a];
            std::vector<double> d(n, 0.0);
            for (int m = 0; m < n; ++m) {
                double acc = 0.0;
                for (int j = 0; j < n; ++j) {
                    if (n % 2 == 0 && j == n / 2) continue;
                    const double k = wavenumber(j, n, I.L);
                    acc -= k * std::sin(k * m * (I.L / n));
                }
                d[m] = acc / n;
            }
            RC(upload(h, &I.dker[a], d));
        }
    }
    for (int s = 0; s < I.n_slots; ++s)
        for (int a = 0; a < 6; ++a)
            if (!std::isfinite(rp[6 * s + a])) return fail(h, TWA_EINVAL, "twa_particles_set: non-finite state");
    std::vector<double> q(rp, rp + (size_t)6 * I.n_slots);
    for (int s = 0; s < I.n_slots; ++s)
        for (int a = 0; a < 3; ++a) {
            if (a >= I.dim) {
                q[6 * s + a] = 0.0;
                q[6 * s + 3 + a] = 0.0;
            } else {
                q[6 * s + a] = std::fmod(q[6 * s + a], I.L);
                if (q[6 * s + a] < 0.0) q[6 * s + a] += I.L;
            }
        }
    CU(cudaMemcpyAsync(I.prt, q.data(), q.size() * sizeof(double), cudaMemcpyHostToDevice, (cudaStream_t)stream));
    // the particles need the potential in real space before every step: the plane pipeline keeps it
    // so, the axis pipeline would transform it back and forth each step (every call restarts the
    // Poisson field from the batch, so the switch is safe between calls)
    if (I.mode == MODE_3D && I.n[0] == I.n[1] && I.n[0] >= 16 && I.n[0] <= 256) I.mode = MODE_3DP;
    if (h->gexec) {
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
    }
    return TWA_OK;
}

int twa_particles_get(twa_handle* h, int inst, double* rp, void* stream) {
    if (!h) return fail(nullptr, TWA_EINVAL, "null handle");
    if (!rp || inst < 0 || inst >= (int)h->in.size()) return fail(h, TWA_EINVAL, "twa_particles_get: bad argument");
    Inst& I = h->in[inst];
    if (!I.prt) return fail(h, TWA_EINVAL, "twa_particles_get: no particles set on this instance");
    cudaStream_t st = (cudaStream_t)stream;
    CU(cudaMemcpyAsync(rp, I.prt, (size_t)I.n_slots * 6 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    return TWA_OK;
}

int twa_phase_moments(twa_handle* h, int inst, const void* psi, double* var_a, double* phi2, double* totals,
                      void* stream) {
    if (!h) return fail(nullptr, TWA_EINVAL, "null handle");
    if (!psi || !totals || inst < 0 || inst >= (int)h->in.size())
        return fail(h, TWA_EINVAL, "twa_phase_moments: bad argument");
    if (misaligned(psi)) return fail(h, TWA_EINVAL, "twa_phase_moments: psi must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    Inst& I = h->in[inst];
    const double weyl = 1.0 / (2.0 * h->p.n_tot * I.dV);
    if (h->p.precision == TWA_F32)
        launch_phase_moments(inst_psi(I, const_cast<void*>(psi)), I.cells, I.n_slots, weyl, I.dV, var_a, phi2, I.part_r,
                             totals, st);
    else
        launch_phase_moments_f64(static_cast<const double2*>(psi) + I.off, I.cells, I.n_slots, weyl, I.dV, var_a, phi2,
                                 I.part_r, totals, st);
    h->launches = 2;
    CU(cudaGetLastError());
    return TWA_OK;
}

int twa_advance_adaptive(twa_handle* h, void* psi_work, int n_out, int out_every, double c_f, double* series,
                         double* times, void* stream) {
    if (!h) return fail(nullptr, TWA_EINVAL, "null handle");
    if (!psi_work || !series || !times || n_out < 0 || out_every <= 0 || !(c_f > 0.0))
        return fail(h, TWA_EINVAL, "twa_advance_adaptive: bad argument (need n_out >= 0, out_every > 0, c_f > 0)");
    if (h->p.precision != TWA_F32) return fail(h, TWA_EINVAL, "twa_advance_adaptive: FP32 path only");
    if (misaligned(psi_work)) return fail(h, TWA_EINVAL, "twa_advance_adaptive: psi must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    const double dt0 = h->p.dt;
    long long total = 0;
    h->launches = 0;
    CU(cudaMemsetAsync(h->d_counter, 0, sizeof(int), st));
    for (size_t i = 0; i < h->in.size(); ++i) {
        Inst& I = h->in[i];
        float2* f = inst_psi(I, psi_work);
        RC(poisson_init(h, I, f, st));
        RC(moments_f32(h, I, f, 0.0, nullptr, h->d_cur + i * TWA_NSCALARS, st));
    }
    launch_store_series(h->d_cur, series, h->d_counter, (int)h->in.size() * TWA_NSCALARS, st);
    ++h->launches;
    times[0] = 0.0;
    double t = 0.0, dt_prev = 0.0;
    int rc = 0;
    for (int o = 1; o <= n_out && rc == 0; ++o) {
        double dt = 0.0;
        if ((rc = adaptive_dt(h, psi_work, c_f, st, &dt))) break;
        if (!(dt > 0.0) || !std::isfinite(dt)) {
            rc = fail(h, TWA_ENONFINITE, "twa_advance_adaptive: no finite time step (non-finite potential)");
            break;
        }
        if ((rc = set_dt(h, dt, st))) break;
        // the pending closing half kick of the previous interval (dt_prev / 2) merges with this
        // interval's opening half kick (dt / 2)
        const double a_first = (o == 1) ? 0.5 : 0.5 + 0.5 * dt_prev / dt;
        total += h->launches;
        h->launches = 0;
        if ((rc = run_interval_f32(h, psi_work, out_every, a_first, series, st))) break;
        t += out_every * dt;
        times[o] = t;
        dt_prev = dt;
    }
    if (rc == 0 && n_out >= 1)
        for (auto& I : h->in)
            if ((rc = closing_kick(h, I, inst_psi(I, psi_work), 0.5, st))) break;
    total += h->launches;
    const int rc2 = set_dt(h, dt0, st);
    h->launches = total;
    if (rc) return rc;
    if (rc2) return rc2;
    CU(cudaGetLastError());
    return TWA_OK;
}

int twa_run(twa_handle* h, const void* psi_cl, uint64_t seed, int n_steps, int out_every, void* psi_work,
            double* series, void* stream) {
    if (!h) return fail(nullptr, TWA_EINVAL, "null handle");
    if (!psi_cl || !psi_work || !series || out_every <= 0 || n_steps < 0 || n_steps % out_every)
        return fail(h, TWA_EINVAL, "twa_run: bad argument (n_steps must be a multiple of out_every)");
    RC(twa_sample(h, psi_cl, seed, psi_work, stream));
    const long long ns = h->launches;
    RC(twa_advance(h, psi_work, n_steps, out_every, series, stream));
    h->launches += ns;
    return TWA_OK;
}

int twa_sync_status(twa_handle* h, void* stream) {
    if (!h) return fail(nullptr, TWA_EINVAL, "null handle");
    CU(cudaStreamSynchronize((cudaStream_t)stream));
    int w = 0;
    CU(cudaMemcpy(&w, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    CU(cudaMemset(h->d_err, 0, sizeof(int)));
    if (w & TWA_ERR_TIMEOUT_BIT)
        return fail(h, TWA_ETIMEOUT, "a device-side wait (persistent batch launch or TMA tile copy) gave up (wait limit " +
                                         std::to_string(h->wait_limit_s) + " s); the batch's fields are undefined");
    if (w & 1) return fail(h, TWA_ENONFINITE, "a moments pass met a non-finite field value");
    return TWA_OK;
}

const char* twa_last_error(const twa_handle* h) { return h ? h->err.c_str() : g_create_error.c_str(); }

int twa_set_batch_mode(twa_handle* h, int mode) {
    if (!h) return fail(nullptr, TWA_EINVAL, "null handle");
    if (mode < TWA_BATCH_SERIAL || mode > TWA_BATCH_PERSISTENT) return fail(h, TWA_EINVAL, "twa_set_batch_mode: bad mode");
    if (mode == TWA_BATCH_PERSISTENT && !batch_eligible(h))
        return fail(h, TWA_EINVAL,
                    "twa_set_batch_mode: the persistent launch needs FP32 2D instances with axes of 256 to 2048 cells "
                    "and no test particles");
    h->fork = mode == TWA_BATCH_FORK;
    h->persist = mode == TWA_BATCH_PERSISTENT;
    if (h->gexec) {
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
    }
    return TWA_OK;
}

int twa_get_batch_mode(const twa_handle* h) {
    if (!h) return TWA_EINVAL;
    return h->persist ? TWA_BATCH_PERSISTENT : (h->fork ? TWA_BATCH_FORK : TWA_BATCH_SERIAL);
}

int twa_set_wait_limit(twa_handle* h, double seconds) {
    if (!h) return fail(nullptr, TWA_EINVAL, "null handle");
    if (!(seconds > 0.0) || seconds > 60.0) return fail(h, TWA_EINVAL, "twa_set_wait_limit: need 0 < seconds <= 60");
    h->wait_limit_s = seconds;
    if (h->gexec) {  // captured launches carry the old limit
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
    }
    return TWA_OK;
}

int twa_debug_stall_next_tma(twa_handle* h) {
    if (!h) return fail(nullptr, TWA_EINVAL, "null handle");
    if (h->p.precision != TWA_F32) return fail(h, TWA_EINVAL, "twa_debug_stall_next_tma: FP32 handles only");
    h->stall_tma = true;
    return TWA_OK;
}

int twa_debug_stall_next_batch(twa_handle* h) {
    if (!h) return fail(nullptr, TWA_EINVAL, "null handle");
    if (!batch_eligible(h)) return fail(h, TWA_EINVAL, "twa_debug_stall_next_batch: the handle has no persistent launch");
    h->stall_next = true;
    return TWA_OK;
}

}  // extern "C"

// Record a failure of a handle-free entry point, reported by twa_last_error(NULL).
void twa_set_global_error(const std::string& msg) { g_create_error = msg; }

// ---------------------------------------------------------------------------------------------
// Stream averages of user functions (Appendix B's synthesizer), compiled at run time.
struct twa_observable {
    twa::ObsProgram* prog = nullptr;
    int flags = 0;
    double* part = nullptr;  // per-block partial sums, allocated on the first evaluation
};

namespace {
constexpr int kObsBlocks = 152 * 8;
}

extern "C" {

int twa_observable_create(twa_observable** out, const char* f_re, const char* f_im, int flags) {
    if (!out || !f_re || (flags & ~(TWA_OBS_OF_MEAN | TWA_OBS_MODES | TWA_OBS_FP32)))
        return fail(nullptr, TWA_EINVAL, "twa_observable_create: bad argument");
    *out = nullptr;
    std::string msg;
    twa::ObsProgram* prog = nullptr;
    const int rc = twa::obs_compile(f_re, f_im, (flags & TWA_OBS_FP32) != 0, &prog, &msg);
    if (rc) return fail(nullptr, rc == -1 ? TWA_EINVAL : TWA_ECUDA, msg);
    twa_observable* ob = new twa_observable();
    ob->prog = prog;
    ob->flags = flags;
    *out = ob;
    return TWA_OK;
}

int twa_observable_destroy(twa_observable* ob) {
    if (!ob) return TWA_OK;
    if (ob->part) cudaFree(ob->part);
    twa::obs_free(ob->prog);
    delete ob;
    return TWA_OK;
}

int twa_observable_eval(twa_observable* ob, twa_handle* h, int inst, const void* psi, double* per_cell, double* f_cl,
                        double* total, void* stream) {
    if (!h) return fail(nullptr, TWA_EINVAL, "null handle");
    if (!ob || !psi || !total || inst < 0 || inst >= (int)h->in.size())
        return fail(h, TWA_EINVAL, "twa_observable_eval: bad argument");
    if (misaligned(psi)) return fail(h, TWA_EINVAL, "twa_observable_eval: psi must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    h->launches = 0;
    Inst& I = h->in[inst];
    if (!ob->part) CU(cudaMalloc(&ob->part, sizeof(double) * 2 * kObsBlocks));
    const void* src = nullptr;
    double scale = 1.0, w = I.dV;
    bool f64 = false;
    if (ob->flags & TWA_OBS_MODES) {
        if (h->p.precision != TWA_F32 || !I.spec)
            return fail(h, TWA_EINVAL, "twa_observable_eval: Fourier amplitudes need the FP32 path and want_modes");
        // a_k = sqrt(n_tot dV / cells) DFT(psi)_k for every slot, as the moments form them
        float2* f = inst_psi(I, const_cast<void*>(psi));
        RC(run_pass(h, I, f, 0, OP_KICK_FWD_OUT, 0.0, I.vc, I.spec, I.n_pairs, st, 0, I.mode == MODE_1D ? 1 : 0));
        for (int ax = 1; ax < I.dim; ++ax) RC(run_pass(h, I, f, ax, OP_FWD, 0.0, I.spec, nullptr, I.n_slots, st));
        h->launches += I.dim;
        src = I.spec;
        scale = std::sqrt(h->p.n_tot * I.dV / (double)I.cells);
        w = 1.0;
    } else if (h->p.precision == TWA_F32) {
        src = inst_psi(I, const_cast<void*>(psi));
    } else {
        src = static_cast<const double2*>(psi) + I.off;
        f64 = true;
    }
    std::string msg;
    if (twa::obs_launch(ob->prog, f64, src, I.cells, I.n_slots, (ob->flags & TWA_OBS_OF_MEAN) ? 1 : 0, scale, I.n,
                        per_cell, f_cl, ob->part, kObsBlocks, w, total, st, &msg))
        return fail(h, TWA_ECUDA, msg);
    h->launches += 2;
    return TWA_OK;
}

}  // extern "C"

extern "C" {

int twa_profile_enable(twa_handle* h, int on) {
    if (!h) return fail(nullptr, TWA_EINVAL, "null handle");
    CU(cudaDeviceSynchronize());
    for (auto& r : h->prof_pending) {
        h->prof_pool.push_back(r.a);
        h->prof_pool.push_back(r.b);
    }
    h->prof_pending.clear();
    for (int i = 0; i < PROF_NOPS; ++i) {
        h->prof_launches[i] = 0;
        h->prof_ms[i] = 0.0;
    }
    h->prof_on = on != 0;
    return TWA_OK;
}

int twa_profile_read(twa_handle* h, int op, long long* launches, double* total_ms, double* bytes_per_cell,
                     long long* fields_per_launch, long long* cells) {
    if (!h) return fail(nullptr, TWA_EINVAL, "null handle");
    if (op < 0 || op >= PROF_NOPS) return fail(h, TWA_EINVAL, "twa_profile_read: bad op");
    for (auto& r : h->prof_pending) {
        CU(cudaEventSynchronize(r.b));
        float ms = 0.f;
        CU(cudaEventElapsedTime(&ms, r.a, r.b));
        h->prof_launches[r.op] += 1;
        h->prof_ms[r.op] += ms;
        h->prof_fields[r.op] = r.fields;
        h->prof_cells[r.op] = r.cells;
        h->prof_pool.push_back(r.a);
        h->prof_pool.push_back(r.b);
    }
    h->prof_pending.clear();
    // Algorithmic DRAM bytes per cell of one launched field (a pair of slots or one slot):
    // every complex value read or written once (8 bytes), the Poisson field once per pair.
    static const double bpc[OP_COUNT + PL_COUNT] = {
        16.0,  // OP_DRIFT: psi read + write
        40.0,  // OP_KICK_DRIFT: W read, 2 x (psi read + write)
        40.0,  // OP_KICK_DRIFT_VINV
        40.0,  // OP_DRIFT_RHO: 2 x (psi read + write), W write
        24.0,  // OP_RHO_FWD: 2 x psi read, W write
        16.0,  // OP_FWD
        16.0,  // OP_FWD_MUL_INV
        16.0,  // OP_INV
        40.0,  // OP_KICK_VINV: W read, 2 x (psi read + write)
        40.0,  // OP_KICK_FWD_OUT: W read, 2 x (psi read + spectrum write)
        48.0,  // OP_STEPS_1D: per pair and step if the fields streamed (they stay on chip)
        16.0,  // OP_MUL_INV
        40.0,  // PL_KICK_DRIFT: W read once from DRAM, 2 x (psi read + write); row/column re-reads hit L2
        16.0,  // PL_POISSON: W read + write
    };
    if (launches) *launches = h->prof_launches[op];
    if (total_ms) *total_ms = h->prof_ms[op];
    if (bytes_per_cell) *bytes_per_cell = bpc[op];
    if (fields_per_launch) *fields_per_launch = h->prof_fields[op];
    if (cells) *cells = h->prof_cells[op];
    return TWA_OK;
}

long long twa_last_launch_count(const twa_handle* h) { return h ? h->launches : 0; }

int twa_poisson_multiplier(const float* k2, float* m, long long n, void* stream) {
    twa_handle* h = nullptr;
    if (!k2 || !m || n < 0) return fail(h, TWA_EINVAL, "twa_poisson_multiplier: bad argument");
    launch_poisson_multiplier(k2, m, n, (cudaStream_t)stream);
    CU(cudaGetLastError());
    return TWA_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Autotuner: for every pass of the FP32 pipelines, time each instantiated lines-per-CTA variant on
// the handle's own buffers and keep the fastest.  Results are cached in a flat JSON object keyed by
// "N,axis,op,dims" so later handles with the same shapes skip the timing.
namespace {

std::string tune_key(const Inst& I, int axis, int op) {
    std::ostringstream s;
    s << I.n[0] << "x" << I.n[1] << "x" << I.n[2] << ":slots" << I.n_slots << ":axis" << axis << ":op" << op;
    return s.str();
}

std::map<std::string, int> read_cache(const char* path) {
    std::map<std::string, int> m;
    if (!path) return m;
    std::ifstream f(path);
    if (!f) return m;
    std::string txt((std::istreambuf_iterator<char>(f)), std::istreambuf_iterator<char>());
    size_t i = 0;
    while ((i = txt.find('"', i)) != std::string::npos) {
        const size_t j = txt.find('"', i + 1);
        if (j == std::string::npos) break;
        const std::string k = txt.substr(i + 1, j - i - 1);
        const size_t c = txt.find(':', j);
        if (c == std::string::npos) break;
        m[k] = std::atoi(txt.c_str() + c + 1);
        i = txt.find_first_of(",}", c);
        if (i == std::string::npos) break;
    }
    return m;
}

void write_cache(const char* path, const std::map<std::string, int>& m) {
    if (!path) return;
    std::ofstream f(path);
    f << "{\n";
    size_t n = 0;
    for (const auto& kv : m) f << "  \"" << kv.first << "\": " << kv.second << (++n < m.size() ? ",\n" : "\n");
    f << "}\n";
}

}  // namespace

namespace {

struct TunePass {
    int axis, op, fields;  // axis 3 = xy-plane pass (op = plane op)
    float2* buf;
    float2* out;
};

int time_variant(twa_handle* h, Inst& I, float2* f, const TunePass& ps, int l, cudaStream_t st, cudaEvent_t e0,
                 cudaEvent_t e1, float* ms) {
    const int ns = (ps.op == OP_STEPS_1D && ps.axis == 0) ? 4 : 0;
    auto once = [&]() -> int {
        if (ps.axis == 3) return run_plane(h, I, f, ps.op, 0.0, st, l);
        return run_pass(h, I, f, ps.axis, ps.op, 0.0, ps.buf, ps.out, ps.fields, st, ns, l);
    };
    RC(once());
    CU(cudaEventRecord(e0, st));
    for (int r = 0; r < 3; ++r) RC(once());
    CU(cudaEventRecord(e1, st));
    CU(cudaEventSynchronize(e1));
    CU(cudaEventElapsedTime(ms, e0, e1));
    return 0;
}

int tune_passes(twa_handle* h, Inst& I, float2* f, const std::vector<TunePass>& passes, std::map<std::string, int>& cache,
                cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1) {
    const int cand[] = {1, 2, 4, 8, 16, 32, 64, 128, 256, 512, PIPE_FLAG | 1, PIPE_FLAG | 2, PIPE_FLAG | 4,
                        PIPE_FLAG | 8, PIPE_FLAG | 16, PIPE_FLAG | 32, PIPE_FLAG | 64, DUAL_FLAG | 4, DUAL_FLAG | 8,
                        DUAL_FLAG | 16, DUAL_FLAG | 32, DUAL_FLAG | 64, DUAL_FLAG | 128, DUAL_FLAG | 256,
                        PIPE_FLAG | TMA_FLAG | 1, PIPE_FLAG | TMA_FLAG | 2, PIPE_FLAG | TMA_FLAG | 4,
                        PIPE_FLAG | TMA_FLAG | 8, PIPE_FLAG | TMA_FLAG | 16, PIPE_FLAG | TMA_FLAG | 32,
                        PIPE_FLAG | TMA_FLAG | 64};
    for (const auto& ps : passes) {
        const int N = I.n[ps.axis == 3 ? 0 : ps.axis];
        auto ok = [&](int l) {
            if (ps.axis == 3) return (l & PIPE_FLAG) == 0 && plane_variant_ok(N, ps.op, l);
            if (!variant_ok(N, ps.op, ps.axis > 0, l)) return false;
            const int ll = l & ~(PIPE_FLAG | DUAL_FLAG | TMA_FLAG);
            if (l & PIPE_FLAG) {
                long long stride = 1;
                for (int b = 0; b < ps.axis; ++b) stride *= I.n[b];
                if ((I.cells / N) % ll != 0 || (ps.axis > 0 && stride % ll != 0)) return false;
            }
            return !(ps.op != OP_STEPS_1D && ps.axis == 0 && ll > I.cells / I.n[0]);
        };
        const std::string key = tune_key(I, ps.axis, ps.op);
        auto hit = cache.find(key);
        if (hit != cache.end() && ok(hit->second)) {
            I.lines[key_of(ps.axis, ps.op)] = hit->second;
            continue;
        }
        float best = 1e30f;
        int best_l = 0;
        for (int l : cand) {
            if (!ok(l)) continue;
            float ms = 0.f;
            RC(time_variant(h, I, f, ps, l, st, e0, e1, &ms));
            if (ms < best) {
                best = ms;
                best_l = l;
            }
        }
        if (best_l) {
            I.lines[key_of(ps.axis, ps.op)] = best_l;
            cache[key] = best_l;
        }
    }
    return 0;
}

}  // namespace

extern "C" int twa_autotune(twa_handle* h, void* psi, const char* cache_path, void* stream) {
    if (!h) return fail(nullptr, TWA_EINVAL, "null handle");
    if (!psi) return fail(h, TWA_EINVAL, "twa_autotune: null buffer");
    if (misaligned(psi)) return fail(h, TWA_EINVAL, "twa_autotune: psi must be 16-byte aligned");
    if (h->p.precision != TWA_F32) return TWA_OK;
    cudaStream_t st = (cudaStream_t)stream;
    std::map<std::string, int> cache = read_cache(cache_path);
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    for (auto& I : h->in) {
        float2* f = inst_psi(I, psi);
        // Each candidate is timed on a prefix of the pass's fields holding at least 8 GB (far above
        // the L2), so the tuner's cost stays bounded on the largest batches (512^3 x 64 streams is
        // 70 GB); every batch of up to 8 GB per pass is timed whole.
        const long long unit = (long long)I.cells * (long long)sizeof(float2);
        const long long cap = (8LL << 30) / unit + 1;
        const int Pn = (int)std::min<long long>(I.n_pairs, cap), Sn = (int)std::min<long long>(I.n_slots, cap);
        std::vector<TunePass> passes;
        if (I.mode == MODE_1D) {
            passes = {{0, OP_STEPS_1D, Pn, I.vc, nullptr}};
        } else if (I.mode == MODE_2D) {
            passes = {{0, OP_KICK_DRIFT, Pn, I.vc, nullptr}, {1, OP_DRIFT_RHO, Pn, I.vc, nullptr},
                      {0, OP_FWD_MUL_INV, Pn, I.vc, nullptr}, {1, OP_INV, Pn, I.vc, nullptr},
                      {1, OP_RHO_FWD, Pn, I.vc, nullptr}};
        } else {
            // both 3D pipelines: the axis passes and, for square xy planes, the fused plane passes
            passes = {{0, OP_KICK_DRIFT_VINV, Pn, I.vc, nullptr}, {1, OP_DRIFT, Sn, I.vc, nullptr},
                      {2, OP_DRIFT_RHO, Pn, I.vc, nullptr}, {0, OP_FWD, Pn, I.vc, nullptr},
                      {1, OP_FWD_MUL_INV, Pn, I.vc, nullptr}, {2, OP_INV, Pn, I.vc, nullptr},
                      {2, OP_RHO_FWD, Pn, I.vc, nullptr}, {0, OP_INV, Pn, I.vc, nullptr},
                      {0, OP_KICK_VINV, Pn, I.vc, nullptr}};
            if (I.mode == MODE_3DP || I.mode == MODE_3DH) {
                passes.push_back({3, PL_KICK_DRIFT, Pn, I.vc, nullptr});
                passes.push_back({3, PL_POISSON, Pn, I.vc, nullptr});
                passes.push_back({0, OP_KICK_DRIFT, Pn, I.vc, nullptr});
            }
        }
        if (I.spec) {
            passes.push_back({0, OP_KICK_FWD_OUT, Pn, I.vc, I.spec});
            for (int ax = 1; ax < I.dim; ++ax) passes.push_back({ax, OP_FWD, Sn, I.spec, nullptr});
        }
        RC(tune_passes(h, I, f, passes, cache, st, e0, e1));
        if (I.mode == MODE_3DP || I.mode == MODE_3D || I.mode == MODE_3DH) {
            // pick the fastest 3D pipeline by timing two whole steps of each (cache value 0 axis,
            // 1 plane, 2 axis passes for the fields with the plane Poisson pass)
            const std::string key = tune_key(I, 9, 0);
            auto hit = cache.find(key);
            const bool eligible = I.n[0] == I.n[1] && I.n[0] >= 16 && I.n[0] <= 256;
            const int modes[3] = {MODE_3D, MODE_3DP, MODE_3DH};
            if (!eligible) {
                I.mode = MODE_3D;
            } else if (hit != cache.end() && hit->second >= 0 && hit->second <= 2) {
                I.mode = modes[hit->second];
            } else {
                float t[3] = {0.f, 0.f, 0.f};
                for (int m = 0; m < 3; ++m) {
                    I.mode = modes[m];
                    RC(steps_f32(h, I, f, 1, 1.0, st));
                    CU(cudaEventRecord(e0, st));
                    RC(steps_f32(h, I, f, 2, 1.0, st));
                    CU(cudaEventRecord(e1, st));
                    CU(cudaEventSynchronize(e1));
                    CU(cudaEventElapsedTime(&t[m], e0, e1));
                }
                // a pipeline other than the axis one is taken only when it is clearly faster (3 %),
                // so near-ties do not flip between runs
                int best = 0;
                for (int m = 1; m < 3; ++m)
                    if (t[m] < 0.97f * t[0] && t[m] < (best ? t[best] : t[0])) best = m;
                I.mode = modes[best];
                cache[key] = best;
            }
        }
        CU(cudaMemsetAsync(I.vc, 0, (size_t)I.n_pairs * I.cells * sizeof(float2), st));
    }
    const bool can_persist = batch_eligible(h);
    if (h->in.size() > 1 || can_persist) {
        // how the instances run: one after another (0), on parallel streams (1, several instances),
        // or as one persistent launch over a work list (2, 2D batches); two steps of each are timed
        std::string key = "batch";
        for (const auto& I : h->in)
            key += ":" + std::to_string(I.n[0]) + "x" + std::to_string(I.n[1]) + "x" + std::to_string(I.n[2]) +
                   "s" + std::to_string(I.n_slots);
        auto hit = cache.find(key);
        if (hit != cache.end() && (hit->second != 2 || can_persist) && (hit->second != 1 || h->in.size() > 1)) {
            h->fork = hit->second == 1;
            h->persist = hit->second == 2;
        } else {
            float t[3] = {0.f, 1e30f, 1e30f};
            auto steps_all = [&](int n) -> int {
                if (h->persist) return batch_steps(h, psi, n, 1.0, st);
                Fork fk{h, st, false};
                RC(fk.open(h->in.size()));
                for (size_t i = 0; i < h->in.size(); ++i) {
                    cudaStream_t s;
                    RC(fk.stream(i, &s));
                    RC(steps_f32(h, h->in[i], inst_psi(h->in[i], psi), n, 1.0, s));
                    RC(fk.join(i));
                }
                return 0;
            };
            for (int m = 0; m < 3; ++m) {
                if ((m == 1 && h->in.size() < 2) || (m == 2 && !can_persist)) continue;
                h->fork = (m == 1);
                h->persist = (m == 2);
                RC(steps_all(1));
                CU(cudaEventRecord(e0, st));
                RC(steps_all(2));
                CU(cudaEventRecord(e1, st));
                CU(cudaEventSynchronize(e1));
                CU(cudaEventElapsedTime(&t[m], e0, e1));
            }
            // a mode other than one-after-another is kept only when it is clearly faster (3 %)
            int best = 0;
            for (int m = 1; m < 3; ++m)
                if (t[m] < 0.97f * t[best]) best = m;
            h->fork = best == 1;
            h->persist = best == 2;
            cache[key] = best;
        }
        for (auto& I : h->in) CU(cudaMemsetAsync(I.vc, 0, (size_t)I.n_pairs * I.cells * sizeof(float2), st));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (h->gexec) {
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
    }
    write_cache(cache_path, cache);
    CU(cudaStreamSynchronize(st));
    return TWA_OK;
}
