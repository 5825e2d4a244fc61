// fft_engine.cuh - register-resident Stockham FFT of one line, exchanged through shared memory.
//
// The split-step of Sec. III.B.2 needs, per step and per field, forward and inverse FFTs along
// every axis (kinetic factor) and the FFTs of the Poisson solve.  Each line of length N is held by
// T = N / RMAX threads with RMAX complex values each in registers.  A transform is a sequence of
// Stockham autosort stages (radix R_s, sub-transform length Ns = prod of earlier radices): every
// butterfly j takes x[j + r N/R], multiplies by W_{Ns R}^{r (j mod Ns)}, does an in-register
// radix-R DFT and lands at (j / Ns) Ns R + (j mod Ns) + r Ns.  Between stages the values are
// exchanged through a padded shared-memory line (one extra float2 per 16 to avoid bank
// conflicts).  The forward transform ends in the layout the inverse starts from, so a pointwise
// operation in Fourier space between them (kinetic phase, Poisson multiplier) needs no data
// movement.  All transforms are unnormalized; scale factors live in the pointwise tables.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace twa {

// Packed two-lane FP32 arithmetic (PTX .f32x2, sm_100 and later): one instruction applies the same
// operation to both components of a float2.  The transforms are bound by instruction issue, and
// the additions of a butterfly and most of its constant products pair up this way.
__device__ __forceinline__ float2 f2_add(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 f2_mul(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
// a * b + c lane by lane, each lane rounded once
__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mov.b64 rc, {%6, %7};\n\tfma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return f2_add(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return f2_sub(a, b); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
// a * (hi + lo) for a constant carried as a float pair hi + lo (lo = remainder of the exact value):
// the small product a * lo enters the innermost fma, so the result carries the constant to about
// twice float precision and every product is rounded once inside an fma.  Without this, the
// rounding of the twiddle constants biases every transform the same way and the error of the
// split step grows linearly in the number of steps.
__device__ __forceinline__ float2 cmul_c(float2 a, float2 hi, float2 lo) {
    const float lx = fmaf(a.x, lo.x, -a.y * lo.y);
    const float ly = fmaf(a.x, lo.y, a.y * lo.x);
    return make_float2(fmaf(a.x, hi.x, fmaf(-a.y, hi.y, lx)), fmaf(a.x, hi.y, fmaf(a.y, hi.x, ly)));
}

// cos and sin of 2 pi j / 32 (mathematical constants rounded to float).
constexpr float kCos32[32] = {
    1.f, 0.98078528040323043f, 0.92387953251128674f, 0.83146961230254524f, 0.70710678118654757f,
    0.55557023301960229f, 0.38268343236508984f, 0.19509032201612833f, 0.f, -0.19509032201612819f,
    -0.38268343236508973f, -0.55557023301960196f, -0.70710678118654746f, -0.83146961230254535f,
    -0.92387953251128674f, -0.98078528040323043f, -1.f, -0.98078528040323043f, -0.92387953251128685f,
    -0.83146961230254546f, -0.70710678118654768f, -0.55557023301960218f, -0.38268343236509034f,
    -0.19509032201612866f, 0.f, 0.1950903220161283f, 0.38268343236509f, 0.55557023301960184f,
    0.70710678118654735f, 0.83146961230254524f, 0.92387953251128652f, 0.98078528040323032f};
constexpr float kSin32[32] = {
    0.f, 0.19509032201612825f, 0.38268343236508978f, 0.55557023301960218f, 0.70710678118654746f,
    0.83146961230254524f, 0.92387953251128674f, 0.98078528040323043f, 1.f, 0.98078528040323043f,
    0.92387953251128674f, 0.83146961230254546f, 0.70710678118654757f, 0.55557023301960218f,
    0.38268343236508989f, 0.19509032201612861f, 0.f, -0.19509032201612836f, -0.38268343236508967f,
    -0.55557023301960196f, -0.70710678118654746f, -0.83146961230254524f, -0.92387953251128652f,
    -0.98078528040323032f, -1.f, -0.98078528040323043f, -0.92387953251128663f, -0.83146961230254546f,
    -0.70710678118654768f, -0.55557023301960218f, -0.38268343236509039f, -0.19509032201612872f};

// cos(2 pi j / 32) - kCos32[j] and sin(2 pi j / 32) - kSin32[j], rounded to float.
constexpr float kCos32Lo[32] = {0.000000000e+00f, 2.973947311e-08f, 2.830749035e-08f, 1.687026374e-08f, 1.210161715e-08f, -1.176952125e-08f, 6.223350946e-09f, -1.670471400e-09f, 0.000000000e+00f, 1.670471539e-09f, -6.223350835e-09f, 1.176952158e-08f, -1.210161704e-08f, -1.687026385e-08f, -2.830749035e-08f, -2.973947311e-08f, 0.000000000e+00f, -2.973947311e-08f, -2.830749046e-08f, -1.687026396e-08f, -1.210161726e-08f, 1.176952136e-08f, -6.223351445e-09f, 1.670471067e-09f, 0.000000000e+00f, -1.670471428e-09f, 6.223351112e-09f, -1.176952169e-08f, 1.210161693e-08f, 1.687026374e-08f, 2.830749013e-08f, 2.973947300e-08f};
constexpr float kSin32Lo[32] = {0.000000000e+00f, -1.670471483e-09f, 6.223350890e-09f, -1.176952136e-08f, 1.210161704e-08f, 1.687026374e-08f, 2.830749035e-08f, 2.973947311e-08f, 0.000000000e+00f, 2.973947311e-08f, 2.830749035e-08f, 1.687026396e-08f, 1.210161715e-08f, -1.176952136e-08f, 6.223351001e-09f, -1.670471123e-09f, 0.000000000e+00f, 1.670471372e-09f, -6.223350779e-09f, 1.176952158e-08f, -1.210161704e-08f, -1.687026374e-08f, -2.830749013e-08f, -2.973947300e-08f, 0.000000000e+00f, -2.973947311e-08f, -2.830749024e-08f, -1.687026396e-08f, -1.210161726e-08f, 1.176952136e-08f, -6.223351501e-09f, 1.670471012e-09f};

// a * (c + i s) for a compile-time constant carried as hi (c, s) + lo (cl, sl), in packed form:
// a (c, c) + (a.y, a.x) (-s, s), with the lo part entering the innermost products as in cmul_c.
__device__ __forceinline__ float2 cmul_k(float2 a, float c, float s, float cl, float sl) {
    const float2 as = make_float2(a.y, a.x);
    const float2 l = f2_fma(as, make_float2(-sl, sl), f2_mul(a, make_float2(cl, cl)));
    return f2_fma(a, make_float2(c, c), f2_fma(as, make_float2(-s, s), l));
}
// a * (sx + i sy) c for signs sx, sy = +-1 and c = cos(pi / 4) carried as ch + cl: the rotation is
// u = a + (sy / sx) i a (exact up to one rounding of the sum), then u * sx c.
__device__ __forceinline__ float2 cmul_45(float2 a, float sx, float sy, float ch, float cl) {
    const float sg = sy * sx;
    const float2 u = f2_fma(make_float2(a.y, a.x), make_float2(-sg, sg), a);
    return f2_fma(u, make_float2(sx * ch, sx * ch), f2_mul(u, make_float2(sx * cl, sx * cl)));
}

// a * W_R^K with W_R = exp(-2 pi i / R) (forward) or exp(+2 pi i / R) (inverse); R | 32.
template <int K, int R, bool INV>
__device__ __forceinline__ float2 twc(float2 a) {
    constexpr int J = (K * (32 / R)) % 32;
    if constexpr (J == 0) {
        return a;
    } else if constexpr (J == 8) {  // -i forward, +i inverse
        return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
    } else if constexpr (J == 16) {
        return make_float2(-a.x, -a.y);
    } else if constexpr (J == 24) {
        return INV ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
    } else if constexpr (J % 8 == 4) {
        constexpr float sx = kCos32[J] > 0.f ? 1.f : -1.f;
        constexpr float sy = ((INV ? kSin32[J] : -kSin32[J]) > 0.f) ? 1.f : -1.f;
        constexpr float ch = kCos32[4], cl = kCos32Lo[4];
        return cmul_45(a, sx, sy, ch, cl);
    } else {
        constexpr float c = kCos32[J], cl = kCos32Lo[J];
        constexpr float s = INV ? kSin32[J] : -kSin32[J];
        constexpr float sl = INV ? kSin32Lo[J] : -kSin32Lo[J];
        return cmul_k(a, c, s, cl, sl);
    }
}

template <int R, bool INV, int K = 0>
struct Combine {
    __device__ __forceinline__ static void run(float2* v, const float2* e, const float2* o) {
        if constexpr (K < R / 2) {
            constexpr int J = (K * (32 / R)) % 32;
            if constexpr (J == 8 || J == 24) {
                // a rotation by +-i is a swap and a sign: fold it into scalar additions
                const float2 t = twc<K, R, INV>(o[K]);
                v[K] = make_float2(e[K].x + t.x, e[K].y + t.y);
                v[K + R / 2] = make_float2(e[K].x - t.x, e[K].y - t.y);
            } else if constexpr (J == 16) {
                v[K] = csub(e[K], o[K]);
                v[K + R / 2] = cadd(e[K], o[K]);
            } else {
                const float2 t = twc<K, R, INV>(o[K]);
                v[K] = cadd(e[K], t);
                v[K + R / 2] = csub(e[K], t);
            }
            Combine<R, INV, K + 1>::run(v, e, o);
        }
    }
};

// In-register radix-R DFT (R = 2..32), natural order in and out, by even/odd splitting.
template <int R, bool INV>
__device__ __forceinline__ void dft(float2* v) {
    if constexpr (R == 2) {
        const float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if constexpr (R > 2) {
        float2 e[R / 2], o[R / 2];
#pragma unroll
        for (int i = 0; i < R / 2; ++i) {
            e[i] = v[2 * i];
            o[i] = v[2 * i + 1];
        }
        dft<R / 2, INV>(e);
        dft<R / 2, INV>(o);
        Combine<R, INV>::run(v, e, o);
    }
}

// Stage plans: radices in forward order, RMAX values per thread, T = N / RMAX threads per line.
template <int N> struct Plan;
#define TWA_PLAN(N_, RMAX_, S_, ...)                                   \
    template <> struct Plan<N_> {                                      \
        static constexpr int RMAX = RMAX_, S = S_, T = N_ / RMAX_;     \
        static constexpr int R[S_] = {__VA_ARGS__};                    \
    };
TWA_PLAN(8, 8, 1, 8)
TWA_PLAN(16, 16, 1, 16)
TWA_PLAN(32, 16, 2, 16, 2)
TWA_PLAN(64, 8, 2, 8, 8)
TWA_PLAN(128, 16, 2, 16, 8)
TWA_PLAN(256, 16, 2, 16, 16)
TWA_PLAN(512, 16, 3, 16, 8, 4)
TWA_PLAN(1024, 16, 3, 16, 16, 4)
TWA_PLAN(2048, 16, 3, 16, 16, 8)
#undef TWA_PLAN

// Shared-memory slot of element i of a line of length n: one padding slot per 16 elements, and for
// n = 64 and 128 (T = 8 threads per line, four lines per warp in row passes) one per 8 plus one per
// 64, which makes the exchanges of both stage orders (forward 16|8, inverse 8|16) conflict-free.
__host__ __device__ constexpr int pad_n(int n, int i) {
    return (n == 64 || n == 128) ? i + (i >> 3) + (i >> 6) : i + (i >> 4);
}
// Shared-memory line stride.  Column passes (lanes = lines): with 16 or more lines per CTA, odd,
// so the 16 lanes of a 64-bit access phase fall in distinct banks; with fewer lines (long lines,
// few per CTA), congruent to 16 / lines modulo 16, so the lines of an access phase start in
// disjoint windows of banks.  Row passes (lanes = positions, T < 16 threads per line): the lines
// sharing an access phase start 2 T banks apart, so each uses its own window of banks.
__host__ __device__ constexpr int line_stride(int n, int lines = 16) {
    return lines >= 16 ? ((pad_n(n, n) & 1) ? pad_n(n, n) : pad_n(n, n) + 1)
                       : pad_n(n, n) + ((16 / lines - pad_n(n, n) % 16) % 16 + 16) % 16;
}
__host__ __device__ constexpr int line_stride_rows(int n, int t) {
    return (t >= 16) ? pad_n(n, n) : pad_n(n, n) + ((t - pad_n(n, n) % 16) % 16 + 16) % 16;
}

template <int N, bool INV, int s>
struct StageInfo {
    using P = Plan<N>;
    static constexpr int R = INV ? P::R[P::S - 1 - s] : P::R[s];
    static constexpr int NS = StageInfo<N, INV, s - 1>::NS * StageInfo<N, INV, s - 1>::R;
};
template <int N, bool INV>
struct StageInfo<N, INV, 0> {
    using P = Plan<N>;
    static constexpr int R = INV ? P::R[P::S - 1] : P::R[0];
    static constexpr int NS = 1;
};

// Twiddle table of length-N transforms, stage-major: for the forward and then the inverse stage
// order, every stage s >= 1 (radix R, sub-transform length NS) holds (R - 1) x NS entries
// W_N^(r k N / (NS R)), r = 1..R-1 (rows), k = 0..NS-1 (consecutive), as float4 (hi.re, hi.im,
// lo.re, lo.im).  Consecutive threads of a stage read consecutive entries.  tw_exponent gives the
// power of W_N = exp(-2 pi i / N) stored at an index (-1 past the end).
// radix s of the forward stage order (1 past the last stage); a constant expression, so device code
// may use it at run time
template <int N, int s>
__host__ __device__ constexpr int plan_radix() {
    if constexpr (s < Plan<N>::S) return Plan<N>::R[s];
    else return 1;
}
template <int N>
__host__ __device__ constexpr int tw_exponent(int idx) {
    constexpr int S = Plan<N>::S;
    const int Rf[3] = {plan_radix<N, 0>(), plan_radix<N, 1>(), plan_radix<N, 2>()};
    for (int dir = 0; dir < 2; ++dir) {
        int ns = 1;
        for (int st = 0; st < S; ++st) {
            const int R = dir ? Rf[S - 1 - st] : Rf[st];
            if (st > 0) {
                const int cnt = (R - 1) * ns;
                if (idx < cnt) return ((idx / ns + 1) * (idx % ns) * (N / (ns * R))) % N;
                idx -= cnt;
            }
            ns *= R;
        }
    }
    return -1;
}
// first entry of stage s of the forward (INV = false) or inverse stage order
template <int N, bool INV, int s>
__host__ __device__ constexpr int tw_offset() {
    constexpr int S = Plan<N>::S;
    const int Rf[3] = {plan_radix<N, 0>(), plan_radix<N, 1>(), plan_radix<N, 2>()};
    int off = 0;
    for (int dir = 0; dir < 2; ++dir) {
        int ns = 1;
        for (int st = 0; st < S; ++st) {
            const int R = dir ? Rf[S - 1 - st] : Rf[st];
            if (dir == (INV ? 1 : 0) && st == s) return off;
            if (st > 0) off += (R - 1) * ns;
            ns *= R;
        }
    }
    return -1;
}

// number of entries of the table (a constant expression)
template <int N>
__host__ __device__ constexpr int tw_entries() {
    int e = 0;
    while (tw_exponent<N>(e) >= 0) ++e;
    return e;
}
// tw_exponent for a run-time length (table builders); -1 for lengths without a plan
__host__ __device__ inline int tw_exponent_n(int n, int idx) {
    switch (n) {
        case 8: return tw_exponent<8>(idx);
        case 16: return tw_exponent<16>(idx);
        case 32: return tw_exponent<32>(idx);
        case 64: return tw_exponent<64>(idx);
        case 128: return tw_exponent<128>(idx);
        case 256: return tw_exponent<256>(idx);
        case 512: return tw_exponent<512>(idx);
        case 1024: return tw_exponent<1024>(idx);
        case 2048: return tw_exponent<2048>(idx);
        default: return -1;
    }
}

// Position along the line of register slot `slot` in the natural layout (forward input,
// inverse output) and in the spectral layout (forward output, inverse input).
template <int N>
__device__ __forceinline__ int pos_nat(int t, int slot) {
    using P = Plan<N>;
    constexpr int R0 = P::R[0];
    return t + P::T * (slot / R0) + (slot % R0) * (N / R0);
}
template <int N>
__device__ __forceinline__ int pos_spec(int t, int slot) {
    using P = Plan<N>;
    constexpr int RL = P::R[P::S - 1];
    return t + P::T * (slot / RL) + (slot % RL) * (N / RL);
}

// WARP: every line lies inside one warp (T <= 32, contiguous lanes); MASK names the lanes that
// exist in a CTA smaller than a warp.
template <bool WARP, unsigned MASK>
__device__ __forceinline__ void line_sync() {
    if constexpr (WARP) __syncwarp(MASK);
    else __syncthreads();
}

template <int N, bool INV, int s, bool WARP, unsigned MASK, bool TS = false>
struct FftStage {
    using P = Plan<N>;
    static constexpr int RMAX = P::RMAX, T = P::T, S = P::S;
    using SI = StageInfo<N, INV, s>;
    static constexpr int R = SI::R, NS = SI::NS;
    static constexpr int TWO = tw_offset<N, INV, s>();  // this stage's block of the twiddle table

    __device__ __forceinline__ static void run(float2 (&v)[RMAX], int t, float2* sm, const float4* __restrict__ tw) {
        constexpr int B = RMAX / R;
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int j = t + T * b;
            if constexpr (NS > 1) {
                const int k = j & (NS - 1);
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    // TS: the table is in shared memory; otherwise a read-only global load (L1)
                    const float4 w = TS ? tw[TWO + (r - 1) * NS + k] : __ldg(&tw[TWO + (r - 1) * NS + k]);
                    v[b * R + r] = INV ? cmul_c(v[b * R + r], make_float2(w.x, -w.y), make_float2(w.z, -w.w))
                                       : cmul_c(v[b * R + r], make_float2(w.x, w.y), make_float2(w.z, w.w));
                }
            }
            dft<R, INV>(&v[b * R]);
        }
        if constexpr (s + 1 < S) {
            constexpr int R2 = StageInfo<N, INV, s + 1>::R;
            constexpr int B2 = RMAX / R2;
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const int j = t + T * b;
                const int base = (j / NS) * NS * R + (j & (NS - 1));
#pragma unroll
                for (int r = 0; r < R; ++r) sm[pad_n(N, base + r * NS)] = v[b * R + r];
            }
            line_sync<WARP, MASK>();
#pragma unroll
            for (int b = 0; b < B2; ++b) {
                const int j = t + T * b;
#pragma unroll
                for (int r = 0; r < R2; ++r) v[b * R2 + r] = sm[pad_n(N, j + r * (N / R2))];
            }
            line_sync<WARP, MASK>();
            FftStage<N, INV, s + 1, WARP, MASK, TS>::run(v, t, sm, tw);
        }
    }
};

// The same stage on two lines held by the same threads (the two fields of a pair), interleaved: each
// twiddle is read once for both.  The table reads are the largest share of the shared-memory
// wavefronts of the heavy passes (a 128-bit read costs four per warp, whatever its broadcast), so
// serving two fields per read relieves the L1 data pipe those passes are bound by.
template <int N, bool INV, int s, bool WARP, unsigned MASK, bool TS = false>
struct FftStage2 {
    using P = Plan<N>;
    static constexpr int RMAX = P::RMAX, T = P::T, S = P::S;
    using SI = StageInfo<N, INV, s>;
    static constexpr int R = SI::R, NS = SI::NS;
    static constexpr int TWO = tw_offset<N, INV, s>();

    __device__ __forceinline__ static void run(float2 (&v)[RMAX], float2 (&u)[RMAX], int t, float2* smv, float2* smu,
                                               const float4* __restrict__ tw) {
        constexpr int B = RMAX / R;
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int j = t + T * b;
            if constexpr (NS > 1) {
                const int k = j & (NS - 1);
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    const float4 w = TS ? tw[TWO + (r - 1) * NS + k] : __ldg(&tw[TWO + (r - 1) * NS + k]);
                    const float2 hi = INV ? make_float2(w.x, -w.y) : make_float2(w.x, w.y);
                    const float2 lo = INV ? make_float2(w.z, -w.w) : make_float2(w.z, w.w);
                    v[b * R + r] = cmul_c(v[b * R + r], hi, lo);
                    u[b * R + r] = cmul_c(u[b * R + r], hi, lo);
                }
            }
            dft<R, INV>(&v[b * R]);
            dft<R, INV>(&u[b * R]);
        }
        if constexpr (s + 1 < S) {
            constexpr int R2 = StageInfo<N, INV, s + 1>::R;
            constexpr int B2 = RMAX / R2;
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const int j = t + T * b;
                const int base = (j / NS) * NS * R + (j & (NS - 1));
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    smv[pad_n(N, base + r * NS)] = v[b * R + r];
                    smu[pad_n(N, base + r * NS)] = u[b * R + r];
                }
            }
            line_sync<WARP, MASK>();
#pragma unroll
            for (int b = 0; b < B2; ++b) {
                const int j = t + T * b;
#pragma unroll
                for (int r = 0; r < R2; ++r) {
                    v[b * R2 + r] = smv[pad_n(N, j + r * (N / R2))];
                    u[b * R2 + r] = smu[pad_n(N, j + r * (N / R2))];
                }
            }
            line_sync<WARP, MASK>();
            FftStage2<N, INV, s + 1, WARP, MASK, TS>::run(v, u, t, smv, smu, tw);
        }
    }
};

template <int N, bool INV, bool WARP, unsigned MASK = 0xffffffffu, bool TS = false>
__device__ __forceinline__ void fft_line2(float2 (&v)[Plan<N>::RMAX], float2 (&u)[Plan<N>::RMAX], int t, float2* smv,
                                          float2* smu, const float4* __restrict__ tw) {
    FftStage2<N, INV, 0, WARP, MASK, TS>::run(v, u, t, smv, smu, tw);
}

// Forward (INV = false) or inverse transform of one line held as in pos_nat / pos_spec.
template <int N, bool INV, bool WARP, unsigned MASK = 0xffffffffu, bool TS = false>
__device__ __forceinline__ void fft_line(float2 (&v)[Plan<N>::RMAX], int t, float2* sm, const float4* __restrict__ tw) {
    FftStage<N, INV, 0, WARP, MASK, TS>::run(v, t, sm, tw);
}

}  // namespace twa
