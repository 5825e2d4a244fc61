/*
 * twa.h - C ABI of the GB300 truncated-Wigner (TWA) ensemble library (libtwa.so).
 *
 * Method (arXiv:2310.07119): a coherent state is represented by an ensemble of
 * classical fields drawn from its Wigner function (Sec. III.A, Eq.
 * eqn_stream_ensemble); every field evolves independently under the normalized
 * Schroedinger-Poisson equations (Sec. III.C, Eq. mft_normed)
 *     d psi/dt = -i ( -hbar/2 lap + V/hbar ) psi,    lap V = C |psi|^2,
 * integrated by the pseudo-spectral kick-drift-kick split step of Sec. III.B.2;
 * symmetric-operator expectation values are ensemble averages of Weyl symbols
 * (Sec. III.B.3, Eq. E[op]) and the size of the quantum correction is Q(t)
 * (Eq. Q).  "hbar" below always means hbar/m.
 *
 * Data layout (all device memory is owned by the caller unless stated):
 *   field      : one realization on an nx*ny*nz grid, x fastest, interleaved
 *                complex (float2 for TWA_F32, double2 for TWA_F64_PLAIN);
 *   batch      : for each instance i (in order), (n_real[i] + 1) fields:
 *                slot 0 is the classical field psi_cl (evolved without noise,
 *                Sec. II.C), slots 1..n_real[i] the sampled streams.
 *                Instance i starts at element offset sum_{j<i} (n_real[j]+1)*cells[j].
 *   psi_cl     : for each instance, one complex128 field (FP64 input),
 *                normalized to sum |psi|^2 dV = 1 (Sec. III.B.1).
 *
 * Every call returns 0 (TWA_OK) or a negative TWA_E* code; the message of the
 * last failure is available from twa_last_error().  All calls that take a
 * stream are asynchronous with respect to the host: they enqueue kernels on
 * that stream and return.  Device-side failures (non-finite fields) are
 * recorded in a device error word and reported by twa_sync_status().
 * There is no CPU fallback: without a CUDA device every call fails with
 * TWA_ECUDA.
 */
#ifndef TWA_H
#define TWA_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TWA_OK           0
#define TWA_EINVAL      -1   /* bad argument: null pointer, non-power-of-two or unsupported size */
#define TWA_ENOMEM      -2   /* device allocation failed */
#define TWA_ECUDA       -3   /* a CUDA runtime call failed (message has the CUDA error) */
#define TWA_ETIMEOUT    -4   /* a device-side wait gave up (reported through twa_sync_status) */
#define TWA_ENONFINITE  -5   /* a moments pass met a non-finite field value */

/* Alignment: the calls that take a handle return TWA_EINVAL when a field buffer (psi, psi_cl,
   psi_work) does not start on a 16-byte boundary; cudaMalloc and PyTorch allocations do.  Other
   device pointers need the alignment of their element type. */

#define TWA_F32          0   /* batched FP32 path: fused Stockham passes, realization pairs */
#define TWA_F64_PLAIN    1   /* comparator: complex128, one realization per launch, no fusion */

/* Number of FP64 scalars written per instance per output by twa_moments / twa_run. */
#define TWA_NSCALARS     8
#define TWA_S_Q          0   /* Q of Eq. Q: sum_g dV (mean|psi|^2 - |mean psi|^2) - M/(2 n) */
#define TWA_S_CORR       1   /* ||<rho> - rho_cl||_2 / ||rho_cl||_2 */
#define TWA_S_MASS       2   /* mean over streams of sum_g |psi|^2 dV (1 up to rounding) */
#define TWA_S_MASS_CL    3   /* sum_g |psi_cl|^2 dV */
#define TWA_S_NONFINITE  4   /* number of non-finite field values met (stored as double) */
#define TWA_S_NK_SUM     5   /* sum_k <n_k> (total occupation, ~ n_tot); 0 if modes are off */
#define TWA_S_DRHO_L2    6   /* ||<rho> - rho_cl||_2 */
#define TWA_S_RHOCL_L2   7   /* ||rho_cl||_2 */

/* Periodic box of Sec. III.B.1: dim axes of n[a] cells (powers of two, 8..2048;
   unused axes = 1), side L on every axis, dx = L / n[a]. */
typedef struct {
    int dim;
    int n[3];
    double L;
} twa_grid;

/* Physical and numerical parameters shared by all instances of a handle.
   hbar_m : hbar/m; C : coupling in lap V = C |psi|^2 (C = 4 pi G M_tot, Eq. mft_normed);
   dt     : time step of the split step (Sec. III.B.2);
   n_tot  : simulated particle number n^s_tot, used only by the sampling (Eq. sample);
   noise_conv : 0 = complex variance 1/2 per mode (coherent-state Wigner function),
                1 = variance 1/2 per real component (Eq. sample as printed);
   precision  : TWA_F32 or TWA_F64_PLAIN;
   want_modes : nonzero to allocate the spectral scratch used for per-mode moments. */
typedef struct {
    double hbar_m;
    double C;
    double dt;
    double n_tot;
    int noise_conv;
    int precision;
    int want_modes;
} twa_params;

/* Device FP64 outputs of one instance's moments (Eq. E[op]); any pointer may be NULL to skip it.
   nk_cl[cells]    = |a_k|^2 of the classical field (slot 0), same normalization (needs want_modes)
   rho_mean[cells] = mean_s |psi_s|^2 - 1/(2 n dV)   (Weyl symbol of psi^dag psi)
   psi_mean[2*cells] = mean_s psi_s                    (interleaved re, im)
   rho_cl[cells]   = |psi_cl|^2
   nk_mean[cells]  = mean_s |a_k|^2 - 1/2, a_k = sqrt(n dV / M) DFT(psi)_k (needs want_modes)
   nk_var[cells]   = mean |a|^4 - mean |a|^2 - (mean |a|^2 - 1/2)^2  (Var of a^dag a)
   scalars[TWA_NSCALARS] as defined above. Mode arrays are in FFT order (x fastest). */
typedef struct {
    double* rho_mean;
    double* psi_mean;
    double* rho_cl;
    double* nk_mean;
    double* nk_var;
    double* scalars;
    double* nk_cl;
} twa_moments_out;

typedef struct twa_handle twa_handle;

/* Create a handle for n_inst instances (grids[i], n_real[i] sampled streams each) sharing *p.
   The handle owns its scratch: the Poisson buffer (8 bytes per cell per pair of slots in
   FP32), the spectral scratch when want_modes is set, twiddle and phase tables, and the
   graph and autotune state.  Must be called with the target device current.
   Errors: TWA_EINVAL (sizes), TWA_ENOMEM, TWA_ECUDA. */
int twa_create(twa_handle** out, const twa_grid* grids, const twa_params* p,
               int n_inst, const int* n_real);

/* Release everything the handle owns (never caller memory).  Accepts NULL. */
int twa_destroy(twa_handle* h);

/* Element count (complex elements) of the batch buffer for all instances. */
size_t twa_batch_elems(const twa_handle* h);

/* Sec. III.B.1, Eq. sample: slot 0 of every instance <- psi_cl (rounded to the path's
   precision); slot s >= 1 <- psi_cl + sigma (zR + i zI), with zR, zI standard normals from
   Philox4x32-10 (key = seed, counter = (cell, s, instance, 0)) through Box-Muller in FP64,
   sigma^2 = v / (2 n_tot dV) per real component, v = 1/2 (noise_conv 0) or 1 (noise_conv 1).
   psi_cl: device complex128, instances concatenated; psi: device batch buffer. */
int twa_sample(twa_handle* h, const void* psi_cl, uint64_t seed, void* psi, void* stream);

/* Advance every field of the batch by n_steps kick-drift-kick steps of Sec. III.B.2:
   V(psi) -> exp(-i V dt / 2 hbar) -> FFT -> exp(-i hbar k^2 dt / 2) -> iFFT -> V(psi)
   -> exp(-i V dt / 2 hbar), with V_k = -C rho_k / k^2, V_0 = 0.  Adjacent half kicks are
   merged.  psi is read and written in place; asynchronous, no host synchronization. */
int twa_step_batch(twa_handle* h, void* psi, int n_steps, void* stream);

/* Ensemble moments of instance `inst` of the (synchronized) batch psi into *out
   (Sec. III.B.3, Eq. Q).  Reductions accumulate in FP64 in a fixed order (bitwise
   reproducible).  Per-mode outputs need want_modes. */
int twa_moments(twa_handle* h, int inst, const void* psi, const twa_moments_out* out, void* stream);

/* Continue a synchronized batch psi by n_steps KDK steps with moments at the start and every
   out_every steps: scalars go to series[(o * n_inst + i) * TWA_NSCALARS + j] (device FP64) for
   o = 0..n_steps/out_every.  Half kicks are merged across steps and the pending half kick is
   applied on the fly by the moments; psi ends synchronized.  On the FP32 path every output
   interval after the first is captured once as a CUDA graph and replayed (unless the pass
   profiler is on).  n_steps must be a multiple of out_every. */
int twa_advance(twa_handle* h, void* psi, int n_steps, int out_every, double* series, void* stream);

/* Continue a synchronized FP32 batch by n_out output intervals of out_every KDK steps with the
   dynamic time step of Sec. III.B.2 (the Delta t rule), chosen before each interval from the
   batch at its start and kept for the interval:
       dt = 2 pi c_f min[ hbar_m / max|V| ,  L dx / (pi hbar_m) ]
   with max|V| over every stream and cell of an instance, dx its smallest cell side, and the
   minimum taken over instances (all instances share the time axis).  The second bound keeps the
   gradient of the kinetic phase from aliasing (the printed term lacks one factor of L; for
   c_f = 1/pi it is the footnote's dt < 4 pi / (hbar k_max dk)); c_f > 0 is the caller's safety
   factor (the paper does not state its value).  Merged half kicks carry the step change.
   series: as for twa_advance (n_out + 1 outputs, device FP64); times: HOST array of n_out + 1
   doubles receiving the time of each output (times[0] = 0).  Reads max|V| back before every
   interval, so the call synchronizes `stream` n_out times and is not graph-captured; the handle's
   own dt and phase tables are restored before it returns.  FP32 path only (TWA_EINVAL
   otherwise); TWA_ENONFINITE if the potential is not finite. */
int twa_advance_adaptive(twa_handle* h, void* psi, int n_out, int out_every, double c_f, double* series,
                         double* times, void* stream);

/* Test particles (Sec. III.D, Eq. cl_int): one particle per slot of instance `inst` (slot 0 moves
   in the classical field's potential), dp/dt = -grad V_s(r), dr/dt = p (unit mass, normalized
   units), advanced by every later twa_step_batch / twa_advance / twa_advance_adaptive / twa_run in
   step with the field (leapfrog, half kicks merged like the field's).  grad V: the spectral
   derivative of V on the grid along each axis (Nyquist mode excluded) at the grid points around r,
   interpolated multilinearly; FP64 state and sums.  rp: HOST array [n_real + 1][6] = (r_x, r_y, r_z,
   p_x, p_y, p_z); positions are wrapped into [0, L), unused axes ignored.  FP32 path only.  Set the
   particles after twa_autotune (the tuner's timing steps would move them; setting them also moves
   a 3D instance with square xy planes to the plane pipeline, whose potential is real between
   steps); the 1D path then runs its on-chip steps one launch per step.  twa_particles_get synchronizes `stream`; it returns a
   synchronized state after any of the calls above. */
int twa_particles_set(twa_handle* h, int inst, const double* rp, void* stream);
int twa_particles_get(twa_handle* h, int inst, double* rp, void* stream);

/* Amplitude and phase variances of instance `inst` of a synchronized batch (Eq. varA, Eq. varPhi):
   per cell over the streams, A_s = |psi_s| with mean <A> and variance <dA^2>, and dphi_s =
   arg(psi_s conj(<psi>)) in (-pi, pi] (the phase relative to the ensemble-mean field; reference 0
   where that vanishes) with mean square <dphi^2>; with <rho> the Weyl-corrected mean density,
       totals[0] = sum_g dV <rho> <dA^2> / <A>,   totals[1] = sum_g dV <rho> <dphi^2> / (pi^2 / 3)
   (the printed pi / sqrt(3) read as the variance of a uniform phase, so a fully random phase gives
   the total mass).  var_a[cells], phi2[cells]: optional per-cell <dA^2> and <dphi^2>.  All outputs
   device FP64; sums in double-float (FP32 path) or FP64, fixed order.  Uses the instance's moment
   scratch: do not overlap with twa_moments of the same instance on another stream. */
int twa_phase_moments(twa_handle* h, int inst, const void* psi, double* var_a, double* phi2, double* totals,
                      void* stream);

/* Full run (Sec. III.B): twa_sample(psi_cl, seed) into psi_work, then twa_advance. */
int twa_run(twa_handle* h, const void* psi_cl, uint64_t seed, int n_steps, int out_every,
            void* psi_work, double* series, void* stream);

/* Pass profiler.  While enabled, every FP32 line pass is bracketed by CUDA events on its own
   stream and graph capture is skipped; twa_profile_read accumulates, per pass kind (op), the
   number of launches and their total device time in ms since the last enable.  Ops are numbered
   as in the library's pass table (TWA_PROF_NOPS kinds); bytes_per_cell receives the pass's
   algorithmic DRAM traffic in bytes per cell of one launched field (pair or slot). */
#define TWA_PROF_NOPS 14
int twa_profile_enable(twa_handle* h, int on);
int twa_profile_read(twa_handle* h, int op, long long* launches, double* total_ms, double* bytes_per_cell,
                     long long* fields_per_launch, long long* cells);

/* Allocation-free 1D step (no counterpart in the paper; an interface for callers that cannot
   allocate device memory where they step: a process whose device memory is owned by its own pool,
   a loop that must not risk an allocation failure or the synchronization cudaMalloc/cudaFree can
   cause).  Same computation as twa_step_batch on a one-instance 1D FP32 handle with these grid and
   params: psi is the caller's synchronized batch of n_real + 1 fields of grid->n[0] cells (float2,
   slot 0 = classical field), advanced in place by n_steps KDK steps on `stream`.  No handle is
   used: the Poisson buffer and the FFT and phase tables live in static device arrays of the
   library (TWA_STATIC_SCRATCH_ELEMS complex values plus about 106 KB of tables), held by every GPU
   that loads the library until the process exits.  The first call on a device looks up the device
   addresses of those arrays (make that first call before any stream capture).  Every call
   rebuilds the tables and the Poisson field; calls whose work overlaps on the GPU share the arrays
   and race.  Errors: TWA_EINVAL when psi is not 16-byte aligned, grid->dim != 1, precision !=
   TWA_F32, n[0] is not a power of two in [8, 2048], (n_real + 2) / 2 * n[0] >
   TWA_STATIC_SCRATCH_ELEMS, or (n_real + 2) / 2 > 65535 (message via twa_last_error(NULL)); all
   of these are found before anything is launched.  TWA_ECUDA on a CUDA failure (a failed launch
   of the Poisson passes returns before psi is touched). */
#define TWA_STATIC_SCRATCH_ELEMS (1 << 19)
int twa_step_batch_1d_static(const twa_grid* grid, const twa_params* p, int n_real, void* psi,
                             int n_steps, void* stream);

/* ---- Learned correction surrogate (no counterpart in the paper) --------------------------------
   A Fourier neural operator on the grid of Fourier modes of a grid^3 field: features of a TWA run
   (classical occupation, a few-stream correction estimate, ...) -> the ensemble correction spectrum
   <n_k> - n_k^cl.  h_0 = P x + p; z_l = Re A^H (R_l . A h_l) + W_l h_l + b_l; h_{l+1} = gelu(z_l)
   (l < layers-1); y = Q h_L + q, with A the unitary 3D DFT restricted to |m_a| < modes.  Weights are
   kept as an FP32 master vector and a BF16 copy used by the kernels (FP32 accumulation).  Flat
   parameter order: P (width x c_in), p, then per layer R ((2 modes)^3 x width x width, re/im), W_l
   (width x width), b_l, then Q (c_out x width), q.  Tensors are device float [B][C][grid^3].
   Requires 2 (2 modes)^3 <= grid^3. */
typedef struct {
    int grid;
    int width;
    int modes;
    int layers;
    int c_in;
    int c_out;
} twa_fno_config;
typedef struct twa_fno twa_fno;
int twa_fno_create(twa_fno** out, const twa_fno_config* cfg, uint64_t seed);
int twa_fno_destroy(twa_fno* f);
long long twa_fno_num_params(const twa_fno* f);
/* copy a flat FP32 parameter vector (device) in (resets the AdamW state) or out (which = 0: parameters,
   1: accumulated gradients) */
int twa_fno_set_params(twa_fno* f, const float* src, void* stream);
int twa_fno_get_params(twa_fno* f, float* dst, int which, void* stream);
/* forward for a batch of B inputs x[B][c_in][grid^3] -> y[B][c_out][grid^3]; keeps the activations
   (x must stay valid until the matching backward) */
int twa_fno_forward(twa_fno* f, const float* x, int B, float* y, void* stream);
/* backward of the last forward: accumulates parameter gradients; dx (optional) = dL/dx */
int twa_fno_backward(twa_fno* f, const float* dy, int B, float* dx, void* stream);
int twa_fno_zero_grad(twa_fno* f, void* stream);
/* AdamW step on the accumulated gradients (bias-corrected moments, decoupled weight decay) */
int twa_fno_adamw(twa_fno* f, float lr, float beta1, float beta2, float eps, float weight_decay, void* stream);
/* mean squared error of y against t (n floats) into *loss (device float); dy (optional) = dL/dy */
int twa_fno_mse(twa_fno* f, const float* y, const float* t, long long n, float* loss, float* dy, void* stream);
const char* twa_fno_last_error(const twa_fno* f);
/* The contractions along the contiguous axis of the truncated DFT (the forward transform of the
   real input rows and the real part of the adjoint's last axis) run as GEMMs on the tensor cores
   (TF32 operands, FP32 accumulation; see twa_tc_gemm) when their shapes allow: the forward when grid
   is a multiple of 32 (up to 128), the adjoint when 4 modes is.  twa_fno_tensor_core_shapes returns
   which (bit 0 forward, bit 1 adjoint); twa_fno_set_tensor_cores(f, 0) routes both back to the
   CUDA-core kernels (for comparisons).  twa_fno_sync_status blocks on `stream` and reports
   TWA_ETIMEOUT if a bounded wait of those GEMMs gave up since the last call, else TWA_OK. */
int twa_fno_set_tensor_cores(twa_fno* f, int on);
int twa_fno_tensor_core_shapes(const twa_fno* f);
int twa_fno_sync_status(twa_fno* f, void* stream);

/* Input features x[4][grid^3] of one snapshot from device FP64 per-mode occupations (FFT order),
   with nu = n_tot / grid^3: x0 = log10(1 + n_cl) / 8, x1 = (n_est - n_cl) / (n_cl + nu) (the
   few-stream correction estimate, relative), x2 = log10(n_tot) - 9, x3 = |m| / (grid/2); and, if t is
   not NULL, the target t[grid^3] = (n_ref - n_cl) / (n_cl + nu) from a reference ensemble. */
int twa_fno_features(const double* nk_cl, const double* nk_est, const double* nk_ref, double n_tot, int grid,
                     float* x, float* t, void* stream);

/* Tensor-core GEMM of tall-skinny FP32 matrices (no counterpart in the paper; the surrogate's DFT
   contractions use it, and tests call it directly): C[p][j] (+ C[p][j] if accumulate) =
   sum_k A[p][k] Bt[j][k] for p < P, j < N.  A: device, row stride lda floats; Bt: device [Np][K],
   rows N..Np-1 ignored (zero them); C: device, row stride ldc floats.  Operands are rounded to TF32
   (10-bit mantissa) by the tensor cores, products summed in FP32 in tensor memory (tcgen05); A and Bt
   tiles are moved by TMA.  Shapes: K a multiple of 32 up to 128, Np a multiple of 16 in [16, 256]
   with 128 K (256 + Np) + 1024 <= 232448 bytes of tiles (Np <= 192 at K = 128); A and Bt 16-byte aligned, lda * 4 a multiple of 16 (TWA_EINVAL otherwise).  Asynchronous on stream;
   a device-side wait that runs out (2 s) sets bit 4 of *err (device int). */
int twa_tc_gemm(const float* A, long long P, long long K, long long lda, const float* Bt, int N, int Np, float* C,
                long long ldc, int accumulate, int* err, void* stream);

/* Block on `stream` and report device-side failures recorded since the last call (TWA_ETIMEOUT: a
   bounded wait of the persistent launch gave up; TWA_ENONFINITE) or TWA_OK.  Clears the device
   error word. */
int twa_sync_status(twa_handle* h, void* stream);

/* How the instances of a batch run their steps (chosen by twa_autotune, or set here):
     TWA_BATCH_SERIAL     : one instance after another, one launch per pass;
     TWA_BATCH_FORK       : instances on parallel streams (parallel graph branches);
     TWA_BATCH_PERSISTENT : every step of every instance in one persistent launch per call (per output
                            interval of twa_advance) that walks a work list of (step, pass, instance,
                            pair of streams, tile of lines) items, Sec. III.A's independent streams
                            scheduled as data flow: an item starts once its pair's earlier passes are
                            done, so passes of different pairs and instances overlap.  Available for FP32
                            handles whose instances are all 2D with axes of 256 to 2048 cells and carry
                            no test particles (TWA_EINVAL otherwise).  Its device-side waits are bounded
                            (twa_set_wait_limit); a wait that runs out stops the launch and
                            twa_sync_status reports TWA_ETIMEOUT (the batch's fields are then undefined).
   The pass profiler runs the passes one by one whatever the mode.  twa_get_batch_mode returns the mode. */
#define TWA_BATCH_SERIAL      0
#define TWA_BATCH_FORK        1
#define TWA_BATCH_PERSISTENT  2
int twa_set_batch_mode(twa_handle* h, int mode);
int twa_get_batch_mode(const twa_handle* h);

/* Longest time a CTA of the persistent launch waits for a dependency, or a CTA of a TMA tile pass for
   its tile, before it gives up (default 2 s, 0 < seconds <= 60; counted in SM clock cycles at the
   device's peak clock). */
int twa_set_wait_limit(twa_handle* h, double seconds);

/* Fault injection for tests of the failure path: the next persistent launch of this handle waits for
   one tile that no work item produces, so its waits run out after the wait limit, the launch stops and
   twa_sync_status reports TWA_ETIMEOUT.  Nothing faults: the GPU stays usable and later calls run
   normally.  TWA_EINVAL if the handle has no persistent launch. */
int twa_debug_stall_next_batch(twa_handle* h);

/* Fault injection for tests of the failure path of the TMA tile pipelines: the next pass that runs a
   TMA variant (eagerly, outside a graph capture) expects 16 bytes per tile more than its copies
   deliver, so its CTAs' waits run out after the wait limit, the pass stops (the fields it was to
   update are undefined) and twa_sync_status reports TWA_ETIMEOUT.  Nothing faults: the GPU stays
   usable and later calls run normally.  TWA_EINVAL for an FP64 handle. */
int twa_debug_stall_next_tma(twa_handle* h);

/* Message of the last failure on this handle (or of the last twa_create failure if h is NULL). */
const char* twa_last_error(const twa_handle* h);

/* Autotune the FP32 pass shapes (lines per CTA, plain or pipelined variant) for every instance,
   the 3D pipeline (axis or plane passes) and, for several instances, whether they run on parallel
   streams, by timing candidates on `stream` with scratch fields; the choice is kept in the handle
   and, if cache_path is not NULL, merged into that JSON file (read first if it exists).  psi: a
   batch buffer the tuner may overwrite. */
int twa_autotune(twa_handle* h, void* psi, const char* cache_path, void* stream);

/* Number of kernel launches the last twa_step_batch / twa_run / twa_moments call enqueued. */
long long twa_last_launch_count(const twa_handle* h);

/* Stream averages of user functions (Appendix B: the synthesizer that evaluates arbitrary
   functions of the streams' fields and averages them across the streams, applied to every
   stream before averaging or to the averaged field).  f = f_re + i f_im is given as two C
   expressions (f_im NULL or "" means 0) in the double variables re, im (the field value), the
   long long i (index of the cell or mode, x fastest) and n (cells), and the ints nx, ny, nz;
   the CUDA math functions (sqrt, exp, atan2, pow, ...) are available.  Expressions are limited
   to arithmetic: brackets, braces, ';', '#', quotes, "->", "__" and pointer casts are refused.
   twa_observable_create compiles f with NVRTC (libnvrtc, opened on first use) for the current
   device.  Errors: TWA_EINVAL (bad flags, a refused or non-compiling expression; the compiler log
   is in twa_last_error(NULL)), TWA_ECUDA (no NVRTC or device).  flags: */
#define TWA_OBS_OF_MEAN 1  /* f of the streams' mean field, not the mean of f over the streams */
#define TWA_OBS_MODES   2  /* f of the Fourier amplitudes a_k = sqrt(n_tot dV / cells) DFT(psi)_k
                              (the number-unit amplitudes of the mode moments; FP32 path with
                              want_modes) instead of the field psi(x) */
#define TWA_OBS_FP32    4  /* evaluate f in FP32 (re, im float) and sum over the streams as float
                              pairs: about 1e-7 relative per value, much faster than FP64; math
                              functions then take float arguments (pow(x, 2.0f), not 2.0, which
                              is an ambiguous overload the compiler log reports) */
typedef struct twa_observable twa_observable;
int twa_observable_create(twa_observable** out, const char* f_re, const char* f_im, int flags);

/* Evaluate on instance `inst` of a synchronized batch psi, asynchronously on `stream`.  Over the
   sampled streams s = 1..n_real, per cell (or mode) c: per_cell[c] = (1/n_real) sum_s f(psi_s(c))
   or, with TWA_OBS_OF_MEAN, f((1/n_real) sum_s psi_s(c)); f_cl[c] = f(psi_0(c)) of the classical
   slot; total = sum_c per_cell[c] dV (position space) or sum_c per_cell[c] (modes).  per_cell and
   f_cl (device, 2 * cells doubles, complex interleaved) may be NULL; total (device, 2 doubles) may
   not.  Streams are summed in slot order and the total in a fixed order, so results are
   reproducible.  The evaluation is in FP64 (GB300's FP64 rate is 1/64 of FP32: expensive
   functions of 10^8-10^9 stream values take milliseconds to tens of milliseconds).  With
   TWA_OBS_MODES the handle's spectral scratch is overwritten.  An observable keeps one buffer of
   partial sums: evaluate it on one stream at a time.  Errors: TWA_EINVAL, TWA_ECUDA. */
int twa_observable_eval(twa_observable* ob, twa_handle* h, int inst, const void* psi, double* per_cell,
                        double* f_cl, double* total, void* stream);

/* Release an observable (accepts NULL). */
int twa_observable_destroy(twa_observable* ob);

/* Diagnostic: m[i] = 1/k2[i] for n device floats, computed as the FP32 transform passes compute
   the Poisson multiplier of Eq. mft_normed (a reciprocal approximation refined by one
   Newton-Raphson step; 0 where k2[i] <= 0), so tests can hold that arithmetic against IEEE
   division.  Asynchronous on `stream`.  Errors: TWA_EINVAL (null pointer, n < 0), TWA_ECUDA. */
int twa_poisson_multiplier(const float* k2, float* m, long long n, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* TWA_H */
