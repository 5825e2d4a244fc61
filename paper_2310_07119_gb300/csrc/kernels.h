// kernels.h - host launchers shared by the C ABI implementation (internal header).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace twa {

constexpr int NP_REAL = 6;   // per-block partial sums of the position-space moments
constexpr int NP_MODES = 2;  // per-block partial sums of the per-mode moments

int launch_sample_f32(const double2* psi_cl, float2* psi, long long cells, int n_slots, uint64_t seed,
                      int inst, double sigma, cudaStream_t st);
int launch_sample_f64(const double2* psi_cl, double2* psi, long long cells, int n_slots, uint64_t seed,
                      int inst, double sigma, cudaStream_t st);
int launch_kick_pairs(float2* psi, const float2* buf, long long cells, int n_slots, float kick, float kick_lo,
                      cudaStream_t st);
int moments_blocks(long long cells);
int launch_moments_real(const float2* psi, const float2* buf, long long cells, int n_slots, float kick,
                        float kick_lo, double inv_ns, double weyl, double* rho_mean, double* psi_mean, double* rho_cl,
                        double* part, cudaStream_t st);
int launch_moments_modes(const float2* spec, long long cells, int n_slots, double anorm2, double inv_ns,
                         double* nk_mean, double* nk_var, double* nk_cl, double* part, cudaStream_t st);
int launch_finish_scalars(const double* part_r, int nb_r, const double* part_m, int nb_m, double dV,
                          double q_offset, double* scalars, int* err_word, cudaStream_t st);
int launch_store_series(const double* cur, double* series, int* counter, int n, cudaStream_t st);
// scalars of outputs row0 .. row0 + n_outputs - 1 of one instance of a whole 1D run (k_run1d partials)
int launch_finish_run1d(const double* part, const double* part_cl, const double* part_bad, int n_pairs, int N,
                        int n_outputs, double inv_ns, double weyl, double dV, double q_offset, double n_tot_modes,
                        double* series, int row0, int inst, int n_inst, int* err_word, cudaStream_t st);
// max over the batch of |re| and |im| of n complex values, folded into *vmax (float bits; *vmax must
// start at 0 or at an earlier maximum)
int launch_max_abs(const float2* buf, long long n, unsigned* vmax, cudaStream_t st);
// m[i] = the transform passes' Poisson multiplier for k2[i]
int launch_poisson_multiplier(const float* k2, float* m, long long n, cudaStream_t st);
// test particles of one instance (one per slot), W the packed Poisson field in real space
int launch_particles(const float2* W, long long cells, const int* n, int dim, double L, const double* const* ker,
                     double fscale, double kick_dt, double drift_dt, int n_slots, double* prt, cudaStream_t st);
// amplitude and phase variances of one synchronized instance; part: moments_blocks(cells) * 2 doubles
int launch_phase_moments(const float2* psi, long long cells, int n_slots, double weyl, double dV, double* var_a,
                         double* phi2, double* part, double* out, cudaStream_t st);
int launch_phase_moments_f64(const double2* psi, long long cells, int n_slots, double weyl, double dV,
                             double* var_a, double* phi2, double* part, double* out, cudaStream_t st);

// Plain FP64 comparator path (one realization per launch, no fusion).
struct Geom64 {
    int dim;
    int n[3];
    long long cells;
};
struct Tables64 {
    const double2* tw[3];     // exp(-2 pi i m / n_a) per axis
    const double2* ph[3];     // exp(-i hbar k_a^2 dt / 2) per axis (FFT order)
    const double* k2[3];      // k_a^2 per axis
};
int launch_f64_fft3(double2* f, const Geom64& g, const Tables64& t, bool inverse, cudaStream_t st, long long* nl);
int launch_f64_kinetic(double2* f, const Geom64& g, const Tables64& t, cudaStream_t st, long long* nl);
int launch_f64_rho(const double2* psi, double2* work, long long cells, cudaStream_t st, long long* nl);
int launch_f64_poisson_mul(double2* work, const Geom64& g, const Tables64& t, double mulc, cudaStream_t st,
                           long long* nl);
int launch_f64_kick(double2* psi, const double2* work, long long cells, double kick, cudaStream_t st, long long* nl);
int launch_f64_moments_accum(const double2* psi, const double2* work, long long cells, double kick, int first,
                             double* acc /*3*cells*/, double* bad, cudaStream_t st, long long* nl);
int launch_f64_modes_accum(const double2* spec, long long cells, double anorm2, int first, double* acc2 /*2*cells*/,
                           cudaStream_t st, long long* nl);
int launch_f64_moments_finish(const double* acc, const double* acc2, const double2* psi0, long long cells, int n_real,
                              double weyl, double dV, double q_offset, double* rho_mean, double* psi_mean,
                              double* rho_cl, double* nk_mean, double* nk_var, double* part_r, double* part_m,
                              const double* bad, double* scalars, int* err_word, cudaStream_t st, long long* nl);

}  // namespace twa
