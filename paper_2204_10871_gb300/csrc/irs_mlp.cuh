// irs_mlp.cuh -- the learned far-far field (irs_mlp.cu), used by IRS_MLP plans.
#pragma once

#include "irs_common.cuh"

namespace irs {

constexpr int MLP_NF = 32;      // Fourier frequencies
constexpr int MLP_W = 64;       // hidden width
constexpr int MLP_OUT = 8;      // 4 complex series coefficients
constexpr int MLP_NPARAM = 13000;
constexpr int MLP_KFF = 4;      // far-far terms carried by the network
constexpr int MLP_KEXACT = 12;  // far-far terms summed exactly for cells near the rectangle's corners
constexpr double MLP_RF_DEFAULT = 8.0;  // window radius R_f in cells (irs_params.window of an
                                        // IRS_MLP plan): lenses within R_f/2 are summed directly
                                        // in full, beyond R_f the network carries them

// What the far-field finalize needs from the network for one map.
struct MlpFar {
  const float2* U;          // [nray cells][MLP_KFF] learned coefficients (theta_E units, tau^k)
  const int32_t* corner;    // [nray cells] index into `exact` or -1
  const double2* exact;     // [corner cells][MLP_KEXACT] exact far-far coefficients
  double rf;                // window radius (cells)
  int active;               // 1: the network replaces the FFT far field
};

// Lens weight of the direct ring: 1 inside R/2, 0 beyond R, and between them
// the C-infinity step w = b / (a + b), a = exp(-1/t), b = exp(-1/(1 - t)),
// t = 2r/R - 1.  Flat at 1 near the cell, so lenses that enter or leave the
// 3 x 3 near block as the cell moves never reach the far-far remainder, and
// smooth to every order in between, so the remainder's spectrum has no
// power-law tail from the taper.
__device__ __forceinline__ double mlp_ring_weight(double r, double R) {
  if (r <= 0.5 * R) return 1.0;
  if (r >= R) return 0.0;
  const double t = 2.0 * r / R - 1.0;
  const double a = exp(-1.0 / t), b = exp(-1.0 / (1.0 - t));
  return b / (a + b);
}

// host side (irs_mlp.cu)
irs_status mlp_plan(irs_plan_t* P, double gx0, double gy0, double h, int ncx, int ncy, int nrcx, int nrcy,
                    int ox, int oy, int64_t n_samples);
void mlp_destroy(irs_plan_t* P);
bool mlp_trained(const irs_plan_t* P);
irs_status mlp_prepare(irs_plan_t* P, const double* xy, const double* mass, int64_t n, double gx0, double gy0,
                       double h, int nrcx, int nrcy, int ox, int oy, MlpFar* far, cudaStream_t s);
irs_status mlp_set_params(irs_plan_t* P, const float* theta, const float* freq);
irs_status mlp_get_params(irs_plan_t* P, float* theta, float* freq);
irs_status mlp_grad(irs_plan_t* P, const float* x, const float* t, int64_t n, float* grad, double* loss,
                    cudaStream_t s);
irs_status mlp_forward(irs_plan_t* P, const float* x, int64_t n, float* y, cudaStream_t s);
irs_status mlp_train(irs_plan_t* P, const double* xy, const double* mass, int64_t n, int64_t n_samples,
                     int32_t steps, uint64_t seed, irs_mlp_report* rep, cudaStream_t s);
// level-1 cell side of an INTERP / MLP plan (irs_interp.cu)
double interp_cell_side(const irs_plan_t* P);

}  // namespace irs
