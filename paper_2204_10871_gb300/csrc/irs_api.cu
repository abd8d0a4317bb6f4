// irs_api.cu -- host side of the C ABI declared in include/irs.h: parameter
// validation, FP64 sizing of the image/lens plane (flow chart of Sec. 2.4),
// workspace ownership and the stream-ordered launch sequence of each method.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "irs_common.cuh"
#include "irs_interp.cuh"

using irs::Geo;

namespace {

irs_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return IRS_OK;
  if (e == cudaErrorMemoryAllocation) return IRS_ERR_OOM;
  return IRS_ERR_CUDA;
}

#define IRS_TRY(expr)                            \
  do {                                           \
    cudaError_t e_ = (expr);                     \
    if (e_ != cudaSuccess) return cuda_status(e_); \
  } while (0)

bool finite_all(const irs_params* p) {
  const double v[] = {p->kappa_star, p->kappa_s, p->gamma, p->src_x0, p->src_x1,
                      p->src_y0,     p->src_y1,  p->rays_per_pixel, p->border, p->cell_mult};
  for (double x : v)
    if (!isfinite(x)) return false;
  return true;
}

}  // namespace

// Sizing, flow chart of Sec. 2.4:
//   P = 10 sqrt(kappa_*)                      ("Protective Border")
//   I_x = (S_x + 2P)/|1 - kappa - gamma|, I_y = (S_y + 2P)/|1 - kappa + gamma|
//   Delta x3 = sqrt(s_x s_y / N_av), N_av rays per unlensed source pixel;
//   the plane is widened to a whole number of rays per side and centred on
//   the image of the source-region centre under the mean lens map.
irs_status irs::size_plane(irs_plan_t* P) {
  const irs_params& p = P->p;
  P->kappa = p.kappa_s + p.kappa_star;
  P->border = p.border < 0 ? 10.0 * sqrt(p.kappa_star) : p.border;
  P->lambda1 = 1.0 - P->kappa - p.gamma;
  P->lambda2 = 1.0 - P->kappa + p.gamma;
  if (fabs(P->lambda1) < 1e-6 || fabs(P->lambda2) < 1e-6) return IRS_ERR_DEGENERATE;
  const double Sx = p.src_x1 - p.src_x0, Sy = p.src_y1 - p.src_y0;
  P->ix0 = (Sx + 2.0 * P->border) / fabs(P->lambda1);
  P->iy0 = (Sy + 2.0 * P->border) / fabs(P->lambda2);
  Geo& g = P->g;
  g.sx = Sx / p.npix_x;
  g.sy = Sy / p.npix_y;
  g.dx3 = sqrt(g.sx * g.sy / p.rays_per_pixel);
  const double fx = ceil(P->ix0 / g.dx3 - 1e-9), fy = ceil(P->iy0 / g.dx3 - 1e-9);
  if (!(fx < 4.0e12 && fy < 4.0e12) || fx * fy > 9.0e15) return IRS_ERR_OVERFLOW;
  g.nrx = fx < 1 ? 1 : (int64_t)fx;
  g.nry = fy < 1 ? 1 : (int64_t)fy;
  P->ix = (double)g.nrx * g.dx3;
  P->iy = (double)g.nry * g.dx3;
  g.cx = 0.5 * (p.src_x0 + p.src_x1) / P->lambda1;
  g.cy = 0.5 * (p.src_y0 + p.src_y1) / P->lambda2;
  g.a1 = g.cx - 0.5 * P->ix;
  g.a2 = g.cx + 0.5 * P->ix;
  g.b1 = g.cy - 0.5 * P->iy;
  g.b2 = g.cy + 0.5 * P->iy;
  P->circle_r = 0.5 * sqrt(P->ix * P->ix + P->iy * P->iy);
  g.src_x0 = p.src_x0;
  g.src_y0 = p.src_y0;
  g.kappa_s = p.kappa_s;
  g.gamma = p.gamma;
  g.npix_x = p.npix_x;
  g.npix_y = p.npix_y;
  g.plane = p.plane;
  g.inv_sx = (float)(1.0 / g.sx);
  g.inv_sy = (float)(1.0 / g.sy);
  g.lam_s1 = (float)(1.0 - p.kappa_s - p.gamma);
  g.lam_s2 = (float)(1.0 - p.kappa_s + p.gamma);
  if (p.plane == IRS_PLANE_CIRCLE) {
    g.kstar_scale = 1.0 / (P->circle_r * P->circle_r);
    P->n_star_suggested = (int64_t)llround(p.kappa_star * P->circle_r * P->circle_r);
  } else {
    g.kstar_scale = M_PI / (P->ix * P->iy);
    P->n_star_suggested = (int64_t)llround(p.kappa_star * P->ix * P->iy / M_PI);
  }
  return IRS_OK;
}

namespace {

irs_status alloc_workspace(irs_plan_t* P) {
  P->br_ntx = (P->g.nrx + irs::BR_TX - 1) / irs::BR_TX;
  P->br_nty = (P->g.nry + irs::BR_TY - 1) / irs::BR_TY;
  P->br_ntiles = P->br_ntx * P->br_nty;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  };
  const size_t o_msum = take(sizeof(double));
  const size_t o_mpart = take(sizeof(double) * irs::MSUM_BLOCKS);
  const size_t o_status = take(sizeof(int));
  size_t o_tiles = 0;
  if (P->p.method == IRS_BRUTE) o_tiles = take(sizeof(irs::TileRec) * (size_t)P->br_ntiles);
  P->ws_bytes = off;
  if (cudaMalloc(&P->ws, P->ws_bytes) != cudaSuccess) {
    cudaGetLastError();
    P->ws = nullptr;
    return IRS_ERR_OOM;
  }
  char* b = static_cast<char*>(P->ws);
  P->d_msum = reinterpret_cast<double*>(b + o_msum);
  P->d_mpart = reinterpret_cast<double*>(b + o_mpart);
  P->d_status = reinterpret_cast<int*>(b + o_status);
  P->d_tiles = P->p.method == IRS_BRUTE ? reinterpret_cast<irs::TileRec*>(b + o_tiles) : nullptr;
  if (cudaMemset(P->ws, 0, P->ws_bytes) != cudaSuccess) return IRS_ERR_CUDA;
  return IRS_OK;
}

irs_status check_lenses(const double* xy, const double* mass, int64_t n) {
  if (n < 0) return IRS_ERR_ARG;
  if (n > 0 && (!xy || !mass)) return IRS_ERR_ARG;
  if (n > 0 && ((uintptr_t)xy & 15u)) return IRS_ERR_ARG;  // read as double2
  if (n > ((int64_t)1 << 31)) return IRS_ERR_OVERFLOW;
  return IRS_OK;
}

void mark(irs_plan_t* P, int slot, cudaStream_t s) {
  if (P->timing) cudaEventRecord(P->ev[slot], s);
}

// One map (or one band of lattice rows) in stream order: mass sum -> per-tile
// or per-cell setup -> [cells -> far field] -> ray pass -> magnification.
irs_status run_map(irs_plan_t* P, const double* xy, const double* mass, int64_t n, int64_t row0,
                   int64_t row1, uint32_t* counts, float* mag, cudaStream_t s, bool clear) {
  irs_status st = check_lenses(xy, mass, n);
  if (st != IRS_OK) return st;
  const size_t npix = (size_t)P->g.npix_x * P->g.npix_y;
  if (clear) IRS_TRY(cudaMemsetAsync(counts, 0, npix * sizeof(uint32_t), s));
  P->launches = 2;  // mass sum
  mark(P, irs::EV_START, s);
  IRS_TRY(irs::launch_mass_sum(P, mass, n, s, xy));
  if (P->p.method == IRS_BRUTE) {
    IRS_TRY(irs::launch_brute_setup(P, s));
    mark(P, irs::EV_PREP, s);
    mark(P, irs::EV_CELLS, s);
    mark(P, irs::EV_FIN, s);
    mark(P, irs::EV_FAR, s);
    mark(P, irs::EV_RAY0, s);
    IRS_TRY(irs::launch_brute_map(P, xy, mass, n, row0, row1, counts, s));
    P->launches += row1 > row0 ? 2 : 1;
    mark(P, irs::EV_RAY1, s);
  } else {
    st = irs::interp_run(P, xy, mass, n, row0, row1, counts, s);
    if (st != IRS_OK) return st;
  }
  mark(P, irs::EV_MAG, s);
  if (mag) IRS_TRY(irs::launch_magnify(P, counts, mag, s));
  if (mag) P->launches += 1;
  mark(P, irs::EV_END, s);
  P->timed_rays = (row1 - row0) * P->g.nrx;
  P->has_mag = mag != nullptr;
  return IRS_OK;
}

}  // namespace

extern "C" {

const char* irs_status_str(irs_status s) {
  switch (s) {
    case IRS_OK: return "ok";
    case IRS_ERR_ARG: return "invalid argument";
    case IRS_ERR_DEGENERATE: return "degenerate lens map (|1 - kappa -+ gamma| < 1e-6)";
    case IRS_ERR_OOM: return "device allocation failed";
    case IRS_ERR_CUDA: return "CUDA runtime error";
    case IRS_ERR_TIMEOUT: return "bounded device wait timed out";
    case IRS_ERR_OVERFLOW: return "size exceeds the kernels' index range";
    case IRS_ERR_NOT_TRAINED: return "far-field network not trained";
    case IRS_ERR_UNSUPPORTED: return "unsupported option";
  }
  return "unknown status";
}

irs_status irs_plan(const irs_params* params, void* stream, irs_plan_t** out) {
  (void)stream;
  if (!params || !out) return IRS_ERR_ARG;
  *out = nullptr;
  const irs_params& p = *params;
  if (!finite_all(params)) return IRS_ERR_ARG;
  if (p.npix_x <= 0 || p.npix_y <= 0 || !(p.rays_per_pixel > 0)) return IRS_ERR_ARG;
  if ((int64_t)p.npix_x * p.npix_y >= ((int64_t)1 << 32) - 1) return IRS_ERR_OVERFLOW;
  if (!(p.src_x1 > p.src_x0) || !(p.src_y1 > p.src_y0)) return IRS_ERR_ARG;
  if (p.kappa_star < 0 || p.kappa_s < 0 || p.n_star < 0) return IRS_ERR_ARG;
  if (p.plane != IRS_PLANE_RECT && p.plane != IRS_PLANE_CIRCLE) return IRS_ERR_ARG;
  if (p.method != IRS_BRUTE && p.method != IRS_INTERP && p.method != IRS_MLP) return IRS_ERR_ARG;
  if (p.flags != 0) return IRS_ERR_ARG;
  for (int k = 0; k < 6; ++k)
    if (p.reserved[k] != 0) return IRS_ERR_ARG;
  if (p.cell_mult < 0 || p.far_order < 0 || p.window < 0) return IRS_ERR_ARG;

  irs_plan_t* P = new (std::nothrow) irs_plan_t();
  if (!P) return IRS_ERR_OOM;
  memset(P, 0, sizeof(*P));
  P->p = p;
  irs_status st = irs::size_plane(P);
  if (st == IRS_OK && cudaGetDevice(&P->device) != cudaSuccess) st = IRS_ERR_CUDA;
  if (st == IRS_OK &&
      cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, P->device) != cudaSuccess)
    st = IRS_ERR_CUDA;
  if (st == IRS_OK) st = alloc_workspace(P);
  if (st == IRS_OK && p.method == IRS_BRUTE && (p.kernel_variant < 0 || p.kernel_variant >= irs::brute_num_variants()))
    st = IRS_ERR_ARG;
  if (st == IRS_OK && p.method == IRS_BRUTE && !irs::brute_variant_fits(p.kernel_variant, 2.0 * P->circle_r))
    st = IRS_ERR_UNSUPPORTED;
  if (st == IRS_OK) P->br_grid = irs::brute_grid_size(P->num_sms, p.method == IRS_BRUTE ? p.kernel_variant : 0);
  if (st == IRS_OK && p.method != IRS_BRUTE) st = irs::interp_plan(P);
  if (st != IRS_OK) {
    irs_plan_destroy(P);
    return st;
  }
  *out = P;
  return IRS_OK;
}

irs_status irs_plan_info_get(const irs_plan_t* P, irs_plan_info* info) {
  if (!P || !info) return IRS_ERR_ARG;
  memset(info, 0, sizeof(*info));
  info->lens_x0 = P->g.a1;
  info->lens_x1 = P->g.a2;
  info->lens_y0 = P->g.b1;
  info->lens_y1 = P->g.b2;
  info->center_x = P->g.cx;
  info->center_y = P->g.cy;
  info->border = P->border;
  info->dx_ray = P->g.dx3;
  info->pix_x = P->g.sx;
  info->pix_y = P->g.sy;
  info->circle_r = P->circle_r;
  info->n_rays_x = P->g.nrx;
  info->n_rays_y = P->g.nry;
  info->n_rays = P->g.nrx * P->g.nry;
  info->n_star_suggested = P->n_star_suggested;
  irs::interp_fill_info(P, info);
  info->workspace_bytes = (int64_t)P->ws_bytes + irs::interp_workspace_bytes(P);
  return IRS_OK;
}

irs_status irs_make_map(irs_plan_t* P, const double* xy, const double* mass, int64_t n,
                        uint32_t* counts, float* mag, void* stream) {
  if (!P || !counts) return IRS_ERR_ARG;
  return run_map(P, xy, mass, n, 0, P->g.nry, counts, mag, static_cast<cudaStream_t>(stream), true);
}

irs_status irs_make_map_rows(irs_plan_t* P, const double* xy, const double* mass, int64_t n,
                             int64_t row0, int64_t row1, uint32_t* counts, void* stream) {
  if (!P || !counts) return IRS_ERR_ARG;
  if (row0 < 0 || row1 < row0 || row1 > P->g.nry) return IRS_ERR_ARG;
  return run_map(P, xy, mass, n, row0, row1, counts, nullptr, static_cast<cudaStream_t>(stream),
                 false);
}

irs_status irs_magnify(irs_plan_t* P, const uint32_t* counts, float* mag, void* stream) {
  if (!P || !counts || !mag) return IRS_ERR_ARG;
  IRS_TRY(irs::launch_magnify(P, counts, mag, static_cast<cudaStream_t>(stream)));
  return IRS_OK;
}

irs_status irs_plan_set_timing(irs_plan_t* P, int32_t enable) {
  if (!P) return IRS_ERR_ARG;
  if (enable && !P->ev[0]) {
    for (int k = 0; k < irs::EV_COUNT; ++k) IRS_TRY(cudaEventCreate(&P->ev[k]));
  }
  P->timing = enable ? 1 : 0;
  return IRS_OK;
}

irs_status irs_plan_timings(irs_plan_t* P, irs_timings* out) {
  if (!P || !out) return IRS_ERR_ARG;
  memset(out, 0, sizeof(*out));
  if (!P->ev[0] || P->timed_rays < 0) return IRS_OK;
  IRS_TRY(cudaEventSynchronize(P->ev[irs::EV_END]));
  auto ms = [&](int a, int b) {
    float t = 0.f;
    cudaEventElapsedTime(&t, P->ev[a], P->ev[b]);
    return t;
  };
  out->ms_total = ms(irs::EV_START, irs::EV_END);
  out->ms_prep = ms(irs::EV_START, irs::EV_PREP);
  out->ms_cells = ms(irs::EV_PREP, irs::EV_CELLS);
  out->ms_farfield = ms(irs::EV_CELLS, irs::EV_FAR);
  out->ms_raypass = ms(irs::EV_RAY0, irs::EV_RAY1);
  out->ms_magnify = P->has_mag ? ms(irs::EV_MAG, irs::EV_END) : 0.f;
  out->ms_finalize = ms(irs::EV_FIN, irs::EV_FAR);
  out->rays = P->timed_rays;
  out->launches = P->launches;
  out->valid = 1;
  return IRS_OK;
}

irs_status irs_shoot_rays(irs_plan_t* P, const double* xy, const double* mass, int64_t n,
                          const int64_t* ray_idx, int64_t n_idx, double* beta, int64_t* pixel,
                          void* stream) {
  if (!P || n_idx < 0 || (n_idx > 0 && (!ray_idx || !beta))) return IRS_ERR_ARG;
  irs_status st = check_lenses(xy, mass, n);
  if (st != IRS_OK) return st;
  if (n_idx == 0) return IRS_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  IRS_TRY(irs::launch_mass_sum(P, mass, n, s, xy));
  if (P->p.method == IRS_BRUTE) {
    IRS_TRY(irs::launch_brute_setup(P, s));
    IRS_TRY(irs::launch_brute_dump(P, xy, mass, n, ray_idx, n_idx, beta, pixel, s));
    return IRS_OK;
  }
  return irs::interp_shoot_rays(P, xy, mass, n, ray_idx, n_idx, beta, pixel, s);
}

irs_status irs_plan_sync(irs_plan_t* P, void* stream) {
  if (!P) return IRS_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  IRS_TRY(cudaStreamSynchronize(s));
  IRS_TRY(cudaGetLastError());
  int status = 0;
  IRS_TRY(cudaMemcpy(&status, P->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (status != 0) {
    const int zero = 0;
    IRS_TRY(cudaMemcpy(P->d_status, &zero, sizeof(int), cudaMemcpyHostToDevice));
    return (irs_status)status;
  }
  return IRS_OK;
}

irs_status irs_plan_destroy(irs_plan_t* P) {
  if (!P) return IRS_OK;
  cudaDeviceSynchronize();
  irs_batch_forget_plan(P);
  irs::interp_destroy(P);
  for (int k = 0; k < irs::EV_COUNT; ++k)
    if (P->ev[k]) cudaEventDestroy(P->ev[k]);
  if (P->ws) cudaFree(P->ws);
  delete P;
  return IRS_OK;
}

}  // extern "C"
