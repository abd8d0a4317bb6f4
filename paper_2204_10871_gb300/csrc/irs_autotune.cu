// irs_autotune.cu -- choose the level-1 cell size and the ray-pass kernel
// variant of the interpolated method by timing them on the caller's lenses.
//
// Candidates: level-1 cell sizes times the ray-pass variants (rays per
// thread, level-2 sub-cells, sub-cell terms, CTAs per SM, binning, shared
// reciprocals), skipping cells wider than both 2 theta_E and the paper rule's
// cell (FP32 near-field precision).  The ray pass deals 32-column strips of a
// cell to warps, so where the rule's cell is at least 128 rays wide the sizes
// are the multiples of 32 rays from 0.5 to 1.25 rule cells (no idle lanes in
// a cell's last strip) and the rule itself; narrower rule cells take the
// multipliers 0.5 ... 2 of the rule.  Each cell size makes one plan, one
// warm-up and one timed map restricted to a band of lattice rows holding
// about 1e9 rays (the whole lattice when smaller), then times every variant's
// ray pass alone on that band's cells; a candidate's cost per map is the
// measured cell-list and far-field time plus its ray-pass time scaled to the
// full lattice.  Results
// are kept in a JSON-lines cache file keyed by a coarse signature of the
// parameters, so a sweep over many similar maps tunes once.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <iterator>
#include <mutex>
#include <string>
#include <vector>

#include "irs_common.cuh"
#include "irs_interp.cuh"

namespace {

const double CELL_MULTS[] = {0.5, 0.6, 0.70710678, 0.85, 1.0, 1.2, 1.41421356, 2.0};
constexpr int STRIP_RAYS = 32;  // columns of a ray-pass work unit (one per lane)

// Cell multipliers to try for a rule cell of `rule_rays` ray spacings.  The
// plan takes k = ceil(mult * rule_rays) rays per side, so (k - 1/2) / rule_rays
// gives exactly k.
std::vector<double> cell_candidates(double rule_rays) {
  std::vector<double> m;
  if (rule_rays >= 4.0 * STRIP_RAYS) {
    for (int k = 2 * STRIP_RAYS; k <= 1024; k += STRIP_RAYS)
      if (k >= 0.5 * rule_rays && k <= 1.25 * rule_rays) m.push_back(((double)k - 0.5) / rule_rays);
    m.push_back(1.0);
  } else {
    m.assign(std::begin(CELL_MULTS), std::end(CELL_MULTS));
  }
  return m;
}
constexpr double BAND_RAYS = 1.0e9;
std::mutex g_file_mu;

// Coarse signature: parameters that change the balance between the near sum,
// the far field and the ray count, bucketed so that similar maps share it.
std::string signature(const irs_params& p, int64_t n) {
  char buf[256];
  const double nav = p.rays_per_pixel;
  snprintf(buf, sizeof buf, "plane%d-ks%.2f-kss%.2f-g%.2f-px%dx%d-nav%d-nlog%d-area%.0f",
           p.plane, floor(p.kappa_star * 20.0 + 0.5) / 20.0, floor(p.kappa_s * 20.0 + 0.5) / 20.0,
           floor(fabs(p.gamma) * 20.0 + 0.5) / 20.0, p.npix_x, p.npix_y,
           (int)floor(log2(nav > 1 ? nav : 1) * 2.0 + 0.5), n > 0 ? (int)floor(log2((double)n) * 2 + 0.5) : -1,
           floor(log2((p.src_x1 - p.src_x0) * (p.src_y1 - p.src_y0)) * 2.0 + 0.5));
  return std::string(buf);
}

bool cache_lookup(const char* path, const std::string& key, double* mult, int* variant, double* ms) {
  if (!path || !*path) return false;
  std::lock_guard<std::mutex> lock(g_file_mu);
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char line[1024];
  bool found = false;
  while (fgets(line, sizeof line, f)) {
    char k[512];
    double m, t;
    int v;
    if (sscanf(line, "{\"key\": \"%511[^\"]\", \"cell_mult\": %lf, \"kernel_variant\": %d, \"ms\": %lf}",
               k, &m, &v, &t) == 4 &&
        key == k) {
      *mult = m;
      *variant = v;
      *ms = t;
      found = true;  // the last entry for a key wins
    }
  }
  fclose(f);
  return found;
}

void cache_store(const char* path, const std::string& key, double mult, int variant, double ms) {
  if (!path || !*path) return;
  std::lock_guard<std::mutex> lock(g_file_mu);
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "{\"key\": \"%s\", \"cell_mult\": %.8f, \"kernel_variant\": %d, \"ms\": %.6f}\n",
          key.c_str(), mult, variant, ms);
  fclose(f);
}

// Estimated milliseconds per full map for one candidate, or a negative value
// when the candidate cannot be planned.
// Largest level-1 cell side a candidate may have: FP32 cell-relative
// coordinates carry ~h 2^-24 of position error, which a lens at distance r
// amplifies by m / r^2 in the near sum; beyond 2 theta_E (or the paper rule's
// own cell, if larger) near-lens rays would lose the 1e-5 theta_E precision.
constexpr double MAX_CELL_SIDE = 2.0;

// Estimated milliseconds per full map of every ray-pass variant at one cell
// size (ms[v], negative when a variant cannot run), or false when the size
// cannot be planned.  One plan per size: a band map gives the far field's
// and the per-cell series' times (the same for every variant), then each
// variant's ray pass alone is timed on the band's cells (one warm-up launch,
// one timed).
bool measure_size(const irs_params& base, double mult, const double* xy, const double* mass, int64_t n,
                  uint32_t* counts, double h_rule, cudaStream_t s, std::vector<double>& ms) {
  ms.assign(irs::interp_num_variants(), -1.0);
  irs_params p = base;
  p.method = IRS_INTERP;
  p.cell_mult = mult;
  p.kernel_variant = 0;
  irs_plan_t* P = nullptr;
  if (irs_plan(&p, s, &P) != IRS_OK) return false;
  irs_plan_info info;
  irs_plan_info_get(P, &info);
  if (info.cell_x > fmax(MAX_CELL_SIDE, h_rule) * (1.0 + 1e-9)) {
    irs_plan_destroy(P);
    return false;
  }
  int64_t rows = (int64_t)ceil(BAND_RAYS / (double)info.n_rays_x);
  if (rows < 2 * info.rays_per_cell_y) rows = 2 * info.rays_per_cell_y;
  if (rows > info.n_rays_y) rows = info.n_rays_y;
  const int64_t r0 = (info.n_rays_y - rows) / 2 / (info.rays_per_cell_y) * info.rays_per_cell_y;
  const int64_t r1 = r0 + rows < info.n_rays_y ? r0 + rows : info.n_rays_y;
  const double scale = (double)info.n_rays_y / (double)(r1 - r0);
  const int64_t k = info.rays_per_cell_y;
  const double cell_scale = (double)((info.n_rays_y + k - 1) / k) / (double)((r1 + k - 1) / k - r0 / k);
  double base_ms = -1.0;  // everything but the ray pass, scaled to the whole lattice
  irs_plan_set_timing(P, 1);
  for (int rep = 0; rep < 2; ++rep) {
    if (irs_make_map_rows(P, xy, mass, n, r0, r1, counts, s) != IRS_OK) break;
    irs_timings t;
    if (irs_plan_timings(P, &t) != IRS_OK || !t.valid) break;
    if (rep == 1)
      base_ms = (double)(t.ms_total - t.ms_raypass - t.ms_finalize) + (double)t.ms_finalize * cell_scale;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (base_ms >= 0 && cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
    for (int v = 0; v < irs::interp_num_variants(); ++v) {
      if (irs::interp_set_variant(P, v) != IRS_OK) continue;
      float ray = -1.f;
      for (int rep = 0; rep < 2; ++rep) {
        if (irs::interp_raypass_rows(P, r0, r1, counts, s, e0, e1) != IRS_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ray, e0, e1) != cudaSuccess) {
          ray = -1.f;
          break;
        }
      }
      if (ray >= 0.f) ms[v] = base_ms + (double)ray * scale;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaGetLastError();
  if (irs_plan_sync(P, s) != IRS_OK) ms.assign(ms.size(), -1.0);
  irs_plan_destroy(P);
  return true;
}

}  // namespace

extern "C" irs_status irs_autotune(const irs_params* params, const double* lens_xy, const double* mass,
                                   int64_t n, const char* cache_path, irs_params* tuned,
                                   irs_tune_result* result, void* stream) {
  if (!params || !tuned || n < 0 || (n > 0 && (!lens_xy || !mass))) return IRS_ERR_ARG;
  *tuned = *params;
  irs_tune_result r;
  memset(&r, 0, sizeof r);
  if (!cache_path || !*cache_path) cache_path = getenv("IRS_AUTOTUNE_CACHE");
  if (params->method == IRS_BRUTE) {  // nothing to choose at run time
    if (result) *result = r;
    return IRS_OK;
  }
  const std::string key = signature(*params, n);
  double mult = 0, ms = 0;
  int variant = 0;
  if (cache_lookup(cache_path, key, &mult, &variant, &ms)) {
    tuned->cell_mult = mult;
    tuned->kernel_variant = variant;
    r.cell_mult = mult;
    r.kernel_variant = variant;
    r.ms_per_map = ms;
    r.from_cache = 1;
    if (result) *result = r;
    return IRS_OK;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint32_t* counts = nullptr;
  const size_t npix = (size_t)params->npix_x * params->npix_y;
  if (cudaMalloc(&counts, npix * sizeof(uint32_t)) != cudaSuccess) {
    cudaGetLastError();
    return IRS_ERR_OOM;
  }
  // the paper rule's cell side, the reference for the size guard
  double h_rule = 0.0, rule_rays = 0.0;
  {
    irs_params p = *params;
    p.method = IRS_INTERP;
    p.cell_mult = 1.0;
    p.kernel_variant = 0;
    irs_plan_t* P = nullptr;
    if (irs_plan(&p, s, &P) == IRS_OK) {
      irs_plan_info info;
      irs_plan_info_get(P, &info);
      h_rule = info.cell_x;
      rule_rays = irs::interp_rule_rays(P);
      irs_plan_destroy(P);
    }
  }
  double best = -1.0;
  std::vector<double> ms_v;
  for (double m : cell_candidates(rule_rays)) {
    if (!measure_size(*params, m, lens_xy, mass, n, counts, h_rule, s, ms_v)) continue;
    for (int v = 0; v < (int)ms_v.size(); ++v) {
      const double t = ms_v[(size_t)v];
      if (t < 0) continue;
      r.candidates++;
      if (m == 1.0 && v == 0) r.ms_default = t;
      if (best < 0 || t < best) {
        best = t;
        mult = m;
        variant = v;
      }
    }
  }
  cudaFree(counts);
  if (best < 0) return IRS_ERR_CUDA;
  tuned->cell_mult = mult;
  tuned->kernel_variant = variant;
  r.cell_mult = mult;
  r.kernel_variant = variant;
  r.ms_per_map = best;
  cache_store(cache_path, key, mult, variant, best);
  if (result) *result = r;
  return IRS_OK;
}
