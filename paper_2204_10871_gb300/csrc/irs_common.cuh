// irs_common.cuh -- shared definitions of the CUDA library (not of the oracle).
//
// Complex notation used throughout the kernels: z = theta_1 + i theta_2.  A
// point lens m at z_i deflects by m (theta - theta_i)/|theta - theta_i|^2,
// which is conj(m / (z - z_i)), so the lens sum of Eq. (alpha1) is
// conj(L(z)) with L(z) = sum_i m_i / (z - z_i) analytic away from the lenses.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/irs.h"

namespace irs {

// ---------------------------------------------------------------- geometry
// Everything a kernel needs to know about one plan, passed by value.
struct Geo {
  double a1, a2, b1, b2;   // image/lens rectangle
  double cx, cy;           // rectangle centre (= circle centre)
  double dx3;              // ray spacing
  double src_x0, src_y0;   // source region origin
  double sx, sy;           // source pixel sides
  double kappa_s, gamma;
  double kstar_scale;      // kappa_*^act = kstar_scale * sum(m): pi/A (rect) or 1/R^2 (circle)
  int64_t nrx, nry;        // ray lattice
  int32_t npix_x, npix_y;
  int32_t plane;           // irs_plane
  int32_t pad_;
  float inv_sx, inv_sy;    // 1 / pixel side (FP32)
  float lam_s1, lam_s2;    // 1 - kappa_s - gamma, 1 - kappa_s + gamma
};

// ---------------------------------------------------------------- FP32 helpers
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Knuth's TwoSum: s + e == a + b exactly (round-to-nearest, no contraction).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Split an FP64 value into FP32 hi + lo with hi + lo == x to ~2^-48 relative.
__device__ __host__ __forceinline__ void split_df(double x, float& hi, float& lo) {
  hi = (float)x;
  lo = (float)(x - (double)hi);
}

// Warp-aggregated increment of counts[key] for every lane with valid == true:
// lanes that share a pixel elect one leader that adds their number.
__device__ __forceinline__ void bin_warp(uint32_t* counts, bool valid, uint32_t key) {
  const uint32_t k = valid ? key : 0xFFFFFFFFu;
  const unsigned peers = __match_any_sync(0xFFFFFFFFu, k);
  const int lane = threadIdx.x & 31;
  if (valid && lane == __ffs(peers) - 1) atomicAdd(counts + key, (uint32_t)__popc(peers));
}

// Key forms (~0u = no pixel) for the ray pass.  The leader of each group of
// equal keys is its lowest lane: no lower lane (lane_lt = its lane mask) shares it.
__device__ __forceinline__ void bin_warp_key(uint32_t* counts, uint32_t key, unsigned lane_lt) {
  const unsigned peers = __match_any_sync(0xFFFFFFFFu, key);
  if (key != 0xFFFFFFFFu && (peers & lane_lt) == 0u) atomicAdd(counts + key, (uint32_t)__popc(peers));
}

// Run-length variant: lanes hold consecutive columns of one row, so equal
// pixels usually come in runs; the first lane of each run of equal keys adds
// the run's length (non-adjacent equal keys add separately).
__device__ __forceinline__ void bin_warp_runs_key(uint32_t* counts, uint32_t key, int lane) {
  const uint32_t prev = __shfl_up_sync(0xFFFFFFFFu, key, 1);
  const bool head = (lane == 0) || (key != prev);
  const unsigned heads = __ballot_sync(0xFFFFFFFFu, head);
  if (key != 0xFFFFFFFFu && head) {
    const unsigned later = heads & ~((2u << lane) - 1u);  // heads after this lane
    const int next = later ? __ffs(later) - 1 : 32;
    atomicAdd(counts + key, (uint32_t)(next - lane));
  }
}

// Pixel of a ray from its position relative to the base pixel's lower-left
// corner (brel1, brel2 in theta_E): floor per axis, so a ray on a pixel edge
// belongs to the pixel above / to the right of it.
__device__ __forceinline__ bool pixel_from_rel(const Geo& g, int32_t ix, int32_t iy, float brel1,
                                               float brel2, uint32_t& key, int64_t& pix) {
  pix = -1;
  if (!(isfinite(brel1) && isfinite(brel2))) return false;
  const float f1 = floorf(brel1 * g.inv_sx), f2 = floorf(brel2 * g.inv_sy);
  if (!(fabsf(f1) < 1.0e9f && fabsf(f2) < 1.0e9f)) return false;
  const int64_t px = (int64_t)ix + (int64_t)f1, py = (int64_t)iy + (int64_t)f2;
  if (px < 0 || px >= g.npix_x || py < 0 || py >= g.npix_y) return false;
  pix = py * (int64_t)g.npix_x + px;
  key = (uint32_t)pix;
  return true;
}

// Pixel keys of two rays at once.  (t + 1.5 2^23) rounded toward -inf keeps
// floor(t) in its mantissa for |t| < 2^22: its bit pattern is
// 0x4B400000 + floor(t).  So with the base folded in, bx = ix - 0x4B400000
// (mod 2^32), the pixel index along an axis is bits + bx, and one unsigned
// range test rejects every ray off the map: a NaN or infinite t and any
// |t| >= 2^22 give a pattern that lands >= 8.7e8 away from the base, which
// no map reaches (|ix|, npix < 2^22 -- a map of 4e6 pixels per side).
constexpr float PIX_MAGIC = 12582912.0f;  // 1.5 2^23
constexpr uint32_t PIX_MAGIC_BITS = 0x4B400000u;
__device__ __forceinline__ void pixel_keys2(float2 t1, float2 t2, uint32_t bx, uint32_t by, uint32_t npix_x,
                                            uint32_t npix_y, uint32_t& ka, uint32_t& kb) {
  const float2 f1 = __fadd2_rd(t1, make_float2(PIX_MAGIC, PIX_MAGIC));
  const float2 f2 = __fadd2_rd(t2, make_float2(PIX_MAGIC, PIX_MAGIC));
  const uint32_t pxa = __float_as_uint(f1.x) + bx, pya = __float_as_uint(f2.x) + by;
  const uint32_t pxb = __float_as_uint(f1.y) + bx, pyb = __float_as_uint(f2.y) + by;
  ka = (pxa < npix_x && pya < npix_y) ? pya * npix_x + pxa : 0xFFFFFFFFu;
  kb = (pxb < npix_x && pyb < npix_y) ? pyb * npix_x + pxb : 0xFFFFFFFFu;
}

// pixel_keys2 plus each ray's bin in a box of hbx x hby pixels (lhx, lhy: the
// box origin folded with the floor's bit pattern offset, as bx, by); ~0u for
// rays off the map or outside the box.
__device__ __forceinline__ void pixel_keys2_box(float2 t1, float2 t2, uint32_t bx, uint32_t by,
                                                uint32_t npix_x, uint32_t npix_y, uint32_t lhx, uint32_t lhy,
                                                uint32_t hbx, uint32_t hby, uint32_t& ka, uint32_t& kb,
                                                uint32_t& la, uint32_t& lb) {
  const float2 f1 = __fadd2_rd(t1, make_float2(PIX_MAGIC, PIX_MAGIC));
  const float2 f2 = __fadd2_rd(t2, make_float2(PIX_MAGIC, PIX_MAGIC));
  const uint32_t ua = __float_as_uint(f1.x), va = __float_as_uint(f2.x);
  const uint32_t ub = __float_as_uint(f1.y), vb = __float_as_uint(f2.y);
  const uint32_t pxa = ua + bx, pya = va + by, pxb = ub + bx, pyb = vb + by;
  const bool ina = pxa < npix_x && pya < npix_y, inb = pxb < npix_x && pyb < npix_y;
  ka = ina ? pya * npix_x + pxa : 0xFFFFFFFFu;
  kb = inb ? pyb * npix_x + pxb : 0xFFFFFFFFu;
  const uint32_t xa = ua + lhx, ya = va + lhy, xb = ub + lhx, yb = vb + lhy;
  la = (ina && xa < hbx && ya < hby) ? ya * hbx + xa : 0xFFFFFFFFu;
  lb = (inb && xb < hbx && yb < hby) ? yb * hbx + xb : 0xFFFFFFFFu;
}

// Both rays of a row pair (keys ka, kb): lanes whose two keys are equal add
// 2 to it, the others 1 to ka, in one __match_any_sync on ka (the leader adds
// its peers plus its peers of weight 2); the kb of lanes whose keys differ
// go through a second match, run only when such a lane exists.
__device__ __forceinline__ void bin_warp_pair(uint32_t* counts, uint32_t ka, uint32_t kb, unsigned lane_lt) {
  const unsigned same = __ballot_sync(0xFFFFFFFFu, ka == kb);
  const unsigned peers = __match_any_sync(0xFFFFFFFFu, ka);
  if (ka != 0xFFFFFFFFu && (peers & lane_lt) == 0u)
    atomicAdd(counts + ka, (uint32_t)(__popc(peers) + __popc(peers & same)));
  if (same != 0xFFFFFFFFu) bin_warp_key(counts, ka == kb ? 0xFFFFFFFFu : kb, lane_lt);
}

// bin_warp_key into a shared-memory sub-histogram where the leader's ray has
// a box bin (lkey; equal keys have equal bins), into the map otherwise.
__device__ __forceinline__ void bin_warp_key_box(uint32_t* counts, uint32_t* hist, uint32_t key, uint32_t lkey,
                                                 unsigned lane_lt) {
  const unsigned peers = __match_any_sync(0xFFFFFFFFu, key);
  if (key != 0xFFFFFFFFu && (peers & lane_lt) == 0u) {
    const uint32_t n = (uint32_t)__popc(peers);
    if (lkey != 0xFFFFFFFFu) atomicAdd(hist + lkey, n);
    else atomicAdd(counts + key, n);
  }
}

// ---------------------------------------------------------------- brute force
constexpr int BR_TX = 32;             // tile columns: one per lane
constexpr int BR_TY = 64;             // tile rows: 64/R warps of R rows per thread
constexpr int BR_LT = 256;            // lenses per shared-memory stage (= FP32 partial length)
constexpr int BR_PAIRED = 4;          // rows per thread that share one reciprocal per two rows
constexpr int SHEET_TERMS = 8;        // Taylor terms t^1..t^8 of the sheet's analytic part
constexpr int MAX_NEAR = 4;           // rectangle corners evaluated per ray

// Per-tile constants computed in FP64 by the setup kernel.
struct __align__(16) TileRec {
  float cx_hi, cx_lo, cy_hi, cy_lo;   // beta of the tile centre without the lens sum, relative
                                      // to the base pixel's corner (double-float)
  int32_t ix, iy;                     // base pixel
  int32_t n_near, pad_;
  float T[SHEET_TERMS][2];            // Taylor coefficients of the sheet's analytic part, t^1..
  float near[MAX_NEAR][4];            // (z_T - c).re, .im, a_c, 0 of corners handled per ray
};

// Geometry of brute-force tile `tile` (row-major over tiles): first ray (i0, j0),
// one past the last valid ray (i1, j1), and the lattice coordinate of its centre.
struct TileGeo {
  int64_t i0, j0, i1, j1;
  double ci, cj;
};
__device__ __forceinline__ TileGeo tile_geo(const Geo& g, int64_t tile, int64_t ntx) {
  TileGeo t;
  const int64_t tx = tile % ntx, ty = tile / ntx;
  t.i0 = tx * BR_TX;
  t.j0 = ty * BR_TY;
  t.i1 = min(t.i0 + (int64_t)BR_TX, g.nrx);
  t.j1 = min(t.j0 + (int64_t)BR_TY, g.nry);
  t.ci = 0.5 * (double)(t.i0 + t.i1);
  t.cj = 0.5 * (double)(t.j0 + t.j1);
  return t;
}

}  // namespace irs

// ---------------------------------------------------------------- host side
namespace irs {
// timing event slots of irs_plan::ev
enum { EV_START = 0, EV_PREP, EV_CELLS, EV_FIN, EV_FAR, EV_RAY0, EV_RAY1, EV_MAG, EV_END, EV_COUNT };
}  // namespace irs

struct irs_plan {
  irs_params p;
  irs::Geo g;
  // FP64 sizing (flow chart)
  double kappa, border, lambda1, lambda2, ix0, iy0, ix, iy, circle_r;
  int64_t n_star_suggested;
  // brute-force tiling
  int64_t br_ntx, br_nty, br_ntiles;
  int br_grid;
  // device workspace
  void* ws;
  size_t ws_bytes;
  double* d_msum;          // [1] sum of masses
  double* d_mpart;         // [MSUM_BLOCKS] partial sums
  irs::TileRec* d_tiles;   // [br_ntiles]
  int* d_status;           // sticky device error
  int device;
  int num_sms;
  // INTERP state (irs_interp.cu)
  void* interp;
  // bumped whenever a device buffer that kernels address is reallocated, so
  // that captured graphs holding the old addresses are never replayed
  uint64_t ws_gen;
  // learned far field state (irs_mlp.cu), IRS_MLP plans only
  void* mlp;
  // stage timing (irs_plan_set_timing)
  int timing;
  cudaEvent_t ev[irs::EV_COUNT];
  int64_t timed_rays;
  int has_mag;
  int launches;  // kernel launches of the last map
};

namespace irs {
constexpr int MSUM_BLOCKS = 128;
constexpr int MSUM_THREADS = 256;

// launchers implemented in irs_brute.cu
// Sum of the masses into d_msum; with lens positions `xy` given (2n doubles),
// also the check that every lens lies in the plan's lens region (IRS_ERR_ARG
// into d_status otherwise).
cudaError_t launch_mass_sum(const irs_plan_t* P, const double* mass, int64_t n, cudaStream_t s,
                            const double* xy = nullptr);
cudaError_t launch_brute_setup(const irs_plan_t* P, cudaStream_t s);
cudaError_t launch_brute_map(const irs_plan_t* P, const double* xy, const double* mass, int64_t n,
                             int64_t row0, int64_t row1, uint32_t* counts, cudaStream_t s);
cudaError_t launch_brute_dump(const irs_plan_t* P, const double* xy, const double* mass, int64_t n,
                              const int64_t* idx, int64_t nidx, double* beta, int64_t* pix,
                              cudaStream_t s);
cudaError_t launch_magnify(const irs_plan_t* P, const uint32_t* counts, float* mag, cudaStream_t s);
int brute_grid_size(int num_sms, int variant);
int brute_num_variants();
// false when the variant's FP32 products of squared distances could leave the
// FP32 range on a plane of this diagonal (theta_E), or the variant is unknown
bool brute_variant_fits(int variant, double plane_diag);
// FP64 sizing of the plane and lattice (irs_api.cu)
irs_status size_plane(irs_plan_t* P);
// the flow chart's level-1 cell side in ray spacings, before the cell
// multiplier (irs_interp.cu; 0 for plans without interpolation state)
double interp_rule_rays(const irs_plan_t* P);
}  // namespace irs

// cached batch graphs that use a plan are dropped with it (irs_batch.cu)
void irs_batch_forget_plan(const irs_plan_t* plan);
