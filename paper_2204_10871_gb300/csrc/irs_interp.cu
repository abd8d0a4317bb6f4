// irs_interp.cu -- the interpolated method of arXiv:2204.10871, Sec. 2.4
// ("Interpolation algorithm" and the flow chart's level-1/2/3 grids),
// re-designed for GB300.
//
//  level 1  square cells of k x k rays, side h = k Delta x3 with k from the
//           paper's Delta x1 = min(L0, min(I_x, I_y)/10), L0 = sqrt(A/N_*).
//           Lenses are binned into cells (counting sort, CSR, deterministic
//           order inside a cell).  A ray's "nearby lenses" are those of its own
//           cell and the 8 neighbours; they are summed directly per ray.
//  far      every other lens and the negative sheet are summed once per cell
//           into a Taylor series G_C(t) = sum_k c_k t^k about the cell centre:
//             cells at Chebyshev distance 2..W: each lens directly (P2L);
//             beyond W: multipole moments of each cell (P2M) translated to the
//             target cell by a convolution over the regular cell grid (M2L),
//             evaluated with FFTs, double-float for the low multipole and
//             local orders and FP32 for the rest (IP_PD, IP_KD below);
//             the rectangle sheet: its analytic part g(z), whose Taylor
//             coefficients are closed-form (rational for order >= 2).
//           The per-cell sums (window lenses, sheet, first series terms)
//           accumulate in FP64.
//  level 2  each cell's series is re-centred on Q x Q sub-cells (the paper's
//           level-2 grid points) with K2 terms, in shared memory per CTA.
//  level 3  the rays: one CTA per cell; near lenses broadcast from shared
//           memory, FP32 pair sums, sub-cell Horner, pixel, warp-aggregated
//           atomic binning.
//
// Per ray, with t = z - z_C (complex) and tau = t / h:
//   conj(beta) = B_C + (1 - kappa_s) conj(t) - gamma t - L_near(t) + sum_{k>=1} c_k tau^k
// where B_C = (1-kappa_s) conj(z_C) - gamma z_C + c_0 (rectangle), and
// L_near(t) = sum_near m_i / (t - t_i).  The kappa_* conj(z) parts of the
// matrix term and of the sheet cancel exactly and never appear.
#include <math.h>
#include <string.h>

#include <new>

#include "irs_df.cuh"
#include "irs_fft.cuh"
#include "irs_interp.cuh"
#include "irs_mlp.cuh"

namespace irs {

namespace {

constexpr int IP_KMAX = 32;        // local series terms (max)
constexpr int IP_P = 18;           // multipole terms per cell
constexpr int IP_KF = 14;          // local terms produced by the M2L (cells >= 4 apart:
                                   // truncation (0.71 / 3.29)^14 ~ 5e-10 of a cell's field)
// Precision split of the convolution.  Multipole order j reaches the local
// term k through kernels of order j + k, each cell >= 4 cells away, so its
// share of term k is at most (0.71 / 4)^j = 0.18^j of the monopole's; local
// term k moves a ray by at most 0.71^k times its value.  Only the low orders
// carry sums that FP32 cannot hold to 1e-7 theta_E (term 0 is a potential-like
// sum over the whole plane, term 1 grows with its logarithm): multipole
// planes j < IP_PD and local planes k < IP_KD, with the kernel planes their
// products need, are transformed and multiplied in double-float; every other
// plane and product in FP32 (the j >= 4 share of term 0 is below 1e-3 of it,
// so FP32 adds ~1e-10 relative; terms k >= 3 are stored as FP32 anyway).
constexpr int IP_PD = 4;
constexpr int IP_KD = 3;
constexpr int IP_NKD = IP_PD + IP_KD - 1;  // kernel orders n = j + k of the double-float products
constexpr int IP_NEAR_MAX = 1024;  // lenses of a 3x3 block held in shared memory
constexpr int IP_KMAX_RAYS = 1024;  // rays along a cell side (row table in shared memory)
constexpr int IP_THREADS = 256;
constexpr int IP_MAX_CORNER = 4;

constexpr int DEFAULT_K = 24;
constexpr int DEFAULT_W = 3;

struct __align__(16) CellRec {
  float bx_hi, bx_lo, by_hi, by_lo;  // beta of the centre (without L_near) relative to the base pixel
  int32_t ix, iy;                    // base pixel
  int32_t n_corner, pad_;
  float corner[IP_MAX_CORNER][4];    // (z_C - c).re, .im, a_c, 0: corners evaluated per ray
};

static_assert(sizeof(CellRec) % 4 == 0 && sizeof(CellRec) / 4 <= 32, "a warp copies a cell record word by word");

struct IpGeo {
  int64_t k;           // rays per cell side
  double h;            // cell side
  int32_t ncx, ncy;    // cell grid
  int32_t ox, oy;      // first ray cell
  int32_t nrcx, nrcy;  // ray cells
  double gx0, gy0;     // grid origin (lower-left corner of cell (0,0))
  int K, P, W;
  int variant;  // ray-pass kernel variant (R, Q, K2)
  float hf;     // (float) h
  float inv_k;  // 1 / k in FP32 (correctly rounded)
  int32_t nrow;  // row-pair entries of the ray pass's row table: (k + 1)/2 + IP_ROW_PAD
  int32_t pad_;
  // privatised binning (BIN 2): half extents, in pixels, of the box around a
  // cell's centre that holds its rays' pixels under the mean lens map, with
  // room for the near lenses' and the far field's spread
  float box_hx, box_hy;
};

struct InterpState {
  IpGeo ig;
  double rule_rays;  // the flow chart's Delta x1 in ray spacings, before the multiplier
  Fft2d fft;
  void* ws;
  size_t ws_bytes;
  void* lens_ws;
  size_t lens_ws_bytes;
  int64_t cap;
  int32_t* cell_count;
  int32_t* cell_start;
  int32_t* cell_cursor;
  int32_t* scan_blocks;
  int32_t* lens_cell;
  int32_t* sorted_idx;
  float4* lens_rel;
  double2* lens_pos;
  double* lens_m;
  float4* lens_pdf;  // positions as complex double-float (x.hi, x.lo, y.hi, y.lo)
  float2* lens_mdf;  // masses as double-float
  // far-field convolution: complex double-float (float4, irs_df.cuh) for
  // the low orders, FP32 (float2) for the rest
  float4* mpole_d;  // [PD][ncells]    multipoles j < PD
  float2* mpole_f;  // [P-PD][ncells]  multipoles j >= PD
  float4* spec_d;   // [PD][Ny][Nx]    their spectra; then local spectra k < KD
  float2* spec_f;   // [P-PD][Ny][Nx]  their spectra; then local spectra KD <= k < KF
  float4* kspec_d;  // [NKD][Ny][Nx]   kernel spectra n < NKD, normalised by 1/(Nx Ny)
  float2* kspec_f;  // [P+KF-1][Ny][Nx] every kernel spectrum in FP32
  float4* conv_d;   // [KD][ncells]    local terms k < KD
  float2* conv_f;   // [KF-KD][ncells] local terms KD <= k < KF
  CellRec* recs;   // [nray cells]
  float2* coef;    // [nray cells][K]
  // the rectangle sheet's corner series per ray cell divided by kappa_*
  // (geometry only; k_ip_sheet_table), rectangular planes only
  double2* sheet_d;     // [nray cells][FIN_K64] terms k < FIN_K64
  float2* sheet_f;      // [nray cells][K - FIN_K64] the rest
  uint8_t* sheet_near;  // [nray cells] bit q: corner q evaluated per ray instead
  int grid_ray;
};

InterpState* S_(irs_plan_t* P) { return static_cast<InterpState*>(P->interp); }
const InterpState* S_(const irs_plan_t* P) { return static_cast<const InterpState*>(P->interp); }

// ------------------------------------------------------------ complex FP64
struct cd {
  double re, im;
};
__device__ __forceinline__ cd cmul(cd a, cd b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__device__ __forceinline__ cd crecip(cd a) {
  const double d = a.re * a.re + a.im * a.im;
  return {a.re / d, -a.im / d};
}

// ------------------------------------------------------------ cell lists
__device__ __forceinline__ int cell_of(const IpGeo& ig, double x, double y) {
  long long cx = (long long)floor((x - ig.gx0) / ig.h);
  long long cy = (long long)floor((y - ig.gy0) / ig.h);
  cx = cx < 0 ? 0 : (cx >= ig.ncx ? ig.ncx - 1 : cx);  // lenses off the grid: edge cell
  cy = cy < 0 ? 0 : (cy >= ig.ncy ? ig.ncy - 1 : cy);
  return (int)(cy * ig.ncx + cx);
}

__global__ void k_ip_count(IpGeo ig, const double2* __restrict__ xy, int64_t n,
                           int32_t* __restrict__ lens_cell, int32_t* __restrict__ count) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double2 p = xy[i];
  const int c = cell_of(ig, p.x, p.y);
  lens_cell[i] = c;
  atomicAdd(count + c, 1);
}

// exclusive scan of int32 in three passes (block scan, scan of block sums, add)
constexpr int SCAN_B = 1024;
__global__ void k_scan_local(const int32_t* __restrict__ in, int32_t* __restrict__ out, int64_t n,
                             int32_t* __restrict__ block_sums) {
  __shared__ int32_t sh[SCAN_B];
  const int64_t i = (int64_t)blockIdx.x * SCAN_B + threadIdx.x;
  const int32_t v = i < n ? in[i] : 0;
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int off = 1; off < SCAN_B; off <<= 1) {
    int32_t t = threadIdx.x >= (unsigned)off ? sh[threadIdx.x - off] : 0;
    __syncthreads();
    sh[threadIdx.x] += t;
    __syncthreads();
  }
  if (i < n) out[i] = sh[threadIdx.x] - v;
  if (threadIdx.x == SCAN_B - 1) block_sums[blockIdx.x] = sh[SCAN_B - 1];
}
__global__ void k_scan_blocks(int32_t* __restrict__ block_sums, int64_t nb, int32_t* __restrict__ total) {
  if (threadIdx.x != 0) return;
  int32_t s = 0;
  for (int64_t b = 0; b < nb; ++b) {
    const int32_t v = block_sums[b];
    block_sums[b] = s;
    s += v;
  }
  *total = s;
}
__global__ void k_scan_add(int32_t* __restrict__ out, int64_t n, const int32_t* __restrict__ block_sums) {
  const int64_t i = (int64_t)blockIdx.x * SCAN_B + threadIdx.x;
  if (i < n) out[i] += block_sums[blockIdx.x];
}

__global__ void k_ip_scatter(const int32_t* __restrict__ lens_cell, int64_t n,
                             int32_t* __restrict__ cursor, int32_t* __restrict__ sorted_idx) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int pos = atomicAdd(cursor + lens_cell[i], 1);
  sorted_idx[pos] = (int32_t)i;
}

// Insertion sort of each cell's lens indices: the order inside a cell no
// longer depends on the atomics, so every map is bitwise reproducible.
__global__ void k_ip_sortcells(const int32_t* __restrict__ start, int64_t ncells,
                               int32_t* __restrict__ sorted_idx) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncells) return;
  const int a = start[c], b = start[c + 1];
  for (int i = a + 1; i < b; ++i) {
    const int32_t v = sorted_idx[i];
    int j = i - 1;
    while (j >= a && sorted_idx[j] > v) {
      sorted_idx[j + 1] = sorted_idx[j];
      --j;
    }
    sorted_idx[j + 1] = v;
  }
}

__global__ void k_ip_fill(IpGeo ig, const double2* __restrict__ xy, const double* __restrict__ mass,
                          const int32_t* __restrict__ sorted_idx, const int32_t* __restrict__ lens_cell,
                          int64_t n, float4* __restrict__ rel, double2* __restrict__ pos,
                          double* __restrict__ m_out, float4* __restrict__ pos_df, float2* __restrict__ m_df) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int32_t i = sorted_idx[p];
  const int c = lens_cell[i];
  const int cx = c % ig.ncx, cy = c / ig.ncx;
  const double zx = ig.gx0 + (cx + 0.5) * ig.h, zy = ig.gy0 + (cy + 0.5) * ig.h;
  const double2 q = xy[i];
  const double m = mass[i];
  rel[p] = make_float4((float)(q.x - zx), (float)(q.y - zy), (float)m, 0.f);
  pos[p] = q;
  m_out[p] = m;
  pos_df[p] = dfc_from_double(q.x, q.y);
  m_df[p] = df_from_double(m);
}

// ------------------------------------------------------------ far field
// P2M: a_j = sum_i m_i ((z_i - z_S)/h)^j for the lenses of cell S; orders
// j < IP_PD in FP64 (stored double-float), the rest in FP32 from the FP32
// offset (|d| <= 0.71; they are stored and convolved in FP32).
__global__ void k_ip_p2m(IpGeo ig, const int32_t* __restrict__ start, const double2* __restrict__ pos,
                         const double* __restrict__ m, float4* __restrict__ mpole_d,
                         float2* __restrict__ mpole_f) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t ncells = (int64_t)ig.ncx * ig.ncy;
  if (c >= ncells) return;
  const int cx = (int)(c % ig.ncx), cy = (int)(c / ig.ncx);
  const double zx = ig.gx0 + (cx + 0.5) * ig.h, zy = ig.gy0 + (cy + 0.5) * ig.h;
  cd a[IP_PD];
  float2 af[IP_P - IP_PD];
#pragma unroll
  for (int j = 0; j < IP_PD; ++j) a[j] = {0.0, 0.0};
#pragma unroll
  for (int j = 0; j < IP_P - IP_PD; ++j) af[j] = make_float2(0.f, 0.f);
  const double inv_h = 1.0 / ig.h;
  for (int p = start[c]; p < start[c + 1]; ++p) {
    const cd d = {(pos[p].x - zx) * inv_h, (pos[p].y - zy) * inv_h};
    cd pw = {m[p], 0.0};
#pragma unroll
    for (int j = 0; j < IP_PD; ++j) {
      a[j].re += pw.re;
      a[j].im += pw.im;
      pw = cmul(pw, d);
    }
    const float2 df = make_float2((float)d.re, (float)d.im);
    float2 pf = make_float2((float)pw.re, (float)pw.im);  // m d^PD
#pragma unroll
    for (int j = 0; j < IP_P - IP_PD; ++j) {
      af[j].x += pf.x;
      af[j].y += pf.y;
      pf = make_float2(fmaf(pf.x, df.x, -pf.y * df.y), fmaf(pf.x, df.y, pf.y * df.x));
    }
  }
#pragma unroll
  for (int j = 0; j < IP_PD; ++j) mpole_d[(int64_t)j * ncells + c] = dfc_from_double(a[j].re, a[j].im);
#pragma unroll
  for (int j = 0; j < IP_P - IP_PD; ++j) mpole_f[(int64_t)j * ncells + c] = af[j];
}

// Translation kernels on the padded grid, scaled by n! / (Nx Ny):
// K'_n[e] = n! (-e)^-(n+1) / (Nx Ny) for offsets e (cell units, wrapped) with
// Chebyshev norm > W, else 0 (the n! is one factor of the M2L's binomial,
// below; the 1/(Nx Ny) normalises the inverse FFT and keeps every spectrum
// far inside the FP32 exponent range).  Orders n < nkd in double-float (kg_d),
// every order in FP32 (kg_f).
__global__ void k_ip_kernel_grid(int Nx, int Ny, int W, int nker, int nkd, float4* __restrict__ kg_d,
                                 float2* __restrict__ kg_f) {
  const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t G = (int64_t)Nx * Ny;
  if (f >= G) return;
  const int ex = (int)(f % Nx), ey = (int)(f / Nx);
  const int sx = ex < Nx / 2 ? ex : ex - Nx, sy = ey < Ny / 2 ? ey : ey - Ny;
  const bool far = abs(sx) > W || abs(sy) > W;
  cd inv = {0.0, 0.0};
  if (far) inv = crecip(cd{-(double)sx, -(double)sy});
  cd pw = inv;
  double fact = 1.0 / (double)G;  // n! / (Nx Ny)
  for (int n = 0; n < nker; ++n) {
    if (n > 0) fact *= (double)n;
    const double re = far ? pw.re * fact : 0.0, im = far ? pw.im * fact : 0.0;
    if (n < nkd) kg_d[(int64_t)n * G + f] = dfc_from_double(re, im);
    kg_f[(int64_t)n * G + f] = make_float2((float)re, (float)im);
    pw = cmul(pw, inv);
  }
}

// Pointwise M2L in frequency space:
//   C_k = sum_j (-1)^j binom(j+k, k) A_j Kh_{j+k},  j < P, k < KF,
// with binom(j+k, k) = (j+k)! / (j! k!): the (j+k)! sits in the kernel
// spectra, so each term is one complex multiply-add of (-1)^j A_j / j! and
// the scaled kernel, and C_k takes the 1/k! at the end.  Products with
// j < PD and k < KD in double-float, the others in FP32 (the FP32 operands
// of the double-float planes are their high parts); the FP32 share of
// C_k, k < KD, joins the double-float sum before the scaling.
__global__ void __launch_bounds__(128) k_ip_m2l_freq(int64_t G, float4* __restrict__ spec_d,
                                                     float2* __restrict__ spec_f,
                                                     const float4* __restrict__ kspec_d,
                                                     const float2* __restrict__ kspec_f) {
  const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= G) return;
  float4 Ad[IP_PD], Cd[IP_KD];
  float2 Af[IP_P], Cf[IP_KF];
  double ifact = 1.0;  // 1/j!, folded at compile time
#pragma unroll
  for (int j = 0; j < IP_P; ++j) {
    if (j > 0) ifact /= (double)j;
    const double sc = ((j & 1) ? -1.0 : 1.0) * ifact;
    if (j < IP_PD) {
      Ad[j] = dfc_scale(spec_d[(int64_t)j * G + f], df_from_double(sc));
      Af[j] = make_float2(Ad[j].x, Ad[j].z);
    } else {
      const float2 v = spec_f[(int64_t)(j - IP_PD) * G + f];
      Af[j] = make_float2(v.x * (float)sc, v.y * (float)sc);
    }
  }
#pragma unroll
  for (int k = 0; k < IP_KD; ++k) Cd[k] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int k = 0; k < IP_KF; ++k) Cf[k] = make_float2(0.f, 0.f);
#pragma unroll
  for (int nn = 0; nn < IP_P + IP_KF - 1; ++nn) {
    const float2 kf = kspec_f[(int64_t)nn * G + f];
    const float4 kd = nn < IP_NKD ? kspec_d[(int64_t)nn * G + f] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int j = 0; j < IP_P; ++j) {
      const int k = nn - j;
      if (k < 0 || k >= IP_KF) continue;
      if (j < IP_PD && k < IP_KD) {
        Cd[k] = dfc_add(Cd[k], dfc_mul(Ad[j], kd));
      } else {
        Cf[k].x = fmaf(Af[j].x, kf.x, fmaf(-Af[j].y, kf.y, Cf[k].x));
        Cf[k].y = fmaf(Af[j].x, kf.y, fmaf(Af[j].y, kf.x, Cf[k].y));
      }
    }
  }
  double kfact = 1.0;  // 1/k!
#pragma unroll
  for (int k = 0; k < IP_KF; ++k) {
    if (k > 0) kfact /= (double)k;
    if (k < IP_KD) {
      const float4 c = dfc_add(Cd[k], make_float4(Cf[k].x, 0.f, Cf[k].y, 0.f));
      spec_d[(int64_t)k * G + f] = dfc_scale(c, df_from_double(kfact));
    } else {
      spec_f[(int64_t)(k - IP_KD) * G + f] = make_float2(Cf[k].x * (float)kfact, Cf[k].y * (float)kfact);
    }
  }
}

// Series terms of the per-cell finalize accumulated in FP64; the others in
// FP32.  A window lens sits >= 1.5 cells from the cell centre and a ray
// <= 0.71 cells from it, so term k of a lens contributes at most
// (m/d) 0.47^k: FP32 rounding of the terms k >= 3 moves a ray's deflection by
// <= 1e-7 x 0.1 of that lens's field, and every term k >= 1 is stored as FP32
// for the ray pass anyway.  Terms 0..2 (the constant, which sets the ray's
// beta, and the two largest slopes) keep FP64.
constexpr int FIN_K64 = 3;
constexpr int FIN_K32 = IP_KMAX - FIN_K64;
static_assert(IP_KD >= FIN_K64, "FP32 local planes feed only FP32 accumulators");

// 1/a for complex a, |a| >~ 1e-19 (cell or theta_E units): an FP32 seed for
// 1/|a|^2 refined by one FP64 Newton step (relative error ~1e-14), instead of
// two FP64 divisions.
__device__ __forceinline__ cd crecip_nr(cd a) {
  const double q = a.re * a.re + a.im * a.im;
  double r = (double)rcp_approx((float)q);
  r = r * fma(-q, r, 2.0);
  return {a.re * r, -a.im * r};
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// 1/(re + i im) in double-float: conj / |.|^2, the reciprocal of |.|^2 from
// the FP32 reciprocal of its high part and one Newton step r + r (1 - q r)
// (quadratic convergence: ~2^-47 relative).  |.| >= 1 here (window lenses
// are at least a cell away, in cell units).
__device__ __forceinline__ float4 dfc_recip(float2 re, float2 im) {
  const float2 q = df_add(df_mul(re, re), df_mul(im, im));
  const float2 r0 = make_float2(__frcp_rn(q.x), 0.f);
  const float2 e = df_sub(make_float2(1.f, 0.f), df_mul(q, r0));
  const float2 r = df_add(r0, df_mul(r0, e));
  return dfc_make(df_mul(re, r), df_neg(df_mul(im, r)));
}

// Corners of the lens rectangle (a1, b1), (a2, b1), (a1, b2), (a2, b2) and
// the signs of their a_c / kappa_* * pi.
__device__ __forceinline__ double sheet_corner_x(const Geo& g, int q) { return (q & 1) ? g.a2 : g.a1; }
__device__ __forceinline__ double sheet_corner_y(const Geo& g, int q) { return (q & 2) ? g.b2 : g.b1; }
__device__ __forceinline__ double sheet_corner_sign(int q) { return (q == 0 || q == 3) ? 1.0 : -1.0; }

// Per ray cell: the four corner terms of the sheet's analytic part,
// sum_c -i (a_c / kappa_*) (z - c) Log(z - c), as a series in tau = (z -
// z_C)/h: terms k < FIN_K64 in FP64, the next K - FIN_K64 in FP32.  They
// depend on the plan's geometry alone, so a plan builds them once and each
// map scales them by its kappa_*.  A corner within 4 x 0.71 h of the centre
// is left out (bit q of `near`): the ray pass evaluates it per ray.
__global__ void k_ip_sheet_table(Geo g, IpGeo ig, double2* __restrict__ sheet_d, float2* __restrict__ sheet_f,
                                 uint8_t* __restrict__ sheet_near, int64_t nrc) {
  const int64_t rc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (rc >= nrc) return;
  const int cx = (int)(rc % ig.nrcx) + ig.ox, cy = (int)(rc / ig.nrcx) + ig.oy;
  const double zx = ig.gx0 + (cx + 0.5) * ig.h, zy = ig.gy0 + (cy + 0.5) * ig.h;
  const double h = ig.h;
  const int nsf = ig.K - FIN_K64;
  cd acc[FIN_K64];
  float2 accf[FIN_K32];
#pragma unroll
  for (int k = 0; k < FIN_K64; ++k) acc[k] = {0.0, 0.0};
#pragma unroll
  for (int k = 0; k < FIN_K32; ++k) accf[k] = make_float2(0.f, 0.f);
  unsigned near = 0;
  const double rho = 4.0 * 0.70710678118654752 * h;
  for (int q = 0; q < 4; ++q) {
    const double ac = sheet_corner_sign(q) / M_PI;
    const cd w = {zx - sheet_corner_x(g, q), zy - sheet_corner_y(g, q)};
    if (hypot(w.re, w.im) < rho) {
      near |= 1u << q;
      continue;
    }
    // Log(z - c) on the branch that is continuous with the rectangle's
    // interior: the principal cuts of the two right-hand corners run along
    // the top and bottom edges, so a cell centre beyond those edges (a
    // ragged last cell row) takes the argument across the cut.
    double arg = atan2(w.im, w.re);
    if (q == 3 && w.re < 0.0 && w.im > 0.0) arg -= 2.0 * M_PI;  // (a2, b2), centre above b2
    if (q == 1 && w.re < 0.0 && w.im < 0.0) arg += 2.0 * M_PI;  // (a2, b1), centre below b1
    const cd L = {0.5 * log(w.re * w.re + w.im * w.im), arg};
    const cd wl = cmul(w, L);
    acc[0].re += ac * wl.im;
    acc[0].im -= ac * wl.re;
    acc[1].re += ac * L.im * h;
    acc[1].im -= ac * (L.re + 1.0) * h;
    const cd inv = crecip_nr(w);
    const cd ih = {inv.re * h, inv.im * h};
    cd pw = {inv.re * h * h, inv.im * h * h};  // h^n / w^(n-1) at n = 2
    // n = 2 in FP64 (FIN_K64 = 3), n >= 3 in FP32
    acc[2].re += ac * 0.5 * pw.im;
    acc[2].im -= ac * 0.5 * pw.re;
    pw = cmul(pw, ih);
    const float2 ihf = make_float2((float)ih.re, (float)ih.im);
    float2 pf = make_float2((float)pw.re, (float)pw.im);
    const float acf = (float)ac;
#pragma unroll
    for (int k = 0; k < FIN_K32; ++k) {
      const int n = k + FIN_K64;
      const float cf = ((n & 1) ? -1.0f : 1.0f) / (float)(n * (n - 1));
      accf[k].x += acf * cf * pf.y;
      accf[k].y -= acf * cf * pf.x;
      pf = cmulf(pf, ihf);
    }
  }
#pragma unroll
  for (int k = 0; k < FIN_K64; ++k) sheet_d[rc * FIN_K64 + k] = make_double2(acc[k].re, acc[k].im);
#pragma unroll
  for (int k = 0; k < FIN_K32; ++k) {
    if (k >= nsf) break;
    sheet_f[rc * nsf + k] = accf[k];
  }
  sheet_near[rc] = (uint8_t)near;
}

// Per ray cell of [rc0, rc1): window P2L, M2L result, sheet series, centre
// term, base pixel.  NF: FP32 series terms computed (k = FIN_K64 ...
// FIN_K64 + NF - 1; at least K - FIN_K64).
template <int NF>
__global__ void __launch_bounds__(64)
k_ip_finalize(Geo g, IpGeo ig, const double* __restrict__ msum, const int32_t* __restrict__ start,
              const double2* __restrict__ pos, const double* __restrict__ m, const float4* __restrict__ pos_df,
              const float2* __restrict__ m_df, const float4* __restrict__ conv_d,
              const float2* __restrict__ conv_f, MlpFar far, const double2* __restrict__ sheet_d,
              const float2* __restrict__ sheet_f, const uint8_t* __restrict__ sheet_near,
              CellRec* __restrict__ recs, float2* __restrict__ coef, int64_t rc0, int64_t rc1) {
  const int64_t rc = rc0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (rc >= rc1) return;
  const int cx = (int)(rc % ig.nrcx) + ig.ox, cy = (int)(rc / ig.nrcx) + ig.oy;
  const int64_t ncells = (int64_t)ig.ncx * ig.ncy;
  const int64_t c = (int64_t)cy * ig.ncx + cx;
  const double zx = ig.gx0 + (cx + 0.5) * ig.h, zy = ig.gy0 + (cy + 0.5) * ig.h;
  const double h = ig.h, inv_h = 1.0 / h;
  const int K = ig.K;

  // coefficients of tau^k before the 1/h of the lens parts: k < FIN_K64 in
  // FP64, the rest in FP32 (terms past K are computed and dropped)
  cd acc[FIN_K64];
  float2 accf[NF];
  float4 accd[FIN_K64];  // the window's terms k < FIN_K64 in double-float (series mode)
#pragma unroll
  for (int k = 0; k < FIN_K64; ++k) {
    acc[k] = {0.0, 0.0};
    accd[k] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
#pragma unroll
  for (int k = 0; k < NF; ++k) accf[k] = make_float2(0.f, 0.f);
  const float2 zx_df = df_from_double(zx), zy_df = df_from_double(zy), ih_df = df_from_double(inv_h);
  // direct ring: lenses of cells at Chebyshev distance 2..W (series mode), or
  // every lens outside the near block weighted by w(r) out to R_f (network
  // mode).  The (cell, lens) pairs are walked as one sequence per thread, one
  // lens per step, so that the lanes of a warp, whose windows hold different
  // numbers of lenses per cell, stay busy until their own lenses run out.
  const int Wd = far.active ? (int)ceil(far.rf) + 1 : ig.W;
  const int side = 2 * Wd + 1, nwin = side * side;
  int q = -1, p = 0, pend = 0;  // window cell (row-major), lens range left in it
  while (true) {
    while (p >= pend && ++q < nwin) {
      const int dy = q / side - Wd, dx = q % side - Wd;
      const int x = cx + dx, y = cy + dy;
      if ((abs(dx) <= 1 && abs(dy) <= 1) || x < 0 || x >= ig.ncx || y < 0 || y >= ig.ncy) continue;
      const int64_t s = (int64_t)y * ig.ncx + x;
      p = start[s];
      pend = start[s + 1];
    }
    if (q >= nwin) break;
    const int pl = p++;  // this step's lens (the step always advances)
    float2 invf, pf;
    if (far.active) {  // network mode: the ring weight wants |d| in FP64
      const cd d = {(pos[pl].x - zx) * inv_h, (pos[pl].y - zy) * inv_h};
      const double wm = m[pl] * mlp_ring_weight(hypot(d.re, d.im), far.rf);
      if (wm == 0.0) continue;
      const cd inv = crecip_nr(d);
      cd pw = {wm * inv.re, wm * inv.im};  // + m d^-(k+1)
#pragma unroll
      for (int k = 0; k < FIN_K64; ++k) {
        acc[k].re += pw.re;
        acc[k].im += pw.im;
        pw = cmul(pw, inv);
      }
      invf = make_float2((float)inv.re, (float)inv.im);
      pf = make_float2((float)pw.re, (float)pw.im);
    } else {  // series mode: the same terms in double-float on the FP32 pipes
      const float4 q4 = pos_df[pl];
      const float2 dre = df_mul(df_sub(make_float2(q4.x, q4.y), zx_df), ih_df);
      const float2 dim = df_mul(df_sub(make_float2(q4.z, q4.w), zy_df), ih_df);
      const float4 inv = dfc_recip(dre, dim);
      float4 pw = dfc_scale(inv, m_df[pl]);  // + m d^-(k+1)
#pragma unroll
      for (int k = 0; k < FIN_K64; ++k) {
        accd[k] = dfc_add(accd[k], pw);
        pw = dfc_mul(pw, inv);
      }
      invf = make_float2(inv.x, inv.z);
      pf = make_float2(pw.x, pw.z);
    }
#pragma unroll
    for (int k = 0; k < NF; ++k) {
      accf[k].x += pf.x;
      accf[k].y += pf.y;
      pf = cmulf(pf, invf);
    }
  }
#pragma unroll
  for (int k = 0; k < FIN_K64; ++k) {
    acc[k].re += df_to_double(dfc_re(accd[k]));
    acc[k].im += df_to_double(dfc_im(accd[k]));
  }
  // outer cells through the FFT convolution (series mode)
  if (!far.active) {
#pragma unroll
    for (int k = 0; k < IP_KF; ++k) {
      if (k >= K) break;
      if (k < IP_KD) {
        const float4 v = conv_d[(int64_t)k * ncells + c];
        if (k < FIN_K64) {
          acc[k].re += df_to_double(dfc_re(v));
          acc[k].im += df_to_double(dfc_im(v));
        } else {
          accf[k - FIN_K64].x += v.x + v.y;
          accf[k - FIN_K64].y += v.z + v.w;
        }
      } else {
        const float2 v = conv_f[(int64_t)(k - IP_KD) * ncells + c];
        accf[k - FIN_K64].x += v.x;
        accf[k - FIN_K64].y += v.y;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < FIN_K64; ++k) {
    acc[k].re *= inv_h;
    acc[k].im *= inv_h;
  }
  const float inv_hf = (float)inv_h;
#pragma unroll
  for (int k = 0; k < NF; ++k) {
    accf[k].x *= inv_hf;
    accf[k].y *= inv_hf;
  }
  // network mode away from corners: G = -L_ring - U - kappa_* conj(z_C); the
  // sheet's g cancels against the definition of U
  const bool learned = far.active && far.corner[rc] < 0;
  if (far.active && !learned) {  // corner zone: exact far-far sum, then the sheet as usual
    const double2* ex = far.exact + (int64_t)far.corner[rc] * MLP_KEXACT;
#pragma unroll
    for (int k = 0; k < MLP_KEXACT; ++k) {
      if (k >= K) break;
      if (k < FIN_K64) {
        acc[k].re -= ex[k].x;
        acc[k].im -= ex[k].y;
      } else {
        accf[k - FIN_K64].x -= (float)ex[k].x;
        accf[k - FIN_K64].y -= (float)ex[k].y;
      }
    }
  }

  const double ks = g.kstar_scale * msum[0];
  const double kap = g.kappa_s + ks;
  CellRec r;
  r.n_corner = 0;
  r.pad_ = 0;
  for (int q = 0; q < IP_MAX_CORNER; ++q) r.corner[q][0] = r.corner[q][1] = r.corner[q][2] = r.corner[q][3] = 0.f;
  cd B;
  if (learned) {
    const double ks0 = g.kstar_scale * msum[0];
#pragma unroll
    for (int k = 0; k < MLP_KFF; ++k) {
      if (k >= K) break;
      const float2 u = far.U[rc * MLP_KFF + k];
      if (k < FIN_K64) {
        acc[k].re -= (double)u.x;
        acc[k].im -= (double)u.y;
      } else {
        accf[k - FIN_K64].x -= u.x;
        accf[k - FIN_K64].y -= u.y;
      }
    }
    acc[0].re -= ks0 * zx;  // kappa_* conj(z_C)
    acc[0].im += ks0 * zy;
    B = {(1.0 - g.kappa_s - g.gamma) * zx, -(1.0 - g.kappa_s + g.gamma) * zy};
  } else if (g.plane == IRS_PLANE_CIRCLE) {
    B = {(1.0 - g.kappa_s - g.gamma) * zx - ks * g.cx, -(1.0 - g.kappa_s + g.gamma) * zy + ks * g.cy};
  } else {
    // sheet: g(z) = kappa_* (z - 2 a2) + sum_c -i a_c (z - c) Log(z - c); adds
    // g_k h^k.  a_c = +-kappa_* / pi, so the corner sums are kappa_* times a
    // per-plan table (k_ip_sheet_table); corners near the cell go to the rays.
    acc[0].re += ks * (zx - 2.0 * g.a2);
    acc[0].im += ks * zy;
    acc[1].re += ks * h;
    if (ks != 0.0) {
      const unsigned near = sheet_near[rc];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (!((near >> q) & 1u)) continue;
        r.corner[r.n_corner][0] = (float)(zx - sheet_corner_x(g, q));
        r.corner[r.n_corner][1] = (float)(zy - sheet_corner_y(g, q));
        r.corner[r.n_corner][2] = (float)(ks / M_PI * sheet_corner_sign(q));
        r.n_corner++;
      }
#pragma unroll
      for (int k = 0; k < FIN_K64; ++k) {
        const double2 t = sheet_d[rc * FIN_K64 + k];
        acc[k].re += ks * t.x;
        acc[k].im += ks * t.y;
      }
      const int nsf = K - FIN_K64;
      const float ksf = (float)ks;
#pragma unroll
      for (int k = 0; k < NF; ++k) {
        if (k >= nsf) break;
        const float2 t = sheet_f[rc * nsf + k];
        accf[k].x = fmaf(ksf, t.x, accf[k].x);
        accf[k].y = fmaf(ksf, t.y, accf[k].y);
      }
    }
    B = {(1.0 - g.kappa_s - g.gamma) * zx, -(1.0 - g.kappa_s + g.gamma) * zy};
  }
  B.re += acc[0].re;
  B.im += acc[0].im;
  const double m1 = (1.0 - kap - g.gamma) * zx, m2 = (1.0 - kap + g.gamma) * zy;
  double fx = floor((m1 - g.src_x0) / g.sx), fy = floor((m2 - g.src_y0) / g.sy);
  fx = fmin(fmax(fx, -1.0e9), 1.0e9);
  fy = fmin(fmax(fy, -1.0e9), 1.0e9);
  r.ix = (int32_t)fx;
  r.iy = (int32_t)fy;
  split_df(B.re - (g.src_x0 + fx * g.sx), r.bx_hi, r.bx_lo);
  split_df(-B.im - (g.src_y0 + fy * g.sy), r.by_hi, r.by_lo);
  recs[rc] = r;
#pragma unroll
  for (int k = 0; k < FIN_K64 + NF; ++k) {
    if (k >= K) break;
    coef[rc * K + k] = k < FIN_K64 ? make_float2((float)acc[k].re, (float)acc[k].im) : accf[k - FIN_K64];
  }
}

// ------------------------------------------------------------ ray pass
enum { IP_MAP = 0, IP_DUMP = 1 };

struct IpRayArgs {
  const int32_t* start;
  const float4* rel;
  const CellRec* recs;
  const float2* coef;
  uint32_t* counts;
  int* status;
  int64_t row0, row1;
  int64_t rc_base;  // first ray cell of the work range
  const int64_t* idx;
  double* beta_out;
  int64_t* pix_out;
  int64_t nwork;
};

// Kernel variants of the ray pass (the autotuner picks one per plan):
// rays per thread R, level-2 sub-cells per side Q, sub-cell series terms K2.
// The truncation is (sub-cell half-diagonal / distance to the nearest far
// lens)^K2 of that lens's field: Q = 8, 10, 12, 16 give ratios 0.083, 0.067,
// 0.057, 0.042, so 8, 7, 6 and 6 terms stay at or below ~3e-8; variants 11
// and 13-15 trade one Horner step per ray for bounds of 1.7e-7 (16 sub-cells,
// 5 terms), 3.3e-7 (14) and 7.3e-7 (12), the last with fewer sub-cells to
// re-centre per cell; variant 16 takes one more step off with 4 terms on 16
// sub-cells (3.1e-6, more sub-cells to re-centre).
// MINB: CTAs per SM the register budget is sized for; BIN: warp binning by
// __match_any_sync (0), by runs of equal pixels (1), or by __match_any_sync
// into a shared-memory sub-histogram over the cell's pixel box, flushed to
// the map once per cell, with global atomics for rays outside the box (2),
// or by row pairs (3: a pair whose two rays share a pixel adds 2 in one
// __match_any_sync; a second one runs only when some lane's pair differs);
// NPR: how many of a
// thread's R/2 row pairs share one reciprocal per lens, 1/(r_a^2 r_b^2) (the
// near sum is bound by the MUFU's 16 reciprocals per SM per clock; a shared
// reciprocal trades one MUFU op for FP32 work on a pipe that is half idle).
#define IP_VARIANTS(X)                                                                       \
  X(0, 8, 12, 6, 3, 0, 0) X(1, 8, 10, 7, 3, 0, 0) X(2, 8, 16, 6, 3, 0, 2)                       \
  X(3, 8, 16, 6, 3, 0, 4) X(4, 8, 16, 6, 2, 1, 0) X(5, 8, 16, 6, 3, 1, 0)                      \
  X(6, 8, 16, 6, 3, 1, 2) X(7, 8, 16, 6, 3, 0, 0) X(8, 4, 16, 6, 4, 0, 0)                      \
  X(9, 8, 8, 8, 3, 0, 0) X(10, 8, 12, 6, 4, 0, 0) X(11, 8, 16, 5, 3, 0, 0)                    \
  X(12, 8, 16, 5, 3, 2, 0) X(13, 8, 16, 5, 3, 3, 0) X(14, 8, 12, 5, 3, 3, 0) X(15, 8, 14, 5, 3, 3, 0) \
  X(16, 8, 16, 4, 3, 3, 0)
constexpr int IP_NVARIANT = 17;

// Advance a (strip, row group) position by `by` units of a row-major
// nstrip-wide unit grid.
__device__ __forceinline__ void step_unit(int& st, int& rg, int by, int nstrip) {
  st += by;
  while (st >= nstrip) {
    st -= nstrip;
    ++rg;
  }
}

// Row table of a cell, one entry per pair of cell rows (2l, 2l + 1).
struct __align__(16) IpRowPair {
  float4 sg;  // (sigma_y, sigma_y', -sigma_y, -sigma_y'), sigma_y = (l + 1/2) Q / k - v - 1/2
  float4 ty;  // (tau_y h, tau_y' h, y0, y0'), y0 = by_lo + lambda_2 tau_y h: the row's share of beta_2
  int2 v;     // (v Q, v' Q): level-2 row offsets
};

// Row pairs of the row table past the cell's last: a thread's R / 2 pairs
// are read without clamping the index (R <= 2 IP_ROW_PAD).
constexpr int IP_ROW_PAD = 4;

// Row stride (float2) of the per-cell table of scaled series coefficients:
// odd, so that the K2 rows a warp reads at once fall in distinct banks.
constexpr int IP_CB_STRIDE = IP_KMAX + 1;

// Dynamic shared memory of the ray pass (bytes, 16-byte aligned blocks):
// near lenses as (-x, -x, -y, -y) and (-m, -m) pairs, the level-2 series
// as conj duplicated (c.re, c.re, -c.im, -c.im), the row table and the
// level-1 series scaled for the re-centring, one row per level-2 term.
// Bins of the privatised sub-histogram (BIN 2): a cell whose pixel box is
// larger bins globally.
constexpr int IP_HIST_MAX = 2048;

// The row table holds `nrow` entries, sized per plan from its cell side
// (IpGeo::nrow), so that small cells leave shared memory for more CTAs; the
// privatised binning adds its sub-histogram at the end.
template <int Q, int K2, int BIN>
struct IpSmem {
  static constexpr size_t near_xy = 0;
  static constexpr size_t near_m = near_xy + sizeof(float4) * IP_NEAR_MAX;
  static constexpr size_t sub = near_m + sizeof(float2) * IP_NEAR_MAX;
  static constexpr int nrow_max = IP_KMAX_RAYS / 2 + IP_ROW_PAD;
  static constexpr size_t row_sg = sub + sizeof(float4) * Q * Q * K2;
  static __host__ __device__ constexpr size_t coef(int nrow) { return row_sg + sizeof(IpRowPair) * nrow; }
  static __host__ __device__ constexpr size_t hist(int nrow) {
    return (coef(nrow) + sizeof(float2) * K2 * IP_CB_STRIDE + 15) / 16 * 16;
  }
  static __host__ __device__ constexpr size_t bytes(int nrow) {
    return hist(nrow) + (BIN == 2 ? sizeof(uint32_t) * IP_HIST_MAX : 0);
  }
  static constexpr size_t bytes_max = bytes(nrow_max);
};

// One level-1 cell: gather the 3x3 block's lenses, re-centre the series on the
// sub-cells, then every ray of rows [jlo, jhi) of the cell.  In DUMP mode the
// thread holding ray (want_i, want_j) writes its beta and pixel to slot `work`.
//
// Each thread takes one lattice column and R rows; rows go in pairs through
// the packed FP32x2 instructions (two rows share the column's dx and sigma_x),
// which round exactly as the scalar ones.  The accumulators hold -alpha (the
// masses are stored negated) and the level-2 Horner runs on the conjugate, so
// no negation is issued per ray.
template <int MODE, int R, int Q, int K2, int BIN, int NPR>
__device__ __forceinline__ void ip_cell(const Geo& g, const IpGeo& ig, const IpRayArgs& a, int64_t rc,
                                        int64_t want_i, int64_t want_j, int64_t work) {
  static_assert(R % 2 == 0, "rows go in pairs");
  static_assert(NPR >= 0 && NPR <= R / 2, "paired row pairs");
  using L = IpSmem<Q, K2, BIN>;
  extern __shared__ __align__(16) unsigned char ip_smem[];
  float4* nxy_s = reinterpret_cast<float4*>(ip_smem + L::near_xy);
  float2* nm_s = reinterpret_cast<float2*>(ip_smem + L::near_m);
  float4* sub_s = reinterpret_cast<float4*>(ip_smem + L::sub);
  IpRowPair* row_s = reinterpret_cast<IpRowPair*>(ip_smem + L::row_sg);
  float2* cb_s = reinterpret_cast<float2*>(ip_smem + L::coef(ig.nrow));
  uint32_t* hist_s = reinterpret_cast<uint32_t*>(ip_smem + L::hist(ig.nrow));
  __shared__ CellRec rec_s;
  __shared__ int blk_start[9], blk_off[10];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t k = ig.k;
  // Every FP32 step of the cell's ray geometry below is written with explicit
  // rounding (__fadd_rn, __fmul_rn, __fdiv_rn, fmaf): implicit contraction
  // would depend on how the compiler places the code in each kernel that
  // inlines this function, and the single-map and batched ray passes must
  // give the same maps bit for bit.
  const float hf = ig.hf;
  const float inv_k = ig.inv_k;

  const int rcx = (int)(rc % ig.nrcx), rcy = (int)(rc / ig.nrcx);
  const int cx = rcx + ig.ox, cy = rcy + ig.oy;
  const int64_t i0 = (int64_t)rcx * k, j0 = (int64_t)rcy * k;
  const int64_t i1 = min(i0 + k, g.nrx);
  int64_t jlo = j0, jhi = min(j0 + k, g.nry);
  if (MODE == IP_MAP) {
    jlo = max(jlo, a.row0);
    jhi = min(jhi, a.row1);
    if (jlo >= jhi) return;  // uniform over the CTA
  }
  __syncthreads();  // previous cell's shared data no longer read
  if (warp == 0) {
    // lane q < 9 takes cell q of the 3x3 block (row-major from the lower
    // left); the block's lens offsets are the exclusive prefix sum of the counts
    int s0 = 0, cnt = 0;
    if (lane < 9) {
      const int x = cx + (lane % 3) - 1, y = cy + (lane / 3) - 1;
      if (x >= 0 && x < ig.ncx && y >= 0 && y < ig.ncy) {
        const int64_t s = (int64_t)y * ig.ncx + x;
        s0 = a.start[s];
        cnt = a.start[s + 1] - s0;
      }
    }
    int inc = cnt;
#pragma unroll
    for (int d = 1; d < 16; d <<= 1) {
      const int v = __shfl_up_sync(0xFFFFFFFFu, inc, d);
      if (lane >= d) inc += v;
    }
    if (lane < 9) {
      blk_start[lane] = s0;
      blk_off[lane] = inc - cnt;
    }
    if (lane == 8) {
      int off = inc;
      if (off > IP_NEAR_MAX) {
        atomicCAS(a.status, 0, (int)IRS_ERR_OVERFLOW);  // the first error stays
        off = IP_NEAR_MAX;
      }
      blk_off[9] = off;
    }
  } else if (warp == 1 && lane < (int)(sizeof(CellRec) / 4)) {
    reinterpret_cast<uint32_t*>(&rec_s)[lane] = reinterpret_cast<const uint32_t*>(a.recs + rc)[lane];
  }
  // Level 2 re-centres the cell series sum_kk c_kk w^kk (w in cell units,
  // terms from 1: term 0 sits in the cell's base) on the sub-cell centres
  // eps: with w = eps + sigma / Q the coefficient of sigma^n is
  // Q^-n sum_kk binom(kk, n) c_kk eps^(kk - n).  First the per-cell table
  // cb[n][kk] = Q^-n binom(kk, n) c_kk (binomials exact in FP32 for kk < 32).
  const float inv_q = __fdiv_rn(1.0f, (float)Q);
  for (int t = tid; t < K2 * ig.K; t += blockDim.x) {
    const int nn = t / ig.K, kk = t % ig.K;
    float2 v = make_float2(0.f, 0.f);
    if (kk >= nn && kk >= 1) {
      int b = 1;  // binom(kk, nn), exact integer steps
      for (int i = 1; i <= nn; ++i) b = b * (kk - nn + i) / i;
      float sc = (float)b;
      for (int i = 0; i < nn; ++i) sc = __fmul_rn(sc, inv_q);
      const float2 c = a.coef[rc * ig.K + kk];
      v = make_float2(__fmul_rn(c.x, sc), __fmul_rn(c.y, sc));
    }
    cb_s[nn * IP_CB_STRIDE + kk] = v;
  }
  __syncthreads();
  const int n_near = blk_off[9];
  for (int t = tid; t < n_near; t += blockDim.x) {
    int q = 0;
    while (q < 8 && t >= blk_off[q + 1]) ++q;
    const float4 v = a.rel[blk_start[q] + (t - blk_off[q])];
    const float ox = __fmul_rn((float)((q % 3) - 1), hf), oy = __fmul_rn((float)((q / 3) - 1), hf);
    const float x = __fadd_rn(v.x, ox), y = __fadd_rn(v.y, oy);
    nxy_s[t] = make_float4(-x, -x, -y, -y);
    nm_s[t] = make_float2(-v.z, -v.z);
  }
  // then per (sub-cell, n) the polynomial sum_j cb[n][n + j] eps^j by Horner,
  // two sub-cells of one sub-cell row at a time (Q is even) through packed
  // FP32x2 instructions: the same roundings as two scalar Horner chains
  static_assert(Q % 2 == 0, "sub-cells go in pairs along a row");
  for (int t = tid; t < Q * Q * K2 / 2; t += blockDim.x) {
    const int sp = t / K2, nn = t % K2;
    const int sa = 2 * sp;  // sub-cells sa, sa + 1: same row, adjacent columns
    const float er_a = __fmaf_rn(__fadd_rn((float)(sa % Q), 0.5f), inv_q, -0.5f);
    const float er_b = __fmaf_rn(__fadd_rn((float)(sa % Q + 1), 0.5f), inv_q, -0.5f);
    const float ei = __fmaf_rn(__fadd_rn((float)(sa / Q), 0.5f), inv_q, -0.5f);
    const float2 ER = make_float2(er_a, er_b), EI = make_float2(ei, ei), NEI = make_float2(-ei, -ei);
    const float2* cb = cb_s + nn * IP_CB_STRIDE;
    float2 SR = make_float2(0.f, 0.f), SI = make_float2(0.f, 0.f);
#pragma unroll 2
    for (int kk = ig.K - 1; kk >= nn; --kk) {
      const float2 c = cb[kk];
      const float2 NR = __ffma2_rn(SR, ER, __ffma2_rn(SI, NEI, make_float2(c.x, c.x)));
      SI = __ffma2_rn(SR, EI, __ffma2_rn(SI, ER, make_float2(c.y, c.y)));
      SR = NR;
    }
    sub_s[sa * K2 + nn] = make_float4(SR.x, SR.x, -SI.x, -SI.x);
    sub_s[(sa + 1) * K2 + nn] = make_float4(SR.y, SR.y, -SI.y, -SI.y);
  }
  // row table: t_y = tau_y h, sigma_y = (l + 1/2) Q / k - v - 1/2, v Q, rows of
  // the whole cell side in pairs and R / 2 pairs past it (rows past the cell
  // side are never binned; their sub-cell row is clamped to Q - 1)
  static_assert(R <= 2 * IP_ROW_PAD, "row table padding");
  const int npair_cell = (int)((k + 1) >> 1) + R / 2;
  for (int pr = tid; pr < npair_cell; pr += blockDim.x) {
    float tyv[2], sg[2], y0[2];
    int vq[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int l = 2 * pr + j;
      const float sv = __fmul_rn(__fadd_rn((float)l, 0.5f), __fmul_rn((float)Q, inv_k));
      const int v = min(__float2int_rd(sv), Q - 1);
      tyv[j] = __fmul_rn(fmaf((float)l, inv_k, fmaf(0.5f, inv_k, -0.5f)), hf);
      y0[j] = __fmaf_rn(g.lam_s2, tyv[j], rec_s.by_lo);
      sg[j] = __fsub_rn(__fsub_rn(sv, (float)v), 0.5f);
      vq[j] = v * Q;
    }
    row_s[pr].sg = make_float4(sg[0], sg[1], -sg[0], -sg[1]);
    row_s[pr].ty = make_float4(tyv[0], tyv[1], y0[0], y0[1]);
    row_s[pr].v = make_int2(vq[0], vq[1]);
  }
  // privatised binning: the cell's pixel box [hx0, hx0 + hbx) x [hy0, hy0 + hby)
  // around the centre's pixel offset (relative to the base pixel; no box when
  // it exceeds the sub-histogram) and its bins cleared; lhx, lhy turn a ray's
  // floor bit pattern into its box column and row
  int32_t hx0 = 0, hy0 = 0, hbx = 0, hby = 0;
  uint32_t lhx = 0, lhy = 0;
  if (BIN == 2 && MODE == IP_MAP) {
    const float cx_pix = __fmul_rn(rec_s.bx_hi, g.inv_sx), cy_pix = __fmul_rn(rec_s.by_hi, g.inv_sy);
    hx0 = __float2int_rd(__fsub_rn(cx_pix, ig.box_hx));
    hy0 = __float2int_rd(__fsub_rn(cy_pix, ig.box_hy));
    hbx = __float2int_rd(__fadd_rn(cx_pix, ig.box_hx)) - hx0 + 1;
    hby = __float2int_rd(__fadd_rn(cy_pix, ig.box_hy)) - hy0 + 1;
    if (hbx * hby > IP_HIST_MAX) hbx = hby = 0;
    lhx = (uint32_t)0u - PIX_MAGIC_BITS - (uint32_t)hx0;
    lhy = (uint32_t)0u - PIX_MAGIC_BITS - (uint32_t)hy0;
    for (int t = tid; t < hbx * hby; t += blockDim.x) hist_s[t] = 0u;
  }
  __syncthreads();

  // base pixel of this cell for the 32-bit pixel test, folded with the
  // floor's bit pattern offset (pixel_keys2)
  const int32_t rix = rec_s.ix, riy = rec_s.iy;
  const uint32_t rbx = (uint32_t)rix - PIX_MAGIC_BITS, rby = (uint32_t)riy - PIX_MAGIC_BITS;
  // the cell centre's beta (hi parts) in pixel units
  const float bxs = __fmul_rn(rec_s.bx_hi, g.inv_sx), bys = __fmul_rn(rec_s.by_hi, g.inv_sy);

  const int n_corner = rec_s.n_corner;
  const unsigned lane_lt = (1u << lane) - 1u;
  // cell-local 32-bit lattice indices: columns [0, kx), rows [ylo, yhi); units
  // start on an even row so that row pairs line up with the table
  const int kx = (int)(i1 - i0), ylo = (int)(jlo - j0), yhi = (int)(jhi - j0);
  const int ylo2 = ylo & ~1;
  const float c_tau = fmaf(0.5f, inv_k, -0.5f);  // tau = (l + 1/2)/k - 1/2
  const float qk = __fmul_rn((float)Q, inv_k);   // sub-cell index = floor((l + 1/2) Q / k)
  const float fnan = __int_as_float(0x7fffffff);
  // work units (32-column strip x R-row group), dealt round-robin to warps
  const int nwarps = blockDim.x / 32;
  const int nstrip = (kx + 31) / 32;
  const int nrg = (yhi - ylo2 + R - 1) / R;
  const int nunit = nstrip * nrg;
  // (strip, row group) of the warp's first unit, then stepped by nwarps units
  // at a time: no integer division per unit
  int st = warp % nstrip, rg = warp / nstrip;
  for (int unit = warp; unit < nunit; unit += nwarps, step_unit(st, rg, nwarps, nstrip)) {
    const int cl = st * 32 + lane;
    const int rl0 = ylo2 + rg * R;
    const int p0 = rl0 >> 1;
    const float su = __fmul_rn(__fadd_rn((float)cl, 0.5f), qk);
    const int u = min(__float2int_rd(su), Q - 1);
    const float sgr = __fsub_rn(__fsub_rn(su, (float)u), 0.5f);
    // rays outside the cell's columns get a NaN x, rays outside its rows a NaN
    // y accumulator: both reach beta whatever the near sum does and fail the
    // pixel test
    const float tx = cl < kx ? __fmul_rn(fmaf((float)cl, inv_k, c_tau), hf) : fnan;
    const float x0 = __fmaf_rn(g.lam_s1, tx, rec_s.bx_lo);  // the column's share of beta_1
    const float2 TX = make_float2(tx, tx), SGR = make_float2(sgr, sgr), X0 = make_float2(x0, x0);
    float2 TY[R / 2], NAX[R / 2], NAY[R / 2];
#pragma unroll
    for (int i = 0; i < R / 2; ++i) {
      const float4 t = row_s[p0 + i].ty;
      TY[i] = make_float2(t.x, t.y);
      NAX[i] = make_float2(0.f, 0.f);
      NAY[i] = make_float2(0.f, 0.f);
    }
    if (rl0 < ylo || rl0 + R > yhi) {  // a group at the band's edge (uniform over the warp)
#pragma unroll
      for (int i = 0; i < R / 2; ++i) {
        const int ra = rl0 + 2 * i;
        NAY[i] = make_float2(ra >= ylo && ra < yhi ? 0.f : fnan, ra + 1 < yhi ? 0.f : fnan);
      }
    }
#pragma unroll 2
    for (int q = 0; q < n_near; ++q) {
      const float4 Lq = nxy_s[q];
      const float2 NM = nm_s[q];
      const float2 DX = __fadd2_rn(TX, make_float2(Lq.x, Lq.y));
      const float2 DX2 = __fmul2_rn(DX, DX);
      const float2 NLY = make_float2(Lq.z, Lq.w);
#pragma unroll
      for (int i = 0; i < R / 2; ++i) {
        const float2 DY = __fadd2_rn(TY[i], NLY);
        const float2 R2 = __ffma2_rn(DY, DY, DX2);
        float2 W;
        if (i < NPR) {  // -m/r_a^2 = -m r_b^2 / (r_a^2 r_b^2), and the same for b
          const float mi = NM.x * rcp_approx(R2.x * R2.y);
          W = __fmul2_rn(make_float2(R2.y, R2.x), make_float2(mi, mi));
        } else {
          W = __fmul2_rn(NM, make_float2(rcp_approx(R2.x), rcp_approx(R2.y)));
        }
        NAX[i] = __ffma2_rn(W, DX, NAX[i]);
        NAY[i] = __ffma2_rn(W, DY, NAY[i]);
      }
    }
    // tail in groups of HP row pairs: level-2 series (conj, in sigma), sheet
    // corners, beta and pixel keys, binning; the chains of a group interleave
    constexpr int HP = R / 2 < 2 ? R / 2 : 2;
#pragma unroll
    for (int h = 0; h < R / 2; h += HP) {
      float2 QR[HP], QI[HP];
      {
        float4 SG[HP];  // (sigma_y, -sigma_y) of the pair
        int va[HP];
        bool aligned = true;  // no pair straddles a sub-cell row: uniform over the warp
#pragma unroll
        for (int i = 0; i < HP; ++i) {
          SG[i] = row_s[p0 + h + i].sg;
          const int2 v = row_s[p0 + h + i].v;
          va[i] = (v.x + u) * K2;
          aligned = aligned && (v.x == v.y);
        }
        if (aligned) {
#pragma unroll
          for (int i = 0; i < HP; ++i) {
            const float4 dl = sub_s[va[i] + K2 - 1];
            QR[i] = make_float2(dl.x, dl.y);
            QI[i] = make_float2(dl.z, dl.w);
          }
#pragma unroll
          for (int nn = K2 - 2; nn >= 0; --nn) {
#pragma unroll
            for (int i = 0; i < HP; ++i) {
              const float4 dn = sub_s[va[i] + nn];
              const float2 sgi = make_float2(SG[i].x, SG[i].y), nsgi = make_float2(SG[i].z, SG[i].w);
              const float2 t1 = __ffma2_rn(QI[i], sgi, make_float2(dn.x, dn.y));
              const float2 t2 = __ffma2_rn(QI[i], SGR, make_float2(dn.z, dn.w));
              const float2 nr = __ffma2_rn(QR[i], SGR, t1);
              QI[i] = __ffma2_rn(QR[i], nsgi, t2);
              QR[i] = nr;
            }
          }
        } else {
          int vb[HP];
#pragma unroll
          for (int i = 0; i < HP; ++i) vb[i] = (row_s[p0 + h + i].v.y + u) * K2;
#pragma unroll
          for (int i = 0; i < HP; ++i) {
            const float4 ea = sub_s[va[i] + K2 - 1], eb = sub_s[vb[i] + K2 - 1];
            QR[i] = make_float2(ea.x, eb.x);
            QI[i] = make_float2(ea.z, eb.z);
          }
#pragma unroll
          for (int nn = K2 - 2; nn >= 0; --nn) {
#pragma unroll
            for (int i = 0; i < HP; ++i) {
              const float4 ea = sub_s[va[i] + nn], eb = sub_s[vb[i] + nn];
              const float2 sgi = make_float2(SG[i].x, SG[i].y), nsgi = make_float2(SG[i].z, SG[i].w);
              const float2 t1 = __ffma2_rn(QI[i], sgi, make_float2(ea.x, eb.x));
              const float2 t2 = __ffma2_rn(QI[i], SGR, make_float2(ea.z, eb.z));
              const float2 nr = __ffma2_rn(QR[i], SGR, t1);
              QI[i] = __ffma2_rn(QR[i], nsgi, t2);
              QR[i] = nr;
            }
          }
        }
      }
      if (n_corner) {  // corners of the sheet near this cell, per ray (uniform over the CTA)
#pragma unroll
        for (int i = 0; i < HP; ++i) {
          float qr[2] = {QR[i].x, QR[i].y}, qi[2] = {QI[i].x, QI[i].y};
          const float4 t = row_s[p0 + h + i].ty;
          const float tyr[2] = {t.x, t.y};
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            for (int c = 0; c < n_corner; ++c) {
              const float wr = __fadd_rn(rec_s.corner[c][0], tx), wi = __fadd_rn(rec_s.corner[c][1], tyr[j]);
              const float lr = __fmul_rn(0.5f, logf(fmaf(wr, wr, __fmul_rn(wi, wi)))), li = atan2f(wi, wr);
              const float plr = fmaf(wr, lr, -__fmul_rn(wi, li)), pli = fmaf(wr, li, __fmul_rn(wi, lr));
              qr[j] = fmaf(rec_s.corner[c][2], pli, qr[j]);
              qi[j] = fmaf(rec_s.corner[c][2], plr, qi[j]);
            }
          }
          QR[i] = make_float2(qr[0], qr[1]);
          QI[i] = make_float2(qi[0], qi[1]);
        }
      }
      // beta relative to the base pixel, (by_hi, by_hi) + ((x0, y0) + L_local -
      // alpha_near), in pixel units, then the pixel key of every ray (~0
      // where none)
      uint32_t key[2 * HP], lkey[2 * HP];
#pragma unroll
      for (int i = 0; i < HP; ++i) {
        const float4 t = row_s[p0 + h + i].ty;
        const float2 y0 = make_float2(t.z, t.w);
        const float2 SX = __fadd2_rn(X0, __fadd2_rn(NAX[h + i], QR[i]));
        const float2 SY = __fadd2_rn(y0, __fadd2_rn(NAY[h + i], QI[i]));
        const float2 T1 = __ffma2_rn(SX, make_float2(g.inv_sx, g.inv_sx), make_float2(bxs, bxs));
        const float2 T2 = __ffma2_rn(SY, make_float2(g.inv_sy, g.inv_sy), make_float2(bys, bys));
        if (BIN == 2 && MODE == IP_MAP)
          pixel_keys2_box(T1, T2, rbx, rby, (uint32_t)g.npix_x, (uint32_t)g.npix_y, lhx, lhy, (uint32_t)hbx,
                          (uint32_t)hby, key[2 * i], key[2 * i + 1], lkey[2 * i], lkey[2 * i + 1]);
        else
          pixel_keys2(T1, T2, rbx, rby, (uint32_t)g.npix_x, (uint32_t)g.npix_y, key[2 * i], key[2 * i + 1]);
        if (MODE == IP_DUMP) {
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            if (i0 + cl == want_i && j0 + rl0 + 2 * (h + i) + j == want_j) {
              const double b1 = (double)rec_s.bx_hi + (double)(j ? SX.y : SX.x);
              const double b2 = (double)rec_s.by_hi + (double)(j ? SY.y : SY.x);
              a.beta_out[2 * work] = (g.src_x0 + (double)rix * g.sx) + b1;
              a.beta_out[2 * work + 1] = (g.src_y0 + (double)riy * g.sy) + b2;
              if (a.pix_out) a.pix_out[work] = key[2 * i + j] != 0xFFFFFFFFu ? (int64_t)key[2 * i + j] : -1;
            }
          }
        }
      }
      if (MODE == IP_MAP) {
#pragma unroll
        if (BIN == 3) {
#pragma unroll
          for (int i = 0; i < HP; ++i) bin_warp_pair(a.counts, key[2 * i], key[2 * i + 1], lane_lt);
        } else {
#pragma unroll
          for (int r = 0; r < 2 * HP; ++r) {
            if (BIN == 2) bin_warp_key_box(a.counts, hist_s, key[r], lkey[r], lane_lt);
            else if (BIN == 1) bin_warp_runs_key(a.counts, key[r], lane);
            else bin_warp_key(a.counts, key[r], lane_lt);
          }
        }
      }
    }
  }
  if (BIN == 2 && MODE == IP_MAP && hbx > 0) {
    // flush the cell's sub-histogram: one global add per non-empty bin (bins
    // off the map never receive a ray: only on-map keys reach the box)
    __syncthreads();
    for (int t = tid; t < hbx * hby; t += blockDim.x) {
      const uint32_t v = hist_s[t];
      if (v) {
        const int by = t / hbx, bx = t - by * hbx;
        atomicAdd(a.counts + (int64_t)(riy + hy0 + by) * g.npix_x + (rix + hx0 + bx), v);
      }
    }
  }
}

// One map: persistent grid over its ray cells (MAP) or requested rays (DUMP).
template <int MODE, int R, int Q, int K2, int MINB, int BIN, int NPR>
__global__ void __launch_bounds__(IP_THREADS, MINB) k_ip_ray(Geo g, IpGeo ig, IpRayArgs a) {
  for (int64_t work = blockIdx.x; work < a.nwork; work += gridDim.x) {
    if (MODE == IP_MAP) {
      ip_cell<IP_MAP, R, Q, K2, BIN, NPR>(g, ig, a, a.rc_base + work, -1, -1, work);
    } else {
      const int64_t f = a.idx[work];
      if (f < 0 || f >= g.nrx * g.nry) {  // not a lattice ray: report it, touch nothing else
        if (threadIdx.x == 0) {
          a.beta_out[2 * work] = a.beta_out[2 * work + 1] = nan("");
          if (a.pix_out) a.pix_out[work] = -1;
        }
        continue;
      }
      const int64_t wi = f % g.nrx, wj = f / g.nrx;
      ip_cell<IP_DUMP, R, Q, K2, BIN, NPR>(g, ig, a, (wj / ig.k) * ig.nrcx + wi / ig.k, wi, wj, work);
    }
  }
}

// Many maps: one persistent launch; CTAs pull (map, cell) items from a global
// counter, so maps of any size and cost share the GPU without a tail per map.
struct MapDesc {
  Geo g;
  IpGeo ig;
  IpRayArgs a;
  int64_t item0;  // index of the map's first item in the concatenated list
};

template <int R, int Q, int K2, int MINB, int BIN, int NPR>
__global__ void __launch_bounds__(IP_THREADS, MINB)
k_ip_ray_batch(const MapDesc* __restrict__ maps, int nmaps, int64_t nitems,
               unsigned long long* __restrict__ queue) {
  __shared__ MapDesc md;
  __shared__ long long item_s;
  __shared__ int map_s;
  if (threadIdx.x == 0) map_s = -1;
  for (;;) {
    __syncthreads();  // everyone is done with md / item_s
    if (threadIdx.x == 0) {
      const long long it = (long long)atomicAdd(queue, 1ull);
      item_s = it;
      if (it < nitems) {
        int lo = 0, hi = nmaps - 1;  // last map with item0 <= it
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (maps[mid].item0 <= it) lo = mid; else hi = mid - 1;
        }
        if (lo != map_s) {  // items of one map are contiguous: copy on change only
          md = maps[lo];
          map_s = lo;
        }
      }
    }
    __syncthreads();
    const long long it = item_s;
    if (it >= nitems) break;
    ip_cell<IP_MAP, R, Q, K2, BIN, NPR>(md.g, md.ig, md.a, md.a.rc_base + (it - md.item0), -1, -1, it);
  }
}

// Dynamic shared memory above the 48 KB default: set once per instantiation,
// before any launch or graph capture that uses it.
#define IP_DECL_ATTR(V, R, Q, K2, MINB, BIN, NPR)                                                           \
  case V: {                                                                                            \
    const int b = (int)IpSmem<Q, K2, BIN>::bytes_max;                                                      \
    e = cudaFuncSetAttribute(k_ip_ray<IP_MAP, R, Q, K2, MINB, BIN, NPR>,                                   \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, b);                         \
    if (e == cudaSuccess)                                                                              \
      e = cudaFuncSetAttribute(k_ip_ray<IP_DUMP, R, Q, K2, MINB, BIN, NPR>,                                \
                               cudaFuncAttributeMaxDynamicSharedMemorySize, b);                       \
    if (e == cudaSuccess)                                                                              \
      e = cudaFuncSetAttribute(k_ip_ray_batch<R, Q, K2, MINB, BIN, NPR>,                                   \
                               cudaFuncAttributeMaxDynamicSharedMemorySize, b);                       \
    break;                                                                                             \
  }
cudaError_t ip_ray_attributes(int variant) {
  cudaError_t e = cudaErrorInvalidValue;
  switch (variant) { IP_VARIANTS(IP_DECL_ATTR) default: break; }
  return e;
}

#define IP_DECL_OCC(V, R, Q, K2, MINB, BIN, NPR)                                                       \
  case V:                                                                                         \
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ip_ray<IP_MAP, R, Q, K2, MINB, BIN, NPR>, \
                                                  IP_THREADS, IpSmem<Q, K2, BIN>::bytes(nrow));        \
    break;
// CTAs per SM of a variant whose row table has `nrow` entries
int ip_ray_occupancy(int variant, int nrow) {
  int per_sm = 0;
  switch (variant) { IP_VARIANTS(IP_DECL_OCC) default: break; }
  return per_sm > 0 ? per_sm : 1;
}

#define IP_DECL_BYTES(V, R, Q, K2, MINB, BIN, NPR) \
  case V:                                          \
    return IpSmem<Q, K2, BIN>::bytes(nrow);
size_t ip_ray_smem(int variant, int nrow) {
  switch (variant) { IP_VARIANTS(IP_DECL_BYTES) default: break; }
  return 0;
}

#define IP_DECL_LAUNCH(V, R, Q, K2, MINB, BIN, NPR)                                                           \
  case V:                                                                                                \
    if (mode == IP_MAP)                                                                                  \
      k_ip_ray<IP_MAP, R, Q, K2, MINB, BIN, NPR><<<(unsigned)grid, IP_THREADS, IpSmem<Q, K2, BIN>::bytes(ig.nrow), \
                                                   s>>>(g, ig, a);                                           \
    else                                                                                                 \
      k_ip_ray<IP_DUMP, R, Q, K2, MINB, BIN, NPR><<<(unsigned)grid, IP_THREADS, IpSmem<Q, K2, BIN>::bytes(ig.nrow), \
                                                    s>>>(g,                                                  \
                                                                                                 ig, a); \
    break;
cudaError_t launch_ip_ray(int variant, int mode, int64_t grid, cudaStream_t s, const Geo& g,
                          const IpGeo& ig, const IpRayArgs& a) {
  switch (variant) { IP_VARIANTS(IP_DECL_LAUNCH) default: return cudaErrorInvalidValue; }
  return cudaGetLastError();
}

#define IP_DECL_BATCH(V, R, Q, K2, MINB, BIN, NPR)                                                       \
  case V:                                                                                           \
    k_ip_ray_batch<R, Q, K2, MINB, BIN, NPR><<<(unsigned)grid, IP_THREADS, IpSmem<Q, K2, BIN>::bytes(nrow), s>>>( \
        maps, nmaps, nitems, queue);                                                                \
    break;
cudaError_t launch_ip_ray_batch(int variant, int64_t grid, cudaStream_t s, const MapDesc* maps,
                                int nmaps, int64_t nitems, unsigned long long* queue, int nrow) {
  switch (variant) { IP_VARIANTS(IP_DECL_BATCH) default: return cudaErrorInvalidValue; }
  return cudaGetLastError();
}

// ------------------------------------------------------------ host helpers
irs_status alloc_lens_buffers(irs_plan_t* P, InterpState* S, int64_t cap) {
  ++P->ws_gen;  // the lens buffers move: graphs captured on the old ones are stale
  if (S->lens_ws) cudaFree(S->lens_ws);
  S->lens_ws = nullptr;
  cap = cap < 256 ? 256 : cap;
  size_t off = 0;
  auto take = [&](size_t b) {
    size_t o = off;
    off += (b + 255) & ~(size_t)255;
    return o;
  };
  const size_t o_cell = take(sizeof(int32_t) * cap), o_sidx = take(sizeof(int32_t) * cap);
  const size_t o_rel = take(sizeof(float4) * cap), o_pos = take(sizeof(double2) * cap);
  const size_t o_m = take(sizeof(double) * cap);
  const size_t o_pdf = take(sizeof(float4) * cap), o_mdf = take(sizeof(float2) * cap);
  if (cudaMalloc(&S->lens_ws, off) != cudaSuccess) {
    cudaGetLastError();
    S->lens_ws = nullptr;
    S->cap = 0;
    return IRS_ERR_OOM;
  }
  char* b = static_cast<char*>(S->lens_ws);
  S->lens_cell = reinterpret_cast<int32_t*>(b + o_cell);
  S->sorted_idx = reinterpret_cast<int32_t*>(b + o_sidx);
  S->lens_rel = reinterpret_cast<float4*>(b + o_rel);
  S->lens_pos = reinterpret_cast<double2*>(b + o_pos);
  S->lens_m = reinterpret_cast<double*>(b + o_m);
  S->lens_pdf = reinterpret_cast<float4*>(b + o_pdf);
  S->lens_mdf = reinterpret_cast<float2*>(b + o_mdf);
  S->lens_ws_bytes = off;
  S->cap = cap;
  return IRS_OK;
}

void mark(irs_plan_t* P, int slot, cudaStream_t s) {
  if (P->timing) cudaEventRecord(P->ev[slot], s);
}

#define IP_TRY(expr)                                                     \
  do {                                                                   \
    cudaError_t e_ = (expr);                                             \
    if (e_ != cudaSuccess) return e_ == cudaErrorMemoryAllocation ? IRS_ERR_OOM : IRS_ERR_CUDA; \
  } while (0)

// kernel launches of one map, reported through irs_plan_timings
int far_launches(int64_t n) { return (n > 0 ? 4 : 0) + 3 + 1 + 2 + 1 + 2 + 1; }  // series mode

// Cell lists and far field; the per-cell finalize covers ray cells
// [rc0, rc1) only (rc1 < 0: all of them).
irs_status build_cells_and_far(irs_plan_t* P, const double* xy, const double* mass, int64_t n,
                               cudaStream_t s, int64_t rc0 = 0, int64_t rc1 = -1) {
  InterpState* S = S_(P);
  const IpGeo& ig = S->ig;
  const int64_t ncells = (int64_t)ig.ncx * ig.ncy;
  if (n > S->cap) {
    cudaStreamSynchronize(s);
    irs_status st = alloc_lens_buffers(P, S, n + n / 4);
    if (st != IRS_OK) return st;
  }
  const double2* xy2 = reinterpret_cast<const double2*>(xy);
  IP_TRY(cudaMemsetAsync(S->cell_count, 0, sizeof(int32_t) * ncells, s));
  if (n > 0) k_ip_count<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(ig, xy2, n, S->lens_cell, S->cell_count);
  const int64_t nb = (ncells + SCAN_B - 1) / SCAN_B;
  k_scan_local<<<(unsigned)nb, SCAN_B, 0, s>>>(S->cell_count, S->cell_start, ncells, S->scan_blocks);
  k_scan_blocks<<<1, 32, 0, s>>>(S->scan_blocks, nb, S->cell_start + ncells);
  k_scan_add<<<(unsigned)nb, SCAN_B, 0, s>>>(S->cell_start, ncells, S->scan_blocks);
  IP_TRY(cudaGetLastError());
  if (n > 0) {
    IP_TRY(cudaMemcpyAsync(S->cell_cursor, S->cell_start, sizeof(int32_t) * ncells,
                           cudaMemcpyDeviceToDevice, s));
    k_ip_scatter<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(S->lens_cell, n, S->cell_cursor, S->sorted_idx);
    k_ip_sortcells<<<(unsigned)((ncells + 255) / 256), 256, 0, s>>>(S->cell_start, ncells, S->sorted_idx);
    k_ip_fill<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(ig, xy2, mass, S->sorted_idx, S->lens_cell, n,
                                                         S->lens_rel, S->lens_pos, S->lens_m, S->lens_pdf,
                                                         S->lens_mdf);
  }
  IP_TRY(cudaGetLastError());
  mark(P, EV_CELLS, s);
  // far field: the network (trained IRS_MLP plans) or the FFT series
  MlpFar far{};
  if (P->p.method == IRS_MLP && mlp_trained(P)) {
    irs_status st = mlp_prepare(P, xy, mass, n, ig.gx0, ig.gy0, ig.h, ig.nrcx, ig.nrcy, ig.ox, ig.oy, &far, s);
    if (st != IRS_OK) return st;
  } else {
    k_ip_p2m<<<(unsigned)((ncells + 127) / 128), 128, 0, s>>>(ig, S->cell_start, S->lens_pos, S->lens_m,
                                                             S->mpole_d, S->mpole_f);
    IP_TRY(cudaGetLastError());
    IP_TRY(fft2d_forward(S->mpole_d, ig.ncx, ig.ncy, ncells, S->spec_d, S->fft, IP_PD, s));
    IP_TRY(fft2d_forward(S->mpole_f, ig.ncx, ig.ncy, ncells, S->spec_f, S->fft, IP_P - IP_PD, s));
    const int64_t G = (int64_t)S->fft.Nx * S->fft.Ny;
    k_ip_m2l_freq<<<(unsigned)((G + 127) / 128), 128, 0, s>>>(G, S->spec_d, S->spec_f, S->kspec_d, S->kspec_f);
    IP_TRY(cudaGetLastError());
    IP_TRY(fft2d_inverse(S->spec_d, S->fft, ig.ncx, ig.ncy, S->conv_d, ncells, IP_KD, s));
    IP_TRY(fft2d_inverse(S->spec_f, S->fft, ig.ncx, ig.ncy, S->conv_f, ncells, IP_KF - IP_KD, s));
  }
  const int64_t nrc = (int64_t)ig.nrcx * ig.nrcy;
  if (rc1 < 0 || rc1 > nrc) rc1 = nrc;
  mark(P, EV_FIN, s);
  if (rc1 > rc0) {
    // the default K = 24 needs 21 FP32 terms; larger K the full FIN_K32
    const unsigned nb = (unsigned)((rc1 - rc0 + 63) / 64);
    if (ig.K - FIN_K64 <= 21)
      k_ip_finalize<21><<<nb, 64, 0, s>>>(P->g, ig, P->d_msum, S->cell_start, S->lens_pos, S->lens_m,
                                          S->lens_pdf, S->lens_mdf, S->conv_d, S->conv_f, far, S->sheet_d,
                                          S->sheet_f, S->sheet_near, S->recs, S->coef, rc0, rc1);
    else
      k_ip_finalize<FIN_K32><<<nb, 64, 0, s>>>(P->g, ig, P->d_msum, S->cell_start, S->lens_pos, S->lens_m,
                                               S->lens_pdf, S->lens_mdf, S->conv_d, S->conv_f, far,
                                               S->sheet_d, S->sheet_f, S->sheet_near, S->recs, S->coef, rc0,
                                               rc1);
  }
  IP_TRY(cudaGetLastError());
  mark(P, EV_FAR, s);
  return IRS_OK;
}

IpRayArgs ray_args(irs_plan_t* P) {
  InterpState* S = S_(P);
  IpRayArgs a{};
  a.start = S->cell_start;
  a.rel = S->lens_rel;
  a.recs = S->recs;
  a.coef = S->coef;
  a.status = P->d_status;
  return a;
}

}  // namespace

// ------------------------------------------------------------ entry points
irs_status interp_plan(irs_plan_t* P) {
  InterpState* S = new (std::nothrow) InterpState();
  if (!S) return IRS_ERR_OOM;
  memset(S, 0, sizeof(*S));
  P->interp = S;
  IpGeo& ig = S->ig;
  const irs_params& p = P->p;
  const Geo& g = P->g;
  const double Ix = P->ix, Iy = P->iy;
  int64_t nstar = p.n_star > 0 ? p.n_star : P->n_star_suggested;
  if (nstar < 1) nstar = 1;
  // level-1 resolution, flow chart: Delta x1 = min(L0, min(I_x, I_y)/10)
  const double L0 = sqrt(Ix * Iy / (double)nstar);
  const double dx1_rule = fmin(L0, fmin(Ix, Iy) / 10.0);
  S->rule_rays = dx1_rule / g.dx3;
  double dx1 = dx1_rule * (p.cell_mult > 0 ? p.cell_mult : 1.0);
  int64_t k = (int64_t)ceil(dx1 / g.dx3 - 1e-9);
  if (k < 4) k = 4;
  if (k > IP_KMAX_RAYS) k = IP_KMAX_RAYS;  // the ray pass keeps a row table per cell
  ig.k = k;
  ig.nrow = (int32_t)((k + 1) / 2) + IP_ROW_PAD;
  ig.h = (double)k * g.dx3;
  // a cell of side h maps to |1 - kappa -+ gamma| h under the mean lens map
  // (declared kappa_*); half of that in pixels, grown by half for the far
  // field's and the near lenses' spread, plus two pixels
  ig.box_hx = (float)(0.75 * fabs(P->lambda1) * ig.h / g.sx + 2.0);
  ig.box_hy = (float)(0.75 * fabs(P->lambda2) * ig.h / g.sy + 2.0);
  ig.hf = (float)ig.h;
  ig.inv_k = 1.0f / (float)k;
  ig.nrcx = (int32_t)((g.nrx + k - 1) / k);
  ig.nrcy = (int32_t)((g.nry + k - 1) / k);
  // lens region: the rectangle, or the circumscribed circle's bounding box
  int64_t ox = 0, oy = 0, ex = 0, ey = 0;
  if (p.plane == IRS_PLANE_CIRCLE) {
    const double R = P->circle_r;
    ox = (int64_t)ceil((g.a1 - (g.cx - R)) / ig.h);
    oy = (int64_t)ceil((g.b1 - (g.cy - R)) / ig.h);
    ex = (int64_t)ceil(((g.cx + R) - (g.a1 + ig.nrcx * ig.h)) / ig.h);
    ey = (int64_t)ceil(((g.cy + R) - (g.b1 + ig.nrcy * ig.h)) / ig.h);
    ox = ox < 0 ? 0 : ox;
    oy = oy < 0 ? 0 : oy;
    ex = ex < 0 ? 0 : ex;
    ey = ey < 0 ? 0 : ey;
  }
  // the ray pass's pixel keys (pixel_keys2) need every ray that lands to be
  // within 2^22 pixels of its cell's base pixel: maps below 2^21 pixels per
  // side and protective borders below 2^20 pixels
  if (g.npix_x >= (1 << 21) || g.npix_y >= (1 << 21) || P->border >= 1048576.0 * fmin(g.sx, g.sy))
    return IRS_ERR_OVERFLOW;
  const int64_t ncx = ox + ig.nrcx + ex, ncy = oy + ig.nrcy + ey;
  if (ncx > FFT_MAX_LEN / 2 || ncy > FFT_MAX_LEN / 2) return IRS_ERR_OVERFLOW;
  ig.ncx = (int32_t)ncx;
  ig.ncy = (int32_t)ncy;
  ig.ox = (int32_t)ox;
  ig.oy = (int32_t)oy;
  ig.gx0 = g.a1 - (double)ox * ig.h;
  ig.gy0 = g.b1 - (double)oy * ig.h;
  ig.K = p.far_order > 0 ? p.far_order : DEFAULT_K;
  // `window` is the direct window of the series form; an IRS_MLP plan reads it
  // as the learned split's radius R_f instead (its untrained fallback keeps
  // the default window)
  ig.W = (p.window > 0 && p.method != IRS_MLP) ? p.window : DEFAULT_W;
  ig.P = IP_P;
  if (ig.K > IP_KMAX || ig.K < 8) return IRS_ERR_ARG;
  ig.variant = p.kernel_variant;
  if (ig.variant < 0 || ig.variant >= IP_NVARIANT) return IRS_ERR_ARG;
  if (ig.W < 1) ig.W = 1;

  Fft2d& f = S->fft;
  // padded lengths >= 2n - 1 (linear convolution), of the form 2^a 3^b
  f.Nx = fft_good_size(2 * ncx - 1, &f.n3x, &f.n2x);
  f.Ny = fft_good_size(2 * ncy - 1, &f.n3y, &f.n2y);
  if (f.Nx < 0 || f.Ny < 0) return IRS_ERR_OVERFLOW;
  if (fft_setup_attributes() != cudaSuccess) return IRS_ERR_CUDA;
  if (fft_twiddles(f.Nx, &f.tw_x) != cudaSuccess) return IRS_ERR_OOM;
  if (fft_twiddles(f.Ny, &f.tw_y) != cudaSuccess) return IRS_ERR_OOM;

  const int64_t ncells = ncx * ncy, nrc = (int64_t)ig.nrcx * ig.nrcy;
  const int64_t G = (int64_t)f.Nx * f.Ny;
  size_t off = 0;
  auto take = [&](size_t b) {
    size_t o = off;
    off += (b + 255) & ~(size_t)255;
    return o;
  };
  const size_t o_cnt = take(sizeof(int32_t) * ncells), o_start = take(sizeof(int32_t) * (ncells + 1));
  const size_t o_cur = take(sizeof(int32_t) * ncells);
  const size_t o_sb = take(sizeof(int32_t) * ((ncells + SCAN_B - 1) / SCAN_B + 1));
  static_assert(IP_KD <= IP_PD && IP_KF - IP_KD <= IP_P - IP_PD, "local spectra overwrite multipole spectra");
  const size_t o_mpd = take(sizeof(float4) * IP_PD * ncells), o_mpf = take(sizeof(float2) * (IP_P - IP_PD) * ncells);
  const size_t o_cvd = take(sizeof(float4) * IP_KD * ncells), o_cvf = take(sizeof(float2) * (IP_KF - IP_KD) * ncells);
  const size_t o_spd = take(sizeof(float4) * IP_PD * G), o_spf = take(sizeof(float2) * (IP_P - IP_PD) * G);
  const size_t o_ksd = take(sizeof(float4) * IP_NKD * G), o_ksf = take(sizeof(float2) * (IP_P + IP_KF - 1) * G);
  const size_t o_rec = take(sizeof(CellRec) * nrc), o_coef = take(sizeof(float2) * ig.K * nrc);
  const bool rect = p.plane == IRS_PLANE_RECT;
  const size_t o_shd = take(rect ? sizeof(double2) * FIN_K64 * nrc : 0);
  const size_t o_shf = take(rect ? sizeof(float2) * (ig.K - FIN_K64) * nrc : 0);
  const size_t o_shn = take(rect ? sizeof(uint8_t) * nrc : 0);
  if (cudaMalloc(&S->ws, off) != cudaSuccess) {
    cudaGetLastError();
    S->ws = nullptr;
    return IRS_ERR_OOM;
  }
  S->ws_bytes = off;
  char* b = static_cast<char*>(S->ws);
  S->cell_count = reinterpret_cast<int32_t*>(b + o_cnt);
  S->cell_start = reinterpret_cast<int32_t*>(b + o_start);
  S->cell_cursor = reinterpret_cast<int32_t*>(b + o_cur);
  S->scan_blocks = reinterpret_cast<int32_t*>(b + o_sb);
  S->mpole_d = reinterpret_cast<float4*>(b + o_mpd);
  S->mpole_f = reinterpret_cast<float2*>(b + o_mpf);
  S->conv_d = reinterpret_cast<float4*>(b + o_cvd);
  S->conv_f = reinterpret_cast<float2*>(b + o_cvf);
  S->spec_d = reinterpret_cast<float4*>(b + o_spd);
  S->spec_f = reinterpret_cast<float2*>(b + o_spf);
  S->kspec_d = reinterpret_cast<float4*>(b + o_ksd);
  S->kspec_f = reinterpret_cast<float2*>(b + o_ksf);
  S->recs = reinterpret_cast<CellRec*>(b + o_rec);
  S->coef = reinterpret_cast<float2*>(b + o_coef);
  S->sheet_d = rect ? reinterpret_cast<double2*>(b + o_shd) : nullptr;
  S->sheet_f = rect ? reinterpret_cast<float2*>(b + o_shf) : nullptr;
  S->sheet_near = rect ? reinterpret_cast<uint8_t*>(b + o_shn) : nullptr;
  irs_status st = alloc_lens_buffers(P, S, nstar + nstar / 4 + 256);
  if (st != IRS_OK) return st;
  // translation kernels and their spectra, once per plan
  const int nker = ig.P + IP_KF - 1;
  k_ip_kernel_grid<<<(unsigned)((G + 255) / 256), 256>>>(f.Nx, f.Ny, ig.W, nker, IP_NKD, S->kspec_d, S->kspec_f);
  if (cudaGetLastError() != cudaSuccess) return IRS_ERR_CUDA;
  if (fft2d_forward(S->kspec_d, f.Nx, f.Ny, G, S->kspec_d, f, IP_NKD, 0) != cudaSuccess) return IRS_ERR_CUDA;
  if (fft2d_forward(S->kspec_f, f.Nx, f.Ny, G, S->kspec_f, f, nker, 0) != cudaSuccess) return IRS_ERR_CUDA;
  if (rect && nrc > 0) {  // the sheet's corner series, once per plan
    k_ip_sheet_table<<<(unsigned)((nrc + 127) / 128), 128>>>(g, ig, S->sheet_d, S->sheet_f, S->sheet_near, nrc);
    if (cudaGetLastError() != cudaSuccess) return IRS_ERR_CUDA;
  }
  if (cudaDeviceSynchronize() != cudaSuccess) return IRS_ERR_CUDA;
  if (ip_ray_attributes(ig.variant) != cudaSuccess) return IRS_ERR_CUDA;
  S->grid_ray = P->num_sms * ip_ray_occupancy(ig.variant, ig.nrow);
  if (p.method == IRS_MLP) {
    if (p.plane != IRS_PLANE_RECT) return IRS_ERR_UNSUPPORTED;
    irs_status st2 = mlp_plan(P, ig.gx0, ig.gy0, ig.h, ig.ncx, ig.ncy, ig.nrcx, ig.nrcy, ig.ox, ig.oy, 1 << 20);
    if (st2 != IRS_OK) return st2;
  }
  return IRS_OK;
}

double interp_cell_side(const irs_plan_t* P) { return S_(P) ? S_(P)->ig.h : 0.0; }
double interp_rule_rays(const irs_plan_t* P) { return S_(P) ? S_(P)->rule_rays : 0.0; }

void interp_fill_info(const irs_plan_t* P, irs_plan_info* info) {
  const InterpState* S = S_(P);
  if (!S) return;
  info->cell_x = info->cell_y = S->ig.h;
  info->ncell_x = S->ig.ncx;
  info->ncell_y = S->ig.ncy;
  info->rays_per_cell_x = info->rays_per_cell_y = (int32_t)S->ig.k;
  info->far_order = S->ig.K;
  info->window = S->ig.W;
}

int64_t interp_workspace_bytes(const irs_plan_t* P) {
  const InterpState* S = S_(P);
  return S ? (int64_t)(S->ws_bytes + S->lens_ws_bytes) : 0;
}

irs_status interp_run(irs_plan_t* P, const double* xy, const double* mass, int64_t n, int64_t row0,
                      int64_t row1, uint32_t* counts, cudaStream_t s) {
  InterpState* S = S_(P);
  mark(P, EV_PREP, s);
  // only the cell rows the band touches need their series
  const int64_t k = S->ig.k;
  const int64_t rc0 = row1 > row0 ? (row0 / k) * S->ig.nrcx : 0;
  const int64_t rc1 = row1 > row0 ? ((row1 + k - 1) / k) * S->ig.nrcx : 0;
  irs_status st = build_cells_and_far(P, xy, mass, n, s, rc0, rc1);
  if (st != IRS_OK) return st;
  mark(P, EV_RAY0, s);
  P->launches += far_launches(n) - (rc1 > rc0 ? 0 : 1) + (row1 > row0 ? 1 : 0);
  if (row1 > row0) {
    IpRayArgs a = ray_args(P);
    a.counts = counts;
    a.row0 = row0;
    a.row1 = row1;
    a.rc_base = rc0;
    a.nwork = rc1 - rc0;
    const int64_t grid = (rc1 - rc0) < S->grid_ray ? (rc1 - rc0) : S->grid_ray;
    if (launch_ip_ray(S->ig.variant, IP_MAP, grid, s, P->g, S->ig, a) != cudaSuccess) return IRS_ERR_CUDA;
  }
  mark(P, EV_RAY1, s);
  return IRS_OK;
}

irs_status interp_set_variant(irs_plan_t* P, int variant) {
  InterpState* S = S_(P);
  if (!S || variant < 0 || variant >= IP_NVARIANT) return IRS_ERR_ARG;
  if (ip_ray_attributes(variant) != cudaSuccess) return IRS_ERR_CUDA;
  S->ig.variant = variant;
  P->p.kernel_variant = variant;
  S->grid_ray = P->num_sms * ip_ray_occupancy(variant, S->ig.nrow);
  return IRS_OK;
}

irs_status interp_raypass_rows(irs_plan_t* P, int64_t row0, int64_t row1, uint32_t* counts, cudaStream_t s,
                               cudaEvent_t e0, cudaEvent_t e1) {
  InterpState* S = S_(P);
  if (!S || row0 < 0 || row1 <= row0 || row1 > P->g.nry) return IRS_ERR_ARG;
  const int64_t k = S->ig.k;
  const int64_t rc0 = (row0 / k) * S->ig.nrcx, rc1 = ((row1 + k - 1) / k) * S->ig.nrcx;
  IpRayArgs a = ray_args(P);
  a.counts = counts;
  a.row0 = row0;
  a.row1 = row1;
  a.rc_base = rc0;
  a.nwork = rc1 - rc0;
  const int64_t grid = (rc1 - rc0) < S->grid_ray ? (rc1 - rc0) : S->grid_ray;
  if (cudaEventRecord(e0, s) != cudaSuccess) return IRS_ERR_CUDA;
  if (launch_ip_ray(S->ig.variant, IP_MAP, grid, s, P->g, S->ig, a) != cudaSuccess) return IRS_ERR_CUDA;
  if (cudaEventRecord(e1, s) != cudaSuccess) return IRS_ERR_CUDA;
  return IRS_OK;
}

irs_status interp_shoot_rays(irs_plan_t* P, const double* xy, const double* mass, int64_t n,
                             const int64_t* idx, int64_t nidx, double* beta, int64_t* pix,
                             cudaStream_t s) {
  InterpState* S = S_(P);
  irs_status st = build_cells_and_far(P, xy, mass, n, s);
  if (st != IRS_OK) return st;
  IpRayArgs a = ray_args(P);
  a.idx = idx;
  a.beta_out = beta;
  a.pix_out = pix;
  a.nwork = nidx;
  const int64_t grid = nidx < S->grid_ray ? nidx : S->grid_ray;
  return launch_ip_ray(S->ig.variant, IP_DUMP, grid, s, P->g, S->ig, a) == cudaSuccess ? IRS_OK
                                                                                     : IRS_ERR_CUDA;
}

irs_status interp_ensure_capacity(irs_plan_t* P, int64_t n) {
  InterpState* S = S_(P);
  if (n <= S->cap) return IRS_OK;
  if (cudaDeviceSynchronize() != cudaSuccess) return IRS_ERR_CUDA;
  return alloc_lens_buffers(P, S, n + n / 4);
}

irs_status interp_prepare(irs_plan_t* P, const double* xy, const double* mass, int64_t n,
                          cudaStream_t s) {
  return build_cells_and_far(P, xy, mass, n, s);
}

int interp_variant(const irs_plan_t* P) { return S_(P)->ig.variant; }
int interp_row_entries(const irs_plan_t* P) { return S_(P)->ig.nrow; }
int interp_num_variants() { return IP_NVARIANT; }

size_t interp_desc_bytes(int nmaps) { return sizeof(MapDesc) * (size_t)(nmaps > 0 ? nmaps : 1); }

int64_t interp_fill_descs(irs_plan_t* const* plans, uint32_t* const* counts, int nmaps, void* host) {
  MapDesc* d = static_cast<MapDesc*>(host);
  int64_t items = 0;
  for (int k = 0; k < nmaps; ++k) {
    InterpState* S = S_(plans[k]);
    memset(&d[k], 0, sizeof(MapDesc));
    d[k].g = plans[k]->g;
    d[k].ig = S->ig;
    d[k].a = ray_args(plans[k]);
    d[k].a.counts = counts[k];
    d[k].a.row0 = 0;
    d[k].a.row1 = plans[k]->g.nry;
    d[k].a.rc_base = 0;
    d[k].a.nwork = (int64_t)S->ig.nrcx * S->ig.nrcy;
    d[k].item0 = items;
    items += d[k].a.nwork;
  }
  return items;
}

irs_status interp_batch_launch(int variant, const void* dev_descs, int nmaps, int64_t nitems,
                               unsigned long long* queue, int num_sms, int nrow, cudaStream_t s) {
  if (nmaps <= 0 || nitems <= 0) return IRS_OK;
  int64_t grid = (int64_t)num_sms * ip_ray_occupancy(variant, nrow);
  if (grid > nitems) grid = nitems;
  if (cudaMemsetAsync(queue, 0, sizeof(unsigned long long), s) != cudaSuccess) return IRS_ERR_CUDA;
  return launch_ip_ray_batch(variant, grid, s, static_cast<const MapDesc*>(dev_descs), nmaps, nitems,
                             queue, nrow) == cudaSuccess
             ? IRS_OK
             : IRS_ERR_CUDA;
}

void interp_destroy(irs_plan_t* P) {
  mlp_destroy(P);
  InterpState* S = S_(P);
  if (!S) return;
  if (S->ws) cudaFree(S->ws);
  if (S->lens_ws) cudaFree(S->lens_ws);
  if (S->fft.tw_x) cudaFree(S->fft.tw_x);
  if (S->fft.tw_y) cudaFree(S->fft.tw_y);
  delete S;
  P->interp = nullptr;
}

}  // namespace irs
