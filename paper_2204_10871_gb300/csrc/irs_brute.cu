// irs_brute.cu -- plain ("ordinary GPU IRS") ray pass: every ray sums every
// lens (arXiv:2204.10871, Sec. 1 and the "ordinary GPU-based IRS code" of
// Sec. 3.1), with the rectangular negative sheet of Eq. (alpha1) / Appendix A.
//
// Layout of the work: the ray lattice is cut into tiles of 32 x 64 rays.  A
// CTA of 64/R warps owns one tile at a time (persistent grid); lane l takes
// column i0 + l and each warp R consecutive rows (R = 16 in the default
// variant), so a thread carries R rays that share their x offset.  Lenses stream through shared memory 256 at a
// time as FP32 positions relative to the tile centre (converted from the
// caller's FP64 once per tile and stage) and are broadcast to all warps.
//
// Precision plan: per pair FP32 with rcp.approx on the SFU (one reciprocal
// per ray, or one per two or four rows of a column through products of
// their squared distances); each 256-lens
// stage is summed in FP32 and folded into a TwoSum (hi, lo) accumulator; the
// sheet, the smooth terms and the pixel base of the tile centre are FP64 in
// the setup kernel and reach the rays as double-float constants plus an
// FP32 Taylor series of the sheet's analytic part in the ray's offset t.
#include <math.h>

#include "irs_common.cuh"

namespace irs {

// ------------------------------------------------------------ mass sum (FP64)
// Deterministic two-pass sum of the masses: fixed strides per thread, fixed
// reduction tree, fixed order of the block partials.  With lens positions
// given, the same pass checks that every lens lies in the plan's lens region
// (the rectangle that is both image and lens plane, Sec. 2.2, or the
// circumscribed circle), with a margin of 1e-9 of the plane's extent for
// positions drawn on its edges: a lens outside it (or a NaN position) sets
// IRS_ERR_ARG in the plan's status word unless an earlier error is there.
struct LensRegion {
  double x0, x1, y0, y1;  // rectangle, margin included
  double cx, cy, r2;      // circle: centre and squared radius, margin included
  int32_t circle;
  int32_t check;          // 0: positions not given, no check
};

__device__ __forceinline__ bool lens_inside(const LensRegion& L, double2 p) {
  if (L.circle) {
    const double dx = p.x - L.cx, dy = p.y - L.cy;
    return dx * dx + dy * dy <= L.r2;  // false for NaN
  }
  return p.x >= L.x0 && p.x <= L.x1 && p.y >= L.y0 && p.y <= L.y1;
}

__global__ void k_mass_partial(const double* __restrict__ mass, const double2* __restrict__ xy, int64_t n,
                               LensRegion region, int* __restrict__ status, double* __restrict__ part) {
  __shared__ double sh[MSUM_THREADS];
  double s = 0.0;
  bool outside = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
    s += mass[k];
    if (region.check) outside |= !lens_inside(region, xy[k]);
  }
  if (__syncthreads_or(outside) && threadIdx.x == 0) atomicCAS(status, 0, (int)IRS_ERR_ARG);
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = MSUM_THREADS / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_mass_final(const double* __restrict__ part, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < MSUM_BLOCKS; ++b) s += part[b];
    out[0] = s;
  }
}

cudaError_t launch_mass_sum(const irs_plan_t* P, const double* mass, int64_t n, cudaStream_t s,
                            const double* xy) {
  LensRegion L{};
  const Geo& g = P->g;
  const double ext = fmax(fmax(fabs(g.a1), fabs(g.a2)), fmax(fmax(fabs(g.b1), fabs(g.b2)),
                                                             fmax(g.a2 - g.a1, g.b2 - g.b1)));
  const double tol = 1e-9 * ext;
  L.x0 = g.a1 - tol;
  L.x1 = g.a2 + tol;
  L.y0 = g.b1 - tol;
  L.y1 = g.b2 + tol;
  L.cx = g.cx;
  L.cy = g.cy;
  L.r2 = (P->circle_r + tol) * (P->circle_r + tol);
  L.circle = g.plane == IRS_PLANE_CIRCLE;
  L.check = xy != nullptr && n > 0;
  k_mass_partial<<<MSUM_BLOCKS, MSUM_THREADS, 0, s>>>(mass, reinterpret_cast<const double2*>(xy), n, L,
                                                      P->d_status, P->d_mpart);
  k_mass_final<<<1, 32, 0, s>>>(P->d_mpart, P->d_msum);
  return cudaGetLastError();
}

// ------------------------------------------------------------ FP64 complex
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
// principal Log
__device__ __forceinline__ cd clog_p(cd a) {
  return {0.5 * log(a.re * a.re + a.im * a.im), atan2(a.im, a.re)};
}

// ------------------------------------------------------------ tile setup
// Analytic part of the positive rectangle sheet (complex form derived from the
// appendix integrals): inside the rectangle,
//   conj(alpha_sheet)(z) = kappa_* conj(z) + g(z),
//   g(z) = kappa_* (z - 2 a2) + sum_c phi_c(z),
//   phi_c(z) = -i a_c (z - c) Log(z - c),   a_c = (kappa_*/pi) s_c,
// with corner signs s = +1 at (a1,b1) and (a2,b2), -1 at (a2,b1) and (a1,b2).
// Derivatives: phi_c' = -i a_c (Log(z-c) + 1),
//              phi_c^(n) = -i a_c (-1)^n (n-2)! / (z-c)^(n-1)  (n >= 2).
// Corners closer than 6 tile half-diagonals are left out of the series and
// evaluated per ray instead (the series would converge slowly there).
__global__ void k_brute_setup(Geo g, const double* __restrict__ msum, int64_t ntx, int64_t ntiles,
                              TileRec* __restrict__ recs) {
  const int64_t tile = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tile >= ntiles) return;
  const TileGeo tg = tile_geo(g, tile, ntx);
  const double ks = g.kstar_scale * msum[0];  // kappa_*^act = pi sum(m) / A of the lenses passed in
  const double kap = g.kappa_s + ks;
  const double zx = g.a1 + tg.ci * g.dx3, zy = g.b1 + tg.cj * g.dx3;

  // base pixel from the mean lens map of the tile centre
  const double m1 = (1.0 - kap - g.gamma) * zx, m2 = (1.0 - kap + g.gamma) * zy;
  double fx = floor((m1 - g.src_x0) / g.sx), fy = floor((m2 - g.src_y0) / g.sy);
  fx = fmin(fmax(fx, -1.0e9), 1.0e9);
  fy = fmin(fmax(fy, -1.0e9), 1.0e9);
  const double base_x = g.src_x0 + fx * g.sx, base_y = g.src_y0 + fy * g.sy;

  TileRec r;
  r.ix = (int32_t)fx;
  r.iy = (int32_t)fy;
  r.n_near = 0;
  r.pad_ = 0;
  for (int k = 0; k < SHEET_TERMS; ++k) r.T[k][0] = r.T[k][1] = 0.f;
  for (int k = 0; k < MAX_NEAR; ++k) r.near[k][0] = r.near[k][1] = r.near[k][2] = r.near[k][3] = 0.f;

  double cre, cim;  // conj(beta) of the centre without the lens sum
  if (g.plane == IRS_PLANE_CIRCLE) {
    // Eq. (alpha) + k_* theta_c:  conj(beta) = (1-k_s) conj(z) - g z - k_* conj(z_c) - L
    cre = (1.0 - g.kappa_s - g.gamma) * zx - ks * g.cx;
    cim = -(1.0 - g.kappa_s + g.gamma) * zy + ks * g.cy;
  } else {
    // Eq. (alpha1): conj(beta) = (1-k) conj(z) - g z - L + conj(alpha_sheet,+)
    cd T0 = {ks * (2.0 * zx - 2.0 * g.a2), 0.0};  // kappa_* (conj z + z - 2 a2)
    cd T[SHEET_TERMS];
    for (int k = 0; k < SHEET_TERMS; ++k) T[k] = {0.0, 0.0};
    T[0].re = ks;  // derivative of kappa_* (z - 2 a2)
    const double half_diag = 0.5 * g.dx3 * hypot((double)(tg.i1 - tg.i0), (double)(tg.j1 - tg.j0));
    const double rho = 6.0 * fmax(half_diag, g.dx3);
    const double cxs[4] = {g.a1, g.a2, g.a1, g.a2};
    const double cys[4] = {g.b1, g.b1, g.b2, g.b2};
    const double sgn[4] = {1.0, -1.0, -1.0, 1.0};
    for (int c = 0; c < 4; ++c) {
      const double ac = ks / M_PI * sgn[c];
      const cd w = {zx - cxs[c], zy - cys[c]};
      if (ac == 0.0) continue;
      if (hypot(w.re, w.im) < rho && r.n_near < MAX_NEAR) {
        r.near[r.n_near][0] = (float)w.re;
        r.near[r.n_near][1] = (float)w.im;
        r.near[r.n_near][2] = (float)ac;
        r.n_near++;
        continue;
      }
      cd L = clog_p(w);
      // branch continuous with the rectangle's interior (tile centres are
      // inside it, so this only guards the two right-hand corners' cuts)
      if (c == 3 && w.re < 0.0 && w.im > 0.0) L.im -= 2.0 * M_PI;
      if (c == 1 && w.re < 0.0 && w.im < 0.0) L.im += 2.0 * M_PI;
      const cd wl = cmul(w, L);
      T0.re += ac * wl.im;  // -i a_c (w L)
      T0.im -= ac * wl.re;
      T[0].re += ac * L.im;  // -i a_c (L + 1)
      T[0].im -= ac * (L.re + 1.0);
      const cd inv = crecip(w);
      cd pw = inv;
      for (int n = 2; n <= SHEET_TERMS; ++n) {
        const double coef = ((n & 1) ? -1.0 : 1.0) / (double)(n * (n - 1));
        T[n - 1].re += ac * coef * pw.im;
        T[n - 1].im -= ac * coef * pw.re;
        pw = cmul(pw, inv);
      }
    }
    cre = (1.0 - kap - g.gamma) * zx + T0.re;
    cim = -(1.0 - kap + g.gamma) * zy + T0.im;
    for (int k = 0; k < SHEET_TERMS; ++k) {
      r.T[k][0] = (float)T[k].re;
      r.T[k][1] = (float)T[k].im;
    }
  }
  split_df(cre - base_x, r.cx_hi, r.cx_lo);
  split_df(-cim - base_y, r.cy_hi, r.cy_lo);
  recs[tile] = r;
}

cudaError_t launch_brute_setup(const irs_plan_t* P, cudaStream_t s) {
  const int64_t nt = P->br_ntiles;
  const int threads = 128;
  const int64_t blocks = (nt + threads - 1) / threads;
  k_brute_setup<<<(unsigned)blocks, threads, 0, s>>>(P->g, P->d_msum, P->br_ntx, nt, P->d_tiles);
  return cudaGetLastError();
}

// ------------------------------------------------------------ ray pass
enum { MODE_MAP = 0, MODE_DUMP = 1 };

// Variants: R rows per thread (the tile stays 32 x 64: 64/R warps per CTA),
// PAIRED rows per thread that share one reciprocal per two rows, QUAD groups
// of four packed rows that share one reciprocal per four rows, and PACK: the
// other rows go two at a time through the packed FP32x2 instructions (the two
// rows share dx and dx^2; fewer issue slots, the same FP32-pipe work).  The
// TwoSum accumulators live in shared memory (updated once per 256-lens stage).
// TPSM: resident threads per SM the register budget is sized for.
//
// Balance of the pair sum per lens and warp (32 lanes x R rows): the MUFU
// unit takes 8 cycles per warp-wide reciprocal, the FP32 pipe 1 cycle per
// scalar and 2 per packed instruction.  An unshared packed row pair costs 5
// packed instructions (10 FP32 cycles) and 2 reciprocals (16 MUFU cycles); a
// quad, two row pairs, 12 packed and 2 scalar instructions (26 FP32 cycles)
// and 1 reciprocal (8 MUFU cycles):
//   variant 11 (2 paired rows x 2, 6 packed pairs): MUFU 112, FP32  88 cycles
//   variant 0 (1 quad, 6 packed pairs):             MUFU 104, FP32  90 cycles
//   variant 10 (2 quads, 4 packed pairs):           MUFU  80, FP32  96 cycles
// bounding the pair sum at 71, 77 and 83 % of the FP32 peak.  Measured on
// the 1e5-lens band (one GB300, 2070 MHz): 59.7 % (variant 11), 62.3 %
// (variant 0, the default), 60.6 % (variant 10): with two quads the FP32
// pipe's longer dependent chains cost more than the MUFU cycles they save.
#define BR_VARIANTS(X)                                                                         \
  X(0, 16, 0, 1, 1, 512) X(1, 16, 8, 0, 0, 512) X(2, 8, 4, 0, 0, 512) X(3, 8, 2, 0, 0, 512)      \
  X(4, 16, 4, 0, 0, 512) X(5, 16, 2, 0, 0, 512) X(6, 16, 8, 0, 1, 512) X(7, 16, 6, 0, 1, 512)     \
  X(8, 16, 2, 0, 1, 512) X(9, 16, 4, 0, 1, 640) X(10, 16, 0, 2, 1, 512) X(11, 16, 4, 0, 1, 512)  \
  X(12, 16, 0, 3, 1, 512) X(13, 8, 0, 1, 1, 512) X(14, 16, 2, 1, 1, 512) X(15, 16, 4, 1, 1, 512)
constexpr int BR_NVARIANT = 16;

// Plane diagonal (theta_E) up to which the four-row products of squared
// distances stay inside the FP32 range with a wide margin ((1e4)^8 = 1e32).
constexpr double BR_QUAD_MAX_DIAG = 1.0e4;

template <int MODE, int R, int PAIRED, int QUAD, int PACK, int TPSM>
__global__ void __launch_bounds__(32 * (BR_TY / R), TPSM / (32 * (BR_TY / R)))
k_brute(Geo g, const double2* __restrict__ xy, const double* __restrict__ mass, int64_t n,
        const TileRec* __restrict__ recs, int64_t ntx, int64_t nwork, int64_t row0, int64_t row1,
        uint32_t* __restrict__ counts, const int64_t* __restrict__ idx,
        double* __restrict__ beta_out, int64_t* __restrict__ pix_out) {
  constexpr int NT = 32 * (BR_TY / R);
  static_assert(PAIRED % 2 == 0 && (!PACK || (R - PAIRED) % 2 == 0), "rows go in pairs");
  static_assert(QUAD == 0 || PACK, "quads are packed");
  static_assert(PAIRED + 4 * QUAD <= R, "rows");
  // packed row pairs after the PAIRED scalar rows: the first 2 QUAD of them
  // form the quads
  constexpr int NPK = PACK ? (R - PAIRED) / 2 : 0;
  // lens records: (x, y, m, 0) for the scalar form; with PACK, (-x, -x, -y, -y)
  // and (m, m) -- the duplicates feed the packed instructions and the scalar
  // rows read one half (t + (-x) == t - x)
  __shared__ float4 lens_s[BR_LT];
  __shared__ float2 lensm_s[PACK ? BR_LT : 1];
  __shared__ float acc_s[4][R][NT];  // x hi, x lo, y hi, y lo
  __shared__ TileRec rec;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  for (int64_t work = blockIdx.x; work < nwork; work += gridDim.x) {
    int64_t tile, want_i = -1, want_j = -1;
    if (MODE == MODE_MAP) {
      tile = (row0 / BR_TY) * ntx + work;  // tile rows covering [row0, row1)
    } else {
      const int64_t f = idx[work];
      if (f < 0 || f >= g.nrx * g.nry) {  // not a lattice ray: report it, touch nothing else
        if (tid == 0) {
          beta_out[2 * work] = beta_out[2 * work + 1] = nan("");
          if (pix_out) pix_out[work] = -1;
        }
        continue;
      }
      want_i = f % g.nrx;
      want_j = f / g.nrx;
      tile = (want_j / BR_TY) * ntx + want_i / BR_TX;
    }
    const TileGeo tg = tile_geo(g, tile, ntx);
    const double zx = g.a1 + tg.ci * g.dx3, zy = g.b1 + tg.cj * g.dx3;
    const int64_t col = tg.i0 + lane;
    const float tx = (float)(((double)col + 0.5 - tg.ci) * g.dx3);
    const float2 TX2 = make_float2(tx, tx);
    float ty[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      ty[r] = (float)(((double)(tg.j0 + warp * R + r) + 0.5 - tg.cj) * g.dx3);
      acc_s[0][r][tid] = acc_s[1][r][tid] = acc_s[2][r][tid] = acc_s[3][r][tid] = 0.f;
    }
    float2 TYP[NPK > 0 ? NPK : 1];
#pragma unroll
    for (int q = 0; q < NPK; ++q) TYP[q] = make_float2(ty[PAIRED + 2 * q], ty[PAIRED + 2 * q + 1]);

    __syncthreads();  // previous tile's readers of rec / lens_s are done
    if (tid == 0) rec = recs[tile];

    for (int64_t base = 0; base < n; base += BR_LT) {
      float4 v[BR_LT / NT];
#pragma unroll
      for (int q = 0; q < BR_LT / NT; ++q) {
        const int64_t k = base + q * NT + tid;
        // padding: massless, and far enough that it is never on a ray, near
        // enough that products of four squared distances stay finite (a
        // product overflowing to inf would turn 0 x inf into NaN)
        v[q] = make_float4(4096.f, 4096.f, 0.f, 0.f);
        if (k < n) {
          const double2 p = xy[k];
          v[q] = make_float4((float)(p.x - zx), (float)(p.y - zy), (float)mass[k], 0.f);
        }
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < BR_LT / NT; ++q) {
        if (PACK) {
          lens_s[q * NT + tid] = make_float4(-v[q].x, -v[q].x, -v[q].y, -v[q].y);
          lensm_s[q * NT + tid] = make_float2(v[q].z, v[q].z);
        } else {
          lens_s[q * NT + tid] = v[q];
        }
      }
      __syncthreads();
      float pax[R], pay[R];
      float2 PAX[NPK > 0 ? NPK : 1], PAY[NPK > 0 ? NPK : 1];
#pragma unroll
      for (int r = 0; r < R; ++r) pax[r] = pay[r] = 0.f;
#pragma unroll
      for (int q = 0; q < NPK; ++q) PAX[q] = PAY[q] = make_float2(0.f, 0.f);
      // lenses in this stage, rounded up to the unroll (padding is massless)
      const int cnt = (int)min((int64_t)BR_LT, ((n - base) + 7) & ~(int64_t)7);
#pragma unroll 2
      for (int jl = 0; jl < cnt; ++jl) {
        float4 L = lens_s[jl];
        float2 M, DX, DX2;
        float dx, dx2;
        if (PACK) {
          M = lensm_s[jl];
          DX = __fadd2_rn(TX2, make_float2(L.x, L.y));
          DX2 = __fmul2_rn(DX, DX);
          dx = DX.x;
          dx2 = DX2.x;
        } else {  // scalar layout: (x, y, m, 0) -> the same quantities
          M = make_float2(L.z, L.z);
          dx = tx - L.x;
          dx2 = dx * dx;
          L.z = -L.y;
        }
        // rows 0..PAIRED-1: one reciprocal for two rows, 1/(r_a^2 r_b^2), to move
        // work from the SFU (MUFU) to the FP32 pipe; remaining rows: one each
#pragma unroll
        for (int r = 0; r < PAIRED; r += 2) {
          const float dya = ty[r] + L.z, dyb = ty[r + 1] + L.z;
          const float r2a = fmaf(dya, dya, dx2), r2b = fmaf(dyb, dyb, dx2);
          const float mR = M.x * rcp_approx(r2a * r2b);
          const float wa = r2b * mR, wb = r2a * mR;
          pax[r] = fmaf(wa, dx, pax[r]);
          pay[r] = fmaf(wa, dya, pay[r]);
          pax[r + 1] = fmaf(wb, dx, pax[r + 1]);
          pay[r + 1] = fmaf(wb, dyb, pay[r + 1]);
        }
        // quads: rows (a, b) and (c, d) as two packed pairs sharing one
        // reciprocal of r_a^2 r_b^2 r_c^2 r_d^2; with P = (r_a^2 r_c^2, r_b^2 r_d^2)
        // and Q = m/(r_a^2 r_b^2 r_c^2 r_d^2) (P.y, P.x), m/r^2 of (a, b) is
        // Q (r_c^2, r_d^2) and of (c, d) is Q (r_a^2, r_b^2)
#pragma unroll
        for (int g4 = 0; g4 < QUAD; ++g4) {
          const float2 DYa = __fadd2_rn(TYP[2 * g4], make_float2(L.z, L.w));
          const float2 DYc = __fadd2_rn(TYP[2 * g4 + 1], make_float2(L.z, L.w));
          const float2 R2a = __ffma2_rn(DYa, DYa, DX2), R2c = __ffma2_rn(DYc, DYc, DX2);
          const float2 P4 = __fmul2_rn(R2a, R2c);
          const float mR = M.x * rcp_approx(P4.x * P4.y);
          const float2 Q4 = __fmul2_rn(make_float2(mR, mR), make_float2(P4.y, P4.x));
          const float2 Wa = __fmul2_rn(Q4, R2c), Wc = __fmul2_rn(Q4, R2a);
          PAX[2 * g4] = __ffma2_rn(Wa, DX, PAX[2 * g4]);
          PAY[2 * g4] = __ffma2_rn(Wa, DYa, PAY[2 * g4]);
          PAX[2 * g4 + 1] = __ffma2_rn(Wc, DX, PAX[2 * g4 + 1]);
          PAY[2 * g4 + 1] = __ffma2_rn(Wc, DYc, PAY[2 * g4 + 1]);
        }
        if (PACK) {
#pragma unroll
          for (int q = 2 * QUAD; q < NPK; ++q) {
            const float2 DY = __fadd2_rn(TYP[q], make_float2(L.z, L.w));
            const float2 R2 = __ffma2_rn(DY, DY, DX2);
            const float2 W = __fmul2_rn(M, make_float2(rcp_approx(R2.x), rcp_approx(R2.y)));
            PAX[q] = __ffma2_rn(W, DX, PAX[q]);
            PAY[q] = __ffma2_rn(W, DY, PAY[q]);
          }
        } else {
#pragma unroll
          for (int r = PAIRED; r < R; ++r) {
            const float dy = ty[r] + L.z;
            const float r2 = fmaf(dy, dy, dx2);
            const float w = M.x * rcp_approx(r2);
            pax[r] = fmaf(w, dx, pax[r]);
            pay[r] = fmaf(w, dy, pay[r]);
          }
        }
      }
      if (PACK) {
#pragma unroll
        for (int q = 0; q < NPK; ++q) {
          pax[PAIRED + 2 * q] = PAX[q].x;
          pax[PAIRED + 2 * q + 1] = PAX[q].y;
          pay[PAIRED + 2 * q] = PAY[q].x;
          pay[PAIRED + 2 * q + 1] = PAY[q].y;
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        float s, e;
        two_sum(acc_s[0][r][tid], pax[r], s, e);
        acc_s[0][r][tid] = s;
        acc_s[1][r][tid] += e;
        two_sum(acc_s[2][r][tid], pay[r], s, e);
        acc_s[2][r][tid] = s;
        acc_s[3][r][tid] += e;
      }
    }
    __syncthreads();  // rec visible

    // ---- per-ray: smooth terms, sheet series, near corners, pixel
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t row = tg.j0 + warp * R + r;
      const bool inside = (col < tg.i1) && (row < tg.j1) && (row >= row0) && (row < row1);
      // P(t) = sum_n T_n t^n by Horner, complex FP32
      float pr = 0.f, pi = 0.f;
#pragma unroll
      for (int k = SHEET_TERMS - 1; k >= 0; --k) {
        const float ar = rec.T[k][0] + pr, ai = rec.T[k][1] + pi;
        pr = ar * tx - ai * ty[r];
        pi = ar * ty[r] + ai * tx;
      }
      for (int c = 0; c < rec.n_near; ++c) {
        const float wr = rec.near[c][0] + tx, wi = rec.near[c][1] + ty[r];
        const float lr = 0.5f * logf(wr * wr + wi * wi), li = atan2f(wi, wr);
        const float plr = wr * lr - wi * li, pli = wr * li + wi * lr;  // w Log w
        pr += rec.near[c][2] * pli;                                    // -i a_c (w Log w)
        pi -= rec.near[c][2] * plr;
      }
      const float axh = acc_s[0][r][tid], axl = acc_s[1][r][tid];
      const float ayh = acc_s[2][r][tid], ayl = acc_s[3][r][tid];
      float s1, e1, s2, e2;
      two_sum(rec.cx_hi, -axh, s1, e1);
      two_sum(rec.cy_hi, -ayh, s2, e2);
      const float b1 = s1 + (((e1 + rec.cx_lo) - axl) + (g.lam_s1 * tx + pr));
      const float b2 = s2 + (((e2 + rec.cy_lo) - ayl) + (g.lam_s2 * ty[r] - pi));
      uint32_t key = 0;
      int64_t pix = -1;
      const bool ok = inside && pixel_from_rel(g, rec.ix, rec.iy, b1, b2, key, pix);
      if (MODE == MODE_MAP) {
        bin_warp(counts, ok, key);
      } else {
        if (col == want_i && row == want_j) {
          beta_out[2 * work] = (g.src_x0 + (double)rec.ix * g.sx) + (double)b1;
          beta_out[2 * work + 1] = (g.src_y0 + (double)rec.iy * g.sy) + (double)b2;
          if (pix_out) pix_out[work] = pix;
        }
      }
    }
  }
}

#define BR_DECL_OCC(V, R, PAIRED, QUAD, PACK, TPSM)                                             \
  case V:                                                                                       \
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm,                                  \
                                                      k_brute<MODE_MAP, R, PAIRED, QUAD, PACK, TPSM>, \
                                                      32 * (BR_TY / R), 0) != cudaSuccess)      \
      per_sm = 1;                                                                               \
    break;
int brute_num_variants() { return BR_NVARIANT; }

#define BR_DECL_QUAD(V, R, PAIRED, QUAD, PACK, TPSM) \
  case V:                                            \
    return QUAD;
static int brute_quads(int variant) {
  switch (variant) { BR_VARIANTS(BR_DECL_QUAD) default: break; }
  return 0;
}

// A variant with four-row reciprocals multiplies four squared distances: it
// serves planes whose diagonal (the largest ray-lens distance; every lens is
// inside the plane) keeps that product in the FP32 range.
bool brute_variant_fits(int variant, double plane_diag) {
  if (variant < 0 || variant >= BR_NVARIANT) return false;
  return brute_quads(variant) == 0 || plane_diag <= BR_QUAD_MAX_DIAG;
}

int brute_grid_size(int num_sms, int variant) {
  int per_sm = 0;
  switch (variant) { BR_VARIANTS(BR_DECL_OCC) default: break; }
  return num_sms * (per_sm < 1 ? 1 : per_sm);
}

#define BR_DECL_LAUNCH(V, R, PAIRED, QUAD, PACK, TPSM)                                         \
  case V:                                                                                      \
    if (mode == MODE_MAP)                                                                      \
      k_brute<MODE_MAP, R, PAIRED, QUAD, PACK, TPSM><<<(unsigned)grid, 32 * (BR_TY / R), 0, s>>>( \
          P->g, xy2, mass, n, P->d_tiles, P->br_ntx, nwork, row0, row1, counts, idx, beta, pix); \
    else                                                                                       \
      k_brute<MODE_DUMP, R, PAIRED, QUAD, PACK, TPSM><<<(unsigned)grid, 32 * (BR_TY / R), 0, s>>>( \
          P->g, xy2, mass, n, P->d_tiles, P->br_ntx, nwork, row0, row1, counts, idx, beta, pix); \
    break;
static cudaError_t launch_brute(const irs_plan_t* P, int mode, int64_t grid, const double* xy,
                                const double* mass, int64_t n, int64_t nwork, int64_t row0,
                                int64_t row1, uint32_t* counts, const int64_t* idx, double* beta,
                                int64_t* pix, cudaStream_t s) {
  const double2* xy2 = reinterpret_cast<const double2*>(xy);
  switch (P->p.kernel_variant) {
    BR_VARIANTS(BR_DECL_LAUNCH)
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_brute_map(const irs_plan_t* P, const double* xy, const double* mass, int64_t n,
                             int64_t row0, int64_t row1, uint32_t* counts, cudaStream_t s) {
  if (row1 <= row0) return cudaSuccess;
  const int64_t tr0 = row0 / BR_TY, tr1 = (row1 + BR_TY - 1) / BR_TY;
  const int64_t nwork = (tr1 - tr0) * P->br_ntx;
  const int64_t grid = nwork < P->br_grid ? nwork : P->br_grid;
  return launch_brute(P, MODE_MAP, grid, xy, mass, n, nwork, row0, row1, counts, nullptr, nullptr,
                      nullptr, s);
}

cudaError_t launch_brute_dump(const irs_plan_t* P, const double* xy, const double* mass, int64_t n,
                              const int64_t* idx, int64_t nidx, double* beta, int64_t* pix,
                              cudaStream_t s) {
  const int64_t grid = nidx < P->br_grid ? nidx : P->br_grid;
  return launch_brute(P, MODE_DUMP, grid, xy, mass, n, nidx, 0, P->g.nry, nullptr, idx, beta, pix, s);
}

// ------------------------------------------------------------ magnification
// Mag_ij = N_ij * S_I / S_S with S_I = dx3^2 and S_S = s_x s_y ("Calculate the
// magnification of each pixel", Sec. 2.4).
__global__ void k_magnify(const uint32_t* __restrict__ counts, float* __restrict__ mag, int64_t npix,
                          float ratio) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < npix; k += stride)
    mag[k] = (float)counts[k] * ratio;
}

cudaError_t launch_magnify(const irs_plan_t* P, const uint32_t* counts, float* mag, cudaStream_t s) {
  const int64_t npix = (int64_t)P->g.npix_x * P->g.npix_y;
  const float ratio = (float)(P->g.dx3 * P->g.dx3 / (P->g.sx * P->g.sy));
  int64_t blocks = (npix + 255) / 256;
  const int64_t cap = (int64_t)P->num_sms * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  k_magnify<<<(unsigned)blocks, 256, 0, s>>>(counts, mag, npix, ratio);
  return cudaGetLastError();
}

}  // namespace irs
