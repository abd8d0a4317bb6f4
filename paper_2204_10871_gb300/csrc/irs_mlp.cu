// irs_mlp.cu -- learned far-far field for IRS_MLP plans (no counterpart in
// arXiv:2204.10871, which interpolates the whole far field from its level-2
// grid).
//
// Split of the lens sum for a level-1 cell C with centre z_C (cell units r):
//   near    the 3x3 block, per ray (unchanged);
//   ring    every other lens with weight w(r), w = 1 for r <= R/2, a C-infinity
//           step to 0 at R = R_f (mlp_ring_weight): summed directly into the
//           cell series (FP64);
//   far-far every lens with weight 1 - w(r).  Its series, minus the sheet's
//           analytic part g and the constant kappa_* conj(z_C) that the far
//           continuum carries, is a smooth function U(z_C) of the cell centre
//           (the weights depend on z_C, not on the ray), which a coordinate
//           network with Fourier features learns from direct sums.
// Cells within 1.5 R_f of a rectangle corner, where U carries the corner's
// (z - c) Log(z - c) singularity, use the exact direct far-far sum instead.
//
// Network: features [sin, cos](pi B x) with 32 frequencies, three tanh layers
// of width 64, a linear head of 8 outputs (U's first 4 complex coefficients,
// standardised).  Training: BF16 operands on the tensor cores
// (mma.sync.m16n8k16) with FP32 accumulation, FP32 master weights and AdamW.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <new>
#include <vector>

#include "irs_interp.cuh"
#include "irs_mlp.cuh"

namespace irs {

namespace {

constexpr int OFF_W1 = 0, OFF_B1 = 4096, OFF_W2 = 4160, OFF_B2 = 8256, OFF_W3 = 8320,
              OFF_B3 = 12416, OFF_W4 = 12480, OFF_B4 = 12992;
constexpr int MLP_WARPS = 4;                 // warps per CTA, 16 samples each
constexpr int MLP_CTA = MLP_WARPS * 32;
constexpr int MLP_TILE = 16 * MLP_W;         // one [16][64] FP32 activation tile
constexpr int FF_THREADS = 256;

struct MlpState {
  float* theta;   // FP32 master weights (packed as the reference network)
  float* adam_m;
  float* adam_v;
  float* grad;
  float* freq;    // [32][2]
  float* out_mean;  // [8]
  float* out_std;   // [8]
  double* loss;   // [1] loss accumulator
  float2* xs;     // training inputs
  float* ts;      // training targets (standardised)
  int64_t n_samples;
  float2* U;      // [nrc][MLP_KFF]
  float2* cell_x;   // [nrc] network inputs at the ray-cell centres
  float* cell_y;    // [nrc][8] network outputs
  int32_t* corner;  // [nrc]
  double2* exact;   // [ncorner][MLP_KEXACT]
  double2* corner_pts;  // [ncorner] cell centres
  int64_t ncorner;
  double cx, cy, half;  // input normalisation: x = (z - centre) / half
  double rf;            // window radius R_f in cells
  int trained;
  void* ws;
};

MlpState* M_(irs_plan_t* P) { return static_cast<MlpState*>(P->mlp); }

// ------------------------------------------------------------ seeded draws
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
__device__ __forceinline__ double u01(uint64_t x) { return (double)(splitmix64(x) >> 11) * 0x1.0p-53; }

// ------------------------------------------------------------ far-far direct sum
// out[p][k] = -sum_i (1 - w(r_i)) m_i h^k / d_i^(k+1),  d_i = z_i - z_p (k < KO):
// the tau^k coefficients of the weighted far-far lens field about z_p.  FP32
// pair terms with double-float positions, FP64 accumulation per 256-lens stage.
template <int KO>
__global__ void __launch_bounds__(FF_THREADS) k_ff_direct(const double2* __restrict__ xy,
                                                          const double* __restrict__ mass, int64_t n,
                                                          const double2* __restrict__ pts, int64_t npts,
                                                          double h, double R, double2* __restrict__ out) {
  __shared__ float4 L_s[FF_THREADS];  // xh, yh, xl, yl
  __shared__ float m_s[FF_THREADS];
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = p < npts;
  const double2 zc = live ? pts[p] : make_double2(0.0, 0.0);
  const float cxh = (float)zc.x, cyh = (float)zc.y;
  const float cxl = (float)(zc.x - (double)cxh), cyl = (float)(zc.y - (double)cyh);
  const float inv_h = (float)(1.0 / h);
  const float R2 = (float)(R * R), Rh2 = (float)(0.25 * R * R);
  double accd[KO][2];
#pragma unroll
  for (int k = 0; k < KO; ++k) accd[k][0] = accd[k][1] = 0.0;
  for (int64_t base = 0; base < n; base += FF_THREADS) {
    const int64_t i = base + threadIdx.x;
    __syncthreads();
    if (i < n) {
      const double2 q = xy[i];
      const float xh = (float)q.x, yh = (float)q.y;
      L_s[threadIdx.x] = make_float4(xh, yh, (float)(q.x - (double)xh), (float)(q.y - (double)yh));
      m_s[threadIdx.x] = (float)mass[i];
    } else {
      L_s[threadIdx.x] = make_float4(1.0e15f, 1.0e15f, 0.f, 0.f);
      m_s[threadIdx.x] = 0.f;
    }
    __syncthreads();
    float acc[KO][2];
#pragma unroll
    for (int k = 0; k < KO; ++k) acc[k][0] = acc[k][1] = 0.f;
    const int cnt = (int)min((int64_t)FF_THREADS, n - base);
    for (int j = 0; j < cnt; ++j) {
      const float4 L = L_s[j];
      // d in cell units
      const float dx = ((L.x - cxh) + (L.z - cxl)) * inv_h, dy = ((L.y - cyh) + (L.w - cyl)) * inv_h;
      const float r2 = dx * dx + dy * dy;
      float wgt = m_s[j];
      if (r2 < R2) {
        if (r2 <= Rh2) continue;  // inside R/2: entirely in the direct ring
        // far-far share 1 - w of the ring weight (mlp_ring_weight)
        const float t = 2.0f * sqrtf(r2) / (float)R - 1.0f;
        const float ea = expf(-1.0f / t), eb = expf(-1.0f / (1.0f - t));
        wgt *= ea / (ea + eb);
      }
      const float ir = rcp_approx(r2);
      const float ur = dx * ir, ui = -dy * ir;  // 1/d
      float pr = ur * wgt, pi = ui * wgt;       // w m / d
#pragma unroll
      for (int k = 0; k < KO; ++k) {
        acc[k][0] -= pr;
        acc[k][1] -= pi;
        const float nr = pr * ur - pi * ui, ni = pr * ui + pi * ur;
        pr = nr;
        pi = ni;
      }
    }
#pragma unroll
    for (int k = 0; k < KO; ++k) {
      accd[k][0] += (double)acc[k][0];
      accd[k][1] += (double)acc[k][1];
    }
  }
  if (live) {
    // cell units -> theta_E: (1/h) per lens term
    for (int k = 0; k < KO; ++k) out[p * KO + k] = make_double2(accd[k][0] / h, accd[k][1] / h);
  }
}

// Sheet series g_k h^k (k < KO) of the positive rectangle sheet about z (inside
// the rectangle), all four corners, interior-consistent branches.
__device__ void sheet_series(const Geo& g, double ks, double zx, double zy, double h, int KO,
                             double2* gk) {
  for (int k = 0; k < KO; ++k) gk[k] = make_double2(0.0, 0.0);
  gk[0] = make_double2(ks * (zx - 2.0 * g.a2), ks * zy);
  if (KO > 1) gk[1].x += ks * h;
  const double cxs[4] = {g.a1, g.a2, g.a1, g.a2};
  const double cys[4] = {g.b1, g.b1, g.b2, g.b2};
  const double sgn[4] = {1.0, -1.0, -1.0, 1.0};
  for (int q = 0; q < 4; ++q) {
    const double ac = ks / M_PI * sgn[q];
    if (ac == 0.0) continue;
    const double wr = zx - cxs[q], wi = zy - cys[q];
    double arg = atan2(wi, wr);
    if (q == 3 && wr < 0.0 && wi > 0.0) arg -= 2.0 * M_PI;
    if (q == 1 && wr < 0.0 && wi < 0.0) arg += 2.0 * M_PI;
    const double lr = 0.5 * log(wr * wr + wi * wi), li = arg;
    const double plr = wr * lr - wi * li, pli = wr * li + wi * lr;
    gk[0].x += ac * pli;
    gk[0].y -= ac * plr;
    if (KO > 1) {
      gk[1].x += ac * li * h;
      gk[1].y -= ac * (lr + 1.0) * h;
    }
    const double d = wr * wr + wi * wi;
    const double ir = wr / d * h, ii = -wi / d * h;  // h / w
    double pr = ir * h, pi = ii * h;                   // h^2 / w at n = 2
    for (int nn = 2; nn < KO; ++nn) {
      const double cf = ((nn & 1) ? -1.0 : 1.0) / (double)(nn * (nn - 1));
      gk[nn].x += ac * cf * pi;
      gk[nn].y -= ac * cf * pr;
      const double nr = pr * ir - pi * ii, ni = pr * ii + pi * ir;
      pr = nr;
      pi = ni;
    }
  }
}

// Random training points inside the rectangle (seeded, counter-based).
__global__ void k_mlp_points(Geo g, uint64_t seed, int64_t np, double2* __restrict__ pts) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  const double u = u01(seed ^ (2 * (uint64_t)i)), v = u01(seed ^ (2 * (uint64_t)i + 1));
  pts[i] = make_double2(g.a1 + u * (g.a2 - g.a1), g.b1 + v * (g.b2 - g.b1));
}

// Targets U_k = L_ff,k - g_k h^k - kappa_* conj(z) delta_k0, inputs x = (z - c)/half.
__global__ void k_mlp_targets(Geo g, const double* __restrict__ msum, const double2* __restrict__ pts,
                              const double2* __restrict__ lff, int64_t np, double h, double cx,
                              double cy, double half, float2* __restrict__ xs, double* __restrict__ u) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  const double ks = g.kstar_scale * msum[0];
  const double2 z = pts[i];
  double2 gk[MLP_KFF];
  sheet_series(g, ks, z.x, z.y, h, MLP_KFF, gk);
  for (int k = 0; k < MLP_KFF; ++k) {
    double2 t = lff[i * MLP_KFF + k];
    t.x -= gk[k].x;
    t.y -= gk[k].y;
    if (k == 0) {
      t.x -= ks * z.x;
      t.y += ks * z.y;
    }
    u[i * MLP_OUT + 2 * k] = t.x;
    u[i * MLP_OUT + 2 * k + 1] = t.y;
  }
  xs[i] = make_float2((float)((z.x - cx) / half), (float)((z.y - cy) / half));
}

__global__ void k_mlp_moments(const double* __restrict__ u, int64_t np, double* __restrict__ mom) {
  // mom[o] += sum u, mom[8 + o] += sum u^2 (one output per warp lane group)
  __shared__ double s1[MLP_OUT][32], s2[MLP_OUT][32];
  const int o = threadIdx.x >> 5, lane = threadIdx.x & 31;  // blockDim = 256 -> 8 outputs
  double a = 0.0, b = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * 32 + lane; i < np; i += (int64_t)gridDim.x * 32) {
    const double v = u[i * MLP_OUT + o];
    a += v;
    b += v * v;
  }
  s1[o][lane] = a;
  s2[o][lane] = b;
  __syncthreads();
  if (lane == 0) {
    double sa = 0.0, sb = 0.0;
    for (int k = 0; k < 32; ++k) {
      sa += s1[o][k];
      sb += s2[o][k];
    }
    atomicAdd(&mom[o], sa);
    atomicAdd(&mom[MLP_OUT + o], sb);
  }
}

__global__ void k_mlp_standardise(const double* __restrict__ u, int64_t np, const float* __restrict__ mean,
                                  const float* __restrict__ sd, float* __restrict__ t) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np * MLP_OUT) return;
  const int o = (int)(i % MLP_OUT);
  t[i] = (float)((u[i] - (double)mean[o]) / (double)sd[o]);
}

// ------------------------------------------------------------ tensor-core tiles
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16(float c[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// acc[nt] (16 x 8 tiles) += A (16 x K) * B (K x 8 NT) on one warp; A(m, k) =
// A[m ars + k acs] (0 for m >= mv or k >= kv), B(k, n) = B[k brs + n bcs]
// (0 for k >= kv); operands rounded to BF16, products accumulated in FP32.
// Fragment layouts of mma.m16n8k16: A rows gid / gid+8, cols 2 tig (+1, +8, +9);
// B rows 2 tig (+1, +8, +9), col gid; C rows gid / gid+8, cols 2 tig (+1).
template <int NT>
__device__ __forceinline__ void warp_gemm(const float* A, int ars, int acs, int mv, const float* B, int brs,
                                          int bcs, int K, int kv, float (*acc)[4]) {
  const int lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
  auto a = [&](int m, int k) { return (m < mv && k < kv) ? A[m * ars + k * acs] : 0.f; };
  auto b = [&](int k, int n) { return k < kv ? B[k * brs + n * bcs] : 0.f; };
  for (int k0 = 0; k0 < K; k0 += 16) {
    const int c0 = k0 + 2 * tig;
    const uint32_t a0 = pack_bf16(a(gid, c0), a(gid, c0 + 1));
    const uint32_t a1 = pack_bf16(a(gid + 8, c0), a(gid + 8, c0 + 1));
    const uint32_t a2 = pack_bf16(a(gid, c0 + 8), a(gid, c0 + 9));
    const uint32_t a3 = pack_bf16(a(gid + 8, c0 + 8), a(gid + 8, c0 + 9));
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      const int n = nt * 8 + gid;
      const uint32_t b0 = pack_bf16(b(c0, n), b(c0 + 1, n));
      const uint32_t b1 = pack_bf16(b(c0 + 8, n), b(c0 + 9, n));
      mma_bf16(acc[nt], a0, a1, a2, a3, b0, b1);
    }
  }
}

// C-fragment element q of tile nt: row and column in the 16 x (8 NT) result.
__device__ __forceinline__ int frag_row(int q) { return ((threadIdx.x & 31) >> 2) + (q >= 2 ? 8 : 0); }
__device__ __forceinline__ int frag_col(int nt, int q) { return nt * 8 + 2 * ((threadIdx.x & 31) & 3) + (q & 1); }

// Forward pass of 16 samples on one warp.  act: [4][16][64] (features, h1,
// h2, h3); W: packed FP32 weights in shared memory.  y[q] = output element
// (frag_row(q), frag_col(0, q)) of the 16 x 8 head.
__device__ void mlp_forward_warp(const float* W, const float* freq, const float2* x16, int ns, float* act,
                                 float y[4]) {
  const int lane = threadIdx.x & 31;
  float* F = act;
  for (int e = lane; e < 16 * MLP_NF; e += 32) {
    const int s = e / MLP_NF, j = e % MLP_NF;
    float sv = 0.f, cv = 0.f;
    if (s < ns) {
      const float a = 3.14159265358979f * (freq[2 * j] * x16[s].x + freq[2 * j + 1] * x16[s].y);
      sincosf(a, &sv, &cv);
    }
    F[s * MLP_W + j] = sv;
    F[s * MLP_W + MLP_NF + j] = cv;
  }
  __syncwarp();
  const int woff[3] = {OFF_W1, OFF_W2, OFF_W3}, boff[3] = {OFF_B1, OFF_B2, OFF_B3};
  for (int l = 0; l < 3; ++l) {
    const float* Hin = act + l * MLP_TILE;
    float* Hout = act + (l + 1) * MLP_TILE;
    float acc[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
    warp_gemm<8>(Hin, MLP_W, 1, 16, W + woff[l], 1, MLP_W, MLP_W, MLP_W, acc);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int o = frag_col(nt, q);
        Hout[frag_row(q) * MLP_W + o] = tanhf(acc[nt][q] + W[boff[l] + o]);
      }
    __syncwarp();
  }
  float acc4[1][4] = {{0.f, 0.f, 0.f, 0.f}};
  warp_gemm<1>(act + 3 * MLP_TILE, MLP_W, 1, 16, W + OFF_W4, 1, MLP_W, MLP_W, MLP_W, acc4);
#pragma unroll
  for (int q = 0; q < 4; ++q) y[q] = acc4[0][q] + W[OFF_B4 + frag_col(0, q)];
}

// Fused forward + backward of a batch; weight gradients accumulate in shared
// memory per CTA, then once per CTA into `grad`.  Samples: idx[b] when given,
// else a seeded draw per (step, slot).
__global__ void __launch_bounds__(MLP_CTA) k_mlp_train(const float* __restrict__ theta,
                                                       const float* __restrict__ freq,
                                                       const float2* __restrict__ xs,
                                                       const float* __restrict__ ts, int64_t n_samples,
                                                       int64_t batch, uint64_t seed, int ordered,
                                                       float* __restrict__ grad, double* __restrict__ loss) {
  extern __shared__ float smem[];
  float* W = smem;                          // MLP_NPARAM
  float* G = W + MLP_NPARAM;                // MLP_NPARAM gradient accumulator
  float* actall = G + MLP_NPARAM;           // warps x (4 + 1) tiles + dy
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int k = tid; k < MLP_NPARAM; k += blockDim.x) {
    W[k] = theta[k];
    G[k] = 0.f;
  }
  __syncthreads();
  float* act = actall + warp * (5 * MLP_TILE + 16 * MLP_OUT);
  float* DZ = act + 4 * MLP_TILE;
  float* DY = DZ + MLP_TILE;
  __shared__ float2 xw[MLP_WARPS][16];
  __shared__ int64_t sid[MLP_WARPS][16];
  const int64_t b0 = ((int64_t)blockIdx.x * MLP_WARPS + warp) * 16;
  int ns = 0;
  if (lane < 16) {
    const int64_t b = b0 + lane;
    int64_t s = -1;
    if (b < batch)
      s = ordered ? b : (int64_t)(splitmix64(seed ^ (uint64_t)b * 0x2545F4914F6CDD1Dull) % (uint64_t)n_samples);
    sid[warp][lane] = s;
    xw[warp][lane] = s >= 0 ? xs[s] : make_float2(0.f, 0.f);
  }
  __syncwarp();
  for (int k = 0; k < 16; ++k) ns += sid[warp][k] >= 0 ? 1 : 0;
  float y[4];
  mlp_forward_warp(W, freq, xw[warp], ns, act, y);
  // loss and dL/dy (mean over the whole batch and the 8 outputs)
  const float scale = 2.0f / (float)(batch * MLP_OUT);
  float lsum = 0.f;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int s = frag_row(q), o = frag_col(0, q);
    float d = 0.f;
    if (s < ns) {
      d = y[q] - ts[sid[warp][s] * MLP_OUT + o];
      lsum += d * d;
    }
    DY[s * MLP_OUT + o] = d * scale;
  }
  for (int off = 16; off; off >>= 1) lsum += __shfl_xor_sync(0xFFFFFFFFu, lsum, off);
  if (lane == 0 && ns > 0) atomicAdd(loss, (double)lsum);
  __syncwarp();
  float* H[4] = {act, act + MLP_TILE, act + 2 * MLP_TILE, act + 3 * MLP_TILE};
  // head: dW4[o][i] = sum_s dy[s][o] h3[s][i]; db4; dh3 = dy W4
  {
    float acc[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
    warp_gemm<8>(DY, 1, MLP_OUT, MLP_OUT, H[3], MLP_W, 1, 16, 16, acc);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int q = 0; q < 2; ++q) atomicAdd(&G[OFF_W4 + frag_row(q) * MLP_W + frag_col(nt, q)], acc[nt][q]);
    if (lane < MLP_OUT) {
      float sb = 0.f;
      for (int s = 0; s < 16; ++s) sb += DY[s * MLP_OUT + lane];
      atomicAdd(&G[OFF_B4 + lane], sb);
    }
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
    warp_gemm<8>(DY, MLP_OUT, 1, 16, W + OFF_W4, MLP_W, 1, 16, MLP_OUT, acc);
    __syncwarp();
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int s = frag_row(q), i = frag_col(nt, q);
        const float h = H[3][s * MLP_W + i];
        DZ[s * MLP_W + i] = acc[nt][q] * (1.f - h * h);
      }
    __syncwarp();
  }
  const int woff[3] = {OFF_W1, OFF_W2, OFF_W3}, boff[3] = {OFF_B1, OFF_B2, OFF_B3};
  for (int l = 2; l >= 0; --l) {
    // dW_l[o][i] = sum_s dz[s][o] Hin[s][i] in four 16-row tiles of o; db_l
    const float* Hin = H[l];
    for (int mt = 0; mt < 4; ++mt) {
      float acc[8][4];
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
      warp_gemm<8>(DZ + mt * 16, 1, MLP_W, 16, Hin, MLP_W, 1, 16, 16, acc);
#pragma unroll
      for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int q = 0; q < 4; ++q)
          atomicAdd(&G[woff[l] + (mt * 16 + frag_row(q)) * MLP_W + frag_col(nt, q)], acc[nt][q]);
    }
    for (int o = lane; o < MLP_W; o += 32) {
      float sb = 0.f;
      for (int s = 0; s < 16; ++s) sb += DZ[s * MLP_W + o];
      atomicAdd(&G[boff[l] + o], sb);
    }
    if (l == 0) break;
    // dH_{l} = dz W_l, then dz_{l-1} = dH (1 - h^2)
    float acc[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
    warp_gemm<8>(DZ, MLP_W, 1, 16, W + woff[l], MLP_W, 1, MLP_W, MLP_W, acc);
    __syncwarp();
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int s = frag_row(q), i = frag_col(nt, q);
        const float h = Hin[s * MLP_W + i];
        DZ[s * MLP_W + i] = acc[nt][q] * (1.f - h * h);
      }
    __syncwarp();
  }
  __syncthreads();
  for (int k = tid; k < MLP_NPARAM; k += blockDim.x)
    if (G[k] != 0.f) atomicAdd(&grad[k], G[k]);
}

__global__ void k_adamw(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                        float* __restrict__ g, float lr, float b1, float b2, float eps, float wd, float c1,
                        float c2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= MLP_NPARAM) return;
  const float gk = g[k];
  const float mk = b1 * m[k] + (1.f - b1) * gk;
  const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
  m[k] = mk;
  v[k] = vk;
  theta[k] -= lr * ((mk / c1) / (sqrtf(vk / c2) + eps) + wd * theta[k]);
  g[k] = 0.f;
}

// Network output at arbitrary inputs (standardised units), 16 per warp.
__global__ void __launch_bounds__(MLP_CTA) k_mlp_eval(const float* __restrict__ theta,
                                                      const float* __restrict__ freq,
                                                      const float2* __restrict__ x, int64_t n,
                                                      float* __restrict__ y_out) {
  extern __shared__ float smem[];
  float* W = smem;
  float* actall = W + MLP_NPARAM;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int k = tid; k < MLP_NPARAM; k += blockDim.x) W[k] = theta[k];
  __syncthreads();
  float* act = actall + warp * 4 * MLP_TILE;
  __shared__ float2 xw[MLP_WARPS][16];
  const int64_t b0 = ((int64_t)blockIdx.x * MLP_WARPS + warp) * 16;
  const int ns = (int)min((int64_t)16, n - b0);
  if (ns <= 0) return;
  if (lane < 16) xw[warp][lane] = lane < ns ? x[b0 + lane] : make_float2(0.f, 0.f);
  __syncwarp();
  float y[4];
  mlp_forward_warp(W, freq, xw[warp], ns, act, y);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int s = frag_row(q);
    if (s < ns) y_out[(b0 + s) * MLP_OUT + frag_col(0, q)] = y[q];
  }
}

// Learned coefficients of every ray cell: U = y * sd + mean at the cell centre.
__global__ void k_mlp_cell_inputs(double gx0, double gy0, double h, int nrcx, int ox, int oy, int64_t nrc,
                                  double cx, double cy, double half, float2* __restrict__ x) {
  const int64_t rc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (rc >= nrc) return;
  const int cxi = (int)(rc % nrcx) + ox, cyi = (int)(rc / nrcx) + oy;
  const double zx = gx0 + (cxi + 0.5) * h, zy = gy0 + (cyi + 0.5) * h;
  x[rc] = make_float2((float)((zx - cx) / half), (float)((zy - cy) / half));
}

__global__ void k_mlp_cell_outputs(const float* __restrict__ y, int64_t nrc, const float* __restrict__ mean,
                                   const float* __restrict__ sd, float2* __restrict__ U) {
  const int64_t rc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (rc >= nrc) return;
  for (int k = 0; k < MLP_KFF; ++k)
    U[rc * MLP_KFF + k] = make_float2(y[rc * MLP_OUT + 2 * k] * sd[2 * k] + mean[2 * k],
                                      y[rc * MLP_OUT + 2 * k + 1] * sd[2 * k + 1] + mean[2 * k + 1]);
}

size_t train_smem() {
  return sizeof(float) * (2 * MLP_NPARAM + MLP_WARPS * (5 * MLP_TILE + 16 * MLP_OUT));
}
size_t eval_smem() { return sizeof(float) * (MLP_NPARAM + MLP_WARPS * 4 * MLP_TILE); }

}  // namespace

// ------------------------------------------------------------ host side
irs_status mlp_plan(irs_plan_t* P, double gx0, double gy0, double h, int ncx, int ncy, int nrcx,
                    int nrcy, int ox, int oy, int64_t n_samples) {
  MlpState* M = new (std::nothrow) MlpState();
  if (!M) return IRS_ERR_OOM;
  memset(M, 0, sizeof(*M));
  P->mlp = M;
  (void)ncx;
  (void)ncy;
  const int64_t nrc = (int64_t)nrcx * nrcy;
  M->n_samples = n_samples;
  M->cx = P->g.cx;
  M->cy = P->g.cy;
  M->half = 0.5 * fmax(P->g.a2 - P->g.a1, P->g.b2 - P->g.b1);
  // corner zones: ray cells whose centre lies within 1.5 R_f cells of a corner
  std::vector<int32_t> corner((size_t)nrc, -1);
  std::vector<double2> pts;
  M->rf = P->p.window > 0 ? (double)P->p.window : MLP_RF_DEFAULT;
  const double lim = 1.5 * M->rf * h;
  const double cxs[4] = {P->g.a1, P->g.a2, P->g.a1, P->g.a2}, cys[4] = {P->g.b1, P->g.b1, P->g.b2, P->g.b2};
  for (int64_t rc = 0; rc < nrc; ++rc) {
    const double zx = gx0 + ((int)(rc % nrcx) + ox + 0.5) * h, zy = gy0 + ((int)(rc / nrcx) + oy + 0.5) * h;
    for (int q = 0; q < 4; ++q)
      if (hypot(zx - cxs[q], zy - cys[q]) < lim) {
        corner[(size_t)rc] = (int32_t)pts.size();
        pts.push_back(make_double2(zx, zy));
        break;
      }
  }
  M->ncorner = (int64_t)pts.size();
  size_t off = 0;
  auto take = [&](size_t b) {
    size_t o = off;
    off += (b + 255) & ~(size_t)255;
    return o;
  };
  const size_t o_theta = take(4 * MLP_NPARAM), o_m = take(4 * MLP_NPARAM), o_v = take(4 * MLP_NPARAM),
               o_g = take(4 * MLP_NPARAM), o_f = take(4 * 2 * MLP_NF), o_mean = take(4 * MLP_OUT),
               o_sd = take(4 * MLP_OUT), o_loss = take(8 * 2), o_xs = take(sizeof(float2) * n_samples),
               o_ts = take(sizeof(float) * MLP_OUT * n_samples), o_U = take(sizeof(float2) * MLP_KFF * nrc),
               o_c = take(sizeof(int32_t) * nrc), o_ex = take(sizeof(double2) * MLP_KEXACT * (M->ncorner + 1)),
               o_pts = take(sizeof(double2) * (M->ncorner + 1)), o_cx = take(sizeof(float2) * nrc),
               o_cy = take(sizeof(float) * MLP_OUT * nrc);
  if (cudaMalloc(&M->ws, off) != cudaSuccess) {
    cudaGetLastError();
    M->ws = nullptr;
    return IRS_ERR_OOM;
  }
  char* b = static_cast<char*>(M->ws);
  M->theta = reinterpret_cast<float*>(b + o_theta);
  M->adam_m = reinterpret_cast<float*>(b + o_m);
  M->adam_v = reinterpret_cast<float*>(b + o_v);
  M->grad = reinterpret_cast<float*>(b + o_g);
  M->freq = reinterpret_cast<float*>(b + o_f);
  M->out_mean = reinterpret_cast<float*>(b + o_mean);
  M->out_std = reinterpret_cast<float*>(b + o_sd);
  M->loss = reinterpret_cast<double*>(b + o_loss);
  M->xs = reinterpret_cast<float2*>(b + o_xs);
  M->ts = reinterpret_cast<float*>(b + o_ts);
  M->U = reinterpret_cast<float2*>(b + o_U);
  M->corner = reinterpret_cast<int32_t*>(b + o_c);
  M->exact = reinterpret_cast<double2*>(b + o_ex);
  M->corner_pts = reinterpret_cast<double2*>(b + o_pts);
  M->cell_x = reinterpret_cast<float2*>(b + o_cx);
  M->cell_y = reinterpret_cast<float*>(b + o_cy);
  if (cudaMemset(M->ws, 0, off) != cudaSuccess) return IRS_ERR_CUDA;
  if (cudaMemcpy(M->corner, corner.data(), sizeof(int32_t) * nrc, cudaMemcpyHostToDevice) != cudaSuccess)
    return IRS_ERR_CUDA;
  if (!pts.empty() &&
      cudaMemcpy(M->corner_pts, pts.data(), sizeof(double2) * pts.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return IRS_ERR_CUDA;
  if (cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)train_smem()) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_mlp_eval, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)eval_smem()) !=
          cudaSuccess)
    return IRS_ERR_CUDA;
  return IRS_OK;
}

void mlp_destroy(irs_plan_t* P) {
  MlpState* M = M_(P);
  if (!M) return;
  if (M->ws) cudaFree(M->ws);
  delete M;
  P->mlp = nullptr;
}

bool mlp_trained(const irs_plan_t* P) {
  const MlpState* M = static_cast<const MlpState*>(P->mlp);
  return M && M->trained;
}

// Per map: exact far-far sums at the corner-zone cells and the network's
// coefficients at every ray cell.
irs_status mlp_prepare(irs_plan_t* P, const double* xy, const double* mass, int64_t n, double gx0, double gy0,
                       double h, int nrcx, int nrcy, int ox, int oy, MlpFar* far, cudaStream_t s) {
  MlpState* M = M_(P);
  float2* scratch_x = M->cell_x;
  float* scratch_y = M->cell_y;
  const int64_t nrc = (int64_t)nrcx * nrcy;
  if (M->ncorner > 0 && n > 0)
    k_ff_direct<MLP_KEXACT><<<(unsigned)((M->ncorner + FF_THREADS - 1) / FF_THREADS), FF_THREADS, 0, s>>>(
        reinterpret_cast<const double2*>(xy), mass, n, M->corner_pts, M->ncorner, h, M->rf, M->exact);
  else if (M->ncorner > 0)
    cudaMemsetAsync(M->exact, 0, sizeof(double2) * MLP_KEXACT * M->ncorner, s);
  k_mlp_cell_inputs<<<(unsigned)((nrc + 255) / 256), 256, 0, s>>>(gx0, gy0, h, nrcx, ox, oy, nrc, M->cx, M->cy,
                                                                 M->half, scratch_x);
  const int64_t blocks = (nrc + 16 * MLP_WARPS - 1) / (16 * MLP_WARPS);
  k_mlp_eval<<<(unsigned)blocks, MLP_CTA, eval_smem(), s>>>(M->theta, M->freq, scratch_x, nrc, scratch_y);
  k_mlp_cell_outputs<<<(unsigned)((nrc + 255) / 256), 256, 0, s>>>(scratch_y, nrc, M->out_mean, M->out_std, M->U);
  if (cudaGetLastError() != cudaSuccess) return IRS_ERR_CUDA;
  far->U = M->U;
  far->corner = M->corner;
  far->exact = M->exact;
  far->rf = M->rf;
  far->active = 1;
  return IRS_OK;
}

irs_status mlp_set_params(irs_plan_t* P, const float* theta, const float* freq) {
  MlpState* M = M_(P);
  if (!M) return IRS_ERR_UNSUPPORTED;
  if (theta && cudaMemcpy(M->theta, theta, 4 * MLP_NPARAM, cudaMemcpyHostToDevice) != cudaSuccess)
    return IRS_ERR_CUDA;
  if (freq && cudaMemcpy(M->freq, freq, 4 * 2 * MLP_NF, cudaMemcpyHostToDevice) != cudaSuccess)
    return IRS_ERR_CUDA;
  return IRS_OK;
}

irs_status mlp_get_params(irs_plan_t* P, float* theta, float* freq) {
  MlpState* M = M_(P);
  if (!M) return IRS_ERR_UNSUPPORTED;
  if (theta && cudaMemcpy(theta, M->theta, 4 * MLP_NPARAM, cudaMemcpyDeviceToHost) != cudaSuccess)
    return IRS_ERR_CUDA;
  if (freq && cudaMemcpy(freq, M->freq, 4 * 2 * MLP_NF, cudaMemcpyDeviceToHost) != cudaSuccess)
    return IRS_ERR_CUDA;
  return IRS_OK;
}

irs_status mlp_grad(irs_plan_t* P, const float* x, const float* t, int64_t n, float* grad, double* loss,
                    cudaStream_t s) {
  MlpState* M = M_(P);
  if (!M) return IRS_ERR_UNSUPPORTED;
  if (n <= 0 || !x || !t || !grad || !loss) return IRS_ERR_ARG;
  if (cudaMemsetAsync(grad, 0, 4 * MLP_NPARAM, s) != cudaSuccess) return IRS_ERR_CUDA;
  if (cudaMemsetAsync(loss, 0, 8, s) != cudaSuccess) return IRS_ERR_CUDA;
  const int64_t blocks = (n + 16 * MLP_WARPS - 1) / (16 * MLP_WARPS);
  k_mlp_train<<<(unsigned)blocks, MLP_CTA, train_smem(), s>>>(M->theta, M->freq, reinterpret_cast<const float2*>(x),
                                                              t, n, n, 0, 1, grad, loss);
  return cudaGetLastError() == cudaSuccess ? IRS_OK : IRS_ERR_CUDA;
}

irs_status mlp_forward(irs_plan_t* P, const float* x, int64_t n, float* y, cudaStream_t s) {
  MlpState* M = M_(P);
  if (!M) return IRS_ERR_UNSUPPORTED;
  if (n <= 0) return IRS_OK;
  const int64_t blocks = (n + 16 * MLP_WARPS - 1) / (16 * MLP_WARPS);
  k_mlp_eval<<<(unsigned)blocks, MLP_CTA, eval_smem(), s>>>(M->theta, M->freq, reinterpret_cast<const float2*>(x),
                                                           n, y);
  return cudaGetLastError() == cudaSuccess ? IRS_OK : IRS_ERR_CUDA;
}

namespace {
// host-side seeded draws for the initial weights and the Fourier matrix
uint64_t hmix(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
double hu01(uint64_t x) { return (double)(hmix(x) >> 11) * 0x1.0p-53; }
}  // namespace

irs_status mlp_train(irs_plan_t* P, const double* xy, const double* mass, int64_t n, int64_t n_samples,
                     int32_t steps, uint64_t seed, irs_mlp_report* rep, cudaStream_t s) {
  MlpState* M = M_(P);
  if (!M) return IRS_ERR_UNSUPPORTED;
  if (n_samples <= 0) n_samples = M->n_samples;
  if (n_samples > M->n_samples || n_samples < 1024) return IRS_ERR_ARG;
  if (steps <= 0) steps = 3000;
  const int64_t n_valid = 16384, n_all = n_samples + n_valid;
  irs_mlp_report r;
  memset(&r, 0, sizeof r);
  r.samples = n_samples;
  r.steps = steps;
  const double h = interp_cell_side(P);
  cudaEvent_t e0, e1, e2;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventCreate(&e2);
  // temporaries (training is synchronous and outside any capture)
  double2 *pts = nullptr, *lff = nullptr;
  double *u = nullptr, *mom = nullptr;
  float2* xv = nullptr;
  float* yv = nullptr;
  irs_status st = IRS_OK;
  if (cudaMalloc(&pts, sizeof(double2) * n_all) != cudaSuccess ||
      cudaMalloc(&lff, sizeof(double2) * MLP_KFF * n_all) != cudaSuccess ||
      cudaMalloc(&u, sizeof(double) * MLP_OUT * n_all) != cudaSuccess ||
      cudaMalloc(&mom, sizeof(double) * 2 * MLP_OUT) != cudaSuccess ||
      cudaMalloc(&xv, sizeof(float2) * n_valid) != cudaSuccess ||
      cudaMalloc(&yv, sizeof(float) * MLP_OUT * n_valid) != cudaSuccess)
    st = IRS_ERR_OOM;
  std::vector<double> hu;
  std::vector<float> hy;
  if (st == IRS_OK) {
    cudaEventRecord(e0, s);
    launch_mass_sum(P, mass, n, s);
    k_mlp_points<<<(unsigned)((n_all + 255) / 256), 256, 0, s>>>(P->g, seed * 0x9E3779B97F4A7C15ull + 1, n_all, pts);
    if (n > 0)
      k_ff_direct<MLP_KFF><<<(unsigned)((n_all + FF_THREADS - 1) / FF_THREADS), FF_THREADS, 0, s>>>(
          reinterpret_cast<const double2*>(xy), mass, n, pts, n_all, h, M->rf, lff);
    else
      cudaMemsetAsync(lff, 0, sizeof(double2) * MLP_KFF * n_all, s);
    // training inputs go to M->xs; the held-out ones follow in xv
    k_mlp_targets<<<(unsigned)((n_samples + 255) / 256), 256, 0, s>>>(P->g, P->d_msum, pts, lff, n_samples, h,
                                                                     M->cx, M->cy, M->half, M->xs, u);
    k_mlp_targets<<<(unsigned)((n_valid + 255) / 256), 256, 0, s>>>(P->g, P->d_msum, pts + n_samples,
                                                                   lff + MLP_KFF * n_samples, n_valid, h, M->cx,
                                                                   M->cy, M->half, xv, u + MLP_OUT * n_samples);
    cudaMemsetAsync(mom, 0, sizeof(double) * 2 * MLP_OUT, s);
    k_mlp_moments<<<256, 256, 0, s>>>(u, n_samples, mom);
    cudaEventRecord(e1, s);
    double hm[2 * MLP_OUT];
    if (cudaMemcpyAsync(hm, mom, sizeof hm, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      st = IRS_ERR_CUDA;
    float mean[MLP_OUT], sd[MLP_OUT];
    double t2 = 0.0;
    for (int o = 0; o < MLP_OUT && st == IRS_OK; ++o) {
      const double mu = hm[o] / (double)n_samples;
      const double var = fmax(hm[MLP_OUT + o] / (double)n_samples - mu * mu, 1e-30);
      mean[o] = (float)mu;
      sd[o] = (float)sqrt(var);
      t2 += hm[MLP_OUT + o] / (double)n_samples;
    }
    r.target_rms = sqrt(t2 / MLP_OUT);
    // initial weights (fan-in uniform, zero biases) and Fourier matrix N(0, 8^2)
    std::vector<float> th(MLP_NPARAM, 0.f), fq(2 * MLP_NF);
    const int woff[4] = {OFF_W1, OFF_W2, OFF_W3, OFF_W4}, wrows[4] = {MLP_W, MLP_W, MLP_W, MLP_OUT};
    for (int l = 0; l < 4; ++l)
      for (int k = 0; k < wrows[l] * MLP_W; ++k)
        th[woff[l] + k] = (float)((2.0 * hu01(seed ^ (0x1000000ull * (l + 1) + k)) - 1.0) / 8.0);
    for (int k = 0; k < MLP_NF; ++k) {
      const double a = hu01(seed ^ (0xF00000000ull + 2 * k)), b = hu01(seed ^ (0xF00000000ull + 2 * k + 1));
      const double rr = sqrt(-2.0 * log(fmax(a, 1e-300)));
      fq[2 * k] = (float)(8.0 * rr * cos(2.0 * M_PI * b));
      fq[2 * k + 1] = (float)(8.0 * rr * sin(2.0 * M_PI * b));
    }
    if (st == IRS_OK &&
        (cudaMemcpy(M->out_mean, mean, sizeof mean, cudaMemcpyHostToDevice) != cudaSuccess ||
         cudaMemcpy(M->out_std, sd, sizeof sd, cudaMemcpyHostToDevice) != cudaSuccess ||
         cudaMemcpy(M->theta, th.data(), 4 * MLP_NPARAM, cudaMemcpyHostToDevice) != cudaSuccess ||
         cudaMemcpy(M->freq, fq.data(), 4 * 2 * MLP_NF, cudaMemcpyHostToDevice) != cudaSuccess ||
         cudaMemset(M->adam_m, 0, 4 * MLP_NPARAM) != cudaSuccess ||
         cudaMemset(M->adam_v, 0, 4 * MLP_NPARAM) != cudaSuccess ||
         cudaMemset(M->grad, 0, 4 * MLP_NPARAM) != cudaSuccess))
      st = IRS_ERR_CUDA;
    if (st == IRS_OK) {
      k_mlp_standardise<<<(unsigned)((n_samples * MLP_OUT + 255) / 256), 256, 0, s>>>(u, n_samples, M->out_mean,
                                                                                     M->out_std, M->ts);
      const int64_t batch = 4096;
      const int64_t blocks = batch / (16 * MLP_WARPS);
      const float lr0 = 2e-3f, b1 = 0.9f, b2 = 0.999f;
      double lsum_first = 0, lsum_last = 0;
      int nfirst = 0, nlast = 0;
      for (int step = 1; step <= steps; ++step) {
        const float warm = step < 100 ? (float)step / 100.f : 1.f;
        const float lr = lr0 * warm * 0.5f * (1.f + cosf(3.14159265f * (float)step / (float)steps));
        cudaMemsetAsync(M->loss, 0, 8, s);
        k_mlp_train<<<(unsigned)blocks, MLP_CTA, train_smem(), s>>>(M->theta, M->freq, M->xs, M->ts, n_samples,
                                                                    batch, seed ^ (0xABCDull * step), 0,
                                                                    M->grad, M->loss);
        k_adamw<<<(MLP_NPARAM + 255) / 256, 256, 0, s>>>(M->theta, M->adam_m, M->adam_v, M->grad, lr, b1, b2,
                                                         1e-8f, 0.f, 1.f - powf(b1, (float)step),
                                                         1.f - powf(b2, (float)step));
        if (step <= 20 || step > steps - 20) {
          double l = 0;
          cudaMemcpyAsync(&l, M->loss, 8, cudaMemcpyDeviceToHost, s);
          cudaStreamSynchronize(s);
          l /= (double)(batch * MLP_OUT);
          if (step <= 20) {
            lsum_first += l;
            ++nfirst;
          } else {
            lsum_last += l;
            ++nlast;
          }
        }
      }
      cudaEventRecord(e2, s);
      r.loss_first = nfirst ? lsum_first / nfirst : 0;
      r.loss_final = nlast ? lsum_last / nlast : 0;
      // held-out error in physical units
      k_mlp_eval<<<(unsigned)((n_valid + 63) / 64), MLP_CTA, eval_smem(), s>>>(M->theta, M->freq, xv, n_valid, yv);
      hu.resize((size_t)MLP_OUT * n_valid);
      hy.resize((size_t)MLP_OUT * n_valid);
      if (cudaMemcpyAsync(hu.data(), u + MLP_OUT * n_samples, sizeof(double) * hu.size(), cudaMemcpyDeviceToHost,
                          s) != cudaSuccess ||
          cudaMemcpyAsync(hy.data(), yv, sizeof(float) * hy.size(), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess)
        st = IRS_ERR_CUDA;
      double num = 0, den = 0;
      for (size_t k = 0; k < hu.size() && st == IRS_OK; ++k) {
        const int o = (int)(k % MLP_OUT);
        const double pred = (double)hy[k] * sd[o] + mean[o];
        num += (pred - hu[k]) * (pred - hu[k]);
        den += hu[k] * hu[k];
      }
      r.valid_rel_rms = den > 0 ? sqrt(num / den) : 0;
      float ms1 = 0, ms2 = 0;
      cudaEventElapsedTime(&ms1, e0, e1);
      cudaEventElapsedTime(&ms2, e1, e2);
      r.ms_samples = ms1;
      r.ms_train = ms2;
      if (st == IRS_OK) M->trained = 1;
      r.trained = M->trained;
    }
  }
  cudaFree(pts);
  cudaFree(lff);
  cudaFree(u);
  cudaFree(mom);
  cudaFree(xv);
  cudaFree(yv);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaEventDestroy(e2);
  if (rep) *rep = r;
  if (st == IRS_OK && cudaGetLastError() != cudaSuccess) st = IRS_ERR_CUDA;
  return st;
}

}  // namespace irs

extern "C" {

irs_status irs_mlp_train(irs_plan_t* plan, const double* lens_xy, const double* mass, int64_t n,
                         int64_t n_samples, int32_t steps, uint64_t seed, irs_mlp_report* report,
                         void* stream) {
  if (!plan || n < 0 || (n > 0 && (!lens_xy || !mass || ((uintptr_t)lens_xy & 15u)))) return IRS_ERR_ARG;
  if (plan->p.method != IRS_MLP || !plan->mlp) return IRS_ERR_UNSUPPORTED;
  return irs::mlp_train(plan, lens_xy, mass, n, n_samples, steps, seed, report,
                        static_cast<cudaStream_t>(stream));
}

irs_status irs_mlp_params(irs_plan_t* plan, const float* theta_in, const float* freq_in, float* theta_out,
                          float* freq_out) {
  if (!plan) return IRS_ERR_ARG;
  if (!plan->mlp) return IRS_ERR_UNSUPPORTED;
  irs_status st = irs::mlp_set_params(plan, theta_in, freq_in);
  if (st != IRS_OK) return st;
  return irs::mlp_get_params(plan, theta_out, freq_out);
}

irs_status irs_mlp_grad(irs_plan_t* plan, const float* x, const float* t, int64_t n, float* grad,
                        double* loss_sum, void* stream) {
  if (!plan) return IRS_ERR_ARG;
  if (!plan->mlp) return IRS_ERR_UNSUPPORTED;
  return irs::mlp_grad(plan, x, t, n, grad, loss_sum, static_cast<cudaStream_t>(stream));
}

irs_status irs_mlp_forward(irs_plan_t* plan, const float* x, int64_t n, float* y, void* stream) {
  if (!plan || n < 0 || (n > 0 && (!x || !y))) return IRS_ERR_ARG;
  if (!plan->mlp) return IRS_ERR_UNSUPPORTED;
  return irs::mlp_forward(plan, x, n, y, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
