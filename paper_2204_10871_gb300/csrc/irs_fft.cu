// irs_fft.cu -- complex 2-D FFTs of length 2^a 3^b for the far-field
// convolution on the level-1 cell grid, in double-float arithmetic
// (irs_df.cuh: 48-bit significands on the FP32 pipes).
//
// A CTA loads B lines of length L = 3^n3 2^n2 (B*L <= 9216 complex values,
// 144 KB) into shared memory in mixed-radix digit-reversed order, runs n3
// radix-3 then n2 radix-2 in-place decimation-in-time stages with a twiddle
// table W_L^t (t < L/2; W_L^(t + L/2) = -W_L^t) staged beside them, and writes
// the lines back.  Rows are contiguous lines; columns are strided lines, loaded
// B adjacent columns at a time so that each row segment is one coalesced
// 16*B-byte access.  Zero padding is implicit: input elements at or beyond
// `in_len` read as 0, and only the first `out_len` outputs of a line are
// written.
#include <math.h>

#include <vector>

#include "irs_df.cuh"
#include "irs_fft.cuh"

namespace irs {

namespace {

// Where input element e goes for the in-place decimation-in-time stages (n3
// radix-3 stages, then n2 radix-2): the n2 low bits of e reversed, times 3^n3,
// plus the n3 base-3 digits of e >> n2 reversed.  (For n3 = 0 this is the
// bit reversal; for n3 > 0 the permutation is not its own inverse.)
__device__ __forceinline__ unsigned digit_pos(unsigned e, int n3, int n2, unsigned pow3) {
  const unsigned lo = e & ((1u << n2) - 1u);
  unsigned hi = e >> n2, r3 = 0;
  for (int i = 0; i < n3; ++i) {
    const unsigned q = hi / 3u;
    r3 = r3 * 3u + (hi - 3u * q);
    hi = q;
  }
  return r3 + pow3 * (n2 > 0 ? (__brev(lo) >> (32 - n2)) : 0u);
}

// W_L^t for 0 <= t < L from the half table, conjugated for the inverse
template <bool INV>
__device__ __forceinline__ float4 tw_at(const float4* w, int t, int half) {
  float4 v = t < half ? w[t] : w[t - half];
  if (t >= half) v = make_float4(-v.x, -v.y, -v.z, -v.w);
  if (INV) {
    v.z = -v.z;
    v.w = -v.w;
  }
  return v;
}

template <bool INV>
__global__ void __launch_bounds__(512) k_fft_lines(const float4* in, float4* out, FftLines d,
                                                   const float4* __restrict__ tw) {
  extern __shared__ float4 sm[];
  float4* x = sm;                           // [B][L]
  float4* w = sm + (size_t)d.B * d.L;       // [L/2]
  const int L = d.L, B = d.B, n3 = d.n3, n2 = d.n2, half_L = L / 2;
  unsigned pow3 = 1;
  for (int i = 0; i < n3; ++i) pow3 *= 3u;
  const int64_t line0 = (int64_t)blockIdx.x * B;
  const int64_t goff_in = (int64_t)blockIdx.y * d.in_grid_stride;
  const int64_t goff_out = (int64_t)blockIdx.y * d.out_grid_stride;
  const int nthr = blockDim.x;
  for (int k = threadIdx.x; k < L / 2; k += nthr) w[k] = tw[k];
  // load, digit-reversed
  for (int idx = threadIdx.x; idx < B * L; idx += nthr) {
    int b, e;
    if (d.in_elem_stride == 1) {
      b = idx / L;
      e = idx % L;
    } else {
      b = idx % B;
      e = idx / B;
    }
    const int64_t line = line0 + b;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (line < d.n_lines && e < d.in_len)
      v = in[goff_in + line * d.in_line_stride + (int64_t)e * d.in_elem_stride];
    x[b * L + digit_pos((unsigned)e, n3, n2, pow3)] = v;
  }
  __syncthreads();
  int m_prev = 1;  // span of the sub-transforms done so far
  // radix-3 stages: y_q = sum_r (W_m^(j r) x_r) W_3^(q r);
  // W_3 = -1/2 -+ i sqrt(3)/2, the halving is exact
  const float2 s3 = INV ? make_float2(-8.660253882e-01f, -1.554362505e-08f)
                        : make_float2(8.660253882e-01f, 1.554362505e-08f);  // sqrt(3)/2 = hi + lo
  for (int s = 0; s < n3; ++s) {
    const int m = m_prev * 3, stride = L / m;
    for (int t = threadIdx.x; t < B * (L / 3); t += nthr) {
      const int b = t / (L / 3), k = t % (L / 3);
      const int j = k % m_prev;
      const int i0 = (k / m_prev) * m + j, i1 = i0 + m_prev, i2 = i1 + m_prev;
      const float4 a = x[b * L + i0];
      const float4 p = dfc_mul(x[b * L + i1], tw_at<INV>(w, j * stride, half_L));
      const float4 q = dfc_mul(x[b * L + i2], tw_at<INV>(w, 2 * j * stride, half_L));
      const float4 t1 = dfc_add(p, q);
      const float4 t2 = dfc_sub(a, make_float4(0.5f * t1.x, 0.5f * t1.y, 0.5f * t1.z, 0.5f * t1.w));
      const float4 dd = dfc_sub(p, q);
      const float2 u = df_mul(s3, dfc_im(dd)), v = df_mul(s3, dfc_re(dd));  // s3 Im(dd), s3 Re(dd)
      x[b * L + i0] = dfc_add(a, t1);
      x[b * L + i1] = dfc_make(df_add(dfc_re(t2), u), df_sub(dfc_im(t2), v));
      x[b * L + i2] = dfc_make(df_sub(dfc_re(t2), u), df_add(dfc_im(t2), v));
    }
    __syncthreads();
    m_prev = m;
  }
  // radix-2 stages
  for (int s = 0; s < n2; ++s) {
    const int m = m_prev * 2, stride = L / m;
    for (int t = threadIdx.x; t < B * (L / 2); t += nthr) {
      const int b = t / (L / 2), k = t % (L / 2);
      const int j = k % m_prev;
      const int i0 = (k / m_prev) * m + j, i1 = i0 + m_prev;
      const float4 u = x[b * L + i0];
      const float4 v = dfc_mul(x[b * L + i1], tw_at<INV>(w, j * stride, half_L));
      x[b * L + i0] = dfc_add(u, v);
      x[b * L + i1] = dfc_sub(u, v);
    }
    __syncthreads();
    m_prev = m;
  }
  const bool scaled = d.scale != 1.0;
  const float2 sc = make_float2((float)d.scale, (float)(d.scale - (double)(float)d.scale));
  for (int idx = threadIdx.x; idx < B * L; idx += nthr) {
    int b, e;
    if (d.out_elem_stride == 1) {
      b = idx / L;
      e = idx % L;
    } else {
      b = idx % B;
      e = idx / B;
    }
    const int64_t line = line0 + b;
    if (line < d.n_lines && e < d.out_len) {
      float4 v = x[b * L + e];
      if (scaled) v = dfc_scale(v, sc);
      out[goff_out + line * d.out_line_stride + (int64_t)e * d.out_elem_stride] = v;
    }
  }
}

}  // namespace

int fft_good_size(int64_t n_min, int* n3, int* n2) {
  int64_t best = -1;
  int b3 = 0, b2 = 0;
  int64_t p3 = 1;
  for (int i3 = 0; p3 <= FFT_MAX_LEN; ++i3, p3 *= 3) {
    int64_t v = p3 * 2;
    int i2 = 1;
    while (v < n_min) {
      v *= 2;
      ++i2;
    }
    if (v <= FFT_MAX_LEN && (best < 0 || v < best)) {
      best = v;
      b3 = i3;
      b2 = i2;
    }
  }
  if (best < 0) return -1;
  *n3 = b3;
  *n2 = b2;
  return (int)best;
}

cudaError_t fft_twiddles(int L, float4** d_tw) {
  std::vector<float4> h((size_t)(L / 2 > 0 ? L / 2 : 1));
  for (int k = 0; k < L / 2; ++k) {
    const double a = -2.0 * M_PI * (double)k / (double)L;
    h[k] = dfc_from_double(cos(a), sin(a));
  }
  cudaError_t e = cudaMalloc(d_tw, h.size() * sizeof(float4));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*d_tw, h.data(), h.size() * sizeof(float4), cudaMemcpyHostToDevice);
}

cudaError_t fft_setup_attributes() {
  const int max_smem = (int)(FFT_MAX_ELEMS * sizeof(float4) + FFT_MAX_LEN / 2 * sizeof(float4));
  cudaError_t e = cudaFuncSetAttribute(k_fft_lines<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_fft_lines<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
}

cudaError_t fft_lines(const float4* in, float4* out, FftLines d, int ngrids, const float4* tw,
                      bool inverse, cudaStream_t s) {
  if (d.n_lines <= 0 || ngrids <= 0) return cudaSuccess;
  const int64_t blocks = (d.n_lines + d.B - 1) / d.B;
  const size_t smem = (size_t)d.B * d.L * sizeof(float4) + (size_t)(d.L / 2) * sizeof(float4);
  const int threads = d.B * d.L / 2 >= 512 ? 512 : (d.B * d.L / 2 >= 32 ? d.B * d.L / 2 : 32);
  dim3 grid((unsigned)blocks, (unsigned)ngrids);
  if (inverse)
    k_fft_lines<true><<<grid, threads, smem, s>>>(in, out, d, tw);
  else
    k_fft_lines<false><<<grid, threads, smem, s>>>(in, out, d, tw);
  return cudaGetLastError();
}

// Lines per CTA for a line length L: fill the shared line buffer.
static int lines_per_cta(int L) {
  int B = FFT_MAX_ELEMS / L;
  return B < 1 ? 1 : (B > 16 ? 16 : B);
}

cudaError_t fft2d_forward(const float4* compact, int64_t nx, int64_t ny, int64_t in_grid_stride,
                          float4* spec, const Fft2d& f, int ngrids, cudaStream_t s) {
  // rows: compact rows [0, ny) -> spectrum rows, zero-padded to Nx
  FftLines r{};
  r.L = f.Nx; r.n3 = f.n3x; r.n2 = f.n2x; r.B = lines_per_cta(f.Nx);
  r.n_lines = ny; r.in_len = (int)nx; r.out_len = f.Nx;
  r.in_line_stride = nx; r.in_elem_stride = 1; r.out_line_stride = f.Nx; r.out_elem_stride = 1;
  r.in_grid_stride = in_grid_stride; r.out_grid_stride = (int64_t)f.Nx * f.Ny; r.scale = 1.0;
  cudaError_t e = fft_lines(compact, spec, r, ngrids, f.tw_x, false, s);
  if (e != cudaSuccess) return e;
  // columns: all Nx, rows >= ny read as zero
  FftLines c{};
  c.L = f.Ny; c.n3 = f.n3y; c.n2 = f.n2y; c.B = lines_per_cta(f.Ny);
  c.n_lines = f.Nx; c.in_len = (int)ny; c.out_len = f.Ny;
  c.in_line_stride = 1; c.in_elem_stride = f.Nx; c.out_line_stride = 1; c.out_elem_stride = f.Nx;
  c.in_grid_stride = (int64_t)f.Nx * f.Ny; c.out_grid_stride = (int64_t)f.Nx * f.Ny; c.scale = 1.0;
  return fft_lines(spec, spec, c, ngrids, f.tw_y, false, s);
}

cudaError_t fft2d_inverse(float4* spec, const Fft2d& f, int64_t nx, int64_t ny, float4* compact,
                          int64_t out_grid_stride, int ngrids, cudaStream_t s) {
  FftLines c{};
  c.L = f.Ny; c.n3 = f.n3y; c.n2 = f.n2y; c.B = lines_per_cta(f.Ny);
  c.n_lines = f.Nx; c.in_len = f.Ny; c.out_len = (int)ny;
  c.in_line_stride = 1; c.in_elem_stride = f.Nx; c.out_line_stride = 1; c.out_elem_stride = f.Nx;
  c.in_grid_stride = (int64_t)f.Nx * f.Ny; c.out_grid_stride = (int64_t)f.Nx * f.Ny; c.scale = 1.0;
  cudaError_t e = fft_lines(spec, spec, c, ngrids, f.tw_y, true, s);
  if (e != cudaSuccess) return e;
  FftLines r{};
  r.L = f.Nx; r.n3 = f.n3x; r.n2 = f.n2x; r.B = lines_per_cta(f.Nx);
  r.n_lines = ny; r.in_len = f.Nx; r.out_len = (int)nx;
  r.in_line_stride = f.Nx; r.in_elem_stride = 1; r.out_line_stride = nx; r.out_elem_stride = 1;
  r.in_grid_stride = (int64_t)f.Nx * f.Ny; r.out_grid_stride = out_grid_stride;
  r.scale = 1.0;
  return fft_lines(spec, compact, r, ngrids, f.tw_x, true, s);
}

}  // namespace irs
