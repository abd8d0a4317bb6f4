// irs_fft.cu -- complex 2-D FFTs of length 2^a 3^b for the far-field
// convolution on the level-1 cell grid, in double-float arithmetic
// (irs_df.cuh: 48-bit significands on the FP32 pipes; float4 elements) or in
// FP32 (float2 elements).
//
// A CTA loads B lines of length L = 3^n3 2^n2 into shared memory (B as large
// as keeps the CTA within 52 KB, so that up to four CTAs share an SM; at
// least one line, up to 9216 double-float or FP32 values), runs in-place
// butterfly stages with a twiddle table W_L^t (t < L/2; W_L^(t + L/2) =
// -W_L^t) staged beside them, and writes the lines back.  Neither direction
// permutes: the forward transform runs decimation in frequency (n2 radix-2
// then n3 radix-3 stages) on natural-order input and leaves X[k] at the
// mixed-radix digit reversal of k; the inverse runs decimation in time (n3
// radix-3 then n2 radix-2 stages), which takes its input in exactly that
// order and returns natural order.  The convolution between them is
// pointwise, so the spectra never need sorting.
// Rows are contiguous lines; columns are strided lines, loaded B adjacent
// columns at a time so that each row segment is one coalesced access.  Zero padding is implicit: input elements at or beyond
// `in_len` read as 0, and only the first `out_len` outputs of a line are
// written.
#include <math.h>

#include <vector>

#include "irs_df.cuh"
#include "irs_fft.cuh"

namespace irs {

namespace {

// Complex arithmetic of the two element types: float4 is double-float
// (re.hi, re.lo, im.hi, im.lo), float2 is FP32 (re, im).
__device__ __forceinline__ float4 c_add(float4 a, float4 b) { return dfc_add(a, b); }
__device__ __forceinline__ float4 c_sub(float4 a, float4 b) { return dfc_sub(a, b); }
__device__ __forceinline__ float4 c_mul(float4 a, float4 b) { return dfc_mul(a, b); }
__device__ __forceinline__ float4 c_neg(float4 a) { return make_float4(-a.x, -a.y, -a.z, -a.w); }
__device__ __forceinline__ float4 c_conj(float4 a) { return make_float4(a.x, a.y, -a.z, -a.w); }
__device__ __forceinline__ float4 c_half(float4 a) { return make_float4(0.5f * a.x, 0.5f * a.y, 0.5f * a.z, 0.5f * a.w); }
__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 c_mul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 c_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 c_conj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 c_half(float2 a) { return make_float2(0.5f * a.x, 0.5f * a.y); }

template <class T> __device__ __forceinline__ T c_zero();
template <> __device__ __forceinline__ float4 c_zero<float4>() { return make_float4(0.f, 0.f, 0.f, 0.f); }
template <> __device__ __forceinline__ float2 c_zero<float2>() { return make_float2(0.f, 0.f); }

// twiddle table entry in the element type (the table holds double-float)
template <class T> __device__ __forceinline__ T tw_elem(float4 v);
template <> __device__ __forceinline__ float4 tw_elem<float4>(float4 v) { return v; }
template <> __device__ __forceinline__ float2 tw_elem<float2>(float4 v) { return make_float2(v.x, v.z); }

// output scaling by a real factor
__device__ __forceinline__ float4 c_scale(float4 a, double s) {
  return dfc_scale(a, make_float2((float)s, (float)(s - (double)(float)s)));
}
__device__ __forceinline__ float2 c_scale(float2 a, double s) {
  const float f = (float)s;
  return make_float2(a.x * f, a.y * f);
}

// Radix-3 butterfly on a and the twiddled p, q:
// x0 = a + t1, x1,2 = a - t1/2 -+ i s3 (p - q) with t1 = p + q and
// s3 = +-sqrt(3)/2 (the sign of the transform's exponent).
__device__ __forceinline__ void radix3(float4 a, float4 p, float4 q, bool inv, float4& x0, float4& x1,
                                       float4& x2) {
  const float2 s3 = inv ? make_float2(-8.660253882e-01f, -1.554362505e-08f)
                        : make_float2(8.660253882e-01f, 1.554362505e-08f);  // sqrt(3)/2 = hi + lo
  const float4 t1 = dfc_add(p, q);
  const float4 t2 = dfc_sub(a, c_half(t1));
  const float4 dd = dfc_sub(p, q);
  const float2 u = df_mul(s3, dfc_im(dd)), v = df_mul(s3, dfc_re(dd));  // s3 Im(dd), s3 Re(dd)
  x0 = dfc_add(a, t1);
  x1 = dfc_make(df_add(dfc_re(t2), u), df_sub(dfc_im(t2), v));
  x2 = dfc_make(df_sub(dfc_re(t2), u), df_add(dfc_im(t2), v));
}
__device__ __forceinline__ void radix3(float2 a, float2 p, float2 q, bool inv, float2& x0, float2& x1,
                                       float2& x2) {
  const float s3 = inv ? -0.8660254038f : 0.8660254038f;
  const float2 t1 = c_add(p, q);
  const float2 t2 = c_sub(a, c_half(t1));
  const float2 dd = c_sub(p, q);
  const float u = s3 * dd.y, v = s3 * dd.x;
  x0 = c_add(a, t1);
  x1 = make_float2(t2.x + u, t2.y - v);
  x2 = make_float2(t2.x - u, t2.y + v);
}

// Quotient by a divisor d that is fixed for a loop: umulhi(x, ceil(2^32 / d))
// equals floor(x / d) whenever x d < 2^32 (here x < 2^15 and d < 2^14), with
// no division instruction sequence per element.
struct FastDiv {
  uint32_t d, m;
  __device__ explicit FastDiv(uint32_t dv) : d(dv), m(dv > 1u ? 0xFFFFFFFFu / dv + 1u : 0u) {}
  __device__ __forceinline__ uint32_t div(uint32_t x) const { return d > 1u ? __umulhi(x, m) : x; }
};

// W_L^t for 0 <= t < L from the half table, conjugated for the inverse
template <bool INV, class T>
__device__ __forceinline__ T tw_at(const T* w, int t, int half) {
  T v = t < half ? w[t] : c_neg(w[t - half]);
  return INV ? c_conj(v) : v;
}

template <bool INV, class T>
__global__ void __launch_bounds__(512) k_fft_lines(const T* in, T* out, FftLines d, const float4* __restrict__ tw) {
  extern __shared__ float4 sm_raw[];
  T* x = reinterpret_cast<T*>(sm_raw);  // [B][L]
  T* w = x + (size_t)d.B * d.L;         // [L/2]
  const int L = d.L, B = d.B, n3 = d.n3, n2 = d.n2, half_L = L / 2;
  int pow3 = 1;
  for (int i = 0; i < n3; ++i) pow3 *= 3;
  const int64_t line0 = (int64_t)blockIdx.x * B;
  const int64_t goff_in = (int64_t)blockIdx.y * d.in_grid_stride;
  const int64_t goff_out = (int64_t)blockIdx.y * d.out_grid_stride;
  const int nthr = blockDim.x;
  const FastDiv fdL((uint32_t)L), fdB((uint32_t)B), fd3((uint32_t)(L / 3)), fd2((uint32_t)half_L);
  for (int k = threadIdx.x; k < L / 2; k += nthr) w[k] = tw_elem<T>(tw[k]);
  // load (natural order for the forward transform, the forward transform's
  // output order for the inverse)
  for (int idx = threadIdx.x; idx < B * L; idx += nthr) {
    int b, e;
    if (d.in_elem_stride == 1) {
      b = (int)fdL.div((uint32_t)idx);
      e = idx - b * L;
    } else {
      e = (int)fdB.div((uint32_t)idx);
      b = idx - e * B;
    }
    const int64_t line = line0 + b;
    T v = c_zero<T>();
    if (line < d.n_lines && e < d.in_len)
      v = in[goff_in + line * d.in_line_stride + (int64_t)e * d.in_elem_stride];
    x[b * L + e] = v;
  }
  __syncthreads();
  if (!INV) {
    // decimation in frequency: the transposes of the inverse's stages in
    // reverse order -- a radix-2 butterfly adds and subtracts, then twiddles
    // the difference; a radix-3 butterfly transforms, then twiddles outputs
    // 1 and 2
    for (int s = n2 - 1; s >= 0; --s) {
      const int m_prev = pow3 << s, m = 2 * m_prev, stride = L / m;
      const FastDiv fdm((uint32_t)m_prev);
      for (int t = threadIdx.x; t < B * (L / 2); t += nthr) {
        const int b = (int)fd2.div((uint32_t)t), k = t - b * half_L;
        const int g = (int)fdm.div((uint32_t)k), j = k - g * m_prev;
        const int i0 = g * m + j, i1 = i0 + m_prev;
        const T u = x[b * L + i0], v = x[b * L + i1];
        x[b * L + i0] = c_add(u, v);
        x[b * L + i1] = c_mul(c_sub(u, v), tw_at<INV>(w, j * stride, half_L));
      }
      __syncthreads();
    }
    int m_prev = pow3;
    for (int s = n3 - 1; s >= 0; --s) {
      m_prev /= 3;
      const int m = m_prev * 3, stride = L / m;
      const FastDiv fdm((uint32_t)m_prev);
      for (int t = threadIdx.x; t < B * (L / 3); t += nthr) {
        const int b = (int)fd3.div((uint32_t)t), k = t - b * (L / 3);
        const int g = (int)fdm.div((uint32_t)k), j = k - g * m_prev;
        const int i0 = g * m + j, i1 = i0 + m_prev, i2 = i1 + m_prev;
        T y0, y1, y2;
        radix3(x[b * L + i0], x[b * L + i1], x[b * L + i2], INV, y0, y1, y2);
        x[b * L + i0] = y0;
        x[b * L + i1] = c_mul(y1, tw_at<INV>(w, j * stride, half_L));
        x[b * L + i2] = c_mul(y2, tw_at<INV>(w, 2 * j * stride, half_L));
      }
      __syncthreads();
    }
  } else {
    // decimation in time
    int m_prev = 1;  // span of the sub-transforms done so far
    // radix-3 stages: y_q = sum_r (W_m^(j r) x_r) W_3^(q r);
    // W_3 = -1/2 -+ i sqrt(3)/2, the halving is exact
    for (int s = 0; s < n3; ++s) {
      const int m = m_prev * 3, stride = L / m;
      const FastDiv fdm((uint32_t)m_prev);
      for (int t = threadIdx.x; t < B * (L / 3); t += nthr) {
        const int b = (int)fd3.div((uint32_t)t), k = t - b * (L / 3);
        const int g = (int)fdm.div((uint32_t)k), j = k - g * m_prev;
        const int i0 = g * m + j, i1 = i0 + m_prev, i2 = i1 + m_prev;
        const T a = x[b * L + i0];
        const T p = c_mul(x[b * L + i1], tw_at<INV>(w, j * stride, half_L));
        const T q = c_mul(x[b * L + i2], tw_at<INV>(w, 2 * j * stride, half_L));
        radix3(a, p, q, INV, x[b * L + i0], x[b * L + i1], x[b * L + i2]);
      }
      __syncthreads();
      m_prev = m;
    }
    // radix-2 stages
    for (int s = 0; s < n2; ++s) {
      const int m = m_prev * 2, stride = L / m;
      const FastDiv fdm((uint32_t)m_prev);
      for (int t = threadIdx.x; t < B * (L / 2); t += nthr) {
        const int b = (int)fd2.div((uint32_t)t), k = t - b * half_L;
        const int g = (int)fdm.div((uint32_t)k), j = k - g * m_prev;
        const int i0 = g * m + j, i1 = i0 + m_prev;
        const T u = x[b * L + i0];
        const T v = c_mul(x[b * L + i1], tw_at<INV>(w, j * stride, half_L));
        x[b * L + i0] = c_add(u, v);
        x[b * L + i1] = c_sub(u, v);
      }
      __syncthreads();
      m_prev = m;
    }
  }
  const bool scaled = d.scale != 1.0;
  for (int idx = threadIdx.x; idx < B * L; idx += nthr) {
    int b, e;
    if (d.out_elem_stride == 1) {
      b = (int)fdL.div((uint32_t)idx);
      e = idx - b * L;
    } else {
      e = (int)fdB.div((uint32_t)idx);
      b = idx - e * B;
    }
    const int64_t line = line0 + b;
    if (line < d.n_lines && e < d.out_len) {
      T v = x[b * L + e];
      if (scaled) v = c_scale(v, d.scale);
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
  cudaError_t e = cudaFuncSetAttribute(k_fft_lines<false, float4>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_fft_lines<true, float4>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_fft_lines<false, float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_fft_lines<true, float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  return e;
}

namespace {

template <class T>
cudaError_t fft_lines_t(const T* in, T* out, FftLines d, int ngrids, const float4* tw, bool inverse,
                        cudaStream_t s) {
  if (d.n_lines <= 0 || ngrids <= 0) return cudaSuccess;
  const int64_t blocks = (d.n_lines + d.B - 1) / d.B;
  const size_t smem = (size_t)d.B * d.L * sizeof(T) + (size_t)(d.L / 2) * sizeof(T);
  const int threads = d.B * d.L / 2 >= 512 ? 512 : (d.B * d.L / 2 >= 32 ? d.B * d.L / 2 : 32);
  dim3 grid((unsigned)blocks, (unsigned)ngrids);
  if (inverse)
    k_fft_lines<true, T><<<grid, threads, smem, s>>>(in, out, d, tw);
  else
    k_fft_lines<false, T><<<grid, threads, smem, s>>>(in, out, d, tw);
  return cudaGetLastError();
}

// Lines per CTA for a line length L: as many as keep the CTA's lines and
// twiddle table within a quarter of the SM's shared memory, so that up to four
// CTAs share an SM and hide each other's barriers; at least one line.
constexpr size_t FFT_CTA_BYTES = 52 * 1024;
template <class T>
int lines_per_cta(int L) {
  const size_t tw = (size_t)(L / 2) * sizeof(T), line = (size_t)L * sizeof(T);
  int B = FFT_CTA_BYTES > tw ? (int)((FFT_CTA_BYTES - tw) / line) : 0;
  return B < 1 ? 1 : (B > 16 ? 16 : B);
}

template <class T>
cudaError_t fft2d_forward_t(const T* compact, int64_t nx, int64_t ny, int64_t in_grid_stride, T* spec,
                            const Fft2d& f, int ngrids, cudaStream_t s) {
  // rows: compact rows [0, ny) -> spectrum rows, zero-padded to Nx
  FftLines r{};
  r.L = f.Nx; r.n3 = f.n3x; r.n2 = f.n2x; r.B = lines_per_cta<T>(f.Nx);
  r.n_lines = ny; r.in_len = (int)nx; r.out_len = f.Nx;
  r.in_line_stride = nx; r.in_elem_stride = 1; r.out_line_stride = f.Nx; r.out_elem_stride = 1;
  r.in_grid_stride = in_grid_stride; r.out_grid_stride = (int64_t)f.Nx * f.Ny; r.scale = 1.0;
  cudaError_t e = fft_lines_t(compact, spec, r, ngrids, f.tw_x, false, s);
  if (e != cudaSuccess) return e;
  // columns: all Nx, rows >= ny read as zero
  FftLines c{};
  c.L = f.Ny; c.n3 = f.n3y; c.n2 = f.n2y; c.B = lines_per_cta<T>(f.Ny);
  c.n_lines = f.Nx; c.in_len = (int)ny; c.out_len = f.Ny;
  c.in_line_stride = 1; c.in_elem_stride = f.Nx; c.out_line_stride = 1; c.out_elem_stride = f.Nx;
  c.in_grid_stride = (int64_t)f.Nx * f.Ny; c.out_grid_stride = (int64_t)f.Nx * f.Ny; c.scale = 1.0;
  return fft_lines_t(spec, spec, c, ngrids, f.tw_y, false, s);
}

template <class T>
cudaError_t fft2d_inverse_t(T* spec, const Fft2d& f, int64_t nx, int64_t ny, T* compact, int64_t out_grid_stride,
                            int ngrids, cudaStream_t s) {
  FftLines c{};
  c.L = f.Ny; c.n3 = f.n3y; c.n2 = f.n2y; c.B = lines_per_cta<T>(f.Ny);
  c.n_lines = f.Nx; c.in_len = f.Ny; c.out_len = (int)ny;
  c.in_line_stride = 1; c.in_elem_stride = f.Nx; c.out_line_stride = 1; c.out_elem_stride = f.Nx;
  c.in_grid_stride = (int64_t)f.Nx * f.Ny; c.out_grid_stride = (int64_t)f.Nx * f.Ny; c.scale = 1.0;
  cudaError_t e = fft_lines_t(spec, spec, c, ngrids, f.tw_y, true, s);
  if (e != cudaSuccess) return e;
  FftLines r{};
  r.L = f.Nx; r.n3 = f.n3x; r.n2 = f.n2x; r.B = lines_per_cta<T>(f.Nx);
  r.n_lines = ny; r.in_len = f.Nx; r.out_len = (int)nx;
  r.in_line_stride = f.Nx; r.in_elem_stride = 1; r.out_line_stride = nx; r.out_elem_stride = 1;
  r.in_grid_stride = (int64_t)f.Nx * f.Ny; r.out_grid_stride = out_grid_stride;
  r.scale = 1.0;
  return fft_lines_t(spec, compact, r, ngrids, f.tw_x, true, s);
}

}  // namespace

cudaError_t fft2d_forward(const float4* compact, int64_t nx, int64_t ny, int64_t in_grid_stride, float4* spec,
                          const Fft2d& f, int ngrids, cudaStream_t s) {
  return fft2d_forward_t(compact, nx, ny, in_grid_stride, spec, f, ngrids, s);
}
cudaError_t fft2d_forward(const float2* compact, int64_t nx, int64_t ny, int64_t in_grid_stride, float2* spec,
                          const Fft2d& f, int ngrids, cudaStream_t s) {
  return fft2d_forward_t(compact, nx, ny, in_grid_stride, spec, f, ngrids, s);
}
cudaError_t fft2d_inverse(float4* spec, const Fft2d& f, int64_t nx, int64_t ny, float4* compact,
                          int64_t out_grid_stride, int ngrids, cudaStream_t s) {
  return fft2d_inverse_t(spec, f, nx, ny, compact, out_grid_stride, ngrids, s);
}
cudaError_t fft2d_inverse(float2* spec, const Fft2d& f, int64_t nx, int64_t ny, float2* compact,
                          int64_t out_grid_stride, int ngrids, cudaStream_t s) {
  return fft2d_inverse_t(spec, f, nx, ny, compact, out_grid_stride, ngrids, s);
}

}  // namespace irs
