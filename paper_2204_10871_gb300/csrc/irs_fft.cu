// irs_fft.cu -- FP64 complex 2-D FFTs of power-of-two size for the far-field
// convolution on the level-1 cell grid.
//
// A CTA loads B lines of length L (B*L <= 8192 complex doubles, 128 KB) into
// shared memory in bit-reversed order, runs log2(L) radix-2 butterfly stages
// with a twiddle table staged beside them, and writes the lines back.  Rows
// are contiguous lines; columns are strided lines, loaded B adjacent columns
// at a time so that each row segment is one coalesced 16*B-byte access.
// Zero padding is implicit: input elements at or beyond `in_len` read as 0,
// and only the first `out_len` outputs of a line are written.
#include <math.h>

#include <vector>

#include "irs_fft.cuh"

namespace irs {

namespace {

__device__ __forceinline__ double2 cmul2(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ unsigned bitrev(unsigned x, int bits) { return __brev(x) >> (32 - bits); }

template <bool INV>
__global__ void __launch_bounds__(512) k_fft_lines(const double2* in, double2* out,
                                                   FftLines d, const double2* __restrict__ tw) {
  extern __shared__ double2 sm[];
  double2* x = sm;                           // [B][L]
  double2* w = sm + (size_t)d.B * d.L;       // [L/2]
  const int L = d.L, B = d.B, logL = d.logL;
  const int64_t line0 = (int64_t)blockIdx.x * B;
  const int64_t goff_in = (int64_t)blockIdx.y * d.in_grid_stride;
  const int64_t goff_out = (int64_t)blockIdx.y * d.out_grid_stride;
  const int nthr = blockDim.x;
  for (int k = threadIdx.x; k < L / 2; k += nthr) w[k] = tw[k];
  // load, bit-reversed
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
    double2 v = make_double2(0.0, 0.0);
    if (line < d.n_lines && e < d.in_len)
      v = in[goff_in + line * d.in_line_stride + (int64_t)e * d.in_elem_stride];
    x[b * L + bitrev((unsigned)e, logL)] = v;
  }
  __syncthreads();
  for (int s = 1; s <= logL; ++s) {
    const int half = 1 << (s - 1);
    for (int t = threadIdx.x; t < B * (L / 2); t += nthr) {
      const int b = t / (L / 2), k = t % (L / 2);
      const int j = k & (half - 1);
      const int i0 = ((k >> (s - 1)) << s) + j, i1 = i0 + half;
      double2 tw_ = w[j << (logL - s)];
      if (INV) tw_.y = -tw_.y;
      const double2 u = x[b * L + i0];
      const double2 v = cmul2(x[b * L + i1], tw_);
      x[b * L + i0] = make_double2(u.x + v.x, u.y + v.y);
      x[b * L + i1] = make_double2(u.x - v.x, u.y - v.y);
    }
    __syncthreads();
  }
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
      double2 v = x[b * L + e];
      v.x *= d.scale;
      v.y *= d.scale;
      out[goff_out + line * d.out_line_stride + (int64_t)e * d.out_elem_stride] = v;
    }
  }
}

}  // namespace

int ilog2_exact(int64_t n) {
  int l = 0;
  while (((int64_t)1 << l) < n) ++l;
  return ((int64_t)1 << l) == n ? l : -1;
}

cudaError_t fft_twiddles(int L, double2** d_tw) {
  std::vector<double2> h((size_t)(L / 2 > 0 ? L / 2 : 1));
  for (int k = 0; k < L / 2; ++k) {
    const double a = -2.0 * M_PI * (double)k / (double)L;
    h[k] = make_double2(cos(a), sin(a));
  }
  cudaError_t e = cudaMalloc(d_tw, h.size() * sizeof(double2));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*d_tw, h.data(), h.size() * sizeof(double2), cudaMemcpyHostToDevice);
}

cudaError_t fft_setup_attributes() {
  const int max_smem = (int)(FFT_MAX_ELEMS * sizeof(double2) + FFT_MAX_LEN / 2 * sizeof(double2));
  cudaError_t e = cudaFuncSetAttribute(k_fft_lines<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_fft_lines<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
}

cudaError_t fft_lines(const double2* in, double2* out, FftLines d, int ngrids, const double2* tw,
                      bool inverse, cudaStream_t s) {
  if (d.n_lines <= 0 || ngrids <= 0) return cudaSuccess;
  const int64_t blocks = (d.n_lines + d.B - 1) / d.B;
  const size_t smem = (size_t)d.B * d.L * sizeof(double2) + (size_t)(d.L / 2) * sizeof(double2);
  const int threads = d.B * d.L / 2 >= 512 ? 512 : (d.B * d.L / 2 >= 32 ? d.B * d.L / 2 : 32);
  dim3 grid((unsigned)blocks, (unsigned)ngrids);
  if (inverse)
    k_fft_lines<true><<<grid, threads, smem, s>>>(in, out, d, tw);
  else
    k_fft_lines<false><<<grid, threads, smem, s>>>(in, out, d, tw);
  return cudaGetLastError();
}

// Lines per CTA for a line length L: fill the 8192-element shared buffer.
static int lines_per_cta(int L) {
  int B = FFT_MAX_ELEMS / L;
  return B < 1 ? 1 : (B > 16 ? 16 : B);
}

cudaError_t fft2d_forward(const double2* compact, int64_t nx, int64_t ny, int64_t in_grid_stride,
                          double2* spec, const Fft2d& f, int ngrids, cudaStream_t s) {
  // rows: compact rows [0, ny) -> spectrum rows, zero-padded to Nx
  FftLines r{};
  r.L = f.Nx; r.logL = f.logNx; r.B = lines_per_cta(f.Nx);
  r.n_lines = ny; r.in_len = (int)nx; r.out_len = f.Nx;
  r.in_line_stride = nx; r.in_elem_stride = 1; r.out_line_stride = f.Nx; r.out_elem_stride = 1;
  r.in_grid_stride = in_grid_stride; r.out_grid_stride = (int64_t)f.Nx * f.Ny; r.scale = 1.0;
  cudaError_t e = fft_lines(compact, spec, r, ngrids, f.tw_x, false, s);
  if (e != cudaSuccess) return e;
  // columns: all Nx, rows >= ny read as zero
  FftLines c{};
  c.L = f.Ny; c.logL = f.logNy; c.B = lines_per_cta(f.Ny);
  c.n_lines = f.Nx; c.in_len = (int)ny; c.out_len = f.Ny;
  c.in_line_stride = 1; c.in_elem_stride = f.Nx; c.out_line_stride = 1; c.out_elem_stride = f.Nx;
  c.in_grid_stride = (int64_t)f.Nx * f.Ny; c.out_grid_stride = (int64_t)f.Nx * f.Ny; c.scale = 1.0;
  return fft_lines(spec, spec, c, ngrids, f.tw_y, false, s);
}

cudaError_t fft2d_inverse(double2* spec, const Fft2d& f, int64_t nx, int64_t ny, double2* compact,
                          int64_t out_grid_stride, int ngrids, cudaStream_t s) {
  FftLines c{};
  c.L = f.Ny; c.logL = f.logNy; c.B = lines_per_cta(f.Ny);
  c.n_lines = f.Nx; c.in_len = f.Ny; c.out_len = (int)ny;
  c.in_line_stride = 1; c.in_elem_stride = f.Nx; c.out_line_stride = 1; c.out_elem_stride = f.Nx;
  c.in_grid_stride = (int64_t)f.Nx * f.Ny; c.out_grid_stride = (int64_t)f.Nx * f.Ny; c.scale = 1.0;
  cudaError_t e = fft_lines(spec, spec, c, ngrids, f.tw_y, true, s);
  if (e != cudaSuccess) return e;
  FftLines r{};
  r.L = f.Nx; r.logL = f.logNx; r.B = lines_per_cta(f.Nx);
  r.n_lines = ny; r.in_len = f.Nx; r.out_len = (int)nx;
  r.in_line_stride = f.Nx; r.in_elem_stride = 1; r.out_line_stride = nx; r.out_elem_stride = 1;
  r.in_grid_stride = (int64_t)f.Nx * f.Ny; r.out_grid_stride = out_grid_stride;
  r.scale = 1.0 / ((double)f.Nx * (double)f.Ny);
  return fft_lines(spec, compact, r, ngrids, f.tw_x, true, s);
}

}  // namespace irs
