// irs_fft.cuh -- complex FFTs of length 2^a 3^b (a >= 1) in shared memory
// (irs_fft.cu), in double-float arithmetic on float4 values (re.hi, re.lo,
// im.hi, im.lo; irs_df.cuh) or in FP32 on float2 values (re, im).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace irs {

constexpr int FFT_MAX_ELEMS = 9216;  // double-float complex values of the largest line buffer a CTA
                                     // may hold (144 KB; with its 72 KB twiddle table 216 KB)
constexpr int FFT_MAX_LEN = 9216;    // longest line (3^2 2^10)

// One batched pass of 1-D FFTs over `n_lines` lines of length L.
struct FftLines {
  int L, n3, n2, B;         // line length L = 3^n3 2^n2, lines per CTA
  int in_len, out_len;      // valid input elements (rest zero), outputs written
  int64_t n_lines;
  int64_t in_line_stride, in_elem_stride, out_line_stride, out_elem_stride;
  int64_t in_grid_stride, out_grid_stride;  // between grids of a batch (gridDim.y)
  double scale;  // applied to the outputs (1: none)
};

// A padded Nx x Ny spectrum layout with its twiddle tables.
struct Fft2d {
  int Nx, Ny;        // 3^n3 2^n2 each
  int n3x, n2x, n3y, n2y;
  float4* tw_x;  // W_N^t, t < N/2, as double-float complex
  float4* tw_y;
};

// Smallest length 2^a 3^b >= n_min with a >= 1 and at most FFT_MAX_LEN, or -1;
// its radix-3 and radix-2 stage counts.
int fft_good_size(int64_t n_min, int* n3, int* n2);
cudaError_t fft_twiddles(int L, float4** d_tw);
cudaError_t fft_setup_attributes();
// compact [ngrids][ny][nx] -> padded spectra [ngrids][Ny][Nx], each axis in
// the forward transform's own order (the mixed-radix digit reversal of the
// frequency index): only pointwise products and sums of spectra made by these
// transforms are meaningful before fft2d_inverse, which expects that order
cudaError_t fft2d_forward(const float4* compact, int64_t nx, int64_t ny, int64_t in_grid_stride,
                          float4* spec, const Fft2d& f, int ngrids, cudaStream_t s);
cudaError_t fft2d_forward(const float2* compact, int64_t nx, int64_t ny, int64_t in_grid_stride,
                          float2* spec, const Fft2d& f, int ngrids, cudaStream_t s);
// padded spectra (overwritten) -> compact [ngrids][ny][nx], unnormalised (the
// 1/(Nx Ny) is the caller's)
cudaError_t fft2d_inverse(float4* spec, const Fft2d& f, int64_t nx, int64_t ny, float4* compact,
                          int64_t out_grid_stride, int ngrids, cudaStream_t s);
cudaError_t fft2d_inverse(float2* spec, const Fft2d& f, int64_t nx, int64_t ny, float2* compact,
                          int64_t out_grid_stride, int ngrids, cudaStream_t s);

}  // namespace irs
