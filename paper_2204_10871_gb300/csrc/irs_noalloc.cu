// irs_noalloc.cu -- an allocation-free variant of the brute-force map.
//
// Some callers cannot allocate device memory: code that runs while another
// memory manager owns the device (a framework's caching allocator, or a fixed
// pool carved out at start-up), plug-ins that must not trigger the implicit
// device-wide synchronisation of cudaMalloc / cudaFree, and latency-critical
// loops in which one allocation would stall every stream.  This entry point
// serves them: it takes the parameters directly instead of a plan, and keeps
// all of its scratch (mass partial sums, the status word, the per-tile FP64
// setup records) in one file-scope __device__ array, so it allocates nothing.
// Inputs and outputs are still the caller's buffers.
//
// The array is part of the library image: every GPU that loads the library's
// device code holds its 7.9 MB until the process exits.  CUDA loads device
// code lazily by default, so on a device where nothing of the library has run
// yet, the first call loads it and the array is allocated then, by the
// driver.  Its device address is looked up with cudaGetSymbolAddress on the
// first call made on each device (with that device current).  Make that
// first call before any stream capture and outside latency-critical loops;
// later calls allocate nothing.  All calls
// share the one array and it keeps the last call's contents, so calls whose
// work overlaps on the GPU (different streams, or different host threads
// without ordering) race on it.
#include <math.h>
#include <string.h>

#include <mutex>

#include "irs_common.cuh"

namespace {

// Tiles of 32 x 64 rays: 49,152 tiles cover lattices of up to 100,663,296 rays.
constexpr int64_t NOALLOC_MAX_TILES = 49152;
constexpr size_t OFF_MSUM = 0;
constexpr size_t OFF_MPART = 256;
constexpr size_t OFF_STATUS = OFF_MPART + ((sizeof(double) * irs::MSUM_BLOCKS + 255) & ~(size_t)255);
constexpr size_t OFF_TILES = OFF_STATUS + 256;
constexpr size_t SCRATCH_BYTES = OFF_TILES + sizeof(irs::TileRec) * NOALLOC_MAX_TILES;

static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mutex;
void* g_scratch_addr[MAX_DEVICES];  // device address of g_noalloc_scratch, per device
int g_num_sms[MAX_DEVICES];
int g_grid[MAX_DEVICES];

// Once per device, with that device current: the device address of the array
// (host code must not use the symbol itself) and the launch sizes.
irs_status device_setup(int dev, char** scratch, int* num_sms, int* grid) {
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
      cudaGetLastError();
      return IRS_ERR_CUDA;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return IRS_ERR_CUDA;
    g_num_sms[dev] = sms;
    g_grid[dev] = irs::brute_grid_size(sms, 0);
    g_scratch_addr[dev] = ptr;
  }
  *scratch = static_cast<char*>(g_scratch_addr[dev]);
  *num_sms = g_num_sms[dev];
  *grid = g_grid[dev];
  return IRS_OK;
}

}  // namespace

extern "C" irs_status irs_make_map_brute_noalloc(const irs_params* params, const double* lens_xy,
                                                 const double* mass, int64_t n, uint32_t* counts,
                                                 float* mag, void* stream) {
  if (!params || !counts) return IRS_ERR_ARG;
  const irs_params& p = *params;
  const double v[] = {p.kappa_star, p.kappa_s, p.gamma, p.src_x0, p.src_x1,
                      p.src_y0, p.src_y1, p.rays_per_pixel, p.border};
  for (double x : v)
    if (!isfinite(x)) return IRS_ERR_ARG;
  if (p.npix_x <= 0 || p.npix_y <= 0 || !(p.rays_per_pixel > 0)) return IRS_ERR_ARG;
  if ((int64_t)p.npix_x * p.npix_y >= ((int64_t)1 << 32) - 1) return IRS_ERR_OVERFLOW;
  if (!(p.src_x1 > p.src_x0) || !(p.src_y1 > p.src_y0)) return IRS_ERR_ARG;
  if (p.kappa_star < 0 || p.kappa_s < 0 || p.n_star < 0 || p.flags != 0) return IRS_ERR_ARG;
  for (int k = 0; k < 6; ++k)  // the parameter checks of irs_plan
    if (p.reserved[k] != 0) return IRS_ERR_ARG;
  if (!isfinite(p.cell_mult) || p.cell_mult < 0 || p.far_order < 0 || p.window < 0) return IRS_ERR_ARG;
  if (p.plane != IRS_PLANE_RECT && p.plane != IRS_PLANE_CIRCLE) return IRS_ERR_ARG;
  if (p.method != IRS_BRUTE) return IRS_ERR_UNSUPPORTED;
  if (p.kernel_variant != 0) return IRS_ERR_UNSUPPORTED;  // the default brute kernel only
  if (n < 0 || (n > 0 && (!lens_xy || !mass)) || (n > 0 && ((uintptr_t)lens_xy & 15u)))
    return IRS_ERR_ARG;
  if (n > ((int64_t)1 << 31)) return IRS_ERR_OVERFLOW;

  irs_plan_t P;  // on the stack: nothing here allocates
  memset(&P, 0, sizeof(P));
  P.p = p;
  irs_status st = irs::size_plane(&P);
  if (st != IRS_OK) return st;
  P.br_ntx = (P.g.nrx + irs::BR_TX - 1) / irs::BR_TX;
  P.br_nty = (P.g.nry + irs::BR_TY - 1) / irs::BR_TY;
  P.br_ntiles = P.br_ntx * P.br_nty;
  if (P.br_ntiles > NOALLOC_MAX_TILES) return IRS_ERR_OVERFLOW;  // lattice beyond the scratch
  if (!irs::brute_variant_fits(0, 2.0 * P.circle_r)) return IRS_ERR_UNSUPPORTED;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return IRS_ERR_CUDA;
  if (dev < 0 || dev >= MAX_DEVICES) return IRS_ERR_UNSUPPORTED;
  char* scratch = nullptr;
  st = device_setup(dev, &scratch, &P.num_sms, &P.br_grid);
  if (st != IRS_OK) return st;
  P.device = dev;
  P.d_msum = reinterpret_cast<double*>(scratch + OFF_MSUM);
  P.d_mpart = reinterpret_cast<double*>(scratch + OFF_MPART);
  P.d_status = reinterpret_cast<int*>(scratch + OFF_STATUS);
  P.d_tiles = reinterpret_cast<irs::TileRec*>(scratch + OFF_TILES);

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the partial sums and tile records are rewritten in full by every call;
  // the status word and the caller's count map must start at zero
  if (cudaMemsetAsync(P.d_status, 0, sizeof(int), s) != cudaSuccess) return IRS_ERR_CUDA;
  const size_t npix = (size_t)p.npix_x * p.npix_y;
  if (cudaMemsetAsync(counts, 0, npix * sizeof(uint32_t), s) != cudaSuccess) return IRS_ERR_CUDA;
  if (irs::launch_mass_sum(&P, mass, n, s) != cudaSuccess) return IRS_ERR_CUDA;
  if (irs::launch_brute_setup(&P, s) != cudaSuccess) return IRS_ERR_CUDA;
  if (irs::launch_brute_map(&P, lens_xy, mass, n, 0, P.g.nry, counts, s) != cudaSuccess)
    return IRS_ERR_CUDA;
  if (mag && irs::launch_magnify(&P, counts, mag, s) != cudaSuccess) return IRS_ERR_CUDA;
  return IRS_OK;
}
