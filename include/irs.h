/*
 * irs.h -- C ABI of the GB300 inverse ray-shooting library.
 *
 * The library computes gravitational-microlensing magnification maps by
 * inverse ray-shooting (IRS) as described in Zheng, Chen, Li & Chen,
 * "An Improved GPU-Based Ray-Shooting Code For Gravitational Microlensing"
 * (arXiv:2204.10871): a regular lattice of rays over a rectangular
 * image/lens plane is deflected by point lenses, a smooth convergence
 * kappa_s, an external shear gamma and a negative mass sheet, and the rays
 * landing in each source-plane pixel are counted.
 *
 * Conventions for every entry point:
 *  - All lengths are in Einstein radii of a unit-mass lens.
 *  - Lens positions are interleaved doubles (x0, y0, x1, y1, ...), masses are
 *    doubles; both live in DEVICE memory owned by the caller.
 *  - Maps are row-major [npix_y][npix_x]; counts are uint32, magnifications
 *    float; both in DEVICE memory owned by the caller.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Calls enqueue work and return without waiting for it, except
 *    where noted.  Errors detected on the host are returned at once; errors
 *    raised by kernels are kept in the plan and returned by irs_plan_sync.
 *  - The library never aborts, throws or prints.  A plan is not thread-safe:
 *    use one plan per host thread or serialise calls on it.
 */
#ifndef IRS_GB300_H
#define IRS_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum irs_status {
  IRS_OK = 0,
  IRS_ERR_ARG = 1,          /* invalid argument (NULL pointer, bad size, NaN) */
  IRS_ERR_DEGENERATE = 2,   /* |1 - kappa -+ gamma| < 1e-6: the mean lens map is singular */
  IRS_ERR_OOM = 3,          /* device allocation failed */
  IRS_ERR_CUDA = 4,         /* a CUDA runtime call failed */
  IRS_ERR_TIMEOUT = 5,      /* a bounded device wait gave up */
  IRS_ERR_OVERFLOW = 6,     /* a size exceeds what the kernels index */
  IRS_ERR_NOT_TRAINED = 7,  /* IRS_MLP requested before the far-field network was trained */
  IRS_ERR_UNSUPPORTED = 8   /* combination of options not implemented */
} irs_status;

/* Shape of the lens plane.  RECT: the image rectangle is the lens plane and the
 * negative sheet is the rectangle's closed form (Eq. alpha1 and Appendix A).
 * CIRCLE: lenses fill the circumscribed circle and the sheet is the circular
 * -kappa_* theta of Eq. (alphapart), i.e. the deflection of Eq. (alpha). */
typedef enum irs_plane { IRS_PLANE_RECT = 0, IRS_PLANE_CIRCLE = 1 } irs_plane;

/* How the lens sum is evaluated.  BRUTE: every ray sums every lens.  INTERP:
 * lenses in the ray's level-1 cell and its 8 neighbours are summed per ray,
 * the rest come from a per-cell Taylor series of the far field (Sec. 2.4,
 * "Interpolation algorithm").  MLP: as INTERP with part of the far field
 * taken from a trained coordinate network (falls back to INTERP if untrained). */
typedef enum irs_method { IRS_BRUTE = 0, IRS_INTERP = 1, IRS_MLP = 2 } irs_method;

/* Inputs of the flow chart ("Input parameters", Sec. 2.4). */
typedef struct irs_params {
  double kappa_star;      /* convergence in point lenses, kappa_* (sizes the plane) */
  double kappa_s;         /* smooth convergence kappa_s */
  double gamma;           /* external shear */
  double src_x0, src_x1;  /* source region [x0, x1) x [y0, y1) */
  double src_y0, src_y1;
  int32_t npix_x, npix_y; /* source-plane pixels */
  double rays_per_pixel;  /* rays per source pixel in the unlensed map (N_av) */
  double border;          /* protective border P; < 0 selects the paper's 10 sqrt(kappa_*) */
  int64_t n_star;         /* lens count the cell grid and workspace are sized for; 0 = kappa_* A / pi */
  int32_t plane;          /* irs_plane */
  int32_t method;         /* irs_method */
  uint32_t flags;         /* reserved, must be 0 */
  int32_t far_order;      /* INTERP: terms of the per-cell far-field series; 0 = default */
  double cell_mult;       /* INTERP: level-1 cell side in units of the paper's rule; 0 = default */
  int32_t window;         /* INTERP: cells within this Chebyshev distance sum lenses directly into
                             the series; 0 = default.  MLP: the learned split's radius R_f in
                             cells; 0 = 8 */
  int32_t kernel_variant; /* INTERP: ray-pass variant 0..16 (rays per thread, level-2 sub-cells,
                             sub-cell terms, CTAs per SM, binning -- into the map or into a
                             per-cell shared-memory sub-histogram --, shared reciprocals);
                             irs_autotune picks one.  BRUTE: variant 0..15 (rows per thread,
                             rows sharing a reciprocal by pairs or by fours, packed FP32x2
                             rows); 0 = default.  Variants with four rows per reciprocal (0, 10,
                             12..15) need a plane diagonal <= 1e4 theta_E
                             (IRS_ERR_UNSUPPORTED otherwise) */
  int32_t reserved[6];    /* must be 0 */
} irs_params;

/* Geometry chosen by irs_plan (FP64, host side). */
typedef struct irs_plan_info {
  double lens_x0, lens_x1, lens_y0, lens_y1; /* image/lens rectangle [a1,a2] x [b1,b2] */
  double center_x, center_y;                 /* rectangle centre */
  double border;                             /* P actually used */
  double dx_ray;                             /* level-3 spacing Delta x3 */
  double pix_x, pix_y;                       /* source pixel sides */
  double circle_r;                           /* circumscribed-circle radius */
  double cell_x, cell_y;                     /* level-1 cell sides (INTERP) */
  int64_t n_rays_x, n_rays_y, n_rays;        /* ray lattice */
  int64_t n_star_suggested;                  /* kappa_* A / pi (unit mean mass) */
  int32_t ncell_x, ncell_y;                  /* level-1 grid (INTERP) */
  int32_t rays_per_cell_x, rays_per_cell_y;  /* rays along a cell side (INTERP) */
  int32_t far_order, window;                 /* INTERP series terms and direct window */
  int64_t workspace_bytes;                   /* device memory held by the plan */
} irs_plan_info;

typedef struct irs_plan irs_plan_t;

/* Size the image/lens plane and the ray lattice from `params` (flow chart:
 * protective border P = 10 sqrt(kappa_*), I = (S + 2P)/|1 - kappa -+ gamma|,
 * level-3 spacing; Sec. 2.4) and allocate the plan's device workspace on the
 * current device.  Synchronous (it allocates).  On success *out owns the
 * plan; release it with irs_plan_destroy.  Errors: IRS_ERR_ARG,
 * IRS_ERR_DEGENERATE, IRS_ERR_OOM, IRS_ERR_OVERFLOW. */
irs_status irs_plan(const irs_params* params, void* stream, irs_plan_t** out);

/* Copy the plan's geometry into *info (host memory).  Errors: IRS_ERR_ARG. */
irs_status irs_plan_info_get(const irs_plan_t* plan, irs_plan_info* info);

/* One magnification map (the whole flow chart after sizing, Sec. 2.4):
 * deflect every ray of the lattice by the n lenses (lens_xy: 2n doubles,
 * mass: n doubles, device), bin it into the source pixel it lands in, and
 * write counts (npix_x*npix_y uint32, device, overwritten) and, when `mag` is
 * not NULL, Mag_ij = N_ij S_I / S_S (npix_x*npix_y float, device).  The
 * sheet's density is that of the lenses passed in, pi sum(m) / area.  n may
 * be 0.  Every lens must lie in the plan's lens region -- the rectangle that
 * is both image and lens plane (Sec. 2.2), or the circumscribed circle for
 * IRS_PLANE_CIRCLE -- to within 1e-9 of the plane's extent: the mass-sum pass
 * checks every position on the device, and a lens outside (or a NaN position)
 * makes the next irs_plan_sync return IRS_ERR_ARG.  Asynchronous on `stream`;
 * may grow the workspace (synchronising) if n exceeds the size the plan was
 * made for.  Errors: IRS_ERR_ARG, IRS_ERR_OOM, IRS_ERR_CUDA,
 * IRS_ERR_NOT_TRAINED. */
irs_status irs_make_map(irs_plan_t* plan, const double* lens_xy, const double* mass, int64_t n,
                        uint32_t* counts, float* mag, void* stream);

/* Several maps with their own plans, lenses and outputs (no paper
 * counterpart: many maps of uneven N_*, kappa and gamma).  Each map's mass
 * sum, cell lists and far-field series (or brute-force setup and ray pass) run
 * on forked streams; the interpolated ray passes of all maps run as one
 * persistent launch per kernel variant that pulls (map, cell) items from a
 * global counter.  The sequence is captured into a CUDA graph on the first call
 * with a given set of plans, pointers and lens counts, and later calls with the
 * same set replay the graph (the last 4 sets are kept; destroying a plan drops
 * the graphs that use it).  A plan whose lens buffers were reallocated since
 * (irs_make_map with more lenses than it had room for) is a new set: it is
 * captured again, and no graph holding the old buffers is replayed.  Arrays hold `nmaps` host-side entries; the pointers
 * they hold are device pointers; `mag` (or any mag[k]) may be NULL.  Results
 * equal those of irs_make_map on each map.  Each plan may appear once (its
 * workspace serves one map).  The first call of a set allocates and
 * synchronises; replays only enqueue.  Errors: as irs_make_map, IRS_ERR_ARG
 * for a repeated plan, IRS_ERR_UNSUPPORTED for IRS_MLP plans. */
irs_status irs_make_maps_batched(irs_plan_t* const* plans, int32_t nmaps,
                                 const double* const* lens_xy, const double* const* mass,
                                 const int64_t* n, uint32_t* const* counts, float* const* mag,
                                 void* stream);

/* Chunked sweep (the count map is additive over disjoint sets of rays): add
 * into `counts` (device, NOT cleared) the rays of lattice rows
 * [row0, row1) only.  Used to sweep very large lattices in pieces, to resume
 * a sweep from a saved map plus the next row, and to split one map over
 * several GPUs (each shoots a strip of rows; the count maps are summed).  The
 * sheet density and all per-map constants are recomputed from the lenses on
 * every call; INTERP computes the per-cell series only for the level-1 cell
 * rows the band touches (the global far-field convolution is always whole).
 * Errors: IRS_ERR_ARG (row range outside [0, n_rays_y]), as irs_make_map. */
irs_status irs_make_map_rows(irs_plan_t* plan, const double* lens_xy, const double* mass,
                             int64_t n, int64_t row0, int64_t row1, uint32_t* counts,
                             void* stream);

/* Mag_ij = N_ij S_I / S_S of an existing count map (device in, device out). */
irs_status irs_magnify(irs_plan_t* plan, const uint32_t* counts, float* mag, void* stream);

/* Stage times of the last map made with this plan, from CUDA events recorded
 * on the launching stream (enable with irs_plan_set_timing; synchronises on
 * the events when read).  Fields are milliseconds; ms_raypass is the ray pass
 * kernel alone, the dominant kernel of every method. */
typedef struct irs_timings {
  float ms_total;     /* first to last event of the map */
  float ms_prep;      /* mass sum and per-tile / per-cell setup */
  float ms_cells;     /* INTERP: lens cell lists */
  float ms_farfield;  /* INTERP: far-field series */
  float ms_raypass;   /* ray pass incl. binning */
  float ms_magnify;   /* magnification (0 if not requested) */
  int64_t rays;       /* rays shot by the timed map */
  int32_t valid;      /* 1 when the fields hold a measurement */
  int32_t launches;   /* kernel launches of the map */
  float ms_finalize;  /* INTERP: the per-cell part of ms_farfield (window, sheet series) */
} irs_timings;

irs_status irs_plan_set_timing(irs_plan_t* plan, int32_t enable);
irs_status irs_plan_timings(irs_plan_t* plan, irs_timings* out);

/* Debug / parity path: the source-plane position beta (2 doubles per ray,
 * device) and pixel index (int64, -1 when outside; device; may be NULL) of
 * the lattice rays with flat indices ray_idx[k] = j * n_rays_x + i (device
 * int64).  Each ray is computed by the same kernel code and tiling that
 * irs_make_map uses for the plan's method, so the values are those that
 * were binned.  Errors: IRS_ERR_ARG, IRS_ERR_CUDA. */
irs_status irs_shoot_rays(irs_plan_t* plan, const double* lens_xy, const double* mass, int64_t n,
                          const int64_t* ray_idx, int64_t n_idx, double* beta, int64_t* pixel,
                          void* stream);

/* Autotuner (no paper counterpart; the paper fixes Delta x1 by its rule and
 * Delta x2 = Delta x1 / 20 "after a series of tests", Sec. 2.4): for an
 * INTERP or MLP `params`, time candidate level-1 cell sizes (multiples of 32
 * rays from 0.5 to 1.25 times the paper's rule, and the rule itself; for rule
 * cells under 128 rays, multipliers 0.5 .. 2 of the rule) and ray-pass kernel
 * variants on the given lenses
 * (device arrays as irs_make_map) and write into *tuned a copy of *params with
 * the fastest cell_mult and kernel_variant.  Each candidate's cost per map is
 * its cell size's measured cell-list and far-field time plus its ray-pass time
 * on a band of ~1e9 rays scaled to the whole lattice (one temporary plan per
 * cell size; every variant's ray pass is timed on that plan's cells).  `cache_path` (or, when NULL or
 * empty, the environment variable IRS_AUTOTUNE_CACHE) names a JSON-lines file
 * of earlier results keyed by a coarse signature of the parameters; a hit
 * returns at once, a miss appends the new result.  For IRS_BRUTE, *tuned =
 * *params.  Synchronous; allocates temporary plans.  *result (may be NULL)
 * receives the choice and the estimated milliseconds per map of the choice
 * and of the default (cell_mult 1, variant 0).  Errors: IRS_ERR_ARG,
 * IRS_ERR_OOM, IRS_ERR_CUDA. */
typedef struct irs_tune_result {
  double cell_mult;      /* chosen multiplier of the paper's Delta x1 */
  int32_t kernel_variant;
  int32_t candidates;    /* candidates measured (0 when served from the cache) */
  double ms_per_map;     /* estimated time per map of the choice */
  double ms_default;     /* the same for cell_mult 1, variant 0 (0 if not measured) */
  int32_t from_cache;    /* 1 when the cache answered */
  int32_t pad_;
} irs_tune_result;

irs_status irs_autotune(const irs_params* params, const double* lens_xy, const double* mass,
                        int64_t n, const char* cache_path, irs_params* tuned,
                        irs_tune_result* result, void* stream);

/* ---- Learned far field (no paper counterpart).  An IRS_MLP plan sums, for
 * each level-1 cell, the lenses within a smooth window of R_f cells
 * (irs_params.window, default 8: weight 1 out to R_f/2, a C-infinity step to
 * 0 at R_f) directly and takes the rest of the far field -- the "far-far"
 * part minus the sheet's analytic part -- from a coordinate network: Fourier features
 * [sin, cos](pi B x) of the cell centre (32 frequencies), three tanh layers of
 * width 64, 8 outputs (4 complex series coefficients).  Cells near the
 * rectangle's corners keep an exact direct sum.  Until irs_mlp_train has run,
 * an IRS_MLP plan computes the exact FFT far field of IRS_INTERP (fallback).
 * The network learns the far field of ONE lens field: make maps with the
 * lenses it was trained on.  Its maps are not accurate to the 1e-3 per-pixel
 * magnification of the series form: the network's deflection error is
 * ~1e-2 theta_E where ~1e-6 is needed; use IRS_INTERP for production maps. */
typedef struct irs_mlp_report {
  int64_t samples;       /* training samples (direct sums at random points) */
  int32_t steps;         /* AdamW steps, batch 4096 */
  int32_t trained;       /* 1 on success */
  double loss_first;     /* standardised MSE, mean of the first 20 steps */
  double loss_final;     /* the same, last 20 steps */
  double valid_rel_rms;  /* held-out: RMS(prediction - target) / RMS(target), physical units */
  double target_rms;     /* RMS of the targets (theta_E, per output) */
  double ms_samples;     /* time to generate the samples (GPU direct sums) */
  double ms_train;       /* time of the training loop */
} irs_mlp_report;

/* Train the plan's network on the lens field (device arrays as irs_make_map):
 * n_samples direct-sum targets at seeded random points of the plane (0:
 * 1,048,576, the maximum), `steps` AdamW steps (0: 3000) of 4096 samples with
 * BF16 tensor-core forward/backward kernels, FP32 accumulation and FP32
 * master weights.  Synchronous.  Errors: IRS_ERR_ARG, IRS_ERR_UNSUPPORTED (not
 * an IRS_MLP plan), IRS_ERR_OOM, IRS_ERR_CUDA. */
irs_status irs_mlp_train(irs_plan_t* plan, const double* lens_xy, const double* mass, int64_t n,
                         int64_t n_samples, int32_t steps, uint64_t seed, irs_mlp_report* report,
                         void* stream);

/* Copy the network's 13,000 FP32 parameters (packed W1, b1, W2, b2, W3, b3, W4,
 * b4, row-major W[out][in]) and its 32 x 2 Fourier matrix in (host arrays;
 * NULL leaves a part unchanged) and/or out.  Synchronous.  Errors:
 * IRS_ERR_UNSUPPORTED (not an IRS_MLP plan), IRS_ERR_CUDA. */
irs_status irs_mlp_params(irs_plan_t* plan, const float* theta_in, const float* freq_in,
                          float* theta_out, float* freq_out);

/* Parity path of the training kernel: the loss sum (device double, sum of
 * squared errors) and the gradient of the mean squared error (device float
 * [13000]) over the n inputs x (device float [n][2]) and targets t (device
 * float [n][8]), computed by the same kernel as one training step. */
irs_status irs_mlp_grad(irs_plan_t* plan, const float* x, const float* t, int64_t n, float* grad,
                        double* loss_sum, void* stream);

/* Network outputs y (device float [n][8], standardised units) at inputs x
 * (device float [n][2]). */
irs_status irs_mlp_forward(irs_plan_t* plan, const float* x, int64_t n, float* y, void* stream);

/* Allocation-free brute-force map.  The paper has no counterpart: this serves
 * callers that cannot allocate device memory -- code running while another
 * memory manager owns the device (a caching allocator or a fixed pool),
 * plug-ins that must not trigger cudaMalloc/cudaFree's implicit device-wide
 * synchronisation, and latency-critical loops.  It computes what
 * irs_make_map does for a plan made from `params` with method IRS_BRUTE
 * (counts overwritten, mag written when not NULL), but takes the parameters
 * directly and calls no cudaMalloc, cudaFree or other allocating routine: its
 * scratch is a 7.9 MB file-scope device array that every GPU loading the
 * library holds until exit.  Limit: the ray lattice must fit 49,152 tiles of
 * 32 x 64 rays (about 1.0e8 rays); larger lattices return IRS_ERR_OVERFLOW
 * before any work is enqueued, and planes wider than 1e4 theta_E
 * (diagonal) IRS_ERR_UNSUPPORTED.  The first call on each device looks up the
 * array's device address; where none of the library's device code has run on
 * that device yet, it also loads that code (CUDA loads modules lazily by
 * default), and the array is allocated then.  Make the first call on each
 * device before any stream capture and outside latency-critical loops; later
 * calls allocate nothing.  Lens positions are not checked against the lens
 * region (there is no plan to report a device-side error to).  All calls share
 * the array: calls whose work overlaps on the GPU race.  Errors: IRS_ERR_ARG,
 * IRS_ERR_DEGENERATE, IRS_ERR_OVERFLOW, IRS_ERR_UNSUPPORTED (method other than
 * IRS_BRUTE), IRS_ERR_CUDA. */
irs_status irs_make_map_brute_noalloc(const irs_params* params, const double* lens_xy,
                                      const double* mass, int64_t n, uint32_t* counts,
                                      float* mag, void* stream);

/* Wait for `stream` and return the first error a kernel of this plan raised
 * since the last sync (IRS_OK if none), clearing it: IRS_ERR_ARG for a lens
 * outside the plan's lens region, IRS_ERR_OVERFLOW when the 3 x 3 block of
 * level-1 cells around some cell held more than the 1024 lenses the
 * interpolated ray pass keeps in shared memory (that cell's near sum used the
 * first 1024; the map is not valid).  The plan stays usable. */
irs_status irs_plan_sync(irs_plan_t* plan, void* stream);

/* Free the plan and its workspace (synchronises the device).  NULL is a no-op. */
irs_status irs_plan_destroy(irs_plan_t* plan);

/* Static text for a status code. */
const char* irs_status_str(irs_status status);

#ifdef __cplusplus
}
#endif

#endif /* IRS_GB300_H */
