// irs_interp.cuh -- entry points of the interpolated (cell list + far-field
// series) method, implemented in irs_interp.cu.
#pragma once

#include "irs_common.cuh"

namespace irs {
irs_status interp_plan(irs_plan_t* P);
void interp_fill_info(const irs_plan_t* P, irs_plan_info* info);
int64_t interp_workspace_bytes(const irs_plan_t* P);
// cells -> far field -> ray pass over lattice rows [row0, row1), with the
// plan's timing events marked between stages.
irs_status interp_run(irs_plan_t* P, const double* xy, const double* mass, int64_t n, int64_t row0,
                      int64_t row1, uint32_t* counts, cudaStream_t s);
irs_status interp_shoot_rays(irs_plan_t* P, const double* xy, const double* mass, int64_t n,
                             const int64_t* idx, int64_t nidx, double* beta, int64_t* pix,
                             cudaStream_t s);
void interp_destroy(irs_plan_t* P);

// --- autotuner (irs_autotune.cu)
// switch the plan's ray pass to another kernel variant (same cells and far field)
irs_status interp_set_variant(irs_plan_t* P, int variant);
// the ray pass alone over lattice rows [row0, row1), on the cell records and
// series the last map of these rows left, bracketed by events e0, e1 on `s`
irs_status interp_raypass_rows(irs_plan_t* P, int64_t row0, int64_t row1, uint32_t* counts, cudaStream_t s,
                               cudaEvent_t e0, cudaEvent_t e1);

// --- batched maps (irs_batch.cu)
// grow the lens buffers outside any stream capture
irs_status interp_ensure_capacity(irs_plan_t* P, int64_t n);
// cell lists and far-field series of one map (no ray pass)
irs_status interp_prepare(irs_plan_t* P, const double* xy, const double* mass, int64_t n,
                          cudaStream_t s);
int interp_variant(const irs_plan_t* P);
// row-table entries of the plan's ray pass (shared memory per CTA grows with them)
int interp_row_entries(const irs_plan_t* P);
int interp_num_variants();
// host-side ray-pass descriptors of maps that share a kernel variant; returns
// the total number of (map, cell) work items
size_t interp_desc_bytes(int nmaps);
int64_t interp_fill_descs(irs_plan_t* const* plans, uint32_t* const* counts, int nmaps, void* host);
// one persistent launch over all maps' cells (descriptors already on the
// device); nrow: the largest row table among the maps
irs_status interp_batch_launch(int variant, const void* dev_descs, int nmaps, int64_t nitems,
                               unsigned long long* queue, int num_sms, int nrow, cudaStream_t s);
}  // namespace irs
