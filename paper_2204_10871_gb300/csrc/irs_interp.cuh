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
}  // namespace irs
