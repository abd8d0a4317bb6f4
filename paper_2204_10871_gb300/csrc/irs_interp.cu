// irs_interp.cu -- interpolated method (placeholder until the far field lands).
#include "irs_interp.cuh"

namespace irs {
irs_status interp_plan(irs_plan_t* P) { (void)P; return IRS_ERR_UNSUPPORTED; }
void interp_fill_info(const irs_plan_t* P, irs_plan_info* info) { (void)P; (void)info; }
int64_t interp_workspace_bytes(const irs_plan_t* P) { (void)P; return 0; }
irs_status interp_run(irs_plan_t* P, const double* xy, const double* mass, int64_t n, int64_t row0,
                      int64_t row1, uint32_t* counts, cudaStream_t s) {
  (void)P; (void)xy; (void)mass; (void)n; (void)row0; (void)row1; (void)counts; (void)s;
  return IRS_ERR_UNSUPPORTED;
}
irs_status interp_shoot_rays(irs_plan_t* P, const double* xy, const double* mass, int64_t n,
                             const int64_t* idx, int64_t nidx, double* beta, int64_t* pix,
                             cudaStream_t s) {
  (void)P; (void)xy; (void)mass; (void)n; (void)idx; (void)nidx; (void)beta; (void)pix; (void)s;
  return IRS_ERR_UNSUPPORTED;
}
void interp_destroy(irs_plan_t* P) { (void)P; }
}  // namespace irs
