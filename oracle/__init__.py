"""FP64 CPU oracle for inverse ray-shooting (arXiv:2204.10871).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
benchmark's CPU-baseline leg, never by the library.  See irs_oracle.c for what
each function follows in the paper.
"""
from .oracle import (OracleParams, OraclePlan, make_params, size, sheet_positive, kappa_star_actual,
                     deflection, shoot_rays, make_map, PLANE_RECT, PLANE_CIRCLE)

__all__ = ["OracleParams", "OraclePlan", "make_params", "size", "sheet_positive", "kappa_star_actual",
           "deflection", "shoot_rays", "make_map", "PLANE_RECT", "PLANE_CIRCLE"]
