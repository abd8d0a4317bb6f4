"""ctypes front end of the plain-C FP64 oracle (irs_oracle.c).

Test infrastructure only.  Arrays are numpy float64/int64/uint32; nothing here
touches the CUDA library.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

PLANE_RECT = 0
PLANE_CIRCLE = 1


class OracleParams(C.Structure):
    _fields_ = [("kappa_star", C.c_double), ("kappa_s", C.c_double), ("gamma", C.c_double),
                ("src_x0", C.c_double), ("src_x1", C.c_double),
                ("src_y0", C.c_double), ("src_y1", C.c_double),
                ("npix_x", C.c_int32), ("npix_y", C.c_int32),
                ("rays_per_pixel", C.c_double), ("border", C.c_double),
                ("plane", C.c_int32), ("pad_", C.c_int32)]


class OraclePlan(C.Structure):
    _fields_ = [("kappa", C.c_double), ("border", C.c_double),
                ("lambda1", C.c_double), ("lambda2", C.c_double),
                ("ix0", C.c_double), ("iy0", C.c_double),
                ("sx", C.c_double), ("sy", C.c_double), ("dx3", C.c_double),
                ("ix", C.c_double), ("iy", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double),
                ("a1", C.c_double), ("a2", C.c_double), ("b1", C.c_double), ("b2", C.c_double),
                ("nrx", C.c_int64), ("nry", C.c_int64), ("n_rays", C.c_int64),
                ("circle_r", C.c_double), ("n_star_paper", C.c_double)]


_lib = None


def _L():
    global _lib
    if _lib is None:
        lib = C.CDLL(_build.build())
        dp = C.POINTER(C.c_double)
        i64p = C.POINTER(C.c_int64)
        u32p = C.POINTER(C.c_uint32)
        lib.or_size.argtypes = [C.POINTER(OracleParams), C.POINTER(OraclePlan)]
        lib.or_size.restype = C.c_int
        lib.or_sheet_positive.argtypes = [C.c_double] * 7 + [dp, dp]
        lib.or_sheet_positive.restype = None
        lib.or_kappa_star_actual.argtypes = [C.POINTER(OracleParams), C.POINTER(OraclePlan), dp,
                                             C.c_int64]
        lib.or_kappa_star_actual.restype = C.c_double
        lib.or_deflection.argtypes = [C.POINTER(OracleParams), C.POINTER(OraclePlan), dp, dp,
                                      C.c_int64, C.c_double, C.c_double, C.c_double, dp, dp]
        lib.or_deflection.restype = None
        lib.or_shoot_rays.argtypes = [C.POINTER(OracleParams), C.POINTER(OraclePlan), dp, dp,
                                      C.c_int64, C.c_double, i64p, C.c_int64, dp, dp, i64p]
        lib.or_shoot_rays.restype = None
        lib.or_make_map.argtypes = [C.POINTER(OracleParams), C.POINTER(OraclePlan), dp, dp,
                                    C.c_int64, C.c_int64, C.c_int64, C.c_int64, C.c_int64,
                                    C.c_int, u32p, dp]
        lib.or_make_map.restype = C.c_int64
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _lens_arrays(xy, mass):
    xy = np.ascontiguousarray(np.asarray(xy, dtype=np.float64).reshape(-1, 2))
    mass = np.ascontiguousarray(np.asarray(mass, dtype=np.float64).reshape(-1))
    if xy.shape[0] != mass.shape[0]:
        raise ValueError("lens positions and masses differ in length")
    if xy.shape[0] == 0:  # keep valid pointers for the empty field
        xy = np.zeros((1, 2))
        mass = np.zeros(1)
        return xy, mass, 0
    return xy, mass, xy.shape[0]


def make_params(kappa_star, kappa_s, gamma, src, npix, rays_per_pixel, border=-1.0,
                plane=PLANE_RECT):
    """src = (x0, x1, y0, y1) in Einstein radii; npix = (nx, ny) or n."""
    if isinstance(npix, int):
        npix = (npix, npix)
    return OracleParams(kappa_star, kappa_s, gamma, src[0], src[1], src[2], src[3],
                        int(npix[0]), int(npix[1]), rays_per_pixel, border, int(plane), 0)


def size(params: OracleParams) -> OraclePlan:
    """Sizing of the image/lens plane and the ray lattice (flow chart; N_av counts rays per unlensed source pixel)."""
    plan = OraclePlan()
    rc = _L().or_size(C.byref(params), C.byref(plan))
    if rc == 1:
        raise ValueError("invalid parameters")
    if rc == 2:
        raise ValueError("degenerate lens map: |1 - kappa -+ gamma| < 1e-6")
    return plan


def sheet_positive(a1, a2, b1, b2, kappa, t1, t2):
    """Appendix A closed form: deflection of a positive uniform rectangle."""
    o1, o2 = C.c_double(), C.c_double()
    _L().or_sheet_positive(a1, a2, b1, b2, kappa, t1, t2, C.byref(o1), C.byref(o2))
    return o1.value, o2.value


def kappa_star_actual(params, plan, mass):
    mass = np.ascontiguousarray(np.asarray(mass, dtype=np.float64).reshape(-1))
    if mass.size == 0:
        return 0.0
    return _L().or_kappa_star_actual(C.byref(params), C.byref(plan), _dp(mass), mass.size)


def deflection(params, plan, xy, mass, t1, t2, kstar_act=None):
    """Eq. (alpha1) (rectangle) or Eq. (alpha) (circle) at one point."""
    xy, mass, n = _lens_arrays(xy, mass)
    if kstar_act is None:
        kstar_act = kappa_star_actual(params, plan, mass[:n])
    o1, o2 = C.c_double(), C.c_double()
    _L().or_deflection(C.byref(params), C.byref(plan), _dp(xy), _dp(mass), n, kstar_act,
                       t1, t2, C.byref(o1), C.byref(o2))
    return o1.value, o2.value


def shoot_rays(params, plan, xy, mass, idx):
    """alpha, beta (each (k, 2)) and pixel (k,) for flat lattice indices idx = j*nrx + i."""
    xy, mass, n = _lens_arrays(xy, mass)
    kstar = kappa_star_actual(params, plan, mass[:n])
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64).reshape(-1))
    k = idx.size
    alpha = np.zeros((max(k, 1), 2))
    beta = np.zeros((max(k, 1), 2))
    pix = np.zeros(max(k, 1), dtype=np.int64)
    if k:
        _L().or_shoot_rays(C.byref(params), C.byref(plan), _dp(xy), _dp(mass), n, kstar,
                           idx.ctypes.data_as(C.POINTER(C.c_int64)), k, _dp(alpha), _dp(beta),
                           pix.ctypes.data_as(C.POINTER(C.c_int64)))
    return alpha[:k], beta[:k], pix[:k]


def make_map(params, plan, xy, mass, rows=None, cols=None, threads=None):
    """Brute-force count map and magnification over the lattice rows/cols given
    (default: all rays).  Returns (counts uint32 (ny, nx), mag float64, landed)."""
    xy, mass, n = _lens_arrays(xy, mass)
    if rows is None:
        rows = (0, plan.nry)
    if cols is None:
        cols = (0, plan.nrx)
    if threads is None:
        threads = os.cpu_count() or 1
    counts = np.zeros((params.npix_y, params.npix_x), dtype=np.uint32)
    mag = np.zeros((params.npix_y, params.npix_x), dtype=np.float64)
    landed = _L().or_make_map(C.byref(params), C.byref(plan), _dp(xy), _dp(mass), n,
                              int(rows[0]), int(rows[1]), int(cols[0]), int(cols[1]),
                              int(threads), counts.ctypes.data_as(C.POINTER(C.c_uint32)),
                              _dp(mag))
    return counts, mag, int(landed)
