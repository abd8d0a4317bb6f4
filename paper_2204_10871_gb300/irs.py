"""ctypes binding of the C ABI in include/irs.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of the method: all of the ray-shooting runs in the CUDA library.
Device buffers are torch CUDA tensors (contiguous); streams are torch streams
or raw cudaStream_t integers.  A missing library raises at once: there is no
fallback path.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libirs_gb300.so")

IRS_OK = 0
STATUS_NAMES = {0: "IRS_OK", 1: "IRS_ERR_ARG", 2: "IRS_ERR_DEGENERATE", 3: "IRS_ERR_OOM",
                4: "IRS_ERR_CUDA", 5: "IRS_ERR_TIMEOUT", 6: "IRS_ERR_OVERFLOW",
                7: "IRS_ERR_NOT_TRAINED", 8: "IRS_ERR_UNSUPPORTED"}
IRS_PLANE_RECT, IRS_PLANE_CIRCLE = 0, 1
IRS_BRUTE, IRS_INTERP, IRS_MLP = 0, 1, 2


class IrsParams(C.Structure):
    _fields_ = [("kappa_star", C.c_double), ("kappa_s", C.c_double), ("gamma", C.c_double),
                ("src_x0", C.c_double), ("src_x1", C.c_double),
                ("src_y0", C.c_double), ("src_y1", C.c_double),
                ("npix_x", C.c_int32), ("npix_y", C.c_int32),
                ("rays_per_pixel", C.c_double), ("border", C.c_double),
                ("n_star", C.c_int64), ("plane", C.c_int32), ("method", C.c_int32),
                ("flags", C.c_uint32), ("far_order", C.c_int32), ("cell_mult", C.c_double),
                ("window", C.c_int32), ("kernel_variant", C.c_int32),
                ("reserved", C.c_int32 * 6)]


class IrsPlanInfo(C.Structure):
    _fields_ = [("lens_x0", C.c_double), ("lens_x1", C.c_double),
                ("lens_y0", C.c_double), ("lens_y1", C.c_double),
                ("center_x", C.c_double), ("center_y", C.c_double),
                ("border", C.c_double), ("dx_ray", C.c_double),
                ("pix_x", C.c_double), ("pix_y", C.c_double), ("circle_r", C.c_double),
                ("cell_x", C.c_double), ("cell_y", C.c_double),
                ("n_rays_x", C.c_int64), ("n_rays_y", C.c_int64), ("n_rays", C.c_int64),
                ("n_star_suggested", C.c_int64),
                ("ncell_x", C.c_int32), ("ncell_y", C.c_int32),
                ("rays_per_cell_x", C.c_int32), ("rays_per_cell_y", C.c_int32),
                ("far_order", C.c_int32), ("window", C.c_int32),
                ("workspace_bytes", C.c_int64)]


class IrsTimings(C.Structure):
    _fields_ = [("ms_total", C.c_float), ("ms_prep", C.c_float), ("ms_cells", C.c_float),
                ("ms_farfield", C.c_float), ("ms_raypass", C.c_float), ("ms_magnify", C.c_float),
                ("rays", C.c_int64), ("valid", C.c_int32), ("launches", C.c_int32),
                ("ms_finalize", C.c_float)]


class IrsTuneResult(C.Structure):
    _fields_ = [("cell_mult", C.c_double), ("kernel_variant", C.c_int32),
                ("candidates", C.c_int32), ("ms_per_map", C.c_double), ("ms_default", C.c_double),
                ("from_cache", C.c_int32), ("pad_", C.c_int32)]


class IrsMlpReport(C.Structure):
    _fields_ = [("samples", C.c_int64), ("steps", C.c_int32), ("trained", C.c_int32),
                ("loss_first", C.c_double), ("loss_final", C.c_double),
                ("valid_rel_rms", C.c_double), ("target_rms", C.c_double),
                ("ms_samples", C.c_double), ("ms_train", C.c_double)]


class IrsError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)} ({irs_status_str(status)})")


_lib = None


def _L():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library {LIB_PATH} is not built; run "
                               "paper_2204_10871_gb300.build.build() first")
        lib = C.CDLL(LIB_PATH)
        vp, dp, i64 = C.c_void_p, C.c_void_p, C.c_int64
        lib.irs_plan.argtypes = [C.POINTER(IrsParams), vp, C.POINTER(vp)]
        lib.irs_plan_info_get.argtypes = [vp, C.POINTER(IrsPlanInfo)]
        lib.irs_make_map.argtypes = [vp, dp, dp, i64, vp, vp, vp]
        lib.irs_make_maps_batched.argtypes = [C.POINTER(vp), C.c_int32, C.POINTER(vp),
                                              C.POINTER(vp), C.POINTER(i64), C.POINTER(vp),
                                              C.POINTER(vp), vp]
        lib.irs_shoot_rays.argtypes = [vp, dp, dp, i64, vp, i64, vp, vp, vp]
        lib.irs_make_map_rows.argtypes = [vp, dp, dp, i64, i64, i64, vp, vp]
        lib.irs_magnify.argtypes = [vp, vp, vp, vp]
        lib.irs_plan_set_timing.argtypes = [vp, C.c_int32]
        lib.irs_plan_timings.argtypes = [vp, C.POINTER(IrsTimings)]
        lib.irs_make_map_brute_noalloc.argtypes = [C.POINTER(IrsParams), dp, dp, i64, vp, vp, vp]
        lib.irs_autotune.argtypes = [C.POINTER(IrsParams), dp, dp, i64, C.c_char_p,
                                     C.POINTER(IrsParams), C.POINTER(IrsTuneResult), vp]
        lib.irs_mlp_train.argtypes = [vp, dp, dp, i64, i64, C.c_int32, C.c_uint64,
                                      C.POINTER(IrsMlpReport), vp]
        fp = C.POINTER(C.c_float)
        lib.irs_mlp_params.argtypes = [vp, fp, fp, fp, fp]
        lib.irs_mlp_grad.argtypes = [vp, vp, vp, i64, vp, vp, vp]
        lib.irs_mlp_forward.argtypes = [vp, vp, i64, vp, vp]
        lib.irs_plan_sync.argtypes = [vp, vp]
        lib.irs_plan_destroy.argtypes = [vp]
        lib.irs_status_str.argtypes = [C.c_int]
        lib.irs_status_str.restype = C.c_char_p
        for name in ("irs_plan", "irs_plan_info_get", "irs_make_map", "irs_make_maps_batched",
                     "irs_shoot_rays", "irs_plan_sync", "irs_plan_destroy", "irs_make_map_rows",
                     "irs_magnify", "irs_plan_set_timing", "irs_plan_timings",
                     "irs_make_map_brute_noalloc", "irs_autotune", "irs_mlp_train",
                     "irs_mlp_params", "irs_mlp_grad", "irs_mlp_forward"):
            getattr(lib, name).restype = C.c_int
        _lib = lib
    return _lib


def lib_handle():
    """The loaded ctypes library (loads it on first use)."""
    return _L()


def _check(status, where):
    if status != IRS_OK:
        raise IrsError(status, where)


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _ptr(t, dtype=None, what="tensor"):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{what} must be a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{what} must have dtype {dtype}, got {t.dtype}")
    return C.c_void_p(t.data_ptr())


def make_params(kappa_star, kappa_s, gamma, src, npix, rays_per_pixel, border=-1.0, n_star=0,
                plane=IRS_PLANE_RECT, method=IRS_BRUTE, far_order=0, cell_mult=0.0, window=0,
                kernel_variant=0):
    """Fill an IrsParams; src = (x0, x1, y0, y1), npix = n or (nx, ny)."""
    if isinstance(npix, int):
        npix = (npix, npix)
    return IrsParams(kappa_star, kappa_s, gamma, src[0], src[1], src[2], src[3], int(npix[0]),
                     int(npix[1]), rays_per_pixel, border, int(n_star), int(plane), int(method),
                     0, int(far_order), float(cell_mult), int(window), int(kernel_variant),
                     (C.c_int32 * 6)())


def irs_status_str(status):
    return _L().irs_status_str(int(status)).decode()


def irs_plan(params, stream=None):
    """Create a plan (handle as int).  Raises IrsError on failure."""
    h = C.c_void_p()
    _check(_L().irs_plan(C.byref(params), _stream(stream) if stream is not None else None,
                         C.byref(h)), "irs_plan")
    return h.value


def irs_plan_info_get(plan):
    info = IrsPlanInfo()
    _check(_L().irs_plan_info_get(C.c_void_p(plan), C.byref(info)), "irs_plan_info_get")
    return info


def irs_make_map(plan, lens_xy, mass, counts, mag=None, stream=None):
    """lens_xy: (n, 2) float64, mass: (n,) float64, counts: (ny, nx) uint32,
    mag: (ny, nx) float32 or None -- all CUDA tensors."""
    import torch
    n = int(mass.numel())
    _check(_L().irs_make_map(C.c_void_p(plan), _ptr(lens_xy, torch.float64, "lens_xy") if n else None,
                             _ptr(mass, torch.float64, "mass") if n else None, n,
                             _ptr(counts, torch.uint32, "counts"),
                             _ptr(mag, torch.float32, "mag"), _stream(stream)), "irs_make_map")


def irs_make_map_rows(plan, lens_xy, mass, row0, row1, counts, stream=None):
    """Add the rays of lattice rows [row0, row1) into counts (not cleared)."""
    import torch
    n = int(mass.numel())
    _check(_L().irs_make_map_rows(C.c_void_p(plan),
                                  _ptr(lens_xy, torch.float64, "lens_xy") if n else None,
                                  _ptr(mass, torch.float64, "mass") if n else None, n, int(row0),
                                  int(row1), _ptr(counts, torch.uint32, "counts"),
                                  _stream(stream)), "irs_make_map_rows")


def irs_magnify(plan, counts, mag, stream=None):
    import torch
    _check(_L().irs_magnify(C.c_void_p(plan), _ptr(counts, torch.uint32, "counts"),
                            _ptr(mag, torch.float32, "mag"), _stream(stream)), "irs_magnify")


def irs_plan_set_timing(plan, enable=True):
    _check(_L().irs_plan_set_timing(C.c_void_p(plan), 1 if enable else 0), "irs_plan_set_timing")


def irs_plan_timings(plan):
    t = IrsTimings()
    _check(_L().irs_plan_timings(C.c_void_p(plan), C.byref(t)), "irs_plan_timings")
    return t


def irs_make_maps_batched(plans, lens_xy, mass, counts, mag=None, stream=None):
    """Lists of per-map handles / CUDA tensors, as irs_make_map."""
    import torch
    k = len(plans)
    arr = lambda vals, T=C.c_void_p: (T * max(k, 1))(*vals)
    ns = [int(m.numel()) for m in mass]
    _check(_L().irs_make_maps_batched(
        arr([C.c_void_p(p) for p in plans]), k,
        arr([_ptr(x, torch.float64, "lens_xy") if nn else None for x, nn in zip(lens_xy, ns)]),
        arr([_ptr(x, torch.float64, "mass") if nn else None for x, nn in zip(mass, ns)]),
        arr(ns, C.c_int64), arr([_ptr(c, torch.uint32, "counts") for c in counts]),
        arr([_ptr(m, torch.float32, "mag") for m in mag]) if mag is not None else None,
        _stream(stream)), "irs_make_maps_batched")


def irs_shoot_rays(plan, lens_xy, mass, ray_idx, beta, pixel=None, stream=None):
    """ray_idx: (k,) int64 CUDA; beta: (k, 2) float64 CUDA; pixel: (k,) int64 CUDA or None."""
    import torch
    n = int(mass.numel())
    _check(_L().irs_shoot_rays(C.c_void_p(plan), _ptr(lens_xy, torch.float64, "lens_xy") if n else None,
                               _ptr(mass, torch.float64, "mass") if n else None, n,
                               _ptr(ray_idx, torch.int64, "ray_idx"), int(ray_idx.numel()),
                               _ptr(beta, torch.float64, "beta"), _ptr(pixel, torch.int64, "pixel"),
                               _stream(stream)), "irs_shoot_rays")


def irs_make_map_brute_noalloc(params, lens_xy, mass, counts, mag=None, stream=None):
    """Brute-force map without any device allocation (see include/irs.h): the
    parameters go in directly, scratch is the library's static device array."""
    import torch
    n = int(mass.numel())
    _check(_L().irs_make_map_brute_noalloc(
        C.byref(params), _ptr(lens_xy, torch.float64, "lens_xy") if n else None,
        _ptr(mass, torch.float64, "mass") if n else None, n, _ptr(counts, torch.uint32, "counts"),
        _ptr(mag, torch.float32, "mag"), _stream(stream)), "irs_make_map_brute_noalloc")


def irs_autotune(params, lens_xy, mass, cache_path=None, stream=None):
    """Returns (tuned IrsParams, IrsTuneResult)."""
    import torch
    n = int(mass.numel())
    tuned = IrsParams()
    res = IrsTuneResult()
    _check(_L().irs_autotune(C.byref(params), _ptr(lens_xy, torch.float64, "lens_xy") if n else None,
                             _ptr(mass, torch.float64, "mass") if n else None, n,
                             cache_path.encode() if cache_path else None, C.byref(tuned),
                             C.byref(res), _stream(stream)), "irs_autotune")
    return tuned, res


def irs_mlp_train(plan, lens_xy, mass, n_samples=0, steps=0, seed=1, stream=None):
    import torch
    n = int(mass.numel())
    rep = IrsMlpReport()
    _check(_L().irs_mlp_train(C.c_void_p(plan), _ptr(lens_xy, torch.float64, "lens_xy") if n else None,
                              _ptr(mass, torch.float64, "mass") if n else None, n, int(n_samples),
                              int(steps), int(seed), C.byref(rep), _stream(stream)), "irs_mlp_train")
    return rep


def irs_mlp_params(plan, theta_in=None, freq_in=None):
    """Set (numpy float32 arrays, optional) and return (theta, freq) as numpy arrays."""
    import numpy as np
    fp = C.POINTER(C.c_float)
    tin = None if theta_in is None else np.ascontiguousarray(theta_in, dtype=np.float32)
    fin = None if freq_in is None else np.ascontiguousarray(freq_in, dtype=np.float32)
    tout = np.zeros(13000, dtype=np.float32)
    fout = np.zeros(64, dtype=np.float32)
    _check(_L().irs_mlp_params(C.c_void_p(plan), None if tin is None else tin.ctypes.data_as(fp),
                               None if fin is None else fin.ctypes.data_as(fp),
                               tout.ctypes.data_as(fp), fout.ctypes.data_as(fp)), "irs_mlp_params")
    return tout, fout.reshape(32, 2)


def irs_mlp_grad(plan, x, t, stream=None):
    """x: (n, 2) float32 CUDA, t: (n, 8) float32 CUDA -> (grad (13000,) float32, loss_sum) on CUDA."""
    import torch
    grad = torch.empty(13000, dtype=torch.float32, device=x.device)
    loss = torch.empty(1, dtype=torch.float64, device=x.device)
    _check(_L().irs_mlp_grad(C.c_void_p(plan), _ptr(x, torch.float32, "x"), _ptr(t, torch.float32, "t"),
                             int(x.shape[0]), _ptr(grad), _ptr(loss), _stream(stream)), "irs_mlp_grad")
    return grad, loss


def irs_mlp_forward(plan, x, stream=None):
    import torch
    y = torch.empty((x.shape[0], 8), dtype=torch.float32, device=x.device)
    _check(_L().irs_mlp_forward(C.c_void_p(plan), _ptr(x, torch.float32, "x"), int(x.shape[0]), _ptr(y),
                                _stream(stream)), "irs_mlp_forward")
    return y


def irs_plan_sync(plan, stream=None):
    _check(_L().irs_plan_sync(C.c_void_p(plan), _stream(stream)), "irs_plan_sync")


def irs_plan_destroy(plan):
    _check(_L().irs_plan_destroy(C.c_void_p(plan)), "irs_plan_destroy")


class Plan:
    """Owning wrapper: Plan(params) ... plan.close() (or use as a context manager)."""

    def __init__(self, params, stream=None):
        self.params = params
        self.handle = irs_plan(params, stream)
        self.info = irs_plan_info_get(self.handle)

    def make_map(self, lens_xy, mass, counts=None, mag=None, stream=None, with_mag=True):
        import torch
        shape = (self.params.npix_y, self.params.npix_x)
        dev = mass.device
        if counts is None:
            counts = torch.empty(shape, dtype=torch.uint32, device=dev)
        if mag is None and with_mag:
            mag = torch.empty(shape, dtype=torch.float32, device=dev)
        irs_make_map(self.handle, lens_xy, mass, counts, mag, stream)
        return counts, mag

    def shoot_rays(self, lens_xy, mass, ray_idx, stream=None):
        import torch
        k = int(ray_idx.numel())
        beta = torch.empty((k, 2), dtype=torch.float64, device=ray_idx.device)
        pix = torch.empty((k,), dtype=torch.int64, device=ray_idx.device)
        irs_shoot_rays(self.handle, lens_xy, mass, ray_idx, beta, pix, stream)
        return beta, pix

    def sync(self, stream=None):
        irs_plan_sync(self.handle, stream)

    def close(self):
        if self.handle:
            irs_plan_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
