"""Thin ctypes binding of libflamerec.so (include/flamerec.h).

Argument marshalling only: torch tensors supply device memory and the CUDA
stream; every step of the reconstruction runs in the library's kernels.  There
is no CPU fallback: loading fails loudly when the library is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libflamerec.so")

FR_OK, FR_EINVAL, FR_ENOMEM, FR_ECUDA, FR_ETIMEDOUT, FR_EBUSY, FR_ECANCELED, FR_ERANGE = range(8)
FR_F32, FR_BF16, FR_F16 = 0, 1, 2
FR_KIND_RGB, FR_KIND_TEMP = 0, 1
FR_RULE_PAPER, FR_RULE_GRADIENT = 0, 1
FR_MAX_VIEWS = 32
PHASES = ("setup", "scatter", "pack", "forward", "reduce", "adjust", "apply", "finish")
FR_PHASE_COUNT = len(PHASES)

STATUS_NAMES = {0: "FR_OK", 1: "FR_EINVAL", 2: "FR_ENOMEM", 3: "FR_ECUDA", 4: "FR_ETIMEDOUT",
                5: "FR_EBUSY", 6: "FR_ECANCELED", 7: "FR_ERANGE"}


class FrError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class fr_volume(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("kind", ctypes.c_int32), ("dtype", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("origin", ctypes.c_float * 3), ("h", ctypes.c_float), ("data", ctypes.c_void_p)]


class fr_camera(ctypes.Structure):
    _fields_ = [("pos", ctypes.c_float * 3), ("right", ctypes.c_float * 3), ("up", ctypes.c_float * 3),
                ("fwd", ctypes.c_float * 3), ("tan_half_fov", ctypes.c_float), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32), ("pad_", ctypes.c_int32)]


class fr_problem(ctypes.Structure):
    _fields_ = [("vol", fr_volume), ("cams", ctypes.c_void_p), ("ncam", ctypes.c_int32),
                ("pad_", ctypes.c_int32), ("targets", ctypes.c_void_p), ("bbox", ctypes.c_void_p),
                ("rmse", ctypes.c_void_p), ("hull_tags", ctypes.c_void_p)]


class fr_job_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32), ("alpha_l", ctypes.c_float),
                ("origin", ctypes.c_float * 3), ("h", ctypes.c_float), ("cams", ctypes.c_void_p),
                ("ncam", ctypes.c_int32), ("iters", ctypes.c_int32), ("init_records", ctypes.c_void_p),
                ("targets", ctypes.c_void_p), ("result_records", ctypes.c_void_p), ("rmse", ctypes.c_void_p),
                ("hull_tags", ctypes.c_void_p)]


class fr_job_info(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("iters_done", ctypes.c_int32), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double), ("footprint", ctypes.c_size_t)]


FR_JOB_QUEUED, FR_JOB_RUNNING, FR_JOB_DONE, FR_JOB_CANCELED = range(4)


class fr_params(ctypes.Structure):
    _fields_ = [("step", ctypes.c_float), ("alpha_l", ctypes.c_float), ("alpha_d", ctypes.c_float),
                ("tau", ctypes.c_float), ("g_std", ctypes.c_float), ("flame_thresh", ctypes.c_float),
                ("seed", ctypes.c_uint64), ("clamp_nonneg", ctypes.c_int32), ("rule", ctypes.c_int32),
                ("grad_step", ctypes.c_float), ("update_sigma", ctypes.c_int32),
                ("lut_t_min", ctypes.c_float), ("lut_t_max", ctypes.c_float), ("lut", ctypes.c_void_p),
                ("lut_size", ctypes.c_int32), ("use_hull", ctypes.c_int32),
                ("skip_empty", ctypes.c_int32), ("hull_tags", ctypes.c_void_p), ("hg_g", ctypes.c_float),
                ("sequential_views", ctypes.c_int32), ("tables", ctypes.c_int32)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_F = ctypes.c_float
_S = ctypes.c_int  # fr_status

# name -> (restype, argtypes), exactly the declarations of include/flamerec.h
SIGNATURES = {
    "fr_abi_version": (ctypes.c_int32, []),
    "fr_params_default": (None, [_P]),
    "fr_create": (_S, [_P, _I, _P]),
    "fr_destroy": (_S, [_P]),
    "fr_set_stream": (_S, [_P, _P]),
    "fr_last_error": (ctypes.c_char_p, [_P]),
    "fr_synchronize": (_S, [_P]),
    "fr_prepare_targets": (_S, [_P, _I, _I, _I, _P, _F, _P]),
    "fr_render": (_S, [_P, _P, _P, _I, _P, _P]),
    "fr_render_residual": (_S, [_P, _P, _P, _I, _P, _P, _P, _P, _P, _P]),
    "fr_adjust": (_S, [_P, _P, _P, _I, _P, _P, _I, _P]),
    "fr_apply_update": (_S, [_P, _P, _P, _F, _I, _I, _I]),
    "fr_render_backward": (_S, [_P, _P, _P, _I, _P, _P, _P, _P]),
    "fr_scatter_source": (_S, [_P, _P, _P, _P, _P]),
    "fr_planck_lut": (_S, [_P, _F, _F, _I, _P]),
    "fr_reconstruct": (_S, [_P, _P, _P, _P, _I, _P, _I, _P, _I, _I, _P, _P, _I]),
    "fr_reconstruct_until": (_S, [_P, _P, _P, _P, _I, _P, _I, _P, _I, _F, _I, _P, _P, _I, _P]),
    "fr_count_samples": (_S, [_P, _P, _P, _I, _P, _P, _P]),
    "fr_reconstruct_batch": (_S, [_P, _P, _I, _I, _I, _P, _I]),
    "fr_visual_hull": (_S, [_P, _P, _P, _I, _P, _P, _P]),
    "fr_server_create": (_S, [_P, _P, _I, ctypes.c_size_t, _P]),
    "fr_server_destroy": (_S, [_P]),
    "fr_server_submit": (_S, [_P, _P, _P]),
    "fr_server_step": (_S, [_P, _P, _P]),
    "fr_job_get_info": (_S, [_P, _P]),
    "fr_job_wait": (_S, [_P, _P, _I]),
    "fr_job_cancel": (_S, [_P, _P]),
    "fr_job_release": (_S, [_P, _P]),
    "fr_server_memory": (_S, [_P, _P, _P]),
    "fr_volume_rmse": (_S, [_P, _P, _P, _P, ctypes.c_uint32, _P, _P]),
    "fr_temperature_from_green": (_S, [_P, _P, _P, _P]),
    "fr_camera_from_projection": (_S, [_P, _I, _I, _P]),
    "fr_volume_dims": (_S, [_P, _I, _P, _P, _F, _P, _P, _P]),
    "fr_trace_phases": (_S, [_P, _I]),
    "fr_checks_enabled": (ctypes.c_int32, []),
    "fr_brick_cells": (ctypes.c_int32, []),
    "fr_check_word": (_S, [_P, _P, _I]),
    "fr_set_scratch_limit": (_S, [_P, ctypes.c_size_t]),
    "fr_scratch_bytes": (_S, [_P, _P]),
    "fr_phase_times": (_S, [_P, _P, _I, _P]),
    "fr_table_stats": (_S, [_P, _P]),
    "fr_render_residual_noalloc": (_S, [_I, _P, _P, _P, _I, _P, _P, _P, _P, _P, _P, ctypes.c_char_p,
                                        ctypes.c_size_t]),
    "fr_volume_create": (_S, [_P, _I, _I, _I, _P, _F, _I, _I, _P]),
    "fr_volume_free": (_S, [_P, _P]),
    "fr_volume_upload": (_S, [_P, _P, _P, _I]),
    "fr_volume_download": (_S, [_P, _P, _P, _I]),
    "fr_cams_create": (_S, [_I, _P, _P, _P]),
    "fr_cams_ring": (_S, [_I, _I, _I, _P, _F, _F, _P, _F, _P]),
    "fr_cams_count": (ctypes.c_int32, [_P]),
    "fr_cams_data": (_P, [_P]),
    "fr_cams_destroy": (_S, [_P]),
}

_lib = None


def load():
    """Load the library (building it first if its sources are newer).  With
    FR_LIBRARY_VARIANT=checked in the environment, the bounds-checked build."""
    global _lib
    if _lib is not None:
        return _lib
    from . import build as _build
    path = _build.build(checked=os.environ.get("FR_LIBRARY_VARIANT") == "checked")
    if not os.path.exists(path):
        raise FrError(FR_ECUDA, f"libflamerec.so missing at {path}")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(t):
    """Device (or host) address of a torch tensor or numpy array, or None."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def params(**kw) -> fr_params:
    p = fr_params()
    load().fr_params_default(ctypes.byref(p))
    for k, v in kw.items():
        if k == "lut":
            p.lut = _ptr(v)
            if v is not None:
                p.lut_size = int(v.shape[0])
            continue
        if k == "hull_tags":
            p.hull_tags = _ptr(v)
            continue
        if not hasattr(p, k):
            raise AttributeError(f"fr_params has no field {k}")
        setattr(p, k, v)
    return p


def cameras(cams) -> ctypes.Array:
    """fr_camera array from dicts with pos, right, up, fwd, tan_half_fov, width, height."""
    arr = (fr_camera * len(cams))()
    for c, s in zip(arr, cams):
        for key in ("pos", "right", "up", "fwd"):
            setattr(c, key, (ctypes.c_float * 3)(*[float(x) for x in s[key]]))
        c.tan_half_fov = float(s["tan_half_fov"])
        c.width, c.height = int(s["width"]), int(s["height"])
    return arr


def fr_render_residual_noalloc(device, stream, vol, cams, p, targets, bbox, rendered, residual, sq_err):
    """fr_render_residual without any allocation (fixed library scratch).
    stream: a torch.cuda.Stream (or None for the default stream)."""
    lib = load()
    err = ctypes.create_string_buffer(512)
    h = ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)
    st = lib.fr_render_residual_noalloc(int(device), h, ctypes.byref(vol), cams, len(cams), ctypes.byref(p),
                                        _ptr(targets), _ptr(bbox), _ptr(rendered), _ptr(residual),
                                        _ptr(sq_err), err, len(err))
    if st != FR_OK:
        raise FrError(st, err.value.decode())


_DT = {"float32": FR_F32, "bfloat16": FR_BF16, "float16": FR_F16}


def volume(t, origin, h, kind=FR_KIND_RGB) -> fr_volume:
    """Descriptor of a (nz, ny, nx, C) CUDA tensor (C = 4 for RGB, 2 for TEMP)."""
    if not t.is_cuda or not t.is_contiguous():
        raise FrError(FR_EINVAL, "volume tensor must be a contiguous CUDA tensor")
    nz, ny, nx, ncomp = t.shape
    if ncomp != (4 if kind == FR_KIND_RGB else 2):
        raise FrError(FR_EINVAL, f"kind {kind} needs {4 if kind == FR_KIND_RGB else 2} components, got {ncomp}")
    dt = _DT.get(str(t.dtype).replace("torch.", ""))
    if dt is None:
        raise FrError(FR_EINVAL, f"unsupported storage dtype {t.dtype}")
    v = fr_volume()
    v.nx, v.ny, v.nz, v.kind, v.dtype = nx, ny, nz, kind, dt
    v.origin = (ctypes.c_float * 3)(*[float(x) for x in origin])
    v.h = float(h)
    v.data = t.data_ptr()
    return v


class Cams:
    """A camera set held by the library (fr_cams).  .array is the fr_camera
    array the entry points take; len() is its count."""

    def __init__(self, handle):
        self.lib, self.h = load(), handle
        n = self.lib.fr_cams_count(handle)
        ptr = self.lib.fr_cams_data(handle)
        self.array = ctypes.cast(ptr, ctypes.POINTER(fr_camera * n)).contents

    def __len__(self):
        return len(self.array)

    def as_dicts(self):
        return [dict(pos=list(c.pos), right=list(c.right), up=list(c.up), fwd=list(c.fwd),
                     tan_half_fov=c.tan_half_fov, width=c.width, height=c.height) for c in self.array]

    def close(self):
        if getattr(self, "h", None):
            self.lib.fr_cams_destroy(self.h)
            self.h = None
            self.array = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cams_create(projections, sizes) -> Cams:
    """fr_cams_create: cameras from 3x4 projection matrices and (width, height) pairs."""
    P = np.ascontiguousarray(projections, dtype=np.float64).reshape(-1, 12)
    wh = np.ascontiguousarray(sizes, dtype=np.int32).reshape(-1, 2)
    if len(P) != len(wh):
        raise FrError(FR_EINVAL, "one size per projection")
    h = ctypes.c_void_p()
    st = load().fr_cams_create(len(P), P.ctypes.data, wh.ctypes.data, ctypes.byref(h))
    if st != FR_OK:
        raise FrError(st, "fr_cams_create rejected the projections")
    return Cams(h)


def cams_ring(k, width, height, center=(0.0, 0.0, 0.0), radius=2.0, fov_deg=60.0, elevation_deg=None,
              phase=0.0) -> Cams:
    """fr_cams_ring: k cameras on a ring around `center` looking at it."""
    c = (ctypes.c_float * 3)(*[float(x) for x in center])
    el = None
    if elevation_deg is not None:
        el = np.ascontiguousarray(elevation_deg, dtype=np.float32)
        if el.shape != (k,):
            raise FrError(FR_EINVAL, "one elevation per camera")
    h = ctypes.c_void_p()
    st = load().fr_cams_ring(int(k), int(width), int(height), c, float(radius), float(fov_deg),
                             el.ctypes.data if el is not None else None, float(phase), ctypes.byref(h))
    if st != FR_OK:
        raise FrError(st, "fr_cams_ring rejected its arguments")
    return Cams(h)


def camera_from_projection(P, width, height):
    """fr_camera (as a dict like synth's cameras) from a 3x4 projection matrix."""
    arr = np.ascontiguousarray(P, dtype=np.float64).reshape(12)
    cam = fr_camera()
    st = load().fr_camera_from_projection(arr.ctypes.data, int(width), int(height), ctypes.byref(cam))
    if st != FR_OK:
        raise FrError(st, "projection not representable by the pinhole model (square pixels, no skew, "
                          "centred principal point)")
    return dict(pos=list(cam.pos), right=list(cam.right), up=list(cam.up), fwd=list(cam.fwd),
                tan_half_fov=cam.tan_half_fov, width=cam.width, height=cam.height)


def volume_dims(cams, box_min, box_max, alpha=1.5):
    """Sec. 4.2 volume dimensions: (dims (nx, ny, nz), voxel edge h, pixels per edge n)."""
    fc = cameras(cams)
    lo = (ctypes.c_float * 3)(*box_min)
    hi = (ctypes.c_float * 3)(*box_max)
    dims = (ctypes.c_int32 * 3)()
    h = ctypes.c_float()
    n = (ctypes.c_float * 3)()
    st = load().fr_volume_dims(fc, len(cams), lo, hi, float(alpha), dims, ctypes.byref(h), n)
    if st != FR_OK:
        raise FrError(st, "no volume dimensions (box behind a camera or empty)")
    return tuple(dims), h.value, tuple(n)


def _nvtx(fn):
    """NVTX range named after the entry point around the call (visible in
    Nsight timelines), when torch's CUDA NVTX bindings are present."""
    import functools
    name = fn.__name__

    @functools.wraps(fn)
    def wrapper(*a, **k):
        nv = _nvtx_module()
        if nv is None:
            return fn(*a, **k)
        nv.range_push(name)
        try:
            return fn(*a, **k)
        finally:
            nv.range_pop()
    return wrapper


_NVTX = []


def _nvtx_module():
    if not _NVTX:
        try:
            import torch
            _NVTX.append(torch.cuda.nvtx if torch.cuda.is_available() else None)
        except Exception:  # torch absent or without CUDA: no ranges
            _NVTX.append(None)
    return _NVTX[0]


class Context:
    """An fr_ctx bound to a device and a stream (torch's current one by default)."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        self.lib = load()
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self._stream = stream
        h = ctypes.c_void_p()
        st = self.lib.fr_create(ctypes.byref(h), device, ctypes.c_void_p(stream.cuda_stream))
        if st != FR_OK:
            raise FrError(st, "fr_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.fr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, status):
        if status != FR_OK:
            raise FrError(status, self.lib.fr_last_error(self.h).decode())

    # -- the C ABI, one method per entry point ------------------------------

    def fr_prepare_targets(self, targets, thresh, bbox):
        k, h, w, _ = targets.shape
        self.check(self.lib.fr_prepare_targets(self.h, k, h, w, _ptr(targets), float(thresh), _ptr(bbox)))

    @_nvtx
    def fr_render(self, vol: fr_volume, cams, p: fr_params, out):
        self.check(self.lib.fr_render(self.h, ctypes.byref(vol), cams, len(cams), ctypes.byref(p), _ptr(out)))

    @_nvtx
    def fr_render_residual(self, vol, cams, p, targets, bbox, rendered, residual, sq_err):
        self.check(self.lib.fr_render_residual(self.h, ctypes.byref(vol), cams, len(cams), ctypes.byref(p),
                                               _ptr(targets), _ptr(bbox), _ptr(rendered), _ptr(residual),
                                               _ptr(sq_err)))

    @_nvtx
    def fr_adjust(self, vol, cams, p, residual, iteration, dV):
        self.check(self.lib.fr_adjust(self.h, ctypes.byref(vol), cams, len(cams), ctypes.byref(p),
                                      _ptr(residual), int(iteration), _ptr(dV)))

    def fr_apply_update(self, vol, dV, scale=1.0, with_sigma=False, clamp_nonneg=True, zero_dV=True):
        self.check(self.lib.fr_apply_update(self.h, ctypes.byref(vol), _ptr(dV), float(scale), int(with_sigma),
                                            int(clamp_nonneg), int(zero_dV)))

    @_nvtx
    def fr_render_backward(self, vol, cams, p, L_total, grad_img, grad):
        self.check(self.lib.fr_render_backward(self.h, ctypes.byref(vol), cams, len(cams), ctypes.byref(p),
                                               _ptr(L_total), _ptr(grad_img), _ptr(grad)))

    @_nvtx
    def fr_scatter_source(self, emission, albedo, J, out):
        self.check(self.lib.fr_scatter_source(self.h, ctypes.byref(emission), _ptr(albedo), _ptr(J),
                                              ctypes.byref(out)))

    def fr_planck_lut(self, t_min, t_max, lut):
        self.check(self.lib.fr_planck_lut(self.h, float(t_min), float(t_max), int(lut.shape[0]), _ptr(lut)))

    @_nvtx
    def fr_reconstruct(self, vol, cams, targets, bbox, iters, p, albedo=None, first_iteration=0,
                       rmse=None, targets_are_host=None):
        if targets_are_host is None:
            targets_are_host = not getattr(targets, "is_cuda", False)
        rmse_is_host = rmse is not None and not getattr(rmse, "is_cuda", False)
        self.check(self.lib.fr_reconstruct(self.h, ctypes.byref(vol), _ptr(albedo), cams, len(cams),
                                           _ptr(targets), int(bool(targets_are_host)), _ptr(bbox), int(iters),
                                           int(first_iteration), ctypes.byref(p), _ptr(rmse),
                                           int(rmse_is_host)))

    @_nvtx
    def fr_reconstruct_until(self, vol, cams, targets, bbox, max_iters, stop_delta, p, albedo=None,
                             first_iteration=0, rmse=None, targets_are_host=None):
        """Iterates until the image error changes by less than stop_delta; returns the iterations run."""
        if targets_are_host is None:
            targets_are_host = not getattr(targets, "is_cuda", False)
        rmse_is_host = rmse is not None and not getattr(rmse, "is_cuda", False)
        done = ctypes.c_int32()
        self.check(self.lib.fr_reconstruct_until(self.h, ctypes.byref(vol), _ptr(albedo), cams, len(cams),
                                                 _ptr(targets), int(bool(targets_are_host)), _ptr(bbox),
                                                 int(max_iters), float(stop_delta), int(first_iteration),
                                                 ctypes.byref(p), _ptr(rmse), int(rmse_is_host),
                                                 ctypes.byref(done)))
        return done.value

    def fr_temperature_from_green(self, rgb, p, temp):
        self.check(self.lib.fr_temperature_from_green(self.h, ctypes.byref(rgb), ctypes.byref(p),
                                                      ctypes.byref(temp)))

    def fr_volume_rmse(self, a, b, tags=None, full_mask=0):
        """(rmse per colour channel, key points compared) of two RGB volumes (fr_volume)."""
        out = (ctypes.c_float * 3)()
        n = ctypes.c_int64()
        self.check(self.lib.fr_volume_rmse(self.h, ctypes.byref(a), ctypes.byref(b), _ptr(tags), int(full_mask),
                                           out, ctypes.byref(n)))
        return np.array(list(out), dtype=np.float64), n.value

    def fr_check_word(self, reset=False):
        w = ctypes.c_uint32()
        self.check(self.lib.fr_check_word(self.h, ctypes.byref(w), int(bool(reset))))
        return w.value

    def fr_set_scratch_limit(self, nbytes):
        self.check(self.lib.fr_set_scratch_limit(self.h, int(nbytes)))

    def fr_scratch_bytes(self):
        n = ctypes.c_size_t()
        self.check(self.lib.fr_scratch_bytes(self.h, ctypes.byref(n)))
        return n.value

    def fr_trace_phases(self, on=True):
        self.check(self.lib.fr_trace_phases(self.h, int(bool(on))))

    def fr_phase_times(self):
        """(dict phase name -> milliseconds summed over the recorded calls, calls)."""
        ms = (ctypes.c_float * FR_PHASE_COUNT)()
        calls = ctypes.c_int32()
        self.check(self.lib.fr_phase_times(self.h, ms, FR_PHASE_COUNT, ctypes.byref(calls)))
        return dict(zip(PHASES, list(ms))), calls.value

    def fr_table_stats(self):
        """Sizes of the ray weight tables of the last reconstruction call: dict of
        forward_entries, adjustment_entries, flame_rays, hull_key_points."""
        st = (ctypes.c_uint64 * 4)()
        self.check(self.lib.fr_table_stats(self.h, st))
        return dict(zip(("forward_entries", "adjustment_entries", "flame_rays", "hull_key_points"), list(st)))

    def fr_count_samples(self, vol, cams, p, residual=None):
        n = ctypes.c_int64()
        self.check(self.lib.fr_count_samples(self.h, ctypes.byref(vol), cams, len(cams), ctypes.byref(p),
                                             _ptr(residual), ctypes.byref(n)))
        return n.value

    @_nvtx
    def fr_reconstruct_batch(self, problems, iters, p, first_iteration=0, use_graph=True):
        """problems: sequence of (fr_volume, camera array, targets, bbox, rmse or None[, hull tags or None])."""
        arr = (fr_problem * len(problems))()
        keep = []
        for q, prob in zip(arr, problems):
            vol, cams, targets, bbox, rmse = prob[:5]
            q.vol = vol
            q.cams = ctypes.cast(cams, ctypes.c_void_p)
            q.ncam = len(cams)
            q.targets, q.bbox, q.rmse = _ptr(targets), _ptr(bbox), _ptr(rmse)
            q.hull_tags = _ptr(prob[5]) if len(prob) > 5 else None
            keep.append(cams)
        self.check(self.lib.fr_reconstruct_batch(self.h, arr, len(problems), int(iters), int(first_iteration),
                                                 ctypes.byref(p), int(bool(use_graph))))

    @_nvtx
    def fr_visual_hull(self, vol, cams, targets, p, tags):
        self.check(self.lib.fr_visual_hull(self.h, ctypes.byref(vol), cams, len(cams), _ptr(targets),
                                           ctypes.byref(p), _ptr(tags)))

    def fr_synchronize(self):
        self.check(self.lib.fr_synchronize(self.h))

    def fr_volume_create(self, shape, origin, h, kind=FR_KIND_RGB, dtype=FR_F32) -> fr_volume:
        """A volume whose records the library allocates (zeroed); shape (nx, ny, nz)."""
        v = fr_volume()
        o = (ctypes.c_float * 3)(*[float(x) for x in origin])
        nx, ny, nz = shape
        self.check(self.lib.fr_volume_create(self.h, int(nx), int(ny), int(nz), o, float(h), int(kind), int(dtype),
                                             ctypes.byref(v)))
        return v

    def fr_volume_free(self, vol):
        self.check(self.lib.fr_volume_free(self.h, ctypes.byref(vol)))

    @_nvtx
    def fr_volume_upload(self, vol, src):
        """src: float32 records, a host numpy array or a CUDA tensor."""
        host = isinstance(src, np.ndarray)
        if host:
            src = np.ascontiguousarray(src, dtype=np.float32)
        self.check(self.lib.fr_volume_upload(self.h, ctypes.byref(vol), _ptr(src), int(host)))
        return src

    @_nvtx
    def fr_volume_download(self, vol, dst):
        """dst: float32 records, a host numpy array (filled on return) or a CUDA tensor."""
        host = isinstance(dst, np.ndarray)
        if host and (dst.dtype != np.float32 or not dst.flags["C_CONTIGUOUS"]):
            raise FrError(FR_EINVAL, "dst must be a contiguous float32 array")
        self.check(self.lib.fr_volume_download(self.h, ctypes.byref(vol), _ptr(dst), int(host)))
        return dst


class Job:
    """A submitted job: keeps its host buffers alive until it is released."""

    def __init__(self, server, handle, keep, result, rmse):
        self.server, self.h, self._keep, self.result, self.rmse = server, handle, keep, result, rmse

    def info(self) -> fr_job_info:
        info = fr_job_info()
        self.server.ctx.check(self.server.lib.fr_job_get_info(self.h, ctypes.byref(info)))
        return info

    def wait(self, timeout_ms=60000):
        self.server.ctx.check(self.server.lib.fr_job_wait(self.server.h, self.h, int(timeout_ms)))

    def cancel(self):
        self.server.ctx.check(self.server.lib.fr_job_cancel(self.server.h, self.h))

    def release(self):
        if self.h:
            self.server.ctx.check(self.server.lib.fr_job_release(self.server.h, self.h))
            self.h = None


class Server:
    """fr_server: continuous-batching reconstruction jobs (see include/flamerec.h)."""

    def __init__(self, ctx: Context, p: fr_params, dtype=FR_BF16, budget_bytes=0):
        self.ctx, self.lib = ctx, ctx.lib
        self.dtype = dtype
        self._p = p
        h = ctypes.c_void_p()
        ctx.check(self.lib.fr_server_create(ctx.h, ctypes.byref(p), int(dtype), ctypes.c_size_t(budget_bytes),
                                            ctypes.byref(h)))
        self.h = h

    def submit(self, shape, origin, h, cams, iters, init_records, targets, want_rmse=True, alpha_l=0.0,
               hull_tags=None) -> Job:
        """init_records: host numpy array (nz, ny, nx, 4) in the server's storage type
        (uint16 bit patterns for bf16/f16, float32 otherwise); targets: host float32
        (K, H, W, 3); hull_tags: host uint32 (nz, ny, nx) tags used instead of the
        job's own hull (servers with use_hull).  Returns a Job whose .result
        receives the reconstruction."""
        nx, ny, nz = shape
        init = np.ascontiguousarray(init_records)
        tgt = np.ascontiguousarray(targets, dtype=np.float32)
        result = np.empty_like(init)
        rmse = np.zeros((iters, 3), dtype=np.float32) if want_rmse else None
        fcams = cameras(cams)
        d = fr_job_desc()
        d.nx, d.ny, d.nz = nx, ny, nz
        d.alpha_l = float(alpha_l)
        d.origin = (ctypes.c_float * 3)(*[float(x) for x in origin])
        d.h = float(h)
        d.cams = ctypes.cast(fcams, ctypes.c_void_p)
        d.ncam, d.iters = len(cams), int(iters)
        d.init_records, d.targets, d.result_records = init.ctypes.data, tgt.ctypes.data, result.ctypes.data
        d.rmse = rmse.ctypes.data if rmse is not None else None
        tags = np.ascontiguousarray(hull_tags, dtype=np.uint32) if hull_tags is not None else None
        d.hull_tags = tags.ctypes.data if tags is not None else None
        jh = ctypes.c_void_p()
        self.ctx.check(self.lib.fr_server_submit(self.h, ctypes.byref(d), ctypes.byref(jh)))
        return Job(self, jh, (init, tgt, fcams, tags), result, rmse)

    @_nvtx
    def step(self):
        running, queued = ctypes.c_int(), ctypes.c_int()
        self.ctx.check(self.lib.fr_server_step(self.h, ctypes.byref(running), ctypes.byref(queued)))
        return running.value, queued.value

    def memory(self):
        used, budget = ctypes.c_size_t(), ctypes.c_size_t()
        self.ctx.check(self.lib.fr_server_memory(self.h, ctypes.byref(used), ctypes.byref(budget)))
        return used.value, budget.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.fr_server_destroy(self.h)
            self.h = None
