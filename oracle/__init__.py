"""FP64 CPU oracle for the flame reconstruction loop (arXiv 1809.06417).

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the GPU library: it is a plain C restatement of the paper's steps
(Sec. 3.2 rendering model, Sec. 3.3 reconstruction, Algorithm 2) compiled with
gcc and called through ctypes.  The C source documents each step and every
reading of the paper it takes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "flame_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no target-specific flags), with
    OpenMP when the compiler has it (the pixel loops can then run on several
    threads, see set_threads), else without."""
    os.makedirs(_BUILD, exist_ok=True)
    fresh = os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)
    if fresh and not force:
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off"]
    r = subprocess.run(base + ["-fopenmp", _SRC, "-o", tmp, "-lm"], capture_output=True, text=True)
    if r.returncode != 0:
        subprocess.run(base + [_SRC, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("pad_", ctypes.c_int32), ("origin", ctypes.c_double * 3), ("h", ctypes.c_double)]


class Cam(ctypes.Structure):
    _fields_ = [("pos", ctypes.c_double * 3), ("right", ctypes.c_double * 3),
                ("up", ctypes.c_double * 3), ("fwd", ctypes.c_double * 3),
                ("tan_half_fov", ctypes.c_double), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32)]


class Params(ctypes.Structure):
    _fields_ = [("step", ctypes.c_double), ("alpha_l", ctypes.c_double),
                ("alpha_d", ctypes.c_double), ("tau", ctypes.c_double),
                ("g_std", ctypes.c_double), ("flame_thresh", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("clamp_nonneg", ctypes.c_int32),
                ("pad_", ctypes.c_int32), ("hg_g", ctypes.c_double), ("sequential", ctypes.c_int32),
                ("storage", ctypes.c_int32)]

# 16-bit storage types of orc_round_storage / Params.storage
STORAGE = {None: 0, "f64": 0, "bf16": 1, "f16": 2}
# visual hull: margin (pixels) within which a rectangle edge near a pixel
# centre leaves a tag bit undecided, and the same for a corner near the camera
# plane (voxels).  A float32 evaluation of the projection, one rounding per
# operation, stays within 1.4e-4 pixels and 1e-4 voxels of the double-precision
# one on ring cameras up to 192^3 grids and 768-pixel images
# (tests/test_oracle_hull.py measures it), so decisions outside these margins
# are the same in both precisions.
HULL_EPS = 1e-3
HULL_EPS_Z = 1e-3


class Lut(ctypes.Structure):
    _fields_ = [("lut", ctypes.POINTER(ctypes.c_double)), ("m", ctypes.c_int32),
                ("pad_", ctypes.c_int32), ("t_min", ctypes.c_double), ("t_max", ctypes.c_double)]


_P = ctypes.c_void_p
_I64 = ctypes.c_int64


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        sig = {
            "orc_render": (_I64, [_P, _P, _P, ctypes.c_int, _P, _P, _P]),
            "orc_render_temp": (_I64, [_P, _P, _P, _P, ctypes.c_int, _P, _P]),
            "orc_render_pixels": (_I64, [_P, _P, _P, _P, _I64, _P, _P]),
            "orc_trace_pixel": (_I64, [_P, _P, _P, _P, ctypes.c_int, ctypes.c_int, _I64, _P, _P, _P]),
            "orc_prepare_targets": (None, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _P,
                                           ctypes.c_double, _P, _P]),
            "orc_residual": (None, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P, _P]),
            "orc_update_paper": (_I64, [_P, _P, _P, ctypes.c_int, _P, _P, _P, ctypes.c_int, _P, _P]),
            "orc_set_undecided_margins": (None, [ctypes.c_double, ctypes.c_double]),
            "orc_apply_update": (None, [_I64, _P, _P, ctypes.c_int]),
            "orc_grad": (None, [_P, _P, _P, ctypes.c_int, _P, _P, _P, _P]),
            "orc_grad_temp": (None, [_P, _P, _P, _P, ctypes.c_int, _P, _P, _P, _P]),
            "orc_scatter_J": (None, [_P, _P, _P]),
            "orc_scatter_source": (None, [_I64, _P, _P, _P, _P]),
            "orc_reconstruct": (None, [_P, _P, _P, _P, ctypes.c_int, _P, _P, _P, _P,
                                       ctypes.c_int, ctypes.c_int, _P, _P, _P, ctypes.c_double, _P, _P]),
            "orc_visual_hull": (None, [_P, _P, ctypes.c_int, _P, _P, _P, ctypes.c_double, ctypes.c_double]),
            "orc_set_threads": (None, [ctypes.c_int]),
            "orc_threads": (ctypes.c_int, []),
            "orc_round_storage": (None, [_I64, _P, ctypes.c_int]),
            "orc_volume_rmse": (_I64, [_I64, _P, _P, _P, ctypes.c_uint32, _P]),
            "orc_volume_dims": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.c_double, _P, _P, _P]),
            "orc_scatter_L6": (None, [_P, _P, _P]),
            "orc_hg_weights": (None, [ctypes.c_double, _P, _P]),
            "orc_scatter_source_hg": (None, [_I64, _P, _P, _P, _P, _P]),
            "orc_planck": (ctypes.c_double, [ctypes.c_double, ctypes.c_double]),
            "orc_temp_rgb": (None, [ctypes.c_double, _P]),
            "orc_lut_build": (None, [ctypes.c_double, ctypes.c_double, ctypes.c_int, _P]),
            "orc_green_to_temp": (ctypes.c_double, [_P, ctypes.c_double]),
            "orc_hg_phase": (ctypes.c_double, [ctypes.c_double, ctypes.c_double]),
            "orc_g_draw": (ctypes.c_double, [ctypes.c_uint64, ctypes.c_double, ctypes.c_int,
                                             ctypes.c_int, _I64, _I64]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def make_grid(shape, origin, h) -> Grid:
    g = Grid()
    g.nx, g.ny, g.nz = (int(s) for s in shape)
    g.origin = (ctypes.c_double * 3)(*[float(x) for x in origin])
    g.h = float(h)
    return g


def make_cams(cams) -> ctypes.Array:
    """cams: sequence of dicts with pos, right, up, fwd, tan_half_fov, width, height."""
    arr = (Cam * len(cams))()
    for c, src in zip(arr, cams):
        for key in ("pos", "right", "up", "fwd"):
            setattr(c, key, (ctypes.c_double * 3)(*[float(x) for x in src[key]]))
        c.tan_half_fov = float(src["tan_half_fov"])
        c.width, c.height = int(src["width"]), int(src["height"])
    return arr


def make_params(step=1.0, alpha_l=0.001, alpha_d=1.0, tau=0.0, g_std=0.0,
                flame_thresh=30.0 / 255.0, seed=0, clamp_nonneg=1, hg_g=0.0, sequential=0,
                storage=None) -> Params:
    """storage: None / "f64" (records held in double), "bf16" or "f16" (the
    loop's stored records rounded to that type, as in 16-bit storage)."""
    p = Params()
    p.step, p.alpha_l, p.alpha_d, p.tau = float(step), float(alpha_l), float(alpha_d), float(tau)
    p.g_std, p.flame_thresh, p.seed, p.clamp_nonneg = float(g_std), float(flame_thresh), int(seed), int(clamp_nonneg)
    p.hg_g, p.sequential = float(hg_g), int(sequential)
    p.storage = STORAGE[storage]
    return p


def set_threads(n: int) -> int:
    """Threads for the oracle's pixel and node loops (1 by default); returns
    the count it will use (1 without OpenMP)."""
    lib = _load()
    lib.orc_set_threads(int(n))
    return int(lib.orc_threads())


def round_storage(x, storage):
    """x (float64 array) rounded to a 16-bit storage type ("bf16" or "f16")."""
    a = _f64(x).copy()
    _load().orc_round_storage(a.size, _ptr(a), STORAGE[storage])
    return a


def _npix(cams) -> int:
    return sum(int(c["width"]) * int(c["height"]) for c in cams)


def _check_vol(vol, grid_shape, rec):
    nx, ny, nz = grid_shape
    vol = _f64(vol)
    if vol.shape != (nz, ny, nx, rec):
        raise ValueError(f"volume must be (nz, ny, nx, {rec}) = {(nz, ny, nx, rec)}, got {vol.shape}")
    return vol


class Scene:
    """A grid plus cameras, in the oracle's own structures."""

    def __init__(self, shape, origin, h, cams):
        self.shape = tuple(int(s) for s in shape)  # (nx, ny, nz)
        self.grid = make_grid(shape, origin, h)
        self.cam_list = list(cams)
        self.cams = make_cams(cams)
        self.ncam = len(cams)
        hw = {(int(c["height"]), int(c["width"])) for c in cams}
        self.uniform = len(hw) == 1
        self.height, self.width = next(iter(hw)) if self.uniform else (None, None)

    @property
    def nodes(self):
        nx, ny, nz = self.shape
        return nx * ny * nz

    def image_shape(self):
        if not self.uniform:
            raise ValueError("views differ in size")
        return (self.ncam, self.height, self.width, 3)


def render(scene: Scene, vol, params: Params, return_t=False):
    """Eqs. 5-8: render every view.  vol (nz,ny,nx,4) {S_r,S_g,S_b,sigma}."""
    lib = _load()
    vol = _check_vol(vol, scene.shape, 4)
    out = np.zeros(3 * _npix(scene.cam_list))
    tout = np.zeros(_npix(scene.cam_list)) if return_t else None
    n = lib.orc_render(ctypes.byref(scene.grid), _ptr(vol), scene.cams, scene.ncam,
                       ctypes.byref(params), _ptr(out), _ptr(tout) if return_t else None)
    img = out.reshape(scene.image_shape()) if scene.uniform else out
    if return_t:
        return img, (tout.reshape(scene.image_shape()[:3]) if scene.uniform else tout), int(n)
    return img, int(n)


def render_pixels(scene: Scene, vol, params: Params, vpx):
    """Render only the listed (view, px, py) pixels."""
    lib = _load()
    vol = _check_vol(vol, scene.shape, 4)
    vpx = np.ascontiguousarray(np.asarray(vpx, dtype=np.int32).reshape(-1, 3))
    out = np.zeros((len(vpx), 3))
    n = lib.orc_render_pixels(ctypes.byref(scene.grid), _ptr(vol), scene.cams,
                              ctypes.byref(params), len(vpx), _ptr(vpx), _ptr(out))
    return out, int(n)


def trace_pixel(scene: Scene, vol, params: Params, view, px, py, max_n=100000):
    """Per-segment (T before the segment, length, midpoint) along one ray."""
    lib = _load()
    vol = _check_vol(vol, scene.shape, 4)
    tb, ln, pos = np.zeros(max_n), np.zeros(max_n), np.zeros((max_n, 3))
    n = lib.orc_trace_pixel(ctypes.byref(scene.grid), _ptr(vol), ctypes.byref(scene.cams[view]),
                            ctypes.byref(params), int(px), int(py), max_n, _ptr(tb), _ptr(ln), _ptr(pos))
    n = int(min(n, max_n))
    return tb[:n], ln[:n], pos[:n]


def lut_build(t_min, t_max, m):
    lib = _load()
    lut = np.zeros((m, 3))
    lib.orc_lut_build(float(t_min), float(t_max), int(m), _ptr(lut))
    return lut


def _lut_struct(lut, t_min, t_max):
    lut = _f64(lut)
    L = Lut()
    L.lut = lut.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    L.m, L.t_min, L.t_max = lut.shape[0], float(t_min), float(t_max)
    return L, lut


def green_to_temp(green, lut, t_min, t_max):
    """Sec. 3.3.3: temperatures whose table green value is `green` (array)."""
    lib = _load()
    L, keep = _lut_struct(lut, t_min, t_max)
    g = np.asarray(green, dtype=np.float64)
    out = np.array([lib.orc_green_to_temp(ctypes.byref(L), float(x)) for x in g.ravel()])
    del keep
    return out.reshape(g.shape)


def render_temp(scene: Scene, vol_ts, lut, t_min, t_max, params: Params):
    """Sec. 3.3.3: temperature records (nz,ny,nx,2) {T, sigma} through the table."""
    lib = _load()
    vol_ts = _check_vol(vol_ts, scene.shape, 2)
    L, keep = _lut_struct(lut, t_min, t_max)
    out = np.zeros(3 * _npix(scene.cam_list))
    n = lib.orc_render_temp(ctypes.byref(scene.grid), _ptr(vol_ts), ctypes.byref(L), scene.cams,
                            scene.ncam, ctypes.byref(params), _ptr(out))
    del keep
    return out.reshape(scene.image_shape()), int(n)


def prepare_targets(targets, thresh):
    """Sec. 4.1 pre-processing.  Returns (black-backed targets, mask, bbox)."""
    lib = _load()
    t = _f64(targets).copy()
    k, h, w, _ = t.shape
    mask = np.zeros((k, h, w), dtype=np.uint8)
    bbox = np.zeros((k, 4), dtype=np.int32)
    lib.orc_prepare_targets(k, h, w, _ptr(t), float(thresh), _ptr(mask), _ptr(bbox))
    return t, mask, bbox


def residual(rendered, targets, bbox):
    lib = _load()
    rendered, targets = _f64(rendered), _f64(targets)
    bbox = np.ascontiguousarray(bbox, dtype=np.int32)
    k, h, w, _ = rendered.shape
    res = np.zeros_like(rendered)
    rmse = np.zeros(3)
    lib.orc_residual(k, h, w, _ptr(rendered), _ptr(targets), _ptr(bbox), _ptr(res), _ptr(rmse))
    return res, rmse


def update_paper(scene: Scene, vol, params: Params, res, mask, iteration, with_undecided=False):
    """Eqs. 10-12: the accumulated adjustment dV (nz,ny,nx,3) and samples
    visited; with_undecided: also the per-node bound (nz,ny,nx) on what the
    samples whose cell or existence is undecided at float32-rounding margins
    can move (see set_undecided_margins)."""
    lib = _load()
    vol = _check_vol(vol, scene.shape, 4)
    res = _f64(res)
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    nx, ny, nz = scene.shape
    dV = np.zeros((nz, ny, nx, 3))
    und = np.zeros((nz, ny, nx)) if with_undecided else None
    n = lib.orc_update_paper(ctypes.byref(scene.grid), _ptr(vol), scene.cams, scene.ncam,
                             ctypes.byref(params), _ptr(res), _ptr(mask), int(iteration), _ptr(dV),
                             _ptr(und) if und is not None else None)
    return (dV, int(n), und) if with_undecided else (dV, int(n))


# Margins of the adjustment's undecided samples: a sample within FACE_EPS
# voxels of a cell face, or a ray whose chord / step lies within COUNT_EPS of
# an integer.  A float32 evaluation of the sample positions differs from the
# double-precision one by about 3e-5 voxels at 250 voxels from the camera
# (one unit in the last place there, plus the direction's rounding times the
# distance travelled), and chord / step by a few units in the last place of
# values below 1000.
FACE_EPS = 2e-4
COUNT_EPS = 1e-3


def set_undecided_margins(face_voxels=FACE_EPS, count_segments=COUNT_EPS):
    _load().orc_set_undecided_margins(float(face_voxels), float(count_segments))


def apply_update(vol, dV, clamp_nonneg=True):
    lib = _load()
    vol = _f64(vol).copy()
    dV = _f64(dV)
    lib.orc_apply_update(vol.size // 4, _ptr(vol), _ptr(dV), int(clamp_nonneg))
    return vol


def grad(scene: Scene, vol, params: Params, L_total, gimg):
    """Exact d(loss)/d(node) for RGB records, given d(loss)/d(pixel)."""
    lib = _load()
    vol = _check_vol(vol, scene.shape, 4)
    nx, ny, nz = scene.shape
    g = np.zeros((nz, ny, nx, 4))
    lib.orc_grad(ctypes.byref(scene.grid), _ptr(vol), scene.cams, scene.ncam, ctypes.byref(params),
                 _ptr(_f64(L_total)), _ptr(_f64(gimg)), _ptr(g))
    return g


def grad_temp(scene: Scene, vol_ts, lut, t_min, t_max, params: Params, L_total, gimg):
    lib = _load()
    vol_ts = _check_vol(vol_ts, scene.shape, 2)
    L, keep = _lut_struct(lut, t_min, t_max)
    nx, ny, nz = scene.shape
    g = np.zeros((nz, ny, nx, 2))
    lib.orc_grad_temp(ctypes.byref(scene.grid), _ptr(vol_ts), ctypes.byref(L), scene.cams,
                      scene.ncam, ctypes.byref(params), _ptr(_f64(L_total)), _ptr(_f64(gimg)), _ptr(g))
    del keep
    return g


def scatter_J(scene: Scene, vol):
    lib = _load()
    vol = _check_vol(vol, scene.shape, 4)
    nx, ny, nz = scene.shape
    J = np.zeros((nz, ny, nx, 3))
    lib.orc_scatter_J(ctypes.byref(scene.grid), _ptr(vol), _ptr(J))
    return J


def scatter_source(vol, albedo, J):
    lib = _load()
    vol, albedo, J = _f64(vol), _f64(albedo), _f64(J)
    out = np.zeros_like(vol)
    lib.orc_scatter_source(vol.size // 4, _ptr(vol), _ptr(albedo), _ptr(J), _ptr(out))
    return out


def visual_hull(scene: Scene, mask, with_undecided=False, eps=HULL_EPS, eps_z=HULL_EPS_Z):
    """Algorithm 1: per-node view bits (uint32, (nz, ny, nx)) from flame masks
    (K, H, W).  with_undecided: also the bits that are not fixed to a margin of
    eps pixels (rectangle edges) and eps_z voxels (camera plane)."""
    lib = _load()
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    nx, ny, nz = scene.shape
    tags = np.zeros((nz, ny, nx), dtype=np.uint32)
    amb = np.zeros((nz, ny, nx), dtype=np.uint32)
    lib.orc_visual_hull(ctypes.byref(scene.grid), scene.cams, scene.ncam, _ptr(mask), _ptr(tags), _ptr(amb),
                        float(eps), float(eps_z))
    return (tags, amb) if with_undecided else tags


def reconstruct(scene: Scene, vol, params: Params, targets, mask, bbox, iters,
                albedo=None, first_iteration=0, hull=None, stop_delta=None, with_undecided=False):
    """Algorithm 2 repeated `iters` times with the paper rule; with `hull`
    (visual-hull tags) the records outside the hull are held at 0; with
    stop_delta, stops once the image error changes by less than it (Sec. 3).
    Returns (volume, rmse per iteration run (rows x 3), (forward, adjust)
    samples[, the adjustments' undecided budget summed over the iterations])."""
    lib = _load()
    vol = _check_vol(vol, scene.shape, 4).copy()
    targets = _f64(targets)
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    bbox = np.ascontiguousarray(bbox, dtype=np.int32)
    rmse = np.zeros((iters, 3))
    samples = np.zeros(2, dtype=np.int64)
    alb = _f64(albedo) if albedo is not None else None
    hl = np.ascontiguousarray(hull, dtype=np.uint32) if hull is not None else None
    done = ctypes.c_int(0)
    nx, ny, nz = scene.shape
    und = np.zeros((nz, ny, nx)) if with_undecided else None
    lib.orc_reconstruct(ctypes.byref(scene.grid), _ptr(vol), _ptr(alb) if alb is not None else None,
                        scene.cams, scene.ncam, ctypes.byref(params), _ptr(targets), _ptr(mask),
                        _ptr(bbox), int(iters), int(first_iteration), _ptr(rmse), _ptr(samples),
                        _ptr(hl) if hl is not None else None,
                        float(stop_delta) if stop_delta is not None else -1.0, ctypes.byref(done),
                        _ptr(und) if und is not None else None)
    out = (vol, rmse[:done.value], (int(samples[0]), int(samples[1])))
    return out + (und,) if with_undecided else out


def scatter_L6(scene: Scene, vol):
    """The six directional radiances (nz,ny,nx,6,3), d = 2 axis + (0: +axis, 1: -axis)."""
    vol = _check_vol(vol, scene.shape, 4)
    nx, ny, nz = scene.shape
    out = np.zeros((nz, ny, nx, 6, 3))
    _load().orc_scatter_L6(ctypes.byref(scene.grid), _ptr(vol), _ptr(out))
    return out


def hg_weights(g, omega):
    w = np.zeros(6)
    _load().orc_hg_weights(float(g), _ptr(np.ascontiguousarray(omega, dtype=np.float64)), _ptr(w))
    return w


def scatter_source_hg(vol, albedo, L6, w):
    vol = _f64(vol)
    out = np.zeros_like(vol)
    _load().orc_scatter_source_hg(vol.size // 4, _ptr(vol), _ptr(_f64(albedo)), _ptr(_f64(L6)),
                                  _ptr(np.ascontiguousarray(w, dtype=np.float64)), _ptr(out))
    return out


def volume_dims(cams, box_min, box_max, alpha=1.5):
    """Sec. 4.2 volume dimensions: (dims, h, n per axis); ValueError when a box
    corner is behind a camera."""
    sc = Scene((2, 2, 2), (0.0, 0.0, 0.0), 1.0, cams)
    lo = np.ascontiguousarray(box_min, dtype=np.float64)
    ln = np.ascontiguousarray(np.asarray(box_max, dtype=np.float64) - lo)
    dims = np.zeros(3, dtype=np.int32)
    h = ctypes.c_double()
    n = np.zeros(3)
    if _load().orc_volume_dims(sc.cams, sc.ncam, _ptr(lo), _ptr(ln), float(alpha), _ptr(dims),
                               ctypes.byref(h), _ptr(n)) != 0:
        raise ValueError("a box corner is not in front of a camera")
    return tuple(int(x) for x in dims), h.value, tuple(n)


def volume_rmse(a, b, tags=None, full=None):
    """Volume data error (Sec. 5.1) of the emission channels over the key points
    whose tag equals `full` (all key points without tags).  Returns (rmse3, count)."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    if a.shape != b.shape or a.shape[-1] != 4:
        raise ValueError("volumes must share a (..., 4) shape")
    nodes = a.size // 4
    tg = np.ascontiguousarray(tags, dtype=np.uint32) if tags is not None else None
    if tg is not None and tg.size != nodes:
        raise ValueError("one tag per node")
    out = np.zeros(3)
    n = _load().orc_volume_rmse(nodes, _ptr(a), _ptr(b), _ptr(tg) if tg is not None else None,
                                int(full or 0), _ptr(out))
    return out, int(n)


def planck(lambda_m, temp_k):
    return _load().orc_planck(float(lambda_m), float(temp_k))


def temp_rgb(temp_k):
    out = np.zeros(3)
    _load().orc_temp_rgb(float(temp_k), _ptr(out))
    return out


def hg_phase(g, cos_wi):
    return _load().orc_hg_phase(float(g), float(cos_wi))


def g_draw(seed, g_std, iteration, view, pixel, k):
    return _load().orc_g_draw(int(seed), float(g_std), int(iteration), int(view), int(pixel), int(k))
