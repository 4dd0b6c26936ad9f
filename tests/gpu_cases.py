"""Seeded cases shared by the GPU parity tests: the same inputs go to the
CUDA path (float32 tensors) and to the FP64 oracle (numpy)."""
import numpy as np

from paper_1809_06417_gb300 import synth


class Case:
    def __init__(self, shape, cams, vol, step, origin=None, h=None, albedo=None):
        self.shape = tuple(shape)            # (nx, ny, nz)
        nmax = max(shape)
        self.h = h if h is not None else 1.0 / (nmax - 1)
        self.origin = origin if origin is not None else tuple(-0.5 * (s - 1) * self.h for s in shape)
        self.cams = cams
        self.vol = vol                       # (nz, ny, nx, C) float64
        self.step = step
        self.albedo = albedo

    def vol32(self):
        return self.vol.astype(np.float32)


def tiny_case(seed=1, views=4, side=64, n=32, step=1.0, jitter=0.0):
    """The tiny configuration: 32^3 blobs, 4 ring cameras 64x64, step 1."""
    cams = synth.ring_cameras(views, side, side, elevation_jitter_deg=jitter, seed=seed)
    return Case((n, n, n), cams, synth.blobs_volume(n, seed), step)


def ragged_case(seed=7):
    """Non-cubic grid, image sizes that leave partial tiles, jittered cameras,
    a step that does not divide the chords."""
    shape = (21, 17, 26)
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape
    vol = np.zeros((nz, ny, nx, 4))
    blobs = synth.blobs_volume(26, seed, count=4, radius_range=(2.0, 5.0))
    vol[...] = blobs[:nz, :ny, :nx]
    vol[..., :3] += 0.02 * rng.random((nz, ny, nx, 3))
    cams = synth.ring_cameras(5, 37, 23, radius=2.0, elevation_jitter_deg=12.0, seed=seed, phase=0.3)
    return Case(shape, cams, vol, 0.7)


def plume_case(n=48, views=6, side=96, step=0.5, seed=2):
    vol, alb = synth.plume_volume(n, seed)
    cams = synth.ring_cameras(views, side, side, elevation_jitter_deg=8.0, seed=seed)
    return Case((n, n, n), cams, vol, step, albedo=alb)


def rel_err(gpu, ref):
    """Element-wise error relative to the largest reference magnitude."""
    scale = float(np.max(np.abs(ref)))
    return np.abs(np.asarray(gpu, dtype=np.float64) - ref) / (scale if scale > 0 else 1.0)
