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


def oracle_targets(orc, case, albedo=None, noise=0.0, seed=11, thresh=30 / 255, P=None):
    """Targets rendered by the oracle from the case's ground truth (through its
    in-scattering source when albedo is given), normalised to max 1, plus
    seeded noise; and the oracle's preparation of them.  Returns
    (scene, raw images, prepared targets, mask, bbox)."""
    from paper_1809_06417_gb300 import synth
    sc = orc.Scene(case.shape, case.origin, case.h, case.cams)
    P = P if P is not None else orc.make_params(step=case.step)
    src = case.vol if albedo is None else orc.scatter_source(case.vol, albedo, orc.scatter_J(sc, case.vol))
    img, _ = orc.render(sc, src, P)
    img = img / img.max()
    if noise:
        img = synth.add_noise(img, noise, seed)
    t_ref, mask, bbox = orc.prepare_targets(img, thresh)
    return sc, img, t_ref, mask, bbox


def tags_on_device(torch, tags):
    """uint32 hull tags (nz, ny, nx) as the int32 CUDA tensor fr_params.hull_tags takes."""
    return torch.as_tensor(np.ascontiguousarray(tags, dtype=np.uint32).view(np.int32), device="cuda")


def oracle_lut(orc, torch, t_min, t_max, m):
    """The oracle's colour-temperature table rounded to float32, as the device
    table the library reads (m x 4, fourth column 0) and as the float64 table
    the oracle is given: both sides then interpolate the same values."""
    ref = orc.lut_build(t_min, t_max, m).astype(np.float32)
    dev = torch.zeros((m, 4), device="cuda")
    dev[:, :3] = torch.as_tensor(ref, device="cuda")
    return dev, ref.astype(np.float64)
