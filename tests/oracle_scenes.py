"""Small hand-built scenes for pinning the oracle (single rays, boxes)."""
import math

import numpy as np


def frame_from_dir(d):
    """Orthonormal (fwd, right, up) with fwd along d."""
    f = np.asarray(d, dtype=np.float64)
    f = f / np.linalg.norm(f)
    helper = np.array([0.0, 1.0, 0.0]) if abs(f[1]) < 0.9 else np.array([1.0, 0.0, 0.0])
    r = np.cross(f, helper)
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    return f, r, u


def one_pixel_camera(through, direction, back=50.0, width=1, height=1, fov_deg=1e-3):
    """A camera whose (single, central) pixel ray passes through `through`
    (world units) along `direction`."""
    f, r, u = frame_from_dir(direction)
    pos = np.asarray(through, dtype=np.float64) - back * f
    return dict(pos=pos.tolist(), right=r.tolist(), up=u.tolist(), fwd=f.tolist(),
                tan_half_fov=math.tan(math.radians(fov_deg) / 2), width=width, height=height)


def const_volume(shape, S, sigma):
    nx, ny, nz = shape
    vol = np.zeros((nz, ny, nx, 4))
    vol[..., :3] = np.asarray(S, dtype=np.float64)
    vol[..., 3] = sigma
    return vol


def affine_volume(shape, a, b, sigma=0.0):
    """RGB source a_c + b_c . (i, j, k) at node (i, j, k) (voxel coordinates)."""
    nx, ny, nz = shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    vol = np.zeros((nz, ny, nx, 4))
    for c in range(3):
        vol[..., c] = a[c] + b[c][0] * i + b[c][1] * j + b[c][2] * k
    vol[..., 3] = sigma
    return vol


def chord_through_centre(shape, d):
    """Length (voxel units) of the chord of the node box [0, n-1]^3 along the
    unit direction d through the box centre: it leaves through the first face
    reached, at t = half-width / |d_a|."""
    half = [(n - 1) / 2.0 for n in shape]
    d = np.asarray(d, dtype=np.float64) / np.linalg.norm(d)
    t = min(half[a] / abs(d[a]) for a in range(3) if d[a] != 0.0)
    return 2.0 * t
