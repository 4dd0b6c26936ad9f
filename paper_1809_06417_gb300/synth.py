"""Seeded synthetic inputs: flame-like volumes, camera rings and target noise.

This module holds input recipes only (no rendering, no update rule): both the
GPU path and the CPU oracle consume what it produces.  The paper's own inputs
(a physically simulated fire and captured videos, Sec. 5.1) are not available;
these seeded volumes stand in for them and reuse the paper's camera geometry
(cameras on a ring looking at the volume centre, 60 degree field of view,
Sec. 5.1).

Volumes are numpy arrays shaped (nz, ny, nx, C) with x fastest; grids are
node-centred with spacing h = 1 / (n - 1), i.e. the node box is the unit cube
centred at the origin.  Lengths inside the method are in voxel edge lengths, so
extinction values are per voxel length.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Extinction per voxel length equivalent to the paper's constant sample
# opacity tau = 0.05 at a one-voxel step (Sec. 5.1): -ln(1 - 0.05).
SIGMA_PAPER = -math.log(1.0 - 0.05)


@dataclass
class Scene:
    """Node grid and cameras in world units."""
    shape: tuple          # (nx, ny, nz)
    origin: tuple         # world position of node (0, 0, 0)
    h: float              # node spacing
    cams: list = field(default_factory=list)  # dicts: pos, right, up, fwd, tan_half_fov, width, height


def unit_grid(n: int):
    """Node-centred n^3 grid spanning [-0.5, 0.5]^3."""
    h = 1.0 / (n - 1)
    return (n, n, n), (-0.5, -0.5, -0.5), h


def look_at(pos, target=(0.0, 0.0, 0.0), world_up=(0.0, 1.0, 0.0)):
    pos = np.asarray(pos, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - pos
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(world_up, dtype=np.float64))
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    return f, r, u


def ring_cameras(k: int, width: int, height: int, radius: float = 2.0, fov_deg: float = 60.0,
                 elevation_jitter_deg: float = 0.0, seed: int = 0, phase: float = 0.0):
    """k pinhole cameras evenly spaced on a horizontal ring around the origin.

    With elevation_jitter_deg > 0 each camera is raised or lowered by a seeded
    uniform angle in [-jitter, jitter] (the paper's simulated cameras look
    slightly up or down, Sec. 5.1)."""
    rng = np.random.default_rng(seed)
    cams = []
    for i in range(k):
        th = phase + 2.0 * math.pi * i / k
        el = math.radians(rng.uniform(-elevation_jitter_deg, elevation_jitter_deg)) if elevation_jitter_deg else 0.0
        pos = radius * np.array([math.cos(el) * math.cos(th), math.sin(el), math.cos(el) * math.sin(th)])
        f, r, u = look_at(pos)
        cams.append(dict(pos=pos.tolist(), right=r.tolist(), up=u.tolist(), fwd=f.tolist(),
                         tan_half_fov=math.tan(math.radians(fov_deg) / 2.0), width=int(width), height=int(height)))
    return cams


def _node_coords(n: int):
    """Voxel coordinates of the nodes, broadcastable as (z, y, x)."""
    a = np.arange(n, dtype=np.float64)
    return a[:, None, None], a[None, :, None], a[None, None, :]


# Profiles are cut to zero below this fraction of their peak, so a flame has
# compact support (empty space around it holds exact zeros).
SUPPORT_CUT = 1e-3


def _gauss(z, y, x, c, s):
    g = np.exp(-((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) / (2.0 * s * s))
    return np.where(g < SUPPORT_CUT, 0.0, g)


def value_noise(n: int, rng: np.random.Generator, octaves: int = 4, base_cells: int = 4):
    """Lattice value noise on an n^3 node grid, smoothstep-interpolated; each
    octave doubles the frequency and halves the amplitude.  Range [0, 1]."""
    out = np.zeros((n, n, n))
    amp_total = 0.0
    t = np.linspace(0.0, 1.0, n)
    for o in range(octaves):
        cells = base_cells * (2 ** o)
        amp = 0.5 ** o
        lat = rng.random((cells + 1, cells + 1, cells + 1))
        u = t * cells
        i0 = np.minimum(np.floor(u).astype(np.int64), cells - 1)
        f = u - i0
        s = f * f * (3.0 - 2.0 * f)
        # separable smoothstep blend along z, y, x
        v = lat[i0][:, :, :] * (1 - s)[:, None, None] + lat[i0 + 1] * s[:, None, None]
        v = v[:, i0, :] * (1 - s)[None, :, None] + v[:, i0 + 1, :] * s[None, :, None]
        v = v[:, :, i0] * (1 - s)[None, None, :] + v[:, :, i0 + 1] * s[None, None, :]
        out += amp * v
        amp_total += amp
    return out / amp_total


def blobs_volume(n: int, seed: int, count: int = 3, sigma_peak: float = 0.5,
                 radius_range=(2.0, 6.0), colour=(1.0, 0.55, 0.15)):
    """Tiny-case volume: Gaussian blobs with centres uniform in the inner 60%
    of the box and radii uniform in radius_range voxels.  Returns records
    (n,n,n,4) {q_r, q_g, q_b, sigma}, sigma peaking at sigma_peak."""
    rng = np.random.default_rng(seed)
    z, y, x = _node_coords(n)
    prof = np.zeros((n, n, n))
    emis = np.zeros((n, n, n))
    lo, hi = 0.2 * (n - 1), 0.8 * (n - 1)
    for _ in range(count):
        c = rng.uniform(lo, hi, size=3)
        s = rng.uniform(*radius_range)
        g = _gauss(z, y, x, c, s)
        prof += g
        emis += rng.uniform(0.5, 1.0) * g
    vol = np.zeros((n, n, n, 4))
    vol[..., 3] = sigma_peak * np.minimum(prof, 1.0)
    for ch in range(3):
        vol[..., ch] = colour[ch] * emis
    return vol


def plume_profile(n: int, rng: np.random.Generator, count: int = 8, shift_y: float = 0.0):
    """Rising plume: `count` Gaussian blobs stacked along +y whose radii shrink
    upward, with a little seeded lateral wander."""
    z, y, x = _node_coords(n)
    prof = np.zeros((n, n, n))
    cx = cz = 0.5 * (n - 1)
    for b in range(count):
        frac = b / max(count - 1, 1)
        cy = (0.18 + 0.62 * frac) * (n - 1) + shift_y
        r = (0.13 - 0.08 * frac) * (n - 1)
        wx, wz = rng.normal(0.0, 0.02 * (n - 1), size=2)
        prof = np.maximum(prof, _gauss(z, y, x, (cx + wx, cy, cz + wz), r))
    return prof


def plume_volume(n: int, seed: int, sigma_peak: float = SIGMA_PAPER, albedo_max: float = 0.3,
                 colour=(1.0, 0.55, 0.15), shift_y: float = 0.0):
    """Full-RTE case: plume of 8 blobs modulated by 4-octave value noise.
    Returns (records (n,n,n,4) {q_r,q_g,q_b,sigma}, albedo (n,n,n) in [0, albedo_max])."""
    rng = np.random.default_rng(seed)
    prof = plume_profile(n, rng, shift_y=shift_y)
    noise = value_noise(n, rng)
    dens = prof * (0.6 + 0.4 * noise)
    heat = np.clip(dens * (1.0 + 0.5 * (noise - 0.5)), 0.0, None)
    vol = np.zeros((n, n, n, 4))
    vol[..., 3] = sigma_peak * dens / max(dens.max(), 1e-30)
    for ch in range(3):
        vol[..., ch] = colour[ch] * heat
    albedo = albedo_max * value_noise(n, rng)
    return vol, albedo


def temperature_volume(n: int, seed: int, t_min: float = 800.0, t_max: float = 2000.0,
                       sigma: float = SIGMA_PAPER):
    """Temperature case: T = t_min + (t_max - t_min) * clamp(core * (1 + 0.3 noise), 0, 1)
    with a Gaussian plume core; constant extinction.  Returns (n,n,n,2) {T, sigma}."""
    rng = np.random.default_rng(seed)
    z, y, x = _node_coords(n)
    c = 0.5 * (n - 1)
    core = np.exp(-((x - c) ** 2 + (z - c) ** 2) / (2 * (0.16 * (n - 1)) ** 2)
                  - (y - 0.4 * (n - 1)) ** 2 / (2 * (0.3 * (n - 1)) ** 2))
    noise = value_noise(n, rng) - 0.5
    t = t_min + (t_max - t_min) * np.clip(core * (1.0 + 0.3 * 2.0 * noise), 0.0, 1.0)
    vol = np.zeros((n, n, n, 2))
    vol[..., 0] = t
    vol[..., 1] = sigma
    return vol


def video_frames(frames: int, n: int, seed: int, sigma_peak: float = SIGMA_PAPER,
                 colour=(1.0, 0.55, 0.15)):
    """Batched video case: one plume advected +1 voxel in y per frame (its blobs
    and its noise texture move together) plus a per-frame noise factor.
    Returns a list of (n,n,n,4) records {q_r, q_g, q_b, sigma}."""
    rng = np.random.default_rng(seed)
    base_noise = value_noise(n, rng)
    out = []
    for f in range(frames):
        frng = np.random.default_rng(seed * 100003 + f)
        prof = plume_profile(n, np.random.default_rng(seed), shift_y=float(f) - 0.25 * frames)
        noise = np.roll(base_noise, f, axis=1)
        flicker = 1.0 + 0.1 * (value_noise(n, frng, octaves=1, base_cells=3) - 0.5)
        dens = prof * (0.6 + 0.4 * noise) * flicker
        vol = np.zeros((n, n, n, 4))
        vol[..., 3] = sigma_peak * dens / max(dens.max(), 1e-30)
        heat = np.clip(dens * (1.0 + 0.5 * (noise - 0.5)), 0.0, None)
        for ch in range(3):
            vol[..., ch] = colour[ch] * heat
        out.append(vol)
    return out


def add_noise(images: np.ndarray, std: float, seed: int) -> np.ndarray:
    """Seeded Gaussian pixel noise (the targets of the tiny case carry std 1e-3)."""
    rng = np.random.default_rng(seed)
    return images + rng.normal(0.0, std, size=images.shape)


def random_interior_points(n_nodes_shape, count: int, seed: int, margin: int = 1):
    rng = np.random.default_rng(seed)
    nx, ny, nz = n_nodes_shape
    return np.stack([rng.integers(margin, s - margin, size=count) for s in (nz, ny, nx)], axis=1)


# ---------------------------------------------------------------------------
# Workload configurations (sizes and seeds of the five benchmark settings)
# ---------------------------------------------------------------------------

CONFIGS = {
    # plain method, tiny: 32^3 fp32, 3 blobs, 4 views 64x64, step 1, 10 iterations
    "tiny": dict(n=32, views=4, side=64, step=1.0, iters=10, seed=1, noise=1e-3),
    # plain method, full RTE: 128^3, plume + albedo, 8 views 512x512, step 0.5, 50 iterations
    "full_rte": dict(n=128, views=8, side=512, step=0.5, iters=50, seed=2, noise=0.0),
    # temperature, differentiable: 128^3 T in [800, 2000] K, 8 views 512x512
    "temperature": dict(n=128, views=8, side=512, step=0.5, seed=3),
    # video: 64 frames of 96^3, 8 views 384x384, 20 iterations per frame
    "video": dict(n=96, frames=64, views=8, side=384, step=0.5, iters=20, seed=4),
    # serving: Poisson 20 jobs/s, grids {64,96,128,192}^3, 4-12 views, side 256-768, 20-50 iterations
    "serving": dict(rate=20.0, grids=(64, 96, 128, 192), views=(4, 12), side=(256, 768),
                    iters=(20, 50), seed=5),
}


def serving_stream(count: int, seed: int = 5, rate: float = 20.0, grids=(64, 96, 128, 192),
                   views=(4, 12), side=(256, 768), iters=(20, 50)):
    """Seeded Poisson arrivals of reconstruction jobs with mixed sizes."""
    rng = np.random.default_rng(seed)
    t = 0.0
    jobs = []
    for i in range(count):
        t += rng.exponential(1.0 / rate)
        jobs.append(dict(id=i, arrival=t, n=int(rng.choice(grids)),
                         views=int(rng.integers(views[0], views[1] + 1)),
                         side=int(rng.integers(side[0] // 32, side[1] // 32 + 1) * 32),
                         iters=int(rng.integers(iters[0], iters[1] + 1)),
                         seed=int(rng.integers(0, 2 ** 31))))
    return jobs
