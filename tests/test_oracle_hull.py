"""Pins for the oracle's visual hull (Sec. 4.3.1, Algorithm 1): the tags are a
superset of the exact "some flame ray crosses a cell of this key point" set
(brute-force ray-box tests), every tag is explained by a flame ray through a
slightly larger box, empty and full masks give no and all bits, and the hull
of a sphere seen from a ring of cameras lies between the sphere and its
polygonal bound."""
import math

import numpy as np
import pytest

from paper_1809_06417_gb300 import synth


def _rays(cam, origin, h):
    """All pixel rays of a camera in voxel coordinates (double precision)."""
    W, H, t = cam["width"], cam["height"], cam["tan_half_fov"]
    f, r, u = (np.asarray(cam[k]) for k in ("fwd", "right", "up"))
    px, py = np.meshgrid(np.arange(W), np.arange(H))
    a = (2 * (px + 0.5) / W - 1) * t * W / H
    b = (1 - 2 * (py + 0.5) / H) * t
    d = f[None, None] + a[..., None] * r + b[..., None] * u
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    o = (np.asarray(cam["pos"]) - np.asarray(origin)) / h
    return o, d


def _hits_box(o, d, lo, hi):
    with np.errstate(divide="ignore", invalid="ignore"):
        t0 = (lo - o) / d
        t1 = (hi - o) / d
    tmin = np.nanmax(np.minimum(t0, t1), axis=-1)
    tmax = np.nanmin(np.maximum(t0, t1), axis=-1)
    return tmax >= np.maximum(tmin, 0.0)


def _exact_tags(shape, origin, h, cams, mask, grow=0.0):
    nx, ny, nz = shape
    tags = np.zeros((nz, ny, nx), dtype=np.uint32)
    for v, cam in enumerate(cams):
        o, d = _rays(cam, origin, h)
        dv = d[mask[v].astype(bool)]
        if len(dv) == 0:
            continue
        for k in range(nz):
            for j in range(ny):
                for i in range(nx):
                    lo = np.maximum(np.array([i, j, k]) - 1.0 - grow, 0.0)
                    hi = np.minimum(np.array([i, j, k]) + 1.0 + grow, np.array(shape) - 1.0)
                    if np.any(_hits_box(o, dv, lo, hi)):
                        tags[k, j, i] |= np.uint32(1 << v)
    return tags


def _case(rng, n=7, views=3, side=(13, 11)):
    shape, origin, h = synth.unit_grid(n)
    cams = synth.ring_cameras(views, side[0], side[1], elevation_jitter_deg=15, seed=int(rng.integers(1 << 30)))
    mask = (rng.random((views, side[1], side[0])) < 0.15).astype(np.uint8)
    return shape, origin, h, cams, mask


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tags_cover_every_flame_ray_and_nothing_far(orc, seed):
    rng = np.random.default_rng(seed)
    shape, origin, h, cams, mask = _case(rng)
    tags = orc.visual_hull(orc.Scene(shape, origin, h, cams), mask)
    exact = _exact_tags(shape, origin, h, cams, mask)
    assert np.all((tags & exact) == exact)               # conservative
    loose = _exact_tags(shape, origin, h, cams, mask, grow=1.5)
    assert np.all((tags & ~loose) == 0)                   # but not far off


def test_empty_and_full_masks(orc):
    shape, origin, h = synth.unit_grid(6)
    cams = synth.ring_cameras(3, 10, 10)
    mask = np.zeros((3, 10, 10), dtype=np.uint8)
    mask[1] = 1
    tags = orc.visual_hull(orc.Scene(shape, origin, h, cams), mask)
    assert np.all(tags == 2)


def test_sphere_hull_from_a_ring(orc):
    n, views, side = 24, 8, 48
    shape, origin, h = synth.unit_grid(n)
    cams = synth.ring_cameras(views, side, side)
    R = 0.25  # world units, centred at the origin
    mask = np.zeros((views, side, side), dtype=np.uint8)
    for v, cam in enumerate(cams):
        o, d = _rays(cam, origin, h)
        oc = o - np.asarray([(n - 1) / 2.0] * 3)        # centre in voxel units
        b = np.sum(d * oc, axis=-1)
        c = np.sum(oc * oc) - (R / h) ** 2
        mask[v] = (b * b - c > 0)
    tags = orc.visual_hull(orc.Scene(shape, origin, h, cams), mask)
    inside = tags == (1 << views) - 1
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    dist = np.sqrt((i - (n - 1) / 2) ** 2 + (j - (n - 1) / 2) ** 2 + (k - (n - 1) / 2) ** 2) * h
    assert np.all(inside[dist < R])
    # outside the sphere's polygonal hull (8 views: radius / cos(pi/8)) plus
    # the cells' reach and a perspective margin, nothing is inside
    assert not np.any(inside[dist > R / math.cos(math.pi / 8) + 3 * h])


def _recon_case(orc, n=12, views=4, side=24):
    from paper_1809_06417_gb300 import synth as sy
    shape, origin, h = sy.unit_grid(n)
    cams = sy.ring_cameras(views, side, side, elevation_jitter_deg=10.0, seed=3)
    vol = sy.blobs_volume(n, 3, radius_range=(1.5, 2.5))
    sc = orc.Scene(shape, origin, h, cams)
    P = orc.make_params(step=0.5, alpha_l=5e-3)
    img, _ = orc.render(sc, vol, P)
    img /= img.max()
    targets, mask, bbox = orc.prepare_targets(img, 30 / 255)
    v0 = vol.copy()
    v0[..., :3] = 0.02
    return sc, P, v0, targets, mask, bbox, views


def test_reconstruct_with_full_hull_is_plain_reconstruct(orc):
    """Every key point inside the hull: the hull changes nothing."""
    sc, P, v0, targets, mask, bbox, views = _recon_case(orc)
    full = np.full(v0.shape[:3], (1 << views) - 1, dtype=np.uint32)
    a, ra, _ = orc.reconstruct(sc, v0, P, targets, mask, bbox, 3)
    b, rb, _ = orc.reconstruct(sc, v0, P, targets, mask, bbox, 3, hull=full)
    assert np.array_equal(a, b) and np.array_equal(ra, rb)


def test_reconstruct_with_hull_keeps_outside_empty(orc):
    """Key points outside the hull hold no flame (Sec. 4.3.1): their records are
    0 after every iteration, the extinction inside is untouched, and an empty
    hull leaves an empty volume whose error is the targets' own RMS."""
    sc, P, v0, targets, mask, bbox, views = _recon_case(orc)
    hull = orc.visual_hull(sc, mask)
    inside = hull == (1 << views) - 1
    assert 0 < inside.sum() < inside.size
    got, rmse, _ = orc.reconstruct(sc, v0, P, targets, mask, bbox, 3, hull=hull)
    assert np.all(got[~inside] == 0.0)
    assert np.array_equal(got[inside][:, 3], v0[inside][:, 3])
    assert np.any(got[inside][:, :3] != v0[inside][:, :3])
    none = np.zeros(v0.shape[:3], dtype=np.uint32)
    got0, rmse0, _ = orc.reconstruct(sc, v0, P, targets, mask, bbox, 2, hull=none)
    assert np.all(got0 == 0.0)
    # nothing rendered: the error of each view is the targets' RMS in its box
    sq = np.zeros(3)
    cnt = 0
    for v in range(views):
        x0, y0, x1, y1 = bbox[v]
        if x1 >= x0 and y1 >= y0:
            t = targets[v, y0:y1 + 1, x0:x1 + 1]
            sq += (t ** 2).sum(axis=(0, 1))
            cnt += t.shape[0] * t.shape[1]
    np.testing.assert_allclose(rmse0[0], 255.0 * np.sqrt(sq / cnt), rtol=1e-12)


def test_stop_criterion(orc):
    """Sec. 3 stop criterion: the loop ends after the first iteration whose
    image error differs from the previous one's by less than stop_delta in
    every channel; an infinite threshold stops after two iterations, a zero
    threshold never stops early, and a stopped run is a prefix of the full run."""
    sc, P, v0, targets, mask, bbox, views = _recon_case(orc)
    full, r_full, _ = orc.reconstruct(sc, v0, P, targets, mask, bbox, 8)
    assert r_full.shape == (8, 3)
    _, r_inf, _ = orc.reconstruct(sc, v0, P, targets, mask, bbox, 8, stop_delta=1e30)
    assert r_inf.shape == (2, 3) and np.array_equal(r_inf, r_full[:2])
    _, r_zero, _ = orc.reconstruct(sc, v0, P, targets, mask, bbox, 8, stop_delta=0.0)
    assert np.array_equal(r_zero, r_full)
    step = np.abs(np.diff(r_full, axis=0)).max(axis=1)   # largest channel change per iteration
    assert np.all(np.diff(step) < 0)                      # shrinking steps on this case
    delta = 0.5 * (step[2] + step[3])                     # first met at iteration 4 (index 3 + 1)
    vol, r_mid, _ = orc.reconstruct(sc, v0, P, targets, mask, bbox, 8, stop_delta=delta)
    assert r_mid.shape == (5, 3) and np.array_equal(r_mid, r_full[:5])
    part, _, _ = orc.reconstruct(sc, v0, P, targets, mask, bbox, 5)
    assert np.array_equal(vol, part)


def test_volume_rmse_in_hull(orc):
    """Volume data error (Sec. 5.1) inside the hull: zero for equal volumes, |c|
    for a constant offset c of one channel, blind to any difference outside
    the hull, and taken over every key point without tags."""
    rng = np.random.default_rng(4)
    a = rng.random((6, 7, 5, 4))
    tags = rng.integers(0, 8, size=(6, 7, 5)).astype(np.uint32)
    full = 7
    inside = tags == full
    r, n = orc.volume_rmse(a, a, tags, full)
    assert n == inside.sum() and np.all(r == 0.0)
    b = a.copy()
    b[..., 1] += 0.25
    b[~inside] += rng.normal(size=(np.count_nonzero(~inside), 4)) * 100.0
    r, n = orc.volume_rmse(a, b, tags, full)
    assert np.allclose(r, [0.0, 0.25, 0.0], atol=1e-15)
    b[..., 3] += 5.0                                     # extinction is not compared
    r2, _ = orc.volume_rmse(a, b, tags, full)
    assert np.array_equal(r, r2)
    r3, n3 = orc.volume_rmse(a, a + 0.5, None)
    assert n3 == a.size // 4 and np.allclose(r3, 0.5, atol=1e-15)
    r4, n4 = orc.volume_rmse(a, b, np.zeros_like(tags), full)
    assert n4 == 0 and np.all(r4 == 0.0)
