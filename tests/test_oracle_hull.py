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


def _lattice_uv(shape, origin, h, c, dt):
    """Pixel coordinates (u, v) of every lattice point (z, y, x) in camera c,
    in float64, or in float32 with one rounding per operation in the order a
    float32 kernel takes."""
    nx, ny, nz = shape
    W, H = c["width"], c["height"]
    if dt == np.float32:
        f = np.float32
        o = [(f(c["pos"][a]) - f(origin[a])) * (f(1.0) / f(h)) for a in range(3)]
        X = [np.arange(n, dtype=f) - o[a] for a, n in enumerate((nx, ny, nz))]
        Xk, Xj, Xi = np.meshgrid(X[2], X[1], X[0], indexing="ij")

        def dot(r):
            return (Xi * f(r[0]) + Xj * f(r[1])) + Xk * f(r[2])
        xc, yc, zc = dot(c["right"]), dot(c["up"]), dot(c["fwd"])
        ty = f(c["tan_half_fov"])
        tx = ty * f(W) / f(H)
        u = ((xc / zc) / tx + f(1.0)) * (f(0.5) * f(W)) - f(0.5)
        w = (f(1.0) - (yc / zc) / ty) * (f(0.5) * f(H)) - f(0.5)
    else:
        K, J, I = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        o = (np.asarray(c["pos"]) - np.asarray(origin)) / h
        P = np.stack([I - o[0], J - o[1], K - o[2]], axis=-1)
        xc, yc, zc = P @ np.asarray(c["right"]), P @ np.asarray(c["up"]), P @ np.asarray(c["fwd"])
        ty = c["tan_half_fov"]
        tx = ty * W / H
        u = (xc / zc / tx + 1.0) * 0.5 * W - 0.5
        w = (1.0 - yc / zc / ty) * 0.5 * H - 0.5
    assert np.all(zc > 0)
    return u.astype(np.float64), w.astype(np.float64)


def _numpy_hull(shape, origin, h, cams, mask, dt):
    """The hull rule evaluated independently, vectorised over nodes: every
    lattice point projected once (_lattice_uv), each node's rectangle the
    extremes over its box's eight corners, flame pixels counted with a
    summed-area table.  Returns (tags, u and v of every lattice point)."""
    nx, ny, nz = shape
    tags = np.zeros((nz, ny, nx), dtype=np.uint32)
    K, J, I = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    lo = [np.maximum(a - 1, 0) for a in (I, J, K)]
    hi = [np.minimum(a + 1, n - 1) for a, n in zip((I, J, K), (nx, ny, nz))]
    uvs = []
    for v, c in enumerate(cams):
        W, H = c["width"], c["height"]
        u, w = _lattice_uv(shape, origin, h, c, dt)
        uvs.append((u, w))
        corners = [(ci, cj, ck) for ck in (lo[2], hi[2]) for cj in (lo[1], hi[1]) for ci in (lo[0], hi[0])]
        us = np.stack([u[ck, cj, ci] for ci, cj, ck in corners])
        ws = np.stack([w[ck, cj, ci] for ci, cj, ck in corners])
        x0 = np.clip(np.ceil(us.min(0)), 0, W).astype(np.int64)
        x1 = np.clip(np.floor(us.max(0)), -1, W - 1).astype(np.int64)
        y0 = np.clip(np.ceil(ws.min(0)), 0, H).astype(np.int64)
        y1 = np.clip(np.floor(ws.max(0)), -1, H - 1).astype(np.int64)
        sat = np.zeros((H + 1, W + 1), dtype=np.int64)
        sat[1:, 1:] = np.cumsum(np.cumsum(mask[v].astype(np.int64), axis=0), axis=1)
        ok = (x0 <= x1) & (y0 <= y1)
        cnt = (sat[np.where(ok, y1 + 1, 0), np.where(ok, x1 + 1, 0)] - sat[np.where(ok, y0, 0), np.where(ok, x1 + 1, 0)]
               - sat[np.where(ok, y1 + 1, 0), np.where(ok, x0, 0)] + sat[np.where(ok, y0, 0), np.where(ok, x0, 0)])
        tags |= np.where(ok & (cnt > 0), np.uint32(1 << v), np.uint32(0))
    return tags, uvs


@pytest.mark.parametrize("n,views,side,seed", [(7, 3, 13, 0), (16, 5, 41, 1), (24, 8, 64, 2)])
def test_undecided_bits_cover_every_precision_dependent_decision(orc, n, views, side, seed):
    """An independent evaluation of the rule agrees with the oracle on every
    decided bit, in float64 and in float32 alike; the undecided bits (edge
    within HULL_EPS of a flame pixel centre) are few; and the float32
    projection's error is far inside the margin."""
    rng = np.random.default_rng(seed)
    shape, origin, h = synth.unit_grid(n)
    cams = synth.ring_cameras(views, side, side - 2, elevation_jitter_deg=15, seed=seed)
    mask = (rng.random((views, side - 2, side)) < 0.3).astype(np.uint8)
    tags, und = orc.visual_hull(orc.Scene(shape, origin, h, cams), mask, with_undecided=True)
    t64, uv64 = _numpy_hull(shape, origin, h, cams, mask, np.float64)
    t32, uv32 = _numpy_hull(shape, origin, h, cams, mask, np.float32)
    assert not np.any((t64 ^ tags) & ~und)
    assert not np.any((t32 ^ tags) & ~und)
    assert np.count_nonzero(und) < 0.1 * und.size
    err = max(np.abs(a - b).max() for p, q in zip(uv32, uv64) for a, b in zip(p, q))
    assert err < orc.HULL_EPS / 4, err


def test_float32_projection_error_at_the_benchmark_sizes(orc):
    """The margin holds at the sizes the GPU tests and the benchmark use: the
    float32 projection of every lattice point stays within a quarter of
    HULL_EPS of the float64 one (128^3 with 8 views of 512^2; 192^3 with 12
    views of 768^2, the largest serving job)."""
    for n, views, side, seed in ((128, 8, 512, 2), (192, 12, 768, 5)):
        shape, origin, h = synth.unit_grid(n)
        cams = synth.ring_cameras(views, side, side, elevation_jitter_deg=10.0, seed=seed)
        err = 0.0
        for c in cams[:2]:
            u64, w64 = _lattice_uv(shape, origin, h, c, np.float64)
            u32, w32 = _lattice_uv(shape, origin, h, c, np.float32)
            err = max(err, np.abs(u32 - u64).max(), np.abs(w32 - w64).max())
        print(f"{n}^3, {side}^2: float32 projection error {err:.2e} pixel")
        assert err < orc.HULL_EPS / 4
