"""Pins for the oracle's volume adjustment (Sec. 3.3.2, Eqs. 10-12), the
pre-processing threshold (Sec. 4.1) and the error measure (Sec. 5.1).

The single-cell cases are worked by hand: a 2x2x2-node grid (one cell) and a
ray along +x.  Their expected values follow from the geometry alone."""
import math

import numpy as np
import pytest

from oracle_scenes import const_volume, one_pixel_camera


def _one_cell_scene(orc, h=1.0, y=0.25, z=0.5):
    cam = one_pixel_camera((0.5 * h, y * h, z * h), (1.0, 0.0, 0.0), back=5.0 * h)
    return orc.Scene((2, 2, 2), (0.0, 0.0, 0.0), h, [cam])


def _update(orc, sc, vol, P, dL, iteration=0, mask=None):
    k = sc.ncam
    res = np.zeros((k, sc.height, sc.width, 3))
    res[...] = dL
    if mask is None:
        mask = np.ones((k, sc.height, sc.width), dtype=np.uint8)
    return orc.update_paper(sc, vol, P, res, mask, iteration)


def test_distance_free_counts_samples(orc):
    """alpha_d = 0, no extinction: every key point of the cell gains
    alpha_l * dL once per sample (G = 1, T = 1)."""
    sc = _one_cell_scene(orc)
    P = orc.make_params(step=0.25, alpha_l=0.5, alpha_d=0.0)
    dL = np.array([0.2, -0.4, 1.0])
    dV, n = _update(orc, sc, const_volume((2, 2, 2), (0, 0, 0), 0.0), P, dL)
    assert n == 4
    np.testing.assert_allclose(dV, np.broadcast_to(0.5 * dL * 4, dV.shape), rtol=1e-14)


def test_constant_tau_weights_are_geometric(orc):
    """Constant-tau mode: sample k (1-based) carries T = (1 - tau)^(k-1)
    (Eq. 12), so with alpha_d = 0 each key point gains
    alpha_l dL (1 - (1 - tau)^n) / tau."""
    sc = _one_cell_scene(orc)
    tau, n = 0.05, 4
    P = orc.make_params(step=0.25, alpha_l=1.0, alpha_d=0.0, tau=tau)
    dV, _ = _update(orc, sc, const_volume((2, 2, 2), (0, 0, 0), 0.0), P, 1.0)
    np.testing.assert_allclose(dV, (1.0 - (1.0 - tau) ** n) / tau, rtol=1e-14)


def test_field_mode_transmittance_is_in_front_of_sample(orc):
    """Two samples of length 0.5 in constant extinction s: the first sees
    T = 1 and the second T = exp(-0.5 s)."""
    sc = _one_cell_scene(orc)
    s = 0.8
    P = orc.make_params(step=0.5, alpha_l=1.0, alpha_d=0.0)
    dV, _ = _update(orc, sc, const_volume((2, 2, 2), (0, 0, 0), s), P, 1.0)
    np.testing.assert_allclose(dV, 1.0 + math.exp(-0.5 * s), rtol=1e-14)


def test_single_sample_distance_weights_in_voxel_units(orc):
    """One segment (step longer than the chord) samples the cell at
    (0.5, 0.25, 0.5) voxels.  Its distance to the four key points with j = 0 is
    sqrt(0.25 + 0.0625 + 0.25) = 0.75 and to the four with j = 1 is
    sqrt(0.25 + 0.5625 + 0.25) = sqrt(1.0625), whatever the world spacing h."""
    for h in (1.0, 0.1):
        sc = _one_cell_scene(orc, h=h)
        P = orc.make_params(step=10.0, alpha_l=0.001, alpha_d=1.0)
        dL = np.array([30.0, 10.0, 5.0])
        dV, n = _update(orc, sc, const_volume((2, 2, 2), (0, 0, 0), 0.0), P, dL)
        assert n == 1
        near, far = math.exp(-0.75), math.exp(-math.sqrt(1.0625))
        np.testing.assert_allclose(dV[:, 0, :, :], np.broadcast_to(0.001 * dL * near, (2, 2, 3)), rtol=1e-13)
        np.testing.assert_allclose(dV[:, 1, :, :], np.broadcast_to(0.001 * dL * far, (2, 2, 3)), rtol=1e-13)


def test_alpha_d_scales_the_distance(orc):
    sc = _one_cell_scene(orc)
    P = orc.make_params(step=10.0, alpha_l=1.0, alpha_d=2.5)
    dV, _ = _update(orc, sc, const_volume((2, 2, 2), (0, 0, 0), 0.0), P, 1.0)
    np.testing.assert_allclose(dV[0, 0, 0], math.exp(-2.5 * 0.75), rtol=1e-13)
    np.testing.assert_allclose(dV[0, 1, 0], math.exp(-2.5 * math.sqrt(1.0625)), rtol=1e-13)


def test_line_of_cells_counts(orc):
    """A ray along x at y = z = 0.5 through an n x 2 x 2 grid, step 0.5: each
    cell holds two samples and each interior key point belongs to two cells."""
    n = 6
    cam = one_pixel_camera(((n - 1) / 2.0, 0.5, 0.5), (1.0, 0.0, 0.0), back=20.0)
    sc = orc.Scene((n, 2, 2), (0.0, 0.0, 0.0), 1.0, [cam])
    P = orc.make_params(step=0.5, alpha_l=1.0, alpha_d=0.0)
    dV, cnt = _update(orc, sc, const_volume((n, 2, 2), (0, 0, 0), 0.0), P, 1.0)
    assert cnt == 2 * (n - 1)
    expect = np.full(n, 4.0)
    expect[0] = expect[-1] = 2.0
    for j in range(2):
        for k in range(2):
            np.testing.assert_allclose(dV[k, j, :, 0], expect, rtol=1e-14)


def test_views_accumulate_and_mask_gates(orc):
    """All views add into one adjustment (simultaneous update); non-flame
    pixels adjust nothing (Algorithm 2 adjusts flame rays only)."""
    cam = one_pixel_camera((0.5, 0.25, 0.5), (1.0, 0.0, 0.0), back=5.0)
    sc1 = orc.Scene((2, 2, 2), (0.0, 0.0, 0.0), 1.0, [cam])
    sc2 = orc.Scene((2, 2, 2), (0.0, 0.0, 0.0), 1.0, [cam, cam])
    P = orc.make_params(step=0.3, alpha_l=1.0)
    vol = const_volume((2, 2, 2), (0, 0, 0), 0.2)
    d1, _ = _update(orc, sc1, vol, P, 0.7)
    d2, _ = _update(orc, sc2, vol, P, 0.7)
    np.testing.assert_allclose(d2, 2.0 * d1, rtol=1e-14)
    d3, n3 = _update(orc, sc2, vol, P, 0.7, mask=np.array([[[1]], [[0]]], dtype=np.uint8))
    np.testing.assert_allclose(d3, d1, rtol=1e-14)


def test_gaussian_factor_statistics(orc):
    """G(s) has mean 1 and the requested spread (Eq. 11); 68.3% of draws fall
    within one standard deviation; g_std = 0 gives exactly 1."""
    draws = np.array([orc.g_draw(123, 0.1, it, v, p, k)
                      for it in range(2) for v in range(3) for p in range(40) for k in range(200)])
    n = len(draws)
    assert abs(draws.mean() - 1.0) < 4 * 0.1 / math.sqrt(n)
    assert abs(draws.std() - 0.1) < 0.004
    assert abs(np.mean(np.abs(draws - 1.0) < 0.1) - 0.6827) < 0.01
    assert orc.g_draw(123, 0.0, 1, 2, 3, 4) == 1.0
    # distinct counters give distinct draws; the same counter repeats
    assert orc.g_draw(5, 0.1, 0, 0, 0, 0) != orc.g_draw(5, 0.1, 0, 0, 0, 1)
    assert orc.g_draw(5, 0.1, 3, 1, 7, 9) == orc.g_draw(5, 0.1, 3, 1, 7, 9)


def test_gaussian_factor_multiplies_each_sample(orc):
    """With one sample the update scales by exactly that sample's G."""
    sc = _one_cell_scene(orc)
    P0 = orc.make_params(step=10.0, alpha_l=1.0)
    P1 = orc.make_params(step=10.0, alpha_l=1.0, g_std=0.3, seed=77)
    vol = const_volume((2, 2, 2), (0, 0, 0), 0.0)
    d0, _ = _update(orc, sc, vol, P0, 1.0, iteration=4)
    d1, _ = _update(orc, sc, vol, P1, 1.0, iteration=4)
    G = orc.g_draw(77, 0.3, 4, 0, 0, 0)
    assert G != 1.0
    np.testing.assert_allclose(d1, G * d0, rtol=1e-14)


def test_apply_update_clamps(orc):
    vol = np.zeros((2, 2, 2, 4))
    vol[..., 3] = 0.5
    dV = np.full((2, 2, 2, 3), -1.0)
    dV[0, 0, 0] = [2.0, 3.0, -0.5]
    out = orc.apply_update(vol, dV, clamp_nonneg=True)
    assert np.all(out[..., :3] >= 0.0)
    np.testing.assert_allclose(out[0, 0, 0], [2.0, 3.0, 0.0, 0.5])
    out2 = orc.apply_update(vol, dV, clamp_nonneg=False)
    np.testing.assert_allclose(out2[1, 1, 1], [-1.0, -1.0, -1.0, 0.5])


def test_flame_threshold_and_bbox(orc):
    """Sec. 4.1: pixels brighter than 30 (of 255) in some channel are flame;
    the rest become black.  The error box is the tight box of flame pixels."""
    k, hgt, w = 2, 6, 7
    t = np.zeros((k, hgt, w, 3))
    t[0, 2, 3] = [31 / 255, 0, 0]
    t[0, 4, 1] = [0, 0, 40 / 255]
    t[0, 1, 5] = [30 / 255, 30 / 255, 30 / 255]  # not strictly above: background
    t[1, 0, 0] = [0.01, 0.02, 0.03]
    out, mask, bbox = orc.prepare_targets(t, 30 / 255)
    assert mask[0].sum() == 2 and mask[1].sum() == 0
    assert np.all(out[0, 1, 5] == 0) and np.all(out[1] == 0)
    np.testing.assert_array_equal(bbox[0], [1, 2, 3, 4])
    assert bbox[1][0] > bbox[1][2]


def test_rmse_over_boxes(orc):
    rng = np.random.default_rng(0)
    k, hgt, w = 3, 5, 8
    r = rng.uniform(0, 1, (k, hgt, w, 3))
    t = rng.uniform(0, 1, (k, hgt, w, 3))
    bbox = np.array([[1, 1, 3, 2], [0, 0, 7, 4], [5, 3, 4, 3]], dtype=np.int32)  # last one empty
    res, rmse = orc.residual(r, t, bbox)
    np.testing.assert_allclose(res, t - r, rtol=0, atol=0)
    d = np.concatenate([(t - r)[0, 1:3, 1:4].reshape(-1, 3), (t - r)[1].reshape(-1, 3)])
    np.testing.assert_allclose(rmse, 255.0 * np.sqrt((d ** 2).mean(axis=0)), rtol=1e-13)


def _shifted(cams, delta_world):
    out = []
    for c in cams:
        c = dict(c)
        c["pos"] = [x + delta_world for x in c["pos"]]
        out.append(c)
    return out


def test_undecided_budget_covers_every_flip_of_a_small_shift(orc):
    """Moving every sample by 5e-5 voxels (inside the face margin) moves a
    node's adjustment by at most its undecided budget plus the continuous part
    of the change (distances and transmittances move by that much, about 1e-4
    of the largest node sum); with the margins at zero the same shift exceeds
    the budget at some node -- the budget is what covers the face crossings."""
    from paper_1809_06417_gb300 import synth
    n, views, side = 16, 4, 48
    shape, origin, h = synth.unit_grid(n)
    cams = synth.ring_cameras(views, side, side, elevation_jitter_deg=12.0, seed=5)
    vol = synth.blobs_volume(n, 5, radius_range=(2.0, 4.0))
    P = orc.make_params(step=0.5, alpha_l=0.01)
    sc = orc.Scene(shape, origin, h, cams)
    img, _ = orc.render(sc, vol, P)
    targets, mask, bbox = orc.prepare_targets(img / img.max(), 30 / 255)
    v0 = vol.copy()
    v0[..., :3] *= 0.3
    ren, _ = orc.render(sc, v0, P)
    res, _ = orc.residual(ren, targets, bbox)
    res *= mask[..., None]
    shifted = orc.Scene(shape, origin, h, _shifted(cams, 5e-5 * h))
    dV2, _ = orc.update_paper(shifted, v0, P, res, mask, 0)
    try:
        dV, _, und = orc.update_paper(sc, v0, P, res, mask, 0, with_undecided=True)
        diff = np.abs(dV2 - dV).max(axis=-1)
        cont = 1e-4 * np.abs(dV).max()
        assert np.count_nonzero(und) > 0
        assert np.count_nonzero(und) < 0.2 * und.size
        assert np.all(diff <= und + cont)
        assert np.any(diff > cont)                          # the shift does cross faces
        orc.set_undecided_margins(0.0, 0.0)
        _, _, und0 = orc.update_paper(sc, v0, P, res, mask, 0, with_undecided=True)
        assert np.any(diff > und0 + cont)
    finally:
        orc.set_undecided_margins()
