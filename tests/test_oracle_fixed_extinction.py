"""Pins for the reading the ray weight tables rest on: in the paper-rule loop
(Sec. 3.3.2) the update changes only the emission, so the extinction stays
what the call started with; with G(s) = 1 the rendering of Eqs. 5-8 is then
one linear map of the source records and the adjustment of Eq. 10 one
linear map of the residuals whose weights read the extinction alone, and the
in-scattering source of Sec. 3.2 is linear in the emission.  Both maps can
therefore be computed once per call and reused every iteration.  The last
test builds the two maps as matrices on a tiny grid (one render per node, one
adjustment per pixel) and runs the loop with them against the oracle's own
loop."""
import numpy as np
import pytest

from paper_1809_06417_gb300 import synth


def _scene(orc, shape=(7, 6, 5), views=3, side=(12, 10), seed=3):
    nx, ny, nz = shape
    edge = float(max(shape) - 1)
    cams = synth.ring_cameras(views, side[0], side[1], radius=2.0 * edge, elevation_jitter_deg=10, seed=seed)
    origin = (-(nx - 1) / 2.0, -(ny - 1) / 2.0, -(nz - 1) / 2.0)
    return orc.Scene(shape, origin, 1.0, cams)


def _volumes(shape, seed, n=2):
    """n random volumes sharing one random extinction field."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape
    sig = rng.uniform(0.0, 0.5, (nz, ny, nx))
    vols = rng.uniform(0.0, 1.0, (n, nz, ny, nx, 4))
    vols[..., 3] = sig
    return rng, vols


def test_extinction_stays_fixed_through_the_loop(orc):
    """Three paper-rule iterations with in-scattering change the emission
    and leave every extinction value bit for bit as it was."""
    sc = _scene(orc)
    rng, (v0, g) = _volumes(sc.shape, 31)
    P = orc.make_params(step=0.6, alpha_l=0.02)
    img, _ = orc.render(sc, g, P)
    t, mask, bbox = orc.prepare_targets(img / img.max(), 30.0 / 255.0)
    alb = rng.uniform(0.0, 0.3, v0.shape[:3])
    out, rmse, _ = orc.reconstruct(sc, v0, P, t, mask, bbox, 3, albedo=alb)
    np.testing.assert_array_equal(out[..., 3], v0[..., 3])
    assert np.abs(out[..., :3] - v0[..., :3]).max() > 1e-3          # the emission did move
    assert rmse.shape == (3, 3)


def test_adjustment_is_linear_in_the_residual(orc):
    sc = _scene(orc)
    rng, (v,) = _volumes(sc.shape, 21, n=1)
    P = orc.make_params(step=0.6, alpha_l=0.01, alpha_d=1.0)
    r1, r2 = rng.normal(0.0, 1.0, (2,) + sc.image_shape())
    mask = (rng.uniform(0.0, 1.0, sc.image_shape()[:3]) < 0.7).astype(np.uint8)
    a, n1 = orc.update_paper(sc, v, P, r1, mask, 0)
    b, n2 = orc.update_paper(sc, v, P, r2, mask, 0)
    c, n3 = orc.update_paper(sc, v, P, 2.0 * r1 - 0.5 * r2, mask, 0)
    assert n1 == n2 == n3 > 0
    np.testing.assert_allclose(c, 2.0 * a - 0.5 * b, rtol=1e-11, atol=1e-12 * np.abs(a).max())


def test_adjustment_reads_no_emission(orc):
    """Two volumes with one extinction field and different emission get the
    same adjustment from the same residual: Eq. 10's weight is the
    transmittance and the distance factor, neither of which reads q."""
    sc = _scene(orc)
    rng, (v1, v2) = _volumes(sc.shape, 22)
    P = orc.make_params(step=0.6, alpha_l=0.01, alpha_d=1.0)
    r = rng.normal(0.0, 1.0, sc.image_shape())
    mask = np.ones(sc.image_shape()[:3], dtype=np.uint8)
    a, na = orc.update_paper(sc, v1, P, r, mask, 0)
    b, nb = orc.update_paper(sc, v2, P, r, mask, 0)
    assert na == nb > 0
    np.testing.assert_array_equal(a, b)
    v3 = v1.copy()
    v3[..., 3] *= 1.5                                              # another extinction: other weights
    c, _ = orc.update_paper(sc, v3, P, r, mask, 0)
    assert np.abs(c - a).max() > 1e-6 * np.abs(a).max()


@pytest.mark.parametrize("g_std", [0.0, 0.3])
def test_weights_repeat_across_iterations_only_without_the_drawn_factor(orc, g_std):
    """With G(s) = 1 iteration 0 and iteration 5 adjust alike; with G(s)
    drawn per iteration (Eq. 11) they do not, which is why the tables need
    g_std = 0."""
    sc = _scene(orc)
    rng, (v,) = _volumes(sc.shape, 23, n=1)
    P = orc.make_params(step=0.6, alpha_l=0.01, g_std=g_std, seed=7)
    r = rng.normal(0.0, 1.0, sc.image_shape())
    mask = np.ones(sc.image_shape()[:3], dtype=np.uint8)
    a, _ = orc.update_paper(sc, v, P, r, mask, 0)
    b, _ = orc.update_paper(sc, v, P, r, mask, 5)
    if g_std == 0.0:
        np.testing.assert_array_equal(a, b)
    else:
        assert np.abs(a - b).max() > 1e-3 * np.abs(a).max()


def test_scattering_source_is_linear_in_the_emission(orc):
    """S = q + omega sigma J(q) with J from the axis sweeps: for a fixed
    extinction and albedo, S(2 q1 - 0.5 q2) = 2 S(q1) - 0.5 S(q2)."""
    sc = _scene(orc)
    rng, (v1, v2) = _volumes(sc.shape, 24)
    alb = rng.uniform(0.0, 0.3, v1.shape[:3])
    v12 = v1.copy()
    v12[..., :3] = 2.0 * v1[..., :3] - 0.5 * v2[..., :3]

    def source(v):
        return orc.scatter_source(v, alb, orc.scatter_J(sc, v))[..., :3]

    np.testing.assert_allclose(source(v12), 2.0 * source(v1) - 0.5 * source(v2), rtol=1e-11, atol=1e-13)


def test_loop_equals_the_fixed_matrix_iteration(orc):
    """On a 4^3 grid seen by two 6 x 6 views: A (pixels x nodes) from one
    render of each unit source, W (nodes x pixels) from one adjustment of each
    unit residual under the flame mask; then three iterations of
    V <- clamp(V + W r(t - A V)) (r: the residual inside the flame box) give
    the volume and the error rows of three iterations of the oracle's loop."""
    shape = (4, 4, 4)
    sc = _scene(orc, shape=shape, views=2, side=(6, 6), seed=5)
    rng, (v0, g) = _volumes(shape, 25)
    g[..., :3] *= np.linspace(0.2, 1.0, 4)[None, None, :, None]    # brighter towards +x
    P = orc.make_params(step=0.5, alpha_l=0.05)
    img, _ = orc.render(sc, g, P)
    t, mask, bbox = orc.prepare_targets(img / img.max(), 30.0 / 255.0)
    assert 0 < mask.sum() < mask.size
    ref, rmse_ref, _ = orc.reconstruct(sc, v0, P, t, mask, bbox, 3)

    nodes, kshape = sc.nodes, sc.image_shape()
    npx = kshape[0] * kshape[1] * kshape[2]
    A = np.zeros((npx, nodes))
    for j in range(nodes):
        e = v0.copy()
        e[..., :3] = 0.0
        e.reshape(nodes, 4)[j, :3] = 1.0
        im, _ = orc.render(sc, e, P)
        A[:, j] = im.reshape(npx, 3)[:, 0]
    W = np.zeros((nodes, npx))
    for p in range(npx):
        r = np.zeros(kshape)
        r.reshape(npx, 3)[p, :] = 1.0
        dV, _ = orc.update_paper(sc, v0, P, r, mask, 0)
        W[:, p] = dV.reshape(nodes, 3)[:, 0]
    assert np.count_nonzero(A) > 0 and np.count_nonzero(W) > 0

    v = v0.copy()
    for it in range(3):
        rendered = (A @ v.reshape(nodes, 4)[:, :3]).reshape(kshape)
        res, rmse = orc.residual(rendered, t, bbox)
        np.testing.assert_allclose(rmse, rmse_ref[it], rtol=1e-10)
        dV = (W @ res.reshape(npx, 3)).reshape(v.shape[:3] + (3,))
        v = orc.apply_update(v, dV)
    np.testing.assert_allclose(v, ref, rtol=1e-10, atol=1e-12)
