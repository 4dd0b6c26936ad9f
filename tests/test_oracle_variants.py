"""Pins for the variants the paper mentions without using: Henyey-Greenstein
in-scattering (Eq. 9, g != 0) and per-view sequential (Kaczmarz-order)
updates."""
import numpy as np
import pytest

from paper_1809_06417_gb300 import synth


def test_directional_radiance_closed_form(orc):
    """Zero extinction, constant emission q: the radiance arriving along a line
    is q times the number of unit segments behind the node, in each direction."""
    n = 6
    shape, origin, h = synth.unit_grid(n)
    vol = np.zeros((n, n, n, 4))
    vol[..., 0], vol[..., 1], vol[..., 2] = 0.3, 0.2, 0.1
    sc = orc.Scene(shape, origin, h, synth.ring_cameras(1, 8, 8))
    L6 = orc.scatter_L6(sc, vol)
    i = np.arange(n)
    q = np.array([0.3, 0.2, 0.1])
    np.testing.assert_allclose(L6[0, 0, :, 0], i[:, None] * q, rtol=1e-12)           # +x: i segments behind
    np.testing.assert_allclose(L6[0, 0, :, 1], (n - 1 - i)[:, None] * q, rtol=1e-12)  # -x
    np.testing.assert_allclose(L6[:, 0, 0, 5], (n - 1 - i)[:, None] * q, rtol=1e-12)  # -z
    np.testing.assert_allclose(L6.mean(axis=3), orc.scatter_J(sc, vol), rtol=1e-12)


@pytest.mark.parametrize("g", [0.3, 0.8, -0.5])
def test_hg_weights(orc, g):
    w0 = orc.hg_weights(0.0, [0.6, 0.0, 0.8])
    np.testing.assert_allclose(w0, 1 / 6, rtol=1e-15)
    w = orc.hg_weights(g, [1.0, 0.0, 0.0])
    assert w.sum() == pytest.approx(1.0, rel=1e-15)
    # towards +x: light travelling along +x is scattered forward, along -x backward
    assert w[0] / w[1] == pytest.approx(((1 + g) / (1 - g)) ** 3, rel=1e-12)
    np.testing.assert_allclose(w[2:], w[2], rtol=1e-15)
    assert w[2] / w[1] == pytest.approx(((1 + g) ** 2 / (1 + g * g)) ** 1.5, rel=1e-12)


def _case(orc, n=10, views=3, side=20):
    from gpu_cases import plume_case
    case = plume_case(n=n, views=views, side=side)
    sc = orc.Scene(case.shape, case.origin, case.h, case.cams)
    P = dict(step=case.step, alpha_l=4e-3)
    img, _ = orc.render(sc, case.vol, orc.make_params(**P))
    img /= img.max()
    t, mask, bbox = orc.prepare_targets(img, 30 / 255)
    v0 = case.vol.copy()
    v0[..., :3] = 0.02
    return sc, P, v0, t, mask, bbox, case.albedo


def test_hg_source_with_g_zero_is_isotropic(orc):
    sc, P, v0, t, mask, bbox, alb = _case(orc)
    L6 = orc.scatter_L6(sc, v0)
    iso = orc.scatter_source(v0, alb, orc.scatter_J(sc, v0))
    hg = orc.scatter_source_hg(v0, alb, L6, np.full(6, 1 / 6))
    np.testing.assert_allclose(hg, iso, rtol=1e-13, atol=1e-15)


def test_per_view_loop_reduces_to_the_simultaneous_one(orc):
    """A vanishing asymmetry makes the per-view loop the standard one (every
    view renders the same source, all views update together), and with one view
    the sequential order changes nothing."""
    sc, P, v0, t, mask, bbox, alb = _case(orc)
    a, ra, _ = orc.reconstruct(sc, v0, orc.make_params(**P), t, mask, bbox, 3, albedo=alb)
    b, rb, _ = orc.reconstruct(sc, v0, orc.make_params(**P, hg_g=1e-13), t, mask, bbox, 3, albedo=alb)
    np.testing.assert_allclose(b, a, rtol=1e-9, atol=1e-14)
    np.testing.assert_allclose(rb, ra, rtol=1e-9)
    sc1, P1, v1, t1, m1, b1, al1 = _case(orc, views=1)
    c, rc, _ = orc.reconstruct(sc1, v1, orc.make_params(**P1), t1, m1, b1, 3, albedo=al1)
    d, rd, _ = orc.reconstruct(sc1, v1, orc.make_params(**P1, sequential=1), t1, m1, b1, 3, albedo=al1)
    np.testing.assert_allclose(d, c, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(rd, rc, rtol=1e-12)


def test_variants_reduce_the_error(orc):
    sc, P, v0, t, mask, bbox, alb = _case(orc)
    for extra in (dict(hg_g=0.6), dict(sequential=1), dict(hg_g=-0.4, sequential=1)):
        _, r, _ = orc.reconstruct(sc, v0, orc.make_params(**P, **extra), t, mask, bbox, 5, albedo=alb)
        assert np.all(r[-1] < r[0]), extra
