"""Pins for the colour-temperature mapping (Sec. 3.3.3, Planck's law), the
phase function (Eq. 9) and the in-scattering estimate (Eq. 5, third term)."""
import math

import numpy as np
import pytest

from oracle_scenes import const_volume, one_pixel_camera

WIEN_B = 2.897771955e-3        # m K, CODATA 2018 exact-constant value
STEFAN_BOLTZMANN = 5.670374419e-8  # W m^-2 K^-4, CODATA 2018


@pytest.mark.parametrize("T", [800.0, 1500.0, 2000.0, 5800.0])
def test_planck_wien_displacement(orc, T):
    from scipy.optimize import minimize_scalar
    r = minimize_scalar(lambda x: -orc.planck(math.exp(x), T),
                        bounds=(math.log(1e-7), math.log(1e-4)), method="bounded",
                        options={"xatol": 1e-12})
    assert abs(math.exp(r.x) * T / WIEN_B - 1.0) < 1e-6


@pytest.mark.parametrize("T", [1000.0, 2000.0])
def test_planck_stefan_boltzmann(orc, T):
    """Integrated over all wavelengths, B gives sigma_SB T^4 / pi."""
    from scipy.integrate import quad
    edges = np.geomspace(5e-8, 1e-2, 60)
    tot = sum(quad(lambda l: orc.planck(l, T), a, b, epsabs=0, epsrel=1e-12, limit=200)[0]
              for a, b in zip(edges[:-1], edges[1:]))
    assert abs(tot / (STEFAN_BOLTZMANN * T ** 4 / math.pi) - 1.0) < 1e-7


def test_colour_mapping_normalisation_and_order(orc):
    np.testing.assert_allclose(orc.temp_rgb(2000.0)[1], 1.0, rtol=1e-15)
    Ts = np.linspace(800.0, 2000.0, 241)
    rgb = np.array([orc.temp_rgb(t) for t in Ts])
    # the green channel grows with temperature over the whole range (Sec. 3.3.3)
    assert np.all(np.diff(rgb[:, 1]) > 0)
    # a cool body is red-dominated
    assert rgb[0, 0] > rgb[0, 1] > rgb[0, 2] > 0


def test_lut_interpolation_error_bound(orc):
    """Rendering a homogeneous temperature slab through the table gives
    q(T) (1 - exp(-s l)) / s with q the linear interpolant of the exact
    mapping; its error is at most dT^2/8 max|q''| (linear interpolation bound)."""
    t_min, t_max, m = 800.0, 2000.0, 1024
    lut = orc.lut_build(t_min, t_max, m)
    dT = (t_max - t_min) / (m - 1)
    shape = (5, 5, 5)
    cam = one_pixel_camera((2.0, 2.0, 2.0), (0.0, 1.0, 0.0))
    sc = orc.Scene(shape, (0.0, 0.0, 0.0), 1.0, [cam])
    s = 0.1
    fac = (1.0 - math.exp(-4.0 * s)) / s
    for T in (812.3456, 1234.5678, 1999.0):
        vol = np.zeros((5, 5, 5, 2))
        vol[..., 0], vol[..., 1] = T, s
        img, _ = orc.render_temp(sc, vol, lut, t_min, t_max, orc.make_params(step=0.5))
        exact = orc.temp_rgb(T)
        h = 0.5
        q2 = np.abs(orc.temp_rgb(T + h) - 2 * exact + orc.temp_rgb(T - h)) / h ** 2
        bound = dT ** 2 / 8 * q2 * 1.5 + 1e-12
        assert np.all(np.abs(img[0, 0, 0] / fac - exact) <= bound)
    # clamped outside the table
    vol = np.zeros((5, 5, 5, 2))
    vol[..., 0], vol[..., 1] = 2500.0, s
    img, _ = orc.render_temp(sc, vol, lut, t_min, t_max, orc.make_params(step=0.5))
    np.testing.assert_allclose(img[0, 0, 0] / fac, orc.temp_rgb(t_max), rtol=1e-12)


@pytest.mark.parametrize("g", [-0.6, 0.0, 0.3, 0.85])
def test_phase_function_normalised(orc, g):
    from scipy.integrate import quad
    tot = 2 * math.pi * quad(lambda mu: orc.hg_phase(g, mu), -1, 1, epsabs=0, epsrel=1e-12, limit=200)[0]
    assert abs(tot - 1.0) < 1e-10
    if g == 0.0:
        assert orc.hg_phase(0.0, 0.37) == pytest.approx(1.0 / (4.0 * math.pi), rel=1e-15)


def test_scatter_homogeneous_closed_form(orc):
    """Constant q and s: along each axis the sweep reaches node i with
    q (1 - exp(-s u)) / s, u the number of unit segments behind it, so J is the
    mean over the six directions of that expression."""
    shape = (6, 5, 7)
    nx, ny, nz = shape
    q, s = np.array([0.5, 0.3, 0.1]), 0.25
    sc = orc.Scene(shape, (0, 0, 0), 1.0, [one_pixel_camera((0, 0, 0), (1, 0, 0))])
    J = orc.scatter_J(sc, const_volume(shape, q, s))
    f = lambda u: (1.0 - np.exp(-s * u)) / s
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    tot = f(i) + f(nx - 1 - i) + f(j) + f(ny - 1 - j) + f(k) + f(nz - 1 - k)
    np.testing.assert_allclose(J, tot[..., None] * q / 6.0, rtol=1e-13)


def test_scatter_without_extinction(orc):
    """s = 0: every direction collects q times the distance travelled, and
    the six distances at any node add to 3 (n - 1) for a cube of n nodes."""
    n = 5
    sc = orc.Scene((n, n, n), (0, 0, 0), 1.0, [one_pixel_camera((0, 0, 0), (1, 0, 0))])
    q = np.array([1.0, 2.0, 4.0])
    J = orc.scatter_J(sc, const_volume((n, n, n), q, 0.0))
    np.testing.assert_allclose(J, np.broadcast_to(q * (n - 1) / 2.0, J.shape), rtol=1e-14)


def test_scatter_source(orc):
    rng = np.random.default_rng(5)
    vol = rng.uniform(0, 1, (3, 4, 5, 4))
    J = rng.uniform(0, 1, (3, 4, 5, 3))
    zero = orc.scatter_source(vol, np.zeros((3, 4, 5)), J)
    np.testing.assert_array_equal(zero, vol)
    alb = rng.uniform(0, 0.3, (3, 4, 5))
    out = orc.scatter_source(vol, alb, J)
    np.testing.assert_allclose(out[..., :3], vol[..., :3] + (alb * vol[..., 3])[..., None] * J, rtol=1e-15)
    np.testing.assert_array_equal(out[..., 3], vol[..., 3])


def test_scatter_affine_source_without_extinction(orc):
    """s = 0 and an affine source: each axis sweep is the exact line integral
    (the segment average is the trapezoid rule, exact for affine q), and the
    two opposite directions add to (n - 1) q evaluated at the line's midpoint."""
    shape = (6, 5, 7)
    nx, ny, nz = shape
    a = np.array([1.0, 0.5, 0.25])
    b = np.array([[0.1, -0.05, 0.02], [0.03, 0.04, -0.01], [-0.02, 0.01, 0.05]])  # b[c] . (i, j, k)
    from oracle_scenes import affine_volume
    vol = affine_volume(shape, a, b)
    sc = orc.Scene(shape, (0, 0, 0), 1.0, [one_pixel_camera((0, 0, 0), (1, 0, 0))])
    J = orc.scatter_J(sc, vol)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")

    def q(x, y, z):
        return np.stack([a[c] + b[c][0] * x + b[c][1] * y + b[c][2] * z for c in range(3)], axis=-1)

    expect = ((nx - 1) * q((nx - 1) / 2.0, j, k) + (ny - 1) * q(i, (ny - 1) / 2.0, k)
              + (nz - 1) * q(i, j, (nz - 1) / 2.0)) / 6.0
    np.testing.assert_allclose(J, expect, rtol=1e-13)
