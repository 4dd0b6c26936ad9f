"""Pins for the oracle's forward rendering (Sec. 3.2 Eq. 6; Sec. 3.3.1 Eqs. 7-8,
Eq. 12).  Each expected value comes from a closed form, a library routine or an
invariant, never from the oracle itself."""
import math

import numpy as np
import pytest

from oracle_scenes import affine_volume, chord_through_centre, const_volume, one_pixel_camera


def _scene(orc, shape, cams):
    return orc.Scene(shape, (0.0, 0.0, 0.0), 1.0, cams)


def _centre(shape):
    return [(n - 1) / 2.0 for n in shape]


@pytest.mark.parametrize("step", [1.0, 0.7, 0.5, 0.3, 10.0])
def test_homogeneous_slab_axis_ray(orc, step):
    """Constant source S and extinction s over a chord of length l: the
    optical model integrates to S (1 - exp(-s l)) / s for any step."""
    shape = (5, 6, 7)
    S, s = (0.3, 0.2, 0.1), 0.37
    cam = one_pixel_camera(_centre(shape), (1.0, 0.0, 0.0))
    img, n = orc.render(_scene(orc, shape, [cam]), const_volume(shape, S, s), orc.make_params(step=step))
    l = shape[0] - 1
    expect = np.asarray(S) * (1.0 - math.exp(-s * l)) / s
    np.testing.assert_allclose(img[0, 0, 0], expect, rtol=1e-12)
    assert n == math.ceil(l / step)


@pytest.mark.parametrize("seed", range(6))
def test_homogeneous_slab_oblique(orc, seed):
    rng = np.random.default_rng(seed)
    shape = (9, 7, 8)
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    S, s = rng.uniform(0.1, 1.0, 3), rng.uniform(0.05, 0.8)
    step = rng.uniform(0.2, 1.3)
    cam = one_pixel_camera(_centre(shape), d)
    img, _ = orc.render(_scene(orc, shape, [cam]), const_volume(shape, S, s), orc.make_params(step=step))
    l = chord_through_centre(shape, d)
    np.testing.assert_allclose(img[0, 0, 0], S * (1.0 - math.exp(-s * l)) / s, rtol=1e-11)


def _chord_by_bisection(shape, o, d):
    """Entry and exit parameters of o + t d in the node box, found by
    bracketing on a fine grid and bisecting the inside/outside predicate."""
    hi = np.asarray([n - 1 for n in shape], dtype=np.float64)

    def inside(t):
        p = o + t * d
        return bool(np.all(p >= 0.0) and np.all(p <= hi))

    ts = np.linspace(0.0, 200.0, 200001)
    ins = np.array([inside(t) for t in ts[::50]])
    idx = np.nonzero(ins)[0]
    assert len(idx), "ray misses"
    a_out, a_in = ts[::50][max(idx[0] - 1, 0)], ts[::50][idx[0]]
    b_in, b_out = ts[::50][idx[-1]], ts[::50][min(idx[-1] + 1, len(ins) - 1)]
    for _ in range(80):
        m = 0.5 * (a_out + a_in)
        if inside(m):
            a_in = m
        else:
            a_out = m
        m = 0.5 * (b_in + b_out)
        if inside(m):
            b_in = m
        else:
            b_out = m
    return a_in, b_in


@pytest.mark.parametrize("seed", range(6))
def test_zero_extinction_affine_is_line_integral(orc, seed):
    """With s = 0 the pixel is the line integral of the source.  Trilinear
    interpolation reproduces affine fields and the midpoint rule integrates
    them exactly, so L = chord length * S(chord midpoint), for any ray."""
    rng = np.random.default_rng(100 + seed)
    shape = (6, 5, 7)
    a = rng.uniform(1.0, 2.0, 3)
    b = rng.uniform(-0.1, 0.1, (3, 3))
    vol = affine_volume(shape, a, b)
    through = np.asarray(_centre(shape)) + rng.uniform(-1.5, 1.5, 3)
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    cam = one_pixel_camera(through, d, back=30.0)
    img, _ = orc.render(_scene(orc, shape, [cam]), vol, orc.make_params(step=rng.uniform(0.2, 1.2)))
    o = np.asarray(cam["pos"])
    t0, t1 = _chord_by_bisection(shape, o, d)
    mid = o + 0.5 * (t0 + t1) * d
    expect = (t1 - t0) * (a + b @ mid)
    np.testing.assert_allclose(img[0, 0, 0], expect, rtol=1e-9)


def test_general_field_converges_to_transport_ode(orc):
    """For a non-homogeneous field, the rendered value converges (as the step
    shrinks) to the solution of dL/dt = T S, dT/dt = -s T along the ray with
    trilinearly interpolated fields (scipy's RegularGridInterpolator)."""
    from scipy.integrate import solve_ivp
    from scipy.interpolate import RegularGridInterpolator

    rng = np.random.default_rng(7)
    shape = (8, 8, 8)
    nx, ny, nz = shape
    vol = rng.uniform(0.0, 1.0, (nz, ny, nx, 4))
    vol[..., 3] *= 0.4
    axes = (np.arange(nz), np.arange(ny), np.arange(nx))
    interp = [RegularGridInterpolator(axes, vol[..., c]) for c in range(4)]
    d = np.array([0.8, 0.35, -0.45])
    d /= np.linalg.norm(d)
    through = np.asarray(_centre(shape)) + np.array([0.3, -0.2, 0.45])
    cam = one_pixel_camera(through, d, back=30.0)
    o = np.asarray(cam["pos"])
    t0, t1 = _chord_by_bisection(shape, o, d)

    def rhs(t, y):
        p = o + t * d
        zyx = np.clip(p[::-1], 0.0, [nz - 1, ny - 1, nx - 1])
        S = np.array([interp[c](zyx)[0] for c in range(3)])
        s = interp[3](zyx)[0]
        return np.concatenate([y[3] * S, [-s * y[3]]])

    sol = solve_ivp(rhs, (t0, t1), [0.0, 0.0, 0.0, 1.0], rtol=1e-11, atol=1e-13, max_step=0.01)
    exact = sol.y[:3, -1]
    errs = []
    for step in (0.2, 0.1, 0.05):
        img, _ = orc.render(_scene(orc, shape, [cam]), vol, orc.make_params(step=step))
        errs.append(np.max(np.abs(img[0, 0, 0] - exact) / np.abs(exact)))
    assert errs[-1] < 2e-3
    assert errs[2] < errs[0]


def test_transmittance_bounded_and_non_increasing(orc):
    rng = np.random.default_rng(3)
    shape = (10, 9, 11)
    nx, ny, nz = shape
    vol = rng.uniform(0.0, 1.0, (nz, ny, nx, 4))
    vol[..., 3] = rng.uniform(0.0, 0.6, (nz, ny, nx))
    cams = [one_pixel_camera(_centre(shape), rng.normal(size=3), back=40.0) for _ in range(5)]
    sc = _scene(orc, shape, cams)
    P = orc.make_params(step=0.45)
    img, tfin, _ = orc.render(sc, vol, P, return_t=True)
    for v in range(len(cams)):
        tb, ln, _ = orc.trace_pixel(sc, vol, P, v, 0, 0)
        assert len(tb) > 5
        assert tb[0] == 1.0
        assert np.all(tb <= 1.0) and np.all(tb > 0.0)
        assert np.all(np.diff(tb) <= 0.0)
        assert 0.0 < tfin[v, 0, 0] <= tb[-1]
        assert np.all(img[v] >= 0.0)
        # the segment lengths add up to the chord of the box
        o, d = np.asarray(cams[v]["pos"]), np.asarray(cams[v]["fwd"])
        t0, t1 = _chord_by_bisection(shape, o, d)
        np.testing.assert_allclose(ln.sum(), t1 - t0, rtol=1e-9)


@pytest.mark.parametrize("step,tau", [(1.0, 0.05), (0.7, 0.05), (0.5, 0.2)])
def test_constant_tau_blending(orc, step, tau):
    """Eqs. 7-8 with constant opacity tau: the k-th sample (1-based) sees
    T = (1 - tau)^(k-1) (Eq. 12) and a constant colour V blends to
    V (1 - (1 - tau)^n) after n samples."""
    shape = (5, 5, 5)
    V = np.array([0.9, 0.5, 0.2])
    cam = one_pixel_camera(_centre(shape), (0.0, 0.0, 1.0))
    sc = _scene(orc, shape, [cam])
    P = orc.make_params(step=step, tau=tau)
    vol = const_volume(shape, V, 123.0)  # sigma is ignored in this mode
    img, n = orc.render(sc, vol, P)
    assert n == math.ceil(4.0 / step)
    np.testing.assert_allclose(img[0, 0, 0], V * (1.0 - (1.0 - tau) ** n), rtol=1e-13)
    tb, _, _ = orc.trace_pixel(sc, vol, P, 0, 0, 0)
    np.testing.assert_allclose(tb, (1.0 - tau) ** np.arange(n), rtol=1e-14)


def test_linear_in_source(orc):
    rng = np.random.default_rng(11)
    shape = (7, 6, 5)
    nx, ny, nz = shape
    sig = rng.uniform(0.0, 0.5, (nz, ny, nx))
    v1, v2 = rng.uniform(0, 1, (2, nz, ny, nx, 4))
    v1[..., 3] = v2[..., 3] = sig
    v12 = v1.copy()
    v12[..., :3] = 2.0 * v1[..., :3] - 0.5 * v2[..., :3]
    from paper_1809_06417_gb300 import synth
    cams = synth.ring_cameras(3, 12, 10, radius=2.0 * 6, elevation_jitter_deg=10, seed=1)
    sc = orc.Scene(shape, (-3.0, -2.5, -2.0), 1.0, cams)
    P = orc.make_params(step=0.6)
    a, _ = orc.render(sc, v1, P)
    b, _ = orc.render(sc, v2, P)
    c, _ = orc.render(sc, v12, P)
    np.testing.assert_allclose(c, 2.0 * a - 0.5 * b, rtol=1e-11, atol=1e-13)


def test_camera_orientation(orc):
    """Pixel rows run top to bottom and columns left to right: a source in the
    upper (+y) half lights the top rows; one on the camera's right lights the
    right columns.  The ring camera at 90 degrees sits on +z looking at the
    origin, so its right is +x."""
    from paper_1809_06417_gb300 import synth
    n = 9
    shape, origin, h = synth.unit_grid(n)
    cams = synth.ring_cameras(4, 16, 16)
    sc = orc.Scene(shape, origin, h, cams)
    P = orc.make_params(step=0.5)
    up = np.zeros((n, n, n, 4))
    up[:, n // 2 + 1:, :, 0] = 1.0
    img, _ = orc.render(sc, up, P)
    assert img[:, :8, :, 0].sum() > 0 and img[:, 8:, :, 0].sum() == 0.0
    right = np.zeros((n, n, n, 4))
    right[:, :, n // 2 + 1:, 0] = 1.0
    img, _ = orc.render(sc, right, P)
    cam1 = img[1, :, :, 0]  # camera at +z
    assert cam1[:, 8:].sum() > 0 and cam1[:, :8].sum() == 0.0


def test_background_and_misses_are_black(orc):
    shape = (4, 4, 4)
    cam = one_pixel_camera((10.0, 10.0, 10.0), (0.0, 1.0, 0.0))  # passes beside the box
    img, n = orc.render(_scene(orc, shape, [cam]), const_volume(shape, (1, 1, 1), 0.1), orc.make_params())
    assert n == 0 and np.all(img == 0.0)
    # a ray that starts inside the box is clipped at t = 0
    cam = one_pixel_camera((1.5, 1.5, 1.5), (1.0, 0.0, 0.0), back=0.0)
    img, n = orc.render(_scene(orc, shape, [cam]), const_volume(shape, (1, 1, 1), 0.0), orc.make_params(step=0.5))
    np.testing.assert_allclose(img[0, 0, 0], [1.5, 1.5, 1.5], rtol=1e-12)
    assert n == 3
