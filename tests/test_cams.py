"""Camera sets held by the library (fr_cams_create, fr_cams_ring): host
arithmetic, no device.  A ring equals the seeded input generator's ring given
the same elevations; calibrated 3x4 projections of known cameras give those
cameras back; projections the pinhole model cannot represent, mixed image
sizes and bad ring arguments are refused."""
import math

import numpy as np
import pytest

from paper_1809_06417_gb300 import flamerec as fr, synth


def _close(a, b, tol=2e-6):
    for x, y in zip(a, b):
        for key in ("pos", "right", "up", "fwd"):
            np.testing.assert_allclose(x[key], y[key], atol=tol * max(1.0, np.abs(y[key]).max()))
        assert abs(x["tan_half_fov"] - y["tan_half_fov"]) < 1e-6
        assert (x["width"], x["height"]) == (y["width"], y["height"])


@pytest.mark.parametrize("k,jitter,phase", [(8, 10.0, 0.0), (5, 0.0, 0.3), (12, 20.0, 1.1)])
def test_ring_equals_the_input_generator(k, jitter, phase):
    seed = 7
    ref = synth.ring_cameras(k, 96, 64, radius=2.5, elevation_jitter_deg=jitter, seed=seed, phase=phase)
    rng = np.random.default_rng(seed)        # the generator draws one elevation per camera, in order
    el = [rng.uniform(-jitter, jitter) if jitter else 0.0 for _ in range(k)]
    cams = fr.cams_ring(k, 96, 64, radius=2.5, elevation_deg=el, phase=phase)
    assert len(cams) == k
    _close(cams.as_dicts(), ref)
    cams.close()


def _projection(c):
    """P = K [R | -R C] of a camera dict: square pixels, principal point at
    the image centre, pixel centres at integers, v down."""
    W, H = c["width"], c["height"]
    f = H / (2.0 * c["tan_half_fov"])
    K = np.array([[f, 0.0, 0.5 * (W - 1)], [0.0, f, 0.5 * (H - 1)], [0.0, 0.0, 1.0]])
    R = np.array([c["right"], [-x for x in c["up"]], c["fwd"]])
    C = np.array(c["pos"])
    return K @ np.hstack([R, (-R @ C)[:, None]])


def test_create_from_projections_recovers_the_cameras():
    ref = synth.ring_cameras(6, 80, 60, elevation_jitter_deg=15.0, seed=3)
    P = [3.7 * _projection(c) for c in ref]     # a projection is defined up to scale
    cams = fr.cams_create(P, [(80, 60)] * 6)
    _close(cams.as_dicts(), ref, tol=1e-5)
    cams.close()


def test_refusals():
    ref = synth.ring_cameras(2, 80, 60)
    P = [_projection(c) for c in ref]
    with pytest.raises(fr.FrError):
        fr.cams_create(P, [(80, 60), (64, 64)])        # mixed image sizes
    skewed = P[0].copy()
    skewed[0, 1] += 5.0
    with pytest.raises(fr.FrError):
        fr.cams_create([skewed], [(80, 60)])           # skew: not the pinhole model
    with pytest.raises(fr.FrError):
        fr.cams_ring(0, 64, 64)
    with pytest.raises(fr.FrError):
        fr.cams_ring(4, 64, 64, radius=-1.0)
    with pytest.raises(fr.FrError):
        fr.cams_ring(4, 64, 64, fov_deg=180.0)
    with pytest.raises(fr.FrError):
        fr.cams_ring(2, 64, 64, elevation_deg=[0.0, 90.0])
    assert fr.load().fr_cams_count(None) == 0


def test_ring_geometry_closed_form():
    """Camera i sits at centre + radius (cos el cos th, sin el, cos el sin th)
    and looks at the centre; its axes are orthonormal with right horizontal."""
    centre = (0.1, -0.2, 0.3)
    cams = fr.cams_ring(4, 32, 32, center=centre, radius=2.0, elevation_deg=[0.0, 10.0, -20.0, 5.0],
                        phase=0.25).as_dicts()
    for i, c in enumerate(cams):
        th = 0.25 + 2 * math.pi * i / 4
        el = math.radians([0.0, 10.0, -20.0, 5.0][i])
        want = np.array(centre) + 2.0 * np.array([math.cos(el) * math.cos(th), math.sin(el),
                                                   math.cos(el) * math.sin(th)])
        np.testing.assert_allclose(c["pos"], want, atol=1e-6)
        f, r, u = (np.array(c[k]) for k in ("fwd", "right", "up"))
        np.testing.assert_allclose(f, (np.array(centre) - want) / 2.0, atol=1e-6)
        assert abs(r[1]) < 1e-7
        np.testing.assert_allclose([f @ f, r @ r, u @ u, f @ r, f @ u, r @ u], [1, 1, 1, 0, 0, 0], atol=1e-6)
        assert u[1] > 0
