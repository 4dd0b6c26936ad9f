"""Cameras from 3x4 projections and the volume-dimension rule of Sec. 4.2.

Host arithmetic of the library (no device): the projection round trip through
K [R | -R C] recovers the cameras, projections agree with the pinhole model,
unrepresentable intrinsics are refused; the volume dimensions follow a closed
form for a face-on cube and agree with the oracle's restatement for rings."""
import math

import numpy as np
import pytest

from paper_1809_06417_gb300 import flamerec as fr, synth


def _projection(cam):
    W, H, t = cam["width"], cam["height"], cam["tan_half_fov"]
    f = H / (2.0 * t)
    K = np.array([[f, 0.0, (W - 1) / 2.0], [0.0, f, (H - 1) / 2.0], [0.0, 0.0, 1.0]])
    R = np.stack([np.asarray(cam["right"]), -np.asarray(cam["up"]), np.asarray(cam["fwd"])])
    C = np.asarray(cam["pos"])
    return K @ np.hstack([R, (-R @ C)[:, None]])


def _pixel(cam, X):
    """Pixel of world point X by the camera model's own formula (centres at integers)."""
    rel = np.asarray(X) - np.asarray(cam["pos"])
    xc, yc, zc = rel @ np.asarray(cam["right"]), rel @ np.asarray(cam["up"]), rel @ np.asarray(cam["fwd"])
    ty = cam["tan_half_fov"]
    tx = ty * cam["width"] / cam["height"]
    return ((xc / zc / tx + 1) * cam["width"] / 2 - 0.5, (1 - yc / zc / ty) * cam["height"] / 2 - 0.5)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_projection_round_trip(seed):
    rng = np.random.default_rng(seed)
    cams = synth.ring_cameras(5, 320 + 16 * seed, 240, elevation_jitter_deg=25.0, seed=seed, phase=0.3 * seed)
    for cam in cams:
        P = _projection(cam)
        for scale in (1.0, -3.7, 1e-3):
            back = fr.camera_from_projection(scale * P, cam["width"], cam["height"])
            for key in ("pos", "right", "up", "fwd"):
                np.testing.assert_allclose(back[key], cam[key], atol=2e-6)
            assert back["tan_half_fov"] == pytest.approx(cam["tan_half_fov"], rel=1e-6)
        X = rng.uniform(-0.5, 0.5, size=(20, 3))
        uvw = (P @ np.hstack([X, np.ones((20, 1))]).T).T
        for x, p in zip(X, uvw):
            np.testing.assert_allclose(p[:2] / p[2], _pixel(back, x), atol=2e-3)


def test_projection_with_unrepresentable_intrinsics_is_refused():
    cam = synth.ring_cameras(1, 200, 100)[0]
    P = _projection(cam)
    K_skew = np.array([[1.0, 0.01, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
    K_aspect = np.diag([1.0, 1.01, 1.0])
    K_shift = np.array([[1.0, 0.0, 3.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
    for A in (K_skew, K_aspect, K_shift):
        with pytest.raises(fr.FrError):
            fr.camera_from_projection(A @ P, 200, 100)
    with pytest.raises(fr.FrError):
        fr.camera_from_projection(np.zeros((3, 4)), 200, 100)


def test_volume_dims_face_on_cube_closed_form():
    """One camera on the +z axis at distance D, looking at the origin, and a
    cube of side L centred there.  Front-face edges span L f / (D - L/2)
    pixels (f = H / (2 tan(fov/2))); depth edges at the corners span
    (L/2) f (1/(D - L/2) - 1/(D + L/2))."""
    D, L, W, H = 3.0, 1.0, 512, 384
    t = math.tan(math.radians(50.0) / 2)
    cam = dict(pos=[0.0, 0.0, D], right=[1.0, 0.0, 0.0], up=[0.0, 1.0, 0.0], fwd=[0.0, 0.0, -1.0],
               tan_half_fov=t, width=W, height=H)
    f = H / (2 * t)
    n_face = L * f / (D - L / 2)
    n_depth = (L / 2) * f * (1 / (D - L / 2) - 1 / (D + L / 2))
    dims, h, n = fr.volume_dims([cam], [-L / 2] * 3, [L / 2] * 3, alpha=1.5)
    np.testing.assert_allclose(n, [n_face, n_face, n_depth], rtol=1e-5)
    assert h == pytest.approx(1.5 * L / n_face, rel=1e-6)
    assert dims == (math.ceil(n_face / 1.5 - 1e-6) + 1,) * 3


def test_volume_dims_follow_oracle_and_refuse_boxes_behind(orc):
    for k, side, seed in ((8, 512, 2), (10, 384, 4), (3, 256, 1)):
        cams = synth.ring_cameras(k, side, side, elevation_jitter_deg=10.0, seed=seed)
        lo, hi = [-0.5, -0.45, -0.5], [0.5, 0.55, 0.4]
        got = fr.volume_dims(cams, lo, hi, alpha=1.5)
        ref = orc.volume_dims(cams, lo, hi, alpha=1.5)
        assert got[0] == ref[0]
        assert got[1] == pytest.approx(ref[1], rel=1e-6)
        np.testing.assert_allclose(got[2], ref[2], rtol=1e-5)
    # the paper's rule for the 128^3 full-RTE cameras (8 views of 512^2 at radius 2)
    dims, h, n = fr.volume_dims(synth.ring_cameras(8, 512, 512, elevation_jitter_deg=10.0, seed=2),
                                [-0.5] * 3, [0.5] * 3)
    print("rule for 8 x 512^2 at radius 2:", dims, h, n)
    with pytest.raises(fr.FrError):
        fr.volume_dims(synth.ring_cameras(2, 64, 64, radius=0.3), [-0.5] * 3, [0.5] * 3)
    with pytest.raises(ValueError):
        orc.volume_dims(synth.ring_cameras(2, 64, 64, radius=0.3), [-0.5] * 3, [0.5] * 3)
