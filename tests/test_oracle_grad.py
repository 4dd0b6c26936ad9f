"""Pins for the oracle's exact image gradient (the differentiable variant of
the adjustment): the adjoint identity for the source, which the render is
linear in, and central finite differences for extinction and temperature."""
import numpy as np
import pytest


def _scene(orc, n=(7, 6, 8), k=3, side=(10, 9), jitter=10.0):
    from paper_1809_06417_gb300 import synth
    cams = synth.ring_cameras(k, side[0], side[1], radius=2.0 * max(n), elevation_jitter_deg=jitter, seed=4)
    origin = tuple(-(s - 1) / 2.0 for s in n)
    return orc.Scene(n, origin, 1.0, cams)


def _loss(orc, sc, vol, P, y):
    img, _ = orc.render(sc, vol, P)
    return float(np.sum(img * y)), img


@pytest.mark.parametrize("tau", [0.0, 0.05])
def test_adjoint_identity_for_source(orc, tau):
    """<R S, y> = <S, R^T y> for the (linear) map from node sources S to pixels."""
    rng = np.random.default_rng(1)
    sc = _scene(orc)
    nx, ny, nz = sc.shape
    vol = rng.uniform(0, 1, (nz, ny, nx, 4))
    vol[..., 3] *= 0.5
    P = orc.make_params(step=0.55, tau=tau)
    y = rng.normal(size=sc.image_shape())
    lhs, img = _loss(orc, sc, vol, P, y)
    g = orc.grad(sc, vol, P, img, y)
    rhs = float(np.sum(vol[..., :3] * g[..., :3]))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    if tau > 0:
        assert np.all(g[..., 3] == 0.0)


def test_extinction_gradient_matches_central_differences(orc):
    rng = np.random.default_rng(2)
    sc = _scene(orc)
    nx, ny, nz = sc.shape
    vol = rng.uniform(0, 1, (nz, ny, nx, 4))
    vol[..., 3] = rng.uniform(0.0, 0.6, (nz, ny, nx))
    vol[2:4, 2:4, 2:4, 3] = 0.0  # include zero-extinction nodes
    P = orc.make_params(step=0.45)
    y = rng.normal(size=sc.image_shape())
    _, img = _loss(orc, sc, vol, P, y)
    g = orc.grad(sc, vol, P, img, y)
    eps = 1e-5
    nodes = [(3, 3, 3), (1, 2, 5), (4, 1, 2), (2, 4, 6), (0, 0, 0), (7, 5, 6)]
    for (k, j, i) in nodes:
        for c in (3, 0, 2):
            vp, vm = vol.copy(), vol.copy()
            vp[k, j, i, c] += eps
            vm[k, j, i, c] -= eps
            fd = (_loss(orc, sc, vp, P, y)[0] - _loss(orc, sc, vm, P, y)[0]) / (2 * eps)
            assert abs(fd - g[k, j, i, c]) <= 1e-6 * max(1.0, abs(fd)), (k, j, i, c, fd, g[k, j, i, c])


def test_temperature_gradient_matches_central_differences(orc):
    rng = np.random.default_rng(3)
    sc = _scene(orc, n=(6, 7, 6))
    nx, ny, nz = sc.shape
    lut = orc.lut_build(800.0, 2000.0, 4096)
    vol = np.zeros((nz, ny, nx, 2))
    vol[..., 0] = rng.uniform(900.0, 1900.0, (nz, ny, nx))
    vol[..., 1] = rng.uniform(0.02, 0.3, (nz, ny, nx))
    P = orc.make_params(step=0.5)
    y = rng.normal(size=sc.image_shape())
    img, _ = orc.render_temp(sc, vol, lut, 800.0, 2000.0, P)
    g = orc.grad_temp(sc, vol, lut, 800.0, 2000.0, P, img, y)

    def loss(v):
        return float(np.sum(orc.render_temp(sc, v, lut, 800.0, 2000.0, P)[0] * y))

    for (k, j, i) in [(2, 3, 2), (1, 1, 4), (4, 5, 3), (3, 2, 1)]:
        for c, eps in ((0, 1e-3), (1, 1e-5)):
            vp, vm = vol.copy(), vol.copy()
            vp[k, j, i, c] += eps
            vm[k, j, i, c] -= eps
            fd = (loss(vp) - loss(vm)) / (2 * eps)
            assert abs(fd - g[k, j, i, c]) <= 2e-4 * max(abs(fd), 1e-3), (k, j, i, c, fd, g[k, j, i, c])
