"""The stop criterion of Sec. 3 on the GPU (fr_reconstruct_until): the loop
runs inside one CUDA graph whose conditional while node the device ends.  A
stopped run is a prefix of the fixed-length run, the iteration count follows
the criterion (and the oracle's), and the volumes agree with fr_reconstruct."""
import numpy as np
import pytest

from gpu_cases import plume_case, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fr_ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_06417_gb300 import flamerec as fr
    ctx = fr.Context(0)
    yield fr, ctx
    torch.cuda.synchronize()
    ctx.close()


def _setup(fr, ctx, case, thresh=30 / 255):
    views, side = len(case.cams), case.cams[0]["width"]
    g = torch.as_tensor(case.vol, dtype=torch.float32, device="cuda").contiguous()
    img = torch.zeros((views, side, side, 3), device="cuda")
    fc = fr.cameras(case.cams)
    ctx.fr_render(fr.volume(g, case.origin, case.h), fc, fr.params(step=case.step), img)
    img /= img.max()
    bbox = torch.zeros((views, 4), dtype=torch.int32, device="cuda")
    ctx.fr_prepare_targets(img, thresh, bbox)
    v0 = g.clone()
    v0[..., :3] = 0.01
    return fc, img, bbox, v0


@pytest.mark.parametrize("hull,albedo", [(0, False), (1, True)])
def test_until_is_a_prefix_of_the_fixed_run(fr_ctx, hull, albedo):
    fr, ctx = fr_ctx
    case = plume_case(n=40, views=5, side=72)
    fc, img, bbox, v0 = _setup(fr, ctx, case)
    alb = torch.as_tensor(case.albedo, dtype=torch.float32, device="cuda").contiguous() if albedo else None
    p = fr.params(step=case.step, alpha_l=3e-3, use_hull=hull)

    def fixed(iters):
        v = v0.clone()
        r = np.zeros((iters, 3), dtype=np.float32)
        ctx.fr_reconstruct(fr.volume(v, case.origin, case.h), fc, img, bbox, iters, p, albedo=alb, rmse=r)
        torch.cuda.synchronize()
        return v, r

    def until(max_iters, delta):
        v = v0.clone()
        r = np.zeros((max_iters, 3), dtype=np.float32)
        n = ctx.fr_reconstruct_until(fr.volume(v, case.origin, case.h), fc, img, bbox, max_iters, delta, p,
                                     albedo=alb, rmse=r)
        torch.cuda.synchronize()
        return v, r[:n], n

    v8, r8 = fixed(8)
    _, r_inf, n_inf = until(8, 1e30)
    assert n_inf == 2
    np.testing.assert_allclose(r_inf, r8[:2], rtol=1e-5)
    v_zero, r_zero, n_zero = until(8, 0.0)
    assert n_zero == 8
    np.testing.assert_allclose(r_zero, r8, rtol=1e-5)
    assert np.max(rel_err(v_zero.cpu().numpy(), v8.cpu().numpy())) < 1e-5
    step = np.abs(np.diff(r8.astype(np.float64), axis=0)).max(axis=1)
    k = 3                                           # stop after iteration k + 1 (k + 2 run)
    if not step[k] < step[k - 1]:
        pytest.skip("error steps do not shrink on this case")
    delta = 0.5 * (step[k - 1] + step[k])
    v_mid, r_mid, n_mid = until(8, delta)
    assert n_mid == k + 2, (n_mid, step, delta)
    v5, r5 = fixed(k + 2)
    np.testing.assert_allclose(r_mid, r5, rtol=1e-5)
    assert np.max(rel_err(v_mid.cpu().numpy(), v5.cpu().numpy())) < 1e-5
    print(f"hull={hull} albedo={albedo}: error steps {np.round(step, 4)}, stopped after {n_mid}")


def test_until_follows_the_oracle(orc, fr_ctx):
    fr, ctx = fr_ctx
    case = plume_case(n=28, views=4, side=48)
    sc = orc.Scene(case.shape, case.origin, case.h, case.cams)
    P = orc.make_params(step=case.step, alpha_l=3e-3)
    img, _ = orc.render(sc, case.vol, P)
    img /= img.max()
    t_ref, mask, bbox_ref = orc.prepare_targets(img, 30 / 255)
    v0 = case.vol.copy()
    v0[..., :3] = 0.01
    _, r_full, _ = orc.reconstruct(sc, v0, P, t_ref, mask, bbox_ref, 10)
    step = np.abs(np.diff(r_full, axis=0)).max(axis=1)
    k = int(np.argmax(step < 0.6 * step[0]))           # a threshold well inside the run
    delta = 0.5 * (step[k - 1] + step[k]) if k > 0 else 0.5 * step[0]
    vol_ref, r_ref, _ = orc.reconstruct(sc, v0, P, t_ref, mask, bbox_ref, 10, stop_delta=delta)
    t_dev = torch.as_tensor(img, dtype=torch.float32, device="cuda").contiguous()
    bbox = torch.zeros((len(case.cams), 4), dtype=torch.int32, device="cuda")
    ctx.fr_prepare_targets(t_dev, 30 / 255, bbox)
    v = torch.as_tensor(v0, dtype=torch.float32, device="cuda").contiguous()
    r = np.zeros((10, 3), dtype=np.float32)
    n = ctx.fr_reconstruct_until(fr.volume(v, case.origin, case.h), fr.cameras(case.cams), t_dev, bbox, 10, delta,
                                 fr.params(step=case.step, alpha_l=3e-3), rmse=r)
    torch.cuda.synchronize()
    print(f"oracle stopped after {len(r_ref)}, GPU after {n}")
    assert n == len(r_ref)
    np.testing.assert_allclose(r[:n], r_ref, rtol=1e-3)
    assert np.max(rel_err(v.cpu().numpy()[..., :3], vol_ref[..., :3])) < 1e-3


def test_until_rejects_bad_arguments(fr_ctx):
    fr, ctx = fr_ctx
    case = plume_case(n=20, views=3, side=32)
    fc, img, bbox, v0 = _setup(fr, ctx, case)
    fv = fr.volume(v0, case.origin, case.h)
    for max_iters, delta in ((0, 0.01), (4, -1.0), (4, float("nan")), (4, float("inf"))):
        with pytest.raises(fr.FrError):
            ctx.fr_reconstruct_until(fv, fc, img, bbox, max_iters, delta, fr.params(step=case.step))
