"""Henyey-Greenstein in-scattering (Eq. 9, g != 0) and sequential per-view
(Kaczmarz-order) updates on the GPU, against the oracle's per-view loop; with a
vanishing asymmetry the per-view loop matches the standard one."""
import numpy as np
import pytest

from gpu_cases import plume_case, rel_err, tags_on_device

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


def _run_gpu(fr, ctx, case, t_dev, bbox, v0, iters, **kw):
    v = torch.as_tensor(v0, dtype=torch.float32, device="cuda").contiguous()
    alb = torch.as_tensor(case.albedo, dtype=torch.float32, device="cuda").contiguous()
    rmse = np.zeros((iters, 3), dtype=np.float32)
    ctx.fr_reconstruct(fr.volume(v, case.origin, case.h), fr.cameras(case.cams), t_dev, bbox, iters,
                       fr.params(step=case.step, alpha_l=3e-3, **kw), albedo=alb, rmse=rmse)
    torch.cuda.synchronize()
    return v.cpu().numpy(), rmse


@pytest.mark.parametrize("variant", [dict(hg_g=0.6), dict(hg_g=-0.4), dict(sequential_views=1),
                                     dict(hg_g=0.5, sequential_views=1), dict(sequential_views=1, use_hull=1)])
def test_variant_follows_oracle(orc, fr_ctx, variant):
    fr, ctx = fr_ctx
    case = plume_case(n=32, views=4, side=48)
    sc = orc.Scene(case.shape, case.origin, case.h, case.cams)
    P0 = orc.make_params(step=case.step)
    img, _ = orc.render(sc, case.vol, P0)
    img /= img.max()
    t_ref, mask, bbox_ref = orc.prepare_targets(img, 30 / 255)
    v0 = case.vol.copy()
    v0[..., :3] = 0.01
    okw = dict(hg_g=variant.get("hg_g", 0.0), sequential=variant.get("sequential_views", 0))
    hull = orc.visual_hull(sc, mask) if variant.get("use_hull") else None
    ref, r_ref, _ = orc.reconstruct(sc, v0, orc.make_params(step=case.step, alpha_l=3e-3, **okw), t_ref, mask,
                                    bbox_ref, 3, albedo=case.albedo, hull=hull)
    t_dev = torch.as_tensor(img, dtype=torch.float32, device="cuda").contiguous()
    bbox = torch.zeros((len(case.cams), 4), dtype=torch.int32, device="cuda")
    ctx.fr_prepare_targets(t_dev, 30 / 255, bbox)
    kw = dict(variant)
    if hull is not None:
        kw["hull_tags"] = tags_on_device(torch, hull)   # one tag set for both sides
    got, rmse = _run_gpu(fr, ctx, case, t_dev, bbox, v0, 3, **kw)
    e = rel_err(got[..., :3], ref[..., :3])
    print(f"{variant}: max {e.max():.2e}, rmse {rmse[-1]} vs {r_ref[-1]}")
    np.testing.assert_allclose(rmse, r_ref, rtol=1e-3)
    assert e.max() < 2e-3


def test_vanishing_asymmetry_is_the_standard_loop(fr_ctx):
    fr, ctx = fr_ctx
    case = plume_case(n=40, views=5, side=64)
    g = torch.as_tensor(case.vol, dtype=torch.float32, device="cuda").contiguous()
    img = torch.zeros((5, 64, 64, 3), device="cuda")
    ctx.fr_render(fr.volume(g, case.origin, case.h), fr.cameras(case.cams), fr.params(step=case.step), img)
    img /= img.max()
    bbox = torch.zeros((5, 4), dtype=torch.int32, device="cuda")
    ctx.fr_prepare_targets(img, 30 / 255, bbox)
    v0 = case.vol.copy()
    v0[..., :3] = 0.01
    a, ra = _run_gpu(fr, ctx, case, img, bbox, v0, 3)
    b, rb = _run_gpu(fr, ctx, case, img, bbox, v0, 3, hg_g=1e-7)
    assert np.max(rel_err(b, a)) < 1e-5
    np.testing.assert_allclose(rb, ra, rtol=1e-5)
