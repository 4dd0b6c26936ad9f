"""One context running reconstructions of different sizes, rules and hull
settings one after another gives the results of fresh contexts: the scratch
it keeps between calls (the update accumulator, which every completed call
leaves zero and the next call then does not clear, the flame-ray list, the
brick tables, the reduction counter) carries nothing from one call to the
next."""
import numpy as np
import pytest

from gpu_cases import plume_case, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_06417_gb300 import flamerec
    return flamerec


def _job(fr, ctx, n, views, side, iters, scatter, **kw):
    case = plume_case(n=n, views=views, side=side)
    g = torch.as_tensor(case.vol, dtype=torch.float32, device="cuda").contiguous()
    fc = fr.cameras(case.cams)
    img = torch.zeros((views, side, side, 3), device="cuda")
    ctx.fr_render(fr.volume(g, case.origin, case.h), fc, fr.params(step=case.step), img)
    img /= img.max()
    bbox = torch.zeros((views, 4), dtype=torch.int32, device="cuda")
    ctx.fr_prepare_targets(img, 30 / 255, bbox)
    v = g.clone()
    v[..., :3] = 0.01
    alb = torch.as_tensor(case.albedo, dtype=torch.float32, device="cuda").contiguous() if scatter else None
    rmse = np.zeros((iters, 3), dtype=np.float32)
    ctx.fr_reconstruct(fr.volume(v, case.origin, case.h), fc, img, bbox, iters,
                       fr.params(step=case.step, alpha_l=3e-3, **kw), albedo=alb, rmse=rmse)
    torch.cuda.synchronize()
    return v.cpu().numpy(), rmse


JOBS = [
    dict(n=40, views=5, side=64, iters=3, scatter=True, use_hull=1),
    dict(n=24, views=4, side=48, iters=2, scatter=False),
    dict(n=48, views=6, side=72, iters=2, scatter=True, use_hull=1),
    dict(n=32, views=4, side=64, iters=2, scatter=False, rule=1, grad_step=0.5),
    dict(n=40, views=5, side=64, iters=3, scatter=True, use_hull=1, sequential_views=1),
    dict(n=40, views=5, side=64, iters=3, scatter=True, use_hull=1),
]


def test_reused_context_matches_fresh_contexts(fr):
    ctx = fr.Context(0)
    try:
        got = [_job(fr, ctx, **j) for j in JOBS]
    finally:
        torch.cuda.synchronize()
        ctx.close()
    for j, (v, rmse) in zip(JOBS, got):
        fresh = fr.Context(0)
        try:
            v_ref, rmse_ref = _job(fr, fresh, **j)
        finally:
            torch.cuda.synchronize()
            fresh.close()
        e = rel_err(v, v_ref)
        print(f"{j}: max {e.max():.2e}")
        # the same arithmetic up to the order of the update's atomic sums
        assert e.max() < 1e-5, j
        np.testing.assert_allclose(rmse, rmse_ref, rtol=1e-5)
    # the first and last jobs are the same problem
    np.testing.assert_allclose(got[0][1], got[-1][1], rtol=1e-5)
