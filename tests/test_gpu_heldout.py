"""Held-out view evaluation (the paper's extra evaluation: reconstruct from nine
of ten views, render the tenth).  The reconstruction lowers the error of the
view it never saw well below the empty volume's, and the input views fit
better than the test view."""
import numpy as np
import pytest

from gpu_cases import plume_case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _view_rmse(fr, ctx, fv, cams, p, targets, bbox):
    """255 x RMS of (target - render) inside each view's flame box, pooled."""
    res = torch.empty_like(targets)
    sq = torch.zeros(4, device="cuda")
    ctx.fr_render_residual(fv, cams, p, targets, bbox, None, res, sq)
    s = sq.cpu().numpy().astype(np.float64)
    return 255.0 * np.sqrt(s[:3] / max(s[3], 1.0))


def test_held_out_view():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_06417_gb300 import flamerec as fr
    ctx = fr.Context(0)
    try:
        case = plume_case(n=48, views=10, side=96)
        g = torch.as_tensor(case.vol, dtype=torch.float32, device="cuda").contiguous()
        fc_all = fr.cameras(case.cams)
        img = torch.zeros((10, 96, 96, 3), device="cuda")
        ctx.fr_render(fr.volume(g, case.origin, case.h), fc_all, fr.params(step=case.step), img)
        img /= img.max()
        train, test = list(range(9)), [9]
        t_in = img[train].contiguous()
        t_out = img[test].contiguous()
        b_in = torch.zeros((9, 4), dtype=torch.int32, device="cuda")
        b_out = torch.zeros((1, 4), dtype=torch.int32, device="cuda")
        ctx.fr_prepare_targets(t_in, 30 / 255, b_in)
        ctx.fr_prepare_targets(t_out, 30 / 255, b_out)
        c_in = fr.cameras([case.cams[i] for i in train])
        c_out = fr.cameras([case.cams[i] for i in test])
        v = g.clone()
        v[..., :3] = 0.0
        fv = fr.volume(v, case.origin, case.h)
        pr = fr.params(step=case.step)
        before = _view_rmse(fr, ctx, fv, c_out, pr, t_out, b_out)
        p = fr.params(step=case.step, alpha_l=2e-4 * (48 / 128) * (8 / 9) * (512 / 96) ** 2, use_hull=1)
        rmse = np.zeros((40, 3), dtype=np.float32)
        ctx.fr_reconstruct(fv, c_in, t_in, b_in, 40, p, rmse=rmse)
        after = _view_rmse(fr, ctx, fv, c_out, pr, t_out, b_out)
        fit = _view_rmse(fr, ctx, fv, c_in, pr, t_in, b_in)
        torch.cuda.synchronize()
        print(f"test view RMSE {before.round(2)} -> {after.round(2)}; input views {rmse[0].round(2)} -> {fit.round(2)}")
        assert np.all(after < 0.3 * before)
        assert fit[1] < after[1]
    finally:
        torch.cuda.synchronize()
        ctx.close()
