"""Host-side fault handling and resume on the GPU, without faulting it: a
scratch limit forces an allocation failure (FR_ENOMEM, nothing launched, the
context stays usable), and a reconstruction stopped at an iteration boundary
resumes to the same result, G(s) seeded by the iteration counter."""
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


def _case(fr, ctx):
    case = plume_case(n=40, views=4, side=64)
    g = torch.as_tensor(case.vol, dtype=torch.float32, device="cuda").contiguous()
    img = torch.zeros((4, 64, 64, 3), device="cuda")
    ctx.fr_render(fr.volume(g, case.origin, case.h), fr.cameras(case.cams), fr.params(step=case.step), img)
    img /= img.max()
    bbox = torch.zeros((4, 4), dtype=torch.int32, device="cuda")
    ctx.fr_prepare_targets(img, 30 / 255, bbox)
    return case, g, img, bbox


def test_scratch_limit_refuses_then_recovers(fr):
    ctx = fr.Context(0)
    try:
        case, g, img, bbox = _case(fr, ctx)
        held = ctx.fr_scratch_bytes()
        ctx.fr_set_scratch_limit(held + 1)               # no room for the error partials
        res = torch.full_like(img, 7.0)
        sq = torch.zeros(4, device="cuda")
        fv = fr.volume(g, case.origin, case.h)
        with pytest.raises(fr.FrError) as info:
            ctx.fr_render_residual(fv, fr.cameras(case.cams), fr.params(step=case.step), img, bbox, None, res, sq)
        assert info.value.status == fr.FR_ENOMEM
        torch.cuda.synchronize()
        assert float(res.min()) == 7.0                    # nothing ran
        ctx.fr_set_scratch_limit(0)                       # no limit
        ctx.fr_render_residual(fv, fr.cameras(case.cams), fr.params(step=case.step), img, bbox, None, res, sq)
        torch.cuda.synchronize()
        assert ctx.fr_scratch_bytes() > held
        ref = fr.Context(0)
        res2 = torch.empty_like(img)
        sq2 = torch.zeros(4, device="cuda")
        ref.fr_render_residual(fv, fr.cameras(case.cams), fr.params(step=case.step), img, bbox, None, res2, sq2)
        torch.cuda.synchronize()
        assert torch.equal(res, res2) and torch.equal(sq, sq2)
        ref.close()
    finally:
        torch.cuda.synchronize()
        ctx.close()


def test_resume_at_an_iteration_boundary(fr):
    ctx = fr.Context(0)
    try:
        case, g, img, bbox = _case(fr, ctx)
        p = fr.params(step=case.step, alpha_l=3e-3, g_std=0.2, seed=11, use_hull=1)
        v0 = g.clone()
        v0[..., :3] = 0.0
        straight = v0.clone()
        r6 = np.zeros((6, 3), dtype=np.float32)
        ctx.fr_reconstruct(fr.volume(straight, case.origin, case.h), fr.cameras(case.cams), img, bbox, 6, p, rmse=r6)
        resumed = v0.clone()
        ra = np.zeros((3, 3), dtype=np.float32)
        rb = np.zeros((3, 3), dtype=np.float32)
        fv = fr.volume(resumed, case.origin, case.h)
        ctx.fr_reconstruct(fv, fr.cameras(case.cams), img, bbox, 3, p, rmse=ra)
        checkpoint = resumed.cpu()                        # e.g. written to disk
        resumed.copy_(checkpoint.cuda())
        ctx.fr_reconstruct(fv, fr.cameras(case.cams), img, bbox, 3, p, first_iteration=3, rmse=rb)
        torch.cuda.synchronize()
        assert np.max(rel_err(resumed.cpu().numpy(), straight.cpu().numpy())) < 1e-5
        np.testing.assert_allclose(np.vstack([ra, rb]), r6, rtol=1e-5)
        # a resumed run that forgot the counter draws other G(s) and ends elsewhere
        other = torch.as_tensor(checkpoint).cuda()
        ctx.fr_reconstruct(fr.volume(other, case.origin, case.h), fr.cameras(case.cams), img, bbox, 3, p)
        torch.cuda.synchronize()
        assert np.max(rel_err(other.cpu().numpy(), straight.cpu().numpy())) > 1e-4
    finally:
        torch.cuda.synchronize()
        ctx.close()
