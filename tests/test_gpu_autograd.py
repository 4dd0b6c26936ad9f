"""The differentiable temperature path: 128^3 temperature field in 800-2000 K,
8 views at 512 x 512, Planck colour-temperature table (Sec. 3.3.3), forward and
adjoint through torch.autograd.Function, checked against central finite
differences at 64 random voxels and against the FP64 oracle gradient."""
import numpy as np
import pytest

from gpu_cases import oracle_lut, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_06417_gb300 import autograd as ag, flamerec as fr, synth
    ctx = fr.Context(0)
    lut = torch.zeros((4096, 4), device="cuda")
    ctx.fr_planck_lut(800.0, 2000.0, lut)
    yield fr, ag, synth, ctx, lut
    torch.cuda.synchronize()
    ctx.close()


def _scene(ag, fr, ctx, lut, n, views, side, step, seed):
    from paper_1809_06417_gb300 import synth
    shape, origin, h = synth.unit_grid(n)
    cams = synth.ring_cameras(views, side, side, elevation_jitter_deg=10.0, seed=seed)
    return ag.RenderScene(ctx, cams, origin, h, kind=fr.FR_KIND_TEMP, step=step, lut=lut,
                          lut_t_min=800.0, lut_t_max=2000.0), cams, (shape, origin, h)


def test_autograd_matches_finite_differences_at_full_size(setup):
    fr, ag, synth, ctx, lut = setup
    n, views, side, step = 128, 8, 512, 0.5
    scene, cams, _ = _scene(ag, fr, ctx, lut, n, views, side, step, 3)
    vol_np = synth.temperature_volume(n, 3)
    vol = torch.as_tensor(vol_np, dtype=torch.float32, device="cuda").requires_grad_(True)
    g = torch.Generator(device="cuda").manual_seed(3)
    w = torch.randn(scene.image_shape, generator=g, device="cuda", dtype=torch.float64)
    img = ag.render(vol, scene)
    (img.double() * w).sum().backward()
    grad = vol.grad.detach().double().cpu().numpy()

    rng = np.random.default_rng(64)
    T = vol_np[..., 0]
    interior = np.argwhere((T > 830.0) & (T < 1970.0))
    pick = interior[rng.choice(len(interior), size=64, replace=False)]
    checks = []
    with torch.no_grad():
        base = vol.detach().clone()
        for (k, j, i) in pick:
            for c, eps in ((0, 1.0), (1, 1e-3)):
                vp, vm = base.clone(), base.clone()
                vp[k, j, i, c] += eps
                vm[k, j, i, c] -= eps
                lp = (ag.render(vp, scene).double() * w).sum()
                lm = (ag.render(vm, scene).double() * w).sum()
                fd = float(lp - lm) / (2 * eps)
                checks.append((c, fd, grad[k, j, i, c]))
    for c in (0, 1):
        fd = np.array([x[1] for x in checks if x[0] == c])
        an = np.array([x[2] for x in checks if x[0] == c])
        scale = np.abs(an).max()
        err = np.abs(fd - an) / scale
        print(f"channel {c}: max |fd - grad| / max|grad| = {err.max():.3e} over {len(fd)} voxels")
        assert err.max() < 1e-2
        assert np.corrcoef(fd, an)[0, 1] > 0.999


def test_autograd_matches_oracle_gradient(setup, orc):
    fr, ag, synth, ctx, _ = setup
    lut, lut_ref = oracle_lut(orc, torch, 800.0, 2000.0, 4096)   # one table for both sides
    n, views, side, step = 32, 3, 48, 0.5
    scene, cams, (shape, origin, h) = _scene(ag, fr, ctx, lut, n, views, side, step, 5)
    vol_np = synth.temperature_volume(n, 5)
    vol_np[..., 1] = np.random.default_rng(1).uniform(0.02, 0.2, vol_np.shape[:3])
    vol = torch.as_tensor(vol_np, dtype=torch.float32, device="cuda").requires_grad_(True)
    img = ag.render(vol, scene)
    gimg = np.random.default_rng(2).normal(size=scene.image_shape)
    img.backward(torch.as_tensor(gimg, dtype=torch.float32, device="cuda"))
    sc = orc.Scene(shape, origin, h, cams)
    P = orc.make_params(step=step)
    ref_img, _ = orc.render_temp(sc, vol_np, lut_ref, 800.0, 2000.0, P)
    ref = orc.grad_temp(sc, vol_np, lut_ref, 800.0, 2000.0, P, ref_img, gimg)
    got = vol.grad.detach().double().cpu().numpy()
    for c in (0, 1):
        e = rel_err(got[..., c], ref[..., c])
        print(f"oracle gradient channel {c}: max {e.max():.3e}")
        assert e.max() < 5e-4


def test_gradient_descent_on_temperature_reduces_error(setup):
    """FR_RULE_GRADIENT reconstruction of a temperature field from images of
    the ground truth: the image error falls over the iterations."""
    fr, ag, synth, ctx, lut = setup
    n, views, side, step = 48, 8, 96, 0.5
    scene, cams, (shape, origin, h) = _scene(ag, fr, ctx, lut, n, views, side, step, 7)
    gt = torch.as_tensor(synth.temperature_volume(n, 7), dtype=torch.float32, device="cuda")
    targets = ag.render(gt, scene).detach().contiguous()
    bbox = torch.zeros((views, 4), dtype=torch.int32, device="cuda")
    ctx.fr_prepare_targets(targets, 1e-3, bbox)
    fv_cams = fr.cameras(cams)

    def run(step_size, iters):
        v = gt.clone()
        v[..., 0] = 1400.0
        p = fr.params(step=step, lut=lut, lut_t_min=800.0, lut_t_max=2000.0, rule=fr.FR_RULE_GRADIENT,
                      grad_step=step_size, flame_thresh=1e-3)
        rmse = np.zeros((iters, 3), dtype=np.float32)
        ctx.fr_reconstruct(fr.volume(v, origin, h, kind=fr.FR_KIND_TEMP), fv_cams, targets, bbox, iters, p,
                           rmse=rmse)
        torch.cuda.synchronize()
        return rmse[:, 1]

    # pick the step size from a short sweep, then iterate
    best = min((1e4, 3e4, 1e5, 3e5), key=lambda s: run(s, 4)[-1])
    rmse = run(best, 20)
    print("step", best, "rmse (green) per iteration", rmse)
    assert np.all(np.diff(rmse[:5]) < 0)
    assert rmse[-1] < 0.5 * rmse[0]
