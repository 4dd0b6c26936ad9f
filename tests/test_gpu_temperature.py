"""The paper-literal temperature path (Sec. 3.3.3): reconstruct the green
channel with the paper rule, then read the temperature off the
colour-temperature table.  The inverse on the GPU follows the oracle's on the
same table; the whole path recovers a seeded temperature field, better with
more cameras (the paper's camera-count experiment, on synthetic data)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

T_MIN, T_MAX = 800.0, 2000.0


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_06417_gb300 import flamerec as fr, synth
    ctx = fr.Context(0)
    lut = torch.zeros((1024, 4), device="cuda")
    ctx.fr_planck_lut(T_MIN, T_MAX, lut)
    yield fr, synth, ctx, lut
    torch.cuda.synchronize()
    ctx.close()


def test_green_to_temperature_follows_oracle(orc, setup):
    """Bisection and interpolation in float32 against the oracle on the same
    table: the segment found can differ only at a node, where both segments
    give that node's temperature, and the fraction carries about 1e-7 of a
    table step (1.2 K), so 1e-3 K bounds the difference."""
    fr, synth, ctx, _ = setup
    from gpu_cases import oracle_lut
    lut, lut_np = oracle_lut(orc, torch, T_MIN, T_MAX, 1024)   # one table for both sides
    rng = np.random.default_rng(5)
    n = 40
    g = rng.uniform(-0.1, 1.2, size=(n, n, n)) * rng.choice([1.0, 1e-4, 1e-7], size=(n, n, n))
    rgb = np.zeros((n, n, n, 4), dtype=np.float32)
    rgb[..., 1] = g
    rgb[..., 3] = rng.random((n, n, n))
    shape, origin, h = synth.unit_grid(n)
    src = torch.as_tensor(rgb, device="cuda")
    out = torch.zeros((n, n, n, 2), device="cuda")
    p = fr.params(lut=lut, lut_t_min=T_MIN, lut_t_max=T_MAX)
    ctx.fr_temperature_from_green(fr.volume(src, origin, h), p, fr.volume(out, origin, h, kind=fr.FR_KIND_TEMP))
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    ref = orc.green_to_temp(rgb[..., 1].astype(np.float64), lut_np, T_MIN, T_MAX)
    print("max |dT|", np.abs(got[..., 0] - ref).max())
    np.testing.assert_allclose(got[..., 0], ref, rtol=0, atol=1e-3)
    assert np.array_equal(got[..., 1], rgb[..., 3])


def _green_path(fr, synth, ctx, lut, gt, views, n, side, step, iters):
    """Targets rendered from the temperature field through the table; the green
    channel reconstructed with the paper rule inside the visual hull; the
    temperature read off the table.  Returns (T, inside-hull mask, image RMSE)."""
    shape, origin, h = synth.unit_grid(n)
    cams = synth.ring_cameras(views, side, side, elevation_jitter_deg=10.0, seed=3)
    fc = fr.cameras(cams)
    g = torch.as_tensor(gt, dtype=torch.float32, device="cuda").contiguous()
    pt = dict(lut=lut, lut_t_min=T_MIN, lut_t_max=T_MAX)
    img = torch.zeros((views, side, side, 3), device="cuda")
    ctx.fr_render(fr.volume(g, origin, h, kind=fr.FR_KIND_TEMP), fc, fr.params(step=step, **pt), img)
    thresh = 30 / 255 * float(img.max())
    bbox = torch.zeros((views, 4), dtype=torch.int32, device="cuda")
    ctx.fr_prepare_targets(img, thresh, bbox)
    rec = torch.zeros((n, n, n, 4), device="cuda")
    rec[..., 3] = g[..., 1]
    fv = fr.volume(rec, origin, h)
    tags = torch.zeros((n, n, n), dtype=torch.int32, device="cuda")
    ctx.fr_visual_hull(fv, fc, img, fr.params(flame_thresh=thresh), tags)
    alpha = 2e-4 * (n / 128.0) * (step / 0.5) * (8.0 / views) * (512.0 / side) ** 2
    p = fr.params(step=step, alpha_l=alpha, flame_thresh=thresh, use_hull=1, hull_tags=tags)
    rmse = np.zeros((iters, 3), dtype=np.float32)
    ctx.fr_reconstruct(fv, fc, img, bbox, iters, p, rmse=rmse)
    temp = torch.zeros((n, n, n, 2), device="cuda")
    ctx.fr_temperature_from_green(fv, fr.params(**pt), fr.volume(temp, origin, h, kind=fr.FR_KIND_TEMP))
    torch.cuda.synchronize()
    inside = tags.cpu().numpy().view(np.uint32) == (1 << views) - 1
    return temp.cpu().numpy()[..., 0], inside, rmse


def test_green_path_recovers_temperature_better_with_more_cameras(setup):
    """Compared inside the visual hull (Sec. 5.1), on the key points inside the
    hulls of both camera sets: 28 cameras recover the temperature better than 4.
    (With 30/255 of the brightest pixel as the flame threshold, only the hot
    core, about 1500-2000 K, is visible: green grows like exp(-26600 K / T).)"""
    fr, synth, ctx, lut = setup
    n, side, step, iters = 48, 96, 0.5, 40
    gt = synth.temperature_volume(n, 3)
    runs = {views: _green_path(fr, synth, ctx, lut, gt, views, n, side, step, iters) for views in (4, 28)}
    common = runs[4][1] & runs[28][1]
    assert common.sum() > 100
    err = {}
    for views, (t, inside, rmse) in runs.items():
        assert rmse[-1, 1] < 0.5 * rmse[0, 1]       # the green image error falls
        own = float(np.sqrt(np.mean((t[inside] - gt[..., 0][inside]) ** 2)))
        err[views] = float(np.sqrt(np.mean((t[common] - gt[..., 0][common]) ** 2)))
        print(f"{views} views: temperature RMSE in its hull {own:.1f} K ({inside.sum()} key points), "
              f"in both hulls {err[views]:.1f} K; green image RMSE {rmse[0, 1]:.2f} -> {rmse[-1, 1]:.2f}")
    assert err[28] < 0.8 * err[4]
