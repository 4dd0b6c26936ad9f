"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (float32 arithmetic against float64):
  * rendered radiance: |gpu - ref| <= 1e-4 |ref| + 1e-6 max|ref|.  The
    relative term covers float32 rounding of a few hundred transmittance
    products and sample positions (about 3e-5 voxels at 250 voxels from the
    camera); the small absolute term covers rays grazing the box edge, whose
    tiny values have no meaningful relative error.
  * accumulated node fields (adjustment, gradient): errors relative to the
    field's largest magnitude, since float atomics sum hundreds of terms of
    both signs in arbitrary order.
"""
import numpy as np
import pytest

from gpu_cases import oracle_lut, plume_case, ragged_case, rel_err, tiny_case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_06417_gb300 import flamerec
    flamerec.load()
    return flamerec


@pytest.fixture(scope="module")
def ctx(fr):
    c = fr.Context(0)
    yield c
    torch.cuda.synchronize()
    c.close()


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def oracle_scene(orc, case):
    return orc.Scene(case.shape, case.origin, case.h, case.cams)


def gpu_render(fr, ctx, case, vol=None, dtype=torch.float32, **kw):
    v = dev(case.vol if vol is None else vol, dtype)
    K, W, H = len(case.cams), case.cams[0]["width"], case.cams[0]["height"]
    out = torch.full((K, H, W, 3), -1.0, device="cuda")
    p = fr.params(step=case.step, **kw)
    ctx.fr_render(fr.volume(v, case.origin, case.h), fr.cameras(case.cams), p, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def assert_image_close(gpu, ref, what):
    err = np.abs(gpu - ref)
    bound = 1e-4 * np.abs(ref) + 1e-6 * np.abs(ref).max()
    worst = np.unravel_index(np.argmax(err - bound), err.shape)
    print(f"{what}: max rel-to-max err {err.max() / max(np.abs(ref).max(), 1e-30):.3e}")
    assert np.all(err <= bound), (what, worst, gpu[worst], ref[worst])


@pytest.mark.parametrize("case_fn", [tiny_case, ragged_case, lambda: tiny_case(seed=3, jitter=10.0, step=0.5)])
def test_render_field_mode(orc, fr, ctx, case_fn):
    case = case_fn()
    ref, _ = orc.render(oracle_scene(orc, case), case.vol, orc.make_params(step=case.step))
    got = gpu_render(fr, ctx, case)
    assert np.all(got >= 0.0)
    assert_image_close(got, ref, "render")


def test_render_constant_tau(orc, fr, ctx):
    case = ragged_case()
    ref, _ = orc.render(oracle_scene(orc, case), case.vol, orc.make_params(step=case.step, tau=0.05))
    got = gpu_render(fr, ctx, case, tau=0.05)
    assert_image_close(got, ref, "render tau")


def test_render_low_precision_storage(orc, fr, ctx):
    """bf16 / f16 records: against the oracle fed the same rounded values the
    kernel sees (float32 tolerance), and against the float32 volume within the
    storage tolerance of 1e-2."""
    case = tiny_case(seed=5, jitter=5.0)
    full, _ = orc.render(oracle_scene(orc, case), case.vol, orc.make_params(step=case.step))
    for dt in (torch.bfloat16, torch.float16):
        rounded = torch.as_tensor(case.vol).to(dt).to(torch.float64).numpy()
        ref, _ = orc.render(oracle_scene(orc, case), rounded, orc.make_params(step=case.step))
        got = gpu_render(fr, ctx, case, dtype=dt)
        assert_image_close(got, ref, f"render {dt}")
        assert np.max(rel_err(got, full)) < 1e-2


def test_sample_count_matches_oracle(orc, fr, ctx):
    case = ragged_case()
    _, n_ref = orc.render(oracle_scene(orc, case), case.vol, orc.make_params(step=case.step))
    v = dev(case.vol)
    n = ctx.fr_count_samples(fr.volume(v, case.origin, case.h), fr.cameras(case.cams), fr.params(step=case.step))
    # float32 and float64 may disagree on ceil(chord / step) for chords within
    # rounding of a multiple of the step: allow one sample per thousand rays
    rays = len(case.cams) * case.cams[0]["width"] * case.cams[0]["height"]
    assert abs(n - n_ref) <= max(1, rays // 1000), (n, n_ref)


def _prepared(orc, fr, ctx, case, noise=1e-3, seed=11):
    """Targets rendered by the oracle (+ noise), prepared on both sides."""
    from paper_1809_06417_gb300 import synth
    sc = oracle_scene(orc, case)
    img, _ = orc.render(sc, case.vol, orc.make_params(step=case.step))
    img = synth.add_noise(img / img.max(), noise, seed) if noise else img / img.max()
    t_ref, mask, bbox_ref = orc.prepare_targets(img, 30 / 255)
    t_dev = dev(img)
    bbox = torch.zeros((len(case.cams), 4), dtype=torch.int32, device="cuda")
    ctx.fr_prepare_targets(t_dev, 30 / 255, bbox)
    torch.cuda.synchronize()
    return img, t_ref, mask, bbox_ref, t_dev, bbox


def test_prepare_targets(orc, fr, ctx):
    case = ragged_case()
    img, t_ref, mask, bbox_ref, t_dev, bbox = _prepared(orc, fr, ctx, case)
    np.testing.assert_array_equal(bbox.cpu().numpy(), bbox_ref)
    np.testing.assert_array_equal(t_dev.cpu().numpy(), t_ref.astype(np.float32))


def test_render_residual_and_error(orc, fr, ctx):
    case = tiny_case(seed=2, jitter=6.0)
    img, t_ref, mask, bbox_ref, t_dev, bbox = _prepared(orc, fr, ctx, case)
    # a different volume than the one that made the targets
    vol = case.vol.copy()
    vol[..., :3] *= 0.7
    sc = oracle_scene(orc, case)
    P = orc.make_params(step=case.step)
    ren_ref, _ = orc.render(sc, vol, P)
    res_ref, rmse_ref = orc.residual(ren_ref, t_ref, bbox_ref)
    res_ref = res_ref * mask[..., None]
    v = dev(vol)
    ren = torch.empty_like(t_dev)
    res = torch.empty_like(t_dev)
    sq = torch.zeros(4, device="cuda")
    ctx.fr_render_residual(fr.volume(v, case.origin, case.h), fr.cameras(case.cams), fr.params(step=case.step),
                           t_dev, bbox, ren, res, sq)
    torch.cuda.synchronize()
    assert_image_close(ren.cpu().numpy().astype(np.float64), ren_ref, "rendered")
    r = res.cpu().numpy().astype(np.float64)
    assert np.all(r[mask == 0] == 0.0)
    assert np.max(rel_err(r, res_ref)) < 1e-5
    sq = sq.cpu().numpy().astype(np.float64)
    count = sum(max(0, b[2] - b[0] + 1) * max(0, b[3] - b[1] + 1) for b in bbox_ref)
    assert sq[3] == count
    rmse = 255.0 * np.sqrt(sq[:3] / sq[3])
    np.testing.assert_allclose(rmse, rmse_ref, rtol=1e-4)


def _adjust(fr, ctx, case, vol, residual, iteration=0, **kw):
    v = dev(vol)
    nx, ny, nz = case.shape
    dV = torch.zeros((nz, ny, nx, 4), device="cuda")
    ctx.fr_adjust(fr.volume(v, case.origin, case.h), fr.cameras(case.cams), fr.params(step=case.step, **kw),
                  dev(residual), iteration, dV)
    torch.cuda.synchronize()
    return dV.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("tau,g_std", [(0.0, 0.0), (0.05, 0.0), (0.0, 0.1)])
def test_adjust_paper_rule(orc, fr, ctx, tau, g_std):
    """Eq. 10 accumulated over all flame rays.  The key-point set of a sample
    changes when the sample crosses a cell face, so samples within float32
    rounding of a face may land in the neighbouring cell on one side only; the
    oracle bounds per node what such samples can move (its undecided budget),
    and every node must lie within 1e-5 of the largest node plus that budget."""
    case = tiny_case(seed=4, jitter=8.0, step=0.5)
    img, t_ref, mask, bbox_ref, t_dev, bbox = _prepared(orc, fr, ctx, case)
    vol = case.vol.copy()
    vol[..., :3] *= 0.5
    sc = oracle_scene(orc, case)
    P = orc.make_params(step=case.step, alpha_l=0.01, tau=tau, g_std=g_std, seed=99)
    ren, _ = orc.render(sc, vol, P)
    res, _ = orc.residual(ren, t_ref, bbox_ref)
    res *= mask[..., None]
    dV_ref, _, und = orc.update_paper(sc, vol, P, res, mask, 3, with_undecided=True)
    got = _adjust(fr, ctx, case, vol, res, iteration=3, alpha_l=0.01, tau=tau, g_std=g_std, seed=99)
    assert np.all(got[..., 3] == 0.0)
    scale = np.abs(dV_ref).max()
    err = np.abs(got[..., :3] - dV_ref).max(axis=-1)
    bound = 1e-5 * scale + und
    print(f"adjust tau={tau} g={g_std}: max error / max {err.max() / scale:.3e}, off undecided nodes "
          f"{err[und == 0].max() / scale:.3e}; {np.count_nonzero(und)} nodes with a budget; "
          f"worst error / bound {np.max(err / bound):.3f}")
    assert np.all(err <= bound)


def test_backward_matches_oracle_gradient(orc, fr, ctx):
    case = ragged_case()
    rng = np.random.default_rng(3)
    sc = oracle_scene(orc, case)
    P = orc.make_params(step=case.step)
    L, _ = orc.render(sc, case.vol, P)
    gimg = rng.normal(size=L.shape)
    g_ref = orc.grad(sc, case.vol, P, L, gimg)
    v = dev(case.vol)
    nx, ny, nz = case.shape
    g = torch.zeros((nz, ny, nx, 4), device="cuda")
    ctx.fr_render_backward(fr.volume(v, case.origin, case.h), fr.cameras(case.cams), fr.params(step=case.step),
                           dev(L), dev(gimg), g)
    torch.cuda.synchronize()
    got = g.cpu().numpy().astype(np.float64)
    for c, name in ((slice(0, 3), "source"), (slice(3, 4), "sigma")):
        e = rel_err(got[..., c], g_ref[..., c])
        print(f"backward {name}: max {e.max():.3e}")
        assert e.max() < 2e-4


def test_planck_table(orc, fr, ctx):
    m = 1024
    lut = torch.zeros((m, 4), device="cuda")
    ctx.fr_planck_lut(800.0, 2000.0, lut)
    torch.cuda.synchronize()
    ref = orc.lut_build(800.0, 2000.0, m)
    got = lut.cpu().numpy().astype(np.float64)
    assert np.all(got[:, 3] == 0.0)
    np.testing.assert_allclose(got[:, :3], ref, rtol=2e-5, atol=1e-7 * ref.max())


def test_temperature_render_and_gradient(orc, fr, ctx):
    from paper_1809_06417_gb300 import synth
    n = 24
    vol = synth.temperature_volume(n, 3)
    case = tiny_case(n=n, views=3, side=40, step=0.5, jitter=7.0)
    case.vol = vol
    lut, lut_ref = oracle_lut(orc, torch, 800.0, 2000.0, 4096)   # one table for both sides
    sc = oracle_scene(orc, case)
    P = orc.make_params(step=case.step)
    ref, _ = orc.render_temp(sc, vol, lut_ref, 800.0, 2000.0, P)
    v = dev(vol)
    fv = fr.volume(v, case.origin, case.h, kind=fr.FR_KIND_TEMP)
    p = fr.params(step=case.step, lut=lut, lut_t_min=800.0, lut_t_max=2000.0)
    out = torch.zeros((3, 40, 40, 3), device="cuda")
    ctx.fr_render(fv, fr.cameras(case.cams), p, out)
    torch.cuda.synchronize()
    assert_image_close(out.cpu().numpy().astype(np.float64), ref, "render temperature")
    rng = np.random.default_rng(8)
    gimg = rng.normal(size=ref.shape)
    g_ref = orc.grad_temp(sc, vol, lut_ref, 800.0, 2000.0, P, ref, gimg)
    g = torch.zeros((n, n, n, 2), device="cuda")
    ctx.fr_render_backward(fv, fr.cameras(case.cams), p, dev(ref), dev(gimg), g)
    torch.cuda.synchronize()
    got = g.cpu().numpy().astype(np.float64)
    for c in range(2):
        e = rel_err(got[..., c], g_ref[..., c])
        print(f"temperature grad {c}: max {e.max():.3e}")
        assert e.max() < 5e-4


def test_scatter_source(orc, fr, ctx):
    case = plume_case(n=20)
    sc = oracle_scene(orc, case)
    J_ref = orc.scatter_J(sc, case.vol)
    S_ref = orc.scatter_source(case.vol, case.albedo, J_ref)
    v = dev(case.vol)
    out = torch.zeros_like(v)
    nz, ny, nx = case.vol.shape[:3]
    J = torch.zeros((nz, ny, nx, 4), device="cuda")
    ctx.fr_scatter_source(fr.volume(v, case.origin, case.h), dev(case.albedo), J,
                          fr.volume(out, case.origin, case.h))
    torch.cuda.synchronize()
    assert np.max(rel_err(J.cpu().numpy()[..., :3], J_ref)) < 1e-5
    np.testing.assert_allclose(out.cpu().numpy(), S_ref, rtol=2e-5, atol=1e-6 * np.abs(S_ref).max())


def test_reconstruct_loop_tiny(orc, fr, ctx):
    """Ten iterations of Algorithm 2 (render, residual, adjust, apply): the
    per-iteration error and the final volume follow the oracle."""
    case = tiny_case()
    img, t_ref, mask, bbox_ref, t_dev, bbox = _prepared(orc, fr, ctx, case)
    sc = oracle_scene(orc, case)
    P = orc.make_params(step=case.step, alpha_l=0.01)
    v0 = case.vol.copy()
    v0[..., :3] = 0.0
    vol_ref, rmse_ref, _ = orc.reconstruct(sc, v0, P, t_ref, mask, bbox_ref, 10)
    v = dev(v0)
    rmse = np.zeros((10, 3), dtype=np.float32)
    ctx.fr_reconstruct(fr.volume(v, case.origin, case.h), fr.cameras(case.cams), t_dev, bbox, 10,
                       fr.params(step=case.step, alpha_l=0.01), rmse=rmse)
    torch.cuda.synchronize()
    print("rmse gpu", rmse[:, 1], "\nrmse ref", rmse_ref[:, 1])
    np.testing.assert_allclose(rmse, rmse_ref, rtol=2e-3)
    e = rel_err(v.cpu().numpy()[..., :3], vol_ref[..., :3])
    print(f"reconstruct volume: max {e.max():.3e}")
    assert e.max() < 5e-3


def test_invalid_arguments_are_rejected(fr, ctx):
    """Bad arguments return FR_EINVAL before any launch: a buffer that ends
    before the data it must hold (checked against its device allocation), a
    host pointer, a misaligned volume, a bad camera, a bad step."""
    case = tiny_case()
    v = dev(case.vol)
    out = torch.zeros((4, 64, 64, 3), device="cuda")
    cams = fr.cameras(case.cams)
    p = fr.params(step=case.step)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    big = torch.zeros(16 * 2 ** 20 // 4, device="cuda")  # its own 16 MiB allocation
    tail = big[-1000:]                                   # 4 kB before the allocation ends
    with pytest.raises(fr.FrError, match="FR_EINVAL.*allocation ends"):
        ctx.fr_render(fr.volume(v, case.origin, case.h), cams, p, tail)
    with pytest.raises(fr.FrError, match="FR_EINVAL"):
        ctx.fr_render(fr.volume(v, case.origin, case.h), cams, p, np.zeros((4, 64, 64, 3), np.float32))
    flat = torch.zeros(v.numel() + 1, device="cuda")
    mis = flat[1:].view(v.shape)                         # 4-byte offset: not 16-byte aligned
    with pytest.raises(fr.FrError, match="aligned"):
        ctx.fr_render(fr.volume(mis, case.origin, case.h), cams, p, out)
    bad = fr.cameras(case.cams)
    bad[0].fwd[0] += 0.5
    with pytest.raises(fr.FrError, match="orthonormal"):
        ctx.fr_render(fr.volume(v, case.origin, case.h), bad, p, out)
    with pytest.raises(fr.FrError, match="step"):
        ctx.fr_render(fr.volume(v, case.origin, case.h), cams, fr.params(step=0.0), out)
    # the context is still usable afterwards
    ctx.fr_render(fr.volume(v, case.origin, case.h), cams, p, out)
    torch.cuda.synchronize()
    assert float(out.max()) > 0.0


def test_reconstruct_loop_with_scattering(orc, fr, ctx):
    """Three iterations with the in-scattering source recomputed from the
    current volume each iteration (plume with albedo, jittered cameras,
    half-voxel step): per-iteration error and final volume follow the oracle."""
    case = plume_case(n=40, views=5, side=72)
    sc = oracle_scene(orc, case)
    P = orc.make_params(step=case.step, alpha_l=2e-3)
    src = orc.scatter_source(case.vol, case.albedo, orc.scatter_J(sc, case.vol))
    img, _ = orc.render(sc, src, P)
    img /= img.max()
    t_ref, mask, bbox_ref = orc.prepare_targets(img, 30 / 255)
    v0 = case.vol.copy()
    v0[..., :3] *= 0.3
    vol_ref, rmse_ref, _ = orc.reconstruct(sc, v0, P, t_ref, mask, bbox_ref, 3, albedo=case.albedo)
    t_dev = dev(img)
    bbox = torch.zeros((len(case.cams), 4), dtype=torch.int32, device="cuda")
    ctx.fr_prepare_targets(t_dev, 30 / 255, bbox)
    v = dev(v0)
    rmse = np.zeros((3, 3), dtype=np.float32)
    ctx.fr_reconstruct(fr.volume(v, case.origin, case.h), fr.cameras(case.cams), t_dev, bbox, 3,
                       fr.params(step=case.step, alpha_l=2e-3), albedo=dev(case.albedo), rmse=rmse)
    torch.cuda.synchronize()
    print("rmse gpu", rmse[:, 1], "ref", rmse_ref[:, 1])
    np.testing.assert_allclose(rmse, rmse_ref, rtol=1e-3)
    e = rel_err(v.cpu().numpy()[..., :3], vol_ref[..., :3])
    print(f"reconstruct with scattering: max {e.max():.3e}")
    assert e.max() < 1e-3
