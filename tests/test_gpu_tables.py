"""The ray weight tables of fr_reconstruct (fr_params.tables): with the
extinction fixed and G(s) = 1, rendering (Eqs. 5-8) and the paper rule's
adjustment (Eq. 10) are linear maps whose weights do not change between
iterations, so the loop can build them once per call and stream them.

* Loops on the tables against the FP64 oracle (hull-restricted, with and
  without in-scattering; 16-bit storage against the 16-bit oracle; an empty
  hull and a hull at the grid's upper corner).
* The tables against the marches at the benchmarked size over ten
  iterations, and under the stop criterion.
* The tables' phases in the trace, and the marches taking over when the
  tables would pass the context's scratch limit.
"""
import numpy as np
import pytest

from gpu_cases import oracle_targets, plume_case, rel_err, tags_on_device, tiny_case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TORCH_DT = {"f32": "float32", "bf16": "bfloat16", "f16": "float16"}


@pytest.fixture(scope="module")
def fr_ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_06417_gb300 import flamerec as fr
    ctx = fr.Context(0)
    yield fr, ctx
    torch.cuda.synchronize()
    ctx.close()


def _device_targets(ctx, img, views):
    t_dev = torch.as_tensor(img, dtype=torch.float32, device="cuda").contiguous()
    bbox = torch.zeros((views, 4), dtype=torch.int32, device="cuda")
    ctx.fr_prepare_targets(t_dev, 30 / 255, bbox)
    return t_dev, bbox


@pytest.mark.parametrize("scatter", [False, True])
def test_tables_loop_follows_oracle(orc, fr_ctx, scatter):
    """Six iterations on the tables against the oracle on its hull tags."""
    fr, ctx = fr_ctx
    case = plume_case(n=36, views=6, side=64)
    P = orc.make_params(step=case.step, alpha_l=3e-3)
    sc, img, t_ref, mask, bbox_ref = oracle_targets(orc, case)
    hull = orc.visual_hull(sc, mask)
    v0 = case.vol.copy()
    v0[..., :3] = 0.01
    alb_np = case.albedo if scatter else None
    iters = 6
    vol_ref, rmse_ref, _ = orc.reconstruct(sc, v0, P, t_ref, mask, bbox_ref, iters, hull=hull, albedo=alb_np)
    t_dev, bbox = _device_targets(ctx, img, len(case.cams))
    v = torch.as_tensor(v0, dtype=torch.float32, device="cuda").contiguous()
    rmse = np.zeros((iters, 3), dtype=np.float32)
    alb = torch.as_tensor(case.albedo, dtype=torch.float32, device="cuda").contiguous() if scatter else None
    ctx.fr_reconstruct(fr.volume(v, case.origin, case.h), fr.cameras(case.cams), t_dev, bbox, iters,
                       fr.params(step=case.step, alpha_l=3e-3, use_hull=1, hull_tags=tags_on_device(torch, hull),
                                 tables=2),
                       albedo=alb, rmse=rmse)
    torch.cuda.synchronize()
    got = v.cpu().numpy()
    outside = hull != (1 << len(case.cams)) - 1
    assert np.all(got[outside] == 0.0)
    assert np.array_equal(got[~outside][:, 3], v0[~outside][:, 3].astype(np.float32))
    np.testing.assert_allclose(rmse, rmse_ref, rtol=1e-3)
    e = rel_err(got[..., :3], vol_ref[..., :3])
    print(f"tables loop (scatter={scatter}): max {e.max():.3e}; rmse {rmse[-1]} oracle {rmse_ref[-1]}")
    assert e.max() < 1e-3


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_tables_16bit_loop_follows_16bit_oracle(orc, fr_ctx, storage):
    """Ten iterations of the tiny configuration in its visual hull with 16-bit
    records on the tables, against the oracle keeping 16-bit records, at the
    storage tolerance (1e-2 of the maximum); the storage error against FP64
    records is printed beside it."""
    fr, ctx = fr_ctx
    case = tiny_case()
    alpha, iters = 0.01, 10
    sc, img, t_ref, mask, bbox_ref = oracle_targets(orc, case, noise=1e-3)
    hull = orc.visual_hull(sc, mask)
    v0 = case.vol.copy()
    v0[..., :3] = 0.0
    v0 = orc.round_storage(v0, storage)
    P16 = orc.make_params(step=case.step, alpha_l=alpha, storage=storage)
    P64 = orc.make_params(step=case.step, alpha_l=alpha)
    ref16, r16, _ = orc.reconstruct(sc, v0, P16, t_ref, mask, bbox_ref, iters, hull=hull)
    ref64, _, _ = orc.reconstruct(sc, v0, P64, t_ref, mask, bbox_ref, iters, hull=hull)
    v = torch.as_tensor(v0, dtype=torch.float32, device="cuda").to(getattr(torch, TORCH_DT[storage])).contiguous()
    t_dev, bbox = _device_targets(ctx, img, len(case.cams))
    rmse = np.zeros((iters, 3), dtype=np.float32)
    ctx.fr_reconstruct(fr.volume(v, case.origin, case.h), fr.cameras(case.cams), t_dev, bbox, iters,
                       fr.params(step=case.step, alpha_l=alpha, use_hull=1, hull_tags=tags_on_device(torch, hull),
                                 tables=2), rmse=rmse)
    torch.cuda.synchronize()
    got = v.float().cpu().numpy().astype(np.float64)
    e16 = rel_err(got[..., :3], ref16[..., :3])
    e64 = rel_err(got[..., :3], ref64[..., :3])
    print(f"tables {storage}: volume vs 16-bit oracle max {e16.max():.2e}; vs FP64 records {e64.max():.2e}")
    assert e16.max() < 1e-2
    np.testing.assert_allclose(rmse, r16, rtol=1e-2)
    inside = hull == (1 << len(case.cams)) - 1
    assert np.array_equal(got[inside][:, 3], v0[inside][:, 3])      # extinction untouched in the hull
    assert np.all(got[~inside] == 0.0)


@pytest.mark.parametrize("shape", ["empty", "corner"])
def test_tables_degenerate_hull_follows_oracle(orc, fr_ctx, shape):
    """No key point inside the hull (empty tables: every ray renders black and
    nothing is adjusted) and a 3^3 block at the grid's upper corner."""
    fr, ctx = fr_ctx
    case = plume_case(n=36, views=6, side=64)
    n = case.vol.shape[0]
    P = orc.make_params(step=case.step, alpha_l=3e-3)
    sc, img, t_ref, mask, bbox_ref = oracle_targets(orc, case)
    full = (1 << len(case.cams)) - 1
    hull = np.zeros(case.vol.shape[:3], dtype=np.uint32)
    if shape == "corner":
        hull[n - 3:, n - 3:, n - 3:] = full
    v0 = case.vol.copy()
    v0[..., :3] = 0.01
    vol_ref, rmse_ref, _ = orc.reconstruct(sc, v0, P, t_ref, mask, bbox_ref, 4, hull=hull, albedo=case.albedo)
    t_dev, bbox = _device_targets(ctx, img, len(case.cams))
    v = torch.as_tensor(v0, dtype=torch.float32, device="cuda").contiguous()
    rmse = np.zeros((4, 3), dtype=np.float32)
    alb = torch.as_tensor(case.albedo, dtype=torch.float32, device="cuda").contiguous()
    ctx.fr_reconstruct(fr.volume(v, case.origin, case.h), fr.cameras(case.cams), t_dev, bbox, 4,
                       fr.params(step=case.step, alpha_l=3e-3, use_hull=1, hull_tags=tags_on_device(torch, hull),
                                 tables=2), albedo=alb, rmse=rmse)
    torch.cuda.synchronize()
    got = v.cpu().numpy()
    assert np.all(got[hull != full] == 0.0)
    np.testing.assert_allclose(rmse, rmse_ref, rtol=1e-3)
    e = rel_err(got[..., :3], vol_ref[..., :3])
    assert e.max() < 1e-3


def _plume_setup(fr, ctx, n=128, views=8, side=512, seed=2):
    from paper_1809_06417_gb300 import synth
    case = plume_case(n=n, views=views, side=side, seed=seed)
    g = torch.as_tensor(case.vol, dtype=torch.float32, device="cuda").contiguous()
    alb = torch.as_tensor(case.albedo, dtype=torch.float32, device="cuda").contiguous()
    fc = fr.cameras(case.cams)
    src = torch.empty_like(g)
    J = torch.empty_like(g)
    ctx.fr_scatter_source(fr.volume(g, case.origin, case.h), alb, J, fr.volume(src, case.origin, case.h))
    img = torch.zeros((views, side, side, 3), device="cuda")
    ctx.fr_render(fr.volume(src, case.origin, case.h), fc, fr.params(step=case.step), img)
    img /= img.max()
    img = torch.as_tensor(synth.add_noise(img.cpu().numpy(), 1e-3, seed), dtype=torch.float32,
                          device="cuda").contiguous()
    bbox = torch.zeros((views, 4), dtype=torch.int32, device="cuda")
    ctx.fr_prepare_targets(img, 30 / 255, bbox)
    tags = torch.zeros(g.shape[:3], dtype=torch.int32, device="cuda")
    ctx.fr_visual_hull(fr.volume(g, case.origin, case.h), fc, img, fr.params(), tags)
    v0 = g.clone()
    v0[..., :3] = 0.0
    return case, fc, img, bbox, tags, alb, v0


def test_tables_follow_the_marches_at_full_size(fr_ctx):
    """Ten iterations of the benchmarked setting (128^3, 8 x 512^2, step 0.5,
    in-scattering, hull, skipping) from the zero start, on the tables and
    marching: the same per-iteration errors and volume up to float32 rounding
    (the tables sum each key point's and each ray's terms in another order)."""
    fr, ctx = fr_ctx
    case, fc, img, bbox, tags, alb, v0 = _plume_setup(fr, ctx)
    out = []
    for tables in (1, 2):
        v = v0.clone()
        rmse = np.zeros((10, 3), dtype=np.float32)
        p = fr.params(step=case.step, alpha_l=2e-4, use_hull=1, hull_tags=tags, tables=tables)
        ctx.fr_reconstruct(fr.volume(v, case.origin, case.h), fc, img, bbox, 10, p, albedo=alb, rmse=rmse)
        torch.cuda.synchronize()
        out.append((v.cpu().numpy(), rmse))
    (a, ra), (b, rb) = out
    e = rel_err(b[..., :3], a[..., :3].astype(np.float64))
    print(f"tables against marches, 10 iterations: volume max {e.max():.2e}; rmse {rb[-1]} against {ra[-1]}")
    assert e.max() < 1e-4
    np.testing.assert_allclose(rb, ra, rtol=1e-4)
    outside = tags.cpu().numpy().view(np.uint32) != (1 << len(case.cams)) - 1
    assert np.all(b[outside] == 0.0)


def test_tables_under_the_stop_criterion(fr_ctx):
    """fr_reconstruct_until on the tables (the graph body streams them) stops
    where the marching loop does, with the same errors and volume."""
    fr, ctx = fr_ctx
    case, fc, img, bbox, tags, alb, v0 = _plume_setup(fr, ctx, n=64, views=6, side=160)
    out = []
    for tables in (1, 2):
        v = v0.clone()
        rmse = np.zeros((40, 3), dtype=np.float32)
        p = fr.params(step=case.step, alpha_l=2e-3, use_hull=1, hull_tags=tags, tables=tables)
        n = ctx.fr_reconstruct_until(fr.volume(v, case.origin, case.h), fc, img, bbox, 40, 0.05, p, albedo=alb,
                                     rmse=rmse)
        torch.cuda.synchronize()
        out.append((v.cpu().numpy(), rmse[:n], n))
    (a, ra, na), (b, rb, nb) = out
    print(f"stop criterion: marches {na} iterations, tables {nb}")
    assert na >= 2 and nb == na
    np.testing.assert_allclose(rb, ra, rtol=1e-4)
    assert np.max(rel_err(b[..., :3], a[..., :3].astype(np.float64))) < 1e-4


def test_tables_trace_and_scratch_limit(fr_ctx):
    """The tables' iterations trace as scatter / forward / adjust (the error
    sums and the update run inside the adjustment's launch, no pack); with a scratch limit that
    leaves no room for the tables the same call marches instead, allocates
    nothing more and gives the same result."""
    fr, ctx0 = fr_ctx
    ctx = fr.Context(0)
    try:
        case, fc, img, bbox, tags, alb, v0 = _plume_setup(fr, ctx, n=64, views=6, side=128)
        p = fr.params(step=case.step, alpha_l=2e-3, use_hull=1, hull_tags=tags, tables=2)
        pm = fr.params(step=case.step, alpha_l=2e-3, use_hull=1, hull_tags=tags, tables=1)
        vm = v0.clone()
        rm = np.zeros((4, 3), dtype=np.float32)
        ctx.fr_reconstruct(fr.volume(vm, case.origin, case.h), fc, img, bbox, 4, pm, albedo=alb, rmse=rm)
        torch.cuda.synchronize()
        held = ctx.fr_scratch_bytes()
        ctx.fr_set_scratch_limit(held + 4096)
        vl = v0.clone()
        rl = np.zeros((4, 3), dtype=np.float32)
        ctx.fr_reconstruct(fr.volume(vl, case.origin, case.h), fc, img, bbox, 4, p, albedo=alb, rmse=rl)
        torch.cuda.synchronize()
        assert ctx.fr_scratch_bytes() <= held + 4096
        assert all(v == 0 for v in ctx.fr_table_stats().values())   # the call marched
        np.testing.assert_allclose(rl, rm, rtol=1e-5)
        assert np.max(rel_err(vl.cpu().numpy(), vm.cpu().numpy().astype(np.float64))) < 1e-5
        ctx.fr_set_scratch_limit(0)
        ctx.fr_trace_phases(True)
        vt = v0.clone()
        rt = np.zeros((4, 3), dtype=np.float32)
        ctx.fr_reconstruct(fr.volume(vt, case.origin, case.h), fc, img, bbox, 4, p, albedo=alb, rmse=rt)
        torch.cuda.synchronize()
        ms, calls = ctx.fr_phase_times()
        ctx.fr_trace_phases(False)
        print({k: round(x, 4) for k, x in ms.items()})
        assert calls == 1 and ctx.fr_scratch_bytes() > held
        st = ctx.fr_table_stats()
        print(st)
        assert st["forward_entries"] % 32 == 0 and st["forward_entries"] >= st["adjustment_entries"] > 0
        assert 0 < st["flame_rays"] and 0 < st["hull_key_points"]
        for k in ("setup", "scatter", "forward", "adjust"):
            assert ms[k] > 0.0, k
        assert ms["pack"] == 0.0 and ms["apply"] == 0.0 and ms["reduce"] == 0.0
        np.testing.assert_allclose(rt, rm, rtol=1e-4)
        assert np.max(rel_err(vt.cpu().numpy(), vm.cpu().numpy().astype(np.float64))) < 1e-4
    finally:
        torch.cuda.synchronize()
        ctx.close()
