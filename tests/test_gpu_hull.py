"""Visual hull (Sec. 4.3.1, Algorithm 1) on the GPU against the FP64 oracle.

The kernel projects in float32, the oracle in double precision.  Whether a
pixel centre lies inside a node's rectangle is an integer decision, so the two
agree exactly on every tag bit that the oracle reports as decided (no
rectangle edge within 1e-3 pixel of a pixel centre whose flame decides the
bit); the undecided bits are counted and bounded, and the GPU's bit there must
be one of the two answers.  The reconstruction loop restricted to the hull is
compared with the oracle on one tag set (the oracle's, passed to both)."""
import os

import numpy as np
import pytest

from gpu_cases import oracle_targets, plume_case, rel_err, tags_on_device

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


def _gpu_tags(fr, ctx, shape, origin, h, cams, targets, thresh):
    nx, ny, nz = shape
    vol = torch.zeros((nz, ny, nx, 4), device="cuda")
    tags = torch.zeros((nz, ny, nx), dtype=torch.int32, device="cuda")
    t = torch.as_tensor(np.ascontiguousarray(targets), dtype=torch.float32, device="cuda")
    ctx.fr_visual_hull(fr.volume(vol, origin, h), fr.cameras(cams), t, fr.params(flame_thresh=thresh), tags)
    torch.cuda.synchronize()
    return tags.cpu().numpy().view(np.uint32)


def _compare_tags(got, ref, undecided, what):
    """Exact on decided bits; on undecided bits the GPU's answer is free."""
    wrong = (got ^ ref) & ~undecided
    n_und = int(np.count_nonzero(undecided))
    n_diff = int(np.count_nonzero((got ^ ref) & undecided))
    print(f"{what}: {n_und} of {got.size} nodes with undecided bits ({n_und / got.size:.2e}), "
          f"{n_diff} of them answered the other way")
    assert not np.any(wrong), np.argwhere(wrong)[:5]
    return n_und


@pytest.mark.parametrize("seed", [0, 1])
def test_hull_tags_match_oracle_random_masks(orc, fr_ctx, seed):
    """Random masks seen by 7 cameras with odd image widths: the volume's
    centre node projects exactly onto a pixel centre in every view, so this
    case holds exact ties (undecided by construction)."""
    fr, ctx = fr_ctx
    from paper_1809_06417_gb300 import synth
    rng = np.random.default_rng(seed)
    shape = (19, 23, 17)
    h = 1.0 / 22
    origin = tuple(-0.5 * (s - 1) * h for s in shape)
    cams = synth.ring_cameras(7, 45, 38, elevation_jitter_deg=20.0, seed=seed)
    targets = rng.random((7, 38, 45, 3)) * (rng.random((7, 38, 45, 1)) < 0.2)
    thresh = 0.3
    mask = (targets.max(axis=-1) > thresh).astype(np.uint8)
    ref, und = orc.visual_hull(orc.Scene(shape, origin, h, cams), mask, with_undecided=True)
    got = _gpu_tags(fr, ctx, shape, origin, h, cams, targets.astype(np.float32), thresh)
    n_und = _compare_tags(got, ref, und, f"random masks seed {seed}")
    assert n_und < 0.06 * got.size


def test_hull_tags_match_oracle_full_size(orc, fr_ctx):
    """128^3 nodes, 8 views of 512^2: masks from the oracle's render of the
    full-RTE plume; at most 1e-3 of the nodes hold an undecided bit."""
    fr, ctx = fr_ctx
    from paper_1809_06417_gb300 import synth
    orc.set_threads(os.cpu_count() or 1)
    n, views, side = 128, 8, 512
    shape, origin, h = synth.unit_grid(n)
    cams = synth.ring_cameras(views, side, side, elevation_jitter_deg=10.0, seed=2)
    gt, _ = synth.plume_volume(n, 2)
    sc = orc.Scene(shape, origin, h, cams)
    img, _ = orc.render(sc, gt, orc.make_params(step=0.5))
    targets = img / img.max()
    thresh = 30 / 255
    mask = (targets.max(axis=-1) > thresh).astype(np.uint8)
    ref, und = orc.visual_hull(sc, mask, with_undecided=True)
    got = _gpu_tags(fr, ctx, shape, origin, h, cams, targets, thresh)
    n_und = _compare_tags(got, ref, und, "full size")
    assert n_und < 1e-3 * got.size
    inside = (got == (1 << views) - 1).mean()
    print(f"hull fraction of the volume: {inside:.3f}")
    assert 0.01 < inside < 0.6


@pytest.mark.parametrize("tables", [1, 0], ids=["march", "auto"])
@pytest.mark.parametrize("scatter", [False, True])
def test_reconstruct_with_hull_follows_oracle(orc, fr_ctx, scatter, tables):
    """The hull-restricted loop follows the oracle on the oracle's tags; with
    in-scattering its sweeps also skip the loads of line chunks in bricks
    outside the hull."""
    fr, ctx = fr_ctx
    case = plume_case(n=36, views=6, side=64)
    P = orc.make_params(step=case.step, alpha_l=3e-3)
    sc, img, t_ref, mask, bbox_ref = oracle_targets(orc, case)
    hull = orc.visual_hull(sc, mask)
    v0 = case.vol.copy()
    v0[..., :3] = 0.01
    alb_np = case.albedo if scatter else None
    vol_ref, rmse_ref, _ = orc.reconstruct(sc, v0, P, t_ref, mask, bbox_ref, 4, hull=hull, albedo=alb_np)
    t_dev = torch.as_tensor(img, dtype=torch.float32, device="cuda").contiguous()
    bbox = torch.zeros((len(case.cams), 4), dtype=torch.int32, device="cuda")
    ctx.fr_prepare_targets(t_dev, 30 / 255, bbox)
    v = torch.as_tensor(v0, dtype=torch.float32, device="cuda").contiguous()
    rmse = np.zeros((4, 3), dtype=np.float32)
    alb = torch.as_tensor(case.albedo, dtype=torch.float32, device="cuda").contiguous() if scatter else None
    ctx.fr_reconstruct(fr.volume(v, case.origin, case.h), fr.cameras(case.cams), t_dev, bbox, 4,
                       fr.params(step=case.step, alpha_l=3e-3, use_hull=1, hull_tags=tags_on_device(torch, hull),
                                 tables=tables),
                       albedo=alb, rmse=rmse)
    torch.cuda.synchronize()
    got = v.cpu().numpy()
    outside = hull != (1 << len(case.cams)) - 1
    assert np.all(got[outside] == 0.0)                       # no flame outside the hull
    assert np.array_equal(got[~outside][:, 3], v0[~outside][:, 3].astype(np.float32))
    np.testing.assert_allclose(rmse, rmse_ref, rtol=1e-3)
    e = rel_err(got[..., :3], vol_ref[..., :3])
    print(f"reconstruct with hull (scatter={scatter}, tables={tables}): max {e.max():.3e}, outside fraction {outside.mean():.3f}")
    assert e.max() < 1e-3


def test_reconstruct_with_precomputed_tags_is_identical(fr_ctx):
    """Tags passed in (from fr_visual_hull) give the same iterations as tags
    fr_reconstruct computes itself (up to the order of the adjustment's
    atomic sums, which differs from run to run)."""
    fr, ctx = fr_ctx
    case = plume_case(n=40, views=5, side=72)
    img = torch.zeros((5, 72, 72, 3), device="cuda")
    g = torch.as_tensor(case.vol, dtype=torch.float32, device="cuda").contiguous()
    fc = fr.cameras(case.cams)
    ctx.fr_render(fr.volume(g, case.origin, case.h), fc, fr.params(step=case.step), img)
    img /= img.max()
    bbox = torch.zeros((5, 4), dtype=torch.int32, device="cuda")
    ctx.fr_prepare_targets(img, 30 / 255, bbox)
    tags = torch.zeros(g.shape[:3], dtype=torch.int32, device="cuda")
    ctx.fr_visual_hull(fr.volume(g, case.origin, case.h), fc, img, fr.params(), tags)
    out = []
    for pre in (None, tags):
        v = g.clone()
        v[..., :3] = 0.01
        rmse = np.zeros((3, 3), dtype=np.float32)
        ctx.fr_reconstruct(fr.volume(v, case.origin, case.h), fc, img, bbox, 3,
                           fr.params(step=case.step, alpha_l=3e-3, use_hull=1, hull_tags=pre), rmse=rmse)
        torch.cuda.synchronize()
        out.append((v, rmse))
    a, b = (o[0].cpu().numpy() for o in out)
    assert np.array_equal(a == 0, b == 0)
    assert np.max(rel_err(a, b)) < 1e-5
    np.testing.assert_allclose(out[0][1], out[1][1], rtol=1e-5)


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_volume_rmse_follows_oracle(orc, fr_ctx, dtype):
    """Volume data error in the hull (Sec. 5.1): GPU against the oracle fed the
    same (rounded) records, with random tags, with no tags, and at full size."""
    fr, ctx = fr_ctx
    rng = np.random.default_rng(11)
    for shape in ((13, 17, 11), (128, 128, 128)):
        a = rng.random(shape[::-1] + (4,)).astype(np.float32)
        b = (a + rng.normal(scale=0.1, size=a.shape)).astype(np.float32)
        tags = rng.integers(0, 4, size=shape[::-1]).astype(np.uint32)
        ta = torch.as_tensor(a, device="cuda").to(dtype).contiguous()
        tb = torch.as_tensor(b, device="cuda").to(dtype).contiguous()
        ra, rb = ta.float().cpu().numpy(), tb.float().cpu().numpy()
        tt = torch.as_tensor(tags.view(np.int32), device="cuda")
        h = 1.0 / (max(shape) - 1)
        origin = tuple(-0.5 * (n - 1) * h for n in shape)
        va, vb = fr.volume(ta, origin, h), fr.volume(tb, origin, h)
        for tg, full in ((tt, 3), (None, 0)):
            got, n = ctx.fr_volume_rmse(va, vb, tg, full)
            ref, n_ref = orc.volume_rmse(ra, rb, tags if tg is not None else None, full)
            assert n == n_ref
            np.testing.assert_allclose(got, ref, rtol=1e-5)
    # no key point compared
    got, n = ctx.fr_volume_rmse(va, vb, torch.zeros_like(tt), 3)
    assert n == 0 and np.all(got == 0.0)


@pytest.mark.parametrize("shape", ["empty", "corner"])
def test_reconstruct_with_degenerate_hull_follows_oracle(orc, fr_ctx, shape):
    """Hulls at the edges of the box logic: no key point at all (the hull's box
    is empty: the sweeps, the pack and the update have no node to cover and
    the marches no sample) and a 3^3 block of key points at the grid's upper
    corner (the box reaches the last node on every axis), with in-scattering,
    against the oracle on the same tags."""
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
    vol_ref, rmse_ref, _ = orc.reconstruct(sc, v0, P, t_ref, mask, bbox_ref, 3, hull=hull, albedo=case.albedo)
    t_dev = torch.as_tensor(img, dtype=torch.float32, device="cuda").contiguous()
    bbox = torch.zeros((len(case.cams), 4), dtype=torch.int32, device="cuda")
    ctx.fr_prepare_targets(t_dev, 30 / 255, bbox)
    v = torch.as_tensor(v0, dtype=torch.float32, device="cuda").contiguous()
    rmse = np.zeros((3, 3), dtype=np.float32)
    alb = torch.as_tensor(case.albedo, dtype=torch.float32, device="cuda").contiguous()
    ctx.fr_reconstruct(fr.volume(v, case.origin, case.h), fr.cameras(case.cams), t_dev, bbox, 3,
                       fr.params(step=case.step, alpha_l=3e-3, use_hull=1, hull_tags=tags_on_device(torch, hull)),
                       albedo=alb, rmse=rmse)
    torch.cuda.synchronize()
    got = v.cpu().numpy()
    outside = hull != full
    assert np.all(got[outside] == 0.0)
    np.testing.assert_allclose(rmse, rmse_ref, rtol=1e-3)
    if shape == "corner":
        e = rel_err(got[..., :3], vol_ref[..., :3])
        print(f"corner hull: max {e.max():.3e}, key points {int((~outside).sum())}")
        assert e.max() < 1e-3
