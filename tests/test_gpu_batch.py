"""Batched reconstruction (independent problems such as video frames, one
launch per phase for all of them): each problem's result equals the one it
gets when reconstructed alone, with and without CUDA-graph capture."""
import numpy as np
import pytest

from gpu_cases import rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _problem(fr, ctx, synth, n, views, side, seed, step=0.5):
    shape, origin, h = synth.unit_grid(n)
    cams = synth.ring_cameras(views, side, side, elevation_jitter_deg=8.0, seed=seed)
    gt, _ = synth.plume_volume(n, seed)
    gt_d = torch.as_tensor(gt, dtype=torch.float32, device="cuda").contiguous()
    img = torch.zeros((views, side, side, 3), device="cuda")
    ctx.fr_render(fr.volume(gt_d, origin, h), fr.cameras(cams), fr.params(step=step), img)
    img /= img.max()
    bbox = torch.zeros((views, 4), dtype=torch.int32, device="cuda")
    ctx.fr_prepare_targets(img, 30 / 255, bbox)
    v0 = gt_d.clone()
    v0[..., :3] *= 0.2
    return dict(origin=origin, h=h, cams=cams, targets=img, bbox=bbox, v0=v0)


@pytest.mark.parametrize("use_graph,use_hull", [(False, 0), (True, 0), (True, 1)])
def test_batch_equals_each_problem_alone(use_graph, use_hull):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_06417_gb300 import flamerec as fr, synth
    ctx = fr.Context(0)
    specs = [(24, 3, 40, 11), (32, 5, 56, 12), (20, 4, 33, 13)]
    probs = [_problem(fr, ctx, synth, *s) for s in specs]
    iters, p = 4, fr.params(step=0.5, alpha_l=2e-3, g_std=0.05, seed=9, use_hull=use_hull)
    alone = []
    for q in probs:
        v = q["v0"].clone()
        rmse = np.zeros((iters, 3), dtype=np.float32)
        ctx.fr_reconstruct(fr.volume(v, q["origin"], q["h"]), fr.cameras(q["cams"]), q["targets"], q["bbox"],
                           iters, p, first_iteration=2, rmse=rmse)
        alone.append((v, rmse))
    vols = [q["v0"].clone() for q in probs]
    rmses = [torch.zeros((iters, 3), device="cuda") for _ in probs]
    batch = [(fr.volume(v, q["origin"], q["h"]), fr.cameras(q["cams"]), q["targets"], q["bbox"], r)
             for v, q, r in zip(vols, probs, rmses)]
    ctx.fr_reconstruct_batch(batch, iters, p, first_iteration=2, use_graph=use_graph)
    torch.cuda.synchronize()
    for (va, ra), vb, rb in zip(alone, vols, rmses):
        e = rel_err(vb.cpu().numpy()[..., :3], va.cpu().numpy()[..., :3].astype(np.float64))
        print(f"batch vs alone: volume {e.max():.2e}")
        assert e.max() < 1e-4
        np.testing.assert_allclose(rb.cpu().numpy(), ra, rtol=1e-4)
    ctx.close()


@pytest.mark.parametrize("use_hull", [0, 1])
def test_batch_follows_oracle(orc, use_hull):
    """Each problem of a batch (grids, views and image sizes differing; G(s)
    drawn; the iteration index starting at 2) against orc.reconstruct on the
    same targets, rendered by the oracle; with the hull, each problem carries
    the oracle's tags, so both sides use one tag set."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from gpu_cases import Case, oracle_targets, tags_on_device
    from paper_1809_06417_gb300 import flamerec as fr, synth
    ctx = fr.Context(0)
    specs = [(24, 3, 40, 11), (32, 5, 56, 12), (20, 4, 33, 13)]
    iters = 4
    P = orc.make_params(step=0.5, alpha_l=2e-3, g_std=0.05, seed=9)
    p = fr.params(step=0.5, alpha_l=2e-3, g_std=0.05, seed=9, use_hull=use_hull)
    refs, batch, keep = [], [], []
    for n, views, side, seed in specs:
        shape, origin, h = synth.unit_grid(n)
        cams = synth.ring_cameras(views, side, side, elevation_jitter_deg=8.0, seed=seed)
        case = Case(shape, cams, synth.plume_volume(n, seed)[0], 0.5)
        sc, img, t_ref, mask, bbox_ref = oracle_targets(orc, case)
        tags = orc.visual_hull(sc, mask) if use_hull else None
        v0 = case.vol.copy()
        v0[..., :3] *= 0.2
        refs.append(orc.reconstruct(sc, v0, P, t_ref, mask, bbox_ref, iters, first_iteration=2, hull=tags)[:2])
        v = torch.as_tensor(v0, dtype=torch.float32, device="cuda").contiguous()
        t_dev = torch.as_tensor(img, dtype=torch.float32, device="cuda").contiguous()
        bbox = torch.zeros((views, 4), dtype=torch.int32, device="cuda")
        ctx.fr_prepare_targets(t_dev, 30 / 255, bbox)
        rm = torch.zeros((iters, 3), device="cuda")
        tg = tags_on_device(torch, tags) if use_hull else None
        keep.append((v, rm, t_dev, bbox, tg))
        batch.append((fr.volume(v, origin, h), fr.cameras(cams), t_dev, bbox, rm, tg))
    ctx.fr_reconstruct_batch(batch, iters, p, first_iteration=2, use_graph=True)
    torch.cuda.synchronize()
    for (vol_ref, rmse_ref), (v, rm, *_) in zip(refs, keep):
        got = v.cpu().numpy().astype(np.float64)
        e = rel_err(got[..., :3], vol_ref[..., :3])
        print(f"batch vs oracle (hull={use_hull}): volume {e.max():.2e}, rmse {rm.cpu().numpy()[-1]} "
              f"vs {rmse_ref[-1]}")
        assert e.max() < 1e-3
        np.testing.assert_allclose(rm.cpu().numpy(), rmse_ref, rtol=1e-3)
    ctx.close()


@pytest.mark.parametrize("tables", [1, 2], ids=["march", "tables"])
def test_video_size_batch_follows_oracle(orc, tables):
    """Two frames of the video setting at full size (96^3, 8 views of 384^2,
    the plume advected between them), each in its own hull (the oracle's tags),
    two batched iterations captured in a CUDA graph, marching or on each
    frame's ray weight tables, against orc.reconstruct frame by frame; node by
    node within 1e-4 of the frame's maximum plus the oracle's undecided
    budget."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import os
    from gpu_cases import Case, oracle_targets, tags_on_device
    from paper_1809_06417_gb300 import flamerec as fr, synth
    orc.set_threads(os.cpu_count() or 1)
    ctx = fr.Context(0)
    n, views, side, step, iters = 96, 8, 384, 0.5, 2
    shape, origin, h = synth.unit_grid(n)
    cams = synth.ring_cameras(views, side, side, elevation_jitter_deg=10.0, seed=4)
    frames = synth.video_frames(8, n, 4)[3:5]
    alpha = 2e-4 * (n / 128.0) * (512.0 / side) ** 2
    P = orc.make_params(step=step, alpha_l=alpha)
    p = fr.params(step=step, alpha_l=alpha, use_hull=1, tables=tables)
    refs, batch, keep = [], [], []
    for gt in frames:
        case = Case(shape, cams, gt, step)
        sc, img, t_ref, mask, bbox_ref = oracle_targets(orc, case)
        tags = orc.visual_hull(sc, mask)
        v0 = gt.copy()
        v0[..., :3] = 0.0
        refs.append(orc.reconstruct(sc, v0, P, t_ref, mask, bbox_ref, iters, hull=tags, with_undecided=True))
        v = torch.as_tensor(v0, dtype=torch.float32, device="cuda").contiguous()
        t_dev = torch.as_tensor(img, dtype=torch.float32, device="cuda").contiguous()
        bbox = torch.zeros((views, 4), dtype=torch.int32, device="cuda")
        ctx.fr_prepare_targets(t_dev, 30 / 255, bbox)
        rm = torch.zeros((iters, 3), device="cuda")
        tg = tags_on_device(torch, tags)
        keep.append((v, rm, t_dev, bbox, tg))
        batch.append((fr.volume(v, origin, h), fr.cameras(cams), t_dev, bbox, rm, tg))
    ctx.fr_reconstruct_batch(batch, iters, p, use_graph=True)
    torch.cuda.synchronize()
    for (vol_ref, rmse_ref, _, und), (v, rm, *_) in zip(refs, keep):
        got = v.cpu().numpy().astype(np.float64)
        scale = np.abs(vol_ref[..., :3]).max()
        err = np.abs(got[..., :3] - vol_ref[..., :3]).max(axis=-1)
        bound = 1e-4 * scale + und
        print(f"video frame vs oracle (tables={tables}): max error / max {err.max() / scale:.2e}, worst error / bound "
              f"{np.max(err / bound):.3f}, rmse {rm.cpu().numpy()[-1]} vs {rmse_ref[-1]}")
        assert np.all(err <= bound)
        np.testing.assert_allclose(rm.cpu().numpy(), rmse_ref, rtol=1e-3)
    ctx.close()


@pytest.mark.parametrize("tables", [1, 2], ids=["march", "tables"])
def test_batch_with_an_empty_hull_follows_oracle(orc, tables):
    """A batch whose middle problem has no key point in its hull (its box is
    empty: the batched pack and update cover no node of it; its tables have no
    entry and no adjustment block) beside two with their hulls: each against
    orc.reconstruct on the same tags."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from gpu_cases import Case, oracle_targets, tags_on_device
    from paper_1809_06417_gb300 import flamerec as fr, synth
    ctx = fr.Context(0)
    specs = [(24, 3, 40, 11), (32, 5, 56, 12), (20, 4, 33, 13)]
    iters = 3
    P = orc.make_params(step=0.5, alpha_l=2e-3)
    p = fr.params(step=0.5, alpha_l=2e-3, use_hull=1, tables=tables)
    refs, batch, keep = [], [], []
    for i, (n, views, side, seed) in enumerate(specs):
        shape, origin, h = synth.unit_grid(n)
        cams = synth.ring_cameras(views, side, side, elevation_jitter_deg=8.0, seed=seed)
        case = Case(shape, cams, synth.plume_volume(n, seed)[0], 0.5)
        sc, img, t_ref, mask, bbox_ref = oracle_targets(orc, case)
        tags = orc.visual_hull(sc, mask)
        if i == 1:
            tags = np.zeros_like(tags)
        v0 = case.vol.copy()
        v0[..., :3] *= 0.2
        refs.append(orc.reconstruct(sc, v0, P, t_ref, mask, bbox_ref, iters, hull=tags)[:2])
        v = torch.as_tensor(v0, dtype=torch.float32, device="cuda").contiguous()
        t_dev = torch.as_tensor(img, dtype=torch.float32, device="cuda").contiguous()
        bbox = torch.zeros((views, 4), dtype=torch.int32, device="cuda")
        ctx.fr_prepare_targets(t_dev, 30 / 255, bbox)
        rm = torch.zeros((iters, 3), device="cuda")
        tg = tags_on_device(torch, tags)
        keep.append((v, rm, t_dev, bbox, tg))
        batch.append((fr.volume(v, origin, h), fr.cameras(cams), t_dev, bbox, rm, tg))
    ctx.fr_reconstruct_batch(batch, iters, p, use_graph=True)
    torch.cuda.synchronize()
    for i, ((vol_ref, rmse_ref), (v, rm, *_)) in enumerate(zip(refs, keep)):
        got = v.cpu().numpy().astype(np.float64)
        if i == 1:
            assert np.all(got == 0.0) and np.all(vol_ref == 0.0)
        else:
            assert rel_err(got[..., :3], vol_ref[..., :3]).max() < 1e-3
        np.testing.assert_allclose(rm.cpu().numpy(), rmse_ref, rtol=1e-3)
    ctx.close()
