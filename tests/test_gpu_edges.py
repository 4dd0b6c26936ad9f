"""Degenerate and extreme inputs through the C ABI, against the oracle where
there is something to compare: the smallest grid (2^3 nodes, one cell), one-
pixel images, the largest number of views (32), a step longer than the box,
cameras that see no part of the volume, targets without a flame pixel, and a
zero-iteration call."""
import numpy as np
import pytest

from gpu_cases import Case, rel_err

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


def _render_both(orc, fr, ctx, case):
    sc = orc.Scene(case.shape, case.origin, case.h, case.cams)
    ref, n_ref = orc.render(sc, case.vol, orc.make_params(step=case.step))
    v = torch.as_tensor(case.vol, dtype=torch.float32, device="cuda").contiguous()
    K, H, W = len(case.cams), case.cams[0]["height"], case.cams[0]["width"]
    out = torch.full((K, H, W, 3), -1.0, device="cuda")
    p = fr.params(step=case.step)
    fv = fr.volume(v, case.origin, case.h)
    ctx.fr_render(fv, fr.cameras(case.cams), p, out)
    n = ctx.fr_count_samples(fv, fr.cameras(case.cams), fr.params(step=case.step, skip_empty=0))
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64), ref, n, n_ref


def _close(got, ref):
    err = np.abs(got - ref)
    assert np.all(err <= 1e-4 * np.abs(ref) + 1e-6 * max(np.abs(ref).max(), 1e-30))


def test_smallest_grid(orc, fr_ctx):
    fr, ctx = fr_ctx
    from paper_1809_06417_gb300 import synth
    rng = np.random.default_rng(1)
    vol = rng.random((2, 2, 2, 4)) * np.array([1.0, 0.5, 0.2, 0.8])
    case = Case((2, 2, 2), synth.ring_cameras(3, 17, 9, elevation_jitter_deg=20, seed=1), vol, 0.3)
    got, ref, n, n_ref = _render_both(orc, fr, ctx, case)
    assert n == n_ref and n > 0
    _close(got, ref)


def test_one_pixel_images_and_32_views(orc, fr_ctx):
    fr, ctx = fr_ctx
    from paper_1809_06417_gb300 import synth
    vol = synth.blobs_volume(12, 4)
    case = Case((12, 12, 12), synth.ring_cameras(32, 1, 1, elevation_jitter_deg=30, seed=4), vol, 0.5)
    got, ref, n, n_ref = _render_both(orc, fr, ctx, case)
    assert n == n_ref and got.shape == (32, 1, 1, 3)
    _close(got, ref)
    assert np.all(ref[..., 0] > 0)                   # every pixel looks at the centre


def test_step_longer_than_the_box(orc, fr_ctx):
    fr, ctx = fr_ctx
    from paper_1809_06417_gb300 import synth
    vol = synth.blobs_volume(10, 5)
    case = Case((10, 10, 10), synth.ring_cameras(3, 16, 16, seed=5), vol, 40.0)
    got, ref, n, n_ref = _render_both(orc, fr, ctx, case)
    assert n == n_ref
    _close(got, ref)


def test_cameras_that_see_nothing(fr_ctx):
    fr, ctx = fr_ctx
    from paper_1809_06417_gb300 import synth
    cams = synth.ring_cameras(2, 24, 24)
    for c in cams:                                    # look straight away from the volume
        c["fwd"] = [-x for x in c["fwd"]]
        c["right"] = [-x for x in c["right"]]
    shape, origin, h = synth.unit_grid(16)
    v = torch.as_tensor(synth.blobs_volume(16, 2), dtype=torch.float32, device="cuda").contiguous()
    out = torch.full((2, 24, 24, 3), -1.0, device="cuda")
    fv = fr.volume(v, origin, h)
    ctx.fr_render(fv, fr.cameras(cams), fr.params(step=0.5), out)
    assert float(out.abs().max()) == 0.0
    assert ctx.fr_count_samples(fv, fr.cameras(cams), fr.params(step=0.5, skip_empty=0)) == 0


def test_targets_without_flame_and_zero_iterations(fr_ctx):
    fr, ctx = fr_ctx
    from paper_1809_06417_gb300 import synth
    shape, origin, h = synth.unit_grid(20)
    cams = synth.ring_cameras(3, 32, 32, seed=3)
    v0 = torch.as_tensor(synth.blobs_volume(20, 3), dtype=torch.float32, device="cuda").contiguous()
    targets = torch.zeros((3, 32, 32, 3), device="cuda")
    bbox = torch.zeros((3, 4), dtype=torch.int32, device="cuda")
    ctx.fr_prepare_targets(targets, 30 / 255, bbox)
    b = bbox.cpu().numpy()
    assert np.all(b[:, 0] > b[:, 2])                  # empty boxes
    v = v0.clone()
    rmse = np.full((3, 3), -1.0, dtype=np.float32)
    fv = fr.volume(v, origin, h)
    ctx.fr_reconstruct(fv, fr.cameras(cams), targets, bbox, 3, fr.params(step=0.5, alpha_l=1e-2), rmse=rmse)
    torch.cuda.synchronize()
    assert torch.equal(v, v0)                         # no flame ray, no adjustment
    assert np.all(rmse == 0.0)                        # no pixel in any box
    n = ctx.fr_reconstruct_until(fv, fr.cameras(cams), targets, bbox, 6, 0.01, fr.params(step=0.5), rmse=rmse)
    assert n == 2
    ctx.fr_reconstruct(fv, fr.cameras(cams), targets, bbox, 0, fr.params(step=0.5))
    torch.cuda.synchronize()
    assert torch.equal(v, v0)
