"""The allocation-free rendering entry point, checked against the allocating one.

fr_render_residual_noalloc serves callers that cannot allocate device memory
while they render (a process whose device memory all belongs to its own pool,
a latency-critical loop that forbids cudaMalloc/cudaFree after start-up).  It
must give the same rendered image, residual and squared-error sums as
fr_render_residual, call after call, although its scratch is one fixed array
shared by all calls.  This file is collected last so that a stop-at-first-
failure run has already run every other test."""
import numpy as np
import pytest

from gpu_cases import ragged_case, rel_err, tiny_case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _targets(fr, ctx, fv, case, p, scale):
    """Targets from the CUDA render of the case's volume, prepared on the GPU."""
    K, W, H = len(case.cams), case.cams[0]["width"], case.cams[0]["height"]
    img = torch.zeros((K, H, W, 3), device="cuda")
    ctx.fr_render(fv, fr.cameras(case.cams), p, img)
    img = img * (scale / float(img.max()))
    bbox = torch.zeros((K, 4), dtype=torch.int32, device="cuda")
    ctx.fr_prepare_targets(img, 30 / 255, bbox)
    return img, bbox


def _both(fr, ctx, case, vol_scale, dtype=torch.float32, kind=None, extra=None):
    """Render with residual through both entry points on the same inputs (the
    volume's colour, or its temperature, scaled by vol_scale)."""
    kind = fr.FR_KIND_RGB if kind is None else kind
    p = fr.params(step=case.step, **(extra or {}))
    g = torch.as_tensor(case.vol, dtype=torch.float32, device="cuda").to(dtype).contiguous()
    targets, bbox = _targets(fr, ctx, fr.volume(g, case.origin, case.h, kind=kind), case, p, 1.0)
    vol = case.vol.copy()
    if kind == fr.FR_KIND_RGB:
        vol[..., :3] *= vol_scale
    else:
        vol[..., 0] *= vol_scale
    v = torch.as_tensor(vol, dtype=torch.float32, device="cuda").to(dtype).contiguous()
    fv = fr.volume(v, case.origin, case.h, kind=kind)
    cams = fr.cameras(case.cams)
    out = []
    for which in ("alloc", "noalloc"):
        ren = torch.full_like(targets, -7.0)
        res = torch.full_like(targets, -7.0)
        sq = torch.full((4,), -7.0, device="cuda")
        if which == "alloc":
            ctx.fr_render_residual(fv, cams, p, targets, bbox, ren, res, sq)
        else:
            fr.fr_render_residual_noalloc(0, torch.cuda.current_stream(), fv, cams, p, targets, bbox, ren, res, sq)
        torch.cuda.synchronize()
        out.append((ren.cpu().numpy().astype(np.float64), res.cpu().numpy().astype(np.float64),
                    sq.cpu().numpy().astype(np.float64)))
    return out


def _check(out):
    (ren_a, res_a, sq_a), (ren_b, res_b, sq_b) = out
    err = np.abs(ren_b - ren_a)
    assert np.all(err <= 1e-4 * np.abs(ren_a) + 1e-6 * np.abs(ren_a).max())
    assert np.max(rel_err(res_b, res_a)) < 1e-5
    assert sq_b[3] == sq_a[3] and sq_a[3] > 0
    np.testing.assert_allclose(sq_b[:3], sq_a[:3], rtol=1e-5)


def test_noalloc_matches_allocating_entry_point_on_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_06417_gb300 import flamerec as fr
    ctx = fr.Context(0)
    # two calls in a row: the second uses a smaller image (fewer tiles) and a
    # different volume, so stale partials of the first call would show up
    for case, scale in ((tiny_case(seed=2, jitter=6.0), 0.6), (ragged_case(), 0.8)):
        _check(_both(fr, ctx, case, scale))
    ctx.close()


def test_noalloc_16bit_records_and_temperature():
    """BF16 and FP16 records, constant-opacity mode, and temperature records
    mapped through the colour-temperature table, each twice in a row."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_06417_gb300 import flamerec as fr, synth
    ctx = fr.Context(0)
    for dt in (torch.bfloat16, torch.float16):
        _check(_both(fr, ctx, tiny_case(seed=3, jitter=4.0), 0.7, dtype=dt))
        _check(_both(fr, ctx, ragged_case(), 0.9, dtype=dt, extra=dict(tau=0.05)))
    lut = torch.zeros((1024, 4), device="cuda")
    ctx.fr_planck_lut(800.0, 2000.0, lut)
    case = tiny_case(n=24, views=3, side=40, step=0.5, jitter=7.0)
    case.vol = synth.temperature_volume(24, 3)
    for scale in (0.95, 0.9):
        _check(_both(fr, ctx, case, scale, kind=fr.FR_KIND_TEMP,
                     extra=dict(lut=lut, lut_t_min=800.0, lut_t_max=2000.0)))
    ctx.close()


def test_noalloc_rejects_images_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_06417_gb300 import flamerec as fr, synth
    case = tiny_case()
    v = _dev(case.vol)
    # 32 views of 1024 x 1024 need 32 * 64 * 128 tiles, beyond the fixed scratch
    cams = fr.cameras(synth.ring_cameras(32, 1024, 1024))
    with pytest.raises(fr.FrError, match="FR_EINVAL.*fixed scratch"):
        fr.fr_render_residual_noalloc(0, None, fr.volume(v, case.origin, case.h), cams, fr.params(step=1.0),
                                      None, None, None, None, None)
