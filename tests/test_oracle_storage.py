"""Pins for the oracle's 16-bit storage rounding and for its threaded loops.

Rounding (round_storage, the records of a loop in 16-bit storage): hand-worked
ties and spacings of bfloat16 (8 significant bits) and IEEE binary16 (11 bits,
subnormals below 2^-14), numpy's binary16 conversion of doubles, torch's
bfloat16 conversion of float32 values (a single rounding there), and a loop
whose kept records are all representable and stay within the rounding's reach
of the double-precision loop.

Threads (set_threads): pixels are independent, so renders are identical for
any thread count; the adjustment's per-thread sums are added in thread order,
which regroups the sums (FP64 rounding only)."""
import numpy as np
import pytest

from paper_1809_06417_gb300 import synth


def test_bf16_ties_and_spacing(orc):
    x = np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 1 + 2 ** -8 + 2 ** -30, 0.75, 2.0 ** -100,
                  3.0 * 2 ** 40, 0.0, 255.0, 257.0])
    want = np.array([1.0, 1 + 2 ** -6, -1.0, 1 + 2 ** -7, 0.75, 2.0 ** -100, 3.0 * 2 ** 40, 0.0, 255.0, 256.0])
    np.testing.assert_array_equal(orc.round_storage(x, "bf16"), want)


def test_f16_ties_spacing_and_subnormals(orc):
    q = 2.0 ** -24                                 # spacing below the smallest normal, 2^-14
    x = np.array([1 + 2 ** -11, 1 + 3 * 2 ** -11, 2049.0, 2051.0, 3.5 * q, 2.5 * q, 0.4 * q, 2 ** -14 + 0.5 * q])
    want = np.array([1.0, 1 + 2 ** -9, 2048.0, 2052.0, 4 * q, 2 * q, 0.0, 2 ** -14])
    np.testing.assert_array_equal(orc.round_storage(x, "f16"), want)


def test_rounding_agrees_with_library_conversions(orc):
    rng = np.random.default_rng(0)
    x = rng.normal(size=20000) * np.exp(rng.uniform(-30, 10, size=20000))
    # numpy converts a double to binary16 with one correct rounding
    np.testing.assert_array_equal(orc.round_storage(x, "f16"), x.astype(np.float16).astype(np.float64))
    torch = pytest.importorskip("torch")
    x32 = x.astype(np.float32).astype(np.float64)   # float32 values: torch rounds them to bf16 once
    got = orc.round_storage(x32, "bf16")
    ref = torch.from_numpy(x32.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("storage,ulp", [("bf16", 2.0 ** -8), ("f16", 2.0 ** -11)])
def test_loop_in_16bit_storage_keeps_representable_records(orc, storage, ulp):
    n, views, side = 12, 4, 24
    shape, origin, h = synth.unit_grid(n)
    cams = synth.ring_cameras(views, side, side, elevation_jitter_deg=10.0, seed=3)
    gt, alb = synth.plume_volume(n, 3)
    sc = orc.Scene(shape, origin, h, cams)
    P = orc.make_params(step=0.5, alpha_l=5e-3)
    img, _ = orc.render(sc, gt, P)
    targets, mask, bbox = orc.prepare_targets(img / img.max(), 30 / 255)
    v0 = orc.round_storage(gt * np.array([0.0, 0.0, 0.0, 1.0]), storage)
    P16 = orc.make_params(step=0.5, alpha_l=5e-3, storage=storage)
    a, ra, _ = orc.reconstruct(sc, v0, P16, targets, mask, bbox, 4, albedo=alb)
    b, rb, _ = orc.reconstruct(sc, v0, P, targets, mask, bbox, 4, albedo=alb)
    np.testing.assert_array_equal(orc.round_storage(a, storage), a)   # every kept record in the type
    assert np.array_equal(a[..., 3], v0[..., 3])
    # a few roundings of at most half a unit each per iteration
    err = np.abs(a[..., :3] - b[..., :3]).max() / np.abs(b[..., :3]).max()
    assert 0.0 < err < 8 * ulp
    np.testing.assert_allclose(ra, rb, rtol=8 * ulp)


def test_threads_leave_renders_unchanged_and_regroup_updates(orc):
    n, views, side = 16, 3, 40
    shape, origin, h = synth.unit_grid(n)
    cams = synth.ring_cameras(views, side, side, elevation_jitter_deg=10.0, seed=4)
    gt, alb = synth.plume_volume(n, 4)
    sc = orc.Scene(shape, origin, h, cams)
    P = orc.make_params(step=0.5, alpha_l=5e-3, g_std=0.1, seed=3)
    img, _ = orc.render(sc, gt, P)
    targets, mask, bbox = orc.prepare_targets(img / img.max(), 30 / 255)
    v0 = gt.copy()
    v0[..., :3] *= 0.3
    out = {}
    try:
        for t in (1, 4):
            used = orc.set_threads(t)
            ren, ns = orc.render(sc, v0, P)
            res, _ = orc.residual(ren, targets, bbox)
            dV, na = orc.update_paper(sc, v0, P, res * mask[..., None], mask, 1)
            vol, rm, samples = orc.reconstruct(sc, v0, P, targets, mask, bbox, 3, albedo=alb)
            tags = orc.visual_hull(sc, mask)
            out[t] = (used, ren, ns, dV, na, vol, rm, samples, tags)
    finally:
        orc.set_threads(1)
    a, b = out[1], out[4]
    assert np.array_equal(a[1], b[1]) and a[2] == b[2]        # renders and sample counts
    assert a[4] == b[4] and a[7] == b[7]
    assert np.array_equal(a[8], b[8])                         # hull tags
    assert np.max(np.abs(a[3] - b[3])) <= 1e-12 * np.abs(a[3]).max()
    assert np.max(np.abs(a[5] - b[5])) <= 1e-12 * np.abs(a[5]).max()
    np.testing.assert_allclose(a[6], b[6], rtol=1e-12)
