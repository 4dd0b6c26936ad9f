"""The benchmarked workload itself against the FP64 oracle: 128^3 nodes of the
seeded full-RTE plume (emission, extinction, scattering albedo), 8 jittered
ring cameras of 512 x 512, a half-voxel step.

* One render with residual of a mid-reconstruction volume through its
  in-scattering source (Eq. 5): image element by element at the radiance
  tolerance, residual and the error sums.
* Two iterations of fr_reconstruct in the launch configuration the benchmark
  times -- in-scattering source, visual hull (the oracle's tags, given to both
  sides), empty-brick skipping, the ray weight tables (and, beside them, the
  marches with the adjustment over half rays) -- against orc.reconstruct on
  the same tags: per-iteration error and the updated volume.

The oracle runs on every host core (its pixel loops are independent; see
oracle.set_threads).
"""
import os

import numpy as np
import pytest

from gpu_cases import rel_err, tags_on_device

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N, VIEWS, SIDE, STEP, SEED, ALPHA_L = 128, 8, 512, 0.5, 2, 2e-4


@pytest.fixture(scope="module")
def full(orc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_06417_gb300 import flamerec as fr, synth
    orc.set_threads(os.cpu_count() or 1)
    shape, origin, h = synth.unit_grid(N)
    gt, alb = synth.plume_volume(N, SEED)
    cams = synth.ring_cameras(VIEWS, SIDE, SIDE, elevation_jitter_deg=10.0, seed=SEED)
    sc = orc.Scene(shape, origin, h, cams)
    P = orc.make_params(step=STEP, alpha_l=ALPHA_L)
    src = orc.scatter_source(gt, alb, orc.scatter_J(sc, gt))
    img, _ = orc.render(sc, src, P)
    scale = float(img.max())
    img = synth.add_noise(img / scale, 1e-3, SEED)
    t_ref, mask, bbox_ref = orc.prepare_targets(img, 30 / 255)
    tags = orc.visual_hull(sc, mask)
    ctx = fr.Context(0)
    t_dev = torch.as_tensor(img, dtype=torch.float32, device="cuda").contiguous()
    bbox = torch.zeros((VIEWS, 4), dtype=torch.int32, device="cuda")
    ctx.fr_prepare_targets(t_dev, 30 / 255, bbox)
    torch.cuda.synchronize()
    assert np.array_equal(bbox.cpu().numpy(), bbox_ref)
    d = dict(fr=fr, ctx=ctx, sc=sc, P=P, gt=gt, alb=alb, scale=scale, cams=cams, origin=origin, h=h, img=img,
             t_ref=t_ref, mask=mask, bbox_ref=bbox_ref, tags=tags, t_dev=t_dev, bbox=bbox)
    yield d
    torch.cuda.synchronize()
    ctx.close()


def _start(full):
    """A mid-reconstruction state: half the ground truth's emission on the
    targets' scale inside the hull, nothing outside it."""
    v0 = full["gt"].copy()
    v0[..., :3] *= 0.5 / full["scale"]
    outside = full["tags"] != (1 << VIEWS) - 1
    v0[outside] = 0.0
    return v0


def test_full_size_render_residual_follows_oracle(orc, full):
    fr, ctx, sc, P = full["fr"], full["ctx"], full["sc"], full["P"]
    v0 = _start(full)
    src_ref = orc.scatter_source(v0, full["alb"], orc.scatter_J(sc, v0))
    ren_ref, n_ref = orc.render(sc, src_ref, P)
    res_ref, rmse_ref = orc.residual(ren_ref, full["t_ref"], full["bbox_ref"])
    res_ref *= full["mask"][..., None]
    v = torch.as_tensor(v0, dtype=torch.float32, device="cuda").contiguous()
    alb = torch.as_tensor(full["alb"], dtype=torch.float32, device="cuda").contiguous()
    src = torch.empty_like(v)
    J = torch.empty((N, N, N, 4), device="cuda")
    ctx.fr_scatter_source(fr.volume(v, full["origin"], full["h"]), alb, J, fr.volume(src, full["origin"], full["h"]))
    ren = torch.empty_like(full["t_dev"])
    res = torch.empty_like(full["t_dev"])
    sq = torch.zeros(4, device="cuda")
    ctx.fr_render_residual(fr.volume(src, full["origin"], full["h"]), fr.cameras(full["cams"]),
                           fr.params(step=STEP), full["t_dev"], full["bbox"], ren, res, sq)
    torch.cuda.synchronize()
    got = ren.cpu().numpy().astype(np.float64)
    err = np.abs(got - ren_ref)
    bound = 1e-4 * np.abs(ren_ref) + 1e-6 * np.abs(ren_ref).max()
    print(f"full-size render: {n_ref} samples, max error / max {err.max() / np.abs(ren_ref).max():.3e}, "
          f"worst error / bound {np.max(err / bound):.3f}")
    assert np.all(err <= bound)
    r = res.cpu().numpy().astype(np.float64)
    assert np.all(r[full["mask"] == 0] == 0.0)
    assert np.max(rel_err(r, res_ref)) < 1e-5
    q = sq.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(255.0 * np.sqrt(q[:3] / q[3]), rmse_ref, rtol=1e-4)


@pytest.fixture(scope="module")
def ref2(orc, full):
    """The oracle's two iterations from the mid-reconstruction start, with its
    undecided budget (shared by the marching and the table runs)."""
    v0 = _start(full)
    vol_ref, rmse_ref, samples, und = orc.reconstruct(full["sc"], v0, full["P"], full["t_ref"], full["mask"],
                                                      full["bbox_ref"], 2, albedo=full["alb"], hull=full["tags"],
                                                      with_undecided=True)
    return dict(v0=v0, vol=vol_ref, rmse=rmse_ref, samples=samples, und=und)


@pytest.mark.parametrize("tables", [1, 2], ids=["march", "tables"])
def test_full_size_reconstruct_iterations_follow_oracle(orc, full, ref2, tables):
    """fr_reconstruct as the benchmark calls it (hull tags given, empty bricks
    skipped, in-scattering) for two iterations, marching every iteration
    (the adjustment over half rays) or streaming the ray weight tables built
    at the start of the call.  Which eight key points a sample updates
    (Eq. 10) is an integer decision: of the 7e7 adjustment samples, those
    within float32 rounding of a cell face (or the last sample of a ray whose
    chord is within rounding of a whole number of steps) may update the
    neighbouring cell's key points on one side only.  The oracle bounds, per
    node, what those samples can move (its undecided budget); every node must
    lie within 1e-4 of the volume's maximum plus its budget."""
    fr, ctx = full["fr"], full["ctx"]
    v0, vol_ref, rmse_ref, samples, und = ref2["v0"], ref2["vol"], ref2["rmse"], ref2["samples"], ref2["und"]
    iters = 2
    v = torch.as_tensor(v0, dtype=torch.float32, device="cuda").contiguous()
    alb = torch.as_tensor(full["alb"], dtype=torch.float32, device="cuda").contiguous()
    p = fr.params(step=STEP, alpha_l=ALPHA_L, use_hull=1, hull_tags=tags_on_device(torch, full["tags"]),
                  skip_empty=1, tables=tables)
    rmse = np.zeros((iters, 3), dtype=np.float32)
    ctx.fr_reconstruct(fr.volume(v, full["origin"], full["h"]), fr.cameras(full["cams"]), full["t_dev"],
                       full["bbox"], iters, p, albedo=alb, rmse=rmse)
    torch.cuda.synchronize()
    got = v.cpu().numpy().astype(np.float64)
    scale = np.abs(vol_ref[..., :3]).max()
    err = np.abs(got[..., :3] - vol_ref[..., :3]).max(axis=-1)
    bound = 1e-4 * scale + und
    flagged = und > 0
    moved = np.abs(vol_ref[..., :3] - v0[..., :3]).max() / scale
    print(f"oracle samples (forward, adjustment) {samples}; rmse gpu {rmse.tolist()} oracle {rmse_ref.tolist()}")
    print(f"full-size volume after {iters} iterations, tables={tables} (the update moved it by {moved:.3e} of its "
          f"max): max error / max {err.max() / scale:.3e}; nodes with an undecided budget {flagged.sum()} "
          f"({flagged.mean():.2e}); max error / max off them {err[~flagged].max() / scale:.3e}; "
          f"worst error / bound {np.max(err / bound):.3f}")
    # the first row is the error of the render of v0; the next ones follow updates
    np.testing.assert_allclose(rmse[0], rmse_ref[0], rtol=1e-4)
    np.testing.assert_allclose(rmse, rmse_ref, rtol=1e-3)
    assert np.all(err <= bound)
    # the budget is small where it is not zero: a few samples' weights
    print(f"budget on flagged nodes / max: p50 {np.median(und[flagged]) / scale:.2e}, "
          f"p99.9 {np.quantile(und[flagged], 0.999) / scale:.2e}")
    assert np.quantile(und[flagged], 0.999) < 2e-2 * scale
    outside = full["tags"] != (1 << VIEWS) - 1
    assert np.all(got[outside] == 0.0)
    assert np.array_equal(got[..., 3], v0[..., 3].astype(np.float32))


@pytest.fixture(scope="module")
def ref_bf16(orc, full):
    """The oracle's two iterations keeping BF16 records, and with FP64 records."""
    sc, P = full["sc"], full["P"]
    v0 = orc.round_storage(_start(full), "bf16")
    P16 = orc.make_params(step=STEP, alpha_l=ALPHA_L, storage="bf16")
    ref16, r16, _ = orc.reconstruct(sc, v0, P16, full["t_ref"], full["mask"], full["bbox_ref"], 2,
                                    albedo=full["alb"], hull=full["tags"])
    ref64, _, _ = orc.reconstruct(sc, v0, P, full["t_ref"], full["mask"], full["bbox_ref"], 2,
                                  albedo=full["alb"], hull=full["tags"])
    return dict(v0=v0, ref16=ref16, r16=r16, ref64=ref64)


@pytest.mark.parametrize("tables", [1, 2], ids=["march", "tables"])
def test_full_size_bf16_records_follow_the_16bit_oracle(orc, full, ref_bf16, tables):
    """The benchmarked workload with BF16 records (FP32 arithmetic): two
    iterations against the oracle keeping BF16 records, at the storage
    tolerance of 1e-2 of the volume's maximum; the error against the FP64
    loop with double-precision records is printed beside it."""
    fr, ctx = full["fr"], full["ctx"]
    v0, ref16, r16, ref64 = ref_bf16["v0"], ref_bf16["ref16"], ref_bf16["r16"], ref_bf16["ref64"]
    iters = 2
    v = torch.as_tensor(v0, dtype=torch.float32, device="cuda").to(torch.bfloat16).contiguous()
    alb = torch.as_tensor(full["alb"], dtype=torch.float32, device="cuda").contiguous()
    p = fr.params(step=STEP, alpha_l=ALPHA_L, use_hull=1, hull_tags=tags_on_device(torch, full["tags"]),
                  tables=tables)
    rmse = np.zeros((iters, 3), dtype=np.float32)
    ctx.fr_reconstruct(fr.volume(v, full["origin"], full["h"]), fr.cameras(full["cams"]), full["t_dev"],
                       full["bbox"], iters, p, albedo=alb, rmse=rmse)
    torch.cuda.synchronize()
    got = v.float().cpu().numpy().astype(np.float64)
    e16 = rel_err(got[..., :3], ref16[..., :3])
    e64 = rel_err(got[..., :3], ref64[..., :3])
    print(f"full-size BF16 (tables={tables}): volume vs BF16 oracle max {e16.max():.2e} (p99.99 {np.quantile(e16, 0.9999):.2e}); "
          f"vs FP64 records {e64.max():.2e}; rmse gpu {rmse[-1]} oracle {r16[-1]}")
    assert e16.max() < 1e-2
    np.testing.assert_allclose(rmse, r16, rtol=1e-2)
