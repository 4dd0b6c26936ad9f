"""Reconstruction with 16-bit voxel storage (BF16 or FP16 records, float32
arithmetic) against the FP64 oracle that keeps its records in the same type.

The oracle rounds every record the loop stores -- the volume on entry and
after each update, the in-scattering source each time it is formed -- to the
storage type (oracle.round_storage); the GPU rounds the same records from
float32.  Where a value lies within float32 rounding of a rounding boundary
of the 16-bit type the two sides may round it to neighbouring values, one unit
in the last place apart (2^-8 relative for BF16, 2^-11 for FP16), and such a
difference then propagates through the later iterations; the comparison is
therefore made at the storage tolerance, 1e-2 of the field's maximum.  The
error of each 16-bit result against the FP64 loop with double-precision
records (the storage error itself) is printed beside it."""
import numpy as np
import pytest

from gpu_cases import oracle_targets, plume_case, rel_err, tiny_case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TORCH_DT = {"bf16": "bfloat16", "f16": "float16"}


@pytest.fixture(scope="module")
def fr_ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_06417_gb300 import flamerec as fr
    ctx = fr.Context(0)
    yield fr, ctx
    torch.cuda.synchronize()
    ctx.close()


@pytest.mark.parametrize("storage", ["bf16", "f16"])
@pytest.mark.parametrize("workload", ["tiny", "plume_scatter"])
def test_16bit_storage_loop_follows_oracle(orc, fr_ctx, storage, workload):
    fr, ctx = fr_ctx
    if workload == "tiny":
        # the tiny configuration: 32^3 blobs, 4 views of 64^2, step 1, 10 iterations
        case, alpha, albedo, noise = tiny_case(), 0.01, None, 1e-3
    else:
        # full-RTE physics at a small size: plume with albedo, in-scattering source
        case, alpha, noise = plume_case(n=32, views=4, side=48), 3e-3, 0.0
        albedo = case.albedo
    iters = 10
    sc, img, t_ref, mask, bbox_ref = oracle_targets(orc, case, albedo=albedo, noise=noise)
    v0 = case.vol.copy()
    v0[..., :3] = 0.0
    v0 = orc.round_storage(v0, storage)          # the stored start: every record a 16-bit value
    P16 = orc.make_params(step=case.step, alpha_l=alpha, storage=storage)
    P64 = orc.make_params(step=case.step, alpha_l=alpha)
    ref16, r16, _ = orc.reconstruct(sc, v0, P16, t_ref, mask, bbox_ref, iters, albedo=albedo)
    ref64, r64, _ = orc.reconstruct(sc, v0, P64, t_ref, mask, bbox_ref, iters, albedo=albedo)
    dt = getattr(torch, TORCH_DT[storage])
    v = torch.as_tensor(v0, dtype=torch.float32, device="cuda").to(dt).contiguous()
    assert np.array_equal(v.float().cpu().numpy(), v0.astype(np.float32))   # exact in the type
    t_dev = torch.as_tensor(img, dtype=torch.float32, device="cuda").contiguous()
    bbox = torch.zeros((len(case.cams), 4), dtype=torch.int32, device="cuda")
    ctx.fr_prepare_targets(t_dev, 30 / 255, bbox)
    alb = torch.as_tensor(albedo, dtype=torch.float32, device="cuda").contiguous() if albedo is not None else None
    rmse = np.zeros((iters, 3), dtype=np.float32)
    ctx.fr_reconstruct(fr.volume(v, case.origin, case.h), fr.cameras(case.cams), t_dev, bbox, iters,
                       fr.params(step=case.step, alpha_l=alpha), albedo=alb, rmse=rmse)
    torch.cuda.synchronize()
    got = v.float().cpu().numpy().astype(np.float64)
    e16 = rel_err(got[..., :3], ref16[..., :3])
    e64 = rel_err(got[..., :3], ref64[..., :3])
    s64 = rel_err(ref16[..., :3], ref64[..., :3])
    print(f"{workload} {storage}: volume vs 16-bit oracle max {e16.max():.2e} (p99.9 "
          f"{np.quantile(e16, 0.999):.2e}); vs FP64 records max {e64.max():.2e}; oracle's own storage "
          f"error {s64.max():.2e}; rmse gpu {rmse[-1]} oracle {r16[-1]} fp64 {r64[-1]}")
    assert e16.max() < 1e-2
    np.testing.assert_allclose(rmse, r16, rtol=1e-2)
    assert np.array_equal(got[..., 3], v0[..., 3])                  # extinction untouched
