"""Volumes held by the library: fr_volume_create / upload / download / free.

Float32 records go in and come out; 16-bit storage rounds them to nearest even
inside the library, which must equal torch's float32 -> bfloat16 / float16
conversion bit for bit (both are the IEEE round-to-nearest-even of one float32
value).  A reconstruction on a library-held volume equals the same
reconstruction on a caller-held one."""
import numpy as np
import pytest

from gpu_cases import rel_err, tiny_case

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


DTYPES = {0: torch.float32, 1: torch.bfloat16, 2: torch.float16}


@pytest.mark.parametrize("dtype", [0, 1, 2])
@pytest.mark.parametrize("kind,shape", [(0, (17, 9, 12)), (1, (3, 3, 3)), (1, (20, 16, 8))])
def test_upload_download_round_trip(fr_ctx, dtype, kind, shape):
    fr, ctx = fr_ctx
    comp = 4 if kind == 0 else 2
    nx, ny, nz = shape
    rng = np.random.default_rng(dtype * 10 + kind)
    # normal values over many binades (no float32 subnormals: the kernels flush those)
    x = (rng.normal(size=(nz, ny, nx, comp)) * np.exp(rng.uniform(-12, 8, size=(nz, ny, nx, comp))))
    x = x.astype(np.float32)
    want = torch.from_numpy(x).to(DTYPES[dtype]).to(torch.float32).numpy()
    vol = ctx.fr_volume_create(shape, (-0.5, -0.5, -0.5), 0.1, kind=kind, dtype=dtype)
    out = np.full_like(x, np.nan)
    ctx.fr_volume_download(vol, out)
    assert np.all(out == 0.0)                                   # created zeroed
    ctx.fr_volume_upload(vol, x)                                # from host memory
    ctx.fr_volume_download(vol, out)
    np.testing.assert_array_equal(out, want)
    # device to device, and the stored records themselves
    ctx.fr_volume_upload(vol, torch.as_tensor(x * 0.5, device="cuda"))
    dev_out = torch.full((nz, ny, nx, comp), float("nan"), device="cuda")
    ctx.fr_volume_download(vol, dev_out)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(dev_out.cpu().numpy(), torch.from_numpy(x * 0.5).to(DTYPES[dtype]).float().numpy())
    ctx.fr_volume_free(vol)
    assert vol.data is None
    with pytest.raises(fr.FrError, match="FR_EINVAL"):
        ctx.fr_volume_free(vol)


def test_refusals(fr_ctx):
    fr, ctx = fr_ctx
    t = torch.zeros((4, 4, 4, 4), device="cuda")
    with pytest.raises(fr.FrError, match="not created by fr_volume_create"):
        ctx.fr_volume_free(fr.volume(t, (0, 0, 0), 1.0))
    with pytest.raises(fr.FrError, match="FR_EINVAL"):
        ctx.fr_volume_create((1, 4, 4), (0, 0, 0), 1.0)
    with pytest.raises(fr.FrError, match="FR_EINVAL"):
        ctx.fr_volume_create((4, 4, 4), (0, 0, 0), 0.0)
    vol = ctx.fr_volume_create((4, 4, 4), (0, 0, 0), 1.0, dtype=fr.FR_BF16)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    big = torch.zeros(16 * 2 ** 20 // 4, device="cuda")   # its own 16 MiB allocation
    tail = big[-64:]                                      # 256 bytes before it ends; 1 KiB are read
    with pytest.raises(fr.FrError, match="FR_EINVAL.*allocation ends"):
        ctx.fr_volume_upload(vol, tail)
    with pytest.raises(fr.FrError, match="FR_EINVAL.*aligned"):
        ctx.fr_volume_upload(vol, big[1:257])              # 4-byte offset
    ctx.fr_volume_free(vol)


@pytest.mark.parametrize("dtype", [0, 1])
def test_reconstruct_on_a_library_volume(fr_ctx, dtype):
    fr, ctx = fr_ctx
    case = tiny_case()
    K, S = len(case.cams), case.cams[0]["width"]
    g = torch.as_tensor(case.vol, dtype=torch.float32, device="cuda").contiguous()
    img = torch.zeros((K, S, S, 3), device="cuda")
    fc = fr.cameras(case.cams)
    ctx.fr_render(fr.volume(g, case.origin, case.h), fc, fr.params(step=case.step), img)
    img /= img.max()
    bbox = torch.zeros((K, 4), dtype=torch.int32, device="cuda")
    ctx.fr_prepare_targets(img, 30 / 255, bbox)
    v0 = case.vol.astype(np.float32)
    v0[..., :3] = 0.0
    p = fr.params(step=case.step, alpha_l=0.01)
    mine = torch.as_tensor(v0, device="cuda").to(DTYPES[dtype]).contiguous()
    ctx.fr_reconstruct(fr.volume(mine, case.origin, case.h), fc, img, bbox, 5, p)
    lib = ctx.fr_volume_create(case.shape, case.origin, case.h, dtype=dtype)
    ctx.fr_volume_upload(lib, v0)
    ctx.fr_reconstruct(lib, fc, img, bbox, 5, p)
    out = np.empty_like(v0)
    ctx.fr_volume_download(lib, out)
    ctx.fr_volume_free(lib)
    ref = mine.float().cpu().numpy().astype(np.float64)
    assert np.max(rel_err(out, ref)) < (1e-5 if dtype == 0 else 1e-2)
