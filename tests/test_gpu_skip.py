"""Empty-brick skipping in the forward march (RGB records, field mode): renders
with and without it are bitwise identical -- a sample whose eight corner
records are all zero adds exactly nothing and leaves the transmittance
unchanged -- and the samples it evaluates are those whose cell lies in a brick
(of fr_brick_cells()^3 cells) holding a non-zero record (counted on the host in float64)."""
import numpy as np
import pytest

from gpu_cases import plume_case

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


def _host_count(vol, cams, origin, h, step, B):
    """Samples of all pixel rays whose cell is in an occupied brick of B^3 cells."""
    nz, ny, nx = vol.shape[:3]
    occ_node = np.any(vol != 0, axis=-1)
    nb = [(n - 2) // B + 1 for n in (nx, ny, nz)]
    occ = np.zeros((nb[2], nb[1], nb[0]), dtype=bool)
    k, j, i = np.nonzero(occ_node)
    for dk in (-1, 0):
        for dj in (-1, 0):
            for di in (-1, 0):
                ci, cj, ck = i + di, j + dj, k + dk
                ok = (ci >= 0) & (ci <= nx - 2) & (cj >= 0) & (cj <= ny - 2) & (ck >= 0) & (ck <= nz - 2)
                occ[ck[ok] // B, cj[ok] // B, ci[ok] // B] = True
    total = evaluated = 0
    hi = np.array([nx - 1, ny - 1, nz - 1], dtype=np.float64)
    for cam in cams:
        W, H, t = cam["width"], cam["height"], cam["tan_half_fov"]
        f, r, u = (np.asarray(cam[key], dtype=np.float64) for key in ("fwd", "right", "up"))
        px, py = np.meshgrid(np.arange(W), np.arange(H))
        a = ((2 * (px + 0.5) / W - 1) * t * W / H).ravel()
        b = ((1 - 2 * (py + 0.5) / H) * t).ravel()
        d = f[None] + a[:, None] * r + b[:, None] * u
        d /= np.linalg.norm(d, axis=-1, keepdims=True)
        o = (np.asarray(cam["pos"]) - np.asarray(origin)) / h
        with np.errstate(divide="ignore", invalid="ignore"):
            t0 = (0.0 - o) / d
            t1 = (hi - o) / d
        tin = np.maximum(np.nanmax(np.minimum(t0, t1), axis=-1), 0.0)
        tout = np.nanmin(np.maximum(t0, t1), axis=-1)
        hit = tout > tin
        chord = (tout - tin)[hit]
        p0 = o + tin[hit, None] * d[hit]
        dd = d[hit]
        n = np.ceil(chord / step).astype(np.int64)
        total += int(n.sum())
        for ks in range(int(n.max())):
            live = ks < n
            ta = ks * step
            tb = np.minimum(ta + step, chord[live])
            tm = 0.5 * (ta + tb)
            p = p0[live] + tm[:, None] * dd[live]
            c = np.clip(np.floor(p), 0, hi - 1).astype(np.int64)
            evaluated += int(occ[c[:, 2] // B, c[:, 1] // B, c[:, 0] // B].sum())
    return total, evaluated


def _clear_outside_sphere(vol, radius_frac):
    n = vol.shape[0]
    z, y, x = np.meshgrid(*(np.arange(n),) * 3, indexing="ij")
    c = 0.5 * (n - 1)
    out = (x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2 > (radius_frac * (n - 1)) ** 2
    v = vol.copy()
    v[out] = 0.0
    return v


def _render(fr, ctx, vol_t, origin, h, cams, step, skip):
    img = torch.zeros((len(cams), cams[0]["height"], cams[0]["width"], 3), device="cuda")
    ctx.fr_render(fr.volume(vol_t, origin, h), fr.cameras(cams), fr.params(step=step, skip_empty=skip), img)
    return img


@pytest.mark.parametrize("n,views,side,radius,dtype", [
    (40, 4, 64, 0.30, torch.float32),     # ragged last brick (39 cells)
    (48, 6, 96, 0.45, torch.float32),
    (48, 6, 96, 0.45, torch.bfloat16),
    (57, 3, 50, 0.25, torch.float16),     # 56 cells: whole bricks, odd image
])
def test_skip_is_bitwise_exact_and_counts_occupied_samples(fr_ctx, n, views, side, radius, dtype):
    fr, ctx = fr_ctx
    case = plume_case(n=n, views=views, side=side)
    vol = _clear_outside_sphere(case.vol, radius)
    vt = torch.as_tensor(vol, dtype=torch.float32, device="cuda").to(dtype).contiguous()
    a = _render(fr, ctx, vt, case.origin, case.h, case.cams, case.step, 1)
    b = _render(fr, ctx, vt, case.origin, case.h, case.cams, case.step, 0)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert float(a.max()) > 0
    fv = fr.volume(vt, case.origin, case.h)
    cams = fr.cameras(case.cams)
    s_all = ctx.fr_count_samples(fv, cams, fr.params(step=case.step, skip_empty=0))
    s_eval = ctx.fr_count_samples(fv, cams, fr.params(step=case.step, skip_empty=1))
    stored = vt.float().cpu().numpy()
    h_all, h_eval = _host_count(stored, case.cams, case.origin, case.h, case.step, fr.load().fr_brick_cells())
    print(f"n={n}: samples {s_all}, evaluated {s_eval} ({s_eval / s_all:.3f}); host {h_all}, {h_eval}")
    assert s_eval < s_all
    assert abs(s_all - h_all) <= 1e-4 * h_all
    assert abs(s_eval - h_eval) <= 1e-3 * h_eval


def test_skip_all_empty_and_tau_mode(fr_ctx):
    """An all-zero volume renders black with no sample evaluated; constant-tau
    mode (whose transmittance falls in empty space) does not skip."""
    fr, ctx = fr_ctx
    case = plume_case(n=33, views=3, side=40)
    z = torch.zeros((33, 33, 33, 4), device="cuda")
    img = _render(fr, ctx, z, case.origin, case.h, case.cams, case.step, 1)
    assert float(img.abs().max()) == 0.0
    fv = fr.volume(z, case.origin, case.h)
    cams = fr.cameras(case.cams)
    assert ctx.fr_count_samples(fv, cams, fr.params(step=case.step)) == 0
    vol = torch.as_tensor(_clear_outside_sphere(case.vol, 0.3), dtype=torch.float32, device="cuda").contiguous()
    fv = fr.volume(vol, case.origin, case.h)
    full = ctx.fr_count_samples(fv, cams, fr.params(step=case.step, skip_empty=0))
    assert ctx.fr_count_samples(fv, cams, fr.params(step=case.step, tau=0.05)) == full


def test_full_size_hull_cleared_plume_bitwise(fr_ctx):
    """The benchmark's shape: 128^3 plume cleared outside a sphere, 8 x 512^2."""
    fr, ctx = fr_ctx
    from paper_1809_06417_gb300 import synth
    n, views, side, step = 128, 8, 512, 0.5
    shape, origin, h = synth.unit_grid(n)
    cams = synth.ring_cameras(views, side, side, elevation_jitter_deg=10.0, seed=2)
    gt, _ = synth.plume_volume(n, 1002)
    vt = torch.as_tensor(_clear_outside_sphere(gt, 0.35), dtype=torch.float32, device="cuda").contiguous()
    a = _render(fr, ctx, vt, origin, h, cams, step, 1)
    b = _render(fr, ctx, vt, origin, h, cams, step, 0)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    fv = fr.volume(vt, origin, h)
    fc = fr.cameras(cams)
    s_all = ctx.fr_count_samples(fv, fc, fr.params(step=step, skip_empty=0))
    s_eval = ctx.fr_count_samples(fv, fc, fr.params(step=step))
    print(f"full size: evaluated fraction {s_eval / s_all:.3f}")


def test_hull_reconstruct_same_with_and_without_skipping(fr_ctx):
    """fr_reconstruct restricted to the visual hull, whose forward skips empty
    bricks and whose adjustment skips bricks outside the hull, gives the same
    volume and errors as with skipping off (up to the order of the atomic
    sums), and evaluates fewer samples."""
    fr, ctx = fr_ctx
    case = plume_case(n=64, views=6, side=128)
    g = torch.as_tensor(case.vol, dtype=torch.float32, device="cuda").contiguous()
    fc = fr.cameras(case.cams)
    img = torch.zeros((6, 128, 128, 3), device="cuda")
    ctx.fr_render(fr.volume(g, case.origin, case.h), fc, fr.params(step=case.step), img)
    img /= img.max()
    bbox = torch.zeros((6, 4), dtype=torch.int32, device="cuda")
    ctx.fr_prepare_targets(img, 30 / 255, bbox)
    tags = torch.zeros(g.shape[:3], dtype=torch.int32, device="cuda")
    ctx.fr_visual_hull(fr.volume(g, case.origin, case.h), fc, img, fr.params(), tags)
    alb = torch.as_tensor(case.albedo, dtype=torch.float32, device="cuda").contiguous()
    out = []
    for skip in (1, 0):
        v = g.clone()
        v[..., :3] = 0.0
        p = fr.params(step=case.step, alpha_l=2e-3, use_hull=1, hull_tags=tags, skip_empty=skip)
        rmse = np.zeros((4, 3), dtype=np.float32)
        fv = fr.volume(v, case.origin, case.h)
        ctx.fr_reconstruct(fv, fc, img, bbox, 4, p, albedo=alb, rmse=rmse)
        n_f = ctx.fr_count_samples(fv, fc, p)
        n_a = ctx.fr_count_samples(fv, fc, p, residual=img)
        torch.cuda.synchronize()
        out.append((v.cpu().numpy(), rmse, n_f, n_a))
    (a, ra, fa, aa), (b, rb, fb, ab) = out
    from gpu_cases import rel_err
    print(f"forward samples {fa} of {fb}, adjustment samples {aa} of {ab}; "
          f"max diff {np.max(rel_err(a, b)):.2e}")
    assert np.array_equal(a == 0, b == 0)
    assert np.max(rel_err(a, b)) < 1e-5
    np.testing.assert_allclose(ra, rb, rtol=1e-5)
    assert fa < fb and aa < ab
