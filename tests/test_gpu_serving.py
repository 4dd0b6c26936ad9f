"""The continuous-batching server on the GPU: a job's result is the same alone
and in a mix of other jobs (1e-2 with bf16 storage, float32 rounding with
float32 storage), matches fr_reconstruct, respects the memory budget, and
handles refusal, cancellation and bounded waits."""
import numpy as np
import pytest

from gpu_cases import rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _records(x, dtype):
    t = torch.as_tensor(x, dtype=torch.float32)
    if dtype == "f32":
        return t.numpy().copy()
    return t.to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16).copy()


def _as_float(rec, dtype):
    if dtype == "f32":
        return rec.astype(np.float64)
    return torch.from_numpy(rec.view(np.int16)).view(torch.bfloat16).float().numpy().astype(np.float64)


def _job_inputs(fr, ctx, synth, n, views, side, seed, step=0.5):
    shape, origin, h = synth.unit_grid(n)
    cams = synth.ring_cameras(views, side, side, elevation_jitter_deg=8.0, seed=seed)
    gt, _ = synth.plume_volume(n, seed)
    gt_d = torch.as_tensor(gt, dtype=torch.float32, device="cuda").contiguous()
    img = torch.zeros((views, side, side, 3), device="cuda")
    ctx.fr_render(fr.volume(gt_d, origin, h), fr.cameras(cams), fr.params(step=step), img)
    img /= img.max()
    init = gt.copy()
    init[..., :3] = 0.0
    return dict(shape=shape, origin=origin, h=h, cams=cams, targets=img.cpu().numpy(), init=init)


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_06417_gb300 import flamerec as fr, synth
    ctx = fr.Context(0)
    jobs = [_job_inputs(fr, ctx, synth, *spec) for spec in [(32, 4, 48, 21), (24, 6, 40, 22), (40, 3, 64, 23)]]
    yield fr, ctx, jobs
    torch.cuda.synchronize()
    ctx.close()


def _submit(srv, q, iters, dtype):
    return srv.submit(q["shape"], q["origin"], q["h"], q["cams"], iters, _records(q["init"], dtype), q["targets"])


@pytest.mark.parametrize("dtype,tol", [("f32", 1e-4), ("bf16", 1e-2)])
def test_same_result_alone_and_in_the_mix(env, dtype, tol):
    fr, ctx, jobs = env
    p = fr.params(step=0.5, alpha_l=2e-3)
    code = fr.FR_F32 if dtype == "f32" else fr.FR_BF16
    srv = fr.Server(ctx, p, dtype=code)
    alone = _submit(srv, jobs[0], 8, dtype)
    alone.wait()
    srv.close()
    srv = fr.Server(ctx, p, dtype=code)
    others = [_submit(srv, jobs[1], 5, dtype)]
    srv.step()
    srv.step()
    mixed = _submit(srv, jobs[0], 8, dtype)          # joins while another job runs
    others.append(_submit(srv, jobs[2], 12, dtype))  # arrives later, leaves later
    for j in [mixed] + others:
        j.wait()
    a, b = _as_float(alone.result, dtype), _as_float(mixed.result, dtype)
    e = rel_err(b[..., :3], a[..., :3])
    print(f"{dtype}: alone vs mix max {e.max():.2e}; rmse alone {alone.rmse[-1]}, mix {mixed.rmse[-1]}")
    assert e.max() < tol
    np.testing.assert_allclose(mixed.rmse, alone.rmse, rtol=max(tol, 1e-4))
    assert np.all(b[..., 3] == a[..., 3])  # extinction untouched
    srv.close()


@pytest.mark.parametrize("use_hull", [0, 1])
def test_server_matches_reconstruct(env, use_hull):
    fr, ctx, jobs = env
    q = jobs[1]
    p = fr.params(step=0.5, alpha_l=2e-3, use_hull=use_hull)
    srv = fr.Server(ctx, p, dtype=fr.FR_F32)
    job = _submit(srv, q, 6, "f32")
    job.wait()
    srv.close()
    v = torch.as_tensor(q["init"], dtype=torch.float32, device="cuda").contiguous()
    t = torch.as_tensor(q["targets"], device="cuda").contiguous()
    bbox = torch.zeros((len(q["cams"]), 4), dtype=torch.int32, device="cuda")
    ctx.fr_prepare_targets(t, 30 / 255, bbox)
    rmse = np.zeros((6, 3), dtype=np.float32)
    ctx.fr_reconstruct(fr.volume(v, q["origin"], q["h"]), fr.cameras(q["cams"]), t, bbox, 6, p, rmse=rmse)
    torch.cuda.synchronize()
    e = rel_err(job.result[..., :3], v.cpu().numpy()[..., :3].astype(np.float64))
    assert e.max() < 1e-4
    np.testing.assert_allclose(job.rmse, rmse, rtol=1e-4)


def test_budget_admission_refusal_cancel_and_wait(env):
    fr, ctx, jobs = env
    p = fr.params(step=0.5, alpha_l=2e-3)
    probe = fr.Server(ctx, p, dtype=fr.FR_F32)
    j = _submit(probe, jobs[2], 2, "f32")
    foot = j.info().footprint
    j.wait()
    probe.close()
    # a budget that holds one job of this size at a time
    srv = fr.Server(ctx, p, dtype=fr.FR_F32, budget_bytes=int(foot * 1.5))
    a = _submit(srv, jobs[2], 3, "f32")
    b = _submit(srv, jobs[2], 3, "f32")
    c = _submit(srv, jobs[2], 3, "f32")
    running, queued = srv.step()
    assert running == 1 and queued == 2
    used, budget = srv.memory()
    assert 0 < used <= budget
    c.cancel()
    with pytest.raises(fr.FrError, match="FR_EBUSY"):
        c.release()
    with pytest.raises(fr.FrError, match="FR_ETIMEDOUT"):
        b.wait(timeout_ms=0)
    a.wait()
    b.wait()
    assert a.info().state == fr.FR_JOB_DONE and b.info().state == fr.FR_JOB_DONE
    assert b.info().t_admit >= a.info().t_done - 1e-6   # b waited for a's memory
    srv.step()
    assert c.info().state == fr.FR_JOB_CANCELED
    c.release()
    assert srv.memory()[0] == 0
    # a job larger than the whole budget is refused at submission
    small = fr.Server(ctx, p, dtype=fr.FR_F32, budget_bytes=foot // 4)
    with pytest.raises(fr.FrError, match="FR_ENOMEM"):
        _submit(small, jobs[2], 3, "f32")
    small.close()
    srv.close()


@pytest.mark.parametrize("dtype,use_hull", [("f32", 0), ("f32", 1), ("bf16", 1)])
def test_served_job_follows_oracle(orc, env, dtype, use_hull):
    """One served job (raw frames prepared by the server at admission) against
    orc.reconstruct on targets the oracle rendered: float32 storage at the
    loop tolerance, BF16 storage against the oracle keeping BF16 records at
    the storage tolerance; with the hull the job carries the oracle's tags."""
    fr, ctx, _ = env
    from gpu_cases import Case, oracle_targets
    from paper_1809_06417_gb300 import synth
    n, views, side, seed, iters = 24, 6, 40, 22, 6
    shape, origin, h = synth.unit_grid(n)
    cams = synth.ring_cameras(views, side, side, elevation_jitter_deg=8.0, seed=seed)
    case = Case(shape, cams, synth.plume_volume(n, seed)[0], 0.5)
    sc, img, t_ref, mask, bbox_ref = oracle_targets(orc, case)
    tags = orc.visual_hull(sc, mask) if use_hull else None
    init = case.vol.copy()
    init[..., :3] = 0.0
    storage = "bf16" if dtype == "bf16" else None
    if storage:
        init = orc.round_storage(init, storage)
    P = orc.make_params(step=0.5, alpha_l=2e-3, storage=storage)
    ref, r_ref, _ = orc.reconstruct(sc, init, P, t_ref, mask, bbox_ref, iters, hull=tags)
    srv = fr.Server(ctx, fr.params(step=0.5, alpha_l=2e-3, use_hull=use_hull),
                    dtype=fr.FR_F32 if dtype == "f32" else fr.FR_BF16)
    job = srv.submit(shape, origin, h, cams, iters, _records(init, dtype), img.astype(np.float32), hull_tags=tags)
    job.wait()
    srv.close()
    got = _as_float(job.result, dtype)
    tol = 1e-3 if dtype == "f32" else 1e-2
    e = rel_err(got[..., :3], ref[..., :3])
    print(f"served {dtype} hull={use_hull}: volume vs oracle {e.max():.2e}; rmse {job.rmse[-1]} vs {r_ref[-1]}")
    assert e.max() < tol
    np.testing.assert_allclose(job.rmse, r_ref, rtol=tol)
