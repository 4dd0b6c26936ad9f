"""Phase tracing of fr_reconstruct: the library's events split the device time
of a call into its phases; their sum matches the time measured around the call
and each phase that ran has a positive share.  With in-scattering and the
visual hull the pair pack runs inside the last sweep (no pack phase); without
in-scattering it is a phase of its own."""
import numpy as np
import pytest

from gpu_cases import plume_case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_phase_times_cover_the_call():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_06417_gb300 import flamerec as fr
    ctx = fr.Context(0)
    try:
        case = plume_case(n=64, views=6, side=128)
        g = torch.as_tensor(case.vol, dtype=torch.float32, device="cuda").contiguous()
        fc = fr.cameras(case.cams)
        img = torch.zeros((6, 128, 128, 3), device="cuda")
        ctx.fr_render(fr.volume(g, case.origin, case.h), fc, fr.params(step=case.step), img)
        img /= img.max()
        bbox = torch.zeros((6, 4), dtype=torch.int32, device="cuda")
        ctx.fr_prepare_targets(img, 30 / 255, bbox)
        alb = torch.as_tensor(case.albedo, dtype=torch.float32, device="cuda").contiguous()
        v = g.clone()
        v[..., :3] = 0
        fv = fr.volume(v, case.origin, case.h)
        p = fr.params(step=case.step, alpha_l=2e-3, use_hull=1)
        ctx.fr_reconstruct(fv, fc, img, bbox, 1, p, albedo=alb)      # warm-up
        torch.cuda.synchronize()
        ctx.fr_trace_phases(True)
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(2):
            ctx.fr_reconstruct(fv, fc, img, bbox, 3, p, albedo=alb)
        e1.record(stream)
        torch.cuda.synchronize()
        ms, calls = ctx.fr_phase_times()
        total = e0.elapsed_time(e1)
        print({k: round(x, 4) for k, x in ms.items()}, "calls", calls, "total", round(total, 4))
        assert calls == 2
        for k in ("setup", "scatter", "forward", "reduce", "adjust", "apply", "finish"):
            assert ms[k] > 0.0, k
        assert ms["pack"] == 0.0
        assert sum(ms.values()) <= total * 1.001
        assert sum(ms.values()) > 0.8 * total
        # read again: the record was dropped
        ms2, calls2 = ctx.fr_phase_times()
        assert calls2 == 0 and sum(ms2.values()) == 0.0
        # without in-scattering: a pack phase of its own, no sweeps
        ctx.fr_reconstruct(fv, fc, img, bbox, 2, p)
        torch.cuda.synchronize()
        ms4, calls4 = ctx.fr_phase_times()
        assert calls4 == 1 and ms4["pack"] > 0.0 and ms4["scatter"] == 0.0 and ms4["forward"] > 0.0
        # tracing off: nothing is recorded
        ctx.fr_trace_phases(False)
        ctx.fr_reconstruct(fv, fc, img, bbox, 1, p, albedo=alb)
        ms3, calls3 = ctx.fr_phase_times()
        assert calls3 == 0
    finally:
        torch.cuda.synchronize()
        ctx.close()
