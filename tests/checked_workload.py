"""Runs the library's entry points on small seeded cases and prints the
bounds-check word as JSON; run with FR_LIBRARY_VARIANT=checked to load the
bounds-checked build (used by test_gpu_checked.py)."""
import json
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from gpu_cases import plume_case, ragged_case  # noqa: E402
from paper_1809_06417_gb300 import flamerec as fr, synth  # noqa: E402


def main():
    ctx = fr.Context(0)
    words = {}
    # render / residual / adjust / backward on a ragged case, f32 and bf16
    case = ragged_case()
    fc = fr.cameras(case.cams)
    K, H, W = len(case.cams), case.cams[0]["height"], case.cams[0]["width"]
    for dt in (torch.float32, torch.bfloat16):
        v = torch.as_tensor(case.vol, dtype=torch.float32, device="cuda").to(dt).contiguous()
        fv = fr.volume(v, case.origin, case.h)
        img = torch.zeros((K, H, W, 3), device="cuda")
        ctx.fr_render(fv, fc, fr.params(step=case.step), img)
        bbox = torch.zeros((K, 4), dtype=torch.int32, device="cuda")
        t = (img / img.max()).contiguous()
        ctx.fr_prepare_targets(t, 30 / 255, bbox)
        res = torch.empty_like(t)
        sq = torch.zeros(4, device="cuda")
        ctx.fr_render_residual(fv, fc, fr.params(step=case.step), t, bbox, None, res, sq)
        dV = torch.zeros(v.shape[:3] + (4,), device="cuda")
        ctx.fr_adjust(fv, fc, fr.params(step=case.step), res, 0, dV)
        grad = torch.zeros(v.shape[:3] + (4,), device="cuda")
        ctx.fr_render_backward(fv, fc, fr.params(step=case.step), img, res, grad)
        fr.fr_render_residual_noalloc(0, torch.cuda.current_stream(), fv, fc, fr.params(step=case.step), t, bbox,
                                      None, res, sq)
    words["render_adjust_backward"] = ctx.fr_check_word(reset=True)
    # the loop: hull, skipping, scattering, variants, stop criterion
    case = plume_case(n=36, views=5, side=56)
    g = torch.as_tensor(case.vol, dtype=torch.float32, device="cuda").contiguous()
    fc = fr.cameras(case.cams)
    img = torch.zeros((5, 56, 56, 3), device="cuda")
    ctx.fr_render(fr.volume(g, case.origin, case.h), fc, fr.params(step=case.step), img)
    img /= img.max()
    bbox = torch.zeros((5, 4), dtype=torch.int32, device="cuda")
    ctx.fr_prepare_targets(img, 30 / 255, bbox)
    alb = torch.as_tensor(case.albedo, dtype=torch.float32, device="cuda").contiguous()
    for kw in (dict(), dict(use_hull=1), dict(use_hull=1, tables=2), dict(use_hull=1, hg_g=0.5),
               dict(use_hull=1, sequential_views=1)):
        v = g.clone()
        v[..., :3] = 0.0
        fv = fr.volume(v, case.origin, case.h)
        p = fr.params(step=case.step, alpha_l=3e-3, **kw)
        ctx.fr_reconstruct(fv, fc, img, bbox, 3, p, albedo=alb)
        ctx.fr_reconstruct_until(fv, fc, img, bbox, 4, 0.01, p, albedo=alb)
        ctx.fr_count_samples(fv, fc, p)
    tags = torch.zeros(g.shape[:3], dtype=torch.int32, device="cuda")
    ctx.fr_visual_hull(fr.volume(g, case.origin, case.h), fc, img, fr.params(), tags)
    ctx.fr_volume_rmse(fr.volume(g, case.origin, case.h), fr.volume(g, case.origin, case.h), tags, 31)
    words["loop"] = ctx.fr_check_word(reset=True)
    # batched problems and the server
    probs, keep = [], []
    for n, views, side, seed in ((20, 3, 30, 1), (24, 4, 36, 2)):
        c2 = plume_case(n=n, views=views, side=side, seed=seed)
        g2 = torch.as_tensor(c2.vol, dtype=torch.float32, device="cuda").contiguous()
        im2 = torch.zeros((views, side, side, 3), device="cuda")
        ctx.fr_render(fr.volume(g2, c2.origin, c2.h), fr.cameras(c2.cams), fr.params(step=c2.step), im2)
        im2 /= im2.max()
        b2 = torch.zeros((views, 4), dtype=torch.int32, device="cuda")
        ctx.fr_prepare_targets(im2, 30 / 255, b2)
        v2 = g2.clone()
        v2[..., :3] = 0.0
        keep.append((v2, im2, b2, c2))
        probs.append((fr.volume(v2, c2.origin, c2.h), fr.cameras(c2.cams), im2, b2, None))
    ctx.fr_reconstruct_batch(probs, 3, fr.params(step=0.5, alpha_l=2e-3, use_hull=1), use_graph=True)
    ctx.fr_reconstruct_batch(probs, 3, fr.params(step=0.5, alpha_l=2e-3, use_hull=1, tables=2), use_graph=True)
    srv = fr.Server(ctx, fr.params(step=0.5, alpha_l=2e-3, use_hull=1), dtype=fr.FR_F32)
    jobs = []
    for v2, im2, b2, c2 in keep:
        init = v2.cpu().numpy()
        jobs.append(srv.submit(c2.shape, c2.origin, c2.h, c2.cams, 4, init, im2.cpu().numpy()))
    for j in jobs:
        j.wait()
    srv.close()
    words["batch_server"] = ctx.fr_check_word(reset=True)
    torch.cuda.synchronize()
    print(json.dumps({"checks_enabled": int(fr.load().fr_checks_enabled()), "words": words}))
    ctx.close()


if __name__ == "__main__":
    main()
