"""Benchmark of the reconstruction loop (render -> residual -> adjust -> apply).

Workload (default): the full-RTE setting -- a 128^3 float32 volume holding RGB
emission, extinction and scattering albedo (seeded 8-blob plume with 4-octave
value noise), 8 ring cameras at 512 x 512, a 0.5-voxel ray step, the paper's
adjustment rule.  One step is one whole reconstruction of that setting: 50
iterations (in-scattering source, rendering with fused residual, error
reduction, adjustment, update) from the zero start in one fr_reconstruct call,
which builds the ray weight tables first and streams them every iteration.

Metric: ray samples per second, forward + adjustment: the samples the
iterations stand for (those the marches evaluate per iteration, times the
iterations) over the step's device time; iterations per second are reported
beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--storage f32|bf16]

Under torchrun every rank runs an independent replica (the loop does not
shard within one volume here); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ray samples/s (fwd+adjoint) and recon iters/s at 128^3×8 views; p50/p99 job latency"
WORKLOAD = dict(name="full_rte_128^3_8x512^2", n=128, views=8, side=512, step=0.5, seed=2,
                alpha_l=2e-4, noise=1e-3, hull=True)
# iterations of one step (the full-RTE setting runs 50)
ITERS_PER_STEP = 50
# kernels one step launches: hull clear with the hull's brick marks and box;
# the tables' build (the count march's tile order from each tile's samples
# in the hull's box: 2, count march, four scans of three kernels, the hull's
# list, fill march, entry ends); then per iteration the in-scatter sweeps
# (3, over the box of the hull's bricks), the staging of the hull's source
# records, the forward table's render with the residual, and the adjustment
# table's update with the error reduction (which also writes the rmse) in
# the same launch
KERNELS_SETUP = 1 + 18
KERNELS_PER_ITERATION = 6
# dram__bytes_read.sum + dram__bytes_write.sum per launch from ncu captures of
# the current kernels at this workload (None where the kernel changed since)
NCU_TRAFFIC = {("fwd", "f32"): 415.31e6 + 3.28e6, ("adj", "f32"): 347.77e6 + 4.70e6}
# lts__throughput.avg.pct_of_peak_sustained_elapsed and
# l1tex__throughput.avg.pct_of_peak_sustained_active of the same captures
NCU_L2_L1 = {("fwd", "f32"): (0.3361, 0.8428), ("adj", "f32"): (0.3519, 0.8919)}
# instruction issue peak: 152 SMs x 4 schedulers x 1 warp instruction per clock
# at the 2070 MHz maximum SM clock, in warp instructions per second
ISSUE_PEAK = 152 * 4 * 2.07e9


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--storage", default="f32", choices=["f32", "bf16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the video-batch and serving sections")
    ap.add_argument("--storage-section", action="store_true",
                    help="run the float32 / BF16 comparison even with --no-extras")
    ap.add_argument("--serving-jobs", type=int, default=500)
    ap.add_argument("--no-hull", action="store_true",
                    help="reconstruct the whole box instead of the visual hull (Sec. 4.3.1)")
    ap.add_argument("--no-skip", action="store_true", help="march empty bricks too (same result, slower)")
    ap.add_argument("--march", action="store_true",
                    help="march every iteration instead of building the ray weight tables (fr_params.tables = 1)")
    ap.add_argument("--profile-video", action="store_true",
                    help="run the video batch once with the profiler range around its timed graph only "
                         "(for ncu --profile-from-start off)")
    ap.add_argument("--profile", action="store_true",
                    help="untimed iterations of the step, for ncu captures")
    return ap.parse_args()


def dist_max(x: float) -> float:
    """Maximum of x over the ranks of the default process group (x itself when
    there is none); NCCL reduces on the GPU, gloo on the CPU."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(world_size: int, units_per_rank_step: float, steps: int, t_max: float) -> float:
    """Whole-job throughput of independent replicas: every rank processes the
    same units per step, timed by the slowest rank."""
    return world_size * units_per_rank_step * steps / t_max


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def alpha_for(n, views, side, step):
    """Paper-rule residual scale giving the same per-iteration gain across
    geometries: the adjustment gain grows with views x (pixels per voxel)^2 /
    step x (chord length in voxels), so alpha_l ~ n step / (views side^2),
    anchored at 2e-4 for 128^3, 8 views of 512^2, step 0.5."""
    return 2e-4 * (n / 128.0) * (step / 0.5) * (8.0 / views) * (512.0 / side) ** 2


def make_inputs(storage, rank, local):
    """Seeded ground truth, cameras and targets (rendered on the GPU from the
    ground truth with in-scattering, plus seeded pixel noise)."""
    import torch
    from paper_1809_06417_gb300 import flamerec as fr, synth
    w = WORKLOAD
    n = w["n"]
    shape, origin, h = synth.unit_grid(n)
    gt, albedo = synth.plume_volume(n, w["seed"] + 1000 * rank)
    cams = synth.ring_cameras(w["views"], w["side"], w["side"], elevation_jitter_deg=10.0, seed=w["seed"])
    dt = torch.float32 if storage == "f32" else torch.bfloat16
    ctx = fr.Context(local)
    gt_d = torch.as_tensor(gt, dtype=torch.float32, device="cuda").to(dt).contiguous()
    alb_d = torch.as_tensor(albedo, dtype=torch.float32, device="cuda").contiguous()
    src = torch.empty_like(gt_d)
    J = torch.empty((n, n, n, 4), device="cuda")
    ctx.fr_scatter_source(fr.volume(gt_d, origin, h), alb_d, J, fr.volume(src, origin, h))
    K, S = w["views"], w["side"]
    img = torch.empty((K, S, S, 3), device="cuda")
    fcams = fr.cameras(cams)
    ctx.fr_render(fr.volume(src, origin, h), fcams, fr.params(step=w["step"]), img)
    torch.cuda.synchronize()
    scale = float(img.max())
    img_np = synth.add_noise(img.cpu().numpy() / scale, w["noise"], w["seed"])
    targets = torch.as_tensor(img_np, dtype=torch.float32, device="cuda").contiguous()
    bbox = torch.zeros((K, 4), dtype=torch.int32, device="cuda")
    ctx.fr_prepare_targets(targets, 30 / 255, bbox)
    vol0 = gt_d.clone()
    vol0[..., :3] = 0  # the volume starts at zero (Sec. 3); extinction and albedo known
    # visual hull tags of the job, computed once from its flame masks (Sec. 4.3.1)
    tags = torch.zeros((n, n, n), dtype=torch.int32, device="cuda")
    ctx.fr_visual_hull(fr.volume(vol0, origin, h), fcams, targets, fr.params(), tags)
    del J, src
    return ctx, dict(origin=origin, h=h, cams=cams, fcams=fcams, targets=targets, bbox=bbox, albedo=alb_d,
                     vol0=vol0, gt=gt, gt_albedo=albedo, scale=scale, img_np=img_np, tags=tags)


def method_params(args, I):
    from paper_1809_06417_gb300 import flamerec as fr
    w = WORKLOAD
    hull = w["hull"] and not args.no_hull
    return fr.params(step=w["step"], alpha_l=w["alpha_l"], use_hull=int(hull),
                     hull_tags=I["tags"] if hull else None, skip_empty=int(not args.no_skip),
                     tables=1 if args.march else 0)


def run_ours(args, ws, rank, local):
    import torch
    import torch.distributed as dist
    from paper_1809_06417_gb300 import flamerec as fr
    torch.cuda.set_device(local)
    w = WORKLOAD
    K_IT = ITERS_PER_STEP
    ctx, I = make_inputs(args.storage, rank, local)
    p = method_params(args, I)
    vol = I["vol0"].clone()
    fv = fr.volume(vol, I["origin"], I["h"])
    cams = I["fcams"]
    stream = torch.cuda.current_stream()
    n_adj = ctx.fr_count_samples(fv, cams, p, residual=I["targets"])
    # forward samples the marches evaluate at the zero start (empty bricks skipped)
    n_fwd_before = ctx.fr_count_samples(fv, cams, p)
    flush = torch.empty(384 * 2 ** 20 // 4, dtype=torch.float32, device="cuda")  # > L2 (129 MB)
    rmse_dev = torch.zeros((K_IT, 3), device="cuda")

    def reset(i):
        # the job's start volume and an L2 flush, queued before the step's start event
        vol.copy_(I["vol0"])
        flush.fill_(float(i))

    def step():
        ctx.fr_reconstruct(fv, cams, I["targets"], I["bbox"], K_IT, p, albedo=I["albedo"], rmse=rmse_dev)

    for i in range(args.warmup):
        reset(i)
        step()
    torch.cuda.synchronize()
    stats = ctx.fr_table_stats()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with Clocks(local) as clk:
        t_wall = time.perf_counter()
        for i in range(args.steps):
            reset(i)
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    if ws > 1:
        dist.barrier()
    ms = [a.elapsed_time(b) for a, b in ev]
    t_dev = dist_max(sum(ms) / 1e3)
    rmse_step = rmse_dev.cpu().numpy()
    n_fwd_after = ctx.fr_count_samples(fv, cams, p)
    n_fwd = (n_fwd_before + n_fwd_after) // 2
    n_fwd_box = ctx.fr_count_samples(fv, cams, fr.params(step=w["step"], skip_empty=0))
    # per-phase device time from a second pass of as many steps, with the
    # events the library records on this stream between its launches (kept
    # out of the timed steps above)
    ctx.fr_trace_phases(True)
    for i in range(args.steps):
        reset(i)
        step()
    torch.cuda.synchronize()
    phase_ms, calls = ctx.fr_phase_times()
    ctx.fr_trace_phases(False)
    assert calls == args.steps, (calls, args.steps)
    phase_ms = {k: v / args.steps for k, v in phase_ms.items()}
    traced_ms = sum(phase_ms.values())
    t_fwd, t_adj = phase_ms["forward"] / K_IT / 1e3, phase_ms["adjust"] / K_IT / 1e3
    t_setup = phase_ms["setup"] / 1e3

    # the same job marching every iteration (fr_params.tables = 1), one timed
    # call after a warm-up, with its phases
    pm = method_params(args, I)
    pm.tables = 1
    reset(0)
    ctx.fr_reconstruct(fv, cams, I["targets"], I["bbox"], 2, pm, albedo=I["albedo"])
    reset(1)
    m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    m0.record(stream)
    ctx.fr_reconstruct(fv, cams, I["targets"], I["bbox"], K_IT, pm, albedo=I["albedo"])
    m1.record(stream)
    torch.cuda.synchronize()
    march_ms = m0.elapsed_time(m1)
    reset(2)
    ctx.fr_trace_phases(True)
    ctx.fr_reconstruct(fv, cams, I["targets"], I["bbox"], K_IT, pm, albedo=I["albedo"])
    torch.cuda.synchronize()
    march_phase, _ = ctx.fr_phase_times()
    ctx.fr_trace_phases(False)
    marching = {"ms_per_step": march_ms, "ms_per_iteration": march_ms / K_IT,
                "phase_ms_per_iteration": {k: v / K_IT for k, v in march_phase.items()},
                "note": "the same 50-iteration job with fr_params.tables = 1: the forward march and the "
                        "paper-rule adjustment over half rays every iteration"}

    # end to end through the C ABI with host buffers, every step: the start
    # volume (float32 records, pinned host memory) uploaded into a
    # library-held volume of the storage type, the pinned host targets copied
    # in by fr_reconstruct, the per-iteration RMSE and the reconstructed volume
    # read back.  The job's constants (albedo, flame boxes, hull tags) stay on
    # the device.
    vol_host = torch.as_tensor(I["vol0"].float().cpu()).pin_memory()
    vol_host_np = vol_host.numpy()
    out_host = torch.empty_like(vol_host).pin_memory()
    out_host_np = out_host.numpy()
    tgt_host = I["targets"].cpu().pin_memory()
    rmse_host = np.zeros((K_IT, 3), dtype=np.float32)
    lv = ctx.fr_volume_create((w["n"],) * 3, I["origin"], I["h"],
                              dtype=fr.FR_F32 if args.storage == "f32" else fr.FR_BF16)

    def e2e_step():
        ctx.fr_volume_upload(lv, vol_host_np)
        ctx.fr_reconstruct(lv, cams, tgt_host, I["bbox"], K_IT, p, albedo=I["albedo"], rmse=rmse_host,
                           targets_are_host=True)
        ctx.fr_volume_download(lv, out_host_np)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    torch.cuda.synchronize()
    t_e2e = dist_max(time.perf_counter() - t0)
    e2e_same = bool(np.allclose(out_host_np, vol.float().cpu().numpy(), rtol=0, atol=1e-4 * float(vol.abs().max())))
    ctx.fr_volume_free(lv)
    e2e_h2d = int(vol_host.numel() * 4 + I["targets"].numel() * 4)
    e2e_d2h = int(vol_host.numel() * 4 + K_IT * 12)

    # reconstruction quality after the job (context for the number)
    reset(0)
    step()
    torch.cuda.synchronize()
    rmse_now = rmse_dev.cpu().numpy()[-1:]

    # volume data error inside the hull (Sec. 5.1) against the ground truth's
    # emission on the targets' scale (the targets were divided by `scale`)
    ref = torch.as_tensor(I["gt"], dtype=torch.float32, device="cuda")
    ref[..., :3] /= I["scale"]
    full = (1 << w["views"]) - 1
    v_rmse, v_n = ctx.fr_volume_rmse(fv, fr.volume(ref.contiguous(), I["origin"], I["h"]), I["tags"], full)
    ref_max = float(ref[..., :3].max())
    del ref

    # the visual hull of the job (Sec. 4.3.1, Algorithm 1): the flame masks'
    # summed-area tables and the per-node tags, event-timed over 10 calls
    tags_h = torch.empty_like(I["tags"])
    ctx.fr_visual_hull(fv, cams, I["targets"], fr.params(), tags_h)
    h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h0.record(stream)
    for _ in range(10):
        ctx.fr_visual_hull(fv, cams, I["targets"], fr.params(), tags_h)
    h1.record(stream)
    torch.cuda.synchronize()
    hull_ms = h0.elapsed_time(h1) / 10
    hull_same = bool(torch.equal(tags_h, I["tags"]))
    del tags_h

    # the variants the paper mentions without using, on the same workload:
    # anisotropic in-scattering (Eq. 9) and sequential per-view updates
    variants = {}
    for name, kw in (("hg_g_0.5", dict(hg_g=0.5)), ("sequential_views", dict(sequential_views=1))):
        vol_v = I["vol0"].clone()
        fvv = fr.volume(vol_v, I["origin"], I["h"])
        pv = method_params(args, I)
        for k_, v_ in kw.items():
            setattr(pv, k_, v_)
        r_v = np.zeros((10, 3), dtype=np.float32)
        ctx.fr_reconstruct(fvv, cams, I["targets"], I["bbox"], 2, pv, albedo=I["albedo"])   # warm-up
        torch.cuda.synchronize()
        vol_v.copy_(I["vol0"])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.fr_reconstruct(fvv, cams, I["targets"], I["bbox"], 10, pv, albedo=I["albedo"], rmse=r_v)
        e1.record(stream)
        torch.cuda.synchronize()
        variants[name] = {"ms_per_iteration": e0.elapsed_time(e1) / 10, "rmse_first": [float(x) for x in r_v[0]],
                          "rmse_after_10": [float(x) for x in r_v[-1]]}
        del vol_v

    # the paper's stop criterion (Sec. 3): iterate from the initial volume until
    # the image error changes by less than 0.01 (on 0-255) between iterations,
    # the whole loop in one conditional CUDA graph
    vol_u = I["vol0"].clone()
    fu = fr.volume(vol_u, I["origin"], I["h"])
    max_u = 400
    r_u = np.zeros((max_u, 3), dtype=np.float32)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    n_u = ctx.fr_reconstruct_until(fu, cams, I["targets"], I["bbox"], max_u, 0.01, p, albedo=I["albedo"], rmse=r_u)
    t_u = time.perf_counter() - t0
    until = {"stop_delta": 0.01, "max_iters": max_u, "iterations": n_u, "seconds": t_u,
             "ms_per_iteration": 1e3 * t_u / max(n_u, 1), "rmse_first": [float(x) for x in r_u[0]],
             "rmse_last": [float(x) for x in r_u[max(n_u - 1, 0)]],
             "note": "wall time of one fr_reconstruct_until call, graph instantiation included"}

    storage_cmp = run_storage_comparison(fr, ctx, I, args) if not args.no_extras or args.storage_section else None
    ablation = run_ablation(fr, ctx, I, args)

    samples_step = (n_fwd + n_adj) * K_IT
    value = weak_value(ws, samples_step, args.steps, t_dev)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    # Roofline of the two per-iteration kernels.  Algorithmic bytes per launch
    # (one pass over what each must read and write): the forward reads its
    # table (8-byte entries, 0.4 GB: it cannot stay in L2 and streams from
    # HBM every iteration), the source records and the targets, and writes
    # each flame ray's residual (16 bytes); the adjustment reads its table,
    # the residuals, the hull's entry ends and key points (8 bytes each) and
    # reads and writes the hull's records.
    rec = 16 if args.storage == "f32" else 8
    nodes = w["n"] ** 3
    img_bytes = w["views"] * w["side"] ** 2 * 12
    f_ent, a_ent, n_flame, n_hull = (stats["forward_entries"], stats["adjustment_entries"], stats["flame_rays"],
                                     stats["hull_key_points"])
    kernels = {
        "fwd": dict(name="tab_forward_kernel (forward table: render + residual)", seconds=t_fwd,
                    compulsory={"forward_table_read": 8 * f_ent, "records_read": nodes * rec,
                                "targets_read": img_bytes, "flame_residuals_written": 16 * n_flame},
                    traffic=NCU_TRAFFIC.get(("fwd", args.storage)), l2_l1=NCU_L2_L1.get(("fwd", args.storage))),
        "adj": dict(name="tab_adjust_kernel (adjustment table: paper-rule update, Eqs. 10-11)", seconds=t_adj,
                    compulsory={"adjustment_table_read": 8 * a_ent, "flame_residuals_read": 16 * n_flame,
                                "hull_lists_read": 8 * n_hull, "hull_records_read_written": 2 * rec * n_hull},
                    traffic=NCU_TRAFFIC.get(("adj", args.storage)), l2_l1=NCU_L2_L1.get(("adj", args.storage))),
    }
    for K in kernels.values():
        K["compulsory_bytes"] = sum(K["compulsory"].values())
        K["hbm_frac"] = K["compulsory_bytes"] / K["seconds"] / 1e9 / hbm_peak if K["seconds"] > 0 else None
    dom = max(kernels, key=lambda k: kernels[k]["seconds"])
    K = kernels[dom]
    other = kernels["fwd" if dom == "adj" else "adj"]
    achieved = K["compulsory_bytes"] / K["seconds"] / 1e9
    roofline = {
        "bound": "hbm", "kernel": K["name"], "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
        "frac": achieved / hbm_peak, "traffic": K["traffic"],
        "algorithmic_bytes_per_launch": K["compulsory_bytes"], "algorithmic_bytes": K["compulsory"],
        "launch_ms": 1e3 * K["seconds"], "launches_per_step": K_IT,
        "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks else "fallback 6.8 TB/s",
        "l2_l1_frac": K["l2_l1"],
        "other_kernel": {"name": other["name"], "hbm_frac": other["hbm_frac"], "launch_ms": 1e3 * other["seconds"],
                         "algorithmic_bytes_per_launch": other["compulsory_bytes"], "traffic": other["traffic"]},
        "tables": {"forward_entries": f_ent, "adjustment_entries": a_ent, "flame_rays": n_flame,
                   "hull_key_points": n_hull, "bytes": 8 * (f_ent + a_ent) + 16 * n_flame,
                   "build_ms_per_step": 1e3 * t_setup},
        "note": "achieved = algorithmic bytes of one launch (tables, records, images, residuals) over its "
                "event-timed duration against the measured HBM copy bandwidth; the tables stream from HBM "
                "every iteration, the 128^3 records stay in the 129 MB L2",
    }
    launches = KERNELS_SETUP + KERNELS_PER_ITERATION * K_IT if f_ent else None

    out = {
        "metric": METRIC,
        "value": value,
        "unit": "samples/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * t_dev / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": w["name"], "grid": [w["n"]] * 3, "views": w["views"], "image": [w["side"]] * 2,
                   "step_vox": w["step"], "storage": args.storage, "rule": "paper", "scattering": True,
                   "visual_hull": bool(p.use_hull), "skip_empty_bricks": bool(p.skip_empty),
                   "iterations_per_step": K_IT, "ray_weight_tables": bool(f_ent),
                   "l2": "flushed before every timed step (384 MiB write); inside a step the ray weight tables "
                         "(larger than L2) stream from HBM every iteration",
                   "parallelism": f"replicas{ws}"},
        "recon_iters_per_s": ws * args.steps * K_IT / t_dev,
        "ms_per_iteration": 1e3 * t_dev / args.steps / K_IT,
        "samples_per_iteration": {"fwd": n_fwd, "adj": n_adj, "fwd_before": n_fwd_before, "fwd_after": n_fwd_after,
                                  "fwd_all_in_box": n_fwd_box,
                                  "note": "the samples the marches evaluate per iteration (empty bricks skipped); "
                                          "the tables hold the same samples' weights per ray and key point"},
        "kernel_ms": {"fwd_residual": 1e3 * t_fwd, "adjust_update": 1e3 * t_adj, "tables_build": 1e3 * t_setup},
        "phase_ms_per_step": phase_ms,
        "traced_ms_per_step": traced_ms,
        "marching": marching,
        "e2e": {"value": weak_value(ws, samples_step, args.steps, t_e2e), "unit": "samples/s",
                "h2d_bytes_per_step": e2e_h2d, "d2h_bytes_per_step": e2e_d2h,
                "ms_per_step": 1e3 * t_e2e / args.steps, "same_volume_as_device_path": e2e_same,
                "path": "fr_volume_upload (float32 host records) -> fr_reconstruct (50 iterations, host targets, "
                        "host rmse) -> fr_volume_download (float32 host records), pinned host memory, every step"},
        "gpu_launches": None if launches is None else launches * args.steps,
        "roofline": roofline,
        "clocks": clk.summary(),
        "rmse_first": [float(x) for x in rmse_step[0]],
        "rmse_after": [float(x) for x in rmse_now[0]],
        "until_converged": until,
        "visual_hull": {"ms": hull_ms, "views": w["views"], "grid": [w["n"]] * 3, "image": [w["side"]] * 2,
                        "same_tags_as_setup": hull_same},
        "variants": variants,
        "storage_f32_vs_bf16": storage_cmp,
        "ablation": ablation,
        "volume_rmse_in_hull": {"rmse": [float(x) for x in v_rmse], "key_points": v_n,
                                "relative_to_max": [float(x) / ref_max for x in v_rmse],
                                "after_iterations": K_IT},
        "wall_s": t_wall,
    }
    ctx.close()
    return out


def run_storage_comparison(fr, ctx, I, args, iters=50):
    """The full-RTE configuration as stated: `iters` iterations from the zero
    start with float32 records and with BF16 records (float32 arithmetic), on
    the same targets, hull and parameters, each run as one fr_reconstruct call
    timed with CUDA events; per storage the per-iteration time, the image error
    of the first and last iteration, and the volume data error inside the hull
    against the ground truth on the targets' scale (Sec. 5.1)."""
    import torch
    w = WORKLOAD
    stream = torch.cuda.current_stream()
    ref = torch.as_tensor(I["gt"], dtype=torch.float32, device="cuda")
    ref[..., :3] /= I["scale"]
    fref = fr.volume(ref.contiguous(), I["origin"], I["h"])
    ref_max = float(ref[..., :3].max())
    full = (1 << w["views"]) - 1
    p = method_params(args, I)
    out, vols = {}, {}
    for name, dt in (("f32", torch.float32), ("bf16", torch.bfloat16)):
        warm = I["vol0"].float().to(dt).clone()
        ctx.fr_reconstruct(fr.volume(warm, I["origin"], I["h"]), I["fcams"], I["targets"], I["bbox"], 2, p,
                           albedo=I["albedo"])
        vol = I["vol0"].float().to(dt).clone()    # (a copy: I["vol0"] itself stays the start)
        fv = fr.volume(vol, I["origin"], I["h"])
        rmse = torch.zeros((iters, 3), device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        ctx.fr_reconstruct(fv, I["fcams"], I["targets"], I["bbox"], iters, p, albedo=I["albedo"], rmse=rmse)
        e1.record(stream)
        torch.cuda.synchronize()
        r = rmse.cpu().numpy()
        v_rmse, _ = ctx.fr_volume_rmse(fv, fref, I["tags"], full)
        out[name] = {"ms_per_iteration": e0.elapsed_time(e1) / iters, "rmse_first": [float(x) for x in r[0]],
                     "rmse_last": [float(x) for x in r[-1]],
                     "volume_rmse_in_hull": [float(x) for x in v_rmse],
                     "volume_rmse_in_hull_relative_to_max": [float(x) / ref_max for x in v_rmse]}
        vols[name] = (vol, fv)
        del warm
    d, _ = ctx.fr_volume_rmse(vols["f32"][1], vols["bf16"][1], I["tags"], full)
    out["bf16_minus_f32_volume_rmse_in_hull_relative_to_max"] = [float(x) / ref_max for x in d]
    out["iterations"] = iters
    out["speedup_bf16"] = out["f32"]["ms_per_iteration"] / out["bf16"]["ms_per_iteration"]
    return out


def run_ablation(fr, ctx, I, args, iters=ITERS_PER_STEP):
    """Per-iteration time of the step with parts of the method turned off,
    beside the headline: marching every iteration instead of the ray weight
    tables (same result up to float32 rounding), without empty-brick skipping
    (the marches then evaluate every sample in the box; the tables need the
    hull's bricks) and without the visual hull (the whole box reconstructed).
    One fr_reconstruct call of `iters` iterations each from the zero start,
    timed with CUDA events."""
    import torch
    w = WORKLOAD
    stream = torch.cuda.current_stream()
    out = {}
    for name, kw in (("default", {}), ("no_tables", dict(tables=1)), ("no_skip", dict(skip_empty=0)),
                     ("no_hull", dict(use_hull=0)), ("no_hull_no_skip", dict(use_hull=0, skip_empty=0))):
        p = fr.params(step=w["step"], alpha_l=w["alpha_l"], use_hull=1, hull_tags=I["tags"], skip_empty=1)
        for k, v in kw.items():
            setattr(p, k, v)
        if not p.use_hull:
            p.hull_tags = None
        vol = I["vol0"].clone()
        fv = fr.volume(vol, I["origin"], I["h"])
        ctx.fr_reconstruct(fv, I["fcams"], I["targets"], I["bbox"], 2, p, albedo=I["albedo"])
        vol.copy_(I["vol0"])
        rmse = np.zeros((iters, 3), dtype=np.float32)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        ctx.fr_reconstruct(fv, I["fcams"], I["targets"], I["bbox"], iters, p, albedo=I["albedo"], rmse=rmse)
        e1.record(stream)
        torch.cuda.synchronize()
        out[name] = {"ms_per_iteration": e0.elapsed_time(e1) / iters, "rmse_last": [float(x) for x in rmse[-1]]}
        del vol
    out["iterations"] = iters
    return out


def run_video(fr, ctx, frames=64, n=96, views=8, side=384, iters=20, step=0.5, seed=4, storage="f32",
              profile=False):
    """Batched video frames: every frame reconstructed from its own targets,
    all frames in one batched launch per phase, the 20 iterations captured in
    one CUDA graph."""
    import torch
    from paper_1809_06417_gb300 import synth
    dt = torch.float32 if storage == "f32" else torch.bfloat16
    shape, origin, h = synth.unit_grid(n)
    cams = synth.ring_cameras(views, side, side, elevation_jitter_deg=10.0, seed=seed)
    fcams = fr.cameras(cams)
    gts = synth.video_frames(frames, n, seed)
    # each frame restricted to its own visual hull (Sec. 4.3.1), empty bricks skipped
    p = fr.params(step=step, alpha_l=alpha_for(n, views, side, step), use_hull=1)
    probs, vols, n_fwd, n_adj = [], [], 0, 0
    for f, gt in enumerate(gts):
        g = torch.as_tensor(gt, dtype=torch.float32, device="cuda").to(dt).contiguous()
        img = torch.empty((views, side, side, 3), device="cuda")
        ctx.fr_render(fr.volume(g, origin, h), fcams, fr.params(step=step), img)
        img /= img.max()
        bbox = torch.zeros((views, 4), dtype=torch.int32, device="cuda")
        ctx.fr_prepare_targets(img, 30 / 255, bbox)
        v = g.clone()
        v[..., :3] = 0
        fv = fr.volume(v, origin, h)
        n_fwd += ctx.fr_count_samples(fv, fcams, fr.params(step=step, skip_empty=0))
        n_adj += ctx.fr_count_samples(fv, fcams, p, residual=img)
        rm = torch.zeros((iters, 3), device="cuda")
        vols.append((v, img, bbox, rm))
        probs.append((fv, fcams, img, bbox, rm))
    ctx.fr_reconstruct_batch(probs, 1, p, use_graph=False)  # warm-up (builds scratch)
    torch.cuda.synchronize()
    for v, *_ in vols:
        v[..., :3] = 0
    flush = torch.empty(384 * 2 ** 20 // 4, device="cuda")
    flush.fill_(1.0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    if profile:
        torch.cuda.profiler.start()
    e0.record(stream)
    ctx.fr_reconstruct_batch(probs, iters, p, use_graph=True)
    e1.record(stream)
    torch.cuda.synchronize()
    if profile:
        torch.cuda.profiler.stop()
    t = e0.elapsed_time(e1) / 1e3
    final = np.stack([rm[-1].cpu().numpy() for *_, rm in vols])
    return {"workload": f"video_{frames}x{n}^3_{views}x{side}^2", "frames": frames, "iters_per_frame": iters,
            "seconds": t, "frames_per_s": frames / t,
            "nominal_samples_per_s": (n_fwd + n_adj) * iters / t,   # every in-box sample, skipped ones included
            "samples_per_iteration": {"fwd_all_in_box": n_fwd, "adj_flame_rays": n_adj}, "graph": True,
            "storage": storage, "visual_hull": True,
            "final_rmse_mean": [float(x) for x in final.mean(axis=0)], "launches_per_iteration": 7}


def run_serving(fr, ctx, jobs=500, rate=20.0, seed=5, step=0.5, warmup_s=10.0, pool=64):
    """The serving configuration: reconstruction jobs arrive as a seeded
    Poisson stream at `rate` jobs/s -- `warmup_s` seconds of warm-up jobs, then
    `jobs` measured ones -- each with a grid from {64, 96, 128, 192}^3, 4-12
    views, image side 256-768 and 20-50 iterations, BF16 records, its own
    visual hull, through the continuous-batching server.  A job's scene (grid,
    cameras, targets) comes from a pool of `pool` seeded scenes drawn from the
    same distribution, rendered once up front (host memory); its arrival time
    and iteration count are its own.

    Reported: p50 / p99 latency from arrival (the loop's clock, so waiting for
    a step in flight counts) and service time on the server, throughput while
    the measured jobs were in the system, and, on the measured jobs alone: the
    capacity (all submitted at once to a fresh server) against the plain
    single-job float32 path (fr_reconstruct, one job after another, frames and
    records from host memory as for the server), with each arm's final image
    error (green, 0-255) to compare them at matched error."""
    import torch
    from paper_1809_06417_gb300 import serving, synth
    n_warm = int(round(warmup_s * rate))
    stream = synth.serving_stream(n_warm + jobs, seed=seed, rate=rate)
    plumes, scenes = {}, []
    for js in stream[:pool]:
        n, K, side = js["n"], js["views"], js["side"]
        if n not in plumes:
            plumes[n] = synth.plume_volume(n, seed + n)[0]
        gt = plumes[n]
        shape, origin, h = synth.unit_grid(n)
        cams = synth.ring_cameras(K, side, side, elevation_jitter_deg=10.0, seed=js["seed"], phase=0.1 * js["id"])
        g = torch.as_tensor(gt, dtype=torch.float32, device="cuda").contiguous()
        img = torch.empty((K, side, side, 3), device="cuda")
        ctx.fr_render(fr.volume(g, origin, h), fr.cameras(cams), fr.params(step=step), img)
        img /= img.max()
        init = gt.copy()
        init[..., :3] = 0.0
        scenes.append(dict(n=n, shape=shape, origin=origin, h=h, cams=cams, targets=img.cpu().numpy(),
                           init32=init.astype(np.float32),
                           init16=torch.as_tensor(init, dtype=torch.float32).to(torch.bfloat16)
                           .view(torch.int16).numpy().view(np.uint16).copy(),
                           alpha=alpha_for(n, K, side, step)))
        del g, img
    specs = [dict(js=js, **scenes[i % pool]) for i, js in enumerate(stream)]
    p = fr.params(step=step, alpha_l=2e-4, use_hull=1)   # each job in its own visual hull

    def submitter(sp):
        return lambda srv: srv.submit(sp["shape"], sp["origin"], sp["h"], sp["cams"], sp["js"]["iters"],
                                      sp["init16"], sp["targets"], alpha_l=sp["alpha"])

    # online: Poisson arrivals, continuous batching
    srv = fr.Server(ctx, p, dtype=fr.FR_BF16)
    reqs = [serving.Request(arrival=sp["js"]["arrival"] - stream[0]["arrival"], submit=submitter(sp),
                            warmup=i < n_warm) for i, sp in enumerate(specs)]
    res = serving.run_requests(srv, reqs)
    measured = [r for r in reqs if not r.warmup]
    online_rmse = np.mean([r.job.rmse[-1, 1] for r in measured])
    srv.close()
    meas_specs = specs[n_warm:]
    # capacity: the measured jobs all submitted at once to a fresh server (bf16)
    srv = fr.Server(ctx, p, dtype=fr.FR_BF16)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    handles = [submitter(sp)(srv) for sp in meas_specs]
    for j in handles:
        j.wait(timeout_ms=1800000)
    t_batched = time.perf_counter() - t0
    rmse_batched = np.array([j.rmse[-1, 1] for j in handles])
    srv.close()
    del handles
    # the plain single-job path: one job after another through fr_reconstruct
    # (float32), frames and records from host memory, the result read back
    t0 = time.perf_counter()
    rmse_single = []
    for sp in meas_specs:
        K, side = len(sp["cams"]), sp["cams"][0]["width"]
        v = torch.as_tensor(sp["init32"], device="cuda").contiguous()
        t = torch.as_tensor(sp["targets"], device="cuda").contiguous()
        bbox = torch.zeros((K, 4), dtype=torch.int32, device="cuda")
        ctx.fr_prepare_targets(t, 30 / 255, bbox)
        rm = np.zeros((sp["js"]["iters"], 3), dtype=np.float32)
        ctx.fr_reconstruct(fr.volume(v, sp["origin"], sp["h"]), fr.cameras(sp["cams"]), t, bbox, sp["js"]["iters"],
                           fr.params(step=step, alpha_l=sp["alpha"], use_hull=1), rmse=rm)
        v.cpu()
        rmse_single.append(rm[-1, 1])
    torch.cuda.synchronize()
    t_single = time.perf_counter() - t0
    rmse_single = np.array(rmse_single)
    return {"workload": f"serving_poisson{rate:g}_jobs{jobs}_warmup{warmup_s:g}s", "jobs": jobs,
            "warmup_jobs": n_warm, "rate_jobs_per_s": rate, "scene_pool": pool,
            "p50_latency_s": res.percentile(50), "p99_latency_s": res.percentile(99),
            "p50_service_s": res.percentile(50, res.services), "p99_service_s": res.percentile(99, res.services),
            "jobs_per_s_in_system": res.throughput(), "max_resident": res.max_running, "steps": res.steps,
            "online_final_rmse_green_mean": float(online_rmse),
            "latency_note": "latency from each job's arrival to the end of the server step that completed it "
                            "(loop clock); service from submission to completion (server clock)",
            "capacity": {"batched_bf16_jobs_per_s": jobs / t_batched, "single_f32_jobs_per_s": jobs / t_single,
                         "speedup": t_single / t_batched,
                         "final_rmse_green_mean_batched_bf16": float(rmse_batched.mean()),
                         "final_rmse_green_mean_single_f32": float(rmse_single.mean()),
                         "rmse_ratio_bf16_over_f32": float(rmse_batched.mean() / rmse_single.mean()),
                         "note": "the measured jobs all submitted at t = 0 (saturating arrivals)"},
            "storage": "bf16", "visual_hull": True,
            "mix": "grids {64,96,128,192}^3, 4-12 views, side 256-768, 20-50 iterations"}


def run_temperature_views(fr, ctx, n=128, side=512, step=0.5, iters=50, seed=3, view_counts=(4, 16, 28),
                          t_min=1000.0, t_max=2300.0, alpha_scale=1.0, sigma=None):
    """Paper-literal temperature path (Sec. 3.3.3) against the number of cameras
    (Sec. 5.2: 4, 16 and 28 cameras, temperatures in 1000-2300 K):
    targets rendered from a seeded temperature field through the colour-
    temperature table, the green channel reconstructed with the paper rule
    inside the visual hull, the temperature read off the table; errors inside
    the hull (Sec. 5.1), and on the key points inside every camera set's hull.
    sigma: the constant extinction per voxel length (default the paper's
    tau = 0.05 at a one-voxel step)."""
    import torch
    from paper_1809_06417_gb300 import synth
    sigma = synth.SIGMA_PAPER if sigma is None else sigma
    lut = torch.zeros((1024, 4), device="cuda")
    ctx.fr_planck_lut(t_min, t_max, lut)
    pt = dict(lut=lut, lut_t_min=t_min, lut_t_max=t_max)
    gt = synth.temperature_volume(n, seed, t_min=t_min, t_max=t_max, sigma=sigma)
    shape, origin, h = synth.unit_grid(n)
    g = torch.as_tensor(gt, dtype=torch.float32, device="cuda").contiguous()
    out, temps, hulls = {}, {}, {}
    for views in view_counts:
        cams = synth.ring_cameras(views, side, side, elevation_jitter_deg=10.0, seed=seed)
        fc = fr.cameras(cams)
        img = torch.zeros((views, side, side, 3), device="cuda")
        ctx.fr_render(fr.volume(g, origin, h, kind=fr.FR_KIND_TEMP), fc, fr.params(step=step, **pt), img)
        thresh = 30 / 255 * float(img.max())
        bbox = torch.zeros((views, 4), dtype=torch.int32, device="cuda")
        ctx.fr_prepare_targets(img, thresh, bbox)
        rec = torch.zeros((n, n, n, 4), device="cuda")
        rec[..., 3] = g[..., 1]
        fv = fr.volume(rec, origin, h)
        tags = torch.zeros((n, n, n), dtype=torch.int32, device="cuda")
        ctx.fr_visual_hull(fv, fc, img, fr.params(flame_thresh=thresh), tags)
        p = fr.params(step=step, alpha_l=alpha_scale * alpha_for(n, views, side, step), flame_thresh=thresh,
                      use_hull=1, hull_tags=tags)
        rmse = np.zeros((iters, 3), dtype=np.float32)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.fr_reconstruct(fv, fc, img, bbox, iters, p, rmse=rmse)
        temp = torch.zeros((n, n, n, 2), device="cuda")
        ctx.fr_temperature_from_green(fv, fr.params(**pt), fr.volume(temp, origin, h, kind=fr.FR_KIND_TEMP))
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        temps[views] = temp.cpu().numpy()[..., 0]
        hulls[views] = tags.cpu().numpy().view(np.uint32) == (1 << views) - 1
        inside = hulls[views]
        out[views] = {"seconds": dt, "hull_key_points": int(inside.sum()),
                      "temperature_rmse_in_hull_K": float(np.sqrt(np.mean((temps[views][inside] -
                                                                             gt[..., 0][inside]) ** 2))),
                      "green_image_rmse_first_last": [float(rmse[0, 1]), float(rmse[-1, 1])]}
    common = np.logical_and.reduce([hulls[v] for v in view_counts])
    for views in view_counts:
        out[views]["temperature_rmse_in_all_hulls_K"] = float(
            np.sqrt(np.mean((temps[views][common] - gt[..., 0][common]) ** 2)))
    return {"workload": f"temperature_green_{n}^3_{side}^2_{iters}it", "range_K": [t_min, t_max],
            "sigma_per_voxel": sigma, "common_key_points": int(common.sum()),
            "views": {str(k): v for k, v in out.items()}}


def run_held_out(fr, ctx, n=128, views=10, side=512, step=0.5, iters=50, seed=2):
    """The paper's extra evaluation: reconstruct from nine of ten views (full
    RTE, visual hull) and render the tenth, which the reconstruction never saw."""
    import torch
    from paper_1809_06417_gb300 import synth
    shape, origin, h = synth.unit_grid(n)
    gt, albedo = synth.plume_volume(n, seed)
    cams = synth.ring_cameras(views, side, side, elevation_jitter_deg=10.0, seed=seed)
    g = torch.as_tensor(gt, dtype=torch.float32, device="cuda").contiguous()
    alb = torch.as_tensor(albedo, dtype=torch.float32, device="cuda").contiguous()
    src = torch.empty_like(g)
    J = torch.empty((n, n, n, 4), device="cuda")
    ctx.fr_scatter_source(fr.volume(g, origin, h), alb, J, fr.volume(src, origin, h))
    img = torch.zeros((views, side, side, 3), device="cuda")
    ctx.fr_render(fr.volume(src, origin, h), fr.cameras(cams), fr.params(step=step), img)
    img /= img.max()
    k = views - 1
    t_in, t_out = img[:k].contiguous(), img[k:].contiguous()
    b_in = torch.zeros((k, 4), dtype=torch.int32, device="cuda")
    b_out = torch.zeros((1, 4), dtype=torch.int32, device="cuda")
    ctx.fr_prepare_targets(t_in, 30 / 255, b_in)
    ctx.fr_prepare_targets(t_out, 30 / 255, b_out)
    c_in, c_out = fr.cameras(cams[:k]), fr.cameras(cams[k:])
    v = g.clone()
    v[..., :3] = 0.0
    fv = fr.volume(v, origin, h)

    def view_rmse(cams_, targets, bbox):
        s_ = torch.empty((4,), device="cuda")
        res = torch.empty_like(targets)
        ren = torch.empty_like(targets)
        s_.zero_()
        # the test view is rendered with in-scattering from the current volume
        ctx.fr_scatter_source(fv, alb, J, fr.volume(src, origin, h))
        ctx.fr_render_residual(fr.volume(src, origin, h), cams_, fr.params(step=step), targets, bbox, ren, res, s_)
        q = s_.cpu().numpy().astype(np.float64)
        return [float(x) for x in 255.0 * np.sqrt(q[:3] / max(q[3], 1.0))]

    before = view_rmse(c_out, t_out, b_out)
    p = fr.params(step=step, alpha_l=alpha_for(n, k, side, step), use_hull=1)
    rmse = np.zeros((iters, 3), dtype=np.float32)
    ctx.fr_reconstruct(fv, c_in, t_in, b_in, iters, p, albedo=alb, rmse=rmse)
    after = view_rmse(c_out, t_out, b_out)
    fit = view_rmse(c_in, t_in, b_in)
    return {"workload": f"held_out_{n}^3_{k}+1x{side}^2_{iters}it", "test_view_rmse_before": before,
            "test_view_rmse_after": after, "input_views_rmse_after": fit,
            "input_views_rmse_first": [float(x) for x in rmse[0]]}


def run_differentiable(fr, ctx, n=128, views=8, side=512, step=0.5, seed=3, reps=5):
    """The differentiable temperature path (C3): forward render through the
    colour-temperature table and the exact backward through
    torch.autograd.Function, timed with CUDA events (median of reps)."""
    import torch
    from paper_1809_06417_gb300 import autograd as ag, synth
    shape, origin, h = synth.unit_grid(n)
    lut = torch.zeros((4096, 4), device="cuda")
    ctx.fr_planck_lut(800.0, 2000.0, lut)
    cams = synth.ring_cameras(views, side, side, elevation_jitter_deg=10.0, seed=seed)
    scene = ag.RenderScene(ctx, cams, origin, h, kind=fr.FR_KIND_TEMP, step=step, lut=lut,
                           lut_t_min=800.0, lut_t_max=2000.0)
    vol = torch.as_tensor(synth.temperature_volume(n, seed), dtype=torch.float32,
                          device="cuda").requires_grad_(True)
    w = torch.randn(scene.image_shape, device="cuda")
    stream = torch.cuda.current_stream()
    fwd_ms, bwd_ms = [], []
    for i in range(reps + 1):
        vol.grad = None
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        img = ag.render(vol, scene)
        e1.record(stream)
        (img * w).sum().backward()
        e2.record(stream)
        torch.cuda.synchronize()
        if i:
            fwd_ms.append(e0.elapsed_time(e1))
            bwd_ms.append(e1.elapsed_time(e2))
    n_fwd = ctx.fr_count_samples(scene.volume(vol.detach()), scene.fcams, scene.params)
    return {"workload": f"temperature_autograd_{n}^3_{views}x{side}^2", "forward_ms": statistics.median(fwd_ms),
            "backward_ms": statistics.median(bwd_ms), "samples_per_pass": n_fwd,
            "backward_samples_per_s": n_fwd / (statistics.median(bwd_ms) / 1e3),
            "note": "backward includes the loss and torch's reduction kernels around fr_render_backward"}


class OracleWorkload:
    """The oracle on the benchmarked workload itself: the same seeded plume,
    cameras, noise, hull and parameters, targets rendered by the oracle, the
    volume starting at zero emission and advanced one fr_reconstruct-like
    iteration per step (in-scattering source, render, residual, adjustment,
    update inside the hull).  Set-up runs outside the timed steps."""

    def __init__(self, threads):
        import oracle as orc
        from paper_1809_06417_gb300 import synth
        self.orc = orc
        w = WORKLOAD
        n = w["n"]
        orc.set_threads(threads)
        shape, origin, h = synth.unit_grid(n)
        gt, self.albedo = synth.plume_volume(n, w["seed"])
        cams = synth.ring_cameras(w["views"], w["side"], w["side"], elevation_jitter_deg=10.0, seed=w["seed"])
        self.sc = orc.Scene(shape, origin, h, cams)
        self.P = orc.make_params(step=w["step"], alpha_l=w["alpha_l"])
        src = orc.scatter_source(gt, self.albedo, orc.scatter_J(self.sc, gt))
        img, _ = orc.render(self.sc, src, self.P)
        img = synth.add_noise(img / img.max(), w["noise"], w["seed"])
        self.targets, self.mask, self.bbox = orc.prepare_targets(img, 30 / 255)
        self.tags = orc.visual_hull(self.sc, self.mask)
        self.vol = gt.copy()
        self.vol[..., :3] = 0.0
        self.it = 0

    def step(self, threads):
        """One iteration on `threads` threads: (samples, seconds)."""
        self.orc.set_threads(threads)
        t0 = time.perf_counter()
        self.vol, _, (nf, na) = self.orc.reconstruct(self.sc, self.vol, self.P, self.targets, self.mask, self.bbox, 1,
                                                     albedo=self.albedo, first_iteration=self.it, hull=self.tags)
        dt = time.perf_counter() - t0
        self.it += 1
        return nf + na, dt


def oracle_tiny(threads, iters=10):
    """The tiny configuration (32^3, 4 views of 64^2, step 1, 10 iterations)
    through the oracle, timed in full: (samples, seconds)."""
    import oracle as orc
    from paper_1809_06417_gb300 import synth
    orc.set_threads(threads)
    n = 32
    shape, origin, h = synth.unit_grid(n)
    cams = synth.ring_cameras(4, 64, 64, seed=1)
    gt = synth.blobs_volume(n, 1)
    sc = orc.Scene(shape, origin, h, cams)
    P = orc.make_params(step=1.0, alpha_l=0.01)
    img, _ = orc.render(sc, gt, P)
    t, mask, bbox = orc.prepare_targets(synth.add_noise(img / img.max(), 1e-3, 1), 30 / 255)
    v0 = gt.copy()
    v0[..., :3] = 0.0
    t0 = time.perf_counter()
    _, _, (nf, na) = orc.reconstruct(sc, v0, P, t, mask, bbox, iters)
    return nf + na, time.perf_counter() - t0


def cpu_baseline(full_iters=3):
    """The oracle, as it stands, on the machine's host cores: the benchmarked
    workload over `full_iters` whole iterations on every core (OpenMP), one
    whole iteration on one core, and the tiny configuration's 10 iterations on
    both."""
    cores = os.cpu_count() or 1
    wl = OracleWorkload(cores)
    n_all = t_all = 0
    for _ in range(full_iters):
        n_, t_ = wl.step(cores)
        n_all += n_
        t_all += t_
    n_one, t_one = wl.step(1)
    tn_all, tt_all = oracle_tiny(cores)
    tn_one, tt_one = oracle_tiny(1)
    import oracle as orc
    orc.set_threads(1)
    return {"value": n_all / t_all, "unit": "samples/s", "cores": cores, "kind": "oracle",
            "sample": f"{WORKLOAD['name']}: {full_iters} whole iterations (in-scattering source, render of every "
                      f"pixel, residual, adjustment of every flame ray, update inside the hull) on {cores} threads, "
                      f"{n_all} samples in {t_all:.1f} s",
            "iterations_per_s": full_iters / t_all,
            "single_core": {"value": n_one / t_one, "unit": "samples/s", "cores": 1,
                            "sample": f"one whole iteration, {n_one} samples in {t_one:.1f} s",
                            "iterations_per_s": 1.0 / t_one},
            "tiny_10_iterations": {"all_cores_s": tt_all, "single_core_s": tt_one, "samples": tn_all,
                                   "cores": cores}}


def run_profile(args):
    """The command the ncu captures use: the workload's inputs, then one
    benchmarked step (one fr_reconstruct call of ITERS_PER_STEP iterations,
    the same launches as a timed step), no timing or L2 flush.  Launches:
    make_inputs renders the ground truth once (fwd_single) and computes the
    hull; the step then launches KERNELS_SETUP kernels and
    KERNELS_PER_ITERATION per iteration."""
    import torch
    from paper_1809_06417_gb300 import flamerec as fr
    ctx, I = make_inputs(args.storage, 0, 0)
    p = method_params(args, I)
    vol = I["vol0"].clone()
    fv = fr.volume(vol, I["origin"], I["h"])
    rmse = np.zeros((ITERS_PER_STEP, 3), dtype=np.float32)
    ctx.fr_reconstruct(fv, I["fcams"], I["targets"], I["bbox"], ITERS_PER_STEP, p, albedo=I["albedo"], rmse=rmse)
    torch.cuda.synchronize()
    print(json.dumps({"profile": "ok", "iterations": ITERS_PER_STEP, "rmse_last": [float(x) for x in rmse[-1]],
                      "tables": ctx.fr_table_stats()}))
    ctx.close()


def run_reference(args, ws, rank):
    """The reference arm: the oracle (the paper ships no code) on the same
    workload, metric and unit, every host core, one whole iteration per step."""
    if rank != 0:
        return None
    cores = os.cpu_count() or 1
    wl = OracleWorkload(cores)
    tot_n, tot_t = 0, 0.0
    for i in range(args.warmup + args.steps):
        n, dt = wl.step(cores)
        if i >= args.warmup:
            tot_n += n
            tot_t += dt
    v = tot_n / tot_t
    w = WORKLOAD
    return {"metric": METRIC, "value": v, "unit": "samples/s", "impl": "reference", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": w["name"], "grid": [w["n"]] * 3, "views": w["views"], "image": [w["side"]] * 2,
                       "step_vox": w["step"], "storage": "f64", "rule": "paper", "scattering": True,
                       "visual_hull": True, "parallelism": f"cpu{cores}"},
            "recon_iters_per_s": args.steps / tot_t,
            "cpu_baseline": {"value": v, "unit": "samples/s", "cores": cores, "kind": "oracle",
                             "sample": "one whole iteration of the workload per step (every pixel rendered, every "
                                       "flame ray adjusted), OpenMP over pixel rows"},
            "e2e": {"value": v, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    ws, rank, local = dist_setup()
    if args.profile:
        run_profile(args)
        return
    if args.profile_video:
        from paper_1809_06417_gb300 import flamerec as fr
        ctx = fr.Context(local)
        r = run_video(fr, ctx, storage=args.storage, profile=True)
        print(json.dumps({"frames_per_s": r["frames_per_s"], "seconds": r["seconds"]}))
        ctx.close()
        return
    if args.impl == "reference":
        out = run_reference(args, ws, rank)
        if out is not None:
            print(json.dumps(out))
        return
    if ws > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline()  # before any GPU work: the oracle never forks after CUDA init
    out = run_ours(args, ws, rank, local)
    if rank == 0 and not args.no_extras:
        from paper_1809_06417_gb300 import flamerec as fr, synth
        ctx = fr.Context(local)
        out["video"] = run_video(fr, ctx, storage=args.storage)
        out["serving"] = run_serving(fr, ctx, jobs=args.serving_jobs)
        out["temperature_views"] = run_temperature_views(fr, ctx)
        # the same at the optical depth the paper's extinction gives a 48^3 grid
        out["temperature_views_thin"] = run_temperature_views(fr, ctx, sigma=synth.SIGMA_PAPER * 48.0 / 128.0)
        out["held_out_view"] = run_held_out(fr, ctx)
        out["differentiable"] = run_differentiable(fr, ctx)
        ctx.close()
    if rank == 0:
        out["cpu_baseline"] = cpu
        print(json.dumps(out))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
