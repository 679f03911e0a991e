"""Benchmark of the differentiable RGB-D splatting hot path on one GB300.

Default workload (the Replica-shaped mapping step): 300k Gaussians with SH
degree 3 in a synthetic 8x6x3 m room, one 1200x680 view (fx = fy = 600).  A step
is the whole hot path: forward render (projection, binning, depth sort,
compositing), the L1 colour + depth loss adjoint, and the backward to every
Gaussian parameter and the 6-DoF twist, gradients zeroed first.

Metric: fwd+bwd Mpixel/s = pixels per step / device time per step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

`--impl reference` times the FP64 CPU oracle (the baseline arm) on a bounded
pixel sample of the same workload.  Under torchrun (N > 1) every rank renders
its own replica of the workload (no data-path collective: one view per rank)
and rank 0 reports the aggregate.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

L2_BYTES = 129 * 2**20


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# Algorithmic work per blended (pixel, Gaussian) pair -- a count fixed by the
# definition, not by the implementation (FP32 operations, FMA = 2): the forward
# evaluates q = d^T conic d (2 sub, 3 mul, 2 FMA, 1 mul), alpha (1 mul + exp, 1 mul,
# 1 min) and blends (1 sub, 1 mul, 1 mul, 4 FMA): 25.  The backward recomputes
# alpha (12), recovers T (1 sub, 1 div), and forms the ten adjoints and the
# behind-accumulators (40): 55.
FLOPS_PER_EVAL_FWD = 25
FLOPS_PER_EVAL_BWD = 55
# FP32 peak: SMs x 128 FP32 lanes x 2 (FMA) x clock
FP32_LANES = 128


def sm_count():
    """SMs of the current device (152 on a GB300; also the value host-side tests use)."""
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    except Exception:
        pass
    return 152


def fp32_peak_tflops(mhz):
    return sm_count() * FP32_LANES * 2 * mhz * 1e6 / 1e12


class ClockSampler:
    """SM clock, its maximum, power and clock-event reasons sampled every ~2 ms during
    the timed region, read through NVML (ctypes on libnvidia-ml; read-only calls), or
    through nvidia-smi every 0.1 s where NVML cannot be loaded.  The device is matched
    by UUID so a CUDA_VISIBLE_DEVICES remap cannot point at another GPU."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")
    # NVML clock-event reason bits (nvml.h): sw power cap, hw slowdown, sw thermal, hw thermal
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown"}

    def __init__(self, index=0):
        self.index = index
        self.samples = []  # (sm_mhz, max_mhz, reason names)
        self._stop = threading.Event()
        self._t = None
        self._nvml = None
        self._h = None
        try:
            import ctypes
            import torch
            nv = ctypes.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() == 0:
                h = ctypes.c_void_p()
                uuid = getattr(torch.cuda.get_device_properties(index), "uuid", None)
                ok = False
                if uuid is not None:
                    ok = nv.nvmlDeviceGetHandleByUUID(f"GPU-{uuid}".encode(), ctypes.byref(h)) == 0
                if not ok:
                    ok = nv.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(h)) == 0
                if ok:
                    self._nvml, self._h = nv, h
        except Exception:
            self._nvml = None

    def _sample_nvml(self):
        import ctypes
        nv, h = self._nvml, self._h
        mhz, mx, r = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        if nv.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(mhz)) != 0:  # 1 = NVML_CLOCK_SM
            return
        nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx))
        fn = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            getattr(nv, "nvmlDeviceGetCurrentClocksThrottleReasons")
        names = []
        if fn(h, ctypes.byref(r)) == 0:
            names = [n for bit, n in self.REASONS.items() if r.value & bit]
        self.samples.append((float(mhz.value), float(mx.value), names))

    def _sample_smi(self):
        out = subprocess.run(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True,
                             timeout=5).stdout.strip()
        if not out:
            return
        f = [x.strip() for x in out.split(",")]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        act = [names[i] for i in range(4) if "Active" in f[3 + i] and not f[3 + i].startswith("Not")]
        num = lambda x: float(x) if x.replace(".", "").isdigit() else None  # noqa: E731
        self.samples.append((num(f[0]), num(f[1]), act))

    def _run(self):
        period = 0.002 if self._nvml is not None else 0.1
        while not self._stop.is_set():
            try:
                self._sample_nvml() if self._nvml is not None else self._sample_smi()
            except Exception:
                pass
            self._stop.wait(period)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [s[0] for s in self.samples if s[0] is not None]
        mx = [s[1] for s in self.samples if s[1] is not None]
        reasons = sorted({n for s in self.samples for n in s[2]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples),
                "source": "nvml" if self._nvml is not None else "nvidia-smi"}


def job_ms(ms_local, world, dev=None):
    """Whole-job time of a step: every rank's mean step time, the maximum over the
    ranks (after a barrier, so no rank's number is taken before the others finish)."""
    import torch
    import torch.distributed as dist
    if world <= 1:
        return float(ms_local)
    dist.barrier()
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(pixels_per_rank, ms, world):
    """Whole-job throughput (Mpixel/s): the pixels all ranks rendered in one step over
    the whole-job step time (replicas, so every rank renders the same workload)."""
    return world * pixels_per_rank / (ms * 1e-3) / 1e6


def bench_config(args, world):
    """The workload both arms time (the same dict in both JSON lines)."""
    return {"workload": f"room mapping step, {args.n} Gaussians SH3, {args.width}x{args.height}, fwd+loss+bwd",
            "l2": "GPU arm: flushed between timed steps (2x L2 buffer write, untimed)",
            "parallelism": f"replicas x{world}"}


def build_workload(args):
    w = synth.workload_room_mapping(n=args.n, width=args.width, height=args.height)
    return w


def run_gpu(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import paper_2311_11700_gb300 as G
    from paper_2311_11700_gb300 import build as B
    B.build()

    w = build_workload(args)
    dev = torch.device("cuda", local)
    R = G.Renderer(local, tile=(args.tile_w, args.tile_h))
    R.ctx.set_strip(args.strip_fwd, args.strip_bwd)
    R.ctx.set_binning(args.binning)
    R.ctx.set_persistent(args.persistent)
    if args.tracking_profile > 0:
        # profiling mode: a few eager batched tracking iterations, nothing timed
        print(json.dumps(run_tracking(args, G, R, w["scenes"][0], dev, t_coarse=args.tracking_profile,
                                      t_fine=args.tracking_profile, profile_only=True)))
        return
    R.ctx.set_grad_mode(1)  # the backward writes the gradients (one view renders the scene)
    scene = G.Scene.from_numpy(w["scenes"][0], device=dev)
    view = w["views"][0]
    views = [view]
    rgb, dep = w["targets"][0]
    P = view["width"] * view["height"]
    trgb = torch.as_tensor(rgb.reshape(-1), device=dev)
    tdep = torch.as_tensor(dep.reshape(-1), device=dev)
    # the launch configuration from the library's autotuner, timing the fused step as
    # it runs below (timed here, untimed below)
    tune = R.autotune([scene], views, reps=3, step=dict(target_rgb=trgb, target_depth=tdep, w_c=w["w_c"],
                                                        w_d=w["w_d"], out=True)) if args.autotune else None
    # size the pair list once (one checked forward), then run unchecked steps
    color, depth, acc, ws, mp = R.forward([scene], views)
    st, needed = G.gs_workspace_status(R.ctx, ws)
    mp = max(mp, int(needed * 1.1) + 1024)
    ws = G.alloc_workspace(G.gs_workspace_query(R.ctx, [scene], views, mp), dev)
    loss = torch.zeros(1, device=dev)
    grads = [{k: torch.zeros_like(getattr(scene, k)) for k in G.PARAM_KEYS}]
    dtw = torch.zeros(1, 6, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    def step():
        # forward, L1 loss and backward with one compositing kernel (gs_render_step_l1;
        # 4 % less compositing time than gs_render_forward_l1 + gs_render_backward here);
        # the backward writes this step's gradients (grad mode 1): no zeroing launches
        G.gs_render_step_l1(R.ctx, [scene], views, ws, mp, (color, depth, acc), trgb, tdep, w["w_c"], w["w_d"],
                            loss, grads, dtw, 0)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    st, _ = G.gs_workspace_status(R.ctx, ws)
    if st != G.GS_OK:
        raise RuntimeError(f"workspace status {st}")
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    times = []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)  # evict L2 between timed steps (not timed)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    ms = job_ms(float(np.mean(times)), world, dev)

    # end to end: host buffers in, loss out, through the same C ABI calls
    e2e = measure_e2e(args, G, R, scene, views, w, mp, ws, dev, rgb, dep)

    # stage split: a separate pass with the library's stage events (timing mode 2:
    # the kernels of the timed path), L2 flushed before each step as in the timed
    # loop, then the same pass warm; then one step that counts the work (mode 1)
    G.gs_ctx_set_timing(R.ctx, 2)
    G.gs_ctx_read_timing(R.ctx, reset=True)
    n_prof = max(3, min(args.steps, 20))
    for _ in range(n_prof):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize()
    stages = G.gs_ctx_read_timing(R.ctx, reset=True)
    # the same split warm: steps back to back, no L2 flush between them
    for _ in range(n_prof):
        step()
    torch.cuda.synchronize()
    stages_warm = G.gs_ctx_read_timing(R.ctx, reset=True)
    G.gs_ctx_set_timing(R.ctx, 1)
    step()
    counters = G.gs_workspace_counters(R.ctx, ws)
    G.gs_ctx_set_timing(R.ctx, 0)
    split = {k: round(v[0] / n_prof, 4) for k, v in stages.items() if k != "calls"}
    split_warm = {k: round(v[0] / n_prof, 4) for k, v in stages_warm.items() if k != "calls" and v[0] > 0}
    # the nested stages (tile scan, short and long sorts) lie inside project and tile_sort
    launches_per_step = sum(v[1] for k, v in stages.items() if k not in ("calls",) + NESTED_STAGES) / n_prof

    if rank == 0:
        peaks, src = _peaks()
        value = job_value(P, ms, world)
        line = {
            "metric": "fwd+bwd Mpixel/s at 1200x680, 300k Gaussians (SH3)",
            "value": round(value, 2), "unit": "Mpixel/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded room scene; no dataset)",
            "config": bench_config(args, world),
            "launch": _launch_cfg(R, tune),
            "clocks": clk.summary(),
            "e2e": e2e,
            "gpu_launches": int(round(launches_per_step * args.steps)),
            "stage_ms": split,
            "stage_ms_warm": split_warm,
            "counters": {"visible_splats": counters[0], "pairs": counters[1], "blended_fwd": counters[2],
                         "blended_bwd": counters[3], "bwd_warp_iters": counters[4], "bwd_blend_iters": counters[5],
                         "bwd_reduce_iters": counters[6], "long_segments": counters[7]},
        }
        line["roofline"] = roofline(split, counters, peaks, src, line["clocks"], scene.n,
                                    (scene.sh_degree + 1) ** 2)
        if args.tracking:
            line["tracking"] = run_tracking(args, G, R, w["scenes"][0], dev)
        if args.batched:
            line["batched_mapping"] = run_batched_mapping(args, G, R, dev, flush)
            line["uneven_batch"] = run_uneven(args, G, R, dev, flush)
        if args.cpu_sample > 0:
            line["cpu_baseline"] = cpu_baseline(w, args.cpu_sample)
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def run_tracking(args, G, R, scene_np, dev, n_hyp=16, t_coarse=50, t_fine=50, profile_only=False):
    """Pose-grad iterations per second on the tracking workload: n_hyp pose
    hypotheses around the room view, t_coarse coarse iterations (half resolution,
    10 % of the pixels) then t_fine fine ones (full resolution, Gaussians with
    opacity > 0.5 and a seeded 60 % keep mask); one iteration = forward with the
    fused L1 loss, pose-only backward and the Adam step of all hypotheses.
    Batched: all hypotheses in one call per stage, the whole loop captured in one
    CUDA graph.  Plain: one hypothesis per call, launched eagerly."""
    import torch
    w = synth.workload_tracking(n=args.n, n_hyp=n_hyp, width=args.width, height=args.height)
    scene = G.Scene.from_numpy(w["scene"], device=dev)
    gt, cgt = w["view_gt"], w["coarse_gt"]
    # targets: renders at the true pose (colour and depth)
    tcol, tdep, _, _, _ = R.forward([scene], [cgt])
    fcol, fdep, _, _, _ = R.forward([scene], [gt])
    keep = torch.as_tensor(w["keep_mask"], device=dev)
    fine_mask = torch.zeros(scene.n, dtype=torch.uint8, device=dev)
    G.gs_select_opacity(R.ctx, scene, 0.5, keep, fine_mask)
    fine_scene = G.Scene(*scene.params(), scene.sh_degree, mask=fine_mask)
    cmask = torch.as_tensor(w["coarse_mask"], device=dev)
    T0 = torch.as_tensor(np.stack([synth.perturb_view(gt, x)["T_cw"] for x in w["twists"]]), device=dev)
    lr = [2e-4, 2e-4, 2e-4, 1e-3, 1e-3, 1e-3]

    def pose_step(scn, views, b, tc, td, fused, pose_mode=0):
        """Loss and pose gradient of one iteration: gs_render_step_l1, the fused
        forward + loss + backward, in both stages (coarse, compacted pixels: 1.6 %
        less compositing time than the separate calls; fine: 6.5 %).  fused=False
        takes the separate calls (gs_render_forward_l1 + gs_pose_grad).  pose_mode
        0: the exact twist gradient; 1: the paper's approximation (Eq. pose_grad)."""
        if fused:
            G.gs_render_step_l1(R.ctx, [scn], views, b["ws"], b["mp"], None, tc, td, 1.0, 0.5, b["loss"], None,
                                b["dtw"], pose_mode)
        else:
            G.gs_render_forward_l1(R.ctx, [scn], views, b["ws"], b["mp"], (None, None, None), tc, td, 1.0, 0.5,
                                   b["loss"], (b["dC"], b["dD"], None))
            G.gs_pose_grad(R.ctx, [scn], views, b["ws"], b["mp"], (b["dC"], b["dD"], None), b["dtw"], pose_mode)

    def stage_buffers(base, scn, views):
        P = base["width"] * base["height"] * len(views)
        need = R.forward([scn], views)  # sizes the pair list for this stage
        st, needed = G.gs_workspace_status(R.ctx, need[3])
        mp = int(needed * 1.5) + 4096
        ws = G.alloc_workspace(G.gs_workspace_query(R.ctx, [scn], views, mp), dev)
        return dict(ws=ws, mp=mp, loss=torch.zeros(len(views), device=dev), dC=torch.empty(3 * P, device=dev),
                    dD=torch.empty(P, device=dev), dtw=torch.zeros(len(views), 6, device=dev))

    def batched_setup(pose_mode=0):
        T = T0.clone()
        state = torch.zeros(n_hyp, 16, device=dev)
        cv = [dict(cgt, T_cw_dev=T[v], pixel_mask=cmask) for v in range(n_hyp)]
        fv = [dict(gt, T_cw_dev=T[v]) for v in range(n_hyp)]
        cb = stage_buffers(cgt, scene, cv)
        fb = stage_buffers(gt, fine_scene, fv)
        ct, cd = tcol.repeat(n_hyp), tdep.repeat(n_hyp)
        ft, fd = fcol.repeat(n_hyp), fdep.repeat(n_hyp)

        def iteration(scn, views, b, tc, td, fused):
            pose_step(scn, views, b, tc, td, fused, pose_mode)
            G.gs_pose_adam(R.ctx, T, b["dtw"], state, lr)

        def loop(coarse=True, fine=True):
            for _ in range(t_coarse if coarse else 0):
                iteration(scene, cv, cb, ct, cd, True)
            for _ in range(t_fine if fine else 0):
                iteration(fine_scene, fv, fb, ft, fd, True)

        def reset():
            T.copy_(T0)
            state.zero_()
        return loop, reset, (cb, fb), T

    def plain_setup():
        Ts = [T0[v:v + 1].clone() for v in range(n_hyp)]
        states = [torch.zeros(1, 16, device=dev) for _ in range(n_hyp)]
        cvs = [[dict(cgt, T_cw_dev=Ts[v][0], pixel_mask=cmask)] for v in range(n_hyp)]
        fvs = [[dict(gt, T_cw_dev=Ts[v][0])] for v in range(n_hyp)]
        cbs = [stage_buffers(cgt, scene, cvs[v]) for v in range(n_hyp)]
        fbs = [stage_buffers(gt, fine_scene, fvs[v]) for v in range(n_hyp)]

        def iteration(scn, views, b, tc, td, T, state, fused):
            pose_step(scn, views, b, tc, td, fused)
            G.gs_pose_adam(R.ctx, T, b["dtw"], state, lr)

        def loop():
            for _ in range(t_coarse):
                for v in range(n_hyp):
                    iteration(scene, cvs[v], cbs[v], tcol, tdep, Ts[v], states[v], True)
            for _ in range(t_fine):
                for v in range(n_hyp):
                    iteration(fine_scene, fvs[v], fbs[v], fcol, fdep, Ts[v], states[v], True)

        def reset():
            for v in range(n_hyp):
                Ts[v].copy_(T0[v:v + 1])
                states[v].zero_()
        return loop, reset, cbs + fbs

    def timed(fn, reps):
        stream = torch.cuda.current_stream()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    iters = t_coarse + t_fine
    loop, reset, bufs, _ = batched_setup()
    reset(); loop(); torch.cuda.synchronize()
    if profile_only:  # one more pass, for a profiler's launch list
        reset(); loop(); torch.cuda.synchronize()
        return {"profile": "tracking", "hypotheses": n_hyp, "coarse_iterations": t_coarse, "fine_iterations": t_fine}
    ms_eager = timed(lambda: (reset(), loop()), 3)
    g = torch.cuda.CUDAGraph()
    reset()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        loop()  # warm the capture stream
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        loop()
    torch.cuda.synchronize()
    ms_graph = timed(lambda: (reset(), g.replay()), 5)
    for b in bufs:
        st, needed = G.gs_workspace_status(R.ctx, b["ws"])
        if st != G.GS_OK:
            raise RuntimeError(f"tracking workspace status {st} (pairs needed {needed}, capacity {b['mp']})")
    # stage split per iteration of each stage: a separate eager pass with the library's
    # stage events (timing mode 2), then one more pass that counts the work (mode 1)
    stage_ms, stage_counters = {}, {}
    for mode in (2, 1):
        G.gs_ctx_set_timing(R.ctx, mode)
        G.gs_ctx_read_timing(R.ctx, reset=True)
        reset()
        for name, its, part, b in (("coarse", t_coarse, dict(fine=False), bufs[0]),
                                   ("fine", t_fine, dict(coarse=False), bufs[1])):
            loop(**part)
            torch.cuda.synchronize()
            split = G.gs_ctx_read_timing(R.ctx, reset=True)
            if mode == 2:
                stage_ms[name] = {k: round(v[0] / max(its, 1), 4) for k, v in split.items()
                                  if k != "calls" and v[0] > 0}
            else:
                c = G.gs_workspace_counters(R.ctx, b["ws"])  # the stage's last iteration, all hypotheses
                stage_counters[name] = {"visible_splats": c[0], "pairs": c[1], "blended_fwd": c[2],
                                        "blended_bwd": c[3], "bwd_warp_iters": c[4], "bwd_blend_iters": c[5],
                                        "bwd_reduce_iters": c[6], "long_segments": c[7]}
    G.gs_ctx_set_timing(R.ctx, 0)
    study = pose_study(batched_setup, timed, gt, T0, iters) if not profile_only else None
    ploop, preset, pbufs = plain_setup()
    # the plain form with either compositing form (one small view per call fills few
    # SMs with the one-warp compacted kernels); the faster one is reported
    ms_plain_by = {}
    for mode in (0, 1):
        R.ctx.set_compact(mode)
        preset(); ploop(); torch.cuda.synchronize()
        ms_plain_by[mode] = timed(lambda: (preset(), ploop()), 2)
    R.ctx.set_compact(1)
    ms_plain = min(ms_plain_by.values())
    for b in pbufs:
        st, needed = G.gs_workspace_status(R.ctx, b["ws"])
        if st != G.GS_OK:
            raise RuntimeError(f"tracking workspace status {st}")
    per_s = lambda ms: round(iters / (ms * 1e-3), 2)  # noqa: E731
    return {"metric": "pose-grad iters/s", "unit": "iterations/s (all hypotheses)", "hypotheses": n_hyp,
            "iterations": iters, "coarse": f"{cgt['width']}x{cgt['height']}, 10 % pixels, {t_coarse} its",
            "fine": f"{gt['width']}x{gt['height']}, opacity > 0.5 and 60 % keep, {t_fine} its",
            "batched_graph": per_s(ms_graph), "batched_eager": per_s(ms_eager), "plain_eager": per_s(ms_plain),
            "plain_eager_by_compact_mode": {str(k): per_s(v) for k, v in ms_plain_by.items()},
            "batched_vs_plain": round(ms_plain / ms_graph, 2), "stage_ms_per_iteration": stage_ms,
            "stage_counters": stage_counters, "pose_study": study}


def pose_errors(T, gt):
    """Per hypothesis: camera-centre error (cm) and rotation error (degrees) of the
    world->camera poses T [V, 12] against the view gt."""
    Tg = np.asarray(gt["T_cw"], np.float64).reshape(3, 4)
    cg = -Tg[:, :3].T @ Tg[:, 3]
    out_t, out_r = [], []
    for P in np.asarray(T, np.float64).reshape(-1, 3, 4):
        out_t.append(100.0 * np.linalg.norm(-P[:, :3].T @ P[:, 3] - cg))
        Rr = P[:, :3] @ Tg[:, :3].T
        out_r.append(np.degrees(np.arccos(np.clip((np.trace(Rr) - 1.0) / 2.0, -1.0, 1.0))))
    return np.array(out_t), np.array(out_r)


def pose_study(batched_setup, timed, gt, T0, iters):
    """The exact twist gradient against the paper's approximation (Eq. pose_grad
    drops dSigma'/dP and the colour's view direction) on this tracking workload:
    the same hypotheses, coarse then fine, each loop captured in a CUDA graph;
    iterations/s and the final pose errors (mean and max over the hypotheses)."""
    import torch
    t0, r0 = pose_errors(T0.cpu().numpy(), gt)
    res = {"initial": {"t_err_cm_mean": round(float(t0.mean()), 3), "r_err_deg_mean": round(float(r0.mean()), 4)}}
    for name, mode in (("exact", 0), ("paper", 1)):
        loop, reset, _, T = batched_setup(mode)
        reset(); loop(); torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            reset(); loop()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        with torch.cuda.graph(g):
            loop()
        ms = timed(lambda: (reset(), g.replay()), 3)
        reset(); g.replay(); torch.cuda.synchronize()
        te, re = pose_errors(T.cpu().numpy(), gt)
        res[name] = {"iterations_per_s": round(iters / (ms * 1e-3), 2), "t_err_cm_mean": round(float(te.mean()), 3),
                     "t_err_cm_max": round(float(te.max()), 3), "r_err_deg_mean": round(float(re.mean()), 4),
                     "r_err_deg_max": round(float(re.max()), 4)}
    return res


def _launch_cfg(R, tune):
    """The context's launch configuration (tile, warp strips, binning, compositing
    launch form) and whether the autotuner chose it."""
    return {"tile": "{}x{}".format(*R.ctx.tile), "strip": list(R.ctx.strip),
            "binning": ["per-tile counting sort", "global radix sort"][R.ctx.binning],
            "compositing": ["one CTA per tile", "persistent"][R.ctx.persistent], "autotuned": tune is not None}


def _step_buffers(G, R, scenes, views, dev, headroom=1.25):
    """Workspace (pair list sized by one checked forward), targets-free buffers."""
    import torch
    color, depth, acc, ws, mp = R.forward(scenes, views)
    st, needed = G.gs_workspace_status(R.ctx, ws)
    mp = int(needed * headroom) + 4096
    ws = G.alloc_workspace(G.gs_workspace_query(R.ctx, scenes, views, mp), dev)
    P = sum(v["width"] * v["height"] for v in views)
    return dict(ws=ws, mp=mp, loss=torch.zeros(len(views), device=dev), dC=torch.empty(3 * P, device=dev),
                dD=torch.empty(P, device=dev), dtw=torch.zeros(len(views), 6, device=dev), P=P)


def _mapping_step(G, R, scenes, views, b, trgb, tdep, grads):
    # forward, L1 loss and backward with one compositing kernel
    G.gs_render_step_l1(R.ctx, scenes, views, b["ws"], b["mp"], None, trgb, tdep, 1.0, 0.5, b["loss"], grads,
                        b["dtw"], 0)


def _timed(fn, reps, flush=None):
    import torch
    stream = torch.cuda.current_stream()
    ts = []
    for _ in range(reps):
        if flush is not None:
            flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts))


def run_batched_mapping(args, G, R, dev, flush):
    """8 keyframes of the 1M-Gaussian SH3 room at 1200x680: fwd + loss + bwd with
    gradients accumulated over the views, batched in one call (captured in a CUDA
    graph) vs one view per call; then the expansion step at one keyframe (render,
    unreliable pixels, floater decay, prune at opacity 0.005)."""
    import torch
    w = synth.workload_batched_mapping(n=args.batched_n, n_views=8, width=args.width, height=args.height)
    scene = G.Scene.from_numpy(w["scene"], device=dev)
    views = [dict(v, scene=0) for v in w["views"]]
    trgb = torch.as_tensor(np.concatenate([t[0].reshape(-1) for t in w["targets"]]), device=dev)
    tdep = torch.as_tensor(np.concatenate([t[1].reshape(-1) for t in w["targets"]]), device=dev)
    grads = [{k: torch.zeros_like(getattr(scene, k)) for k in G.PARAM_KEYS}]
    R.ctx.set_grad_mode(0)  # gradients accumulate over the views (and the plain form's calls)
    tune = R.autotune([scene], views, reps=2, step=dict(target_rgb=trgb, target_depth=tdep)) if args.autotune else None
    b = _step_buffers(G, R, [scene], views, dev)

    def batched():
        for g in grads[0].values():
            g.zero_()
        _mapping_step(G, R, [scene], views, b, trgb, tdep, grads)

    batched(); torch.cuda.synchronize()
    ms_eager = _timed(batched, 5, flush)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        batched()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        batched()
    ms_graph = _timed(g.replay, 5, flush)
    st, _ = G.gs_workspace_status(R.ctx, b["ws"])
    if st != G.GS_OK:
        raise RuntimeError(f"batched mapping status {st}")
    # plain: one view per call, separate workspaces, same accumulated gradients
    P1 = views[0]["width"] * views[0]["height"]
    pb = [_step_buffers(G, R, [scene], [v], dev) for v in views]

    def plain():
        for gg in grads[0].values():
            gg.zero_()
        for i, v in enumerate(views):
            _mapping_step(G, R, [scene], [v], pb[i], trgb[3 * P1 * i:3 * P1 * (i + 1)], tdep[P1 * i:P1 * (i + 1)],
                          grads)

    plain(); torch.cuda.synchronize()
    ms_plain = _timed(plain, 5, flush)
    # the expansion step at keyframe 0: render acc/depth, then gs_expand
    v0 = views[0]
    cap = scene.n + v0["width"] * v0["height"]
    K = (scene.sh_degree + 1) ** 2
    out = {"mean": torch.empty(3, cap, device=dev), "log_scale": torch.empty(3, cap, device=dev),
           "quat": torch.empty(4, cap, device=dev), "opacity_logit": torch.empty(cap, device=dev),
           "sh": torch.empty(3 * K, cap, device=dev)}
    count = torch.zeros(4, dtype=torch.int64, device=dev)
    ews = G.alloc_workspace(G.gs_expand_workspace_query(R.ctx, scene.n, v0), dev)
    b0 = _step_buffers(G, R, [scene], [v0], dev)
    acc0 = torch.empty(P1, device=dev)
    dep0 = torch.empty(P1, device=dev)
    obs_rgb, obs_d = trgb[:3 * P1], tdep[:P1]

    def expand():
        G.gs_render_forward(R.ctx, [scene], [v0], b0["ws"], b0["mp"], (None, dep0, acc0))
        G.gs_expand(R.ctx, scene, v0, acc0, dep0, obs_rgb, obs_d, {}, out, cap, count, ews)

    expand(); torch.cuda.synchronize()
    ms_expand = _timed(expand, 5, flush)
    c = count.cpu().numpy()
    px = sum(v["width"] * v["height"] for v in views)
    return {"workload": f"{scene.n} Gaussians SH3 (1M room minus a 1 m^3 hole), 8 keyframes "
                        f"{views[0]['width']}x{views[0]['height']}, fwd+loss+bwd, gradients accumulated",
            "unit": "Mpixel/s", "batched_graph": round(px / (ms_graph * 1e-3) / 1e6, 2),
            "batched_eager": round(px / (ms_eager * 1e-3) / 1e6, 2), "plain_eager": round(px / (ms_plain * 1e-3) / 1e6, 2),
            "batched_vs_plain": round(ms_plain / ms_graph, 2),
            "expand_ms": round(ms_expand, 3), "expand": {"kept": int(c[0]), "added": int(c[1])},
            "launch": _launch_cfg(R, tune)}


def run_uneven(args, G, R, dev, flush):
    """12 views of {320x240, 640x480, 1200x680}, each with its own room of 50k..2M
    SH3 Gaussians: fwd + loss + bwd batched in one call (graph) vs one view per call."""
    import torch
    w = synth.workload_uneven(n_views=12, n_max=args.uneven_nmax)
    scenes = [G.Scene.from_numpy(s, device=dev) for s in w["scenes"]]
    views = w["views"]
    trgb = torch.as_tensor(np.concatenate([t[0].reshape(-1) for t in w["targets"]]), device=dev)
    tdep = torch.as_tensor(np.concatenate([t[1].reshape(-1) for t in w["targets"]]), device=dev)
    grads = [{k: torch.zeros_like(getattr(s, k)) for k in G.PARAM_KEYS} for s in scenes]
    # one configuration for both forms: the one the autotuner picks for the batch;
    # every scene has one view, so the backward writes its gradients
    R.ctx.set_grad_mode(1)
    tune = R.autotune(scenes, views, reps=2, step=dict(target_rgb=trgb, target_depth=tdep)) if args.autotune else None
    b = _step_buffers(G, R, scenes, views, dev)

    def batched():
        _mapping_step(G, R, scenes, views, b, trgb, tdep, grads)

    batched(); torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        batched()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        batched()
    ms_graph = _timed(g.replay, 5, flush)
    offs = np.cumsum([0] + [v["width"] * v["height"] for v in views])
    pb = [_step_buffers(G, R, [scenes[i]], [dict(v, scene=0)], dev) for i, v in enumerate(views)]

    def plain():
        for i, v in enumerate(views):
            _mapping_step(G, R, [scenes[i]], [dict(v, scene=0)], pb[i], trgb[3 * offs[i]:3 * offs[i + 1]],
                          tdep[offs[i]:offs[i + 1]], [grads[i]])

    plain(); torch.cuda.synchronize()
    ms_plain = _timed(plain, 5, flush)
    px = int(offs[-1])
    return {"workload": "12 views of {320x240, 640x480, 1200x680} with their own SH3 rooms of "
                        f"{min(s.n for s in scenes)}..{max(s.n for s in scenes)} Gaussians, fwd+loss+bwd",
            "unit": "Mpixel/s", "batched_graph": round(px / (ms_graph * 1e-3) / 1e6, 2),
            "plain_eager": round(px / (ms_plain * 1e-3) / 1e6, 2), "batched_vs_plain": round(ms_plain / ms_graph, 2),
            "launch": _launch_cfg(R, tune)}


def _capture(stage, key="dram_bytes_per_launch"):
    """A per-launch figure of the stage's kernel from the committed ncu capture
    (profiles/dram_traffic.json): dram__bytes_read.sum + dram__bytes_write.sum, or
    smsp__inst_executed.sum ("warp_instructions_per_launch"); None when the
    kernel's sources changed since that capture (their sha256 differs)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(path):
        return None
    for rec in json.load(open(path)).values():
        if rec.get("stage") != stage:
            continue
        h = hashlib.sha256()
        for f in rec["sources"]:
            h.update(open(os.path.join(ROOT, f), "rb").read())
        return rec.get(key) if h.hexdigest() == rec["sources_sha256"] else None
    return None


def _dram_traffic(stage):
    return _capture(stage)


# Algorithmic bytes of the memory-bound stages: what the method must move, per
# Gaussian of the scene (N), per visible splat (V: touches a tile) and per
# (Gaussian, tile) pair (P), at K SH coefficients per channel.  Fixed by the
# definition, not by the implementation.
#   project      the centre of every Gaussian for the depth test (12 B); the other
#                parameters of the visible ones (log-scale 12, quaternion 16,
#                opacity 4, SH 12 K); the projected splat written (centre 8, conic 12,
#                depth 4, colour 12, opacity 4, footprint 8 = 48 B)
#   emit         the visible splats' footprint rectangle, depth and tile count read
#                (24 B); one (tile | depth key, Gaussian id) pair written (12 B)
#   tile_sort    one read and one write of each pair's key and value (24 B)
#   project_bwd  the parameters (44 + 12 K B) and the blend's 40 B of adjoints read,
#                the parameter gradients (44 + 12 K B) written, per visible splat
NESTED_STAGES = ("tile_scan", "sort_short", "sort_long")
STAGE_KERNELS = {"project": ["k_project_fwd", "k_tile_sums", "k_tile_offsets"], "emit": ["k_emit"],
                 "tile_sort": ["k_tile_sort", "k_tile_sort_mid", "k_tile_sort_large"],
                 "project_bwd": ["k_project_bwd"]}


def stage_bytes(stage, N, V, P, K):
    if stage == "project":
        return 12 * N + (32 + 12 * K) * V + 48 * V
    if stage == "emit":
        return 24 * V + 12 * P
    if stage == "tile_sort":
        return 24 * P
    if stage == "project_bwd":
        return (84 + 12 * K) * V + (44 + 12 * K) * V
    return None


def roofline(split, counters, peaks, src, clocks, N, K):
    """Roofline of every stage of the step, from the live CUDA-event time of the
    stage timing pass (timing mode 2, L2 flushed before each step).  The
    compositing kernels are FP32-ALU bound: achieved = algorithmic FLOPs (blended
    pairs x FLOPs per blended pair) / time against the FP32 peak at the maximum SM
    clock.  The others are HBM bound: achieved = algorithmic bytes (stage_bytes) /
    time against the measured copy bandwidth; traffic = the ncu DRAM bytes of one
    launch of the stage's kernels, while their sources match the capture.  The
    top-level keys describe the stage with the largest share of the step."""
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    V, P = counters[0], counters[1]
    stages = {}
    for st, t_ms in split.items():
        if t_ms <= 0 or st == "setup":
            continue
        t = t_ms * 1e-3
        if st in ("composite_step", "composite_fwd", "composite_bwd"):
            if st == "composite_step":  # forward and backward walks in one kernel
                ev = counters[2] + counters[3]
                flops = counters[2] * FLOPS_PER_EVAL_FWD + counters[3] * FLOPS_PER_EVAL_BWD
            else:
                ev = counters[2] if st == "composite_fwd" else counters[3]
                flops = ev * (FLOPS_PER_EVAL_FWD if st == "composite_fwd" else FLOPS_PER_EVAL_BWD)
            ach = flops / t / 1e12
            peak = fp32_peak_tflops(mhz)
            line = {"kernel": st, "bound": "alu", "achieved": round(ach, 3), "peak": round(peak, 2),
                    "unit": "TFLOP/s", "frac": round(ach / peak, 4), "traffic": _dram_traffic(st),
                    "blended_per_s": round(ev / t / 1e9, 3), "blended_unit": "G blended pairs/s",
                    "peak_note": f"FP32 {sm_count()} SMs x {FP32_LANES} lanes x 2 x {mhz:.0f} MHz (derived, not "
                                 "measured)",
                    "time_ms": round(t_ms, 4)}
            # the kernel is issue-bound: its warp instructions per launch (ncu, same
            # workload) over the live time, against one instruction per clock per scheduler
            inst = _capture(st, "warp_instructions_per_launch")
            if inst is not None:
                ipk = inst / t / 1e12
                ipeak = sm_count() * 4 * mhz * 1e6 / 1e12
                line["issue"] = {"achieved": round(ipk, 4), "peak": round(ipeak, 4),
                                 "unit": "T warp instructions/s", "frac": round(ipk / ipeak, 4),
                                 "note": f"ncu smsp__inst_executed.sum per launch / live time; peak {sm_count()} SMs "
                                         "x 4 x clock"}
            stages[st] = line
            continue
        b = stage_bytes(st, N, V, P, K)
        if b is None:
            continue
        ach = b / t / 1e9
        tr = _dram_traffic(st)
        stages[st] = {"kernel": st, "kernels": STAGE_KERNELS.get(st), "bound": "hbm", "achieved": round(ach, 1),
                      "peak": hbm, "unit": "GB/s", "frac": round(ach / hbm, 4), "traffic": tr,
                      "algorithmic_bytes": int(b), "traffic_ratio": None if tr is None else round(tr / b, 3),
                      "time_ms": round(t_ms, 4), "peak_source": src}
    top = max(stages, key=lambda k: stages[k]["time_ms"])
    line = dict(stages[top])
    line["stages"] = stages
    return line


def cpu_baseline(w, n_pix, seed=0):
    """The FP64 oracle (as it stands) on a seeded pixel sample of the same
    workload: forward + loss + gradients of every parameter and the twist."""
    import torch
    import oracle as O
    view = w["views"][0]
    H, W = view["height"], view["width"]
    rng = np.random.default_rng(seed)
    m = np.zeros(H * W, np.uint8)
    m[rng.choice(H * W, n_pix, replace=False)] = 1
    t0 = time.perf_counter()
    O.render_and_grad(w["scenes"], w["views"], w["targets"], w["w_c"], w["w_d"], pixel_masks=[m.reshape(H, W)])
    dt = time.perf_counter() - t0
    return {"value": round(n_pix / dt / 1e6, 8), "unit": "Mpixel/s", "cores": torch.get_num_threads(),
            "kind": "oracle", "sample": f"{n_pix} seeded random pixels of the 1200x680 view, fwd+loss+bwd "
                                        f"(all 300k Gaussians brute force per pixel), {dt:.1f} s",
            "seconds": round(dt, 4)}


def run_reference(args):
    """The baseline arm: the FP64 CPU oracle, as it stands, on bounded pixel
    samples of the same workload (one seeded sample of args.ref_sample pixels per
    step).  ms_per_step is the measured time of one such step; value is the pixel
    rate it achieves (Mpixel/s); the time a full frame would take at that rate is
    reported apart, as an extrapolation."""
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = build_workload(args)
    samples = []
    for k in range(args.warmup + args.steps):
        r = cpu_baseline(w, args.ref_sample, seed=k)
        if k >= args.warmup:
            samples.append(r)
    step_s = float(np.mean([s["seconds"] for s in samples]))
    v = args.ref_sample / step_s / 1e6
    P = args.width * args.height
    line = {"impl": "reference", "metric": "fwd+bwd Mpixel/s at 1200x680, 300k Gaussians (SH3)",
            "value": round(v, 8), "unit": "Mpixel/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(step_s * 1e3, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded room scene; no dataset)",
            "config": bench_config(args, world),
            "full_frame_ms_extrapolated": round(P / (v * 1e6) * 1e3, 1),
            "cpu_baseline": {"value": round(v, 8), "unit": "Mpixel/s", "cores": torch.get_num_threads(),
                             "kind": "oracle",
                             "sample": f"{args.ref_sample} seeded random pixels of the 1200x680 view per step, "
                                       "fwd+loss+bwd (all 300k Gaussians brute force per pixel)"},
            "e2e": {"value": round(v, 8), "unit": "Mpixel/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def measure_e2e(args, G, R, scene, views, w, mp, ws, dev, rgb, dep):
    """The mapping step end to end through the public calls: every step copies its
    targets from pinned host memory and reads its loss back.  The inputs and the
    loss are double buffered on the device: each step's upload runs on a copy stream
    while the step before it computes, and each step's loss is read back on another
    stream while the next step computes (events order every buffer's reuse), as a
    training loop that streams keyframes from the host would.  All copies lie inside
    the timed region."""
    import torch
    P = views[0]["width"] * views[0]["height"]
    h_rgb = torch.as_tensor(rgb.reshape(-1)).pin_memory()
    h_dep = torch.as_tensor(dep.reshape(-1)).pin_memory()
    h_loss = torch.empty(2).pin_memory()
    trgb = [torch.empty(3 * P, device=dev) for _ in range(2)]
    tdep = [torch.empty(P, device=dev) for _ in range(2)]
    color = torch.empty(3 * P, device=dev)
    depth = torch.empty(P, device=dev)
    acc = torch.empty(P, device=dev)
    loss = [torch.zeros(1, device=dev) for _ in range(2)]
    grads = [{k: torch.zeros_like(getattr(scene, k)) for k in G.PARAM_KEYS}]
    dtw = torch.zeros(1, 6, device=dev)
    stream = torch.cuda.current_stream()
    cstream = torch.cuda.Stream()
    dstream = torch.cuda.Stream()
    copied = [torch.cuda.Event() for _ in range(2)]
    used = [torch.cuda.Event() for _ in range(2)]
    read = [torch.cuda.Event() for _ in range(2)]

    def upload(b, after=None):
        with torch.cuda.stream(cstream):
            if after is not None:
                cstream.wait_event(after)
            cstream.wait_event(used[b])  # the step that read buffer b is done
            trgb[b].copy_(h_rgb, non_blocking=True)
            tdep[b].copy_(h_dep, non_blocking=True)
            copied[b].record(cstream)

    def run(n, start=None):
        if start is not None:
            dstream.wait_event(start)
        for b in range(2):
            read[b].record(dstream)
        upload(0, start)
        for k in range(n):
            b = k & 1
            stream.wait_event(copied[b])
            stream.wait_event(read[b])  # the loss of step k - 2 has reached the host
            if k + 1 < n:
                upload(b ^ 1)
            G.gs_render_step_l1(R.ctx, [scene], views, ws, mp, (color, depth, acc), trgb[b], tdep[b], w["w_c"],
                                w["w_d"], loss[b], grads, dtw, 0)
            used[b].record(stream)  # the step that read buffer b is done
            with torch.cuda.stream(dstream):
                dstream.wait_event(used[b])
                h_loss[b:b + 1].copy_(loss[b], non_blocking=True)
                read[b].record(dstream)
        stream.wait_event(read[(n - 1) & 1])  # the last loss is on the host

    run(3)
    torch.cuda.synchronize()
    n = max(3, args.steps)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    run(n, e0)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / n
    return {"value": round(P / (ms * 1e-3) / 1e6, 2), "unit": "Mpixel/s", "ms_per_step": round(ms, 4),
            "h2d_bytes_per_step": int(h_rgb.numel() * 4 + h_dep.numel() * 4), "d2h_bytes_per_step": 4,
            "overlap": "uploads double-buffered on a copy stream, each under the previous step's compute; "
                       "each loss read back on a third stream under the next step"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gsr", choices=["gsr", "reference"])
    ap.add_argument("--n", type=int, default=300_000)
    ap.add_argument("--width", type=int, default=1200)
    ap.add_argument("--height", type=int, default=680)
    ap.add_argument("--tile-w", type=int, default=16)
    ap.add_argument("--tile-h", type=int, default=16)
    ap.add_argument("--strip-fwd", type=int, default=2, help="warp strip shape of the compositing forward (0..5)")
    ap.add_argument("--strip-bwd", type=int, default=2, help="warp strip shape of the compositing backward (0..5)")
    ap.add_argument("--binning", type=int, default=0, help="0: per-tile counting sort, 1: global radix sort")
    ap.add_argument("--persistent", type=int, default=0,
                    help="launch form of the fused step's compositing kernel: 0 one CTA per tile, 1 persistent")
    ap.add_argument("--autotune", type=int, default=1,
                    help="pick tile / binning / strips with the library's autotuner before timing (overrides the above)")
    ap.add_argument("--cpu-sample", type=int, default=2048, help="pixels of the oracle CPU baseline (0: skip)")
    ap.add_argument("--tracking", type=int, default=1, help="also time the tracking workload (pose-grad iters/s)")
    ap.add_argument("--batched", type=int, default=1, help="also time the batched and uneven mapping workloads")
    ap.add_argument("--batched-n", type=int, default=1_000_000)
    ap.add_argument("--uneven-nmax", type=int, default=2_000_000)
    ap.add_argument("--ref-sample", type=int, default=32, help="pixels per step of the reference arm")
    ap.add_argument("--tracking-profile", type=int, default=0,
                    help="profiling mode: set up the tracking workload, run this many coarse and fine batched "
                         "iterations twice (eager, untimed) and exit")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    run_gpu(args)


if __name__ == "__main__":
    main()
