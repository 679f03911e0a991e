"""Bundle adjustment over a keyframe window (GS-SLAM Sec. 3.3, Eq. BA) and the
coarse-to-fine tracking of a frame (Sec. 3.3) on the library's kernels.

One iteration renders the K selected keyframes of one scene in a single batched
call (device-resident poses), evaluates the BA loss in the forward's epilogue,
runs one backward to the map parameters (accumulated over the keyframes) and to
every keyframe's se(3) twist, steps the map with torch Adam and, in the second
half of the iterations only, every keyframe pose with the library's pose Adam
(exp retraction on the device).  All rendering, loss and gradient work is the
library's CUDA kernels; this module only sequences the calls.

Loss (Eq. BA): (1/K) sum_k sum_m w_d |D_m - D_hat_m| + w_c |C_m - C_hat_m| with the
depth term only where D_m > 0; the paper's weights are photometric 0.8 and
geometric 0.3.  Map learning rates: position 1.6e-5 decaying log-linearly to 1.7e-7
over 100 steps, SH 5e-4, opacity 1e-2, scale 2e-4, rotation 4e-5; pose learning
rates translation 2e-4, rotation 5e-4 (supp. Sec. "Additional Implementation
Details").
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import (PARAM_KEYS, Renderer, Scene, gs_loss_l1, gs_outlier_mask, gs_pose_adam, gs_pose_grad,
               gs_render_backward, gs_render_forward_l1, gs_select_reliable, gs_workspace_query, gs_workspace_status,
               alloc_workspace, GS_ERR_CAPACITY, _check)

MAP_LR = {"mean": 1.6e-5, "log_scale": 2e-4, "quat": 4e-5, "opacity_logit": 1e-2, "sh": 5e-4}
MEAN_LR_FINAL = 1.7e-7
POSE_LR = (2e-4, 2e-4, 2e-4, 5e-4, 5e-4, 5e-4)


def mean_lr(step, total=100, lr0=MAP_LR["mean"], lr1=MEAN_LR_FINAL):
    """Log-linear decay of the position learning rate from lr0 to lr1 over `total` steps
    (0 stays 0)."""
    if lr0 <= 0.0:
        return 0.0
    t = min(max(step / max(total, 1), 0.0), 1.0)
    return math.exp((1 - t) * math.log(lr0) + t * math.log(lr1))


class MapAdam:
    """torch Adam over a scene's five parameter planes (each its own group)."""

    def __init__(self, scene: Scene, lr=None, decay_steps=100):
        lr = dict(MAP_LR, **(lr or {}))
        # the position rate decays from its start by the paper's ratio (1.7e-7 / 1.6e-5)
        self.mean_lr0 = lr["mean"]
        self.mean_lr1 = lr["mean"] * MEAN_LR_FINAL / MAP_LR["mean"]
        self.params = {k: getattr(scene, k) for k in PARAM_KEYS}
        for p in self.params.values():
            p.requires_grad_(False)
        self.opt = torch.optim.Adam([{"params": [p], "lr": lr[k], "name": k} for k, p in self.params.items()],
                                    eps=1e-15)
        self.decay_steps = decay_steps
        self.steps = 0

    def step(self, grads):
        for g in self.opt.param_groups:
            (p,) = g["params"]
            p.grad = grads[g["name"]]
            if g["name"] == "mean":
                g["lr"] = mean_lr(self.steps, self.decay_steps, self.mean_lr0, self.mean_lr1)
        self.opt.step()
        self.steps += 1


def select_keyframes(n_keyframes, K, seed):
    """K keyframes drawn without replacement from the window (all when K >= n)."""
    rng = np.random.default_rng(seed)
    if K >= n_keyframes:
        return list(range(n_keyframes))
    return sorted(rng.choice(n_keyframes, K, replace=False).tolist())


def bundle_adjust(renderer: Renderer, scene: Scene, views, poses, targets, iters=100, K=10, w_c=0.8, w_d=0.3,
                  pose_lr=POSE_LR, seed=0, map_opt: MapAdam | None = None):
    """Eq. BA on a keyframe window.

    views   : keyframe view dicts (intrinsics, size; their T_cw is ignored)
    poses   : float32 CUDA tensor [n_keyframes, 12], world->camera [R | t] row-major,
              updated in place in the second half of the iterations
    targets : per keyframe (rgb [3, H, W], depth [H, W]) numpy or tensors
    Returns the per-iteration BA loss (numpy, length iters) and the selected keyframes.
    The losses stay on the device until the loop ends: after the first iteration (which
    reads the pair count once to size the pair list) no iteration waits for the GPU.
    """
    dev = renderer.device
    sel = select_keyframes(len(views), K, seed)
    k = len(sel)
    batch = [dict(views[i], scene=0, T_cw_dev=poses[i]) for i in sel]
    trgb = torch.cat([torch.as_tensor(np.asarray(targets[i][0], np.float32), device=dev).reshape(-1) for i in sel])
    tdep = torch.cat([torch.as_tensor(np.asarray(targets[i][1], np.float32), device=dev).reshape(-1) for i in sel])
    P = sum(int(v["width"]) * int(v["height"]) for v in batch)
    color, depth = torch.empty(3 * P, device=dev), torch.empty(P, device=dev)
    dC, dD = torch.empty(3 * P, device=dev), torch.empty(P, device=dev)
    loss = torch.zeros(k, device=dev)
    grads = {kk: torch.zeros_like(getattr(scene, kk)) for kk in PARAM_KEYS}
    dtw = torch.zeros(k, 6, device=dev)
    # pose Adam state of the selected keyframes ([k][16]: m, v, step) and their poses
    kf_poses = poses[sel].contiguous()
    state = torch.zeros(k, 16, device=dev)
    opt = map_opt or MapAdam(scene, decay_steps=iters)
    ctx = renderer.ctx
    ctx.set_grad_mode(1)  # the backward writes the gradients; no zeroing between iterations
    ws, mp = renderer.new_workspace([scene], batch)
    losses = torch.zeros(iters, device=dev)
    for it in range(iters):
        batch = [dict(b, T_cw_dev=kf_poses[j]) for j, b in enumerate(batch)]
        for attempt in range(4):
            gs_render_forward_l1(ctx, [scene], batch, ws, mp, (color, depth, None), trgb, tdep, w_c / k, w_d / k,
                                 loss, (dC, dD, None))
            if it > 0:
                break
            st, needed = gs_workspace_status(ctx, ws)  # size the pair list on the first iteration
            if st != GS_ERR_CAPACITY:
                _check(ctx, st)
                break
            renderer.max_pairs = mp = int(needed * 1.25) + 4096
            ws = alloc_workspace(gs_workspace_query(ctx, [scene], batch, mp), dev)
        gs_render_backward(ctx, [scene], batch, ws, mp, (dC, dD, None), [grads], dtw, 0)
        opt.step(grads)
        if it >= iters // 2:  # poses only in the second half (supp. implementation details)
            gs_pose_adam(ctx, kf_poses, dtw, state, pose_lr)
        losses[it] = loss.sum()  # a device copy: no host synchronisation
    poses[sel] = kf_poses
    return losses.cpu().numpy().astype(np.float64), sel


# ----------------------------------------------------------------------------
# coarse-to-fine tracking of one frame (Sec. 3.3)
# ----------------------------------------------------------------------------
def constant_velocity(T_prev2, T_prev1):
    """Pose guess of the next frame from the two last poses (world->camera, 3x4):
    the last pose moved by their relative motion, (T1 T2^-1) T1."""
    def h(T):
        M = np.eye(4)
        M[:3, :] = np.asarray(T, np.float64).reshape(3, 4)
        return M
    A, B = h(T_prev2), h(T_prev1)
    return (B @ np.linalg.inv(A) @ B)[:3, :]


def coarse_view(view):
    """The half-resolution camera whose pixel (u, v) looks through the centre of the
    full-resolution pixel (2u, 2v): focal lengths halved, principal point
    ((c + 0.5) / 2); its observed image is the even-indexed pixels of the frame."""
    return dict(view, width=int(view["width"]) // 2, height=int(view["height"]) // 2, fx=view["fx"] / 2.0,
                fy=view["fy"] / 2.0, cx=(view["cx"] + 0.5) / 2.0, cy=(view["cy"] + 0.5) / 2.0)


def track_frame(renderer: Renderer, scene: Scene, view, T_prev2, T_prev1, obs_rgb, obs_depth, iters_coarse=5,
                iters_fine=5, coarse_fraction=0.25, eps=0.05, outlier_factor=10.0, w_c=0.8, observed_acc=0.5,
                pose_lr=POSE_LR, pose_mode=1, seed=0):
    """Coarse-to-fine pose estimation of one frame (Sec. 3.3, Eq. track_loss, Eq.
    coarse2fine) on the library's kernels.

    1. Constant-velocity guess from the two last poses.
    2. Coarse: iters_coarse Adam steps on the photometric L1 at half resolution over
       a uniform random coarse_fraction of the pixels.
    3. Fine: the Gaussians Eq. coarse2fine keeps (|D - d| <= eps under the coarse
       pose), full resolution, iters_fine Adam steps.
    Pixels are rendered only where the map was observed (accumulated opacity above
    observed_acc at the guess); every iteration ignores the pixels whose loss exceeds
    outlier_factor x the median (supp. tracking hyper-parameters).  pose_mode 1 is the
    paper's approximate pose gradient (view-independent colour, no dSigma'/dP).
    obs_rgb [3, H, W], obs_depth [H, W] CUDA float32.  Returns the pose (3x4 numpy)
    and a per-iteration log (loss, pixels kept)."""
    ctx = renderer.ctx
    dev = renderer.device
    W, H = int(view["width"]), int(view["height"])
    T = torch.as_tensor(constant_velocity(T_prev2, T_prev1).reshape(1, 12), dtype=torch.float32, device=dev)
    state = torch.zeros(1, 16, device=dev)
    dtw = torch.zeros(1, 6, device=dev)
    ctx.set_grad_mode(1)
    log = []

    def observed(v, n_pix):
        _, _, acc, *_ = renderer.forward([scene], [dict(v, T_cw_dev=T[0], pixel_mask=None)],
                                         want=("color", "acc"))
        return (acc > observed_acc).to(torch.uint8).view(int(v["height"]), int(v["width"]))

    def stage(v, scn, trgb, tdep, base_mask, iters):
        P = int(v["width"]) * int(v["height"])
        color, depth = torch.empty(3 * P, device=dev), torch.empty(P, device=dev)
        dC, dD = torch.empty(3 * P, device=dev), torch.empty(P, device=dev)
        keep = torch.empty(P, dtype=torch.uint8, device=dev)
        loss = torch.zeros(1, device=dev)
        fv = dict(v, T_cw_dev=T[0], pixel_mask=base_mask)
        ws, mp = renderer.new_workspace([scn], [fv])
        for _ in range(iters):
            color, depth, _, ws, mp = renderer.forward([scn], [fv], workspace=ws, want=("color", "depth"))
            gs_outlier_mask(ctx, [fv], (color, depth), trgb, tdep, w_c, 0.0, outlier_factor, keep)
            lv = dict(fv, pixel_mask=keep.view(base_mask.shape))
            gs_loss_l1(ctx, [lv], (color, depth, None), trgb, tdep, w_c, 0.0, loss, (dC, dD, None))
            gs_pose_grad(ctx, [scn], [fv], ws, mp, (dC, dD, None), dtw, pose_mode)
            gs_pose_adam(ctx, T, dtw, state, pose_lr)
            log.append((float(loss.item()), int(keep.sum().item())))

    # coarse: even-indexed pixels of the frame, a uniform random subset of them
    cv = coarse_view(view)
    Wc, Hc = int(cv["width"]), int(cv["height"])
    crgb = obs_rgb[:, 0:2 * Hc:2, 0:2 * Wc:2].contiguous().reshape(-1)
    cdep = obs_depth[0:2 * Hc:2, 0:2 * Wc:2].contiguous().reshape(-1)
    rng = np.random.default_rng(seed)
    sub = torch.as_tensor((rng.random((Hc, Wc)) < coarse_fraction).astype(np.uint8), device=dev)
    stage(cv, scene, crgb, cdep, observed(cv, Wc * Hc) & sub, iters_coarse)
    # fine: Eq. coarse2fine selection under the coarse pose, full resolution
    sel = torch.zeros(scene.n, dtype=torch.uint8, device=dev)
    gs_select_reliable(ctx, scene, dict(view, T_cw_dev=T[0]), obs_depth.reshape(-1).contiguous(), eps, sel)
    fine = Scene(*scene.params(), scene.sh_degree, mask=sel)
    stage(view, fine, obs_rgb.reshape(-1).contiguous(), obs_depth.reshape(-1).contiguous(),
          observed(view, W * H), iters_fine)
    return T[0].cpu().numpy().astype(np.float64).reshape(3, 4), log
