"""Helpers shared by the GPU parity tests: running the CUDA path through the C
ABI, reading its saved state, and the near-threshold pixel policy."""
import numpy as np
import torch

# A pixel is compared only when every threshold decision it took is farther from
# its threshold than float32 evaluation can blur (the oracle reports the margins):
#   gate  |q - 9| / (9 (1 + cond))        > 1e-6
#   alpha |a - 1/255| 255 / (1 + cond)    > 1e-5
#   stop  |T(1 - a) - 1e-4| / 1e-4        > 1e-4
#   clamp |o G - 0.99| / (1 + cond)       > 1e-5   (gradients only)
MARGINS = {"m_gate": 1e-6, "m_alpha": 1e-5, "m_stop": 1e-4}
GRAD_MARGINS = dict(MARGINS, m_clamp=1e-5)

COLOR_ABS = 1e-4     # colour: absolute
DEPTH_REL = 1e-4     # depth: relative
GRAD_REL_L2 = 1e-3   # each gradient tensor: relative L2


def resolvable(ref, margins=MARGINS):
    ok = np.ones(ref["m_gate"].shape, bool)
    for k, tol in margins.items():
        ok &= ref[k] > tol
    return ok


def run_forward(G, R, scenes_np, views, masks=None):
    scenes = [G.Scene.from_numpy(s, mask=None if masks is None else masks[i]) for i, s in enumerate(scenes_np)]
    color, depth, acc, ws, mp = R.forward(scenes, views)
    torch.cuda.synchronize()
    return scenes, color, depth, acc, ws, mp


def split_views(views, color, depth, acc):
    """Packed images -> per-view numpy (color [3,H,W], depth [H,W], acc [H,W])."""
    out = []
    o = 0
    for v in views:
        W, H = int(v["width"]), int(v["height"])
        c = color[3 * o:3 * (o + W * H)].view(3, H, W).cpu().numpy() if color is not None else None
        d = depth[o:o + W * H].view(H, W).cpu().numpy() if depth is not None else None
        a = acc[o:o + W * H].view(H, W).cpu().numpy() if acc is not None else None
        out.append((c, d, a))
        o += W * H
    return out


def read_state(G, R, scenes, views, ws, mp):
    """The forward's saved state from the workspace (see gs_workspace_layout)."""
    lay = G.gs_workspace_layout(R.ctx, scenes, views, mp)
    S, T = lay.n_splats, lay.n_tiles
    b = ws.cpu().numpy()

    def arr(off, dtype, count):
        return np.frombuffer(b[off:off + np.dtype(dtype).itemsize * count].tobytes(), dtype=dtype).copy()

    hdr = arr(lay.header, np.uint32, 5)
    rec = arr(lay.rec, np.float32, S * 16).reshape(S, 16)
    rect = arr(lay.rect, np.uint32, S * 4).reshape(S, 4)
    ntiles = arr(lay.ntiles, np.uint32, S)
    dkey = arr(lay.dkey, np.uint32, S)
    ranges = arr(lay.ranges, np.uint32, T * 2).reshape(T, 2)
    pairs = arr(lay.pair_val, np.uint32, int(hdr[2]))
    order = arr(lay.order, np.uint32, T)
    return dict(layout=lay, hdr=hdr, rec=rec, rect=rect, ntiles=ntiles, dkey=dkey, ranges=ranges, pairs=pairs,
                order=order)


def gpu_loss_and_grads(G, R, scenes, views, targets, w_c, w_d, pose_mode=0, want_params=True):
    """Forward, fused L1 loss adjoint and backward through the C ABI."""
    dev = R.device
    color, depth, acc, ws, mp = R.forward(scenes, views)
    trgb = torch.as_tensor(np.concatenate([np.asarray(t[0], np.float32).reshape(-1) for t in targets]), device=dev)
    tdep = torch.as_tensor(np.concatenate([np.asarray(t[1], np.float32).reshape(-1) for t in targets]), device=dev)
    loss = torch.zeros(len(views), device=dev)
    dC, dD = torch.empty_like(color), torch.empty_like(depth)
    G.gs_loss_l1(R.ctx, views, (color, depth, acc), trgb, tdep, w_c, w_d, loss, (dC, dD, None))
    dtw = torch.zeros(len(views), 6, device=dev)
    if want_params:
        grads = [{k: torch.zeros_like(getattr(s, k)) for k in G.PARAM_KEYS} for s in scenes]
        G.gs_render_backward(R.ctx, scenes, views, ws, mp, (dC, dD, None), grads, dtw, pose_mode)
    else:
        grads = None
        G.gs_pose_grad(R.ctx, scenes, views, ws, mp, (dC, dD, None), dtw, pose_mode)
    torch.cuda.synchronize()
    st, _ = G.gs_workspace_status(R.ctx, ws)
    assert st == G.GS_OK
    g_np = None if grads is None else [{k: v.cpu().numpy().astype(np.float64) for k, v in g.items()} for g in grads]
    return dict(loss=loss.cpu().numpy(), grads=g_np, twist=dtw.cpu().numpy().astype(np.float64),
                images=split_views(views, color, depth, acc))


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30))


def image_parity(view, color, depth, acc, ref, pixels):
    """GPU images (color [3,H,W], depth, acc [H,W] numpy) against the oracle on every
    pixel of `pixels` (bool [H,W]).  A pixel whose threshold decisions all lie beyond
    float32 reach (resolvable) is compared with the oracle's render `ref`; any other
    pixel must match one of the outcomes the definition allows when its near
    decisions go either way (oracle.pixel_alternatives on ref's projection).
    Tolerances: colour and opacity COLOR_ABS absolute, depth DEPTH_REL relative.
    Returns (pixels compared, pixels checked against alternatives, pixels with more
    near decisions than the alternatives enumerate)."""
    import oracle as O
    ok = resolvable(ref) & pixels
    if ok.any():
        assert np.abs(color - ref["color"])[:, ok].max() < COLOR_ABS
        rel = np.abs(depth - ref["depth"]) / np.maximum(np.abs(ref["depth"]), 1e-12)
        assert rel[ok & (ref["depth"] > 0)].max(initial=0.0) < DEPTH_REL
        assert np.abs(depth[ok & (ref["depth"] == 0)]).max(initial=0.0) == 0.0
        assert np.abs(acc - ref["acc"])[ok].max() < COLOR_ABS
    near = pixels & ~ok
    unresolved = 0
    for yy, xx in zip(*np.nonzero(near)):
        alts = O.pixel_alternatives(ref["proj"], view, int(xx), int(yy))
        if alts is None:
            unresolved += 1
            continue

        def match(a):
            return (np.abs(color[:, yy, xx] - a["color"]).max() < COLOR_ABS and
                    abs(depth[yy, xx] - a["depth"]) <= DEPTH_REL * abs(a["depth"]) + 1e-9 and
                    abs(acc[yy, xx] - a["acc"]) < COLOR_ABS)
        assert any(match(a) for a in alts), (int(xx), int(yy), color[:, yy, xx], depth[yy, xx], alts)
    return int(pixels.sum()), int(near.sum()), unresolved
