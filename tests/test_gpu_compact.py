"""GPU parity of the compacted-pixel compositing kernels (gs_ctx_set_compact):
identical images, runs and loss adjoints to the warp-strip kernels on sparse and
dense pixel masks, every tile shape and ragged image edges; gradients against the
FP64 oracle on a sparse pixel subset; the backward revisits exactly the forward's
blended pairs."""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from gpu_util import GRAD_MARGINS, GRAD_REL_L2, rel_l2, resolvable, split_views

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_11700_gb300 import build
    build.build()
    import paper_2311_11700_gb300 as g
    return g


def _scene_view(seed, n, W, H):
    sc = synth.room_scene(seed, n=n)
    vw = synth.room_view(W, H, f=0.5 * W)
    return sc, vw


def _fused(G, R, scenes, views, trgb, tdep):
    """Forward with the fused L1 loss: images, loss, adjoints and the workspace."""
    P = sum(v["width"] * v["height"] for v in views)
    color, depth, acc, ws, mp = R.forward(scenes, views)  # sizes the pair list
    loss = torch.zeros(len(views), device="cuda")
    dC, dD, dA = torch.empty(3 * P, device="cuda"), torch.empty(P, device="cuda"), torch.empty(P, device="cuda")
    G.gs_render_forward_l1(R.ctx, scenes, views, ws, mp, (color, depth, acc), trgb, tdep, 1.0, 0.5, loss,
                           (dC, dD, dA))
    torch.cuda.synchronize()
    return dict(color=color, depth=depth, acc=acc, loss=loss, dC=dC, dD=dD, dA=dA, ws=ws, mp=mp)


def _grads(G, R, scenes, views, f):
    grads = [{k: torch.zeros_like(getattr(s, k)) for k in G.PARAM_KEYS} for s in scenes]
    dtw = torch.zeros(len(views), 6, device="cuda")
    G.gs_render_backward(R.ctx, scenes, views, f["ws"], f["mp"], (f["dC"], f["dD"], None), grads, dtw, 0)
    torch.cuda.synchronize()
    st, _ = G.gs_workspace_status(R.ctx, f["ws"])
    assert st == G.GS_OK
    return [{k: v.cpu().numpy().astype(np.float64) for k, v in g.items()} for g in grads], dtw.cpu().numpy()


@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (16, 8), (32, 8)])
@pytest.mark.parametrize("fraction", [0.1, 1.0])
def test_compact_equals_strips(G, tile, fraction):
    """Same images, loss adjoints (bit for bit) and gradients (to summation order)
    from both forms; 101 x 67 leaves ragged tiles on two edges, two views of two
    scenes, one of them with a denser mask."""
    sa, va = _scene_view(81, 3000, 101, 67)
    sb, vb = _scene_view(82, 1500, 64, 40)
    vb["scene"] = 1
    masks = [synth.pixel_subset_mask(83, 101, 67, fraction), synth.pixel_subset_mask(84, 64, 40, min(1.0, 3 * fraction))]
    views = [dict(va, scene=0, pixel_mask=torch.as_tensor(masks[0], device="cuda")),
             dict(vb, pixel_mask=torch.as_tensor(masks[1], device="cuda"))]
    scenes = [G.Scene.from_numpy(sa), G.Scene.from_numpy(sb)]
    tg = [synth.zbuffer_targets(sa, va, 85), synth.zbuffer_targets(sb, vb, 86)]
    trgb = torch.as_tensor(np.concatenate([t[0].reshape(-1) for t in tg]), device="cuda")
    tdep = torch.as_tensor(np.concatenate([t[1].reshape(-1) for t in tg]), device="cuda")
    out = {}
    for mode in (0, 1):
        R = G.Renderer(0, tile)
        R.ctx.set_compact(mode)
        f = _fused(G, R, scenes, views, trgb, tdep)
        out[mode] = (f, _grads(G, R, scenes, views, f))
    f0, f1 = out[0][0], out[1][0]
    for k in ("color", "depth", "acc", "dC", "dD", "dA"):
        assert torch.equal(f0[k], f1[k]), k
    np.testing.assert_allclose(f1["loss"].cpu().numpy(), f0["loss"].cpu().numpy(), rtol=1e-5)
    (g0, t0), (g1, t1) = out[0][1], out[1][1]
    for s in range(2):
        for k in G.PARAM_KEYS:
            assert rel_l2(g1[s][k], g0[s][k]) < 1e-5, (s, k)
    assert rel_l2(t1, t0) < 1e-5
    # masked-out pixels: zero colour, depth and opacity, zero adjoints
    c, d, a = split_views(views, f1["color"], f1["depth"], f1["acc"])[0]
    m = masks[0] == 0
    assert (c[:, m] == 0).all() and (d[m] == 0).all() and (a[m] == 0).all()


def test_compact_always_on_unmasked_views(G):
    """Mode 2 serves views without a pixel mask: every pixel is gathered, 32 at a time."""
    sc, vw = _scene_view(91, 2500, 77, 53)
    scenes = [G.Scene.from_numpy(sc)]
    res = []
    for mode in (0, 2):
        R = G.Renderer(0)
        R.ctx.set_compact(mode)
        c, d, a, *_ = R.forward(scenes, [vw])
        torch.cuda.synchronize()
        res.append((c.clone(), d.clone(), a.clone()))
    for x, y in zip(*res):
        assert torch.equal(x, y)


@pytest.mark.parametrize("pose_mode", [0, 1])
def test_compact_gradients_match_oracle_on_a_sparse_subset(G, pose_mode):
    """The tracking shape: a 10 % pixel subset (intersected with the resolvable
    pixels) through the compacted kernels against the FP64 oracle."""
    sc, vw = _scene_view(93, 2000, 120, 88)
    rgb, dep = synth.zbuffer_targets(sc, vw, 94)
    ref_f = O.render_view(sc, vw)
    ok = resolvable(ref_f, GRAD_MARGINS) & (synth.pixel_subset_mask(95, 120, 88, 0.1) != 0)
    m = ok.astype(np.uint8)
    R = G.Renderer(0)
    assert R.ctx.compact == 1
    v2 = dict(vw, pixel_mask=torch.as_tensor(m, device="cuda"))
    scenes = [G.Scene.from_numpy(sc)]
    color, depth, acc, ws, mp = R.forward(scenes, [v2])
    loss = torch.zeros(1, device="cuda")
    dC, dD = torch.empty_like(color), torch.empty_like(depth)
    G.gs_loss_l1(R.ctx, [v2], (color, depth, acc), torch.as_tensor(rgb.reshape(-1), device="cuda"),
                 torch.as_tensor(dep.reshape(-1), device="cuda"), 1.0, 0.5, loss, (dC, dD, None))
    grads = [{k: torch.zeros_like(getattr(scenes[0], k)) for k in G.PARAM_KEYS}]
    dtw = torch.zeros(1, 6, device="cuda")
    G.gs_render_backward(R.ctx, scenes, [v2], ws, mp, (dC, dD, None), grads, dtw, pose_mode)
    torch.cuda.synchronize()
    ref = O.render_and_grad([sc], [vw], [(rgb, dep)], 1.0, 0.5, pixel_masks=[m],
                            pose_mode="paper" if pose_mode else "exact")
    assert abs(loss.item() - ref["loss"]) / ref["loss"] < 1e-5
    for k in O.PARAM_KEYS:
        e = rel_l2(grads[0][k].cpu().numpy().astype(np.float64), ref["grads"][0][k])
        assert e < GRAD_REL_L2, (k, e)
    assert rel_l2(dtw.cpu().numpy().astype(np.float64), ref["twist"]) < GRAD_REL_L2


def test_compact_backward_revisits_the_forward_pairs(G):
    """With timing on the kernels count blended pairs: equal forward and backward
    counts, and equal to the strip form's count."""
    sc, vw = _scene_view(97, 4000, 160, 96)
    m = synth.pixel_subset_mask(98, 160, 96, 0.1)
    v = dict(vw, pixel_mask=torch.as_tensor(m, device="cuda"))
    counts = []
    for mode in (0, 1):
        R = G.Renderer(0)
        R.ctx.set_compact(mode)
        scenes = [G.Scene.from_numpy(sc)]
        G.gs_ctx_set_timing(R.ctx, True)
        try:
            color, depth, acc, ws, mp = R.forward(scenes, [v])
            dtw = torch.zeros(1, 6, device="cuda")
            G.gs_pose_grad(R.ctx, scenes, [v], ws, mp, (torch.ones_like(color), torch.ones_like(depth), None), dtw,
                           0)
            vis, pairs, nf, nb, *_ = G.gs_workspace_counters(R.ctx, ws)
        finally:
            G.gs_ctx_set_timing(R.ctx, False)
            G.gs_ctx_read_timing(R.ctx, reset=True)
        assert nf == nb > 0
        counts.append(nf)
    assert counts[0] == counts[1]


def test_compact_mode_is_validated(G):
    R = G.Renderer(0)
    with pytest.raises(G.GsrError):
        R.ctx.set_compact(3)
    R.ctx.set_compact(0)
    assert R.ctx.compact == 0
