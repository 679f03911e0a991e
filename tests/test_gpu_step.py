"""GPU tests of gs_render_step_l1 (forward, fused L1 loss and backward in one
compositing kernel): equal to gs_render_forward_l1 + gs_render_backward (images
bit for bit, gradients to float-atomic order) in every tiling, strip, compacted
pixel form, batch and gradient mode; the pose-only form equals gs_pose_grad; the
backward walk revisits exactly the forward's blended pairs; parity with the
FP64 oracle; argument errors."""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from gpu_util import GRAD_MARGINS, GRAD_REL_L2, read_state, rel_l2, resolvable

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_11700_gb300 import build
    build.build()
    import paper_2311_11700_gb300 as g
    return g


def _case(seed=11, masked=False):
    """Two views of two scenes (one of them ragged), SH3, z-buffer targets."""
    sa, va = synth.room_scene(seed, n=3000), synth.room_view(101, 67, f=50.0)
    sb, vb = synth.room_scene(seed + 1, n=1500), synth.room_view(64, 48, f=32.0)
    vb["scene"] = 1
    va = dict(va, scene=0)
    if masked:
        va["pixel_mask"] = torch.as_tensor(synth.pixel_subset_mask(seed + 2, 101, 67, 0.1), device="cuda")
        vb["pixel_mask"] = torch.as_tensor(synth.pixel_subset_mask(seed + 3, 64, 48, 0.3), device="cuda")
    tg = [synth.zbuffer_targets(sa, va, seed + 4), synth.zbuffer_targets(sb, vb, seed + 5)]
    return [sa, sb], [va, vb], tg


def _run(G, R, scenes_np, views, targets, fused, params=True, grad_mode=0):
    R.ctx.set_grad_mode(grad_mode)
    scenes = [G.Scene.from_numpy(s) for s in scenes_np]
    P = sum(v["width"] * v["height"] for v in views)
    color, depth, acc, ws, mp = R.forward(scenes, views)  # sizes the pair list
    trgb = torch.as_tensor(np.concatenate([t[0].reshape(-1) for t in targets]), device="cuda")
    tdep = torch.as_tensor(np.concatenate([t[1].reshape(-1) for t in targets]), device="cuda")
    loss = torch.zeros(len(views), device="cuda")
    grads = [{k: torch.zeros_like(getattr(s, k)) for k in G.PARAM_KEYS} for s in scenes] if params else None
    dtw = torch.zeros(len(views), 6, device="cuda")
    if fused:
        G.gs_render_step_l1(R.ctx, scenes, views, ws, mp, (color, depth, acc), trgb, tdep, 1.0, 0.5, loss, grads, dtw)
    else:
        dC, dD = torch.empty(3 * P, device="cuda"), torch.empty(P, device="cuda")
        G.gs_render_forward_l1(R.ctx, scenes, views, ws, mp, (color, depth, acc), trgb, tdep, 1.0, 0.5, loss,
                               (dC, dD, None))
        if params:
            G.gs_render_backward(R.ctx, scenes, views, ws, mp, (dC, dD, None), grads, dtw)
        else:
            G.gs_pose_grad(R.ctx, scenes, views, ws, mp, (dC, dD, None), dtw)
    torch.cuda.synchronize()
    st, _ = G.gs_workspace_status(R.ctx, ws)
    assert st == G.GS_OK
    return dict(color=color.clone(), depth=depth.clone(), acc=acc.clone(), loss=loss.cpu().numpy(),
                twist=dtw.cpu().numpy().astype(np.float64),
                grads=None if grads is None else [{k: v.cpu().numpy().astype(np.float64) for k, v in g.items()}
                                                  for g in grads])


def _same(a, b, params=True):
    for k in ("color", "depth", "acc"):
        assert torch.equal(a[k], b[k]), k
    np.testing.assert_allclose(a["loss"], b["loss"], rtol=1e-6)
    if params:
        for s in range(len(a["grads"])):
            for k in a["grads"][s]:
                assert rel_l2(a["grads"][s][k], b["grads"][s][k]) < 1e-5, (s, k)
    assert rel_l2(a["twist"], b["twist"]) < 1e-5


@pytest.mark.parametrize("tile,strip", [((16, 16), 2), ((16, 16), 0), ((16, 16), 1), ((16, 16), 4), ((8, 8), 0),
                                        ((16, 8), 0), ((32, 8), 0)])
def test_step_equals_separate_calls(G, tile, strip):
    sc, vw, tg = _case()
    R = G.Renderer(0, tile)
    R.ctx.set_strip(strip, strip)
    _same(_run(G, R, sc, vw, tg, True), _run(G, R, sc, vw, tg, False))


@pytest.mark.parametrize("tile,strip,masked", [((16, 16), 2, False), ((16, 16), 1, False), ((8, 8), 0, False),
                                               ((16, 16), 2, True), ((32, 8), 0, True)])
def test_persistent_step_equals_grid_step(G, tile, strip, masked):
    """The persistent form of the fused step (warps taking (tile, strip) items from
    a ticket; tiles in the compacted-pixel form) gives the grid form's images bit
    for bit and its gradients up to the order of the float atomics, twice in a row
    on the same workspace (the ticket restarts with every call)."""
    sc, vw, tg = _case(41, masked=masked)
    R = G.Renderer(0, tile)
    R.ctx.set_strip(strip, strip)
    grid = _run(G, R, sc, vw, tg, True)
    R.ctx.set_persistent(1)
    for _ in range(2):
        _same(_run(G, R, sc, vw, tg, True), grid)
    R.ctx.set_persistent(0)


@pytest.mark.parametrize("grad_mode", [0, 1])
def test_step_compacted_pixels_and_grad_modes(G, grad_mode):
    sc, vw, tg = _case(21, masked=True)
    R = G.Renderer(0)
    _same(_run(G, R, sc, vw, tg, True, grad_mode=grad_mode), _run(G, R, sc, vw, tg, False, grad_mode=grad_mode))


@pytest.mark.parametrize("masked", [False, True])
def test_step_pose_only_equals_pose_grad(G, masked):
    sc, vw, tg = _case(31, masked=masked)
    R = G.Renderer(0)
    _same(_run(G, R, sc, vw, tg, True, params=False), _run(G, R, sc, vw, tg, False, params=False), params=False)


def test_step_backward_walk_revisits_the_forward_pairs(G):
    sc, vw, tg = _case(41)
    R = G.Renderer(0)
    scenes = [G.Scene.from_numpy(s) for s in sc]
    color, depth, acc, ws, mp = R.forward(scenes, vw)
    trgb = torch.as_tensor(np.concatenate([t[0].reshape(-1) for t in tg]), device="cuda")
    tdep = torch.as_tensor(np.concatenate([t[1].reshape(-1) for t in tg]), device="cuda")
    loss = torch.zeros(2, device="cuda")
    dtw = torch.zeros(2, 6, device="cuda")
    G.gs_ctx_set_timing(R.ctx, True)
    try:
        G.gs_render_step_l1(R.ctx, scenes, vw, ws, mp, None, trgb, tdep, 1.0, 0.5, loss, None, dtw)
        vis, pairs, nf, nb, *_ = G.gs_workspace_counters(R.ctx, ws)
        stages = G.gs_ctx_read_timing(R.ctx, reset=True)
    finally:
        G.gs_ctx_set_timing(R.ctx, False)
    assert nf == nb > 0
    assert stages["composite_step"][1] == 1 and stages["composite_fwd"][1] == 0


def _faint_crowd(n, seed):
    """n wide, faint, anisotropic Gaussians over a 40x36 view: every one blends at every
    pixel with alpha ~0.0041, so the tile lists hold n entries and the runs stay open
    for about 2240 blends (T reaches 1e-4 after that many)."""
    rng = np.random.default_rng(seed)
    W, H, f = 40, 36, 30.0
    vw = synth.make_view(W, H, f, f, W / 2, H / 2, np.concatenate([np.eye(3), np.zeros((3, 1))], 1))
    z = rng.uniform(2.0, 6.0, n)
    px, py = rng.normal(W / 2, 3.0, n), rng.normal(H / 2, 3.0, n)
    mean = np.stack([(px - W / 2) * z / f, (py - H / 2) * z / f, z])
    # anisotropic (axes 1 : 0.8 : 0.6), so that every parameter has a gradient
    sigma = rng.uniform(160.0, 220.0, n) * z / f
    sc = dict(mean=mean.astype(np.float32),
              log_scale=np.log(np.stack([sigma, 0.8 * sigma, 0.6 * sigma])).astype(np.float32),
              quat=rng.normal(0, 1, (4, n)).astype(np.float32),
              opacity_logit=np.full(n, np.log(0.0041 / 0.9959), np.float32),
              sh=rng.normal(0, 1, (3, n)).astype(np.float32), sh_degree=0)
    return sc, dict(vw, scene=0)


def test_step_runs_beyond_the_recorded_culls(G):
    """The fused step's backward walk stages the forward walk's recorded cull ballots
    for the first 64 batches of a list (2048 entries) and culls again beyond them.
    Lists of 3000 entries with runs past 2048 take both paths: the step still equals
    the separate calls (images bit for bit, gradients to float-atomic order), and the
    backward revisits exactly the forward's blended pairs."""
    sc, vw = _faint_crowd(3000, 61)
    tg = [synth.zbuffer_targets(sc, vw, 62)]
    R = G.Renderer(0)
    R.ctx.set_compact(0)
    _same(_run(G, R, [sc], [vw], tg, True), _run(G, R, [sc], [vw], tg, False))
    scenes = [G.Scene.from_numpy(sc)]
    color, depth, acc, ws, mp = R.forward(scenes, [vw])
    st = read_state(G, R, scenes, [vw], ws, mp)
    assert (st["ranges"][:, 1] - st["ranges"][:, 0]).max() > 2048
    trgb = torch.as_tensor(tg[0][0].reshape(-1), device="cuda")
    tdep = torch.as_tensor(tg[0][1].reshape(-1), device="cuda")
    loss = torch.zeros(1, device="cuda")
    dtw = torch.zeros(1, 6, device="cuda")
    G.gs_ctx_set_timing(R.ctx, True)
    try:
        G.gs_render_step_l1(R.ctx, scenes, [vw], ws, mp, None, trgb, tdep, 1.0, 0.5, loss, None, dtw)
        vis, pairs, nf, nb, *_ = G.gs_workspace_counters(R.ctx, ws)
    finally:
        G.gs_ctx_set_timing(R.ctx, False)
        G.gs_ctx_read_timing(R.ctx, reset=True)
    assert nf == nb
    # the mean run is past the 2048 recorded entries
    assert nb / (vw["width"] * vw["height"]) > 2048


def test_step_matches_oracle(G):
    w = synth.workload_plain_2k()
    ref_f = O.render_view(w["scenes"][0], w["views"][0])
    ok = resolvable(ref_f, GRAD_MARGINS).astype(np.uint8)
    ref = O.render_and_grad(w["scenes"], w["views"], w["targets"], w["w_c"], w["w_d"], pixel_masks=[ok])
    R = G.Renderer(0)
    R.ctx.set_compact(0)  # the strip form, although the view has a pixel mask
    vw = [dict(w["views"][0], pixel_mask=torch.as_tensor(ok, device="cuda"))]
    scenes = [G.Scene.from_numpy(w["scenes"][0])]
    color, depth, acc, ws, mp = R.forward(scenes, vw)
    t = w["targets"][0]
    loss = torch.zeros(1, device="cuda")
    grads = [{k: torch.zeros_like(getattr(scenes[0], k)) for k in G.PARAM_KEYS}]
    dtw = torch.zeros(1, 6, device="cuda")
    G.gs_render_step_l1(R.ctx, scenes, vw, ws, mp, None, torch.as_tensor(t[0].reshape(-1), device="cuda"),
                        torch.as_tensor(t[1].reshape(-1), device="cuda"), w["w_c"], w["w_d"], loss, grads, dtw)
    torch.cuda.synchronize()
    assert abs(loss.item() - ref["loss"]) / ref["loss"] < 1e-5
    for k in O.PARAM_KEYS:
        assert rel_l2(grads[0][k].cpu().numpy().astype(np.float64), ref["grads"][0][k]) < GRAD_REL_L2, k
    assert rel_l2(dtw.cpu().numpy().astype(np.float64), ref["twist"]) < GRAD_REL_L2


def test_step_argument_errors(G):
    sc, vw, tg = _case(51)
    R = G.Renderer(0)
    scenes = [G.Scene.from_numpy(s) for s in sc]
    color, depth, acc, ws, mp = R.forward(scenes, vw)
    trgb = torch.zeros(color.numel(), device="cuda")
    tdep = torch.zeros(depth.numel(), device="cuda")
    loss = torch.zeros(2, device="cuda")
    with pytest.raises(G.GsrError):  # neither parameter nor pose gradients requested
        G.gs_render_step_l1(R.ctx, scenes, vw, ws, mp, None, trgb, tdep, 1.0, 0.5, loss, None, None)
    with pytest.raises(G.GsrError):
        G.gs_render_step_l1(R.ctx, scenes, vw, ws, mp, None, trgb, tdep, float("nan"), 0.5, loss, None,
                            torch.zeros(2, 6, device="cuda"))
    # the step leaves no forward state: a following backward is refused
    dtw = torch.zeros(2, 6, device="cuda")
    G.gs_render_step_l1(R.ctx, scenes, vw, ws, mp, None, trgb, tdep, 1.0, 0.5, loss, None, dtw)
    with pytest.raises(G.GsrError):
        G.gs_pose_grad(R.ctx, scenes, vw, ws, mp, (trgb, tdep, None), dtw)
