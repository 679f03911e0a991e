"""CUDA-graph capture of the library's calls.

The batched forms are meant to be captured once and replayed (the benchmark's
batched mapping and tracking legs are). Every kernel of a call is launched with
programmatic stream serialisation and waits for its predecessors at entry, and a
call forks its short segment sorts onto a second stream and joins them with events.
A captured call must therefore give the same results as the same call made eagerly:
images bit for bit, and the gradients up to the order of the float atomics.
"""
import numpy as np
import pytest
import torch

import synth
from gpu_util import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_11700_gb300 import build
    build.build()
    import paper_2311_11700_gb300 as g
    return g


def _keyframes(seed, n_views=3, n=20_000, W=320, H=180):
    sc = synth.room_scene(seed, n=n)
    base = synth.room_view(W, H, f=W / 2.0)
    rng = np.random.default_rng(seed + 1)
    views = [synth.perturb_view(base, rng.normal(0.0, 0.05, 6)) for _ in range(n_views)]
    targets = [synth.zbuffer_targets(sc, v, seed + 10 + i) for i, v in enumerate(views)]
    return sc, views, targets


def _capture(fn):
    """fn() warmed on a side stream, then captured; returns the graph."""
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        fn()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn()
    torch.cuda.synchronize()
    return g


@pytest.mark.parametrize("fused", [True, False], ids=["step_l1", "forward_l1+backward"])
def test_captured_mapping_step_equals_eager(G, fused):
    sc, views, targets = _keyframes(301)
    R = G.Renderer(0)
    R.ctx.set_grad_mode(0)  # three views of one scene: gradients accumulate
    scene = G.Scene.from_numpy(sc)
    color, depth, acc, ws, mp = R.forward([scene], views)
    st, needed = G.gs_workspace_status(R.ctx, ws)
    mp = max(mp, int(needed * 1.2) + 1024)
    ws = G.alloc_workspace(G.gs_workspace_query(R.ctx, [scene], views, mp))
    trgb = torch.as_tensor(np.concatenate([t[0].reshape(-1) for t in targets]), device="cuda")
    tdep = torch.as_tensor(np.concatenate([t[1].reshape(-1) for t in targets]), device="cuda")
    loss = torch.zeros(len(views), device="cuda")
    dC, dD = torch.empty_like(color), torch.empty_like(depth)
    grads = [{k: torch.zeros_like(getattr(scene, k)) for k in G.PARAM_KEYS}]
    dtw = torch.zeros(len(views), 6, device="cuda")

    def step():
        for t in list(grads[0].values()) + [dtw]:
            t.zero_()
        if fused:
            G.gs_render_step_l1(R.ctx, [scene], views, ws, mp, (color, depth, acc), trgb, tdep, 1.0, 0.5, loss,
                                grads, dtw, 0)
        else:
            G.gs_render_forward_l1(R.ctx, [scene], views, ws, mp, (color, depth, acc), trgb, tdep, 1.0, 0.5, loss,
                                   (dC, dD, None))
            G.gs_render_backward(R.ctx, [scene], views, ws, mp, (dC, dD, None), grads, dtw, 0)

    step()
    torch.cuda.synchronize()
    st, _ = G.gs_workspace_status(R.ctx, ws)
    assert st == G.GS_OK
    ref = dict(color=color.clone(), depth=depth.clone(), acc=acc.clone(), loss=loss.clone(),
               grads={k: v.clone() for k, v in grads[0].items()}, twist=dtw.clone())
    g = _capture(step)
    for t in (color, depth, acc, loss, dtw):
        t.fill_(-1.0)
    for _ in range(2):  # replays reuse the workspace: the second must match too
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(color, ref["color"]) and torch.equal(depth, ref["depth"]) and torch.equal(acc, ref["acc"])
        assert torch.allclose(loss, ref["loss"], rtol=1e-5)
        for k in G.PARAM_KEYS:
            assert rel_l2(grads[0][k].cpu().numpy(), ref["grads"][k].cpu().numpy().astype(np.float64)) < 1e-5, k
        assert rel_l2(dtw.cpu().numpy(), ref["twist"].cpu().numpy().astype(np.float64)) < 1e-5
    st, _ = G.gs_workspace_status(R.ctx, ws)
    assert st == G.GS_OK


def test_captured_tracking_iterations_equal_eager(G):
    """Pose hypotheses with device-resident poses: the pose gradient (fused step) and
    the pose Adam step, several iterations captured in one graph."""
    sc, views, targets = _keyframes(311, n_views=4)
    R = G.Renderer(0)
    scene = G.Scene.from_numpy(sc)
    T0 = torch.as_tensor(np.stack([np.asarray(v["T_cw"], np.float32).reshape(12) for v in views]), device="cuda")
    T = T0.clone()
    vdev = [dict(views[0], T_cw_dev=T[i]) for i in range(len(views))]
    color, depth, acc, ws, mp = R.forward([scene], vdev)
    st, needed = G.gs_workspace_status(R.ctx, ws)
    mp = max(mp, int(needed * 1.5) + 1024)
    ws = G.alloc_workspace(G.gs_workspace_query(R.ctx, [scene], vdev, mp))
    # every hypothesis is fitted to the first keyframe's targets
    trgb = torch.as_tensor(np.tile(targets[0][0].reshape(-1), len(views)), device="cuda")
    tdep = torch.as_tensor(np.tile(targets[0][1].reshape(-1), len(views)), device="cuda")
    loss = torch.zeros(len(views), device="cuda")
    dtw = torch.zeros(len(views), 6, device="cuda")
    state = torch.zeros(len(views), 16, device="cuda")
    lr = [2e-4, 2e-4, 2e-4, 1e-3, 1e-3, 1e-3]

    def reset():
        T.copy_(T0)
        state.zero_()
        dtw.zero_()

    def iterations(k=3):
        for _ in range(k):
            G.gs_render_step_l1(R.ctx, [scene], vdev, ws, mp, None, trgb, tdep, 1.0, 0.5, loss, None, dtw, 0)
            G.gs_pose_adam(R.ctx, T, dtw, state, lr)

    reset()
    iterations()
    torch.cuda.synchronize()
    T_eager, l_eager = T.clone(), loss.clone()
    assert not torch.equal(T_eager, T0)  # the poses moved
    g = _capture(iterations)
    reset()
    g.replay()
    torch.cuda.synchronize()
    # the twist sums are float atomics, so Adam sees gradients equal to rounding
    assert torch.allclose(T, T_eager, atol=1e-5, rtol=0)
    assert torch.allclose(loss, l_eager, rtol=1e-4)
    st, _ = G.gs_workspace_status(R.ctx, ws)
    assert st == G.GS_OK
