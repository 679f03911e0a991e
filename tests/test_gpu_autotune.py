"""The autotuner: it picks a configuration from its search space by timing, the
images do not depend on the choice, the choice is cached by batch shape and the
cache survives a save / load round trip."""
import numpy as np
import pytest
import torch

import synth
from gpu_util import run_forward, split_views

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_11700_gb300 import build
    build.build()
    import paper_2311_11700_gb300 as g
    return g


def test_autotune_choice_is_valid_cached_and_result_neutral(G, tmp_path):
    sc = synth.room_scene(51, n=30_000)
    vw = synth.room_view(256, 144, f=128.0)
    R = G.Renderer(0)
    _, c0, d0, a0, *_ = run_forward(G, R, [sc], [vw])
    ref = split_views([vw], c0, d0, a0)[0]
    scenes = [G.Scene.from_numpy(sc)]
    res = R.autotune(scenes, [vw], reps=1)
    assert res["timed"] >= 2 * (6 + 6 + 3 * 2) - 6  # every tiling that fits was timed
    assert res["tile"] in [(16, 16), (16, 8), (8, 8), (32, 8)]
    assert res["binning"] in (0, 1) and res["ms_fwd"] > 0 and res["ms_bwd"] > 0
    if res["tile"] == (16, 16):
        assert 0 <= res["strip"][0] <= 5 and 0 <= res["strip"][1] <= 5
    assert (R.ctx.tile, R.ctx.strip, R.ctx.binning) == (res["tile"], res["strip"], res["binning"])
    # the tuned configuration renders the same images
    _, c1, d1, a1, *_ = run_forward(G, R, [sc], [vw])
    got = split_views([vw], c1, d1, a1)[0]
    for x, y in zip(got, ref):
        assert np.array_equal(x, y)
    # same shape: taken from the cache
    again = R.autotune(scenes, [vw], reps=1)
    assert again["timed"] == 0 and again["tile"] == res["tile"] and again["strip"] == res["strip"]
    # the cache survives a save / load round trip into another context
    path = tmp_path / "tune.txt"
    R.ctx.autotune_save(path)
    R2 = G.Renderer(0)
    R2.ctx.autotune_load(path)
    loaded = R2.autotune(scenes, [vw], reps=1)
    assert loaded["timed"] == 0 and (loaded["tile"], loaded["strip"], loaded["binning"]) == \
        (res["tile"], res["strip"], res["binning"])


def test_step_autotune_times_the_fused_step(G):
    """gs_autotune_step_l1: every strip shape s of 16x16 tiles timed as (s, s) with the
    fused step itself, its own cache keys (parameter step, pose-only step, separate
    calls), and the tuned step renders the untuned forward's images bit for bit."""
    sc = synth.room_scene(52, n=30_000)
    vw = synth.room_view(256, 144, f=128.0)
    R = G.Renderer(0)
    _, c0, d0, a0, *_ = run_forward(G, R, [sc], [vw])
    ref = split_views([vw], c0, d0, a0)[0]
    scenes = [G.Scene.from_numpy(sc)]
    P = vw["width"] * vw["height"]
    gen = torch.Generator(device="cuda").manual_seed(5)
    trgb = torch.rand(3 * P, device="cuda", generator=gen)
    tdep = torch.rand(P, device="cuda", generator=gen) * 4.0
    step = dict(target_rgb=trgb, target_depth=tdep)
    res = R.autotune(scenes, [vw], reps=1, step=step)
    # 16x16: 6 strip shapes, the other tilings one each, both binning modes
    assert res["timed"] == 2 * (6 + 3)
    assert res["tile"] in [(16, 16), (16, 8), (8, 8), (32, 8)] and res["binning"] in (0, 1)
    assert res["strip"][0] == res["strip"][1] and res["ms_fwd"] > 0 and res["ms_bwd"] == 0
    if res["tile"] != (16, 16):
        assert res["strip"] == (0, 0)
    assert (R.ctx.tile, R.ctx.strip, R.ctx.binning) == (res["tile"], res["strip"], res["binning"])
    # the same key again: from the cache; the pose-only step and the separate calls
    # are tuned under keys of their own
    assert R.autotune(scenes, [vw], reps=1, step=step)["timed"] == 0
    assert R.autotune(scenes, [vw], reps=1, step=dict(step, grads=False))["timed"] == 2 * (6 + 3)
    assert R.autotune(scenes, [vw], reps=1)["timed"] > 0
    R.autotune(scenes, [vw], reps=1, step=step)  # back to the parameter step's choice
    assert (R.ctx.tile, R.ctx.strip, R.ctx.binning) == (res["tile"], res["strip"], res["binning"])
    # the tuned fused step writes the untuned forward's images
    ws, mp = R.new_workspace(scenes, [vw])
    out = (torch.empty(3 * P, device="cuda"), torch.empty(P, device="cuda"), torch.empty(P, device="cuda"))
    loss = torch.zeros(1, device="cuda")
    grads = [{k: torch.zeros_like(getattr(scenes[0], k)) for k in G.PARAM_KEYS}]
    G.gs_render_step_l1(R.ctx, scenes, [vw], ws, mp, out, trgb, tdep, 1.0, 0.5, loss, grads, None, 0)
    st, _ = G.gs_workspace_status(R.ctx, ws)
    assert st == G.GS_OK
    got = split_views([vw], *out)[0]
    for x, y in zip(got, ref):
        assert np.array_equal(x, y)
    assert float(loss[0]) > 0
