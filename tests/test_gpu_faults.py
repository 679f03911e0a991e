"""Failure paths on the GPU, forced without a GPU fault.

* A bounded device-side wait that runs out: the context's look-back bound set to
  0 reads (gs_ctx_set_spin_limit) makes every decoupled look-back of binning mode 1
  and of the expansion give up at once.  The call must report GS_ERR_TIMEOUT, leave
  the images unwritten (the later kernels of the call do nothing), and leave the
  GPU healthy: the same context renders correctly once the bound is restored.
* Host-side injection through GSR_FAULT (read when a context is created):
  alloc fails the context's stream creation before anything is enqueued; capacity
  gives the kernels a pair capacity of 0; timeout gives every look-back a bound of 0.
"""
import os

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_11700_gb300 import build
    build.build()
    import paper_2311_11700_gb300 as g
    return g


def _case(n=20_000, W=160, H=120):
    # 20k Gaussians: 10 scan tiles of 2048 splats, so the look-backs have waiters
    return synth.frustum_scene(1000, n=n, width=W, height=H, f=120.0)


def _sentinel(P):
    return (torch.full((3 * P,), -7.0, device="cuda"), torch.full((P,), -7.0, device="cuda"),
            torch.full((P,), -7.0, device="cuda"))


def _render(G, ctx, sc, v, mp):
    P = v["width"] * v["height"]
    ws = G.alloc_workspace(G.gs_workspace_query(ctx, [sc], [v], mp))
    out = _sentinel(P)
    G.gs_render_forward(ctx, [sc], [v], ws, mp, out)
    st, needed = G.gs_workspace_status(ctx, ws)
    return st, needed, out


@pytest.fixture()
def fault_env():
    """Sets GSR_FAULT for the contexts created inside the test, then clears it."""
    old = os.environ.get("GSR_FAULT")

    def set_(v):
        os.environ["GSR_FAULT"] = v
    yield set_
    if old is None:
        os.environ.pop("GSR_FAULT", None)
    else:
        os.environ["GSR_FAULT"] = old


def test_lookback_bound_runs_out_reports_timeout_and_recovers(G):
    s, v = _case()
    sc = G.Scene.from_numpy(s)
    mp = 16 * s["mean"].shape[1]
    ref_ctx = G.Context(0)
    ref_ctx.set_binning(1)
    st, _, ref = _render(G, ref_ctx, sc, v, mp)
    assert st == G.GS_OK
    ctx = G.Context(0)
    ctx.set_binning(1)
    ctx.set_spin_limit(0)
    st, _, out = _render(G, ctx, sc, v, mp)
    assert st == G.GS_ERR_TIMEOUT
    assert "wait" in G.lib().gs_last_error(ctx.handle).decode()
    for t in out:  # the compositing kernel did nothing
        assert (t == -7.0).all()
    # the GPU and the context stay usable: the default bound renders the reference
    ctx.set_spin_limit(1 << 20)
    st, _, again = _render(G, ctx, sc, v, mp)
    assert st == G.GS_OK
    for a, b in zip(again, ref):
        assert torch.equal(a, b)


def test_expansion_lookback_bound_runs_out(G):
    s, v = synth.frustum_scene(1001, n=6000, width=128, height=96, f=96.0)
    ctx = G.Context(0)
    ctx.set_spin_limit(0)
    scene = G.Scene.from_numpy(s)
    P = v["width"] * v["height"]
    cap = scene.n + P
    K = (s["sh_degree"] + 1) ** 2
    out = {"mean": torch.zeros(3, cap, device="cuda"), "log_scale": torch.zeros(3, cap, device="cuda"),
           "quat": torch.zeros(4, cap, device="cuda"), "opacity_logit": torch.zeros(cap, device="cuda"),
           "sh": torch.zeros(3 * K, cap, device="cuda")}
    count = torch.zeros(4, dtype=torch.int64, device="cuda")
    ws = G.alloc_workspace(G.gs_expand_workspace_query(ctx, scene.n, v))
    acc = torch.zeros(P, device="cuda")          # every pixel unreliable: many appended Gaussians
    dep = torch.zeros(P, device="cuda")
    rgb = torch.full((3 * P,), 0.5, device="cuda")
    D = torch.full((P,), 2.0, device="cuda")
    G.gs_expand(ctx, scene, v, acc, dep, rgb, D, {}, out, cap, count, ws)
    torch.cuda.synchronize()
    assert int(ws[:4].view(torch.int32).item()) & 2  # GS_ERR_TIMEOUT bit of the expansion workspace
    assert (count.cpu().numpy()[:3] <= cap).all()


def test_fault_injection_alloc_enqueues_nothing(G, fault_env):
    s, v = _case(n=3000)
    sc = G.Scene.from_numpy(s)
    fault_env("alloc")
    ctx = G.Context(0)
    P = v["width"] * v["height"]
    mp = 16 * s["mean"].shape[1]
    ws = G.alloc_workspace(G.gs_workspace_query(ctx, [sc], [v], mp))
    ws.fill_(0xAB)
    out = _sentinel(P)
    with pytest.raises(G.GsrError) as e:
        G.gs_render_forward(ctx, [sc], [v], ws, mp, out)
    assert e.value.status == G.GS_ERR_CUDA and "injected" in str(e.value)
    torch.cuda.synchronize()
    assert (ws == 0xAB).all()
    for t in out:
        assert (t == -7.0).all()


@pytest.mark.parametrize("binning", [0, 1])
def test_fault_injection_capacity(G, fault_env, binning):
    s, v = _case(n=3000)
    sc = G.Scene.from_numpy(s)
    fault_env("capacity")
    ctx = G.Context(0)
    ctx.set_binning(binning)
    mp = 16 * s["mean"].shape[1]
    st, needed, out = _render(G, ctx, sc, v, mp)
    assert st == G.GS_ERR_CAPACITY and 0 < needed < mp
    for t in out:
        assert (t == -7.0).all()
    # the binding's capacity growth cannot fix it and says so
    R = G.Renderer(0)
    R.ctx = ctx
    with pytest.raises(G.GsrError) as e:
        R.forward([sc], [v])
    assert e.value.status == G.GS_ERR_CAPACITY


@pytest.mark.parametrize("binning,want", [(0, "GS_OK"), (1, "GS_ERR_TIMEOUT")])
def test_fault_injection_timeout(G, fault_env, binning, want):
    """Binning mode 0 has no cross-CTA wait, so only mode 1 reports the timeout."""
    s, v = _case()
    sc = G.Scene.from_numpy(s)
    fault_env("timeout")
    ctx = G.Context(0)
    ctx.set_binning(binning)
    st, _, _ = _render(G, ctx, sc, v, 16 * s["mean"].shape[1])
    assert st == getattr(G, want)
