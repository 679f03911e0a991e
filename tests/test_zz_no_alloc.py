"""The workspace-free forward (gs_render_forward_static) against the regular
forward (gs_render_forward).

gs_render_forward_static is for callers that cannot allocate device memory
when they render (a plug-in whose host application owns the GPU memory budget,
or a per-frame callback where cudaMalloc could block); it uses the library's
static 32 MiB device scratch instead of a caller workspace.  This file is named
to be collected last, so a run that stops at the first failure has run every
other test first.
"""
import numpy as np
import pytest
import torch

import synth
from gpu_util import COLOR_ABS, DEPTH_REL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_11700_gb300 import build
    build.build()
    import paper_2311_11700_gb300 as g
    return g


def _images(P):
    return (torch.full((3 * P,), -1.0, device="cuda"), torch.full((P,), -1.0, device="cuda"),
            torch.full((P,), -1.0, device="cuda"))


def _close(a, b):
    (ca, da, aa), (cb, db, ab) = a, b
    assert torch.isfinite(ca).all() and torch.isfinite(da).all() and torch.isfinite(aa).all()
    assert (ca - cb).abs().max().item() < COLOR_ABS
    rel = ((da - db).abs() / db.abs().clamp_min(1e-6)).max().item()
    assert rel < DEPTH_REL
    assert (aa - ab).abs().max().item() < COLOR_ABS


def test_static_scratch_forward_matches_workspace_forward_twice(G):
    ctx = G.Context(0)
    cases = []
    s0, v0 = synth.frustum_scene(1000, n=2000)                # the 160x120 frustum workload
    s1, v1 = synth.frustum_scene(77, n=5000, width=200, height=150, f=150.0, sh_degree=2)
    for s, v in ((s0, v0), (s1, v1)):
        sc = G.Scene.from_numpy(s)
        P = v["width"] * v["height"]
        mp = 16 * s["mean"].shape[1]
        ws = G.alloc_workspace(G.gs_workspace_query(ctx, [sc], [v], mp))
        ref = _images(P)
        G.gs_render_forward(ctx, [sc], [v], ws, mp, ref)
        st, _ = G.gs_workspace_status(ctx, ws)
        assert st == G.GS_OK
        cases.append((sc, v, mp, ref))
    # two calls in a row, different scenes and sizes: the shared scratch must not
    # carry anything over from the previous call
    for sc, v, mp, ref in cases:
        got = _images(v["width"] * v["height"])
        G.gs_render_forward_static(ctx, [sc], [v], mp, got)
        torch.cuda.synchronize()
        _close(got, ref)


def test_static_scratch_rejects_requests_above_its_size(G):
    ctx = G.Context(0)
    s, v = synth.frustum_scene(1000, n=2000)
    sc = G.Scene.from_numpy(s)
    P = v["width"] * v["height"]
    with pytest.raises(G.GsrError) as e:
        G.gs_render_forward_static(ctx, [sc], [v], 8_000_000, _images(P))  # 64 MB of pair lists
    assert e.value.status == G.GS_ERR_INVALID_ARG
    assert "static" in str(e.value)


def test_static_scratch_reports_device_side_capacity_overflow(G):
    """A pair capacity too small for the view: the static forward returns GS_OK (the
    overflow is only known on the device) and gs_render_forward_static_status then
    reports GS_ERR_CAPACITY with the pairs the call needed; a later call with room
    renders the same images as the workspace forward."""
    ctx = G.Context(0)
    s, v = synth.frustum_scene(1000, n=2000)
    sc = G.Scene.from_numpy(s)
    P = v["width"] * v["height"]
    small = 64
    G.gs_render_forward_static(ctx, [sc], [v], small, _images(P))
    st, needed = G.gs_render_forward_static_status(ctx)
    assert st == G.GS_ERR_CAPACITY and needed > small
    mp = 16 * s["mean"].shape[1]
    ws = G.alloc_workspace(G.gs_workspace_query(ctx, [sc], [v], mp))
    ref = _images(P)
    G.gs_render_forward(ctx, [sc], [v], ws, mp, ref)
    got = _images(P)
    G.gs_render_forward_static(ctx, [sc], [v], mp, got)
    st, needed2 = G.gs_render_forward_static_status(ctx)
    assert st == G.GS_OK and needed2 == needed
    _close(got, ref)
