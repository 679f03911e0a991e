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
