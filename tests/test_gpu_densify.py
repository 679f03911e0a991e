"""Density control on the GPU against the FP64 oracle: the view-space gradient
statistics accumulated by the backward, and the clone / split of gs_densify."""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from oracle import slam_ops as S
from gpu_util import read_state, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_11700_gb300 import build
    build.build()
    import paper_2311_11700_gb300 as g
    return g


def _visible(sc, vw, widen=False):
    """Gaussians the oracle renders in a view: projected, opacity >= 1/255 and a
    footprint box that covers a pixel centre of the image.  widen: the box of the
    half-extents e 1.002 + 2e-3, the most the kernels widen them by (so that float32
    rounding never drops a pixel the definition blends)."""
    pr = O.project(O.to_params(sc), vw)
    idx = pr["index"].numpy()
    mu = pr["mu"].detach().numpy()
    ex, ey = O.footprint_extents(pr["cov2d"].detach().numpy(), pr["opacity"].detach().numpy())
    if widen:
        ex, ey = ex * 1.002 + 2e-3, ey * 1.002 + 2e-3
    tx0, tx1, ty0, ty1 = O.tile_rects(mu[:, 0].astype(np.float32), mu[:, 1].astype(np.float32),
                                      ex.astype(np.float32), ey.astype(np.float32), vw["width"], vw["height"], 16, 16)
    ok = (ex > 0) & (tx1 >= tx0) & (ty1 >= ty0)
    return idx[ok]


def test_view_space_gradient_statistics_match_oracle(G):
    sc = synth.room_scene(81, n=3000)
    views = synth.trajectory_views(82, 2, 96, 64)
    targets = [synth.random_targets(83 + i, 96, 64) for i in range(2)]
    R = G.Renderer(0)
    scene = G.Scene.from_numpy(sc)
    vws = [dict(v, scene=0) for v in views]
    color, depth, acc, ws, mp = R.forward([scene], vws)
    trgb = torch.as_tensor(np.concatenate([t[0].reshape(-1) for t in targets]), device="cuda")
    tdep = torch.as_tensor(np.concatenate([t[1].reshape(-1) for t in targets]), device="cuda")
    loss = torch.zeros(2, device="cuda")
    dC, dD = torch.empty_like(color), torch.empty_like(depth)
    G.gs_loss_l1(R.ctx, vws, (color, depth, acc), trgb, tdep, 1.0, 0.5, loss, (dC, dD, None))
    n = sc["mean"].shape[1]
    vs = torch.full((n,), 0.25, device="cuda")   # statistics accumulate onto what is there
    cnt = torch.full((n,), 1.0, device="cuda")
    G.gs_render_backward(R.ctx, [scene], vws, ws, mp, (dC, dD, None), [{"vs_grad_norm": vs, "vs_count": cnt}])
    torch.cuda.synchronize()
    ref = O.render_and_grad([sc], vws, targets, w_c=1.0, w_d=0.5, want_2d=True)
    want_g, want_c = np.full(n, 0.25), np.ones(n)
    for v, g2 in zip(vws, ref["grads_2d"]):
        pos = {int(i): k for k, i in enumerate(g2["index"])}
        for i in _visible(sc, v):
            want_g[i] += S.ndc_grad_norm(g2["mu"][pos[int(i)]], v["width"], v["height"])
            want_c[i] += 1
    got_c = cnt.cpu().numpy()
    # bit-exact: one count per view whose forward rendered the Gaussian (its tile
    # rectangle, decided in float32 from the kernel's own centre and extents, is not
    # empty), read from the forward's workspace
    st = read_state(G, R, [scene], vws, ws, mp)
    want32 = np.ones(n)
    for k in range(len(vws)):
        o = int(st["layout"].splat_off[k])
        want32 += st["ntiles"][o:o + n] > 0
    np.testing.assert_array_equal(got_c, want32)
    # against the oracle: between its count with the exact footprint boxes and its
    # count with the boxes widened as far as the kernels may widen them
    hi = np.ones(n)
    for v in vws:
        hi[_visible(sc, v, widen=True)] += 1
    assert (got_c >= want_c).all() and (got_c <= hi).all()
    assert (want_c > 1).sum() > 1000
    assert rel_l2(vs.cpu().numpy().astype(np.float64), want_g) < 1e-3


@pytest.mark.parametrize("deg", [0, 3])
def test_densify_matches_oracle(G, deg):
    rng = np.random.default_rng(84 + deg)
    n = 5000
    sc = synth.room_scene(85, n=n, sh_degree=deg)
    sc["log_scale"] = np.log(rng.uniform(0.005, 0.03, (3, n))).astype(np.float32)
    grad_sum = rng.uniform(0, 0.01, n).astype(np.float32)
    count = rng.integers(0, 4, n).astype(np.float32)
    noise = rng.standard_normal((6, n)).astype(np.float32)
    want, counts = S.densify(sc, grad_sum, count, noise)
    assert counts[1] > 100 and counts[2] > 100
    scene = G.Scene.from_numpy(sc)
    cap = counts[0] + counts[1] + 2 * counts[2] + 17
    K3 = 3 * (deg + 1) ** 2
    out = {"mean": torch.zeros(3, cap, device="cuda"), "log_scale": torch.zeros(3, cap, device="cuda"),
           "quat": torch.zeros(4, cap, device="cuda"), "opacity_logit": torch.zeros(cap, device="cuda"),
           "sh": torch.zeros(K3, cap, device="cuda")}
    cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
    d = lambda a: torch.as_tensor(a, device="cuda")  # noqa: E731
    G.gs_densify(G.Context(0), scene, d(grad_sum), d(count), d(noise), out, cap, cnt)
    torch.cuda.synchronize()
    c = cnt.cpu().numpy()
    m = counts[0] + counts[1] + 2 * counts[2]
    assert tuple(c[:3]) == counts and c[3] == m
    got = {k: v.cpu().numpy()[..., :m] for k, v in out.items()}
    np.testing.assert_allclose(got["mean"], want["mean"], rtol=2e-6, atol=2e-6)
    np.testing.assert_allclose(got["log_scale"], want["log_scale"], rtol=0, atol=2e-6)
    for k in ("quat", "opacity_logit", "sh"):
        np.testing.assert_array_equal(got[k], want[k])


def test_densify_capacity_is_reported(G):
    n = 1000
    rng = np.random.default_rng(86)
    sc = synth.room_scene(87, n=n, sh_degree=0)
    scene = G.Scene.from_numpy(sc)
    d = lambda a: torch.as_tensor(a, device="cuda")  # noqa: E731
    cap = 10
    out = {"mean": torch.zeros(3, cap, device="cuda"), "log_scale": torch.zeros(3, cap, device="cuda"),
           "quat": torch.zeros(4, cap, device="cuda"), "opacity_logit": torch.zeros(cap, device="cuda"),
           "sh": torch.zeros(3, cap, device="cuda")}
    cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
    G.gs_densify(G.Context(0), scene, d(np.full(n, 1.0, np.float32)), d(np.ones(n, np.float32)),
                 d(rng.standard_normal((6, n)).astype(np.float32)), out, cap, cnt)
    c = cnt.cpu().numpy()
    assert c[3] > cap and c[0] + c[1] + 2 * c[2] == c[3]
