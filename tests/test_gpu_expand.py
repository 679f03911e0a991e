"""GPU parity of the adaptive expansion (Eq. add_method, Eq. delete_method,
Eq. init-rep, opacity prune) against the FP64 oracle, including a capacity
overflow.  The rendered acc / depth inputs come from the oracle's render."""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from oracle import slam_ops as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_11700_gb300 import build
    build.build()
    import paper_2311_11700_gb300 as g
    return g


def _case(seed=41, n=5000, W=128, H=96):
    full = synth.room_scene(seed, n=n, sh_degree=2)
    vw = synth.room_view(W, H, f=0.5 * W)
    obs_rgb, obs_d = synth.zbuffer_targets(full, vw, seed + 1)
    # the current map: a hole (Gaussians removed) and some low-opacity ones
    rng = np.random.default_rng(seed + 2)
    keep = rng.uniform(0, 1, n) > 0.3
    cur = {k: (v[..., keep].copy() if isinstance(v, np.ndarray) else v) for k, v in full.items()}
    m = cur["opacity_logit"].shape[0]
    low = rng.uniform(0, 1, m) < 0.05
    cur["opacity_logit"][low] = rng.normal(-6.0, 1.0, int(low.sum())).astype(np.float32)
    # floaters in front of the surface
    fl = rng.uniform(0, 1, m) < 0.05
    T = np.asarray(vw["T_cw"], np.float64).reshape(3, 4)
    cam = -T[:, :3].T @ T[:, 3]
    cur["mean"][:, fl] = (cam[:, None] + 0.6 * (cur["mean"][:, fl] - cam[:, None])).astype(np.float32)
    r = O.render_view(cur, vw)
    return cur, vw, r["acc"].astype(np.float32), r["depth"].astype(np.float32), obs_rgb, obs_d


@pytest.mark.parametrize("flags,checker", [(7, False), (1, True), (2, False)])
def test_expand_matches_oracle(G, flags, checker):
    cur, vw, acc, dep, rgb, D = _case()
    params = dict(tau_T=0.5, tau_D=0.1, eta=0.01, gamma=0.1, init_opacity=0.1, density=0.5 if checker else 1.0,
                  prune_opacity=0.005, flags=flags | (8 if checker else 0))
    want, (nk, na) = S.expand(cur, vw, acc, dep, rgb, D, do_add=bool(flags & 1), do_delete=bool(flags & 2),
                              do_prune=bool(flags & 4), checkerboard=checker, density=params["density"])
    ctx = G.Context(0)
    scene = G.Scene.from_numpy(cur)
    cap = scene.n + vw["width"] * vw["height"]
    K = (cur["sh_degree"] + 1) ** 2
    out = {"mean": torch.zeros(3, cap, device="cuda"), "log_scale": torch.zeros(3, cap, device="cuda"),
           "quat": torch.zeros(4, cap, device="cuda"), "opacity_logit": torch.zeros(cap, device="cuda"),
           "sh": torch.zeros(3 * K, cap, device="cuda")}
    count = torch.zeros(4, dtype=torch.int64, device="cuda")
    ws = G.alloc_workspace(G.gs_expand_workspace_query(ctx, scene.n, vw))
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")  # noqa: E731
    G.gs_expand(ctx, scene, vw, t(acc), t(dep), t(rgb), t(D), params, out, cap, count, ws)
    torch.cuda.synchronize()
    c = count.cpu().numpy()
    assert (c[0], c[1]) == (nk, na) and c[2] == c[3] == nk + na
    if flags & 1:
        assert na > 50
    if flags == 2:  # delete only: every Gaussian kept, the floaters decayed
        assert nk == scene.n and (want["opacity_logit"] != cur["opacity_logit"]).sum() > 20
    tot = nk + na
    got = {k: v[..., :tot].cpu().numpy() for k, v in out.items()}
    np.testing.assert_array_equal(got["mean"][:, :nk], want["mean"][:, :nk])
    np.testing.assert_array_equal(got["log_scale"][:, :nk], want["log_scale"][:, :nk])
    np.testing.assert_array_equal(got["quat"], want["quat"])
    np.testing.assert_array_equal(got["sh"][:, :nk], want["sh"][:, :nk])
    np.testing.assert_allclose(got["opacity_logit"], want["opacity_logit"], atol=2e-5)
    np.testing.assert_allclose(got["mean"][:, nk:], want["mean"][:, nk:], rtol=2e-6, atol=2e-6)
    np.testing.assert_allclose(got["log_scale"][:, nk:], want["log_scale"][:, nk:], atol=2e-6)
    np.testing.assert_allclose(got["sh"][:, nk:], want["sh"][:, nk:], atol=2e-5)


def test_expand_capacity_overflow_is_reported(G):
    cur, vw, acc, dep, rgb, D = _case(51)
    ctx = G.Context(0)
    scene = G.Scene.from_numpy(cur)
    _, (nk, na) = S.expand(cur, vw, acc, dep, rgb, D)
    cap = nk + na // 2
    K = (cur["sh_degree"] + 1) ** 2
    out = {"mean": torch.zeros(3, cap, device="cuda"), "log_scale": torch.zeros(3, cap, device="cuda"),
           "quat": torch.zeros(4, cap, device="cuda"), "opacity_logit": torch.zeros(cap, device="cuda"),
           "sh": torch.zeros(3 * K, cap, device="cuda")}
    count = torch.zeros(4, dtype=torch.int64, device="cuda")
    ws = G.alloc_workspace(G.gs_expand_workspace_query(ctx, scene.n, vw))
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")  # noqa: E731
    G.gs_expand(ctx, scene, vw, t(acc), t(dep), t(rgb), t(D), {}, out, cap, count, ws)
    torch.cuda.synchronize()
    c = count.cpu().numpy()
    assert c[2] == cap and c[3] == nk + na
    assert int(ws[:4].view(torch.int32).item()) & 1  # GS_ERR_CAPACITY bit in the expansion workspace
