"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle:
projection, bit-exact per-tile lists, forward images, loss, gradients (exact and
paper pose modes), batched = per-view, tile-size invariance, edge cases."""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from gpu_util import (GRAD_MARGINS, GRAD_REL_L2, gpu_loss_and_grads, image_parity,
                      read_state, rel_l2, resolvable, run_forward, split_views)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_11700_gb300 import build
    build.build()
    import paper_2311_11700_gb300 as g
    return g


@pytest.fixture(scope="module")
def R(G):
    return G.Renderer(0)


@pytest.fixture(scope="module")
def plain2k():
    return synth.workload_plain_2k()


@pytest.fixture(scope="module")
def plain2k_ref(plain2k):
    return O.render_view(plain2k["scenes"][0], plain2k["views"][0])


def _sh3_small(seed=21, n=1500, W=120, H=88):
    """A small SH-degree-3 scene seen from a general pose (view-dependent colour)."""
    sc = synth.room_scene(seed, n=n)
    vw = synth.room_view(W, H, f=0.5 * W)
    return sc, vw


def test_forward_matches_oracle_plain_2k(G, R, plain2k, plain2k_ref):
    sc, vw = plain2k["scenes"], plain2k["views"]
    _, color, depth, acc, ws, mp = run_forward(G, R, sc, vw)
    c, d, a = split_views(vw, color, depth, acc)[0]
    ref = plain2k_ref
    # every pixel: 4 of the 19,200 lie within float32 reach of a threshold and are
    # checked against the outcomes the oracle allows there
    n, near, unresolved = image_parity(vw[0], c, d, a, ref, np.ones(c.shape[1:], bool))
    assert n == 19200 and near <= 4 and unresolved == 0


def test_projection_matches_oracle(G, R):
    sc, vw = _sh3_small()
    scenes, *_, ws, mp = run_forward(G, R, [sc], [vw])
    st = read_state(G, R, scenes, [vw], ws, mp)
    pr = O.project(O.to_params(sc), vw)
    idx = pr["index"].numpy()
    vis = np.nonzero(st["ntiles"][:sc["mean"].shape[1]])[0]
    assert len(vis) > 100 and np.isin(vis, idx).all()
    pos = np.searchsorted(idx, vis)
    rec = st["rec"][vis].astype(np.float64)
    mu = np.stack([rec[:, 0] + rec[:, 7], rec[:, 1] + rec[:, 11]], 1)
    np.testing.assert_allclose(mu, pr["mu"].detach().numpy()[pos], rtol=0, atol=1e-5)
    cond = pr["cond"].numpy()[pos]
    con = pr["conic"].detach().numpy()[pos]
    scale = np.abs(con).max(1, keepdims=True)
    assert (np.abs(rec[:, [2, 3, 4]] - con) / scale / (1 + cond[:, None])).max() < 1e-5
    # the depth key is the correctly rounded float32 camera depth
    assert (st["dkey"][vis] == pr["depth32"][pos].view(np.uint32)).mean() > 0.9999
    np.testing.assert_allclose(rec[:, 5], pr["opacity"].detach().numpy()[pos], rtol=2e-6)
    np.testing.assert_allclose(rec[:, [8, 9, 10]], pr["rgb"].detach().numpy()[pos], atol=2e-5)


@pytest.fixture(scope="module")
def R_radix(G):
    r = G.Renderer(0)
    r.ctx.set_binning(1)
    return r


@pytest.fixture(params=[0, 1], ids=["counting", "radix"])
def RB(request, R, R_radix):
    """The renderer with each binning mode (per-tile counting sort, global radix sort)."""
    return R if request.param == 0 else R_radix


def test_tile_lists_bit_exact_given_the_kernels_keys(G, RB):
    R = RB
    sc, vw = _sh3_small(22, n=3000, W=133, H=71)  # ragged: 9 x 5 tiles with partial edges
    scenes, *_, ws, mp = run_forward(G, R, [sc], [vw])
    st = read_state(G, R, scenes, [vw], ws, mp)
    n = sc["mean"].shape[1]
    rec, rect = st["rec"][:n], st["rect"][:n]
    ex, ey = rect[:, 2].view(np.float32), rect[:, 3].view(np.float32)
    valid = st["ntiles"][:n] > 0
    # the kernel's footprint extents against the definition (q <= min(9, 2 ln(255 o)))
    pr = O.project(O.to_params(sc), vw)
    idx = pr["index"].numpy()
    v = np.nonzero(valid)[0]
    pos = np.searchsorted(idx, v)
    oex, oey = O.footprint_extents(pr["cov2d"].detach().numpy()[pos], pr["opacity"].detach().numpy()[pos])
    cond = pr["cond"].numpy()[pos]
    assert (ex[v] >= oex * (1 + 5e-4 / (1 + 1e-3 * cond))).all() and (ex[v] <= oex * 1.002 + 2e-3).all()
    assert (ey[v] >= oey * (1 + 5e-4 / (1 + 1e-3 * cond))).all() and (ey[v] <= oey * 1.002 + 2e-3).all()
    # the rectangle rule, decided in float32 from the kernel's own centre and extents
    tx0, tx1, ty0, ty1 = O.tile_rects(rec[:, 0], rec[:, 1], ex, ey, vw["width"], vw["height"], 16, 16)
    np.testing.assert_array_equal(rect[v, 0] & 0xffff, tx0[v])
    np.testing.assert_array_equal(rect[v, 0] >> 16, tx1[v])
    np.testing.assert_array_equal(rect[v, 1] & 0xffff, ty0[v])
    np.testing.assert_array_equal(rect[v, 1] >> 16, ty1[v])
    lists = O.tile_lists(rec[:, 0], rec[:, 1], ex, ey, st["dkey"][:n], valid, vw["width"], vw["height"], 16, 16)
    assert int(st["hdr"][2]) == sum(len(l) for l in lists)
    for t, want in enumerate(lists):
        s, e = st["ranges"][t]
        got = st["pairs"][s:e].tolist() if e > s else []
        assert got == want, f"tile {t}"


def _crowd(n, seed):
    """n Gaussians crowded on a 40x36 identity-pose view: 90 % wide ones around the
    centre (each covering most of the 3 x 3 tiles), 10 % small ones scattered; a
    third of the wide ones share one of five camera depths exactly (tie-breaking)."""
    rng = np.random.default_rng(seed)
    W, H, f = 40, 36, 30.0
    vw = synth.make_view(W, H, f, f, W / 2, H / 2, np.concatenate([np.eye(3), np.zeros((3, 1))], 1))
    z = rng.uniform(2.0, 6.0, n)
    tie = rng.random(n) < 0.3
    z[tie] = rng.choice([2.5, 3.0, 3.25, 4.0, 5.5], tie.sum())
    wide = rng.random(n) < 0.9
    px = np.where(wide, rng.normal(W / 2, 2.0, n), rng.uniform(0, W, n))
    py = np.where(wide, rng.normal(H / 2, 2.0, n), rng.uniform(0, H, n))
    mean = np.stack([(px - W / 2) * z / f, (py - H / 2) * z / f, z])
    rad_px = np.where(wide, rng.uniform(5.0, 9.0, n), rng.uniform(0.5, 2.0, n))
    sc = dict(mean=mean.astype(np.float32),
              log_scale=np.tile(np.log(rad_px * z / f / 3.0), (3, 1)).astype(np.float32),
              quat=rng.normal(0, 1, (4, n)).astype(np.float32),
              opacity_logit=rng.normal(0, 1, n).astype(np.float32),
              sh=rng.normal(0, 1, (3, n)).astype(np.float32), sh_degree=0)
    return sc, vw


@pytest.mark.parametrize("binning", [0, 1])
def test_pair_count_and_ranges_consistent_many_tiles(G, binning):
    """4800 tiles (8x8 at 640x480: 19 chunks of the tile scan): the non-empty
    ranges tile the pair list without gaps, the pair count is the sum of the
    Gaussians' tile counts, every list holds only Gaussians whose rectangle covers
    it, and the launch order is a permutation by non-increasing length bucket (8 per
    octave)."""
    R8 = G.Renderer(0, tile=(8, 8))
    R8.ctx.set_binning(binning)
    sc = synth.room_scene(31, n=20_000)
    vw = synth.room_view(640, 480, f=320.0)
    scenes, *_, ws, mp = run_forward(G, R8, [sc], [vw])
    st = read_state(G, R8, scenes, [vw], ws, mp)
    n = sc["mean"].shape[1]
    rg = st["ranges"]
    assert len(rg) == 80 * 60
    npairs = int(st["hdr"][2])
    assert npairs == int(st["ntiles"][:n].sum(dtype=np.int64)) == int(st["hdr"][3])
    ne = rg[rg[:, 1] > rg[:, 0]]  # non-empty tiles, in tile order (empty ones may hold (0, 0))
    assert ne[0, 0] == 0 and ne[-1, 1] == npairs and (ne[1:, 0] == ne[:-1, 1]).all()
    assert (rg[:, 1] >= rg[:, 0]).all()
    # the compositing launch order: every tile once, list-length buckets non-increasing
    order = st["order"].astype(np.int64)
    assert np.array_equal(np.sort(order), np.arange(80 * 60))
    lens = (rg[:, 1] - rg[:, 0]).astype(np.int64)[order]
    m = lens + 1
    k = np.floor(np.log2(m)).astype(np.int64)  # exact for these small integers
    sub = np.where(k >= 3, (m >> np.maximum(k - 3, 0)) & 7, (m << np.maximum(3 - k, 0)) & 7)
    bucket = 8 * k + sub
    assert (np.diff(bucket) <= 0).all()
    # the buckets refine the octaves: list lengths fall within 1/8 of an octave
    assert (np.diff(k) <= 0).all()
    rect = st["rect"][:n]
    for t in range(0, 80 * 60, 97):
        tx, ty = t % 80, t // 80
        ids = st["pairs"][rg[t, 0]:rg[t, 1]]
        r = rect[ids]
        assert ((r[:, 0] & 0xffff) <= tx).all() and ((r[:, 0] >> 16) >= tx).all()
        assert ((r[:, 1] & 0xffff) <= ty).all() and ((r[:, 1] >> 16) >= ty).all()


@pytest.mark.parametrize("n", [3000, 20000])
def test_long_tile_segments_sorted_bit_exact(G, RB, n):
    """With the per-tile counting sort, segments beyond 2048 entries take the large
    segment sort (register chunks, bitonic merges in shared memory) and beyond 8192
    its LSD radix path through global memory; the global radix binning sorts them
    like any other.  All must give the (depth bits, index) order, equal depths to
    the lower index."""
    R = RB
    sc, vw = _crowd(n, 40 + n)
    scenes, *_, ws, mp = run_forward(G, R, [sc], [vw])
    st = read_state(G, R, scenes, [vw], ws, mp)
    rec, rect = st["rec"][:n], st["rect"][:n]
    ex, ey = rect[:, 2].view(np.float32), rect[:, 3].view(np.float32)
    valid = st["ntiles"][:n] > 0
    lists = O.tile_lists(rec[:, 0], rec[:, 1], ex, ey, st["dkey"][:n], valid, vw["width"], vw["height"], 16, 16)
    sizes = [len(l) for l in lists]
    assert max(sizes) > (8192 if n > 16384 else 2048) and min(sizes) < max(sizes)
    dk = st["dkey"][:n]
    assert len(np.unique(dk[valid])) < valid.sum()  # ties present
    assert int(st["hdr"][2]) == sum(sizes)
    for t, want in enumerate(lists):
        s, e = st["ranges"][t]
        got = st["pairs"][s:e].tolist() if e > s else []
        assert got == want, f"tile {t}"
    # the workspace counts the segments the medium and large sorts took (mode 0 only)
    long_segments = G.gs_workspace_counters(R.ctx, ws)[7]
    assert long_segments == (sum(k > 512 for k in sizes) if R.ctx.binning == 0 else 0)


def test_binning_modes_give_identical_renders_and_gradients(G, R, R_radix):
    """The two binning modes build the same lists, so the images are bitwise equal
    and the loss and gradients equal up to the order of float atomics."""
    sc = synth.room_scene(33, n=40_000)
    vw = synth.room_view(320, 184, f=160.0)
    rgb, dep = synth.zbuffer_targets(sc, vw, 34)
    outs = []
    for r in (R, R_radix):
        scenes = [G.Scene.from_numpy(sc)]
        outs.append(gpu_loss_and_grads(G, r, scenes, [vw], [(rgb, dep)], 1.0, 0.5))
    (c0, d0, a0), (c1, d1, a1) = outs[0]["images"][0], outs[1]["images"][0]
    assert np.array_equal(c0, c1) and np.array_equal(d0, d1) and np.array_equal(a0, a1)
    assert abs(outs[0]["loss"][0] - outs[1]["loss"][0]) <= 1e-5 * abs(outs[0]["loss"][0])  # float atomics
    for k in O.PARAM_KEYS:
        assert rel_l2(outs[1]["grads"][0][k], outs[0]["grads"][0][k]) < 1e-5, k
    assert rel_l2(outs[1]["twist"], outs[0]["twist"]) < 1e-5


@pytest.mark.parametrize("pose_mode", [0, 1])
def test_gradients_match_oracle_plain_2k(G, R, plain2k, plain2k_ref, pose_mode):
    w = plain2k
    ok = resolvable(plain2k_ref, GRAD_MARGINS)
    assert (~ok).sum() <= 4  # the loss covers the other 19,196 pixels on both sides
    vw = dict(w["views"][0])
    vw["pixel_mask"] = torch.as_tensor(ok.astype(np.uint8), device="cuda")
    scenes = [G.Scene.from_numpy(w["scenes"][0])]
    out = gpu_loss_and_grads(G, R, scenes, [vw], w["targets"], w["w_c"], w["w_d"], pose_mode)
    ref = O.render_and_grad(w["scenes"], w["views"], w["targets"], w["w_c"], w["w_d"],
                            pixel_masks=[ok.astype(np.uint8)], pose_mode="paper" if pose_mode else "exact")
    assert abs(out["loss"][0] - ref["loss"]) / ref["loss"] < 1e-5
    for k in O.PARAM_KEYS:
        e = rel_l2(out["grads"][0][k], ref["grads"][0][k])
        assert e < GRAD_REL_L2, (k, e)
    assert rel_l2(out["twist"], ref["twist"]) < GRAD_REL_L2


def test_gradients_match_oracle_sh3_general_pose(G, R):
    sc, vw = _sh3_small(23, n=1200, W=96, H=72)
    rgb, dep = synth.zbuffer_targets(sc, vw, 24)
    ref_f = O.render_view(sc, vw)
    ok = resolvable(ref_f, GRAD_MARGINS)
    assert ok.all()  # no pixel of this view lies within float32 reach of a threshold
    v2 = dict(vw)
    v2["pixel_mask"] = torch.as_tensor(ok.astype(np.uint8), device="cuda")
    out = gpu_loss_and_grads(G, R, [G.Scene.from_numpy(sc)], [v2], [(rgb, dep)], 1.0, 0.5)
    ref = O.render_and_grad([sc], [vw], [(rgb, dep)], 1.0, 0.5, pixel_masks=[ok.astype(np.uint8)])
    for k in O.PARAM_KEYS:
        e = rel_l2(out["grads"][0][k], ref["grads"][0][k])
        assert e < GRAD_REL_L2, (k, e)
    assert rel_l2(out["twist"], ref["twist"]) < GRAD_REL_L2


def test_pose_grad_entry_equals_backward_twist(G, R, plain2k):
    w = plain2k
    scenes = [G.Scene.from_numpy(w["scenes"][0])]
    a = gpu_loss_and_grads(G, R, scenes, w["views"], w["targets"], 1.0, 0.5, 0, want_params=True)
    b = gpu_loss_and_grads(G, R, scenes, w["views"], w["targets"], 1.0, 0.5, 0, want_params=False)
    np.testing.assert_allclose(b["twist"], a["twist"], rtol=1e-4, atol=1e-3)


def test_batched_views_equal_one_view_per_call(G, R):
    s1, v1 = _sh3_small(31, n=2000, W=96, H=64)
    s2, _ = _sh3_small(32, n=900)
    v2 = synth.room_view(70, 50, f=40.0)
    v2["scene"] = 1
    v3 = synth.perturb_view(v1, [0.05, 0.0, -0.03, 0.0, 0.02, 0.0])
    v3["scene"] = 0
    scenes = [G.Scene.from_numpy(s1), G.Scene.from_numpy(s2)]
    views = [dict(v1, scene=0), v2, v3]
    color, depth, acc, *_ = R.forward(scenes, views)
    batched = split_views(views, color, depth, acc)
    for i, v in enumerate(views):
        vv = dict(v, scene=0)
        c, d, a, *_ = R.forward([scenes[v["scene"]]], [vv])
        one = split_views([vv], c, d, a)[0]
        for x, y in zip(batched[i], one):
            np.testing.assert_array_equal(x, y)


def test_results_do_not_depend_on_tile_size_or_strip(G):
    sc, vw = _sh3_small(41, n=2500, W=101, H=67)
    outs = []
    for tile, strip in (((16, 16), 0), ((8, 8), 0), ((16, 8), 0), ((32, 8), 0), ((16, 16), 1), ((16, 16), 2),
                        ((16, 16), 3), ((16, 16), 4), ((16, 16), 5)):
        R = G.Renderer(0, tile)
        R.ctx.set_strip(strip, strip)
        c, d, a, *_ = R.forward([G.Scene.from_numpy(sc)], [vw])
        outs.append(split_views([vw], c, d, a)[0])
    ref = O.render_view(sc, vw)
    ok = resolvable(ref)
    for o in outs[1:]:
        assert np.abs(o[0] - outs[0][0])[:, ok].max() < 1e-5
        assert np.abs(o[1] - outs[0][1])[ok].max() < 1e-5 * max(1.0, np.abs(outs[0][1]).max())


def test_capacity_overflow_is_reported_then_recovered(G):
    sc, vw = _sh3_small(51, n=2000, W=96, H=64)
    R = G.Renderer(0)
    R.max_pairs = 64
    scenes = [G.Scene.from_numpy(sc)]
    mp = R.max_pairs
    ws = G.alloc_workspace(G.gs_workspace_query(R.ctx, scenes, [vw], mp))
    color = torch.zeros(3 * 96 * 64, device="cuda")
    G.gs_render_forward(R.ctx, scenes, [vw], ws, mp, (color, None, None))
    st, needed = G.gs_workspace_status(R.ctx, ws)
    assert st == G.GS_ERR_CAPACITY and needed > 64
    c, d, a, ws2, mp2 = R.forward(scenes, [vw])  # grows and re-renders
    assert mp2 >= needed
    ref = O.render_view(sc, vw)
    c, d, a = split_views([vw], c, d, a)[0]
    n, near, unresolved = image_parity(vw, c, d, a, ref, np.ones(d.shape, bool))
    assert unresolved == 0


def test_pixel_mask_and_empty_scene(G, R):
    sc, vw = _sh3_small(61, n=800, W=64, H=48)
    m = np.zeros((48, 64), np.uint8)
    m[5:30, 10:50] = 1
    v = dict(vw, pixel_mask=torch.as_tensor(m, device="cuda"))
    c, d, a, *_ = R.forward([G.Scene.from_numpy(sc)], [v])
    c, d, a = split_views([v], c, d, a)[0]
    assert (c[:, m == 0] == 0).all() and (d[m == 0] == 0).all() and (a[m == 0] == 0).all()
    # every Gaussian behind the camera: background everywhere, nothing accumulated
    behind = dict(sc)
    T = np.asarray(vw["T_cw"], np.float64).reshape(3, 4)
    cam = -T[:, :3].T @ T[:, 3]
    fwd = T[2, :3]
    behind["mean"] = (cam[:, None] - 2.0 * fwd[:, None] + 0 * sc["mean"]).astype(np.float32)
    vb = dict(vw, bg=np.array([0.1, 0.2, 0.3], np.float32))
    c, d, a, *_ = R.forward([G.Scene.from_numpy(behind)], [vb])
    c, d, a = split_views([vb], c, d, a)[0]
    np.testing.assert_allclose(c, np.broadcast_to(np.array([0.1, 0.2, 0.3], np.float32)[:, None, None], c.shape))
    assert (a == 0).all() and (d == 0).all()


def test_loss_value_and_adjoint_match_oracle(G, R, plain2k, plain2k_ref):
    w = plain2k
    scenes = [G.Scene.from_numpy(w["scenes"][0])]
    out = gpu_loss_and_grads(G, R, scenes, w["views"], w["targets"], 1.0, 0.5)
    ref = O.render_and_grad(w["scenes"], w["views"], w["targets"], 1.0, 0.5)
    assert abs(out["loss"][0] - ref["loss"]) / ref["loss"] < 1e-4


def test_autograd_function_matches_abi(G, R, plain2k):
    w = plain2k
    sc = G.Scene.from_numpy(w["scenes"][0])
    params = [p.clone().requires_grad_(True) for p in sc.params()]
    sc2 = sc.with_params(params)
    twist = torch.zeros(1, 6, device="cuda", requires_grad=True)
    color, depth, acc = G.RenderRGBD.apply(R, [sc2], w["views"], twist, 0, *params)
    trgb = torch.as_tensor(w["targets"][0][0].reshape(-1), device="cuda")
    tdep = torch.as_tensor(w["targets"][0][1].reshape(-1), device="cuda")
    loss = (color - trgb).abs().sum() + 0.5 * ((depth - tdep).abs() * (tdep > 0)).sum()
    loss.backward()
    direct = gpu_loss_and_grads(G, R, [sc], w["views"], w["targets"], 1.0, 0.5)
    for p, k in zip(params, G.PARAM_KEYS):
        np.testing.assert_allclose(p.grad.cpu().numpy(), direct["grads"][0][k], rtol=1e-4,
                                   atol=1e-4 * np.abs(direct["grads"][0][k]).max())
    np.testing.assert_allclose(twist.grad.cpu().numpy(), direct["twist"], rtol=1e-4, atol=1e-2)


def _left_jacobian_fd(xi, h=1e-6):
    """The SE(3) left Jacobian at xi by central differences of
    vee(log(exp((xi + d)^) exp(-xi^))) (scipy's matrix exponential and logarithm)."""
    from scipy.linalg import expm, logm

    def hat(x):
        M = np.zeros((4, 4))
        M[:3, :3] = [[0, -x[5], x[4]], [x[5], 0, -x[3]], [-x[4], x[3], 0]]
        M[:3, 3] = x[:3]
        return M

    def vee(M):
        return np.array([M[0, 3], M[1, 3], M[2, 3], M[2, 1], M[0, 2], M[1, 0]])

    E_inv = expm(-hat(xi))
    J = np.zeros((6, 6))
    for k in range(6):
        d = np.zeros(6)
        d[k] = h
        J[:, k] = (vee(np.real(logm(expm(hat(xi + d)) @ E_inv))) -
                   vee(np.real(logm(expm(hat(xi - d)) @ E_inv)))) / (2 * h)
    return J


def test_autograd_function_renders_at_a_nonzero_twist(G, R):
    """RenderRGBD with twist xi != 0 renders at exp(xi^) T (against the oracle's render
    at that pose, near-threshold pixels against its alternatives), and its twist
    gradient is the chain of the left-perturbation gradient at that pose through the
    exponential: J(xi)^T g, with g the oracle's pose gradient at exp(xi^) T and J the
    SE(3) left Jacobian taken by finite differences of scipy's expm / logm."""
    sc, vw = _sh3_small(25, n=1200, W=96, H=72)
    rgb, dep = synth.zbuffer_targets(sc, vw, 26)
    xi = np.array([0.02, -0.015, 0.01, 0.03, -0.02, 0.025])
    T1 = O.se3_exp(torch.as_tensor(xi)).numpy() @ np.vstack([np.asarray(vw["T_cw"], np.float64).reshape(3, 4),
                                                               [0, 0, 0, 1]])
    v1 = dict(vw, T_cw=T1[:3].astype(np.float32).reshape(12))
    ref_f = O.render_view(sc, v1)
    ok = resolvable(ref_f, GRAD_MARGINS)
    assert ok.sum() >= ok.size - 2
    m = torch.as_tensor(ok.astype(np.uint8), device="cuda")
    scene = G.Scene.from_numpy(sc)
    params = [p.clone().requires_grad_(True) for p in scene.params()]
    twist = torch.as_tensor(xi[None].astype(np.float32), device="cuda").requires_grad_(True)
    color, depth, acc = G.RenderRGBD.apply(R, [scene.with_params(params)], [dict(vw, pixel_mask=m)], twist, 0, *params)
    c, d, a = split_views([vw], color.detach(), depth.detach(), acc.detach())[0]
    n, near, unresolved = image_parity(v1, c, d, a, ref_f, ok)
    assert unresolved == 0
    trgb = torch.as_tensor(rgb.reshape(-1), device="cuda")
    tdep = torch.as_tensor(dep.reshape(-1), device="cuda")
    mk = m.reshape(-1).bool()
    loss = ((color.view(3, -1) - trgb.view(3, -1)).abs() * mk).sum() + \
        0.5 * ((depth - tdep).abs() * (tdep > 0) * mk).sum()
    loss.backward()
    ref = O.render_and_grad([sc], [v1], [(rgb, dep)], 1.0, 0.5, pixel_masks=[ok.astype(np.uint8)])
    want = _left_jacobian_fd(xi).T @ ref["twist"][0]
    assert rel_l2(twist.grad.cpu().numpy()[0], want) < GRAD_REL_L2
    # the parameter gradients are those of the render at exp(xi^) T
    for p, k in zip(params, G.PARAM_KEYS):
        assert rel_l2(p.grad.cpu().numpy(), ref["grads"][0][k]) < GRAD_REL_L2, k


def test_fused_forward_loss_equals_separate_loss(G, R, plain2k):
    w = plain2k
    sc = G.Scene.from_numpy(w["scenes"][0])
    views = w["views"]
    P = views[0]["width"] * views[0]["height"]
    trgb = torch.as_tensor(w["targets"][0][0].reshape(-1), device="cuda")
    tdep = torch.as_tensor(w["targets"][0][1].reshape(-1), device="cuda")
    color, depth, acc, ws, mp = R.forward([sc], views)
    loss_a = torch.zeros(1, device="cuda")
    dCa, dDa = torch.empty(3 * P, device="cuda"), torch.empty(P, device="cuda")
    G.gs_loss_l1(R.ctx, views, (color, depth, acc), trgb, tdep, 1.0, 0.5, loss_a, (dCa, dDa, None))
    color2, depth2 = torch.empty_like(color), torch.empty_like(depth)
    loss_b = torch.full((1,), 123.0, device="cuda")
    dCb, dDb = torch.empty_like(dCa), torch.empty_like(dDa)
    G.gs_render_forward_l1(R.ctx, [sc], views, ws, mp, (color2, depth2, None), trgb, tdep, 1.0, 0.5, loss_b,
                           (dCb, dDb, None))
    torch.cuda.synchronize()
    assert torch.equal(color, color2) and torch.equal(depth, depth2)
    assert torch.equal(dCa, dCb) and torch.equal(dDa, dDb)
    assert abs(loss_a.item() - loss_b.item()) <= 1e-5 * loss_a.item()


def test_backward_blends_exactly_the_forward_pairs(G, R):
    """With timing on, the kernels count blended (pixel, Gaussian) pairs: the backward
    must revisit exactly the pairs the forward blended."""
    sc, vw = _sh3_small(71, n=4000, W=160, H=96)
    rgb, dep = synth.zbuffer_targets(sc, vw, 72)
    G.gs_ctx_set_timing(R.ctx, True)
    try:
        out = gpu_loss_and_grads(G, R, [G.Scene.from_numpy(sc)], [vw], [(rgb, dep)], 1.0, 0.5)
        ws_counts = None
    finally:
        G.gs_ctx_set_timing(R.ctx, False)
    stages = G.gs_ctx_read_timing(R.ctx, reset=True)
    assert stages["calls"] >= 1 and stages["composite_fwd"][1] >= 1
    # a fresh forward/backward on a known workspace to read the counters
    G.gs_ctx_set_timing(R.ctx, True)
    try:
        scenes = [G.Scene.from_numpy(sc)]
        color, depth, acc, ws, mp = R.forward(scenes, [vw])
        dC, dD = torch.ones_like(color), torch.ones_like(depth)
        dtw = torch.zeros(1, 6, device="cuda")
        G.gs_pose_grad(R.ctx, scenes, [vw], ws, mp, (dC, dD, None), dtw, 0)
        vis, pairs, nf, nb, *_ = G.gs_workspace_counters(R.ctx, ws)
    finally:
        G.gs_ctx_set_timing(R.ctx, False)
        G.gs_ctx_read_timing(R.ctx, reset=True)
    ref = O.render_view(sc, vw)
    assert nf == nb > 0
    # and the forward blends what the oracle blends (up to pixels at a threshold)
    ok = resolvable(ref)
    assert abs(nf - int(ref["n_contrib"].sum())) <= int(ref["n_contrib"][~ok].sum()) + 0.001 * nf


def test_timing_modes_give_the_same_results(G, R):
    """The counting kernels (timing mode 1) and the plain ones (modes 0 and 2) give
    bit-identical images, the same gradients up to atomic order, and only mode 1
    counts the blended pairs."""
    sc, vw = _sh3_small(73, n=4000, W=160, H=96)
    rgb, dep = synth.zbuffer_targets(sc, vw, 74)
    res = {}
    for mode in (0, 1, 2):
        G.gs_ctx_set_timing(R.ctx, mode)
        try:
            scenes = [G.Scene.from_numpy(sc)]
            out = gpu_loss_and_grads(G, R, scenes, [vw], [(rgb, dep)], 1.0, 0.5)
            _, _, _, ws, _ = R.forward(scenes, [vw])
            res[mode] = (out, G.gs_workspace_counters(R.ctx, ws))
        finally:
            G.gs_ctx_set_timing(R.ctx, 0)
            G.gs_ctx_read_timing(R.ctx, reset=True)
    for mode in (1, 2):
        a, b = res[0][0], res[mode][0]
        for k in range(3):
            assert np.array_equal(a["images"][0][k], b["images"][0][k])
        for k in G.PARAM_KEYS:
            assert rel_l2(b["grads"][0][k], a["grads"][0][k]) < 1e-5
        assert rel_l2(b["twist"], a["twist"]) < 1e-5
    assert res[1][1][2] > 0 and res[2][1][2] == 0 and res[0][1][2] == 0


@pytest.mark.parametrize("strips", [(0, 0), (1, 1), (2, 2), (3, 3), (3, 1), (1, 4), (5, 5)])
def test_gradients_match_oracle_with_other_strips(G, plain2k, plain2k_ref, strips):
    w = plain2k
    R = G.Renderer(0)
    R.ctx.set_strip(*strips)
    R.ctx.set_compact(0)  # the strip kernels, although the view has a pixel mask
    ok = resolvable(plain2k_ref, GRAD_MARGINS)
    vw = dict(w["views"][0])
    vw["pixel_mask"] = torch.as_tensor(ok.astype(np.uint8), device="cuda")
    out = gpu_loss_and_grads(G, R, [G.Scene.from_numpy(w["scenes"][0])], [vw], w["targets"], w["w_c"], w["w_d"])
    ref = O.render_and_grad(w["scenes"], w["views"], w["targets"], w["w_c"], w["w_d"],
                            pixel_masks=[ok.astype(np.uint8)])
    for k in O.PARAM_KEYS:
        assert rel_l2(out["grads"][0][k], ref["grads"][0][k]) < GRAD_REL_L2, k
    assert rel_l2(out["twist"], ref["twist"]) < GRAD_REL_L2


def test_grad_write_mode_overwrites_and_matches_add_mode(G):
    """gs_ctx_set_grad_mode(1): buffers prefilled with garbage receive the gradients
    that add mode accumulates into zeroed buffers (stored directly for a scene
    rendered by one view, zeroed and accumulated for a scene shared by two views);
    a scene no view renders gets zeros."""
    sa = synth.room_scene(61, n=20_000)
    sb = synth.room_scene(62, n=5_000)
    va = synth.room_view(200, 120, f=100.0)
    vb = dict(synth.perturb_view(va, np.array([0.05, 0.0, 0.02, 0.0, 0.03, 0.0])))
    rgb, dep = synth.zbuffer_targets(sa, va, 63)
    rgb2, dep2 = synth.zbuffer_targets(sa, vb, 64)
    cases = [([sa], [va], [(rgb, dep)], "single"), ([sa, sb], [dict(va, scene=0), dict(vb, scene=0)],
                                                    [(rgb, dep), (rgb2, dep2)], "shared")]
    for scs, vws, tg, kind in cases:
        outs = []
        for mode in (0, 1):
            R = G.Renderer(0)
            R.ctx.set_grad_mode(mode)
            scenes = [G.Scene.from_numpy(s) for s in scs]
            color, depth, acc, ws, mp = R.forward(scenes, vws)
            trgb = torch.as_tensor(np.concatenate([np.asarray(t[0], np.float32).reshape(-1) for t in tg]),
                                   device="cuda")
            tdep = torch.as_tensor(np.concatenate([np.asarray(t[1], np.float32).reshape(-1) for t in tg]),
                                   device="cuda")
            loss = torch.zeros(len(vws), device="cuda")
            dC, dD = torch.empty_like(color), torch.empty_like(depth)
            G.gs_loss_l1(R.ctx, vws, (color, depth, acc), trgb, tdep, 1.0, 0.5, loss, (dC, dD, None))
            fill = 0.0 if mode == 0 else 7.0
            grads = [{k: torch.full_like(getattr(s, k), fill) for k in G.PARAM_KEYS} for s in scenes]
            dtw = torch.full((len(vws), 6), fill, device="cuda")
            G.gs_render_backward(R.ctx, scenes, vws, ws, mp, (dC, dD, None), grads, dtw, 0)
            torch.cuda.synchronize()
            outs.append(([{k: v.cpu().numpy() for k, v in g.items()} for g in grads], dtw.cpu().numpy()))
        (g0, t0), (g1, t1) = outs
        for k in G.PARAM_KEYS:
            # two independent runs: the per-splat adjoints are float atomics, so equal up to their order
            assert rel_l2(g1[0][k], g0[0][k]) < 1e-5, k
            assert not (g1[0][k] == 7.0).any(), k  # nothing of the prefill survives
            if kind == "shared":
                assert (g1[1][k] == 0).all() and (g0[1][k] == 0).all(), k  # scene b is rendered by no view
        assert rel_l2(t1, t0) < 1e-5


def test_grad_write_mode_pose_grad_writes_the_twist(G):
    sc = synth.room_scene(65, n=10_000)
    vw = synth.room_view(160, 96, f=80.0)
    rgb, dep = synth.zbuffer_targets(sc, vw, 66)
    res = []
    for mode in (0, 1):
        R = G.Renderer(0)
        R.ctx.set_grad_mode(mode)
        scenes = [G.Scene.from_numpy(sc)]
        color, depth, acc, ws, mp = R.forward(scenes, [vw])
        loss = torch.zeros(1, device="cuda")
        dC, dD = torch.empty_like(color), torch.empty_like(depth)
        G.gs_loss_l1(R.ctx, [vw], (color, depth, acc), torch.as_tensor(rgb.reshape(-1), device="cuda"),
                     torch.as_tensor(dep.reshape(-1), device="cuda"), 1.0, 0.5, loss, (dC, dD, None))
        dtw = torch.full((1, 6), 0.0 if mode == 0 else -3.0, device="cuda")
        G.gs_pose_grad(R.ctx, scenes, [vw], ws, mp, (dC, dD, None), dtw, 0)
        res.append(dtw.cpu().numpy())
    assert rel_l2(res[1], res[0]) < 1e-5 and np.abs(res[0]).max() > 0
