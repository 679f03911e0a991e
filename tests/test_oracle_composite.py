"""Pins of the oracle's compositing (Eq. color_render, Eq. depth, accumulated
opacity), its loss and its tile binning: closed forms, a literal per-pixel
sequential loop on tiny inputs, invariants, the supplement's depth adjoint
(supp. Eq. grad_depth) and brute-force binning."""
import json
import math
import os

import numpy as np
import pytest
import torch

import oracle as O
import synth

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))
F64 = torch.float64


def _proj(mu, conic, depth, opacity, rgb):
    n = len(depth)
    d = dict(index=torch.arange(n), mu=torch.tensor(mu, dtype=F64).reshape(n, 2),
             conic=torch.tensor(conic, dtype=F64).reshape(n, 3), depth=torch.tensor(depth, dtype=F64),
             opacity=torch.tensor(opacity, dtype=F64), rgb=torch.tensor(rgb, dtype=F64).reshape(n, 3),
             cond=torch.ones(n, dtype=F64))
    d["depth32"] = np.asarray(depth, np.float32)
    return d


def _view(W, H, bg=(0, 0, 0)):
    return dict(width=W, height=H, fx=1.0, fy=1.0, cx=0.0, cy=0.0, z_near=0.2,
                bg=np.asarray(bg, np.float32), T_cw=np.zeros(12, np.float32))


def test_single_gaussian_at_pixel_centre():
    bg = (0.25, 0.5, 0.75)
    for o in (0.3, 0.995):
        pr = _proj([[3.5, 2.5]], [[0.2, 0.0, 0.2]], [1.5], [o], [[0.9, 0.1, 0.4]])
        r = O.composite(pr, _view(8, 8, bg), np.array([3]), np.array([2]))
        a = min(0.99, o)
        np.testing.assert_allclose(r["color"].numpy()[0], a * np.array([0.9, 0.1, 0.4]) + (1 - a) * np.array(bg),
                                   rtol=1e-7)  # bg is float32
        assert float(r["depth"][0]) == pytest.approx(1.5 * a, rel=1e-15)
        assert float(r["acc"][0]) == pytest.approx(a, rel=1e-15)


def test_stacked_alpha_095_golden():
    g = GOLDEN["stack_alpha_095"]
    n = g["count"]
    for k in range(1, n + 1):
        pr = _proj([[0.5, 0.5]] * k, [[1.0, 0.0, 1.0]] * k, np.arange(1, k + 1, dtype=float),
                   [g["alpha"]] * k, [[0.3, 0.6, 0.9]] * k)
        r = O.composite(pr, _view(1, 1), np.array([0]), np.array([0]))
        T = float(r["T"][0])
        want = g["T_after"][min(k, len(g["T_after"])) - 1]
        assert T == pytest.approx(want, rel=1e-12)
        assert int(r["n_contrib"][0]) == min(k, g["n_contrib"])
    assert float(r["acc"][0]) == pytest.approx(g["acc"], rel=1e-12)
    np.testing.assert_allclose(r["color"].numpy()[0], np.array([0.3, 0.6, 0.9]) * g["acc"], rtol=1e-12)


def _sequential(pr, view, u, v):
    """The compositing loop written out literally, one pixel at a time."""
    order = np.argsort(pr["depth32"], kind="stable")
    mu = pr["mu"].detach().numpy()[order]
    con = pr["conic"].detach().numpy()[order]
    dep = pr["depth"].detach().numpy()[order]
    opa = pr["opacity"].detach().numpy()[order]
    rgb = pr["rgb"].detach().numpy()[order]
    bg = np.asarray(view["bg"], np.float64)
    out = []
    for uu, vv in zip(u, v):
        px, py = uu + 0.5, vv + 0.5
        T, C, D, n = 1.0, np.zeros(3), 0.0, 0
        for i in range(len(order)):
            dx, dy = px - mu[i, 0], py - mu[i, 1]
            q = con[i, 0] * dx * dx + 2 * con[i, 1] * dx * dy + con[i, 2] * dy * dy
            if q > 9.0:
                continue
            a = min(0.99, opa[i] * math.exp(-0.5 * q))
            if a < 1.0 / 255.0:
                continue
            if T * (1 - a) < 1e-4:
                break
            C += rgb[i] * a * T
            D += dep[i] * a * T
            T *= 1 - a
            n += 1
        out.append((C + T * bg, D, 1 - T, T, n))
    return out


def test_closed_form_composite_equals_sequential_loop():
    rng = np.random.default_rng(7)
    n, W, H = 80, 20, 14
    mu = rng.uniform(-2, [W + 2, H + 2], (n, 2))
    L = rng.standard_normal((n, 2, 2)) * 1.5
    cov = L @ L.transpose(0, 2, 1) + 0.3 * np.eye(2)
    inv = np.linalg.inv(cov)
    conic = np.stack([inv[:, 0, 0], inv[:, 0, 1], inv[:, 1, 1]], 1)
    depth = rng.uniform(0.5, 3, n)
    depth[5] = depth[6]  # a depth tie: index order decides
    opa = rng.uniform(0.05, 1.0, n)
    rgb = rng.uniform(0, 1, (n, 3))
    pr = _proj(mu, conic, depth, opa, rgb)
    vw = _view(W, H, (0.1, 0.2, 0.3))
    uu, vv = np.meshgrid(np.arange(W), np.arange(H))
    u, v = uu.reshape(-1), vv.reshape(-1)
    r = O.composite(pr, vw, u, v)
    ref = _sequential(pr, vw, u, v)
    np.testing.assert_allclose(r["color"].numpy(), np.stack([x[0] for x in ref]), atol=1e-13)
    np.testing.assert_allclose(r["depth"].numpy(), [x[1] for x in ref], atol=1e-13)
    np.testing.assert_allclose(r["acc"].numpy(), [x[2] for x in ref], atol=1e-13)
    np.testing.assert_allclose(r["T"].numpy(), [x[3] for x in ref], atol=1e-13)
    np.testing.assert_array_equal(r["n_contrib"], [x[4] for x in ref])
    assert max(x[4] for x in ref) >= 5 and min(x[3] for x in ref) < 1e-2  # non-trivial stacks


def test_invariants_on_frustum_scene():
    w = synth.workload_plain_2k()
    sc, vw = w["scenes"][0], w["views"][0]
    r = O.render_view(sc, vw)
    T, A = r["T"], r["acc"]
    assert (T > 0).all() and (T <= 1).all()
    np.testing.assert_allclose(A, 1 - T, atol=0)
    # transmittance never increases along a pixel's list
    p = O.to_params(sc)
    pr = O.project(p, vw)
    order = O.depth_order(pr)
    u = np.array([10, 80, 150, 33]); v = np.array([5, 60, 110, 90])
    prev = np.ones(len(u))
    for k in range(0, len(order) + 1, 50):
        rk = O.composite(pr, vw, u, v, order[:k]) if k > 0 else None
        Tk = np.ones(len(u)) if rk is None else rk["T"].numpy()
        assert (Tk <= prev + 1e-15).all()
        prev = Tk


def test_uniform_colour_and_depth_identities():
    """Uniform colour c with a black background renders c * A; a scene with every
    Gaussian at one depth d renders depth d * A (Eq. color_render, Eq. depth)."""
    sc, vw = synth.frustum_scene(5, n=400, width=64, height=48, f=50.0)
    c = np.array([0.3, 0.55, 0.8])
    sc["sh"][0:3] = ((c - 0.5) / 0.28209479177387814)[:, None]
    r = O.render_view(sc, vw)
    np.testing.assert_allclose(r["color"], c[:, None, None] * r["acc"][None], atol=1e-14)
    d = 2.0
    m = sc["mean"].astype(np.float64)
    sc["mean"] = (m / m[2:3] * d).astype(np.float32)
    sc["mean"][2] = d
    r = O.render_view(sc, vw)
    np.testing.assert_allclose(r["depth"], d * r["acc"], rtol=1e-12, atol=1e-15)


def test_supplement_depth_adjoint():
    """supp. Eq. grad_depth: dD/da_i = d_i prod_{j<i}(1-a_j)
    - sum_{k>i} d_k a_k prod_{j<k, j != i}(1-a_j);  dD/dd_i = a_i prod_{j<i}(1-a_j).
    Gaussians centred on the pixel (q = 0) so a_i = o_i; no background, no stop."""
    a = np.array([0.3, 0.5, 0.2, 0.6, 0.4])
    d = np.array([1.0, 1.3, 1.7, 2.2, 2.9])
    n = len(a)
    pr = _proj([[0.5, 0.5]] * n, [[1.0, 0.0, 1.0]] * n, d, a, [[0.5, 0.5, 0.5]] * n)
    opa = pr["opacity"].clone().requires_grad_(True)
    dep = pr["depth"].clone().requires_grad_(True)
    pr["opacity"], pr["depth"] = opa, dep
    r = O.composite(pr, _view(1, 1), np.array([0]), np.array([0]))
    r["depth"].sum().backward()
    T = np.concatenate([[1.0], np.cumprod(1 - a)[:-1]])
    dD_da = np.zeros(n)
    for i in range(n):
        s = 0.0
        for k in range(i + 1, n):
            s += d[k] * a[k] * np.prod([1 - a[j] for j in range(k) if j != i])
        dD_da[i] = d[i] * T[i] - s
    np.testing.assert_allclose(opa.grad.numpy(), dD_da, rtol=1e-13)
    np.testing.assert_allclose(dep.grad.numpy(), a * T, rtol=1e-13)


def test_l1_loss_conventions():
    """Eq. map_loss: sum of |.|; sign(0) = 0; the depth term only where D_obs > 0."""
    C = torch.tensor([[0.5, 0.2, 0.9]], dtype=F64, requires_grad=True)
    D = torch.tensor([1.0, 2.0], dtype=F64, requires_grad=True)
    L = O.l1_loss(torch.cat([C, C]), D, torch.tensor([[0.5, 0.3, 0.1]] * 2, dtype=F64),
                  torch.tensor([0.5, 0.0], dtype=F64), 1.0, 0.5)
    assert float(L) == pytest.approx(2 * (0.1 + 0.8) + 0.5 * 0.5)
    L.backward()
    np.testing.assert_allclose(C.grad.numpy(), [[0.0, -2.0, 2.0]])
    np.testing.assert_allclose(D.grad.numpy(), [0.5, 0.0])


def test_pixel_mask_renders_only_masked_pixels():
    sc, vw = synth.frustum_scene(6, n=200, width=32, height=24, f=25.0)
    mask = np.zeros((24, 32), np.uint8)
    mask[3:9, 5:20] = 1
    full = O.render_view(sc, vw)
    part = O.render_view(sc, vw, pixel_mask=mask)
    m = mask.astype(bool)
    np.testing.assert_array_equal(part["color"][:, m], full["color"][:, m])
    assert (part["color"][:, ~m] == 0).all() and (part["T"][~m] == 1).all()


def test_tile_lists_match_brute_force_pixel_enumeration():
    rng = np.random.default_rng(8)
    n, W, H, tw, th = 300, 53, 37, 16, 8
    mu_x = rng.uniform(-10, W + 10, n).astype(np.float32)
    mu_y = rng.uniform(-10, H + 10, n).astype(np.float32)
    ex = rng.uniform(0.2, 12, n).astype(np.float32)
    ey = rng.uniform(0.2, 12, n).astype(np.float32)
    depth = rng.uniform(0.5, 4, n).astype(np.float32)
    depth[7] = depth[9]
    valid = rng.uniform(0, 1, n) < 0.9
    lists = O.tile_lists(mu_x, mu_y, ex, ey, O.depth_bits(depth), valid, W, H, tw, th)
    tiles_x = (W + tw - 1) // tw
    order = np.lexsort((np.arange(n), depth))
    for t, lst in enumerate(lists):
        tx, ty = t % tiles_x, t // tiles_x
        want = []
        for g in order:
            if not valid[g]:
                continue
            hit = False
            for v in range(ty * th, min(H, ty * th + th)):
                if not (mu_y[g] - ey[g] <= v + 0.5 <= mu_y[g] + ey[g]):
                    continue
                for u in range(tx * tw, min(W, tx * tw + tw)):
                    if mu_x[g] - ex[g] <= u + 0.5 <= mu_x[g] + ex[g]:
                        hit = True
                        break
                if hit:
                    break
            if hit:
                want.append(int(g))
        assert lst == want, t


def test_footprint_box_bounds_every_contributing_pixel():
    """Every pixel where a Gaussian passes both tests (q <= 9 and alpha >= 1/255)
    lies inside its footprint box (brute force over a grid around each Gaussian)."""
    sc, vw = synth.frustum_scene(9, n=60, width=40, height=30, f=30.0)
    pr = O.project(O.to_params(sc), vw)
    ex, ey = O.footprint_extents(pr["cov2d"].detach().numpy(), pr["opacity"].detach().numpy())
    mu = pr["mu"].detach().numpy()
    con = pr["conic"].detach().numpy()
    o = pr["opacity"].detach().numpy()
    for i in range(len(o)):
        g = np.linspace(-40, 40, 801)
        dx, dy = np.meshgrid(g, g)
        q = con[i, 0] * dx * dx + 2 * con[i, 1] * dx * dy + con[i, 2] * dy * dy
        a = np.minimum(0.99, o[i] * np.exp(-0.5 * q))
        ok = (q <= 9) & (a >= 1 / 255)
        if ok.any():
            assert np.abs(dx[ok]).max() <= ex[i] + 1e-9 and np.abs(dy[ok]).max() <= ey[i] + 1e-9
            # and the box is tight: it is reached by the region
            assert np.abs(dx[ok]).max() >= ex[i] - 0.2 and np.abs(dy[ok]).max() >= ey[i] - 0.2


def _comp1(pr, view, u, v):
    r = O.composite(pr, view, np.array([u]), np.array([v]))
    return r["color"].numpy()[0], float(r["depth"][0]), float(r["acc"][0])


def _same(alt, ref):
    c, d, a = ref
    return np.allclose(alt["color"], c, rtol=0, atol=1e-12) and abs(alt["depth"] - d) < 1e-12 and \
        abs(alt["acc"] - a) < 1e-12


def _drop(pr, k):
    keep = [i for i in range(len(pr["depth"])) if i != k]
    t = lambda x: x[keep]  # noqa: E731
    out = {key: t(val) for key, val in pr.items() if key != "depth32"}
    out["depth32"] = pr["depth32"][keep]
    return out


def test_pixel_alternatives_without_near_decisions_is_the_composite():
    """Away from every threshold the walk has one outcome: the closed-form composite."""
    w = synth.workload_plain_2k()
    ref = O.render_view(w["scenes"][0], w["views"][0], pixel_mask=np.eye(120, 160, dtype=bool))
    ok = np.ones(ref["m_gate"].shape, bool)
    for k, tol in (("m_gate", 1e-6), ("m_alpha", 1e-5), ("m_stop", 1e-4)):
        ok &= ref[k] > tol
    pix = np.argwhere(ok & np.eye(120, 160, dtype=bool))[:40]
    assert len(pix) >= 30
    for v, u in pix:
        alts = O.pixel_alternatives(ref["proj"], w["views"][0], int(u), int(v))
        assert len(alts) == 1
        c, d, a = _comp1(ref["proj"], w["views"][0], int(u), int(v))
        np.testing.assert_allclose(alts[0]["color"], c, rtol=1e-12, atol=1e-13)
        assert alts[0]["depth"] == pytest.approx(d, rel=1e-12, abs=1e-13)
        assert alts[0]["acc"] == pytest.approx(a, rel=1e-12, abs=1e-13)


def test_pixel_alternatives_gate_at_three_sigma():
    """A Gaussian whose q is exactly 9 at the pixel (offset 3 along an axis of an
    identity conic): one outcome blends it (the definition, q <= 9), the other is
    the render without it."""
    view = _view(8, 8, (0.1, 0.2, 0.3))
    pr = _proj([[3.5, 2.5], [0.5, 2.5]], [[0.5, 0.0, 0.5], [1.0, 0.0, 1.0]], [1.0, 2.0], [0.6, 0.9],
               [[0.9, 0.1, 0.4], [0.2, 0.8, 0.5]])
    alts = O.pixel_alternatives(pr, view, 3, 2)
    assert len(alts) == 2
    full, without = _comp1(pr, view, 3, 2), _comp1(_drop(pr, 1), view, 3, 2)
    assert any(_same(x, full) for x in alts) and any(_same(x, without) for x in alts)
    assert not np.allclose(full[0], without[0])


def test_pixel_alternatives_alpha_at_one_255th():
    """Opacity exactly 1/255 at the Gaussian's centre: alpha sits on the skip
    threshold, so both the blend and the skip are outcomes."""
    view = _view(4, 4)
    pr = _proj([[1.5, 1.5], [1.5, 1.5]], [[1.0, 0.0, 1.0]] * 2, [1.0, 2.0], [0.5, 1.0 / 255.0],
               [[0.9, 0.1, 0.4], [0.2, 0.8, 0.5]])
    alts = O.pixel_alternatives(pr, view, 1, 1)
    assert len(alts) == 2
    assert any(_same(x, _comp1(pr, view, 1, 1)) for x in alts)
    assert any(_same(x, _comp1(_drop(pr, 1), view, 1, 1)) for x in alts)


def test_pixel_alternatives_stop_at_the_transmittance_floor():
    """Two coincident Gaussians of alpha 0.99 (clamped): after the second, T is
    (1 - 0.99)^2, within rounding of the 1e-4 floor.  One outcome blends both,
    the other stops before the second (T = 0.01)."""
    view = _view(2, 2)
    pr = _proj([[0.5, 0.5]] * 2, [[1.0, 0.0, 1.0]] * 2, [1.0, 2.0], [0.995, 0.995], [[0.3, 0.6, 0.9]] * 2)
    alts = O.pixel_alternatives(pr, view, 0, 0)
    assert len(alts) == 2
    accs = sorted(x["acc"] for x in alts)
    assert accs[0] == pytest.approx(0.99, rel=1e-12) and accs[1] == pytest.approx(1 - 1e-4, rel=1e-12)
    assert any(_same(x, _comp1(_drop(pr, 1), view, 0, 0)) for x in alts)


def test_pixel_alternatives_gives_up_past_max_near():
    """Four Gaussians each on the 3-sigma gate: 2^4 outcomes, more than the
    max_near = 3 the walk enumerates."""
    view = _view(8, 8)
    pr = _proj([[0.5, 2.5], [6.5, 2.5], [3.5, 5.5], [3.5, -0.5]], [[1.0, 0.0, 1.0]] * 4, [1.0, 2.0, 3.0, 4.0],
               [0.9] * 4, [[0.5, 0.5, 0.5]] * 4)
    assert O.pixel_alternatives(pr, view, 3, 2) is None
    assert len(O.pixel_alternatives(pr, view, 3, 2, max_near=4)) == 16
