"""Pins of the oracle's gradients (Eq. pose_grad and the map gradients of
Eq. map_loss): central finite differences in float64 of the oracle's own
forward, for every Gaussian parameter and the 6-DoF twist (exact and paper
modes), and the quaternion form of the pose in the supplement (supp. Eq. q2R,
supp. Eq. grad_q) against the twist at the identity pose."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import synth

F64 = torch.float64


def _tiny_case(seed=11, n=10, W=28, H=20, deg=3, identity=False):
    rng = np.random.default_rng(seed)
    f = 30.0
    if identity:
        T = np.concatenate([np.eye(3), np.zeros((3, 1))], 1)
    else:
        T = synth.look_at((0.3, -0.2, -0.4), (0.0, 0.1, 2.0), up=(0, -1, 0))
    R, t = T[:, :3], T[:, 3]
    # place Gaussians in front of the camera, then express them in world coordinates
    u = rng.uniform(4, W - 4, n)
    v = rng.uniform(3, H - 3, n)
    z = rng.uniform(1.5, 3.0, n)
    Xc = np.stack([(u - W / 2) * z / f, (v - H / 2) * z / f, z], 1)
    Xw = (Xc - t) @ R
    s = synth._attributes(rng, n, deg, high_sigma=0.3)
    s["log_scale"] = rng.uniform(math.log(0.03), math.log(0.12), (3, n)).astype(np.float32)
    s["opacity_logit"] = rng.uniform(-1.0, 1.5, n).astype(np.float32)
    s["mean"] = Xw.T.astype(np.float32).copy()
    view = synth.make_view(W, H, f, f, W / 2, H / 2, T, bg=(0.2, 0.1, 0.3))
    trgb, tdep = synth.random_targets(seed + 1, W, H, 1.0, 3.5)
    trgb[:, ::3, ::2] = 5.0     # far from any render, so no L1 kink sits near a test point
    return s, view, (trgb, tdep)


def _scene64(s):
    return {k: (np.asarray(v, np.float64).copy() if isinstance(v, np.ndarray) else v) for k, v in s.items()}


def _margins_ok(s, view, tol=1e-4):
    r = O.render_view(s, view)
    for k in ("m_gate", "m_alpha", "m_stop", "m_clamp"):
        assert r[k].min() > tol, (k, r[k].min())


@pytest.mark.parametrize("seed", [11, 19])
def test_parameter_gradients_match_central_differences(seed):
    s, view, tg = _tiny_case(seed)
    _margins_ok(s, view)
    g = O.render_and_grad([s], [view], [tg], 1.0, 0.5)
    base = _scene64(s)
    h = 1e-6
    rng = np.random.default_rng(seed)
    for key in O.PARAM_KEYS:
        arr = base[key]
        flat = arr.reshape(-1)
        picks = rng.choice(flat.size, size=min(flat.size, 24), replace=False)
        for i in picks:
            sp = _scene64(s)
            sm = _scene64(s)
            sp[key].reshape(-1)[i] += h
            sm[key].reshape(-1)[i] -= h
            fd = (O.loss_only([sp], [view], [tg]) - O.loss_only([sm], [view], [tg])) / (2 * h)
            an = g["grads"][0][key].reshape(-1)[i]
            assert an == pytest.approx(fd, rel=2e-5, abs=2e-5 * (1 + abs(fd))), (key, i)


@pytest.mark.parametrize("mode", ["exact", "paper"])
def test_twist_gradient_matches_central_differences(mode):
    """d/d eps L(exp(eps^) W) at eps = 0, eps = (rho, phi).  The paper mode is the
    exact derivative of the restricted function whose Sigma' and colour direction
    keep the unperturbed pose (Eq. pose_grad with those terms dropped)."""
    s, view, tg = _tiny_case(13)
    _margins_ok(s, view)
    g = O.render_and_grad([s], [view], [tg], 1.0, 0.5, pose_mode=mode)
    h = 1e-6
    for k in range(6):
        e = np.zeros((1, 6))
        e[0, k] = h
        fd = (O.loss_only([s], [view], [tg], twists=e, pose_mode=mode)
              - O.loss_only([s], [view], [tg], twists=-e, pose_mode=mode)) / (2 * h)
        assert g["twist"][0, k] == pytest.approx(fd, rel=2e-5, abs=1e-4), k
    if mode == "paper":
        ge = O.render_and_grad([s], [view], [tg], 1.0, 0.5, pose_mode="exact")
        assert np.abs(ge["twist"] - g["twist"]).max() > 1e-3  # the dropped terms matter


def test_twist_equals_half_quaternion_gradient_at_identity():
    """With the pose stored as a quaternion q and translation t (supp. Sec. A) and
    R(q) from supp. Eq. q2R, at q = (1,0,0,0), t = 0: dL/dt = dL/drho and
    dL/dq_(i,j,k) = 2 dL/dphi (R(q) = I + 2 [q_vec]_x + O(q^2))."""
    s, view, tg = _tiny_case(14, identity=True)
    g = O.render_and_grad([s], [view], [tg], 1.0, 0.5)
    p = O.to_params(s)
    q = torch.tensor([1.0, 0.0, 0.0, 0.0], dtype=F64, requires_grad=True)
    t = torch.zeros(3, dtype=F64, requires_grad=True)
    R = O.quat_to_rotmat(q)
    pr = O.project(p, view, pose=(R, t))
    W, H = view["width"], view["height"]
    uu, vv = np.meshgrid(np.arange(W), np.arange(H))
    r = O.composite(pr, view, uu.reshape(-1), vv.reshape(-1))
    L = O.l1_loss(r["color"], r["depth"], torch.tensor(tg[0].reshape(3, -1).T.astype(np.float64)),
                  torch.tensor(tg[1].reshape(-1).astype(np.float64)), 1.0, 0.5)
    L.backward()
    np.testing.assert_allclose(t.grad.numpy(), g["twist"][0, :3], rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(q.grad.numpy()[1:], 2 * g["twist"][0, 3:], rtol=1e-9, atol=1e-9)


def test_gradients_accumulate_over_views_of_one_scene():
    s, view, tg = _tiny_case(15)
    view2 = synth.perturb_view(view, [0.01, -0.02, 0.0, 0.01, 0.0, -0.01])
    both = O.render_and_grad([s], [view, view2], [tg, tg])
    one = O.render_and_grad([s], [view], [tg])
    two = O.render_and_grad([s], [view2], [tg])
    for k in O.PARAM_KEYS:
        np.testing.assert_allclose(both["grads"][0][k], one["grads"][0][k] + two["grads"][0][k],
                                   rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(both["twist"], np.concatenate([one["twist"], two["twist"]]), rtol=1e-12)
