"""Pins of the oracle's tracking helpers: the SE(3) exponential against scipy's
matrix exponential, Adam's closed-form first steps, and the reliable-Gaussian
selection of Eq. coarse2fine on a hand-built scene."""
import math

import numpy as np
import pytest

import synth
from oracle import slam_ops as S


def _hat4(xi):
    rho, phi = xi[:3], xi[3:]
    M = np.zeros((4, 4))
    M[:3, :3] = [[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]]
    M[:3, 3] = rho
    return M


@pytest.mark.parametrize("scale", [1e-9, 1e-3, 0.3, 2.0])
def test_se3_exp_matches_matrix_exponential(scale):
    from scipy.linalg import expm
    rng = np.random.default_rng(int(scale * 1e9) % 1000)
    xi = rng.standard_normal(6) * scale
    np.testing.assert_allclose(S.se3_exp_np(xi), expm(_hat4(xi)), atol=1e-13)


def test_adam_first_steps_have_closed_form():
    """With zero moments, step 1 moves each component by -lr * g / (|g| + eps) and a
    repeated gradient keeps that step (mhat = g, vhat = g^2): Adam's scale invariance."""
    T0 = synth.look_at((1.0, 2.0, 1.5), (4.0, 3.0, 1.0))
    g = np.array([0.3, -2.0, 0.0, 1e-3, -5.0, 0.7])
    lr = np.array([2e-4, 2e-4, 2e-4, 1e-3, 1e-3, 1e-3])
    T1, m, v = S.pose_adam_step(T0, g, np.zeros(6), np.zeros(6), 1, lr)
    delta = -lr * g / (np.abs(g) + 1e-8)
    want = (S.se3_exp_np(delta) @ np.vstack([T0, [0, 0, 0, 1]]))[:3]
    np.testing.assert_allclose(T1, want, atol=1e-15)
    T2, m, v = S.pose_adam_step(T1, g, m, v, 2, lr)
    want2 = (S.se3_exp_np(delta) @ np.vstack([T1, [0, 0, 0, 1]]))[:3]
    np.testing.assert_allclose(T2, want2, atol=1e-14)
    # a zero gradient at step 1 leaves the pose
    T3, _, _ = S.pose_adam_step(T0, np.zeros(6), np.zeros(6), np.zeros(6), 1, lr)
    np.testing.assert_allclose(T3, T0, atol=0)


def test_select_reliable_on_a_plane():
    """Identity camera looking at a wall z = 2 m: Gaussians on the wall are reliable,
    floaters 0.3 m in front are not, nor are Gaussians off-image, behind the camera or
    over pixels without a depth reading (Eq. coarse2fine with eps = 0.05 m)."""
    W, H, f = 32, 24, 20.0
    view = synth.make_view(W, H, f, f, W / 2, H / 2, np.concatenate([np.eye(3), np.zeros((3, 1))], 1))
    D = np.full((H, W), 2.0, np.float32)
    D[:, :4] = 0.0  # no reading in the first 4 columns
    # pixel (u, v) -> point at depth z through the pixel's interior
    def at(u, v, z):
        return [(u + 0.3 - W / 2) * z / f, (v + 0.6 - H / 2) * z / f, z]
    pts = [at(10, 5, 2.0), at(20, 12, 2.03), at(8, 8, 1.7), at(2, 3, 2.0), at(40, 3, 2.0), [0, 0, -1.0],
           at(30, 20, 1.96)]
    want = [1, 1, 0, 0, 0, 0, 1]
    n = len(pts)
    sc = dict(mean=np.asarray(pts, np.float32).T.copy(), log_scale=np.full((3, n), -4.0, np.float32),
              quat=np.tile(np.array([[1], [0], [0], [0]], np.float32), (1, n)),
              opacity_logit=np.zeros(n, np.float32), sh=np.zeros((3, n), np.float32), sh_degree=0)
    np.testing.assert_array_equal(S.select_reliable(sc, view, D, 0.05), want)


def test_select_opacity():
    sc = dict(opacity_logit=np.array([-1.0, 0.0, 0.01, 3.0], np.float32))
    np.testing.assert_array_equal(S.select_opacity(sc, 0.5), [0, 0, 1, 1])
    np.testing.assert_array_equal(S.select_opacity(sc, 0.5, keep=np.array([1, 1, 0, 1])), [0, 0, 0, 1])


def _plane_case():
    W, H, f = 24, 16, 16.0
    view = synth.make_view(W, H, f, f, W / 2, H / 2, synth.look_at((0.2, -0.1, 0.0), (0.3, 0.1, 3.0), up=(0, -1, 0)))
    rng = np.random.default_rng(5)
    T = np.asarray(view["T_cw"], np.float64).reshape(3, 4)
    # three Gaussians: on the observed surface, a floater 0.5 m in front, one off-image
    def world(u, v, z):
        Xc = np.array([(u + 0.4 - W / 2) * z / f, (v + 0.7 - H / 2) * z / f, z])
        return T[:, :3].T @ (Xc - T[:, 3])
    pts = np.stack([world(5, 5, 2.0), world(12, 9, 1.5), world(40, 2, 2.0)], 1)
    sc = dict(mean=pts.astype(np.float32), log_scale=np.full((3, 3), -4.0, np.float32),
              quat=np.tile(np.array([[1], [0], [0], [0]], np.float32), (1, 3)),
              opacity_logit=np.array([1.0, 2.0, 0.5], np.float32), sh=rng.normal(0, 1, (12, 3)).astype(np.float32),
              sh_degree=1)
    D = np.full((H, W), 2.0, np.float32)
    D[0, :] = 0.0
    acc = np.full((H, W), 0.9, np.float32)
    acc[3:6, 10:14] = 0.2                      # holes: 12 unreliable pixels
    Dh = np.full((H, W), 2.0, np.float32)
    Dh[10, 2] = 2.5                            # depth disagreement: 1 more
    Dh[0, 3] = 0.5                             # but no depth reading there: not added
    C = rng.uniform(0, 1, (3, H, W)).astype(np.float32)
    return sc, view, acc, Dh, C, D


def test_expand_add_delete_prune_by_hand():
    """Eq. add_method / Eq. delete_method / Eq. init-rep on a hand-built keyframe."""
    sc, view, acc, Dh, C, D = _plane_case()
    out, (nk, na) = S.expand(sc, view, acc, Dh, C, D, tau_T=0.5, tau_D=0.1, eta=0.01, gamma=0.1)
    # the floater (index 1, 0.5 m in front of D = 2) decays 0.88 -> 0.0088 (kept, > 0.005);
    # the surface Gaussian and the off-image one are untouched
    o = 1 / (1 + np.exp(-out["opacity_logit"][:3]))
    np.testing.assert_allclose(o, [1 / (1 + np.exp(-1.0)), 0.01 / (1 + np.exp(-2.0)), 1 / (1 + np.exp(-0.5))],
                               rtol=1e-6)
    assert (nk, na) == (3, 13)
    # the new Gaussians re-project onto their pixel centres at depth D
    T = np.asarray(view["T_cw"], np.float64).reshape(3, 4)
    Xc = T[:, :3] @ out["mean"][:, 3:].astype(np.float64) + T[:, 3:4]
    u = view["fx"] * Xc[0] / Xc[2] + view["cx"]
    v = view["fy"] * Xc[1] / Xc[2] + view["cy"]
    np.testing.assert_allclose(Xc[2], 2.0, rtol=1e-6)
    np.testing.assert_allclose(u - np.floor(u), 0.5, atol=1e-4)
    np.testing.assert_allclose(v - np.floor(v), 0.5, atol=1e-4)
    raster = np.floor(v) * 24 + np.floor(u)
    assert (np.diff(raster) > 0).all()          # raster order
    # init values: colour of the pixel through the SH DC term, scale D / f, identity rotation
    Y00 = 1 / (2 * np.sqrt(np.pi))
    rgb = out["sh"][0:3, 3:] * Y00 + 0.5
    np.testing.assert_allclose(rgb, C[:, np.floor(v).astype(int), np.floor(u).astype(int)], atol=1e-6)
    np.testing.assert_allclose(np.exp(out["log_scale"][:, 3:]), 2.0 / 16.0, rtol=1e-6)
    assert (out["quat"][:, 3:] == np.array([[1], [0], [0], [0]])).all()
    np.testing.assert_allclose(1 / (1 + np.exp(-out["opacity_logit"][3:])), 0.1, rtol=1e-6)
    assert (out["sh"][3:, 3:] == 0).all()
    # with eta small enough the floater is pruned (opacity < 0.005)
    out2, (nk2, na2) = S.expand(sc, view, acc, Dh, C, D, eta=0.001)
    assert nk2 == 2 and na2 == 13
    np.testing.assert_array_equal(out2["mean"][:, :2], sc["mean"][:, [0, 2]])
    # first-frame sampling: the checkerboard half of the unreliable pixels
    out3, (_, na3) = S.expand(sc, view, acc, Dh, C, D, checkerboard=True, density=0.5)
    assert na3 == 7
    np.testing.assert_allclose(np.exp(out3["log_scale"][:, 3:]), 2.0 / 16.0 * np.sqrt(2), rtol=1e-6)


def test_densify_clone_and_split_by_hand():
    """Three Gaussians: below the gradient threshold (kept), small and above it
    (cloned), large and above it (split into two children sampled from it)."""
    q = np.array([[1, 0, 0, 0], [1, 0, 0, 0], [np.cos(0.3), 0, 0, np.sin(0.3)]], np.float32).T.copy()
    ls = np.log(np.array([[0.01, 0.01, 0.01], [0.01, 0.015, 0.005], [0.05, 0.02, 0.01]], np.float32)).T.copy()
    sc = dict(mean=np.array([[0, 0, 1], [1, 0, 2], [0, 1, 3]], np.float32).T.copy(), log_scale=ls, quat=q,
              opacity_logit=np.array([0.1, 0.2, 0.3], np.float32), sh=np.arange(12, dtype=np.float32).reshape(12, 1)
              * np.ones((1, 3), np.float32), sh_degree=1)
    grad_sum = np.array([0.001, 0.009, 0.004], np.float32)
    count = np.array([1, 3, 1], np.float32)   # averages 0.001, 0.003, 0.004
    noise = np.zeros((6, 3), np.float32)
    noise[:, 2] = [1, 0, 0, 0, -1, 2]
    out, (nk, nc, ns) = S.densify(sc, grad_sum, count, noise)
    assert (nk, nc, ns) == (2, 1, 1)
    assert out["mean"].shape == (3, 5)
    # kept: 0 and 1 in order; then the clone of 1; then the two children of 2
    np.testing.assert_array_equal(out["mean"][:, :3], sc["mean"][:, [0, 1, 1]])
    np.testing.assert_array_equal(out["sh"][:, 2], sc["sh"][:, 1])
    # child c = mean + R (s * z_c); R rotates by 0.6 rad about z
    c, s_ = np.cos(0.6), np.sin(0.6)
    Rz = np.array([[c, -s_, 0], [s_, c, 0], [0, 0, 1]])
    sz = np.array([0.05, 0.02, 0.01])
    np.testing.assert_allclose(out["mean"][:, 3], sc["mean"][:, 2] + Rz @ (sz * [1, 0, 0]), atol=1e-6)
    np.testing.assert_allclose(out["mean"][:, 4], sc["mean"][:, 2] + Rz @ (sz * [0, -1, 2]), atol=1e-6)
    np.testing.assert_allclose(np.exp(out["log_scale"][:, 3:]), np.tile(sz[:, None] / 1.6, (1, 2)), rtol=1e-6)
    assert (out["opacity_logit"][3:] == np.float32(0.3)).all()
    # no gradient statistics (count 0): nothing densifies
    out2, counts = S.densify(sc, grad_sum, np.zeros(3, np.float32), noise)
    assert counts == (3, 0, 0)


def test_ndc_gradient_norm():
    np.testing.assert_allclose(S.ndc_grad_norm(np.array([[3.0, 4.0]]), 2.0, 2.0), [5.0])
    np.testing.assert_allclose(S.ndc_grad_norm(np.array([[1e-3, 0.0]]), 640, 480), [0.32])


def test_outlier_mask_by_hand():
    losses = np.array([1.0, 2.0, 3.0, 40.0, 25.0, 0.5, 100.0, 5.0], np.float32)
    mask = np.array([1, 1, 1, 1, 1, 1, 1, 0], np.uint8)
    # masked losses sorted: 0.5 1 2 3 25 40 100 -> lower median (rank 3) = 3, threshold 30
    np.testing.assert_array_equal(S.outlier_mask(losses, mask), [1, 1, 1, 0, 1, 1, 0, 0])
    np.testing.assert_array_equal(S.outlier_mask(losses, np.zeros(8, np.uint8)), np.zeros(8))
    # an even count takes the lower of the two middle values
    np.testing.assert_array_equal(S.outlier_mask(np.array([1, 2, 3, 4], np.float32), np.ones(4), factor=1.0),
                                  [1, 1, 0, 0])


def test_pixel_losses_by_hand():
    c = np.array([[0.5, 0.0], [0.25, 0.0], [1.0, 0.0]], np.float32)
    t = np.array([[0.0, 1.0], [0.0, 0.0], [0.0, 0.0]], np.float32)
    l = S.pixel_losses(c, np.array([2.0, 3.0], np.float32), t, np.array([1.5, 0.0], np.float32), 0.8, 0.3)
    np.testing.assert_allclose(l, [0.8 * 1.75 + 0.3 * 0.5, 0.8 * 1.0], rtol=1e-6)


def test_constant_velocity_continues_a_steady_motion():
    T0 = synth.look_at((1.0, 2.0, 1.5), (4.0, 3.0, 1.0))
    step = S.se3_exp_np(np.array([0.02, -0.01, 0.03, 0.01, 0.02, -0.005]))
    h = lambda T: np.vstack([T, [0, 0, 0, 1]])  # noqa: E731
    T1 = (step @ h(T0))[:3]
    T2 = (step @ h(T1))[:3]
    np.testing.assert_allclose(S.constant_velocity(T0, T1), T2, atol=1e-12)
