"""Pins of the oracle's per-Gaussian geometry against things other than itself:
library rotations and spherical harmonics, closed forms, Monte-Carlo projection
and the derivative formulas printed in the supplement (supp. Sec. A)."""
import json
import math
import os

import numpy as np
import pytest
import torch

import oracle as O

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))
F64 = torch.float64


def _rng(s=0):
    return np.random.default_rng(s)


def test_quat_to_rotmat_matches_scipy_and_is_a_rotation():
    from scipy.spatial.transform import Rotation
    q = _rng(1).standard_normal((64, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    R = O.quat_to_rotmat(torch.tensor(q)).numpy()
    # scipy takes scalar-last quaternions (x, y, z, w)
    R_ref = Rotation.from_quat(np.concatenate([q[:, 1:], q[:, :1]], 1)).as_matrix()
    np.testing.assert_allclose(R, R_ref, atol=1e-14)
    np.testing.assert_allclose(R @ R.transpose(0, 2, 1), np.broadcast_to(np.eye(3), R.shape), atol=1e-14)
    np.testing.assert_allclose(np.linalg.det(R), 1.0, atol=1e-13)


def test_covariance_eigen_decomposition():
    """Sigma = R S S^T R^T: eigenvalues exp(2 s), eigenvectors the columns of R (Eq. covariance)."""
    rng = _rng(2)
    s = rng.uniform(-5, -1, (16, 3))
    q = rng.standard_normal((16, 4))
    Sig = O.covariance_3d(torch.tensor(s), torch.tensor(q)).numpy()
    R = O.quat_to_rotmat(torch.tensor(q / np.linalg.norm(q, axis=1, keepdims=True))).numpy()
    for i in range(16):
        np.testing.assert_allclose(Sig[i], Sig[i].T, atol=1e-18)
        for k in range(3):
            v = R[i][:, k]
            np.testing.assert_allclose(Sig[i] @ v, math.exp(2 * s[i, k]) * v, rtol=1e-12, atol=1e-18)


def _sh_scipy(l, m, d):
    """Real SH with the Condon-Shortley phase kept, from scipy's complex harmonics."""
    from scipy.special import sph_harm_y
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    if m == 0:
        std = sph_harm_y(l, 0, theta, phi).real
    elif m > 0:
        std = math.sqrt(2) * (-1) ** m * sph_harm_y(l, m, theta, phi).real
    else:
        std = math.sqrt(2) * (-1) ** m * sph_harm_y(l, -m, theta, phi).imag
    return (-1) ** abs(m) * std


def test_sh_basis_matches_scipy_up_to_degree_3():
    d = _rng(3).standard_normal((200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y = O.sh_basis(3, torch.tensor(d)).numpy()
    k = 0
    for l in range(4):
        for m in range(-l, l + 1):
            np.testing.assert_allclose(Y[:, k], _sh_scipy(l, m, d), atol=1e-13, err_msg=f"l={l} m={m}")
            k += 1


def test_sh_low_order_golden():
    g = GOLDEN["sh_low_order"]
    d = np.array([[0.36, 0.48, 0.8]])
    Y = O.sh_basis(1, torch.tensor(d)).numpy()[0]
    assert Y[0] == pytest.approx(g["Y00"], abs=1e-15)
    s = g["Y1_signs_m_minus1_0_plus1"]
    np.testing.assert_allclose(Y[1:], g["Y1_coeff"] * np.array([s[0] * 0.48, s[1] * 0.8, s[2] * 0.36]),
                               atol=1e-15)


def _one_gaussian_scene(mean, log_scale, quat=(1, 0, 0, 0), logit=0.0, sh_degree=0, rgb=(0.2, 0.4, 0.6)):
    K = (sh_degree + 1) ** 2
    sh = np.zeros((K * 3, 1), np.float32)
    sh[0:3, 0] = (np.asarray(rgb) - 0.5) / 0.28209479177387814
    return dict(mean=np.asarray(mean, np.float32).reshape(3, 1),
                log_scale=np.asarray(log_scale, np.float32).reshape(3, 1),
                quat=np.asarray(quat, np.float32).reshape(4, 1),
                opacity_logit=np.array([logit], np.float32), sh=sh, sh_degree=sh_degree)


def _view(W, H, f, T=None, cx=None, cy=None):
    T = np.concatenate([np.eye(3), np.zeros((3, 1))], 1) if T is None else np.asarray(T)
    return dict(width=W, height=H, fx=f, fy=f, cx=W / 2 if cx is None else cx, cy=H / 2 if cy is None else cy,
                z_near=0.2, bg=np.zeros(3, np.float32), T_cw=T.reshape(12).astype(np.float32))


def test_isotropic_on_axis_closed_form():
    g = GOLDEN["isotropic_on_axis"]
    sc = _one_gaussian_scene([0, 0, g["z"]], [math.log(g["s"])] * 3)
    vw = _view(g["width"], g["height"], g["f"])
    pr = O.project(O.to_params(sc), vw)
    cov = pr["cov2d"].detach().numpy()[0]
    # float32 inputs: s = exp(float32(log 0.02)) differs from 0.02 by ~1e-7 relative
    assert cov[0] == pytest.approx(g["sigma2d_diag"], rel=1e-6)
    assert cov[2] == pytest.approx(g["sigma2d_diag"], rel=1e-6)
    assert cov[1] == pytest.approx(g["sigma2d_offdiag"], abs=1e-12)
    assert int(pr["radius"][0]) == g["radius"]
    np.testing.assert_allclose(pr["mu"].detach().numpy()[0], g["mu"], atol=1e-12)
    assert float(pr["depth"][0]) == pytest.approx(g["depth"], rel=1e-7)
    # the conic is the inverse of Sigma'
    A, B, C = pr["conic"].detach().numpy()[0]
    np.testing.assert_allclose(np.array([[A, B], [B, C]]) @ np.array([[cov[0], cov[1]], [cov[1], cov[2]]]),
                               np.eye(2), atol=1e-12)


def test_projected_covariance_matches_monte_carlo():
    """For a small Gaussian (s/z ~ 1e-3) the linearised Sigma' = J W Sigma W^T J^T
    (Eq. covariance2d, no low-pass) matches the covariance of exactly projected
    samples to O(s/z); the pose is a general rotation + translation, so this
    checks the world->camera reading of P and the Jacobian J."""
    rng = _rng(4)
    qp = np.array([0.9, 0.2, -0.3, 0.25])
    R = O.quat_to_rotmat(torch.tensor(qp / np.linalg.norm(qp))).numpy()
    t = np.array([0.3, -0.2, 1.0])
    T = np.concatenate([R, t[:, None]], 1)
    Xw = R.T @ (np.array([0.4, -0.25, 3.0]) - t)     # camera-frame point (0.4, -0.25, 3)
    ls = np.log([0.004, 0.002, 0.003])
    q = np.array([0.6, -0.5, 0.4, 0.3])
    sc = _one_gaussian_scene(Xw, ls, q)
    vw = _view(640, 480, 500.0, T)
    vw["T_cw"] = T.reshape(12)  # float64 pose for this test
    pr = O.project(O.to_params(sc), vw, lowpass=0.0, fov_guard=None,
                   pose=(torch.tensor(R), torch.tensor(t)))
    cov = pr["cov2d"].detach().numpy()[0]
    Sig = O.covariance_3d(torch.tensor(np.asarray(sc["log_scale"], np.float64).T),
                          torch.tensor(np.asarray(sc["quat"], np.float64).T)).numpy()[0]
    X = rng.multivariate_normal(np.asarray(sc["mean"], np.float64)[:, 0], Sig, size=400_000)
    Xc = X @ R.T + t
    uv = np.stack([500 * Xc[:, 0] / Xc[:, 2], 500 * Xc[:, 1] / Xc[:, 2]], 1)
    emp = np.cov(uv.T)
    ref = np.array([[cov[0], cov[1]], [cov[1], cov[2]]])
    assert np.abs(emp - ref).max() / np.abs(ref).max() < 1.5e-2
    # and the projected centre is the pinhole projection of the mean
    np.testing.assert_allclose(pr["mu"].detach().numpy()[0], [500 * 0.4 / 3 + 320, 500 * -0.25 / 3 + 240],
                               rtol=1e-6)


def test_supplement_dm_dXc_with_corrected_entry():
    """supp. Sec. A prints dm/dX^c = [[fx/z, 0, -fx x/z], [0, fy/z, -fy y/z^2]]; the
    (0,2) entry must read -fx x/z^2 (the printed -fx x/z is dimensionally wrong).
    Checked on the oracle's own projection at the identity pose (X^c = X)."""
    x, y, z = 0.4, -0.3, 2.5
    fx, fy = 500.0, 450.0
    sc = _one_gaussian_scene([x, y, z], [math.log(0.01)] * 3)
    vw = dict(width=640, height=480, fx=fx, fy=fy, cx=320.0, cy=240.0, z_near=0.2,
              bg=np.zeros(3, np.float32), T_cw=np.concatenate([np.eye(3), np.zeros((3, 1))], 1).reshape(12))
    p = O.to_params(sc)

    def mu_of(X):
        q = dict(p)
        q["mean"] = X[None, :]
        return O.project(q, vw)["mu"][0]

    X0 = p["mean"][0].clone()
    Jm = torch.autograd.functional.jacobian(mu_of, X0).numpy()
    x, y, z = X0.numpy()
    corrected = np.array([[fx / z, 0, -fx * x / z ** 2], [0, fy / z, -fy * y / z ** 2]])
    printed = corrected.copy()
    printed[0, 2] = -fx * x / z
    np.testing.assert_allclose(Jm, corrected, rtol=1e-12)
    assert not np.allclose(Jm, printed)


def _paper_dXc_dq(q, X):
    """supp. Eq. grad_q as printed (row sums of the 3x3 arrays), with the single
    correction of the (2,0) entry of dX^c/dq_i (printed -q_k x; the derivative of
    the third row of supp. Eq. q2R w.r.t. q_i is +2 q_k x)."""
    r, i, j, k = q
    x, y, z = X
    d_r = 2 * np.array([[0, -k * y, j * z], [k * x, 0, -i * z], [-j * x, i * y, 0]])
    d_i = 2 * np.array([[0, j * y, k * z], [j * x, -2 * i * y, -r * z], [+k * x, r * y, -2 * i * z]])
    d_j = 2 * np.array([[-2 * j * x, i * y, r * z], [i * x, 0, k * z], [-r * x, k * y, -2 * j * z]])
    d_k = 2 * np.array([[-2 * k * x, -r * y, i * z], [r * x, -2 * k * y, j * z], [i * x, j * y, 0]])
    return np.stack([m.sum(1) for m in (d_r, d_i, d_j, d_k)], 1)  # (3 rows of X^c, 4 q comps)


def test_supplement_dXc_dq_matches_autograd_of_q2R():
    rng = _rng(5)
    for _ in range(5):
        q = rng.standard_normal(4)
        X = rng.standard_normal(3)
        Jq = torch.autograd.functional.jacobian(
            lambda qq: O.quat_to_rotmat(qq) @ torch.tensor(X), torch.tensor(q)).numpy()
        np.testing.assert_allclose(Jq, _paper_dXc_dq(q, X), atol=1e-12)
    # the printed sign of that entry is wrong: with it the row does not match
    q = np.array([0.3, 0.5, -0.2, 0.7])
    X = np.array([1.0, 0.0, 0.0])
    Jq = torch.autograd.functional.jacobian(
        lambda qq: O.quat_to_rotmat(qq) @ torch.tensor(X), torch.tensor(q)).numpy()
    assert Jq[2, 1] == pytest.approx(2 * q[3] * X[0])
    assert Jq[2, 1] != pytest.approx(-2 * q[3] * X[0])


def _paper_dvecSigma_de(E, S):
    """supp. Eq. grad_m as printed: d vec(Sigma')/d e_ab for Sigma' = E S E^T,
    vec = (00, 01, 10, 11)."""
    e = E
    s = S
    d = {}
    d[(0, 0)] = [2 * e[0, 0] * s[0, 0] + e[0, 1] * s[0, 1] + e[0, 1] * s[1, 0] + e[0, 2] * s[0, 2] + e[0, 2] * s[2, 0],
                 e[1, 0] * s[0, 0] + e[1, 1] * s[0, 1] + e[1, 2] * s[0, 2],
                 e[1, 0] * s[0, 0] + e[1, 1] * s[1, 0] + e[1, 2] * s[2, 0], 0]
    d[(0, 1)] = [e[0, 0] * s[0, 1] + e[0, 0] * s[1, 0] + 2 * e[0, 1] * s[1, 1] + e[0, 2] * s[1, 2] + e[0, 2] * s[2, 1],
                 e[1, 0] * s[1, 0] + e[1, 1] * s[1, 1] + e[1, 2] * s[1, 2],
                 e[1, 0] * s[0, 1] + e[1, 1] * s[1, 1] + e[1, 2] * s[2, 1], 0]
    d[(0, 2)] = [e[0, 0] * s[0, 2] + e[0, 0] * s[2, 0] + e[0, 1] * s[1, 2] + e[0, 1] * s[2, 1] + 2 * e[0, 2] * s[2, 2],
                 e[1, 0] * s[2, 0] + e[1, 1] * s[2, 1] + e[1, 2] * s[2, 2],
                 e[1, 0] * s[0, 2] + e[1, 1] * s[1, 2] + e[1, 2] * s[2, 2], 0]
    d[(1, 0)] = [0, e[0, 0] * s[0, 0] + e[0, 1] * s[1, 0] + e[0, 2] * s[2, 0],
                 e[0, 0] * s[0, 0] + e[0, 1] * s[0, 1] + e[0, 2] * s[0, 2],
                 2 * e[1, 0] * s[0, 0] + e[1, 1] * s[0, 1] + e[1, 1] * s[1, 0] + e[1, 2] * s[0, 2] + e[1, 2] * s[2, 0]]
    d[(1, 1)] = [0, e[0, 0] * s[0, 1] + e[0, 1] * s[1, 1] + e[0, 2] * s[2, 1],
                 e[0, 0] * s[1, 0] + e[0, 1] * s[1, 1] + e[0, 2] * s[1, 2],
                 e[1, 0] * s[0, 1] + e[1, 0] * s[1, 0] + 2 * e[1, 1] * s[1, 1] + e[1, 2] * s[1, 2] + e[1, 2] * s[2, 1]]
    d[(1, 2)] = [0, e[0, 0] * s[0, 2] + e[0, 1] * s[1, 2] + e[0, 2] * s[2, 2],
                 e[0, 0] * s[2, 0] + e[0, 1] * s[2, 1] + e[0, 2] * s[2, 2],
                 e[1, 0] * s[0, 2] + e[1, 0] * s[2, 0] + e[1, 1] * s[1, 2] + e[1, 1] * s[2, 1] + 2 * e[1, 2] * s[2, 2]]
    return d


def test_supplement_dSigma_prime_dE_matches_autograd():
    """All six printed vectors of supp. Eq. grad_m equal the derivative of the
    matrix product E Sigma E^T the oracle evaluates (a general, non-symmetric
    Sigma, so every index of the printed formulas is exercised)."""
    rng = _rng(6)
    E = rng.standard_normal((2, 3))
    S = rng.standard_normal((3, 3))
    Jt = torch.autograd.functional.jacobian(
        lambda ee: (ee @ torch.tensor(S) @ ee.T).reshape(4), torch.tensor(E)).numpy()  # (4, 2, 3)
    d = _paper_dvecSigma_de(E, S)
    for (a, b), vec in d.items():
        np.testing.assert_allclose(Jt[:, a, b], vec, atol=1e-12, err_msg=f"e_{a}{b}")


def test_cull_and_depth_key_in_float32():
    """A Gaussian exactly at z_near is dropped; the sort key is the float32 depth."""
    sc = _one_gaussian_scene([0, 0, 0.2], [math.log(0.01)] * 3)
    vw = _view(64, 48, 50.0)
    pr = O.project(O.to_params(sc), vw)
    assert len(pr["index"]) == 0
    sc = _one_gaussian_scene([0, 0, 0.25], [math.log(0.01)] * 3)
    pr = O.project(O.to_params(sc), vw)
    assert len(pr["index"]) == 1 and pr["depth32"].dtype == np.float32
