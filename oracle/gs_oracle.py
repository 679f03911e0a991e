"""FP64 CPU oracle of GS-SLAM's differentiable RGB-D Gaussian splatting.

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the
CPU-baseline leg of `bench.py` may import this module.  It shares no code with
the CUDA path.

It is the plain definition of what the renderer computes, written in float64
with PyTorch CPU ops.  Every pixel is composited by brute force over ALL kept
Gaussians of its view in depth order: there is no tiling, binning, culling by
screen rectangle or early exit other than the termination rule that is part of
the definition.  Gradients come from torch autograd of this forward (a library
reverse sweep of exactly this function); the tests pin that reverse sweep with
central finite differences and with the supplement's closed-form derivatives.

Paper (GS-SLAM, arXiv 2311.11700) passages followed:
  Eq. scene-rep       Gaussians (X, Sigma, Lambda, Y)                   [Sec. 3.1]
  Eq. covariance      Sigma = R S S^T R^T, R from a quaternion          [Sec. 3.1]
  supp. Eq. q2R       unit quaternion [q_r, q_i, q_j, q_k] -> R         [supp. Sec. A]
  Eq. covariance2d    Sigma' = J W Sigma W^T J^T (W = world->camera)    [Sec. 3.1]
  Eq. color_render    C = sum_i c_i a_i prod_{j<i} (1 - a_j)            [Sec. 3.1]
  Eq. depth           D = sum_i d_i a_i prod_{j<i} (1 - a_j)            [Sec. 3.1]
  Sec. 3.2 adding     accumulated opacity sum_i a_i prod_{j<i}(1 - a_j)
  Eq. map_loss        L1 colour and depth losses                        [Sec. 3.2]
  Eq. track_loss      L1 colour loss over sampled pixels                [Sec. 3.3]
  Eq. pose_grad       gradient w.r.t. the camera pose P                 [Sec. 3.3]
  Eq. add_method / Eq. delete_method / Eq. init-rep                     [Sec. 3.2]
  Eq. coarse2fine     reliable-Gaussian selection                      [Sec. 3.3]

Readings where the paper is silent (inherited rasteriser conventions), fixed as
constants of the definition: alpha = min(0.99, o * exp(-q/2)); a Gaussian with
q > 9 (outside 3 sigma) or alpha < 1/255 is skipped; the Gaussian whose blend
would take T below 1e-4 is not blended and ends the pixel; a low-pass 0.3 px^2
is added to Sigma'; the x/z and y/z used in J are clamped to 1.3 tan(fov/2);
Gaussians with camera depth z <= z_near (0.2 m) are dropped; pixel (u, v) has
its centre at (u + 0.5, v + 0.5); colour is max(0, SH(dir) + 0.5); opacity is
sigmoid(Lambda); scale is exp(log_scale).
"""
from __future__ import annotations

import math

import numpy as np
import torch

F64 = torch.float64

ALPHA_MAX = 0.99
ALPHA_MIN = 1.0 / 255.0
T_MIN = 1e-4
GATE_Q = 9.0          # 3 sigma: q = d^T Sigma'^-1 d <= 9
LOWPASS = 0.3         # px^2 added to the diagonal of Sigma'
FOV_GUARD = 1.3


# ----------------------------------------------------------------------------
# rotations and covariance (Eq. covariance, supp. Eq. q2R)
# ----------------------------------------------------------------------------

def quat_to_rotmat(q: torch.Tensor) -> torch.Tensor:
    """Rotation matrix of a unit quaternion q = [q_r, q_i, q_j, q_k] (supp. Eq. q2R).
    q: (..., 4) -> (..., 3, 3)."""
    r, i, j, k = q.unbind(-1)
    row0 = torch.stack([0.5 - (j * j + k * k), i * j - r * k, i * k + r * j], -1)
    row1 = torch.stack([i * j + r * k, 0.5 - (i * i + k * k), j * k - r * i], -1)
    row2 = torch.stack([i * k - r * j, j * k + r * i, 0.5 - (i * i + j * j)], -1)
    return 2.0 * torch.stack([row0, row1, row2], -2)


def covariance_3d(log_scale: torch.Tensor, quat: torch.Tensor) -> torch.Tensor:
    """Sigma = R S S^T R^T with S = diag(exp(log_scale)) and R = R(q / |q|) (Eq. covariance).
    log_scale: (N, 3), quat: (N, 4) -> (N, 3, 3)."""
    qn = quat / torch.linalg.norm(quat, dim=-1, keepdim=True)
    R = quat_to_rotmat(qn)
    S = torch.diag_embed(torch.exp(log_scale))
    M = R @ S
    return M @ M.transpose(-1, -2)


def hat(w: torch.Tensor) -> torch.Tensor:
    """Skew-symmetric matrix [w]_x with [w]_x v = w x v."""
    z = torch.zeros((), dtype=w.dtype)
    return torch.stack([torch.stack([z, -w[2], w[1]]),
                        torch.stack([w[2], z, -w[0]]),
                        torch.stack([-w[1], w[0], z])])


def se3_exp(xi: torch.Tensor) -> torch.Tensor:
    """4x4 exponential of a twist xi = (rho, phi) (Rodrigues form, float64)."""
    rho, phi = xi[:3], xi[3:]
    th = torch.linalg.norm(phi)
    K = hat(phi)
    I = torch.eye(3, dtype=xi.dtype)
    if float(th) < 1e-12:
        R = I + K
        V = I + 0.5 * K
    else:
        a = torch.sin(th) / th
        b = (1 - torch.cos(th)) / th ** 2
        c = (th - torch.sin(th)) / th ** 3
        R = I + a * K + b * (K @ K)
        V = I + b * K + c * (K @ K)
    T = torch.eye(4, dtype=xi.dtype)
    T = torch.cat([torch.cat([R, (V @ rho)[:, None]], 1), T[3:]], 0)
    return T


# ----------------------------------------------------------------------------
# real spherical harmonics (colour c_i from the coefficients Y_i, Eq. scene-rep)
# ----------------------------------------------------------------------------

def sh_basis(degree: int, d: torch.Tensor) -> torch.Tensor:
    """Real SH basis up to `degree` at unit directions d (N, 3) -> (N, (degree+1)^2),
    coefficient k = l^2 + l + m.

    Convention: the real harmonics built from the associated Legendre functions
    WITH the Condon-Shortley phase (the basis of the 3DGS rasteriser the paper
    extends), i.e. (-1)^|m| times the textbook real harmonics:
        m = 0 : K_l^0 P_l(z)
        m > 0 : (-1)^m sqrt(2) K_l^m Re((x + i y)^m) d^m P_l/dz^m (z)
        m < 0 : (-1)^m sqrt(2) K_l^|m| Im((x + i y)^|m|) d^|m| P_l/dz^|m| (z)
    with K_l^m = sqrt((2l + 1)/(4 pi) (l - m)!/(l + m)!)."""
    x, y, z = d[:, 0], d[:, 1], d[:, 2]
    cols = []
    for l in range(degree + 1):
        Pl = np.polynomial.legendre.Legendre.basis(l).convert(kind=np.polynomial.Polynomial)
        for m in range(-l, l + 1):
            am = abs(m)
            dP = Pl.deriv(am) if am > 0 else Pl
            val = torch.zeros_like(z)
            for p, c in enumerate(dP.coef):
                val = val + float(c) * z ** p
            re, im = torch.ones_like(x), torch.zeros_like(x)
            for _ in range(am):
                re, im = re * x - im * y, re * y + im * x
            K = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
            cs = -1.0 if am % 2 else 1.0
            if m == 0:
                Y = K * val
            elif m > 0:
                Y = cs * math.sqrt(2.0) * K * re * val
            else:
                Y = cs * math.sqrt(2.0) * K * im * val
            cols.append(Y)
    return torch.stack(cols, -1)


# ----------------------------------------------------------------------------
# parameters
# ----------------------------------------------------------------------------

PARAM_KEYS = ("mean", "log_scale", "quat", "opacity_logit", "sh")


def to_params(scene: dict, requires_grad: bool = False) -> dict:
    """float32 SoA planes -> float64 leaf tensors, row per Gaussian:
    mean (N,3), log_scale (N,3), quat (N,4), opacity_logit (N,), sh (N,K,3)."""
    n = scene["mean"].shape[1]
    deg = int(scene["sh_degree"])
    K = (deg + 1) ** 2
    # float32 inputs widen exactly; float64 inputs (finite differences) pass through
    f64 = lambda k: np.asarray(scene[k]).astype(np.float64)  # noqa: E731
    p = {
        "mean": torch.tensor(f64("mean").T.copy()),
        "log_scale": torch.tensor(f64("log_scale").T.copy()),
        "quat": torch.tensor(f64("quat").T.copy()),
        "opacity_logit": torch.tensor(f64("opacity_logit")),
        "sh": torch.tensor(f64("sh").reshape(K, 3, n).transpose(2, 0, 1).copy()),
    }
    for t in p.values():
        t.requires_grad_(requires_grad)
    p["sh_degree"] = deg
    p["n"] = n
    return p


def grads_to_planes(p: dict) -> dict:
    """Leaf gradients back to the SoA plane layout of the inputs (float64 numpy)."""
    out = {}
    for k in PARAM_KEYS:
        g = p[k].grad
        g = torch.zeros_like(p[k]) if g is None else g
        g = g.detach().numpy()
        if k in ("mean", "log_scale", "quat"):
            out[k] = g.T.copy()
        elif k == "opacity_logit":
            out[k] = g.copy()
        else:
            n, K, _ = g.shape
            out[k] = g.transpose(1, 2, 0).reshape(K * 3, n).copy()
    return out


def pose_tensors(view: dict):
    T = torch.tensor(np.asarray(view["T_cw"], np.float32).astype(np.float64)).reshape(3, 4)
    return T[:, :3], T[:, 3]


# ----------------------------------------------------------------------------
# projection (Eq. covariance2d, mean projection m = K P X / d, SH colour)
# ----------------------------------------------------------------------------

def project(p: dict, view: dict, twist: torch.Tensor | None = None, pose_mode: str = "exact",
            gaussian_mask=None, lowpass: float = LOWPASS, fov_guard: float | None = FOV_GUARD,
            pose=None, pose_cov=None) -> dict:
    """Project every Gaussian of parameter set `p` into `view`.

    The pose is W = [R | t] (world -> camera).  With `twist` = (rho, phi) the pose
    is the left perturbation exp(twist^) W; only the derivative at twist = 0 is
    used, for which (I + twist^) W is exact to first order.  pose_mode "paper"
    keeps the twist out of Sigma' and of the view direction of the colour, the
    approximation of Eq. pose_grad (the dSigma'/dP and dc/dP terms dropped).

    Returns the kept Gaussians (z > z_near, det(Sigma') > 0, mask) in index
    order: index, mu (M,2), conic (M,3) = (A, B, C) of [[A,B],[B,C]] = Sigma'^-1,
    cov2d (M,3), depth (M,) the camera z, depth32 (float32 z, the sort key),
    opacity (M,), rgb (M,3), radius (M,), cond (M,) = lambda_max/lambda_min.

    `pose` = (R, t) float64 tensors overrides the view's float32 T_cw (it may carry
    autograd history, e.g. R built from a quaternion).  `pose_cov` = (R, t), when
    given, is the pose used for Sigma' and the colour's view direction instead
    (the restricted function whose exact derivative is the "paper" mode)."""
    R0, t0 = pose_tensors(view) if pose is None else pose
    if twist is None:
        R, t = R0, t0
    else:
        G = torch.eye(3, dtype=F64) + hat(twist[3:])
        R, t = G @ R0, G @ t0 + twist[:3]
    X_all = p["mean"]
    with torch.no_grad():
        z_all = (X_all @ R0.detach().T + t0.detach())[:, 2].numpy()
    z32 = z_all.astype(np.float32)
    keep = z32 > np.float32(view["z_near"])
    if gaussian_mask is not None:
        keep &= np.asarray(gaussian_mask).astype(bool)
    idx = torch.tensor(np.nonzero(keep)[0], dtype=torch.long)

    X = X_all[idx]
    Xc = X @ R.T + t
    x, y, z = Xc.unbind(-1)
    fx, fy, cx, cy = (float(view[k]) for k in ("fx", "fy", "cx", "cy"))
    W_img, H_img = int(view["width"]), int(view["height"])
    mu = torch.stack([fx * x / z + cx, fy * y / z + cy], -1)

    if pose_cov is not None:
        Rq, tq = pose_cov
        R_cov, Xc_cov, cam = Rq, X @ Rq.T + tq, -(Rq.T @ tq)
    elif pose_mode == "paper":
        R_cov, Xc_cov, cam = R0, X @ R0.T + t0, -(R0.T @ t0)
    elif pose_mode == "exact":
        R_cov, Xc_cov, cam = R, Xc, -(R.T @ t)
    else:
        raise ValueError(pose_mode)
    xc, yc, zc = Xc_cov.unbind(-1)
    if fov_guard is None:
        tx, ty = xc, yc
    else:
        limx = fov_guard * W_img / (2.0 * fx)
        limy = fov_guard * H_img / (2.0 * fy)
        tx = zc * torch.clamp(xc / zc, -limx, limx)
        ty = zc * torch.clamp(yc / zc, -limy, limy)
    zero = torch.zeros_like(zc)
    J = torch.stack([torch.stack([fx / zc, zero, -fx * tx / zc ** 2], -1),
                     torch.stack([zero, fy / zc, -fy * ty / zc ** 2], -1)], -2)
    Sigma = covariance_3d(p["log_scale"][idx], p["quat"][idx])
    Sc = R_cov @ Sigma @ R_cov.T
    cov = J @ Sc @ J.transpose(-1, -2)
    a = cov[:, 0, 0] + lowpass
    b = cov[:, 0, 1]
    c = cov[:, 1, 1] + lowpass
    det = a * c - b * b
    conic = torch.stack([c / det, -b / det, a / det], -1)
    with torch.no_grad():
        mid = 0.5 * (a + c)
        disc = torch.sqrt(torch.clamp(mid * mid - det, min=0.1))
        lam_max = mid + disc
        lam_min = torch.clamp(mid - torch.sqrt(torch.clamp(mid * mid - det, min=0.0)), min=1e-30)
        radius = torch.ceil(3.0 * torch.sqrt(lam_max))
        cond = lam_max / lam_min
    opacity = torch.sigmoid(p["opacity_logit"][idx])
    dirs = X - cam
    dirs = dirs / torch.linalg.norm(dirs, dim=-1, keepdim=True)
    Y = sh_basis(p["sh_degree"], dirs)
    rgb = torch.clamp((Y[:, :, None] * p["sh"][idx]).sum(1) + 0.5, min=0.0)

    good = (det > 0).detach().numpy()
    if not good.all():
        sel = torch.tensor(np.nonzero(good)[0], dtype=torch.long)
        idx, mu, conic, z, opacity, rgb = idx[sel], mu[sel], conic[sel], z[sel], opacity[sel], rgb[sel]
        radius, cond = radius[sel], cond[sel]
        a, b, c = a[sel], b[sel], c[sel]
        z32 = z32  # indexed below through idx
    return dict(index=idx, mu=mu, conic=conic, cov2d=torch.stack([a, b, c], -1), depth=z,
                depth32=z32[idx.numpy()], opacity=opacity, rgb=rgb, radius=radius, cond=cond)


DIFF_KEYS = ("mu", "conic", "depth", "opacity", "rgb")


def depth_order(proj: dict) -> np.ndarray:
    """Blend order: ascending (float32 camera depth, Gaussian index)."""
    return np.argsort(proj["depth32"], kind="stable")


# ----------------------------------------------------------------------------
# compositing (Eq. color_render, Eq. depth, accumulated opacity)
# ----------------------------------------------------------------------------

def composite(proj: dict, view: dict, pix_u: np.ndarray, pix_v: np.ndarray, order=None) -> dict:
    """Front-to-back alpha blending of every listed pixel over all projected
    Gaussians in depth order (brute force).

    Per pixel p (centre (u+0.5, v+0.5)), in order: q = d^T conic d with d = p - mu;
    skip if q > 9; alpha = min(0.99, o exp(-q/2)); skip if alpha < 1/255; if
    T (1 - alpha) < 1e-4 stop without blending; else C += c alpha T, D += d alpha T,
    T *= 1 - alpha.  Output C + T bg, D, A = 1 - T, T.

    Written as the closed form of Eq. color_render: with alpha set to 0 for skipped
    and post-stop Gaussians, T_i = prod_{j<i} (1 - alpha_j) and the weights are
    alpha_i T_i.  The stop rule keeps exactly the Gaussians whose inclusive product
    is still >= 1e-4 (a prefix, since the product never increases).

    Also returns, per pixel, the distance of each threshold decision from its
    threshold (used to set aside pixels whose decisions a float32 evaluation may
    take the other way):
      m_gate  = min |q - 9| / (9 (1 + cond))           over tested Gaussians
      m_alpha = min |alpha - 1/255| 255 / (1 + cond)   over tested in-gate Gaussians
      m_stop  = min |T(1 - alpha) - 1e-4| / 1e-4       over tested blend candidates
      m_clamp = min |o exp(-q/2) - 0.99| / (1 + cond)  over blended Gaussians
    ("tested" = up to and including the Gaussian that stops the pixel)."""
    if order is None:
        order = depth_order(proj)
    o = torch.tensor(order, dtype=torch.long)
    mu = proj["mu"][o]
    con = proj["conic"][o]
    dep = proj["depth"][o]
    opa = proj["opacity"][o]
    rgb = proj["rgb"][o]
    cond = proj["cond"][o].detach()
    n = mu.shape[0]
    P = len(pix_u)
    bg = torch.tensor(np.asarray(view["bg"], np.float32).astype(np.float64))
    if n == 0:
        z = torch.zeros(P, dtype=F64)
        return dict(color=bg.expand(P, 3).clone(), depth=z, acc=z, T=torch.ones(P, dtype=F64),
                    n_contrib=np.zeros(P, np.int64),
                    m_gate=np.full(P, np.inf), m_alpha=np.full(P, np.inf),
                    m_stop=np.full(P, np.inf), m_clamp=np.full(P, np.inf))
    px = torch.tensor(np.asarray(pix_u, np.float64) + 0.5)[:, None]
    py = torch.tensor(np.asarray(pix_v, np.float64) + 0.5)[:, None]
    dx = px - mu[None, :, 0]
    dy = py - mu[None, :, 1]
    q = con[None, :, 0] * dx * dx + 2.0 * con[None, :, 1] * dx * dy + con[None, :, 2] * dy * dy
    araw = opa[None, :] * torch.exp(-0.5 * q)
    alpha = torch.clamp(araw, max=ALPHA_MAX)
    with torch.no_grad():
        in_gate = q <= GATE_Q
        cand = in_gate & (alpha >= ALPHA_MIN)
        c_incl = torch.cumprod(torch.where(cand, 1.0 - alpha, torch.ones_like(alpha)), dim=1)
        keep = cand & (c_incl >= T_MIN)
        stops = cand & (c_incl < T_MIN)
        has_stop = stops.any(1)
        first_stop = torch.where(has_stop, stops.int().argmax(1), torch.full((P,), n, dtype=torch.long))
        tested = torch.arange(n)[None, :] <= first_stop[:, None]
        inf = torch.tensor(float("inf"), dtype=F64)
        m_gate = torch.where(tested, (q - GATE_Q).abs() / (GATE_Q * (1 + cond[None])), inf).amin(1)
        m_alpha = torch.where(tested & in_gate, (alpha - ALPHA_MIN).abs() / ALPHA_MIN / (1 + cond[None]),
                              inf).amin(1)
        m_stop = torch.where(tested & cand, (c_incl - T_MIN).abs() / T_MIN, inf).amin(1)
        m_clamp = torch.where(keep, (araw - ALPHA_MAX).abs() / (1 + cond[None]), inf).amin(1)
    a_k = torch.where(keep, alpha, torch.zeros_like(alpha))
    one_m = 1.0 - a_k
    T_incl = torch.cumprod(one_m, dim=1)
    T_before = torch.cat([torch.ones(P, 1, dtype=F64), T_incl[:, :-1]], 1)
    w = a_k * T_before
    T_final = T_incl[:, -1]
    color = w @ rgb + T_final[:, None] * bg[None, :]
    depth = w @ dep
    return dict(color=color, depth=depth, acc=1.0 - T_final, T=T_final,
                n_contrib=keep.sum(1).numpy(),
                m_gate=m_gate.numpy(), m_alpha=m_alpha.numpy(), m_stop=m_stop.numpy(),
                m_clamp=m_clamp.numpy())


def pixel_alternatives(proj: dict, view: dict, u: int, v: int, tol_gate: float = 1e-6, tol_alpha: float = 1e-5,
                       tol_stop: float = 1e-4, max_near: int = 3, order=None):
    """Every output the definition allows at pixel (u, v) when each threshold
    decision that lies within float32 reach of its threshold may go either way.

    A plain front-to-back walk of the pixel's depth-ordered Gaussians in float64
    (Eq. color_render, Eq. depth, accumulated opacity): q = d^T conic d, skip if
    q > 9, alpha = min(0.99, o exp(-q/2)), skip if alpha < 1/255, stop without
    blending if T (1 - alpha) < 1e-4, else blend and T *= 1 - alpha.  A decision
    whose relative margin (the measures of composite(): |q - 9| / (9 (1 + cond)),
    |alpha - 1/255| 255 / (1 + cond), |T (1 - alpha) - 1e-4| / 1e-4) is at most its
    tolerance is taken both ways, one branch of the walk for each.

    Returns a list of dict(color (3,), depth, acc), one per combination of the near
    decisions met along the way (a single entry when none is near), or None when a
    branch meets more than max_near near decisions."""
    if order is None:
        order = depth_order(proj)
    o = np.asarray(order, np.int64)
    mu = proj["mu"].detach().numpy()[o]
    con = proj["conic"].detach().numpy()[o]
    opa = proj["opacity"].detach().numpy()[o]
    rgb = proj["rgb"].detach().numpy()[o]
    dep = proj["depth"].detach().numpy()[o]
    cond = proj["cond"].detach().numpy()[o]
    bg = np.asarray(view["bg"], np.float32).astype(np.float64)
    dx = (u + 0.5) - mu[:, 0]
    dy = (v + 0.5) - mu[:, 1]
    q = con[:, 0] * dx * dx + 2.0 * con[:, 1] * dx * dy + con[:, 2] * dy * dy
    alpha = np.minimum(ALPHA_MAX, opa * np.exp(-0.5 * q))
    in_gate = q <= GATE_Q
    near_gate = np.abs(q - GATE_Q) / (GATE_Q * (1 + cond)) <= tol_gate
    cand_a = alpha >= ALPHA_MIN
    near_a = np.abs(alpha - ALPHA_MIN) / ALPHA_MIN / (1 + cond) <= tol_alpha
    # Gaussians that blend in no branch (clearly outside the gate or below 1/255) are
    # skipped in every branch; the walk visits the rest in order
    rel = np.nonzero((in_gate | near_gate) & (cand_a | near_a))[0]
    outs = []
    overflow = [False]

    def walk(k, T, C, D, n_near):
        while k < len(rel):
            j = rel[k]
            k += 1
            g_opts = (True, False) if near_gate[j] else (bool(in_gate[j]),)
            a_opts = (True, False) if near_a[j] else (bool(cand_a[j]),)
            cands = {ga and aa for ga in g_opts for aa in a_opts}
            if len(cands) == 2:
                if n_near + 1 > max_near:
                    overflow[0] = True
                    return
                n_near += 1
                walk(k, T, C, D, n_near)  # the branch that skips this Gaussian
            elif not cands.pop():
                continue
            c = T * (1.0 - alpha[j])
            stop = c < T_MIN
            if abs(c - T_MIN) / T_MIN <= tol_stop:
                if n_near + 1 > max_near:
                    overflow[0] = True
                    return
                n_near += 1
                outs.append(dict(color=C + T * bg, depth=D, acc=1.0 - T))  # the branch that stops here
                stop = False
            if stop:
                break
            C = C + rgb[j] * alpha[j] * T
            D = D + dep[j] * alpha[j] * T
            T = c
        outs.append(dict(color=C + T * bg, depth=D, acc=1.0 - T))

    walk(0, 1.0, np.zeros(3), 0.0, 0)
    return None if overflow[0] else outs


def _pixel_chunks(view, pixel_mask, chunk_elems, n_gauss):
    W, H = int(view["width"]), int(view["height"])
    if pixel_mask is None:
        lin = np.arange(W * H)
    else:
        lin = np.nonzero(np.asarray(pixel_mask).reshape(-1))[0]
    step = max(1, chunk_elems // max(1, n_gauss))
    for s in range(0, len(lin), step):
        sl = lin[s:s + step]
        yield sl, sl % W, sl // W


def render_view(scene: dict, view: dict, pixel_mask=None, gaussian_mask=None,
                chunk_elems: int = 1 << 22, lowpass=LOWPASS, fov_guard=FOV_GUARD) -> dict:
    """Forward render of one view: colour [3][H][W], depth [H][W], acc [H][W],
    T [H][W], n_contrib [H][W] and the per-pixel threshold margins.  Pixels outside
    `pixel_mask` are not rendered and hold 0 (T holds 1)."""
    with torch.no_grad():
        p = to_params(scene)
        proj = project(p, view, gaussian_mask=gaussian_mask, lowpass=lowpass, fov_guard=fov_guard)
        order = depth_order(proj)
        W, H = int(view["width"]), int(view["height"])
        out = dict(color=np.zeros((3, H * W)), depth=np.zeros(H * W), acc=np.zeros(H * W),
                   T=np.ones(H * W), n_contrib=np.zeros(H * W, np.int64))
        for k in ("m_gate", "m_alpha", "m_stop", "m_clamp"):
            out[k] = np.full(H * W, np.inf)
        for lin, u, v in _pixel_chunks(view, pixel_mask, chunk_elems, len(order)):
            r = composite(proj, view, u, v, order)
            out["color"][:, lin] = r["color"].numpy().T
            out["depth"][lin] = r["depth"].numpy()
            out["acc"][lin] = r["acc"].numpy()
            out["T"][lin] = r["T"].numpy()
            out["n_contrib"][lin] = r["n_contrib"]
            for k in ("m_gate", "m_alpha", "m_stop", "m_clamp"):
                out[k][lin] = r[k]
    out["color"] = out["color"].reshape(3, H, W)
    for k in ("depth", "acc", "T", "n_contrib", "m_gate", "m_alpha", "m_stop", "m_clamp"):
        out[k] = out[k].reshape(H, W)
    out["proj"] = proj
    return out


# ----------------------------------------------------------------------------
# loss (Eq. map_loss / Eq. track_loss) and gradients (Eq. pose_grad)
# ----------------------------------------------------------------------------

def l1_loss(color, depth, t_rgb, t_depth, w_c, w_d):
    """w_c sum |C - C_obs| + w_d sum_{D_obs > 0} |D - D_obs| over the given pixels.
    color (P,3), depth (P,), t_rgb (P,3), t_depth (P,)."""
    lc = (color - t_rgb).abs().sum()
    valid = (t_depth > 0).to(F64)
    ld = ((depth - t_depth).abs() * valid).sum()
    return w_c * lc + w_d * ld


def render_and_grad(scenes, views, targets, w_c=1.0, w_d=0.5, pixel_masks=None, pose_mode="exact",
                    gaussian_masks=None, chunk_elems: int = 1 << 21, want_2d=False):
    """Loss summed over views and its gradient w.r.t. every Gaussian parameter of
    every scene and the left-perturbation twist (rho, phi) of every view.

    views[v]["scene"] (default 0) picks the scene; gradients of a scene seen by
    several views accumulate.  Returns dict(loss, per_view_loss, images, grads
    (list of SoA-plane dicts), twist (V,6) and, with want_2d, the per-view
    gradients w.r.t. the projected quantities keyed by Gaussian index)."""
    params = [to_params(s, requires_grad=True) for s in scenes]
    V = len(views)
    twist = torch.zeros(V, 6, dtype=F64, requires_grad=True)
    per_view, images, g2d = [], [], []
    for v, view in enumerate(views):
        s = int(view.get("scene", 0))
        gm = None if gaussian_masks is None else gaussian_masks[v]
        proj = project(params[s], view, twist=twist[v], pose_mode=pose_mode, gaussian_mask=gm)
        order = depth_order(proj)
        leaves = {k: proj[k].detach().clone().requires_grad_(True) for k in DIFF_KEYS}
        lv = dict(proj)
        lv.update(leaves)
        W, H = int(view["width"]), int(view["height"])
        t_rgb = np.asarray(targets[v][0], np.float32).reshape(3, -1)
        t_dep = np.asarray(targets[v][1], np.float32).reshape(-1)
        pm = None if pixel_masks is None else pixel_masks[v]
        img = dict(color=np.zeros((3, H * W)), depth=np.zeros(H * W), acc=np.zeros(H * W))
        loss_v = 0.0
        for lin, u, vv in _pixel_chunks(view, pm, chunk_elems, len(order)):
            r = composite(lv, view, u, vv, order)
            L = l1_loss(r["color"], r["depth"],
                        torch.tensor(t_rgb[:, lin].T.astype(np.float64)),
                        torch.tensor(t_dep[lin].astype(np.float64)), w_c, w_d)
            L.backward()
            loss_v += float(L.detach())
            img["color"][:, lin] = r["color"].detach().numpy().T
            img["depth"][lin] = r["depth"].detach().numpy()
            img["acc"][lin] = r["acc"].detach().numpy()
        outs, gts = [], []
        for k in DIFF_KEYS:
            if leaves[k].grad is not None:
                outs.append(proj[k])
                gts.append(leaves[k].grad)
        if outs:
            torch.autograd.backward(outs, gts)
        per_view.append(loss_v)
        images.append(dict(color=img["color"].reshape(3, H, W), depth=img["depth"].reshape(H, W),
                           acc=img["acc"].reshape(H, W)))
        if want_2d:
            g2d.append({"index": proj["index"].numpy(),
                        **{k: (leaves[k].grad.numpy() if leaves[k].grad is not None
                               else np.zeros(tuple(leaves[k].shape))) for k in DIFF_KEYS}})
    grads = [grads_to_planes(p) for p in params]
    tw = twist.grad.numpy().copy() if twist.grad is not None else np.zeros((V, 6))
    return dict(loss=float(sum(per_view)), per_view_loss=per_view, images=images, grads=grads,
                twist=tw, grads_2d=g2d)


def loss_only(scenes, views, targets, w_c=1.0, w_d=0.5, pixel_masks=None, twists=None,
              gaussian_masks=None, chunk_elems: int = 1 << 22, lowpass=LOWPASS, fov_guard=FOV_GUARD,
              pose_mode="exact"):
    """The loss alone (no autograd).  With `twists` (V,6) each view's pose is first
    replaced by exp(twist^) W using the exact matrix exponential (for finite
    differences of the pose).  pose_mode "paper" applies the twist to the mean
    projection only (Sigma' and the colour keep the unperturbed pose)."""
    total = 0.0
    with torch.no_grad():
        ps = [to_params(s) for s in scenes]
        for v, view in enumerate(views):
            vw = dict(view)
            if twists is not None:
                T = torch.eye(4, dtype=F64)
                T[:3, :] = torch.tensor(np.asarray(view["T_cw"], np.float32).astype(np.float64)).reshape(3, 4)
                Tn = se3_exp(torch.as_tensor(np.asarray(twists[v], np.float64))) @ T
                pose = (Tn[:3, :3], Tn[:3, 3])
            else:
                pose = None
            s = int(view.get("scene", 0))
            gm = None if gaussian_masks is None else gaussian_masks[v]
            # the perturbed pose stays in float64: finite differences need it
            pose_cov = pose_tensors(view) if (pose_mode == "paper" and pose is not None) else None
            proj = project(ps[s], vw, gaussian_mask=gm, lowpass=lowpass, fov_guard=fov_guard, pose=pose,
                           pose_cov=pose_cov)
            order = depth_order(proj)
            t_rgb = np.asarray(targets[v][0], np.float32).reshape(3, -1)
            t_dep = np.asarray(targets[v][1], np.float32).reshape(-1)
            pm = None if pixel_masks is None else pixel_masks[v]
            for lin, u, vv in _pixel_chunks(view, pm, chunk_elems, len(order)):
                r = composite(proj, vw, u, vv, order)
                total += float(l1_loss(r["color"], r["depth"],
                                       torch.tensor(t_rgb[:, lin].T.astype(np.float64)),
                                       torch.tensor(t_dep[lin].astype(np.float64)), w_c, w_d))
    return total


# ----------------------------------------------------------------------------
# tile binning (the per-tile depth-sorted lists the tiled renderer builds)
# ----------------------------------------------------------------------------

def tile_rects(mu_x, mu_y, ext_x, ext_y, width, height, tile_w, tile_h):
    """Tile rectangle of each Gaussian's footprint box, decided in float32.

    The box covers pixel centres u + 0.5 in [mu - e, mu + e] (e = the half-extent
    of the footprint along that axis):
      u_min = ceil(mu - (e + 0.5)), u_max = floor((mu + e) - 0.5), clipped to the
      image; tiles floor(u / tile_w).  Returns (tx0, tx1, ty0, ty1) inclusive, with
      tx0 > tx1 (or ty0 > ty1) meaning no tile."""
    mx = np.asarray(mu_x, np.float32)
    my = np.asarray(mu_y, np.float32)
    ex = np.asarray(ext_x, np.float32)
    ey = np.asarray(ext_y, np.float32)
    half = np.float32(0.5)
    umin = np.ceil(mx - (ex + half)).astype(np.float64)
    umax = np.floor((mx + ex) - half).astype(np.float64)
    vmin = np.ceil(my - (ey + half)).astype(np.float64)
    vmax = np.floor((my + ey) - half).astype(np.float64)
    umin = np.clip(umin, 0, width)
    umax = np.clip(umax, -1, width - 1)
    vmin = np.clip(vmin, 0, height)
    vmax = np.clip(vmax, -1, height - 1)
    tx0 = np.floor_divide(umin, tile_w).astype(np.int64)
    tx1 = np.where(umax >= umin, np.floor_divide(umax, tile_w), -1).astype(np.int64)
    ty0 = np.floor_divide(vmin, tile_h).astype(np.int64)
    ty1 = np.where(vmax >= vmin, np.floor_divide(vmax, tile_h), -1).astype(np.int64)
    return tx0, tx1, ty0, ty1


def tile_lists(mu_x, mu_y, ext_x, ext_y, depth_bits, valid, width, height, tile_w, tile_h):
    """For every tile (row-major), the Gaussian indices whose footprint box covers a
    pixel centre of the tile, in ascending (depth bits, index) order."""
    tiles_x = (width + tile_w - 1) // tile_w
    tiles_y = (height + tile_h - 1) // tile_h
    tx0, tx1, ty0, ty1 = tile_rects(mu_x, mu_y, ext_x, ext_y, width, height, tile_w, tile_h)
    lists = [[] for _ in range(tiles_x * tiles_y)]
    ids = np.nonzero(np.asarray(valid).astype(bool))[0]
    keys = np.asarray(depth_bits, np.uint32)
    ids = ids[np.lexsort((ids, keys[ids]))]
    for g in ids:
        for ty in range(ty0[g], ty1[g] + 1):
            for tx in range(tx0[g], tx1[g] + 1):
                lists[ty * tiles_x + tx].append(int(g))
    return lists


def footprint_extents(cov2d, opacity):
    """Half-extents of the alpha >= 1/255 region {q <= min(9, 2 ln(255 o))} along x
    and y: sqrt(qlim Sigma'_00), sqrt(qlim Sigma'_11) (0 where o < 1/255)."""
    cov = np.asarray(cov2d, np.float64)
    o = np.asarray(opacity, np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        qlim = np.minimum(GATE_Q, 2.0 * np.log(255.0 * o))
    qlim = np.where(o >= ALPHA_MIN, qlim, 0.0)
    return np.sqrt(qlim * cov[:, 0]), np.sqrt(qlim * cov[:, 2])


def depth_bits(depth32) -> np.ndarray:
    """The float32 depth as its IEEE bit pattern (orders like the value for z > 0)."""
    return np.asarray(depth32, np.float32).view(np.uint32)
