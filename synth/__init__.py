"""Seeded synthetic inputs for the RGB-D Gaussian splatting hot path.

This module only draws inputs: Gaussian parameter sets, camera views, target
images and masks.  It holds none of the renderer's arithmetic and is shared by
the tests, the benchmark and the smoke check.  Both the CUDA path and the FP64
oracle consume what it returns; neither is imported here.

Layouts (float32, component-major "SoA planes", the layout of the C ABI):

  scene["mean"]           [3][N]      world position X (GS-SLAM Eq. scene-rep)
  scene["log_scale"]      [3][N]      log of the scale vector S (Eq. covariance)
  scene["quat"]           [4][N]      rotation quaternion (r, i, j, k), not normalised
  scene["opacity_logit"]  [N]         opacity before the sigmoid
  scene["sh"]             [3K][N]     SH coefficients, plane k*3 + c (K = (deg+1)^2)
  scene["sh_degree"]      int

  view = dict(width, height, fx, fy, cx, cy, z_near, bg[3], T_cw[12])
  T_cw is row-major [R | t], world -> camera, camera looks along +z, y down.

The paper measures on Replica and TUM-RGBD, which are not available here.  The
generators below stand in for them with the shapes of those workloads: rooms of
planes and boxes seen from inside at 1200x680, TUM-like 640x480 views, and the
small frustum scene used for parity.
"""
from __future__ import annotations

import math

import numpy as np

SH_C0 = 0.28209479177387814  # Y_00 = 1 / (2 sqrt(pi)), used only to store a DC colour


def sh_count(degree: int) -> int:
    return (degree + 1) ** 2


# ----------------------------------------------------------------------------
# small host-side geometry used only to place cameras and draw poses
# ----------------------------------------------------------------------------

def _hat(w):
    return np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])


def se3_exp(xi):
    """4x4 matrix exponential of a twist xi = (rho, phi) (float64), for drawing poses."""
    xi = np.asarray(xi, dtype=np.float64)
    rho, phi = xi[:3], xi[3:]
    th = float(np.linalg.norm(phi))
    K = _hat(phi)
    if th < 1e-12:
        R = np.eye(3) + K
        V = np.eye(3) + 0.5 * K
    else:
        a = math.sin(th) / th
        b = (1.0 - math.cos(th)) / th**2
        c = (th - math.sin(th)) / th**3
        R = np.eye(3) + a * K + b * K @ K
        V = np.eye(3) + b * K + c * K @ K
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = V @ rho
    return T


def look_at(eye, target, up=(0.0, 0.0, 1.0)):
    """World->camera [R|t] (3x4, float64) for a camera at `eye` looking at `target`.
    Camera axes: +z forward, +x right, +y down (pinhole convention)."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, np.float64))
    if np.linalg.norm(r) < 1e-9:
        r = np.cross(f, np.array([0.0, 1.0, 0.0]))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)  # down
    R_wc = np.stack([r, d, f], axis=1)
    R_cw = R_wc.T
    t_cw = -R_cw @ eye
    return np.concatenate([R_cw, t_cw[:, None]], axis=1)


def make_view(width, height, fx, fy, cx, cy, T_cw, bg=(0.0, 0.0, 0.0), z_near=0.2):
    T = np.asarray(T_cw, np.float64).reshape(3, 4)
    return dict(width=int(width), height=int(height), fx=float(fx), fy=float(fy),
                cx=float(cx), cy=float(cy), z_near=float(z_near),
                bg=np.asarray(bg, np.float32).copy(),
                T_cw=T.reshape(12).astype(np.float32))


def perturb_view(view, xi):
    """Left-multiply the view's pose by exp(xi^) (a pose hypothesis)."""
    T = np.eye(4)
    T[:3, :] = np.asarray(view["T_cw"], np.float64).reshape(3, 4)
    Tn = se3_exp(xi) @ T
    v = dict(view)
    v["T_cw"] = Tn[:3, :].reshape(12).astype(np.float32)
    v["bg"] = np.asarray(view["bg"], np.float32).copy()
    return v


def scale_view(view, factor):
    """The same camera at a resolution scaled by `factor` (intrinsics scaled)."""
    v = dict(view)
    v["width"] = int(round(view["width"] * factor))
    v["height"] = int(round(view["height"] * factor))
    for k in ("fx", "fy", "cx", "cy"):
        v[k] = float(view[k] * factor)
    v["bg"] = np.asarray(view["bg"], np.float32).copy()
    v["T_cw"] = np.asarray(view["T_cw"], np.float32).copy()
    return v


# ----------------------------------------------------------------------------
# Gaussian attribute draws shared by the scene generators
# ----------------------------------------------------------------------------

def _attributes(rng, n, sh_degree, dc_rgb=None, high_sigma=0.05):
    log_scale = rng.uniform(math.log(0.005), math.log(0.05), size=(3, n))
    q = rng.standard_normal((4, n))
    q /= np.linalg.norm(q, axis=0, keepdims=True)
    opacity_logit = rng.standard_normal(n)
    K = sh_count(sh_degree)
    sh = np.zeros((K * 3, n), np.float64)
    if dc_rgb is None:
        dc_rgb = rng.uniform(0.0, 1.0, size=(3, n))
    sh[0:3] = (dc_rgb - 0.5) / SH_C0
    if K > 1:
        sh[3:] = rng.normal(0.0, high_sigma, size=((K - 1) * 3, n))
    return dict(log_scale=log_scale.astype(np.float32), quat=q.astype(np.float32),
                opacity_logit=opacity_logit.astype(np.float32), sh=sh.astype(np.float32),
                sh_degree=int(sh_degree))


def frustum_scene(seed, n=2000, width=160, height=120, f=120.0, sh_degree=0,
                  zmin=0.5, zmax=4.0):
    """Gaussians uniform in the frustum of an identity-pose pinhole camera
    (the 2,000-Gaussian 160x120 parity workload)."""
    rng = np.random.default_rng(seed)
    cx, cy = width / 2.0, height / 2.0
    u = rng.uniform(0.0, width, n)
    v = rng.uniform(0.0, height, n)
    z = rng.uniform(zmin, zmax, n)
    mean = np.stack([(u - cx) * z / f, (v - cy) * z / f, z])
    s = _attributes(rng, n, sh_degree)
    s["mean"] = mean.astype(np.float32)
    view = make_view(width, height, f, f, cx, cy, np.concatenate([np.eye(3), np.zeros((3, 1))], 1))
    return s, view


def random_targets(seed, width, height, zmin=0.5, zmax=4.0):
    """Uniform random target colour [3][H][W] in [0,1] and depth [H][W] in [zmin,zmax]."""
    rng = np.random.default_rng(seed)
    rgb = rng.uniform(0.0, 1.0, size=(3, height, width)).astype(np.float32)
    depth = rng.uniform(zmin, zmax, size=(height, width)).astype(np.float32)
    return rgb, depth


ROOM = (8.0, 6.0, 3.0)


def _room_quads(rng, n_boxes=20):
    """Planar rectangles (origin, edge a, edge b) of an 8x6x3 m room (z up) with boxes."""
    Lx, Ly, Lz = ROOM
    quads = [
        ((0, 0, 0), (Lx, 0, 0), (0, Ly, 0)),        # floor
        ((0, 0, Lz), (Lx, 0, 0), (0, Ly, 0)),       # ceiling
        ((0, 0, 0), (Lx, 0, 0), (0, 0, Lz)),        # wall y=0
        ((0, Ly, 0), (Lx, 0, 0), (0, 0, Lz)),       # wall y=Ly
        ((0, 0, 0), (0, Ly, 0), (0, 0, Lz)),        # wall x=0
        ((Lx, 0, 0), (0, Ly, 0), (0, 0, Lz)),       # wall x=Lx
    ]
    for _ in range(n_boxes):
        sx, sy, sz = rng.uniform(0.2, 1.5, 3)
        x0 = rng.uniform(0.3, Lx - 0.3 - sx)
        y0 = rng.uniform(0.3, Ly - 0.3 - sy)
        quads += [
            ((x0, y0, sz), (sx, 0, 0), (0, sy, 0)),            # top
            ((x0, y0, 0), (sx, 0, 0), (0, 0, sz)),             # sides
            ((x0, y0 + sy, 0), (sx, 0, 0), (0, 0, sz)),
            ((x0, y0, 0), (0, sy, 0), (0, 0, sz)),
            ((x0 + sx, y0, 0), (0, sy, 0), (0, 0, sz)),
        ]
    return [tuple(np.asarray(p, np.float64) for p in q) for q in quads]


def room_scene(seed, n=300_000, sh_degree=3, jitter=0.01):
    """Replica-shaped room: means area-uniform on the planes and boxes of an 8x6x3 m
    room, jittered N(0, jitter^2); DC colour U[0,1] per surface patch noise, higher
    SH bands N(0, 0.05^2)."""
    rng = np.random.default_rng(seed)
    quads = _room_quads(rng)
    areas = np.array([np.linalg.norm(np.cross(a, b)) for _, a, b in quads])
    idx = rng.choice(len(quads), size=n, p=areas / areas.sum())
    o = np.stack([quads[i][0] for i in range(len(quads))])[idx]
    a = np.stack([quads[i][1] for i in range(len(quads))])[idx]
    b = np.stack([quads[i][2] for i in range(len(quads))])[idx]
    st = rng.uniform(0.0, 1.0, size=(n, 2))
    pts = o + st[:, :1] * a + st[:, 1:] * b + rng.normal(0.0, jitter, size=(n, 3))
    s = _attributes(rng, n, sh_degree)
    s["mean"] = pts.T.astype(np.float32).copy()
    return s


def room_view(width=1200, height=680, f=600.0, eye=(1.2, 3.0, 1.5), target=(8.0, 3.3, 1.3),
              bg=(0.0, 0.0, 0.0)):
    """A camera inside the room at 1.5 m height looking at the x = 8 m wall."""
    return make_view(width, height, f, f, width / 2.0, height / 2.0, look_at(eye, target), bg=bg)


def trajectory_views(seed, n_views=8, width=1200, height=680, f=None):
    """Keyframes on a seeded smooth (sinusoidal) path inside the room, looking at the
    room centre with a little noise."""
    rng = np.random.default_rng(seed)
    f = f if f is not None else width / 2.0
    Lx, Ly, _ = ROOM
    ph = rng.uniform(0, 2 * math.pi, 3)
    views = []
    for k in range(n_views):
        t = 2 * math.pi * k / n_views
        eye = (Lx / 2 + 2.2 * math.sin(t + ph[0]), Ly / 2 + 1.6 * math.cos(0.7 * t + ph[1]),
               1.5 + 0.25 * math.sin(2 * t + ph[2]))
        tgt = np.array([Lx / 2, Ly / 2, 1.2]) + rng.normal(0.0, 0.3, 3)
        # look away from the centre half of the time so walls fill the view
        if k % 2 == 1:
            tgt = 2 * np.asarray(eye) - tgt
            tgt[2] = 1.2
        views.append(make_view(width, height, f, f, width / 2.0, height / 2.0, look_at(eye, tgt)))
    return views


def zbuffer_targets(scene, view, seed, jitter=0.005, splat=1):
    """Cheap target images of a seeded perturbation of `scene` (numpy point z-buffer,
    (2*splat+1)^2 pixels per point, DC colour).  Pixels no point reaches get depth 0
    (no sensor reading) and colour = background."""
    rng = np.random.default_rng(seed)
    W, H = view["width"], view["height"]
    T = np.asarray(view["T_cw"], np.float64).reshape(3, 4)
    X = scene["mean"].astype(np.float64).T + rng.normal(0.0, jitter, size=(scene["mean"].shape[1], 3))
    Xc = X @ T[:, :3].T + T[:, 3]
    z = Xc[:, 2]
    keep = z > view["z_near"]
    u = np.floor(view["fx"] * Xc[keep, 0] / z[keep] + view["cx"]).astype(np.int64)
    v = np.floor(view["fy"] * Xc[keep, 1] / z[keep] + view["cy"]).astype(np.int64)
    zz = z[keep]
    rgb = np.clip(scene["sh"][0:3, keep].astype(np.float64) * SH_C0 + 0.5, 0.0, 1.0)
    order = np.argsort(-zz, kind="stable")  # far first, nearest written last
    out_rgb = np.empty((3, H, W), np.float32)
    out_rgb[:] = np.asarray(view["bg"], np.float32)[:, None, None]
    out_d = np.zeros((H, W), np.float32)
    for du in range(-splat, splat + 1):
        for dv in range(-splat, splat + 1):
            uu, vv = u[order] + du, v[order] + dv
            ok = (uu >= 0) & (uu < W) & (vv >= 0) & (vv < H)
            lin = vv[ok] * W + uu[ok]
            # later (nearer) writes win: numpy fancy assignment keeps the last
            out_d.reshape(-1)[lin] = zz[order][ok]
            for c in range(3):
                out_rgb[c].reshape(-1)[lin] = rgb[c][order][ok]
    return out_rgb, out_d


def pixel_subset_mask(seed, width, height, fraction):
    rng = np.random.default_rng(seed)
    return (rng.uniform(0.0, 1.0, size=(height, width)) < fraction).astype(np.uint8)


def bernoulli_mask(seed, n, p):
    rng = np.random.default_rng(seed)
    return (rng.uniform(0.0, 1.0, size=n) < p).astype(np.uint8)


# ----------------------------------------------------------------------------
# the five workloads (seed = 1000 + index; per-view seed + v)
# ----------------------------------------------------------------------------

def workload_plain_2k():
    """2,000 Gaussians SH0 in a 160x120 identity-pose frustum, random targets,
    loss L1(colour) + 0.5 L1(depth)."""
    seed = 1000
    scene, view = frustum_scene(seed)
    rgb, depth = random_targets(seed + 1, view["width"], view["height"])
    return dict(scenes=[scene], views=[view], targets=[(rgb, depth)], w_c=1.0, w_d=0.5)


def workload_room_mapping(n=300_000, width=1200, height=680):
    """300k SH3 Gaussians in the 8x6x3 m room, one 1200x680 view (fx=fy=600)."""
    seed = 1001
    scene = room_scene(seed, n=n)
    f = 600.0 * width / 1200.0
    view = room_view(width, height, f)
    rgb, depth = zbuffer_targets(scene, view, seed + 1)
    return dict(scenes=[scene], views=[view], targets=[(rgb, depth)], w_c=1.0, w_d=0.5)


def workload_tracking(n=300_000, n_hyp=16, width=1200, height=680, coarse_fraction=0.10,
                      keep_p=0.6, twist_sigma=0.02):
    """Pose hypotheses around the room view: coarse (W/2 x H/2, 10% pixels) then fine
    (W x H, ~30% of Gaussians: opacity > 0.5 and a seeded keep mask)."""
    seed = 1002
    scene = room_scene(1001, n=n)
    f = 600.0 * width / 1200.0
    view_gt = room_view(width, height, f)
    rng = np.random.default_rng(seed)
    twists = rng.normal(0.0, twist_sigma, size=(n_hyp, 6))
    coarse_gt = scale_view(view_gt, 0.5)
    return dict(scene=scene, view_gt=view_gt, coarse_gt=coarse_gt, twists=twists.astype(np.float32),
                coarse_mask=pixel_subset_mask(seed + 1, coarse_gt["width"], coarse_gt["height"],
                                              coarse_fraction),
                keep_mask=bernoulli_mask(seed + 2, n, keep_p))


def workload_batched_mapping(n=1_000_000, n_views=8, width=1200, height=680, hole=True):
    """1M SH3 room, 8 keyframes on a smooth path; for the expansion step a 1 m^3 box of
    Gaussians is removed and 1% of the opacity logits are drawn from N(-7, 1)."""
    seed = 1003
    full = room_scene(seed, n=n)
    views = trajectory_views(seed + 1, n_views, width, height)
    targets = [zbuffer_targets(full, v, seed + 10 + i) for i, v in enumerate(views)]
    cur = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in full.items()}
    if hole:
        rng = np.random.default_rng(seed + 2)
        lo = np.array([rng.uniform(1, 6), rng.uniform(1, 4), 0.0])
        inside = np.all((full["mean"].T >= lo) & (full["mean"].T <= lo + 1.0), axis=1)
        keep = ~inside
        cur = {k: (v[..., keep].copy() if isinstance(v, np.ndarray) else v) for k, v in cur.items()}
        m = cur["opacity_logit"].shape[0]
        low = rng.uniform(0, 1, m) < 0.01
        cur["opacity_logit"][low] = rng.normal(-7.0, 1.0, int(low.sum())).astype(np.float32)
    return dict(full=full, scene=cur, views=views, targets=targets, w_c=1.0, w_d=0.5)


RESOLUTIONS = ((320, 240), (640, 480), (1200, 680))


def workload_uneven(n_views=12, n_min=50_000, n_max=2_000_000, sh_degree=3):
    """12 views with resolutions drawn from {320x240, 640x480, 1200x680}, each with its
    own room of N log-uniform in [n_min, n_max] Gaussians."""
    seed = 1004
    rng = np.random.default_rng(seed)
    scenes, views, targets = [], [], []
    for v in range(n_views):
        W, H = RESOLUTIONS[rng.integers(0, len(RESOLUTIONS))]
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        sc = room_scene(seed + 100 + v, n=n, sh_degree=sh_degree)
        vw = trajectory_views(seed + 200 + v, 1, W, H)[0]
        scenes.append(sc)
        vw["scene"] = v
        views.append(vw)
        targets.append(zbuffer_targets(sc, vw, seed + 300 + v))
    return dict(scenes=scenes, views=views, targets=targets, w_c=1.0, w_d=0.5)
