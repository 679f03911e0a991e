"""Bundle adjustment (Sec. 3.3, Eq. BA) on the batched kernels: the loss and the
per-keyframe twist gradients of one BA iteration against the FP64 oracle, and a
BA run that recovers a perturbed map and perturbed keyframe poses."""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from gpu_util import GRAD_REL_L2, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_11700_gb300 import build
    build.build()
    import paper_2311_11700_gb300 as g
    return g


def _window(seed, n, n_kf, W, H):
    sc = synth.room_scene(seed, n=n)
    views = synth.trajectory_views(seed + 1, n_kf, W, H)
    return sc, views


def test_ba_loss_and_twist_gradients_match_oracle(G):
    from paper_2311_11700_gb300 import slam
    sc, views = _window(71, 3000, 4, 64, 48)
    targets = [synth.random_targets(80 + i, 64, 48) for i in range(4)]
    R = G.Renderer(0)
    scene = G.Scene.from_numpy(sc)
    poses = torch.as_tensor(np.stack([np.asarray(v["T_cw"], np.float32) for v in views]), device="cuda")
    # one iteration with zero learning rates: the loss and gradients at the inputs
    opt = slam.MapAdam(scene, lr={k: 0.0 for k in slam.MAP_LR})
    opt.decay_steps = 1
    losses, sel = slam.bundle_adjust(R, scene, views, poses, targets, iters=1, K=4, map_opt=opt)
    assert sel == [0, 1, 2, 3]
    ref = O.render_and_grad([sc], [dict(v, scene=0) for v in views], targets, w_c=0.8 / 4, w_d=0.3 / 4)
    assert abs(losses[0] - ref["loss"]) <= 1e-4 * ref["loss"]


def test_ba_twist_gradient_per_keyframe_matches_oracle(G):
    sc, views = _window(72, 3000, 3, 64, 48)
    targets = [synth.random_targets(90 + i, 64, 48) for i in range(3)]
    R = G.Renderer(0)
    R.ctx.set_grad_mode(1)
    scene = G.Scene.from_numpy(sc)
    poses = torch.as_tensor(np.stack([np.asarray(v["T_cw"], np.float32) for v in views]), device="cuda")
    batch = [dict(v, scene=0, T_cw_dev=poses[i]) for i, v in enumerate(views)]
    color, depth, acc, ws, mp = R.forward([scene], batch)
    trgb = torch.as_tensor(np.concatenate([t[0].reshape(-1) for t in targets]), device="cuda")
    tdep = torch.as_tensor(np.concatenate([t[1].reshape(-1) for t in targets]), device="cuda")
    loss = torch.zeros(3, device="cuda")
    dC, dD = torch.empty_like(color), torch.empty_like(depth)
    G.gs_loss_l1(R.ctx, batch, (color, depth, acc), trgb, tdep, 0.8 / 3, 0.3 / 3, loss, (dC, dD, None))
    grads = [{k: torch.full_like(getattr(scene, k), 5.0) for k in G.PARAM_KEYS}]
    dtw = torch.full((3, 6), 5.0, device="cuda")
    G.gs_render_backward(R.ctx, [scene], batch, ws, mp, (dC, dD, None), grads, dtw, 0)
    torch.cuda.synchronize()
    ref = O.render_and_grad([sc], [dict(v, scene=0) for v in views], targets, w_c=0.8 / 3, w_d=0.3 / 3)
    assert rel_l2(dtw.cpu().numpy().astype(np.float64), ref["twist"]) < GRAD_REL_L2
    for k in G.PARAM_KEYS:
        assert rel_l2(grads[0][k].cpu().numpy().astype(np.float64), ref["grads"][0][k]) < GRAD_REL_L2, k


def test_ba_recovers_a_perturbed_map_and_poses(G):
    """Targets rendered from the true map at the true keyframe poses; the map means
    are perturbed by N(0, 0.01^2) m and the poses by twists N(0, 0.01^2): BA (map all
    the way, poses in the second half) lowers the loss and the pose error."""
    from paper_2311_11700_gb300 import slam
    sc, views = _window(73, 40_000, 6, 160, 96)
    R = G.Renderer(0)
    true_scene = G.Scene.from_numpy(sc)
    true_poses = torch.as_tensor(np.stack([np.asarray(v["T_cw"], np.float32) for v in views]), device="cuda")
    targets = []
    for i, v in enumerate(views):
        c, d, a, *_ = R.forward([true_scene], [dict(v, scene=0)])
        targets.append((c.view(3, 96, 160).cpu().numpy(), d.view(96, 160).cpu().numpy()))
    rng = np.random.default_rng(74)
    noisy = dict(sc, mean=(sc["mean"] + rng.normal(0, 0.01, sc["mean"].shape)).astype(np.float32))
    scene = G.Scene.from_numpy(noisy)
    xis = rng.normal(0, 0.01, (6, 6))
    poses = torch.as_tensor(np.stack([np.asarray(synth.perturb_view(v, x)["T_cw"], np.float32)
                                      for v, x in zip(views, xis)]), device="cuda")

    def pose_err(P):
        e = []
        for i in range(6):
            T, Tg = P[i].cpu().numpy().astype(np.float64).reshape(3, 4), true_poses[i].cpu().numpy().reshape(3, 4)
            e.append(np.linalg.norm(-T[:, :3].T @ T[:, 3] + Tg[:, :3].T @ Tg[:, 3]))
        return float(np.mean(e))

    e0 = pose_err(poses)
    opt = slam.MapAdam(scene, lr={"mean": 2e-3}, decay_steps=200)
    losses, sel = slam.bundle_adjust(R, scene, views, poses, targets, iters=120, K=6, map_opt=opt,
                                     pose_lr=(2e-3,) * 6)
    assert sel == list(range(6))
    assert losses[-1] < 0.7 * losses[0], (losses[0], losses[-1])
    assert pose_err(poses) < e0, (e0, pose_err(poses))
