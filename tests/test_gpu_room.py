"""End-to-end localisation on the analytic room map (synth.room_map_weights),
whose ground truth is unique: the observed images are the continuous
rendering integral of the closed-form field at seeded ground-truth poses
(tests/room_scene.py, independent of the oracle and of the library), and the
device-driven filter (Alg. 1 with the coarse-to-fine schedule) must end at
the ground truth from the global initial spread (+-1 m, +-180 deg)."""
import math

import numpy as np
import pytest

import synth
from gpu_helpers import lib
from room_scene import observed_image, pixel_rays, render_continuous

pytestmark = pytest.mark.gpu

W = H = 100
FOCAL = 138.9
Q, N = 4, 2000


@pytest.fixture(scope="module")
def M():
    return lib()


@pytest.fixture(scope="module")
def room(M):
    blob, a = synth.room_map_weights(0)
    m = M.Map(blob, max_rays=Q * N * 64, max_samples=192, max_particles=Q * N, max_queries=Q)
    yield m, blob, a.astype(np.float32).astype(np.float64)
    m.close()


@pytest.fixture(scope="module")
def observations(M, room):
    import torch
    _, _, a = room
    gts = [synth.gt_pose(100 + q) for q in range(Q)]
    imgs = [torch.tensor(observed_image(g[0], a, W, H, FOCAL), dtype=torch.float32,
                         device="cuda").contiguous() for g in gts]
    return gts, imgs


@pytest.mark.parametrize("prec,nc,nf,mean_bar,max_bar", [
    ("fp32", 64, 128, 5e-3, 0.08), ("bf16", 64, 128, 1e-2, 0.15), ("bf16", 32, 32, 2e-2, 0.2)])
def test_room_render_close_to_continuous_integral(M, room, prec, nc, nf, mean_bar, max_bar):
    """Renders of the room map stay near the continuous integral: the
    quadrature error of Eq. 1's Riemann sum (FP32: 3e-3 mean with 64 + 128
    samples, as the oracle) plus, for BF16, the rounding of the wall position
    (8 significant bits of m(x) ~ 3 move the wall by ~6e-3)."""
    import torch
    m, _, a = room
    P = synth.random_particles(5, 20)[0]
    px = synth.pixel_set(5, 25, 25, 16)
    o, d = map(np.concatenate, zip(*[pixel_rays(p, FOCAL / 4, FOCAL / 4, 12.5, 12.5, px)
                                      for p in P]))
    ref, _ = render_continuous(o, d, a)
    K = M.intrinsics(FOCAL, FOCAL, W / 2, H / 2, W, H)
    r = m.render(torch.tensor(P, dtype=torch.float32, device="cuda"), K, 0,
                 torch.tensor(px, dtype=torch.int32, device="cuda"),
                 M.UpdateOptions(n_coarse=nc, n_fine=nf, precision=prec)).cpu().numpy()
    e = np.abs(r - ref)
    assert e.mean() <= mean_bar and e.max() <= max_bar, (e.mean(), e.max())


def _localize(M, room, observations, opts, iterations=60, sigma=0.02):
    import torch
    m, _, _ = room
    gts, imgs = observations
    K = M.intrinsics(FOCAL, FOCAL, W / 2, H / 2, W, H)
    sch = M.schedule([0, 1, 2], [64, 64, 64], [N, 1000, 500], n_min=200,
                     iter_caps=[iterations // 3] * 3, refine=[0.02, 0.005, 0.0],
                     iterations=iterations, sigma_t=sigma, sigma_yaw=sigma)
    parts = torch.tensor(np.stack([synth.random_particles(200 + q, N)[0] for q in range(Q)]),
                         dtype=torch.float32, device="cuda")
    log, fin = m.localize(parts, [N] * Q, imgs, K, sch, opts, use_graph=True)
    recs = M.Map.decode_log(log, Q, iterations)
    errs = []
    for q in range(Q):
        est = recs[q][-1]["est"]
        pos = float(np.linalg.norm(np.array(est[:3]) - gts[q][1]))
        yaw = abs((est[3] - gts[q][2] + math.pi) % (2 * math.pi) - math.pi)
        errs.append((pos, math.degrees(yaw)))
        assert recs[q][-1]["stage"] == 2
        assert all(r["status"] == 0 for r in recs[q])
    return errs


def test_room_localization_converges(M, room, observations):
    """Four queries from the global spread, 2000 particles each, 60
    iterations of the BF16 loop (levels 1/4, 1/2, 1 of a 100 x 100 image, 64
    pixels per update): every estimate ends within 10 cm and 5 degrees (the
    paper's rotation threshold, Sec. IV-A)."""
    errs = _localize(M, room, observations,
                     M.UpdateOptions(n_coarse=64, n_fine=64, precision="bf16", seed=1))
    assert all(p < 0.1 and y < 5.0 for p, y in errs), errs


def test_room_localization_with_trained_proposal(M, room, observations):
    """The same run with the learned proposal sampler (64 proposal samples,
    32 guided + 32 importance NeRF samples) distilled on this map from other
    poses: the same accuracy with half the NeRF evaluations of 64 + 64."""
    import torch
    m, _, _ = room
    P = synth.random_particles(21, 256)[0]
    px = synth.pixel_set(21, 25, 25, 64)
    K = M.intrinsics(FOCAL, FOCAL, W / 2, H / 2, W, H)
    m.proposal_set(synth.proposal_init_weights(0))
    m.proposal_train(torch.tensor(P, dtype=torch.float32, device="cuda"),
                     torch.tensor(px, dtype=torch.int32, device="cuda"), K, 0,
                     M.UpdateOptions(n_coarse=64, n_fine=128, precision="fp32"), epochs=40,
                     batch_rays=2048, n_bins=64, lr=3e-3, lr_end=1e-4, seed=1)
    errs = _localize(M, room, observations,
                     M.UpdateOptions(n_coarse=64, n_fine=32, precision="bf16", seed=1,
                                     use_proposal=True, n_proposal=64, n_guided=32))
    assert all(p < 0.1 and y < 5.0 for p, y in errs), errs


def test_room_tracking_with_odometry(M, room):
    """Tracking mode (Sec. III-A motion model with odometry O_t): the camera
    moves 4 cm forward and turns 1.5 degrees per frame for 24 frames; each
    frame the filter predicts with the (noise-free) odometry plus motion
    noise, weights 500 particles with 64 pixels of the half-resolution level
    (BF16, public single-step entry points) and resamples.  Starting 5 cm /
    3 degrees off, the estimate stays within 5 cm and 2 degrees."""
    import torch
    m, _, a = room
    K = M.intrinsics(FOCAL, FOCAL, W / 2, H / 2, W, H)
    step = synth.pose_from_xyz_yaw([[0.0, 0.0, -0.04]], [math.radians(1.5)])[0]
    h = lambda p: np.vstack([np.reshape(p, (3, 4)), [0, 0, 0, 1]])
    gt = synth.pose_from_xyz_yaw([[0.2, 0.1, 0.3]], [0.4])[0]
    n, B = 500, 64
    rng = np.random.default_rng(3)
    start = synth.pose_from_xyz_yaw(np.array([[0.2, 0.1, 0.3]]) + rng.normal(0, 0.05, (n, 3)),
                                    0.4 + rng.normal(0, math.radians(3), n))
    P = torch.tensor(start, dtype=torch.float32, device="cuda")
    odom = torch.tensor(step, dtype=torch.float32, device="cuda")
    opts = M.UpdateOptions(n_coarse=64, n_fine=64, precision="bf16")
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    errs = []
    for t in range(24):
        gt = (h(gt) @ h(step))[:3].reshape(12)
        # the half-resolution level rendered directly (focal / 2, 401 samples
        # of the integral), replicated 2 x 2: its box filter is that image
        half = observed_image(gt, a, W // 2, H // 2, FOCAL / 2, n=401)
        img = torch.tensor(np.repeat(np.repeat(half, 2, 0), 2, 1), dtype=torch.float32,
                           device="cuda").contiguous()
        P = M.predict(P, None, n, 0.01, 0.01, 9, 2 * t, odom=odom)
        px = M.draw_pixels(W // 2, H // 2, B, 9, 2 * t + 1)
        out = m.update(P, img, K, 1, px, opts)
        w = out["w"]
        est = (w[:, None] * P.double()[:, [3, 7, 11]]).sum(0).cpu().numpy()
        Pc = P.cpu().numpy().astype(np.float64)
        yaw = np.arctan2(Pc[:, 2], Pc[:, 0])
        wc = w.cpu().numpy()
        yaw_est = math.atan2((wc * np.sin(yaw)).sum(), (wc * np.cos(yaw)).sum())
        gyaw = math.atan2(gt[2], gt[0])
        errs.append((float(np.linalg.norm(est - gt[[3, 7, 11]])),
                     math.degrees(abs((yaw_est - gyaw + math.pi) % (2 * math.pi) - math.pi))))
        m.resample(w, n, (t * 0.618034) % 1.0, idx=idx)
        P = P[idx.long()].contiguous()
    torch.cuda.synchronize()
    assert all(p < 0.05 and y < 2.0 for p, y in errs[4:]), errs
