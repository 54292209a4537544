"""Device-driven localisation loop (mcl_localize) and the on-device pixel-set
draw.  The loop must reproduce the single-step entry points exactly (same
kernels, same arithmetic, same random streams), follow its schedule, and give
the same result eagerly and as a replayed CUDA graph."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import lib

pytestmark = pytest.mark.gpu

W = H = 400
F = 555.6


@pytest.fixture(scope="module")
def M():
    return lib()


@pytest.fixture(scope="module")
def gm(M):
    m = M.Map(synth.he_init_weights(2), max_rays=2 * 700 * 64, max_samples=192,
              max_particles=2 * 700, max_queries=4)
    yield m
    m.close()


def ctr(q, t, p):
    return (q << 32) | (t << 2) | p


@pytest.mark.parametrize("W_,H_,B,seed,c", [(100, 100, 16, 3, 7), (400, 400, 64, 11, 0),
                                          (7, 3, 21, 1, 2), (200, 200, 256, 5, 9)])
def test_draw_pixels_matches_oracle(M, W_, H_, B, seed, c):
    g = M.draw_pixels(W_, H_, B, seed, c).cpu().numpy()
    assert np.array_equal(g, oracle.pixel_set(W_, H_, B, seed, c))


def _query(M, seed, n, with_gt=True):
    import torch
    P = synth.random_particles(seed, n)[0]
    gt = synth.gt_pose(seed)[0]
    if with_gt:
        P[n // 2] = gt
    return torch.tensor(P, dtype=torch.float32, device="cuda"), gt


def _observation(M, gm, gt):
    import torch
    K = M.intrinsics(F, F, W / 2, H / 2, W, H)
    allpx = np.stack(np.meshgrid(np.arange(W), np.arange(H), indexing="xy"), -1).reshape(-1, 2)
    img = torch.empty(W * H, 3, device="cuda")
    o = M.UpdateOptions(n_coarse=64, n_fine=128, precision="bf16")
    g = torch.tensor(gt[None], dtype=torch.float32, device="cuda")
    for c0 in range(0, W * H, 40000):
        px = torch.tensor(allpx[c0:c0 + 40000], dtype=torch.int32, device="cuda")
        img[c0:c0 + px.shape[0]] = gm.render(g, K, 2, px, o)
    return img.reshape(H, W, 3).contiguous(), K


@pytest.fixture(params=[False, True], ids=["separate", "fused"])
def fused(request, gm):
    """Both ray-epilogue settings of the tensor-core forms: the separate
    sampling / composite kernels (the default) and the fused MLP epilogue
    (mcl_set_fused_epilogue)."""
    gm.set_fused_epilogue(request.param)
    yield request.param
    gm.set_fused_epilogue(False)


def test_one_iteration_equals_single_step_entry_points(M, gm, fused):
    import torch
    N, seed = 300, 1234
    P0, gt = _query(M, 41, N)
    img, K = _observation(M, gm, gt)
    opts = M.UpdateOptions(n_coarse=64, n_fine=128, precision="bf16", seed=seed)
    sch = M.schedule([1], [32], [N], n_min=8, iterations=1)
    parts = P0.clone().reshape(1, N, 12)
    log, fin = gm.localize(parts, [N], [img], K, sch, opts, use_graph=False)
    rec = M.Map.decode_log(log, 1, 1)[0][0]
    # the same iteration through the single-step entry points
    px = M.draw_pixels(W // 2, H // 2, 32, seed, ctr(0, 0, 0))
    out = gm.update(P0, img, K, 1, px, opts)
    n_s = int(out["mask"].sum().item())
    assert rec["n_survivors"] == n_s and rec["n_particles"] == N and rec["n_pixels"] == 32
    n_next = min(max(n_s, 8), N)
    assert int(fin[0].item()) == n_next
    u0 = oracle.uniform(seed, ctr(0, 0, 1), 0)
    idx = gm.resample(out["w"], n_next, u0)
    Pn = M.predict(P0, idx, n_next, 0.05, 0.05, seed, ctr(0, 0, 2))
    torch.cuda.synchronize()
    assert torch.equal(parts[0, :n_next], Pn)
    w = out["w"].cpu().numpy()
    est = (w[:, None] * P0.cpu().numpy()[:, [3, 7, 11]]).sum(0)
    assert np.allclose(rec["est"][:3], est, atol=1e-5)


def test_schedule_invariants_uneven_queries_and_graph_replay(M, gm, fused):
    import torch
    Q, stride = 2, 700
    n0 = [700, 450]
    parts = torch.full((Q, stride, 12), float("nan"), device="cuda")
    imgs = []
    for q in range(Q):
        P, gt = _query(M, 50 + q, n0[q])
        parts[q, :n0[q]] = P
        img, K = _observation(M, gm, gt)
        imgs.append(img)
    sch = M.schedule([0, 1, 2], [16, 32, 64], [700, 350, 175], n_min=64, iter_caps=[3, 3, 10],
                     refine=[0.05, 0.01, 0.0], iterations=8)
    opts = M.UpdateOptions(n_coarse=64, n_fine=128, precision="bf16", seed=99)
    a = parts.clone()
    log_a, fin_a = gm.localize(a, n0, imgs, K, sch, opts, use_graph=False)
    b = parts.clone()
    log_b, fin_b = gm.localize(b, n0, imgs, K, sch, opts, use_graph=True)
    c = parts.clone()
    log_c, fin_c = gm.localize(c, n0, imgs, K, sch, opts, use_graph=True)   # replay
    torch.cuda.synchronize()
    # identical records (bytes) apart from the GPU timer stamps
    import ctypes
    size, off = ctypes.sizeof(M.IterRecord), M.IterRecord.t_start_ns.offset

    def strip(log):
        r = log.reshape(-1, size).clone()
        r[:, off:off + 8] = 0
        return r
    assert torch.equal(strip(log_a), strip(log_b)) and torch.equal(strip(log_b), strip(log_c))
    ts = [r["t_start_ns"] for r in M.Map.decode_log(log_b, Q, 8)[0]]
    assert all(b > a for a, b in zip(ts[:-1], ts[1:]))
    assert torch.equal(fin_a, fin_b) and torch.equal(fin_b, fin_c)
    for q in range(Q):
        k = int(fin_a[q].item())
        assert torch.equal(a[q, :k], b[q, :k]) and torch.equal(b[q, :k], c[q, :k])
    recs = M.Map.decode_log(log_a, Q, 8)
    for q in range(Q):
        r = recs[q]
        assert r[0]["n_particles"] == n0[q]
        for t in range(8):
            st = r[t]["stage"]
            assert r[t]["level"] == [0, 1, 2][st] and r[t]["n_pixels"] == [16, 32, 64][st]
            assert np.all(np.isfinite(r[t]["est"])) and r[t]["status"] == 0
            if t > 0:
                assert st >= r[t - 1]["stage"]
                cap = [700, 350, 175][st]
                assert r[t]["n_particles"] == min(max(r[t - 1]["n_survivors"], 64), cap)
        # the iteration caps force every stage to be visited
        assert r[-1]["stage"] == 2
    assert int(fin_a[0].item()) == min(max(recs[0][-1]["n_survivors"], 64), 175)


def test_gt_particle_pulls_the_estimate(M, gm):
    """A query whose particle set contains the ground truth: after the first
    weighting the estimate sits on the ground truth (its loss is ~0)."""
    import torch
    N = 400
    P0, gt = _query(M, 60, N)
    img, K = _observation(M, gm, gt)
    sch = M.schedule([2], [64], [N], n_min=32, iterations=3)
    opts = M.UpdateOptions(n_coarse=64, n_fine=128, precision="bf16", seed=5)
    parts = P0.clone().reshape(1, N, 12)
    log, fin = gm.localize(parts, [N], [img], K, sch, opts, use_graph=False)
    r = M.Map.decode_log(log, 1, 3)[0]
    assert np.linalg.norm(np.array(r[0]["est"][:3]) - gt[[3, 7, 11]]) < 1e-3


def test_loop_log_replays_through_the_oracle(M, gm):
    """Every record of a 2-query, 8-iteration run against the FP64 oracle's
    statement of the refinement statistic and the schedule (Sec. III-C):
    the particles at the start of iteration t (a run of t iterations) are
    weighted through mcl_update with the iteration's pixel set, and
    orc_loop_statistics of those weights must give the record's spread
    (1e-9 relative), pose estimate and survivor count (exactly), and
    orc_loop_schedule the next record's stage and particle count (exactly)."""
    import torch
    Q, stride, iters = 2, 700, 8
    n0 = [700, 450]
    parts = torch.full((Q, stride, 12), float("nan"), device="cuda")
    imgs = []
    for q in range(Q):
        P, gt = _query(M, 70 + q, n0[q], with_gt=False)
        parts[q, :n0[q]] = P
        img, K = _observation(M, gm, gt)
        imgs.append(img)
    levels, pixels, caps = [0, 1, 2], [16, 32, 64], [700, 350, 175]
    refine, iter_caps, n_min = [0.3, 0.05, 0.0], [3, 3, 10], 64
    sch = M.schedule(levels, pixels, caps, n_min=n_min, iter_caps=iter_caps, refine=refine,
                     iterations=iters)
    seed = 321
    opts = M.UpdateOptions(n_coarse=64, n_fine=128, precision="bf16", seed=seed)
    full = parts.clone()
    log, fin = gm.localize(full, n0, imgs, K, sch, opts, use_graph=False)
    recs = M.Map.decode_log(log, Q, iters)
    # particles at the start of each iteration
    starts = [[parts[q, :n0[q]].clone() for q in range(Q)]]
    for t in range(1, iters):
        p = parts.clone()
        _, f = gm.localize(p, n0, imgs, K, M.schedule(levels, pixels, caps, n_min=n_min,
                                                      iter_caps=iter_caps, refine=refine,
                                                      iterations=t), opts, use_graph=False)
        starts.append([p[q, :int(f[q].item())].clone() for q in range(Q)])
    for q in range(Q):
        stage, it = 0, 0
        for t in range(iters):
            r = recs[q][t]
            Pq = starts[t][q]
            assert r["stage"] == stage and r["n_particles"] == Pq.shape[0]
            B, lev = pixels[stage], levels[stage]
            f = 4 >> lev
            px = M.draw_pixels(W // f, H // f, B, seed, ctr(q, t, 0))
            out = gm.update(Pq.contiguous(), imgs[q], K, lev, px, opts)
            w = out["w"].cpu().numpy()
            mask = out["mask"].cpu().numpy()
            st = oracle.loop_statistics(Pq.cpu().numpy().astype(np.float64), w, mask)
            assert r["spread"] == pytest.approx(st["spread"], rel=1e-9)
            assert np.allclose(r["est"][:3], st["mean"], rtol=0, atol=1e-12)
            assert r["est"][3] == pytest.approx(st["yaw"], abs=1e-12)
            assert r["n_survivors"] == st["n_survivors"]
            nxt = oracle.loop_schedule(stage, it, st["n_survivors"], st["spread"], refine,
                                       iter_caps, caps, n_min, stride)
            stage, it, n_next = nxt
            if t + 1 < iters:
                assert recs[q][t + 1]["stage"] == stage
                assert recs[q][t + 1]["n_particles"] == n_next
            else:
                assert int(fin[q].item()) == n_next
