"""Pins of two composed parts of the FP64 oracle, each against closed forms,
invariants and independent renders (CPU only):

* the learned-proposal render (orc_render_rays_proposal): proposal weights ->
  guided samples -> NeRF MLP -> importance samples -> merged Eq. 1 composite
  and Eq. 5 / F.  Its pieces (inverse CDF, composite, Eq. 5) are pinned in
  test_oracle_pins.py; these tests pin how they are put together;
* the statistics and the schedule step of the coarse-to-fine loop
  (orc_loop_statistics, orc_loop_schedule; Sec. III-C refinement test).
"""
import math

import numpy as np
import pytest

import oracle
import synth


# ------------------------------------------------------ proposal render ---
def _const_map(c, b_rgb):
    """NeRF map with zero trunk: raw density c and colour sigmoid(b_rgb)
    everywhere (closed form)."""
    return synth.blob_from_layers({"sigma": (None, np.array([c])),
                                   "rgb_out": (None, np.asarray(b_rgb, dtype=np.float64))})


def _rays(seed, n):
    rng = np.random.default_rng(seed)
    o = rng.uniform(-1, 1, size=(n, 3))
    d = rng.normal(size=(n, 3))
    d[:, 2] = -np.abs(d[:, 2]) - 0.5
    return o, d


def _crossings(z, c, dn, alpha, tau):
    """Eq. 5 / F on sorted samples z of a ray of constant density c (the last
    interval is 1e10 long): W_k = 1 - exp(-c (z_{k+1} - z_0) |d|) for k < n-1,
    W_{n-1} = 1.  Returns z_trans, z_opaque, F and the smallest distance of
    any W_k to alpha or 1 - alpha (to keep the cases away from ties)."""
    n = len(z)
    W = np.ones(n)
    W[:-1] = 1.0 - np.exp(-c * (z[1:] - z[0]) * dn)
    kt = int(np.argmax(W >= alpha))
    below = np.nonzero(W <= 1.0 - alpha)[0]
    zt = z[kt]
    zo = z[below[-1]] if len(below) else z[0]
    margin = min(np.abs(W - alpha).min(), np.abs(W - (1.0 - alpha)).min())
    return zt, zo, max(zo - zt, tau), margin


def test_proposal_render_guided_samples_closed_form():
    """Zero proposal density: the proposal weights are all zero, so the pdf
    over the interior proposal bins is uniform and the guided samples are
    evenly spaced between the first and last midpoint of the stratified
    proposal samples: z_j = e_0 + j/(n_g - 1) (e_last - e_0).  With no
    importance samples, the final composite runs over exactly these n_g
    samples of a constant-density map, whose Eq. 5 crossings and
    transmittance are closed forms."""
    near, far, n_p, n_g, alpha, tau = 2.0, 6.0, 24, 17, 0.05, 0.1
    c = float(np.float32(0.9))
    b = np.array([0.3, -1.2, 2.0])
    blob = _const_map(c, b)
    pblob = np.zeros(synth.proposal_n_weights(), dtype=np.float32)
    o, d = _rays(3, 6)
    opts = oracle.make_opts(n_coarse=n_p, n_fine=0, alpha=alpha, tau=tau)
    r = oracle.render_rays_proposal(blob, pblob, o, d, opts, n_p=n_p, n_g=n_g)
    e0 = near + (far - near) / n_p
    e1 = near + (far - near) * (n_p - 1) / n_p
    zg = e0 + np.arange(n_g) / (n_g - 1) * (e1 - e0)
    col = 1.0 / (1.0 + np.exp(-b.astype(np.float32).astype(np.float64)))
    for i in range(len(o)):
        dn = np.linalg.norm(d[i])
        zt, zo, F, margin = _crossings(zg, c, dn, alpha, tau)
        assert margin > 1e-6
        assert r["z_trans"][i] == pytest.approx(zt, abs=1e-12)
        assert r["z_opaque"][i] == pytest.approx(zo, abs=1e-12)
        assert r["F"][i] == pytest.approx(F, abs=1e-12)
        assert r["T_last"][i] == pytest.approx(math.exp(-c * (zg[-1] - zg[0]) * dn), rel=1e-12)
        assert r["sigma_last"][i] == pytest.approx(c, rel=1e-15)
        assert np.allclose(r["rgb"][i], col, rtol=0, atol=1e-14)


def test_proposal_render_merges_importance_samples_of_the_guided_pass():
    """With importance samples, they are drawn from the composite weights of
    the guided samples (closed form on a constant-density map; the inverse
    CDF is the pinned orc_sample_pdf) and merged with them: the final Eq. 5
    crossings and transmittance are those of the sorted union.  A render
    that drew them from the proposal weights (uniform here), or composited
    the guided samples alone, fails this."""
    near, far, n_p, n_g, n_f, alpha, tau = 2.0, 6.0, 20, 16, 24, 0.05, 0.1
    c = float(np.float32(2.5))
    blob = _const_map(c, [0.0, 0.5, -0.5])
    pblob = np.zeros(synth.proposal_n_weights(), dtype=np.float32)
    o, d = _rays(4, 5)
    opts = oracle.make_opts(n_coarse=n_p, n_fine=n_f, alpha=alpha, tau=tau)
    r = oracle.render_rays_proposal(blob, pblob, o, d, opts, n_p=n_p, n_g=n_g)
    e0 = near + (far - near) / n_p
    e1 = near + (far - near) * (n_p - 1) / n_p
    zg = e0 + np.arange(n_g) / (n_g - 1) * (e1 - e0)
    checked = 0
    for i in range(len(o)):
        dn = np.linalg.norm(d[i])
        a = 1.0 - np.exp(-c * np.diff(zg) * dn)
        T = np.concatenate([[1.0], np.cumprod(1.0 - a)])
        wg = T * np.concatenate([a, [1.0]])
        zf = oracle.sample_pdf(zg, wg, n_f)
        zm = np.sort(np.concatenate([zg, zf]), kind="stable")
        zt, zo, F, margin = _crossings(zm, c, dn, alpha, tau)
        if margin < 1e-6:
            continue
        checked += 1
        assert r["z_trans"][i] == pytest.approx(zt, abs=1e-12)
        assert r["z_opaque"][i] == pytest.approx(zo, abs=1e-12)
        assert r["F"][i] == pytest.approx(F, abs=1e-12)
        assert r["T_last"][i] == pytest.approx(math.exp(-c * (zm[-1] - zm[0]) * dn), rel=1e-10)
        # the alternatives the composition could get wrong give other answers
        zo_g = _crossings(zg, c, dn, alpha, tau)[1]
        zu = np.sort(np.concatenate([zg, oracle.sample_pdf(zg, np.zeros(n_g), n_f)]))
        assert abs(zo_g - zo) > 1e-6 and abs(_crossings(zu, c, dn, alpha, tau)[1] - zo) > 1e-6
    assert checked >= 3


def test_proposal_render_with_exact_room_proposal_converges_to_continuous_integral():
    """A proposal whose density is exactly the room map's (hand-set,
    synth.room_proposal_weights) guides the samples onto the wall.  The
    guided samples can only resolve the wall to one proposal bin (the
    proposal weight of the bin the wall enters goes to the bin's far edge),
    so the render converges as the proposal bins shrink: with 256 proposal,
    128 guided and 128 importance samples it is within the plain sampler's
    convergence bars of the continuous rendering integral (colour 5e-3,
    z_trans 2e-2 of the wall, F = tau on the sharp wall), and four times
    coarser proposal bins leave a larger error."""
    from room_scene import pixel_rays, render_continuous, wall_hit
    blob, a = synth.room_map_weights(0)
    a32 = a.astype(np.float32).astype(np.float64)
    pblob = synth.room_proposal_weights()
    P = synth.random_particles(6, 2)[0]
    px = synth.pixel_set(6, 25, 25, 12)
    o, d = map(np.concatenate, zip(*[pixel_rays(p, 138.9 / 4, 138.9 / 4, 12.5, 12.5, px)
                                      for p in P]))
    ref, t_left = render_continuous(o, d, a32)
    assert t_left.max() < 1e-6
    err = {}
    for n_p in (64, 256):
        opts = oracle.make_opts(n_coarse=n_p, n_fine=128)
        r = oracle.render_rays_proposal(blob, pblob, o, d, opts, n_p=n_p, n_g=128)
        err[n_p] = np.abs(r["rgb"] - ref).max()
        assert np.allclose(r["F"], 0.1)
    assert err[256] < 5e-3
    assert np.abs(r["z_trans"] - wall_hit(o, d, 3.0)).max() < 2e-2
    assert err[64] > 4 * err[256]


# ------------------------------------------------------ loop statistics ---
def _poses(seed, n):
    P, xyz, yaw = synth.random_particles(seed, n)
    return P.astype(np.float64), xyz, yaw


def test_loop_statistics_uniform_weights_is_the_population_spread():
    P, _, _ = _poses(1, 37)
    st = oracle.loop_statistics(P, np.full(37, 1.0 / 37), np.ones(37))
    ref = oracle.position_spread(P)
    assert np.allclose(st["mean"], ref["mean"], rtol=0, atol=1e-14)
    assert st["spread"] == pytest.approx(ref["trace"], rel=1e-13)
    assert st["n_survivors"] == 37


def test_loop_statistics_two_particles_closed_form():
    """Weights (p, 1 - p) at positions a, b: mean p a + (1 - p) b and spread
    p (1 - p) |a - b|^2."""
    a, b, p = np.array([0.3, -0.2, 0.9]), np.array([-0.5, 0.4, 0.1]), 0.3
    P = synth.pose_from_xyz_yaw([a, b], [0.2, 1.1]).astype(np.float64)
    st = oracle.loop_statistics(P, np.array([p, 1.0 - p]), np.array([1, 0]))
    assert np.allclose(st["mean"], p * a + (1 - p) * b, rtol=0, atol=1e-15)
    assert st["spread"] == pytest.approx(p * (1 - p) * ((a - b) ** 2).sum(), rel=1e-13)
    assert st["n_survivors"] == 1


def test_loop_statistics_point_mass_scale_and_split_invariance():
    P, xyz, yaw = _poses(2, 20)
    w = np.zeros(20)
    w[7] = 1.0
    st = oracle.loop_statistics(P, w, np.zeros(20))
    assert np.allclose(st["mean"], xyz[7], atol=1e-15)
    assert st["spread"] == 0.0
    assert st["yaw"] == pytest.approx((yaw[7] + math.pi) % (2 * math.pi) - math.pi, abs=1e-12)
    assert st["n_survivors"] == 0
    rng = np.random.default_rng(3)
    w = rng.dirichlet(np.ones(20))
    base = oracle.loop_statistics(P, w, w > 0.05)
    scaled = oracle.loop_statistics(P, 7.5 * w, w > 0.05)
    assert np.allclose(scaled["mean"], base["mean"], rtol=0, atol=1e-14)
    assert scaled["spread"] == pytest.approx(base["spread"], rel=1e-13)
    assert scaled["yaw"] == pytest.approx(base["yaw"], abs=1e-13)
    # a particle split into two copies with half its weight each
    P2 = np.concatenate([P, P[4:5]])
    w2 = np.concatenate([w, [w[4] / 2]])
    w2[4] /= 2
    split = oracle.loop_statistics(P2, w2, np.ones(21))
    assert np.allclose(split["mean"], base["mean"], rtol=0, atol=1e-14)
    assert split["spread"] == pytest.approx(base["spread"], rel=1e-12)
    assert split["n_survivors"] == 21


def test_loop_statistics_circular_yaw():
    P = synth.pose_from_xyz_yaw([[0, 0, 0]] * 2, [math.pi - 0.1, -math.pi + 0.1]).astype(np.float64)
    st = oracle.loop_statistics(P, np.array([0.5, 0.5]), np.ones(2))
    assert abs(abs(st["yaw"]) - math.pi) < 1e-12
    P = synth.pose_from_xyz_yaw([[0, 0, 0]] * 3, [0.4, -0.4, 0.0]).astype(np.float64)
    st = oracle.loop_statistics(P, np.array([0.25, 0.25, 0.5]), np.ones(3))
    assert abs(st["yaw"]) < 1e-14
    P = synth.pose_from_xyz_yaw([[0, 0, 0]] * 2, [0.3, 1.3]).astype(np.float64)
    st = oracle.loop_statistics(P, np.array([0.5, 0.5]), np.ones(2))
    assert st["yaw"] == pytest.approx(0.8, abs=1e-12)


def test_loop_schedule_transitions_by_hand():
    sch = dict(refine=[0.05, 0.01, 0.0], iter_cap=[7, 7, 6], n_cap=[1500, 1000, 600],
               n_min=100, stride=1500)
    step = lambda st, it, ns, V: oracle.loop_schedule(st, it, ns, V, **sch)
    assert step(0, 0, 900, 0.2) == (0, 1, 900)            # spread above: stay
    assert step(0, 3, 900, 0.049) == (1, 0, 900)          # spread below: refine
    assert step(0, 3, 900, 0.05) == (0, 4, 900)           # strictly below only
    assert step(0, 6, 1400, 0.9) == (1, 0, 1000)          # cap forces refine; next cap
    assert step(1, 2, 40, 0.5) == (1, 3, 100)             # floor n_min
    assert step(2, 9, 5000, 0.0) == (2, 10, 600)          # last stage never refines
    assert step(1, 0, 700, 0.001) == (2, 0, 600)
    assert oracle.loop_schedule(0, 0, 900, 0.2, [1.0], [5], [800], 10, 700) == (0, 1, 700)
