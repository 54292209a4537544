"""Pins of the FP64 oracle against values fixed by the paper and by
mathematics (closed forms, invariants, special cases, brute force), so that a
dropped term, a wrong sign or index, or a transposed operand in ``oracle/``
fails here.  CPU only."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- RNG -----
def test_splitmix64_published_outputs():
    vals = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt"))
            if l.startswith("0x")]
    assert oracle.splitmix64_stream(0, 3) == vals


def test_cbrng_is_splitmix_stream():
    # value idx of stream (seed, ctr) is output idx+1 of a SplitMix64
    # generator started at seed ^ (first output of a generator started at ctr)
    seed, ctr = 0x1234ABCD, 7
    first_of_ctr = oracle.splitmix64_stream(ctr, 1)[0]
    outs = oracle.splitmix64_stream(seed ^ first_of_ctr, 5)
    assert [oracle.cbrng(seed, ctr, i) for i in range(5)] == outs


def test_normal_moments():
    n = 20000
    z = np.array([oracle.normal(3, 11, m) for m in range(n)])
    assert abs(z.mean()) < 4.0 / math.sqrt(n)
    assert abs(z.var() - 1.0) < 6.0 * math.sqrt(2.0 / n)
    # fourth moment of a standard normal is 3
    assert abs((z ** 4).mean() - 3.0) < 0.25


def test_pixel_set_distinct_in_range_and_full_permutation():
    for (W, H, B) in ((100, 100, 64), (7, 3, 21), (5, 5, 1), (400, 400, 16)):
        px = oracle.pixel_set(W, H, B, 9, 4)
        assert px.shape == (B, 2)
        assert np.all((px[:, 0] >= 0) & (px[:, 0] < W) & (px[:, 1] >= 0) & (px[:, 1] < H))
        q = px[:, 1] * W + px[:, 0]
        assert len(set(q.tolist())) == B
    # B = n: every pixel exactly once
    px = oracle.pixel_set(7, 3, 21, 1, 2)
    assert sorted((px[:, 1] * 7 + px[:, 0]).tolist()) == list(range(21))


def test_pixel_set_uniform_subsets():
    """Floyd's algorithm draws every B-subset with equal probability: for
    n = 5, B = 2 the 10 subsets are equally frequent (chi-square, 9 dof)."""
    from collections import Counter
    cnt = Counter()
    T = 20000
    for c in range(T):
        px = oracle.pixel_set(5, 1, 2, 77, c)
        cnt[tuple(sorted(px[:, 0].tolist()))] += 1
    assert len(cnt) == 10
    exp = T / 10
    chi2 = sum((v - exp) ** 2 / exp for v in cnt.values())
    assert chi2 < 30.0   # 99.95th percentile of chi-square(9) is ~29.7


# ----------------------------------------------------------------- PE -----
def test_pe_closed_form():
    L = 10
    g = oracle.pe([0.0, math.pi / 2, math.pi / 3], L)
    assert g.shape == (63,)
    assert np.allclose(g[:3], [0.0, math.pi / 2, math.pi / 3], atol=0)
    r3 = math.sqrt(3) / 2
    for k in range(L):
        s = g[3 + 6 * k: 6 + 6 * k]
        c = g[6 + 6 * k: 9 + 6 * k]
        # p = 0
        assert s[0] == 0.0 and c[0] == 1.0
        # p = pi/2: 2^k pi/2 is pi/2, pi, 2pi, 4pi, ...
        exp_s1 = 1.0 if k == 0 else 0.0
        exp_c1 = 0.0 if k == 0 else (-1.0 if k == 1 else 1.0)
        assert abs(s[1] - exp_s1) < 1e-12 and abs(c[1] - exp_c1) < 1e-12
        # p = pi/3: 2^k pi/3 mod 2 pi is pi/3, 2pi/3, 4pi/3, 2pi/3, 4pi/3, ...
        if k == 0:
            es, ec = r3, 0.5
        elif k % 2 == 1:
            es, ec = r3, -0.5
        else:
            es, ec = -r3, -0.5
        assert abs(s[2] - es) < 1e-11 and abs(c[2] - ec) < 1e-11


# ---------------------------------------------------------------- MLP -----
def _rand_dirs(rng, n):
    d = rng.normal(size=(n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def test_mlp_bias_only_closed_form():
    rng = np.random.default_rng(1)
    arch = synth.Arch()
    layers = {name: (None, rng.normal(size=fo)) for name, fi, fo in synth.layer_shapes(arch)}
    blob = synth.blob_from_layers(layers)
    x = rng.uniform(-3, 3, size=(5, 3))
    s, rgb = oracle.mlp(blob, x, _rand_dirs(rng, 5))
    b_sig = np.float32(layers["sigma"][1][0])
    b_rgb = layers["rgb_out"][1].astype(np.float32).astype(np.float64)
    assert np.allclose(s, float(b_sig), rtol=0, atol=1e-15)
    assert np.allclose(rgb, 1.0 / (1.0 + np.exp(-b_rgb)), rtol=0, atol=1e-15)


def handset_blob():
    """A map whose outputs have a closed form:
       sigma_raw = |x0| + relu(sin(2 x1)) + 0.5
       rgb = (sigmoid(relu(sin(2 x1))), sigmoid(2 relu(-dz)), sigmoid(-4*0.25+0.1))
    Unit 2 of trunk layer 6 reads gamma(x) entry 10 = sin(2^1 x_1) through the
    skip connection, and rgb_hidden unit 1 reads gamma(d) entry 2 = d_z."""
    a = synth.Arch()
    Wd, gx, gd, Wr = a.trunk_width, a.gx, a.gd, a.rgb_width
    L = {}
    W1 = np.zeros((Wd, gx)); W1[0, 0] = 1.0; W1[1, 0] = -1.0
    L["trunk1"] = (W1, None)
    for l in (2, 3, 4, 5, 7, 8):
        W = np.zeros((Wd, Wd)); W[0, 0] = W[1, 1] = W[2, 2] = 1.0
        L[f"trunk{l}"] = (W, None)
    W6 = np.zeros((Wd, Wd + gx)); W6[0, 0] = W6[1, 1] = 1.0; W6[2, Wd + 10] = 1.0
    L["trunk6"] = (W6, None)
    Ws = np.zeros((1, Wd)); Ws[0, :3] = 1.0
    L["sigma"] = (Ws, np.array([0.5]))
    Wf = np.zeros((Wd, Wd)); Wf[0, 2] = 1.0; Wf[1, 0] = 1.0
    bf = np.zeros(Wd); bf[2] = 0.25
    L["feature"] = (Wf, bf)
    Wh = np.zeros((Wr, Wd + gd)); Wh[0, 0] = 1.0; Wh[1, Wd + 2] = -1.0; Wh[2, 2] = 1.0
    L["rgb_hidden"] = (Wh, None)
    Wo = np.zeros((3, Wr)); Wo[0, 0] = 1.0; Wo[1, 1] = 2.0; Wo[2, 2] = -4.0
    L["rgb_out"] = (Wo, np.array([0.0, 0.0, 0.1]))
    return synth.blob_from_layers(L)


def test_mlp_handset_closed_form():
    rng = np.random.default_rng(2)
    blob = handset_blob()
    x = rng.uniform(-3, 3, size=(64, 3))
    d = _rand_dirs(rng, 64)
    s, rgb = oracle.mlp(blob, x, d)
    sig = lambda t: 1.0 / (1.0 + np.exp(-t))
    r = np.maximum(np.sin(2 * x[:, 1]), 0.0)
    assert np.allclose(s, np.abs(x[:, 0]) + r + 0.5, atol=1e-6)
    assert np.allclose(rgb[:, 0], sig(r), atol=1e-7)
    assert np.allclose(rgb[:, 1], sig(2 * np.maximum(-d[:, 2], 0.0)), atol=1e-7)
    assert np.allclose(rgb[:, 2], sig(-4 * 0.25 + np.float32(0.1)), atol=1e-7)


def test_room_map_closed_form():
    """The analytic room map through the full 8-layer trunk, skip input,
    density head, feature layer and RGB head: density 64 clamp((m - 3)/eps)
    with m = max |x_c|, colour sigmoid(a . f(x)) of the texture features."""
    from room_scene import room_rgb, room_sigma
    blob, a = synth.room_map_weights(0)
    a32 = a.astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(4)
    x = rng.uniform(-4, 4, size=(512, 3))
    x[:64] = rng.uniform(2.99, 3.02, size=(64, 3)) * rng.choice([-1, 1], size=(64, 3))
    d = _rand_dirs(rng, 512)
    s, rgb = oracle.mlp(blob, x, d)
    assert np.allclose(s, room_sigma(x, 3.0, 0.015625, 64.0), rtol=0, atol=1e-12)
    assert np.allclose(rgb, room_rgb(x, a32), rtol=0, atol=1e-12)


def test_room_render_converges_to_continuous_integral():
    """Eq. 1 quadrature with 256 coarse + 256 importance samples on the room
    map approaches the continuous rendering integral (fine trapezoid rule on
    the closed-form field): colour within 5e-3, z_trans within 2e-2 of the
    wall, and F = tau on the sharp wall."""
    from room_scene import pixel_rays, render_continuous, wall_hit
    blob, a = synth.room_map_weights(0)
    a32 = a.astype(np.float32).astype(np.float64)
    P = synth.random_particles(6, 2)[0]
    px = synth.pixel_set(6, 25, 25, 16)
    o, d = map(np.concatenate, zip(*[pixel_rays(p, 138.9 / 4, 138.9 / 4, 12.5, 12.5, px)
                                      for p in P]))
    ref, t_left = render_continuous(o, d, a32)
    assert t_left.max() < 1e-6
    r = oracle.render_rays(blob, o, d, oracle.make_opts(n_coarse=256, n_fine=256))
    assert np.abs(r["rgb"] - ref).max() < 5e-3
    assert np.abs(r["z_trans"] - wall_hit(o, d, 3.0)).max() < 2e-2
    assert np.allclose(r["F"], 0.1)


# ---------------------------------------------------------------- rays ----
def test_ray_closed_form():
    f, cx, cy = 100.0, 50.0, 40.0
    P = synth.pose_from_xyz_yaw([[1.0, 2.0, 3.0]], [0.0])[0]
    o, d = oracle.ray(P, f, f, cx, cy, 50, 40)
    assert np.allclose(o, [1, 2, 3])
    assert np.allclose(d, [0.5 / f, -0.5 / f, -1.0], atol=1e-15)
    # yaw = +90 deg about +y maps camera -z onto world -x
    P = synth.pose_from_xyz_yaw([[0.0, 0.0, 0.0]], [math.pi / 2])[0]
    o, d = oracle.ray(P, f, f, cx, cy, 60, 30)
    dc = np.array([10.5 / f, -(-9.5) / f, -1.0])
    assert np.allclose(d, [dc[2], dc[1], -dc[0]], atol=1e-15)


# ---------------------------------------------------------- compositing ---
def test_composite_constant_density_closed_form():
    n, s, dn = 32, 0.7, 1.3
    z = 2.0 + 4.0 * (np.arange(n) + 0.5) / n
    rgb = np.tile([0.2, 0.5, 0.9], (n, 1))
    w, T, C = oracle.composite(z, np.full(n, s), rgb, dn)
    assert np.allclose(T, np.exp(-s * (z - z[0]) * dn), rtol=1e-14, atol=0)
    # the last interval is 1e10 long, so all light is absorbed
    assert abs(w.sum() - 1.0) < 1e-14
    assert np.allclose(C, [0.2, 0.5, 0.9], atol=1e-14)
    w0, T0, C0 = oracle.composite(z, np.zeros(n), rgb, dn)
    assert np.all(w0 == 0) and np.all(T0 == 1) and np.all(C0 == 0)
    # negative raw density acts as zero density (ReLU)
    w1, _, _ = oracle.composite(z, np.full(n, -2.0), rgb, dn)
    assert np.all(w1 == 0)


def test_composite_invariants_random():
    rng = np.random.default_rng(3)
    for _ in range(20):
        n = int(rng.integers(2, 64))
        z = np.sort(rng.uniform(2, 6, n))
        sg = rng.normal(0, 2, n)
        w, T, C = oracle.composite(z, sg, rng.uniform(0, 1, (n, 3)), rng.uniform(1, 2))
        assert np.all(w >= 0) and w.sum() <= 1 + 1e-14
        assert np.all(np.diff(T) <= 0) and T[0] == 1.0
        assert np.all(C >= 0) and np.all(C <= 1 + 1e-14)


# ----------------------------------------------------------- Eq. 5 / F ----
def test_uncertainty_constant_density_crossings():
    n, dn, alpha, tau = 64, 1.1, 0.05, 0.1
    z = 2.0 + 4.0 * (np.arange(n) + 0.5) / n
    dz = 4.0 / n
    for s in (0.3, 1.7, 4.2, 9.0):
        w, _, _ = oracle.composite(z, np.full(n, s), np.zeros((n, 3)), dn)
        u = oracle.uncertainty(z, w, alpha, tau)
        # W_k = 1 - exp(-s (k+1) dz |d|) for k < n-1 and W_{n-1} = 1
        kt = math.ceil(math.log(1 / (1 - alpha)) / (s * dz * dn)) - 1
        ko = math.floor(math.log(1 / alpha) / (s * dz * dn)) - 1
        kt, ko = min(kt, n - 1), min(ko, n - 2)
        assert u["z_trans"] == pytest.approx(z[kt], abs=1e-12)
        assert u["z_opaque"] == pytest.approx(z[ko], abs=1e-12)
        assert u["F"] == pytest.approx(max(z[ko] - z[kt], tau), abs=1e-12)


def test_uncertainty_special_rays():
    n, alpha, tau = 16, 0.05, 0.1
    z = np.linspace(2, 6, n)
    # empty ray: no weight anywhere -> maximal penalty z_last - z_0
    u = oracle.uncertainty(z, np.zeros(n), alpha, tau)
    assert u["z_trans"] == z[0] and u["z_opaque"] == z[-1]
    assert u["F"] == pytest.approx(z[-1] - z[0])
    # sharp surface: all weight on one sample -> F = tau
    w = np.zeros(n); w[7] = 1.0
    u = oracle.uncertainty(z, w, alpha, tau)
    assert u["z_trans"] == z[7] and u["z_opaque"] == z[6] and u["F"] == tau
    # first sample already opaque
    w = np.zeros(n); w[0] = 1.0
    u = oracle.uncertainty(z, w, alpha, tau)
    assert u["z_trans"] == z[0] and u["z_opaque"] == z[0] and u["F"] == tau


def test_uncertainty_bruteforce_small_rays():
    rng = np.random.default_rng(4)
    for _ in range(500):
        n = 5
        z = np.sort(rng.uniform(2, 6, n))
        w = rng.dirichlet(np.ones(n + 1))[:n] * rng.uniform(0, 1)
        alpha, tau = float(rng.choice([0.05, 0.2])), float(rng.choice([0.01, 0.1, 1.0]))
        W = [sum(w[:k + 1]) for k in range(n)]
        trans = [z[k] for k in range(n) if W[k] >= alpha]
        opq = [z[k] for k in range(n) if W[k] <= 1 - alpha]
        zt = min(trans) if trans else z[0]
        zo = max(opq) if opq else z[0]
        u = oracle.uncertainty(z, w, alpha, tau)
        assert u["z_trans"] == zt and u["z_opaque"] == zo
        assert u["F"] == max(zo - zt, tau)


# --------------------------------------------------- importance sampling --
def test_sample_pdf_uniform_weights_even_spacing():
    nc, nf = 64, 128
    z = 2.0 + 4.0 * (np.arange(nc) + 0.5) / nc
    zf = oracle.sample_pdf(z, np.full(nc, 0.3), nf)
    mids = 0.5 * (z[1:] + z[:-1])
    assert np.allclose(zf, np.linspace(mids[0], mids[-1], nf), atol=1e-12)


def test_sample_pdf_spike_and_monotone():
    nc, nf = 32, 64
    z = 2.0 + 4.0 * (np.arange(nc) + 0.5) / nc
    mids = 0.5 * (z[1:] + z[:-1])
    w = np.zeros(nc); w[10] = 1.0
    zf = oracle.sample_pdf(z, w, nf)
    inside = (zf >= mids[9]) & (zf <= mids[10])
    # 1e-5 floor: each of the 29 other bins holds ~1e-5 of the mass
    assert inside.sum() >= nf - 2
    rng = np.random.default_rng(5)
    for _ in range(20):
        zf = oracle.sample_pdf(z, rng.exponential(size=nc), nf)
        assert np.all(np.diff(zf) >= 0)
        assert zf[0] == pytest.approx(mids[0]) and zf[-1] == pytest.approx(mids[-1])


# ----------------------------------------------------------- weighting ----
SMALL = dict(n_coarse=16, n_fine=16)


# He-init map seed whose density is positive on roughly 80 % of space (the
# global sign of a zero-bias He-init density head depends on the seed).
MAP_SEED = 2


def _scene(seed, N, B, W=40, H=40, f=55.0, factor=1, opts=None):
    blob = synth.he_init_weights(MAP_SEED)
    P, _, _ = synth.random_particles(seed, N)
    gt, _, _ = synth.gt_pose(seed)
    P = np.concatenate([P, gt[None]], 0)
    K4 = (f, f, W / 2, H / 2)
    px = synth.pixel_set(seed, W // factor, H // factor, B)
    opts = opts or oracle.make_opts(**SMALL)
    cols = oracle.render_observation_pixels(blob, gt, K4, factor, px, opts)
    img = oracle.paint_pixels(synth.smooth_image(seed, W, H), px, factor, cols)
    return blob, P, img, K4, px, opts


@pytest.mark.parametrize("factor", [1, 2])
def test_gt_particle_zero_loss_max_weight(factor):
    blob, P, img, K4, px, opts = _scene(11, 6, 8, factor=factor)
    r = oracle.update(blob, P, img, K4, factor, px, opts)
    assert r["S"][-1] == 0.0
    assert np.argmax(r["w"]) == len(P) - 1
    assert r["w"][-1] > 0.999 and r["mask"][-1] == 1
    assert abs(r["w"].sum() - 1.0) < 1e-14


def test_tau_large_equals_no_rejection():
    blob, P, img, K4, px, _ = _scene(12, 6, 8)
    P = P[:-1]  # without the GT particle every S is positive
    a = oracle.update(blob, P, img, K4, 1, px, oracle.make_opts(tau=10.0, **SMALL))
    b = oracle.update(blob, P, img, K4, 1, px, oracle.make_opts(use_rejection=False, **SMALL))
    assert np.all(a["F"] == 10.0) and np.all(b["F"] == 1.0)
    assert np.allclose(a["w"], b["w"], rtol=1e-12, atol=1e-300)


def test_weights_closed_form_and_permutation():
    blob, P, img, K4, px, opts = _scene(13, 3, 8)
    P = P[:-1]
    r = oracle.update(blob, P, img, K4, 1, px, opts)
    # Eq. 6: w_i proportional to (B / S_i)^4, normalised to sum 1
    S = r["S"]
    assert np.allclose(r["w"], S ** -4 / np.sum(S ** -4), rtol=1e-12)
    assert np.allclose(r["logw"], 4 * np.log(8 / S), rtol=1e-14)
    perm = np.array([2, 0, 1])
    rp = oracle.update(blob, P[perm], img, K4, 1, px, opts)
    assert np.allclose(rp["w"], r["w"][perm], rtol=1e-13)
    assert np.allclose(rp["S"], S[perm], rtol=1e-13)


def test_weights_invariant_to_repeating_the_pixel_set():
    """Eq. 6: every pixel taken twice doubles B and every S_i, so the
    log-weights 4 (log B - log S_i) and the normalised weights are unchanged
    (scale invariance of the normalisation)."""
    blob, P, img, K4, px, opts = _scene(16, 4, 8)
    P = P[:-1]
    r1 = oracle.update(blob, P, img, K4, 1, px, opts)
    r2 = oracle.update(blob, P, img, K4, 1, np.concatenate([px, px]), opts)
    assert np.allclose(r2["S"], 2 * r1["S"], rtol=1e-14)
    assert np.allclose(r2["logw"], r1["logw"], rtol=1e-13, atol=1e-13)
    assert np.allclose(r2["w"], r1["w"], rtol=1e-12, atol=1e-300)


def test_update_matches_rendered_rays():
    """S_i is the sum over j of E_ij F_ij with E the squared RGB distance."""
    blob, P, img, K4, px, opts = _scene(14, 2, 4)
    r = oracle.update(blob, P, img, K4, 1, px, opts)
    o, d = [], []
    for i in range(len(P)):
        for (u, v) in px:
            oo, dd = oracle.ray(P[i], *K4, u, v)
            o.append(oo); d.append(dd)
    rr = oracle.render_rays(blob, np.array(o), np.array(d), opts)
    assert np.array_equal(rr["rgb"], r["rgb"])
    obs = img[px[:, 1], px[:, 0]]
    E = ((np.tile(obs, (len(P), 1)) - rr["rgb"]) ** 2).sum(1)
    assert np.allclose(E, r["E"], rtol=1e-14, atol=0)
    assert np.allclose((E * rr["F"]).reshape(len(P), -1).sum(1), r["S"], rtol=1e-14)


def test_nonfinite_particle_gets_no_weight():
    blob, P, img, K4, px, opts = _scene(15, 4, 8)
    P = P[:-1].copy()
    P[2, 3] = np.nan
    r = oracle.update(blob, P, img, K4, 1, px, opts)
    assert not np.isfinite(r["S"][2]) and r["logw"][2] == -np.inf
    assert r["w"][2] == 0.0 and r["mask"][2] == 0
    assert abs(r["w"].sum() - 1.0) < 1e-14


def test_downscale_closed_forms():
    img = np.full((8, 12, 3), 0.37)
    assert np.allclose(oracle.downscale(img, 4), 0.37)
    yy, xx = np.meshgrid(np.arange(8.0), np.arange(12.0), indexing="ij")
    ramp = np.stack([xx, yy, 2 * xx + 3 * yy], -1)
    d = oracle.downscale(ramp, 2)
    cy, cx = np.meshgrid(np.arange(4) * 2 + 0.5, np.arange(6) * 2 + 0.5, indexing="ij")
    assert np.allclose(d, np.stack([cx, cy, 2 * cx + 3 * cy], -1), atol=1e-14)


# ----------------------------------------------------------- resampling ---
def _systematic_exact(w, n_out, u0):
    """Definition: index k is the smallest i with (sum_{m<=i} w_m) / sum(w)
    > (k + u0) / n_out, in exact rational arithmetic."""
    wf = [Fraction(x) for x in w]
    tot = sum(wf)
    cdf, run = [], Fraction(0)
    for x in wf:
        run += x
        cdf.append(run / tot)
    out = []
    for k in range(n_out):
        pos = (k + Fraction(u0)) / n_out
        out.append(next(i for i, c in enumerate(cdf) if c > pos))
    return out


def test_resample_bruteforce_dyadic():
    rng = np.random.default_rng(6)
    for trial in range(300):
        n_in = int(rng.integers(1, 7))
        n_out = int(rng.integers(1, 9))
        w = synth.random_weights(trial, n_in, dyadic_bits=4, zero_frac=0.3)
        u0 = float(rng.integers(0, 64)) / 64.0
        got = oracle.resample(w, n_out, u0).tolist()
        assert got == _systematic_exact(w, n_out, u0), (w, n_out, u0)


def test_resample_large_n_out_exact_integers():
    """N_out in the thousands (k 2^53 exceeds 64 bits): the definition
    evaluated in exact integers for dyadic weights and a dyadic u0."""
    for n_in, n_out, seed in ((5, 3000, 1), (40, 65536, 2), (7, 2049, 3)):
        w = synth.random_weights(seed, n_in, dyadic_bits=6, zero_frac=0.2)
        a = seed * 13 % 64                       # u0 = a / 64
        q = [int(x) for x in w]                  # integer weights (dyadic, scaled)
        C, run = [], 0
        for x in q:
            run += x
            C.append(run)
        T = C[-1]
        # smallest i with C_i / T > (k + a/64) / n_out  <=>  64 C_i n_out > (64 k + a) T
        exp_idx = [next(i for i, c in enumerate(C) if 64 * c * n_out > (64 * k + a) * T)
                   for k in range(n_out)]
        got = oracle.resample(w, n_out, a / 64.0).tolist()
        assert got == exp_idx


def test_resample_copy_counts_large():
    w = synth.random_weights(17, 300)
    for n in (4000, 65536):
        cnt = np.bincount(oracle.resample(w, n, 0.61803), minlength=300)
        assert cnt.sum() == n
        assert np.all(cnt >= np.floor(n * w) - 1e-9) and np.all(cnt <= np.ceil(n * w) + 1e-9)


def test_resample_copy_counts_and_frequencies():
    w = synth.random_weights(7, 50)
    n = 50
    cnt = np.bincount(oracle.resample(w, n, 0.3719), minlength=n)
    assert np.all(cnt >= np.floor(n * w) - 1e-9) and np.all(cnt <= np.ceil(n * w) + 1e-9)
    acc = np.zeros(n)
    grid = (np.arange(500) + 0.5) / 500
    for u0 in grid:
        acc += np.bincount(oracle.resample(w, n, u0), minlength=n)
    assert np.allclose(acc / len(grid), n * w, atol=2.0 / len(grid) + 1e-9)


def test_resample_zero_weights_never_drawn_and_errors():
    w = np.array([0.0, 0.5, 0.0, 0.5])
    idx = oracle.resample(w, 1000, 0.123)
    assert set(idx.tolist()) == {1, 3}
    with pytest.raises(ValueError):
        oracle.resample(np.zeros(4), 4, 0.5)
    with pytest.raises(ValueError):
        oracle.resample(np.array([1.0, np.nan]), 4, 0.5)


# ------------------------------------------------------------- motion -----
def _twist(rho, om):
    M = np.zeros((4, 4))
    M[0, 1], M[0, 2], M[1, 2] = -om[2], om[1], -om[0]
    M[1, 0], M[2, 0], M[2, 1] = om[2], -om[1], om[0]
    M[:3, 3] = rho
    return M


def test_se3_exp_against_matrix_exponential():
    from scipy.linalg import expm
    rng = np.random.default_rng(8)
    for _ in range(50):
        rho = rng.normal(size=3)
        om = rng.normal(size=3) * rng.choice([1e-10, 1e-3, 1.0, 3.0])
        M = oracle.se3_exp(rho, om)
        ref = expm(_twist(rho, om))[:3]
        assert np.allclose(M, ref, atol=1e-12)


def test_predict_identity_and_inverse():
    P, _, _ = synth.random_particles(9, 10)
    assert np.array_equal(oracle.predict(P, np.zeros((10, 4))), P)
    q = np.random.default_rng(9).normal(0, 0.1, (10, 4))
    back = oracle.predict(oracle.predict(P, q), -q)
    assert np.allclose(back, P, atol=1e-14)
    # a pure yaw turns the camera about the world +y axis and keeps t
    yaw = np.zeros((10, 4)); yaw[:, 3] = 0.3
    Q = oracle.predict(P, yaw).reshape(10, 3, 4)
    R0 = P.reshape(10, 3, 4)
    Ry = synth.pose_from_xyz_yaw([[0, 0, 0]], [0.3])[0].reshape(3, 4)[:, :3]
    assert np.allclose(Q[:, :, :3], R0[:, :, :3] @ Ry, atol=1e-14)
    assert np.allclose(Q[:, :, 3], R0[:, :, 3], atol=1e-15)


def test_predict_with_odometry_matrix_product():
    """x_t = x_{t-1} O_t Exp(delta) (Sec. III-A): against 4x4 homogeneous
    products with scipy's matrix exponential of the noise twist."""
    from scipy.linalg import expm
    rng = np.random.default_rng(21)
    P, _, _ = synth.random_particles(21, 12)
    O = synth.pose_from_xyz_yaw([[0.3, -0.1, 0.2]], [0.4])[0]
    q = rng.normal(0, 0.1, (12, 4))
    out = oracle.predict(P, q, odom=O)
    h = lambda m: np.vstack([np.reshape(m, (3, 4)), [0, 0, 0, 1]])
    for i in range(12):
        ref = h(P[i]) @ h(O) @ expm(_twist(q[i, :3], np.array([0.0, q[i, 3], 0.0])))
        assert np.allclose(out[i], ref[:3].reshape(12), atol=1e-13)
    # zero noise: the pure odometry step, and the identity odometry is the default
    assert np.allclose(oracle.predict(P, np.zeros((12, 4)), odom=O),
                       np.stack([(h(P[i]) @ h(O))[:3].reshape(12) for i in range(12)]), atol=1e-14)
    assert np.array_equal(oracle.predict(P, q, odom=np.eye(4)[:3].reshape(12)), oracle.predict(P, q))


def test_position_spread_closed_form():
    P = synth.pose_from_xyz_yaw([[0, 0, 0], [2, 0, 0], [0, 4, 0]], [0, 1, 2])
    s = oracle.position_spread(P)
    assert np.allclose(s["mean"], [2 / 3, 4 / 3, 0])
    # trace of the population covariance
    xs = np.array([[0, 0, 0], [2, 0, 0], [0, 4, 0]], dtype=float)
    assert s["trace"] == pytest.approx(((xs - xs.mean(0)) ** 2).sum() / 3)


# ----------------------------------------------------- proposal sampler ---
def _prop_rays(seed, n):
    rng = np.random.default_rng(seed)
    o = rng.uniform(-1, 1, size=(n, 3))
    d = rng.normal(size=(n, 3))
    d[:, 2] = -np.abs(d[:, 2]) - 0.5
    return o, d


def test_proposal_blob_size():
    assert oracle.prop_n_weights() == synth.proposal_n_weights() == 15105


def test_histogram_closed_form():
    z = np.array([2.05, 2.2, 3.9, 4.1, 5.99, 6.5, 1.0])
    w = np.array([0.1, 0.2, 0.3, 0.1, 0.2, 0.05, 0.05])
    h = oracle.histogram(z, w, 4, 2.0, 6.0)
    # bins [2,3) [3,4) [4,5) [5,6]; z = 6.5 clamps to the last, z = 1 to the first
    assert np.allclose(h, np.array([0.1 + 0.2 + 0.05, 0.3, 0.1, 0.2 + 0.05]) / 1.0)
    assert np.allclose(oracle.histogram(z, np.zeros(7), 4, 2.0, 6.0), 0.25)


def test_proposal_constant_density_loss_closed_form():
    """All weights zero and head bias b: density b everywhere, so the
    composite weights and the cross-entropy have a closed form."""
    b, nb = float(np.float32(0.8)), 16
    blob = np.zeros(15105, dtype=np.float32)
    blob[-1] = b
    o, d = _prop_rays(1, 3)
    rng = np.random.default_rng(2)
    hist = rng.dirichlet(np.ones(nb), size=3)
    loss, grad = oracle.prop_loss_grad(blob, o, d, hist)
    ref = 0.0
    for r in range(3):
        dz = 4.0 / nb * np.linalg.norm(d[r])
        k = np.arange(nb)
        w = np.exp(-b * dz * k) * (1 - np.exp(-b * dz))
        w[-1] = np.exp(-b * dz * (nb - 1))
        ref += -(hist[r] * np.log(w / w.sum() + 1e-8)).sum()
    assert loss == pytest.approx(ref / 3, rel=1e-12)
    # zero network weights: only the head bias gets a gradient
    assert np.all(grad[:-1] == 0.0) and grad[-1] != 0.0


def test_proposal_gradient_matches_finite_differences():
    """Analytic gradient (through the ReLU layers and the Eq. 1 compositing)
    against central differences of the loss, in FP64 on an FP32 blob (the
    step is the exact difference of the two FP32-rounded parameters)."""
    base = synth.proposal_init_weights(3)
    o, d = _prop_rays(4, 2)
    rng = np.random.default_rng(5)
    hist = rng.dirichlet(np.ones(16), size=2)
    f = lambda b: oracle.prop_loss_grad(b, o, d, hist, with_grad=False)[0]
    _, g = oracle.prop_loss_grad(base, o, d, hist)
    idx = np.concatenate([rng.choice(15105, 60, replace=False), [15104, 15103, 0, 2559]])
    checked = 0
    for i in idx:
        h = np.float32(2.0 ** -14 * max(1.0, abs(float(base[i]))))
        bp, bm = base.copy(), base.copy()
        bp[i] = np.float32(base[i] + h)
        bm[i] = np.float32(base[i] - h)
        fd = (f(bp) - f(bm)) / (float(bp[i]) - float(bm[i]))
        # a ReLU kink inside [-h, h] makes the difference quotient one-sided;
        # such parameters are detected by comparing the two one-sided slopes
        f0 = f(base)
        sp = (f(bp) - f0) / (float(bp[i]) - float(base[i]))
        sm = (f0 - f(bm)) / (float(base[i]) - float(bm[i]))
        if abs(sp - sm) > 1e-3 * max(1e-3, abs(sp)):
            continue
        assert abs(fd - g[i]) <= 1e-5 * max(1e-3, abs(g[i])) + 1e-9, (i, fd, g[i])
        checked += 1
    assert checked >= 50


def test_proposal_weights_sum_to_at_most_one():
    blob = synth.proposal_init_weights(6)
    o, d = _prop_rays(7, 5)
    w = oracle.prop_weights(blob, o, d, 64)
    assert np.all(w >= 0) and np.all(w.sum(1) <= 1 + 1e-12)
