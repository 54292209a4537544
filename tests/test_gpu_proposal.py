"""GPU parity of the learned proposal sampler (a project extension; the paper
samples with the basic model's coarse pass): the distillation targets, the
loss and its gradient against the FP64 oracle, rendering with
proposal-guided samples, and the effect of training (loss falls; at an equal
budget of NeRF evaluations the proposal sampler lands closer to the full
hierarchical sampler than the coarse pass it replaces)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import K_ULP, lib

pytestmark = pytest.mark.gpu

NEAR, FAR = 2.0, 6.0
ULP_Z = 4.8e-7   # one FP32 ulp of z in [4, 8)


@pytest.fixture(scope="module")
def M():
    return lib()


@pytest.fixture(scope="module")
def gmap(M):
    m = M.Map(synth.he_init_weights(2), max_rays=70000, max_samples=192, max_particles=4096)
    yield m
    m.close()


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def random_rays(seed, n):
    """Origins in [-1, 1]^3, directions of norm 1 .. 1.3 (pixel rays of a
    camera with focal ~ image size have |d| in that range)."""
    rng = np.random.default_rng(seed)
    o = rng.uniform(-1.0, 1.0, (n, 3))
    d = rng.normal(size=(n, 3))
    d *= rng.uniform(1.0, 1.3, (n, 1)) / np.linalg.norm(d, axis=1, keepdims=True)
    return f32(o), f32(d)


def level_rays(P, K4, factor, px):
    """Oracle rays (o, d) of poses x pixels in (pose, pixel) order."""
    fx, fy, cx, cy = oracle.level_intrinsics(K4, factor)
    o, d = [], []
    for pose in P:
        for u, v in px:
            a, b = oracle.ray(pose, fx, fy, cx, cy, int(u), int(v))
            o.append(a)
            d.append(b)
    return np.array(o), np.array(d)


def scene(seed, N, B, W=100, H=100, focal=138.9, level=2):
    P = f32(synth.random_particles(seed, N)[0])
    factor = 4 >> level
    px = synth.pixel_set(seed, W // factor, H // factor, B)
    K4 = tuple(float(np.float32(k)) for k in (focal, focal, W / 2, H / 2))
    return P, px, K4, factor, level, W, H


def gpu_inputs(M, P, px, K4, W, H):
    import torch
    Pt = torch.tensor(P, dtype=torch.float32, device="cuda")
    pxt = torch.tensor(px, dtype=torch.int32, device="cuda")
    K = M.intrinsics(*K4, W, H)
    return Pt, pxt, K


# ----------------------------------------------------------------- loss, grad
@pytest.mark.parametrize("pseed,nb", [(3, 32), (4, 64)])
def test_loss_and_gradient_match_oracle(M, gmap, pseed, nb):
    """Mean cross-entropy and its gradient w.r.t. all 15105 proposal weights
    against the oracle's FP64 chain rule.  Bars: the loss to 1e-5 relative
    (FP32 log of normalised weights); the gradient to 1e-3 of its norm and
    elementwise to 2e-3 of its largest entry: FP32 accumulation over 64-wide
    dot products and thousands of rows stays near 1e-5, and a ReLU
    pre-activation within FP32 rounding of 0 switches one row's
    contribution to one unit (one row in n * nb)."""
    import torch
    pblob = synth.proposal_init_weights(pseed)
    gmap.proposal_set(pblob)
    n = 96
    o, d = random_rays(pseed, n)
    rng = np.random.default_rng(pseed + 100)
    hist = rng.gamma(0.5, size=(n, nb))
    hist[::7] = 0.0
    hist[::7, rng.integers(0, nb)] = 1.0          # one-hot targets too
    hist = f32(hist / hist.sum(1, keepdims=True))
    L_o, g_o = oracle.prop_loss_grad(pblob, o, d, hist, NEAR, FAR)
    t = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")
    L_g, g_g = gmap.proposal_loss_grad(t(o), t(d), t(hist), NEAR, FAR)
    g_g = g_g.cpu().numpy().astype(np.float64)
    assert abs(L_g - L_o) <= 1e-5 * abs(L_o), (L_g, L_o)
    rel = np.linalg.norm(g_g - g_o) / np.linalg.norm(g_o)
    assert rel <= 1e-3, rel
    assert np.abs(g_g - g_o).max() <= 2e-3 * np.abs(g_o).max()


def test_zero_density_ray_has_no_gradient(M, gmap):
    """A proposal with density <= 0 everywhere (head bias -100, head weights
    0): every ray has W = 0, loss -log(1e-8) per unit of target mass, no
    gradient (the density ReLU is closed)."""
    import torch
    pblob = synth.proposal_init_weights(1).astype(np.float64)
    pblob[-65:-1] = 0.0
    pblob[-1] = -100.0
    pblob = pblob.astype(np.float32)
    gmap.proposal_set(pblob)
    n, nb = 8, 16
    o, d = random_rays(7, n)
    hist = np.full((n, nb), 1.0 / nb)
    t = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")
    L_g, g_g = gmap.proposal_loss_grad(t(o), t(d), t(hist), NEAR, FAR)
    assert abs(L_g + np.log(1e-8)) < 1e-6 * abs(np.log(1e-8))
    assert not g_g.any()


# ------------------------------------------------------------------- targets
@pytest.mark.parametrize("nf,nb", [(0, 16), (32, 64)])
def test_histogram_targets_match_oracle(M, gmap, nf, nb):
    """Re-binned final weights of the full sampler (GPU FP32 form) against
    the oracle's histogram of its own FP64 render.  Without importance
    samples the sample positions are exact midpoints that never sit on a bin
    boundary, so the bar is 1e-4 absolute.  With importance samples it adds
    K_ULP times the oracle's own change when every coarse z moves by one
    FP32 ulp."""
    P, px, K4, factor, level, W, H = scene(11, 8, 16)
    Pt, pxt, K = gpu_inputs(M, P, px, K4, W, H)
    opts = M.UpdateOptions(n_coarse=32, n_fine=nf, precision="fp32")
    h_g = gmap.render_histogram(Pt, K, level, pxt, opts, nb).cpu().numpy().astype(np.float64)
    o, d = level_rays(P, K4, factor, px)
    oo = oracle.make_opts(n_coarse=32, n_fine=nf)
    blob = synth.he_init_weights(2)

    def hist_of(uj):
        r = oracle.render_rays(blob, o, d, oo, uj=uj, debug=True)
        return np.array([oracle.histogram(r["z"][i], r["w"][i], nb, NEAR, FAR)
                         for i in range(len(o))])
    base = np.full((len(o), 32), 0.5)
    h_o = hist_of(base)
    tol = 1e-4
    if nf > 0:
        tol += K_ULP * np.abs(hist_of(base + ULP_Z / ((FAR - NEAR) / 32)) - h_o).max()
    assert np.allclose(h_g.sum(1), 1.0, atol=1e-5)
    assert np.abs(h_g - h_o).max() <= tol, (np.abs(h_g - h_o).max(), tol)


# ----------------------------------------------------------------- rendering
def test_proposal_render_matches_oracle(M, gmap):
    """Colour and F of rays rendered with proposal samples (32 stratified
    proposal samples -> 16 guided -> 16 importance samples) against the
    oracle.  Guided and importance positions come from inverse CDFs, so the
    RGB bar is 1e-4 relative plus K_ULP times the oracle's own change when
    every proposal sample moves by one FP32 ulp; F may move by two decision
    steps."""
    import torch
    pblob = synth.proposal_init_weights(5)
    gmap.proposal_set(pblob)
    P, px, K4, factor, level, W, H = scene(12, 8, 16)
    Pt, pxt, K = gpu_inputs(M, P, px, K4, W, H)
    opts = M.UpdateOptions(n_coarse=32, n_fine=16, precision="fp32", use_proposal=True,
                           n_proposal=32, n_guided=16)
    rgb_g, F_g = gmap.render(Pt, K, level, pxt, opts, with_F=True)
    torch.cuda.synchronize()
    rgb_g = rgb_g.cpu().numpy().astype(np.float64)
    F_g = F_g.cpu().numpy().astype(np.float64)
    o, d = level_rays(P, K4, factor, px)
    blob = synth.he_init_weights(2)
    r = oracle.render_rays_proposal(blob, pblob, o, d, oracle.make_opts(n_coarse=32, n_fine=16),
                                    n_p=32, n_g=16)
    r2 = oracle.render_rays_proposal(blob, pblob, o, d,
                                     oracle.make_opts(n_coarse=32, n_fine=16, near=NEAR + ULP_Z,
                                                      far=FAR + ULP_Z), n_p=32, n_g=16)
    sens = np.abs(r2["rgb"] - r["rgb"]).max()
    tol = 1e-4 * np.abs(r["rgb"]) + max(1e-6, K_ULP * sens)
    err = np.abs(rgb_g - r["rgb"])
    assert np.all(err <= tol), (err.max(), sens)
    f_allow = 2.0 * r["step"] + 2e-5
    assert np.all(np.abs(F_g - r["F"]) <= f_allow * (1 + 1e-6))


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_proposal_densities_vs_oracle(M, gmap, prec):
    """Raw proposal density at points: the FP32 kernel to 1e-4 relative
    (floor 1e-5), the tensor-core kernel (BF16 operands, FP32 accumulation,
    used by the BF16 and FP8 forms) within 0.05 max / 0.01 mean of the
    density spread (8 significant bits through four layers)."""
    import torch
    pblob = synth.proposal_init_weights(6)
    gmap.proposal_set(pblob)
    rng = np.random.default_rng(31)
    x = f32(rng.uniform(-7, 7, size=(4099, 3)))
    s_g = gmap.proposal_query(torch.tensor(x, dtype=torch.float32, device="cuda"), prec)
    s_g = s_g.cpu().numpy().astype(np.float64)
    s_o = oracle.prop_forward(pblob, x)
    if prec == "fp32":
        assert np.all(np.abs(s_g - s_o) <= 1e-4 * np.abs(s_o) + 1e-5)
    else:
        e = np.abs(s_g - s_o) / np.std(s_o)
        assert e.max() <= 0.05 and e.mean() <= 0.01, (e.max(), e.mean())


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_proposal_render_tensor_core_forms_vs_oracle(M, gmap, prec):
    """BF16 / FP8 forms: the proposal runs on the tensor cores in BF16 and
    the NeRF MLP in the form's precision.  The guided samples follow the
    inverse CDF of the rounded proposal weights, so besides the MLP's own
    rounding every guided position moves by a fraction of its bin: bars are
    twice the plain forms' rendered bars with importance samples (BF16: max
    0.16, mean 0.03; FP8: max 0.24, mean 0.04), on rays away from the flip
    band of the seed-2 map."""
    import torch
    pblob = synth.proposal_init_weights(5)
    gmap.proposal_set(pblob)
    P, px, K4, factor, level, W, H = scene(12, 8, 16)
    Pt, pxt, K = gpu_inputs(M, P, px, K4, W, H)
    opts = M.UpdateOptions(n_coarse=32, n_fine=16, precision=prec, use_proposal=True,
                           n_proposal=32, n_guided=16)
    rgb_g = gmap.render(Pt, K, level, pxt, opts).cpu().numpy().astype(np.float64)
    torch.cuda.synchronize()
    o, d = level_rays(P, K4, factor, px)
    r = oracle.render_rays_proposal(synth.he_init_weights(2), pblob, o, d,
                                    oracle.make_opts(n_coarse=32, n_fine=16), n_p=32, n_g=16)
    band = 0.1 if prec == "bf16" else 0.6
    flip = (np.abs(r["sigma_last"]) < band) & (r["T_last"] > 1e-3)
    e = np.abs(rgb_g - r["rgb"])[~flip]
    mx, mn = (0.16, 0.03) if prec == "bf16" else (0.24, 0.04)
    assert flip.mean() <= 0.5 and np.all(np.isfinite(rgb_g))
    assert e.max() <= mx and e.mean() <= mn, (e.max(), e.mean(), flip.mean())


def test_proposal_options_are_checked(M):
    """use_proposal without proposal weights, and sample counts beyond the
    workspace, are argument errors."""
    import torch
    m = M.Map(synth.he_init_weights(2), max_rays=256, max_samples=64)
    try:
        P, px, K4, factor, level, W, H = scene(1, 2, 4)
        Pt, pxt, K = gpu_inputs(M, P, px, K4, W, H)
        opts = M.UpdateOptions(n_coarse=16, n_fine=16, use_proposal=True, n_proposal=32,
                               n_guided=16)
        with pytest.raises(M.MclError) as e:
            m.render(Pt, K, level, pxt, opts)
        assert e.value.code == M.MCL_ERR_ARG
        m.proposal_set(synth.proposal_init_weights(0))
        m.render(Pt, K, level, pxt, opts)
        for bad in (dict(n_guided=64), dict(n_proposal=1), dict(n_proposal=300)):
            o2 = M.UpdateOptions(n_coarse=16, n_fine=16, use_proposal=True, n_proposal=32,
                                 n_guided=16)
            for k, v in bad.items():
                setattr(o2, k, v)
            with pytest.raises(M.MclError):
                m.render(Pt, K, level, pxt, o2)
        with pytest.raises(M.MclError):
            m.proposal_set(np.zeros(10, np.float32))
        back = m.proposal_get()
        assert np.array_equal(back, synth.proposal_init_weights(0))
    finally:
        m.close()
        torch.cuda.synchronize()


# ------------------------------------------------------------------ training
@pytest.fixture(scope="module")
def room(M):
    """The analytic room map (sharp textured walls): sampling matters there."""
    blob, _ = synth.room_map_weights(0)
    m = M.Map(blob, max_rays=70000, max_samples=192, max_particles=4096)
    yield m, blob
    m.close()


@pytest.fixture(scope="module")
def trained(M, room):
    """Distil a proposal from the full 64 + 128 sampler over 256 random
    poses x 64 pixels of the 25 x 25 level of a 100 x 100 image."""
    m, _ = room
    P, px, K4, factor, level, W, H = scene(21, 256, 64, level=0)
    Pt, pxt, K = gpu_inputs(M, P, px, K4, W, H)
    m.proposal_set(synth.proposal_init_weights(0))
    full = M.UpdateOptions(n_coarse=64, n_fine=128, precision="fp32")
    log = m.proposal_train(Pt, pxt, K, level, full, epochs=40, batch_rays=2048, n_bins=64,
                           lr=3e-3, lr_end=1e-4, seed=1)
    return log, m.proposal_get()


def test_training_reduces_loss(M, trained):
    """Cross-entropy per ray starts above that of a uniform proposal
    (log 64 = 4.16 nats) and ends far below it: the walls' weight falls in
    one or two of the 64 bins."""
    log, pblob = trained
    assert np.all(np.isfinite(log)) and np.isfinite(pblob).all()
    assert log[0] > 0.8 * np.log(64)
    assert log[-1] < 0.25 * log[0], log


@pytest.mark.parametrize("n_main", [32, 16])
def test_trained_proposal_beats_coarse_pass_at_equal_budget(M, room, trained, n_main):
    """On held-out poses, n proposal-guided + n importance samples land
    closer (mean RGB error) to the oracle's full 64 + 128 sampler than n
    coarse + n importance samples: the same 2n NeRF evaluations per ray.
    The bar asks for half the error."""
    import torch
    m, blob = room
    _, pblob = trained
    m.proposal_set(pblob)
    P, px, K4, factor, level, W, H = scene(33, 32, 16, level=0)
    Pt, pxt, K = gpu_inputs(M, P, px, K4, W, H)
    o, d = level_rays(P, K4, factor, px)
    ref = oracle.render_rays(blob, o, d, oracle.make_opts(n_coarse=64, n_fine=128))["rgb"]
    plain = M.UpdateOptions(n_coarse=n_main, n_fine=n_main, precision="fp32")
    prop = M.UpdateOptions(n_coarse=n_main, n_fine=n_main, precision="fp32", use_proposal=True,
                           n_proposal=64, n_guided=n_main)
    e_plain = np.abs(m.render(Pt, K, level, pxt, plain).cpu().numpy() - ref).mean()
    e_prop = np.abs(m.render(Pt, K, level, pxt, prop).cpu().numpy() - ref).mean()
    torch.cuda.synchronize()
    assert e_prop < 0.5 * e_plain, (e_prop, e_plain)


def test_training_is_deterministic(M, room):
    """Gradients are reduced in a fixed order: the same inputs and seed give
    bit-identical weights."""
    m, _ = room
    P, px, K4, factor, level, W, H = scene(5, 32, 16, level=0)
    Pt, pxt, K = gpu_inputs(M, P, px, K4, W, H)
    full = M.UpdateOptions(n_coarse=32, n_fine=32, precision="fp32")
    out = []
    for _ in range(2):
        m.proposal_set(synth.proposal_init_weights(2))
        m.proposal_train(Pt, pxt, K, level, full, epochs=3, batch_rays=128, n_bins=32, lr=1e-3,
                         seed=4)
        out.append(m.proposal_get())
    assert np.array_equal(out[0], out[1])
    assert not np.array_equal(out[0], synth.proposal_init_weights(2))
