"""Map fitting (mcl_fit_map, mcl_map_loss_grad, mcl_get_map_weights).

The gradient of the fitting loss
  L = mean_p  w_s (sigma_raw(x_p) - sigma_p)^2 + |rgb(x_p, d_p) - rgb_p|^2
from the library's FP32 backward kernels is compared with central finite
differences of the same loss evaluated by the FP64 oracle (oracle.mlp, the
plain layer structure of Sec. III-A's network), at weights sampled from every
layer.  The fitted weights, read back in the blob layout, are checked by the
oracle against the library's own FP32 and BF16 queries (the tensor-core forms
are rebuilt from them), and the fit is deterministic."""
import numpy as np
import pytest

from gpu_helpers import lib

pytestmark = pytest.mark.gpu

WS = 1e-2     # weight of the density term


@pytest.fixture(scope="module")
def M():
    return lib()


def _points(n, seed):
    import synth
    x, d = synth.room_fit_points(seed, n)
    sig, rgb = synth.room_field(x)
    return x, d, np.concatenate([sig[:, None], rgb], 1).astype(np.float32)


def _oracle_loss(blob, x, dhat, tgt):
    import oracle
    s, c = oracle.mlp(blob, x, dhat)
    return float(np.mean(WS * (s - tgt[:, 0]) ** 2 + ((c - tgt[:, 1:]) ** 2).sum(1)))


def _unit(d):
    d = d.astype(np.float64)
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def test_loss_grad_matches_fp64_finite_differences(M):
    import torch
    import synth
    n = 256
    x, d, tgt = _points(n, 11)
    blob = synth.he_init_weights(4, bias_std=0.05)
    gm = M.Map(blob, max_rays=1024)
    try:
        loss, g = gm.loss_grad(torch.tensor(x, device="cuda"), torch.tensor(d, device="cuda"),
                               torch.tensor(tgt, device="cuda"), sigma_weight=WS)
        g = g.cpu().numpy().astype(np.float64)
    finally:
        gm.close()
    b64 = blob.astype(np.float64)
    xd, dd, td = x.astype(np.float64), _unit(d), tgt.astype(np.float64)
    ref = _oracle_loss(b64, xd, dd, td)
    assert abs(loss - ref) <= 1e-5 * ref, (loss, ref)
    rng = np.random.default_rng(5)
    rows = []
    for name, (ow, ob, fi, fo) in synth.blob_offsets().items():
        # per layer: the two largest-gradient weights, two random weights, a bias
        gw = np.abs(g[ow:ob])
        picks = list(ow + np.argsort(-gw)[:2]) + list(ow + rng.integers(0, fi * fo, 2))
        picks.append(ob + int(rng.integers(0, fo)))
        scale = max(gw.max(), np.abs(g[ob:ob + fo]).max())
        for i in picks:
            # the blob format is FP32: step to the FP32 neighbours of w +- h
            # and divide by the step actually taken
            h = 1e-5 * max(1.0, abs(b64[i]))
            wp, wm = float(np.float32(b64[i] + h)), float(np.float32(b64[i] - h))
            bp, bm = b64.copy(), b64.copy()
            bp[i], bm[i] = wp, wm
            fd = (_oracle_loss(bp, xd, dd, td) - _oracle_loss(bm, xd, dd, td)) / (wp - wm)
            rows.append((name, i, g[i], fd, scale))
    worst = 0.0
    for name, i, gi, fd, scale in rows:
        worst = max(worst, abs(gi - fd) / (scale + 1e-30))
        print(f"{name:8s} {i:7d} gpu {gi: .6e} fd {fd: .6e} layer max {scale:.3e}")
    num = np.sqrt(sum((gi - fd) ** 2 for _, _, gi, fd, _ in rows))
    den = np.sqrt(sum(fd ** 2 for _, _, _, fd, _ in rows))
    print(f"{len(rows)} weights: worst |g - fd| / layer max {worst:.3g}, "
          f"relative L2 {num / den:.3g}")
    for name, i, gi, fd, scale in rows:
        assert abs(gi - fd) <= 1e-3 * scale + 1e-3 * abs(fd), (name, i, gi, fd, scale)
    assert num / den <= 1e-3


@pytest.fixture(scope="module")
def fitted(M):
    """A short fit from He-init weights on 65,536 room-field samples."""
    import torch
    import synth
    x, d, tgt = _points(65536, 1)
    xt, dt, tt = (torch.tensor(a, device="cuda") for a in (x, d, tgt))
    out = {}
    for k in range(2):
        gm = M.Map(synth.he_init_weights(0), max_rays=4096)
        log = gm.fit(xt, dt, tt, steps=300, batch=4096, lr=1e-3, lr_end=3e-4, sigma_weight=WS,
                     seed=7).cpu().numpy()
        out[k] = (gm, log, gm.weights())
    yield out
    for gm, _, _ in out.values():
        gm.close()


def test_fit_lowers_the_loss(fitted):
    _, log, _ = fitted[0]
    assert np.all(np.isfinite(log))
    first, last = float(log[:20].mean()), float(log[-20:].mean())
    print(f"\nloss: first 20 steps {first:.4g}, last 20 steps {last:.4g}")
    assert last < 0.5 * first


def test_fit_is_deterministic(fitted):
    (_, log0, w0), (_, log1, w1) = fitted[0], fitted[1]
    assert np.array_equal(log0, log1)
    assert np.array_equal(w0, w1)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_fitted_weights_drive_every_form(fitted, precision):
    """Queries of the fitted map against the oracle on the weights read back:
    FP32 at the plain form's 1e-4 relative bar; BF16 (the tensor-core form
    rebuilt from the fitted weights) at twice the BF16 format floor."""
    import torch
    import oracle
    import format_floor
    gm, _, w = fitted[0]
    rng = np.random.default_rng(21)
    x = rng.uniform(-4, 4, size=(2048, 3)).astype(np.float32)
    d = rng.normal(size=(2048, 3)).astype(np.float32)
    dd = _unit(d)
    out = gm.query(torch.tensor(x, device="cuda"), torch.tensor(d, device="cuda"),
                   precision).cpu().numpy()
    s_ref, c_ref = oracle.mlp(w, x.astype(np.float64), dd)
    if precision == "fp32":
        assert np.all(np.abs(out[:, 1:] - c_ref) <= 1e-4 * np.abs(c_ref) + 1e-6)
        assert np.all(np.abs(out[:, 0] - s_ref) <= 1e-4 * np.abs(s_ref) + 1e-4)
        return
    s_fl, c_fl = format_floor.mlp_rounded(w, x.astype(np.float64), dd, "bf16")
    spread = float(np.std(s_ref))
    for name, got, flo, ref, norm in (("rgb", out[:, 1:], c_fl, c_ref, 1.0),
                                      ("sigma", out[:, 0], s_fl, s_ref, spread)):
        eg, ef = np.abs(got - ref) / norm, np.abs(flo - ref) / norm
        print(f"\n{name}: gpu mean {eg.mean():.3g} max {eg.max():.3g}; "
              f"floor mean {ef.mean():.3g} max {ef.max():.3g}")
        assert eg.mean() <= 2 * ef.mean() and eg.max() <= 2 * ef.max()


def test_adam_steps_match_the_published_update(M):
    """Two Adam steps of mcl_fit_map over one full batch (the optimiser the
    proposal training uses too) against Adam as Kingma and Ba define it, in
    FP64, driven by the library's own gradients at w0 and w1 (the fit sums
    its batch in a shuffled order, so its gradients differ from loss_grad's
    by FP32 rounding: weights whose gradient is within 1e-5 of the layer's
    largest of zero but not zero, where that rounding could move the step,
    are left out)."""
    import torch
    import synth
    n = 1024
    x, d, tgt = _points(n, 17)
    xt, dt, tt = (torch.tensor(a, device="cuda") for a in (x, d, tgt))
    w0 = synth.he_init_weights(6, bias_std=0.05)
    lr, b1, b2, eps = 1e-3, 0.9, 0.999, 1e-8

    def fitted(steps):
        gm = M.Map(w0, max_rays=4096)
        try:
            gm.fit(xt, dt, tt, steps=steps, batch=n, lr=lr, lr_end=lr, beta1=b1, beta2=b2, eps=eps,
                   sigma_weight=WS, seed=9)
            return gm.weights().astype(np.float64)
        finally:
            gm.close()

    def grad(w):
        gm = M.Map(np.asarray(w, np.float32), max_rays=4096)
        try:
            return gm.loss_grad(xt, dt, tt, sigma_weight=WS)[1].cpu().numpy().astype(np.float64)
        finally:
            gm.close()

    w1, w2 = fitted(1), fitted(2)
    g0, g1 = grad(w0), grad(w1)
    w0d = w0.astype(np.float64)
    # step 1: m = (1 - b1) g, v = (1 - b2) g^2, bias-corrected by 1 - b^1
    m = (1 - b1) * g0
    v = (1 - b2) * g0 * g0
    w1_ref = w0d - lr * (m / (1 - b1)) / (np.sqrt(v / (1 - b2)) + eps)
    # step 2 from the library's w1
    m = b1 * m + (1 - b1) * g1
    v = b2 * v + (1 - b2) * g1 * g1
    w2_ref = w1 - lr * (m / (1 - b1 ** 2)) / (np.sqrt(v / (1 - b2 ** 2)) + eps)
    # (an exactly zero gradient -- a unit no point activates -- steps by exactly 0)
    ok0 = (np.abs(g0) > 1e-5 * np.abs(g0).max()) | (g0 == 0)
    ok1 = (np.abs(g1) > 1e-5 * np.abs(g1).max()) | (g1 == 0)
    keep = ok0 & ok1
    tol = 1e-3 * lr + 4 * np.spacing(np.abs(w0d).astype(np.float32)).astype(np.float64)
    e1 = np.abs(w1 - w1_ref)[keep]
    e2 = np.abs(w2 - w2_ref)[keep]
    print(f"\n{keep.sum()} of {keep.size} weights: step 1 max |dw| {e1.max():.3g}, "
          f"step 2 {e2.max():.3g} (lr {lr})")
    assert keep.mean() > 0.9   # measured 0.926: the rest have near-zero gradients
    assert np.all(e1 <= tol[keep])
    assert np.all(e2 <= tol[keep])
    # and the steps moved the weights by about lr
    moved = keep & (g0 != 0)
    assert 0.5 * lr <= np.median(np.abs(w1 - w0d)[moved]) <= 1.01 * lr
