"""Error floor of a reduced-precision operand format, for deriving the parity
bars of the BF16 and FP8 tensor-core forms (test infrastructure).

The NeRF MLP is evaluated on its plain layer structure (the paper's basic
model: 8 ReLU trunk layers with the skip, density head, linear feature layer,
RGB head) with every matrix-multiply operand -- positional encoding,
activations and weights -- rounded to the format, products accumulated in
FP32, biases, ReLU and the sigmoid in FP32.  Rendering, Eq. 5 / F and the
Eq. 6 weights around it are the FP64 oracle's pinned pieces (composite,
inverse CDF, uncertainty).  Comparing this render with the oracle's own
gives the error that any kernel computing with these operand formats
carries; the GPU forms are then held to a stated multiple of it.

Formats:
  bf16  round to nearest even to 8 significant bits;
  e4m3  per-tensor scaling of each operand (largest magnitude -> 448, the
        format's largest finite value), then round to nearest even to 4
        significant bits, subnormals below 2^-6, saturation at 448.
"""
from __future__ import annotations

import numpy as np

import oracle
import synth


def round_bf16(x):
    x = np.ascontiguousarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32)
    return np.where(np.isfinite(x), out, x)


def round_e4m3(x):
    """Nearest E4M3 value (round half to even), saturating at +-448."""
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    e = np.floor(np.log2(np.maximum(a, 1e-300)))
    e = np.maximum(e, -6.0)                   # subnormal spacing below 2^-6
    q = np.exp2(e - 3.0)                       # 3 mantissa bits
    v = np.round(a / q) * q                    # numpy rounds half to even
    v = np.minimum(v, 448.0)
    return (np.sign(x) * v).astype(np.float32)


def _q(x, fmt):
    """Operand as the format holds it (value in FP32)."""
    if fmt == "bf16":
        return round_bf16(x)
    m = float(np.max(np.abs(x))) if np.size(x) else 0.0
    if m == 0.0:
        return np.asarray(x, dtype=np.float32)
    s = 448.0 / m
    return (round_e4m3(np.asarray(x, dtype=np.float64) * s) / s).astype(np.float32)


def _layers(blob, arch=synth.Arch()):
    out = {}
    off = 0
    for name, fi, fo in synth.layer_shapes(arch):
        W = blob[off:off + fi * fo].reshape(fo, fi).astype(np.float32)
        off += fi * fo
        b = blob[off:off + fo].astype(np.float32)
        off += fo
        out[name] = (W, b)
    return out


def _pe(p, L):
    parts = [p]
    for k in range(L):
        parts.append(np.sin((2.0 ** k) * p))
        parts.append(np.cos((2.0 ** k) * p))
    # order [p, sin(2^0 p), cos(2^0 p), sin(2^1 p), ...], each a 3-vector
    return np.concatenate(parts, axis=-1)


def mlp_rounded(blob, x, dhat, fmt, arch=synth.Arch()):
    """(sigma_raw, rgb) at points x [n,3], unit directions dhat [n,3], with
    the operands of every matrix product rounded to fmt."""
    Ls = _layers(blob, arch)
    mm = lambda a, W: np.matmul(_q(a, fmt), _q(W, fmt).T, dtype=np.float32)
    gx = _pe(np.asarray(x, np.float64), arch.n_freq_xyz).astype(np.float32)
    gd = _pe(np.asarray(dhat, np.float64), arch.n_freq_dir).astype(np.float32)
    h = gx
    for l in range(1, arch.trunk_depth + 1):
        W, b = Ls[f"trunk{l}"]
        h = np.maximum(mm(h, W) + b, 0.0)
        if l == arch.skip_layer:
            h = np.concatenate([h, gx], axis=1)
    Ws, bs = Ls["sigma"]
    sigma = (mm(h, Ws) + bs)[:, 0]
    Wf, bf = Ls["feature"]
    feat = mm(h, Wf) + bf
    Wh, bh = Ls["rgb_hidden"]
    hid = np.maximum(mm(np.concatenate([feat, gd], axis=1), Wh) + bh, 0.0)
    Wo, bo = Ls["rgb_out"]
    rgb = 1.0 / (1.0 + np.exp(-(mm(hid, Wo) + bo).astype(np.float64)))
    return sigma.astype(np.float64), rgb


def _eval_points(blob, o, d, z, fmt):
    x = o[None, :] + z[:, None] * d[None, :]
    dh = np.broadcast_to(d / np.linalg.norm(d), x.shape)
    if fmt == "fp64":
        return oracle.mlp(blob, x, dh)
    return mlp_rounded(blob, x, dh, fmt)


def render_scene(sc, fmt):
    """Per-ray rgb / F and per-particle log-weights of a gpu_helpers scene
    with the MLP in `fmt` ("bf16", "e4m3", or "fp64" for the oracle's MLP)
    and FP64 compositing, inverse CDF, Eq. 5 and Eq. 6 (stratified
    midpoints, no jitter)."""
    op = sc["opts"]
    nc, nf = sc["n_coarse"], sc["n_fine"]
    f = sc["factor"]
    K = oracle.level_intrinsics(sc["K4"], f)
    P, px, img = sc["P"], sc["px"], sc["img"]
    level = oracle.downscale(img, f) if f > 1 else img
    N, B = P.shape[0], px.shape[0]
    zc = op.near_z + (op.far_z - op.near_z) * (np.arange(nc) + 0.5) / nc
    rgb = np.zeros((N * B, 3))
    F = np.zeros(N * B)
    E = np.zeros(N * B)
    for i in range(N):
        for j in range(B):
            o, d = oracle.ray(P[i], *K, int(px[j, 0]), int(px[j, 1]))
            o, d = np.asarray(o), np.asarray(d)
            dn = float(np.linalg.norm(d))
            s1, c1 = _eval_points(sc["blob"], o, d, zc, fmt)
            if nf > 0:
                w1 = oracle.composite(zc, s1, c1, dn)[0]
                zf = oracle.sample_pdf(zc, w1, nf)
                s2, c2 = _eval_points(sc["blob"], o, d, zf, fmt)
                z = np.concatenate([zc, zf])
                s = np.concatenate([s1, s2])
                c = np.concatenate([c1, c2])
                order = np.argsort(z, kind="stable")
                z, s, c = z[order], s[order], c[order]
            else:
                z, s, c = zc, s1, c1
            w, _, col = oracle.composite(z, s, c, dn)
            unc = oracle.uncertainty(z, w, op.alpha, op.tau)
            r = i * B + j
            rgb[r] = col
            F[r] = unc["F"] if sc["use_rejection"] else 1.0
            obs = level[px[j, 1], px[j, 0]]
            E[r] = float(((obs - col) ** 2).sum())
    S = (E * F).reshape(N, B).sum(1)
    logw = 4.0 * (np.log(B) - np.log(np.maximum(S, op.s_min)))
    return dict(rgb=rgb, F=F, E=E, S=S, logw=logw)
