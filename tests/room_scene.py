"""Closed-form renders of the analytic room map (synth.room_map_weights):
the volume-rendering integral of Eq. 1 taken in continuous form along each
ray, with the map's density and colour written out from their definitions
(no MLP, no sample placement of the method), by a fine trapezoid rule over
the short stretch behind the wall where all the weight lies.  Independent of
both the oracle and the CUDA library; used as the observed image of
end-to-end localisation tests and as a pin of the oracle's renderer."""
from __future__ import annotations

import numpy as np


def room_sigma(x, half, eps, density):
    m = np.abs(x).max(-1)
    return density * np.clip((m - half) / eps, 0.0, 1.0)


def room_rgb(x, a, n_tex_freq=4):
    feats = []
    for k in range(n_tex_freq):
        for c in range(3):
            v = (2.0 ** k) * x[..., c]
            feats.append(np.sin(v))
            feats.append(np.cos(v))
    f = np.stack(feats, -1)
    return 1.0 / (1.0 + np.exp(-(f @ a.T)))


def wall_hit(o, d, half):
    """Distance t (in units of d) at which o + t d leaves the cube |x|_inf <= half."""
    with np.errstate(divide="ignore"):
        t = np.where(d != 0.0, (np.sign(d) * half - o) / d, np.inf)
    return t.min(-1)


def render_continuous(o, d, a, half=3.0, eps=0.015625, density=64.0, near=2.0, far=6.0,
                      depth=0.3, n=1201):
    """Colour of rays o, d [n_rays, 3] (d not normalised: the density acts
    per unit of ray length |d| dt, as in Eq. 1's quadrature).  Returns rgb
    [n_rays, 3] and the transmittance left at the end of the integrated
    stretch (~0 for a ray that meets a wall inside [near, far])."""
    o = np.asarray(o, np.float64)
    d = np.asarray(d, np.float64)
    a = np.asarray(a, np.float64)
    dn = np.linalg.norm(d, axis=1)
    th = np.clip(wall_hit(o, d, half), near, far)
    # the stretch [th, th + depth / |d|] covers the ramp and the solid part
    s = np.linspace(0.0, 1.0, n)[None, :]
    t = th[:, None] + s * (depth / dn)[:, None]
    t = np.minimum(t, far)
    x = o[:, None, :] + t[..., None] * d[:, None, :]
    sg = room_sigma(x, half, eps, density) * dn[:, None]
    dt = np.diff(t, axis=1)
    tau = np.concatenate([np.zeros((len(o), 1)),
                          np.cumsum(0.5 * (sg[:, 1:] + sg[:, :-1]) * dt, axis=1)], 1)
    T = np.exp(-tau)
    g = (T * sg)[..., None] * room_rgb(x, a)
    rgb = (0.5 * (g[:, 1:] + g[:, :-1]) * dt[..., None]).sum(1)
    return rgb, T[:, -1]


def pixel_rays(pose, fx, fy, cx, cy, px):
    """Rays through pixel centres (camera looks along -z, +y up), as the
    method's pinhole model reads: d = R [(u + 0.5 - cx)/fx, -(v + 0.5 - cy)/fy, -1]."""
    P = np.asarray(pose, np.float64).reshape(3, 4)
    u = px[:, 0] + 0.5
    v = px[:, 1] + 0.5
    dc = np.stack([(u - cx) / fx, -(v - cy) / fy, -np.ones_like(u)], 1)
    return np.broadcast_to(P[:, 3], dc.shape).copy(), dc @ P[:, :3].T


def observed_image(pose, a, W, H, focal, **kw):
    """Full-resolution observation [H, W, 3] at pose by the continuous integral."""
    px = np.stack(np.meshgrid(np.arange(W), np.arange(H), indexing="xy"), -1).reshape(-1, 2)
    o, d = pixel_rays(pose, focal, focal, W / 2.0, H / 2.0, px)
    rgb = np.zeros((W * H, 3))
    for c0 in range(0, W * H, 2000):
        rgb[c0:c0 + 2000] = render_continuous(o[c0:c0 + 2000], d[c0:c0 + 2000], a, **kw)[0]
    return rgb.reshape(H, W, 3)
