"""Seeded synthetic inputs for the MCL particle-weight update.

This module is the one place both sides of the parity tests take their inputs
from: the FP64 oracle under ``oracle/`` and the CUDA library under
``paper_2406_12202_gb300/``.  It holds none of the method's arithmetic (no
rendering, no weighting, no resampling, no motion model).  It only draws
numbers with numpy's PCG64 generator from a fixed seed and lays them out in the
formats the two sides accept.

Stand-ins.  The paper evaluates on the LLFF and Deep Blending datasets with
trained NeRF-pytorch / Zip-NeRF maps (Sec. IV-A, IV-B).  Neither is available,
so every workload here is synthetic with the paper's structure:

* map: the NeRF MLP of the "basic NeRF model" (Sec. IV-A) with He-normal
  weights (std sqrt(2/fan_in), zero biases) from a seed;
* particles: uniform offsets in [-1, 1]^3 around the origin and a uniform yaw
  in [-pi, pi), the paper's global-localisation initial spread (Sec. IV-A);
* camera: forward-facing pinhole, principal point at the image centre;
* pixel set: B distinct pixels of the level image, shared by every particle
  of one update (Eq. 4 and Eq. 6 index p_j without a particle index);
* observed image: a smooth seeded RGB texture in [0, 1] (tests overwrite the
  sampled pixels with oracle renders at the ground-truth pose).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# --------------------------------------------------------------------------
# Map architecture (the NeRF MLP named by the workload: 8 x 256 trunk, skip
# concatenation of gamma(x) after trunk layer 5, sigma head, 256-wide linear
# feature layer, 128-wide RGB layer fed with [feature, gamma(d)]).
# --------------------------------------------------------------------------


@dataclass(frozen=True)
class Arch:
    n_freq_xyz: int = 10
    n_freq_dir: int = 4
    trunk_depth: int = 8
    trunk_width: int = 256
    skip_layer: int = 5
    rgb_width: int = 128

    @property
    def gx(self) -> int:
        return 3 + 6 * self.n_freq_xyz

    @property
    def gd(self) -> int:
        return 3 + 6 * self.n_freq_dir

    def as_tuple(self):
        return (self.n_freq_xyz, self.n_freq_dir, self.trunk_depth,
                self.trunk_width, self.skip_layer, self.rgb_width)


def layer_shapes(arch: Arch = Arch()):
    """(name, fan_in, fan_out) of every layer in blob order.

    Blob order: trunk1..trunkD, sigma, feature, rgb_hidden, rgb_out.  Trunk
    layer skip+1 takes [h_skip (width), gamma(x)] (that order).  rgb_hidden
    takes [feature (width), gamma(d)] (that order).
    """
    out = []
    for l in range(1, arch.trunk_depth + 1):
        if l == 1:
            fi = arch.gx
        elif l == arch.skip_layer + 1:
            fi = arch.trunk_width + arch.gx
        else:
            fi = arch.trunk_width
        out.append((f"trunk{l}", fi, arch.trunk_width))
    out.append(("sigma", arch.trunk_width, 1))
    out.append(("feature", arch.trunk_width, arch.trunk_width))
    out.append(("rgb_hidden", arch.trunk_width + arch.gd, arch.rgb_width))
    out.append(("rgb_out", arch.rgb_width, 3))
    return out


def n_weights(arch: Arch = Arch()) -> int:
    return sum(fi * fo + fo for _, fi, fo in layer_shapes(arch))


def blob_offsets(arch: Arch = Arch()):
    """name -> (offset of W, offset of b, fan_in, fan_out) in float units."""
    offs, pos = {}, 0
    for name, fi, fo in layer_shapes(arch):
        offs[name] = (pos, pos + fi * fo, fi, fo)
        pos += fi * fo + fo
    return offs


def he_init_weights(seed: int = 0, arch: Arch = Arch(),
                    bias_std: float = 0.0) -> np.ndarray:
    """FP32 weight blob: W ~ N(0, 2/fan_in) per layer ([out][in] row-major),
    biases N(0, bias_std^2) (zero by default).  Drawn in FP64, stored FP32."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for _, fi, fo in layer_shapes(arch):
        W = rng.normal(0.0, math.sqrt(2.0 / fi), size=(fo, fi))
        b = rng.normal(0.0, bias_std, size=fo) if bias_std > 0 else np.zeros(fo)
        parts.append(W.reshape(-1))
        parts.append(b)
    return np.concatenate(parts).astype(np.float32)


def blob_from_layers(layers: dict, arch: Arch = Arch()) -> np.ndarray:
    """Assemble a blob from {name: (W [out,in], b [out])}; missing layers are
    zero.  Used to build hand-set maps with closed-form outputs."""
    parts = []
    for name, fi, fo in layer_shapes(arch):
        W, b = layers.get(name, (None, None))
        W = np.zeros((fo, fi)) if W is None else np.asarray(W, dtype=np.float64)
        b = np.zeros(fo) if b is None else np.asarray(b, dtype=np.float64)
        assert W.shape == (fo, fi), (name, W.shape, (fo, fi))
        assert b.shape == (fo,), (name, b.shape)
        parts.append(W.reshape(-1))
        parts.append(b)
    return np.concatenate(parts).astype(np.float32)


def room_map_weights(seed: int = 0, half: float = 3.0, eps: float = 0.015625,
                     density: float = 64.0, n_tex_freq: int = 4,
                     arch: Arch = Arch()) -> np.ndarray:
    """Hand-set map of the same architecture with a closed form: a textured
    cube room.  With m(x) = max(|x|, |y|, |z|),
        sigma(x) = density * clamp((m(x) - half) / eps, 0, 1)
    (free space inside the room, solid walls beyond it) and, everywhere,
        rgb(x) = sigmoid(sum_f a_f f(x)),
    f running over sin / cos(2^k x_c) for k < n_tex_freq and each axis c,
    with coefficients a_f ~ N(0, 0.45^2) from the seed.  Built only from the
    ReLU units the architecture has (|v| = relu(v) + relu(-v), max(a, b) =
    a + relu(b - a), clamp = relu(t) - relu(t - 1)); the view direction has
    zero weight.  Returns (blob FP32, coefficient matrix a [3, n_features]).
    Camera positions in [-1, 1]^3 with near 2 / far 6 see the walls; the
    texture makes position and yaw identifiable, so a filter on this map has
    a unique answer."""
    Wd, gx, gd, Wr = arch.trunk_width, arch.gx, arch.gd, arch.rgb_width
    rng = np.random.Generator(np.random.PCG64(seed + 179424673))
    feats = [(k, c, kind) for k in range(n_tex_freq) for c in range(3) for kind in (0, 1)]
    nf = len(feats)
    a = rng.normal(0.0, 0.45, size=(3, nf))
    T0 = 8                        # first texture unit (pairs relu(f), relu(-f))
    assert T0 + 2 * nf <= Wd
    tex = np.arange(T0, T0 + 2 * nf)

    def ident(fi):
        W = np.zeros((Wd, fi))
        W[tex, tex] = 1.0
        return W

    L = {}
    W1 = np.zeros((Wd, gx))
    for c in range(3):
        W1[2 * c, c] = 1.0
        W1[2 * c + 1, c] = -1.0
    for i, (k, c, kind) in enumerate(feats):
        col = 3 + 6 * k + c + 3 * kind          # sin(2^k x_c) or cos(2^k x_c)
        W1[T0 + 2 * i, col] = 1.0
        W1[T0 + 2 * i + 1, col] = -1.0
    L["trunk1"] = (W1, np.zeros(Wd))
    W2 = ident(Wd)                              # |x|, |y|, |z|
    for c in range(3):
        W2[c, 2 * c] = W2[c, 2 * c + 1] = 1.0
    L["trunk2"] = (W2, np.zeros(Wd))
    W3 = ident(Wd)                              # |x|, relu(|y| - |x|), |z|
    W3[0, 0] = 1.0
    W3[1, 1], W3[1, 0] = 1.0, -1.0
    W3[2, 2] = 1.0
    L["trunk3"] = (W3, np.zeros(Wd))
    W4 = ident(Wd)                              # max(|x|,|y|), relu(|z| - max(|x|,|y|))
    W4[0, 0] = W4[0, 1] = 1.0
    W4[1, 2], W4[1, 0], W4[1, 1] = 1.0, -1.0, -1.0
    L["trunk4"] = (W4, np.zeros(Wd))
    W5 = ident(Wd)                              # relu(t), relu(t - 1), t = (m - half) / eps
    b5 = np.zeros(Wd)
    W5[0, 0] = W5[0, 1] = 1.0 / eps
    W5[1, 0] = W5[1, 1] = 1.0 / eps
    b5[0] = -half / eps
    b5[1] = -half / eps - 1.0
    L["trunk5"] = (W5, b5)
    W6 = np.zeros((Wd, Wd + gx))                # clamp(t, 0, 1); gamma(x) part unused
    W6[tex, tex] = 1.0
    W6[0, 0], W6[0, 1] = 1.0, -1.0
    L["trunk6"] = (W6, np.zeros(Wd))
    for l in range(7, arch.trunk_depth + 1):
        W = ident(Wd)
        W[0, 0] = 1.0
        L[f"trunk{l}"] = (W, np.zeros(Wd))
    Ws = np.zeros((1, Wd))
    Ws[0, 0] = density
    L["sigma"] = (Ws, np.zeros(1))
    L["feature"] = (np.eye(Wd), np.zeros(Wd))
    beta = np.abs(a).sum(1) + 1.0               # keeps the hidden units positive
    Wh = np.zeros((Wr, Wd + gd))
    for c in range(3):
        for i in range(nf):
            Wh[c, T0 + 2 * i] = a[c, i]
            Wh[c, T0 + 2 * i + 1] = -a[c, i]
    bh = np.zeros(Wr)
    bh[:3] = beta
    L["rgb_hidden"] = (Wh, bh)
    Wo = np.zeros((3, Wr))
    Wo[[0, 1, 2], [0, 1, 2]] = 1.0
    L["rgb_out"] = (Wo, -beta)
    return blob_from_layers(L, arch), a


# --------------------------------------------------------------------------
# Learned proposal sampler: gamma(x) with 6 frequencies (39 inputs), four ReLU
# layers of 64 units, a linear density head.  Blob: P1 W[64][39] b[64],
# P2..P4 W[64][64] b[64], head w[64] b[1].
# --------------------------------------------------------------------------
PROPOSAL_SHAPES = [("p1", 39, 64), ("p2", 64, 64), ("p3", 64, 64), ("p4", 64, 64), ("head", 64, 1)]


def proposal_n_weights() -> int:
    return sum(fi * fo + fo for _, fi, fo in PROPOSAL_SHAPES)


def proposal_init_weights(seed: int = 0, head_bias: float = 1.0) -> np.ndarray:
    """He-normal proposal weights (FP32 blob), zero hidden biases and a
    positive density-head bias so that training starts with density > 0."""
    rng = np.random.Generator(np.random.PCG64(seed + 1299709))
    parts = []
    for name, fi, fo in PROPOSAL_SHAPES:
        parts.append(rng.normal(0.0, math.sqrt(2.0 / fi), size=fo * fi))
        parts.append(np.full(fo, head_bias) if name == "head" else np.zeros(fo))
    return np.concatenate(parts).astype(np.float32)


def room_field(x, seed: int = 0, half: float = 3.0, eps: float = 0.015625,
               density: float = 64.0, n_tex_freq: int = 4):
    """The field that room_map_weights(seed, half, eps, density, n_tex_freq)
    represents, evaluated at points x [n, 3]: density * clamp((max_c |x_c| -
    half) / eps, 0, 1) and sigmoid(a . f(x)) with f = sin / cos(2^k x_c) in
    the map's feature order (FP64).  Samples of it are the targets for
    fitting a map to the room.  Returns (density [n], rgb [n, 3])."""
    x = np.asarray(x, dtype=np.float64)
    _, a = room_map_weights(seed, half, eps, density, n_tex_freq)
    a = a.astype(np.float32).astype(np.float64)
    m = np.abs(x).max(-1)
    sig = density * np.clip((m - half) / eps, 0.0, 1.0)
    feats = []
    for k in range(n_tex_freq):
        for c in range(3):
            v = (2.0 ** k) * x[..., c]
            feats.append(np.sin(v))
            feats.append(np.cos(v))
    f = np.stack(feats, -1)
    return sig, 1.0 / (1.0 + np.exp(-(f @ a.T)))


def room_fit_points(seed: int, n: int, half: float = 3.0):
    """Seeded sample points for fitting a map to the room: half uniform in
    the box [-(half + 0.5), half + 0.5]^3 (free space and walls), half in the
    shell of the walls (one coordinate at +-(half + U(-0.1, 0.3)), the others
    uniform in [-half, half]); unit view directions.  Returns (x [n,3],
    dirs [n,3]) float32."""
    rng = np.random.Generator(np.random.PCG64(seed + 2750159))
    n1 = n // 2
    x1 = rng.uniform(-(half + 0.5), half + 0.5, size=(n1, 3))
    x2 = rng.uniform(-half, half, size=(n - n1, 3))
    axis = rng.integers(0, 3, size=n - n1)
    sign = rng.choice([-1.0, 1.0], size=n - n1)
    x2[np.arange(n - n1), axis] = sign * (half + rng.uniform(-0.1, 0.3, size=n - n1))
    x = np.concatenate([x1, x2])
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return x.astype(np.float32), d.astype(np.float32)


def room_proposal_weights(half: float = 3.0, eps: float = 0.015625,
                          density: float = 64.0) -> np.ndarray:
    """Hand-set proposal blob whose raw density is exactly the room map's
    density, density * clamp((max_c |x_c| - half) / eps, 0, 1), built from
    the proposal network's ReLU units on the identity part of its input
    (gamma(x) entries 0..2 = x): |x_c| = relu(x_c) + relu(-x_c) (layer 1),
    |x|, relu(|y| - |x|), |z| (layer 2), max(|x|, |y|) and
    relu(|z| - max(|x|, |y|)) (layer 3), relu(t) and relu(t - 1) with
    t = (m - half) / eps (layer 4), head density * (relu(t) - relu(t - 1))."""
    L = {n: (np.zeros((fo, fi)), np.zeros(fo)) for n, fi, fo in PROPOSAL_SHAPES}
    W1 = L["p1"][0]
    for c in range(3):
        W1[2 * c, c] = 1.0
        W1[2 * c + 1, c] = -1.0
    W2 = L["p2"][0]
    W2[0, 0] = W2[0, 1] = 1.0                       # |x|
    W2[1, 2] = W2[1, 3] = 1.0                       # relu(|y| - |x|)
    W2[1, 0] = W2[1, 1] = -1.0
    W2[2, 4] = W2[2, 5] = 1.0                       # |z|
    W3 = L["p3"][0]
    W3[0, 0] = W3[0, 1] = 1.0                       # max(|x|, |y|)
    W3[1, 2] = 1.0                                  # relu(|z| - max(|x|, |y|))
    W3[1, 0] = W3[1, 1] = -1.0
    W4, b4 = L["p4"]
    W4[0, 0] = W4[0, 1] = 1.0 / eps
    W4[1, 0] = W4[1, 1] = 1.0 / eps
    b4[0] = -half / eps
    b4[1] = -half / eps - 1.0
    Wh = L["head"][0]
    Wh[0, 0], Wh[0, 1] = density, -density
    parts = []
    for name, fi, fo in PROPOSAL_SHAPES:
        parts.append(L[name][0].reshape(-1))
        parts.append(L[name][1])
    return np.concatenate(parts).astype(np.float32)


# --------------------------------------------------------------------------
# Poses: particle = T(x, y, z) * R_y(yaw), stored as a row-major 3x4 [R | t].
# --------------------------------------------------------------------------


def pose_from_xyz_yaw(xyz, yaw) -> np.ndarray:
    xyz = np.asarray(xyz, dtype=np.float64).reshape(-1, 3)
    yaw = np.asarray(yaw, dtype=np.float64).reshape(-1)
    n = xyz.shape[0]
    P = np.zeros((n, 3, 4))
    c, s = np.cos(yaw), np.sin(yaw)
    P[:, 0, 0] = c
    P[:, 0, 2] = s
    P[:, 1, 1] = 1.0
    P[:, 2, 0] = -s
    P[:, 2, 2] = c
    P[:, :, 3] = xyz
    return P.reshape(n, 12)


def random_particles(seed: int, n: int, extent: float = 1.0):
    """n poses: x, y, z ~ U[-extent, extent], yaw ~ U[-pi, pi).  Returns
    (poses [n,12] float64, xyz [n,3], yaw [n])."""
    rng = np.random.Generator(np.random.PCG64(seed))
    xyz = rng.uniform(-extent, extent, size=(n, 3))
    yaw = rng.uniform(-math.pi, math.pi, size=n)
    return pose_from_xyz_yaw(xyz, yaw), xyz, yaw


def gt_pose(seed: int):
    """Ground-truth pose drawn like a particle (seed offset keeps it distinct
    from the particle draw of the same seed)."""
    P, xyz, yaw = random_particles(seed + 7919, 1)
    return P[0], xyz[0], float(yaw[0])


# --------------------------------------------------------------------------
# Camera, pixels, images.
# --------------------------------------------------------------------------


@dataclass(frozen=True)
class Camera:
    width: int
    height: int
    focal: float

    @property
    def cx(self) -> float:
        return self.width / 2.0

    @property
    def cy(self) -> float:
        return self.height / 2.0


def pixel_set(seed: int, width: int, height: int, B: int) -> np.ndarray:
    """B distinct pixels (u, v) of a width x height image, int32 [B, 2]."""
    rng = np.random.Generator(np.random.PCG64(seed + 104729))
    flat = rng.choice(width * height, size=B, replace=False)
    return np.stack([flat % width, flat // width], axis=1).astype(np.int32)


def smooth_image(seed: int, width: int, height: int, n_waves: int = 6) -> np.ndarray:
    """Smooth RGB texture in [0, 1], float32 [H, W, 3] (sum of random
    low-frequency plane waves squashed into [0, 1])."""
    rng = np.random.Generator(np.random.PCG64(seed + 15485863))
    yy, xx = np.meshgrid(np.arange(height) / height, np.arange(width) / width,
                         indexing="ij")
    img = np.zeros((height, width, 3))
    for c in range(3):
        acc = np.zeros((height, width))
        for _ in range(n_waves):
            kx, ky = rng.uniform(-6, 6, size=2)
            ph = rng.uniform(0, 2 * math.pi)
            acc += np.sin(2 * math.pi * (kx * xx + ky * yy) + ph)
        img[..., c] = 0.5 + 0.5 * np.tanh(acc / math.sqrt(n_waves))
    return img.astype(np.float32)


def jitter_uniforms(seed: int, n: int) -> np.ndarray:
    """n uniforms in [0, 1) for stratified jitter when passed explicitly."""
    rng = np.random.Generator(np.random.PCG64(seed + 32452843))
    return rng.uniform(0.0, 1.0, size=n)


def random_weights(seed: int, n: int, dyadic_bits: int | None = None,
                   zero_frac: float = 0.0) -> np.ndarray:
    """Normalised FP64 particle weights for resampling tests.  With
    dyadic_bits=m every weight is an integer multiple of 2^-m before
    normalisation by a power of two (exactly representable sums)."""
    rng = np.random.Generator(np.random.PCG64(seed + 49979687))
    if dyadic_bits is not None:
        k = rng.integers(0, 1 << dyadic_bits, size=n).astype(np.float64)
        if zero_frac > 0:
            k[rng.uniform(size=n) < zero_frac] = 0.0
        if k.sum() == 0:
            k[0] = 1.0
        return k
    w = rng.exponential(1.0, size=n) ** 3
    if zero_frac > 0:
        w[rng.uniform(size=n) < zero_frac] = 0.0
    if w.sum() == 0:
        w[0] = 1.0
    return w / w.sum()


def resample_u0(seed: int) -> float:
    rng = np.random.Generator(np.random.PCG64(seed + 86028121))
    return float(rng.uniform(0.0, 1.0))


# --------------------------------------------------------------------------
# Workload recipes (sizes of the configurations this library is measured on).
# --------------------------------------------------------------------------

WORKLOADS = {
    # Plain single update: 32 particles x 8 pixels of a 100x100 image,
    # 32 midpoint-stratified coarse samples in [2, 6], no fine pass.
    "c1": dict(N=32, B=8, width=100, height=100, focal=138.9, n_coarse=32,
               n_fine=0, levels=(1,), near=2.0, far=6.0),
    # Full update: 600 particles x 64 pixels of a 400x400 image, 64 coarse +
    # 128 importance samples, uncertainty, rejection, systematic resampling.
    "c2": dict(N=600, B=64, width=400, height=400, focal=555.6, n_coarse=64,
               n_fine=128, levels=(1,), near=2.0, far=6.0),
    # Coarse-to-fine: 1500 initial particles, 3 levels (factors 4, 2, 1 of a
    # 400x400 image) with 16/32/64 pixels per particle.
    "c3": dict(N=1500, B=(16, 32, 64), width=400, height=400, focal=555.6,
               n_coarse=64, n_fine=128, levels=(4, 2, 1), near=2.0, far=6.0,
               iters=20, sigma_t=0.05, sigma_yaw=0.05),
}
