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
