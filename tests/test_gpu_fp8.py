"""FP8 (E4M3 operands, FP32 accumulation) form of the tensor-core NeRF MLP
against the FP64 oracle.

The bars derived from the E4M3 format's own error floor (twice the error of
the plain layer structure with per-tensor-scaled E4M3 operands, every ray
counted) are in test_gpu_format_floor.py; the checks below are coarser
sanity bounds, kept from before that floor was measured.

FP8 bars (stated, derived from the format, not inherited from BF16): E4M3
keeps 4 significant bits, so every operand (positional encoding, weights,
activations) carries a relative rounding of up to 2^-4 (about 1.8 % rms for
round-to-nearest); a 256-term dot product of such operands has about 2.5 %
rms relative error, and nine layers compound this to the order of 10 % of a
pre-activation.  The activation scales come from a calibration pass when the
map is loaded (largest input of each layer over points in [-8, 8]^3 mapped
to 224, half the E4M3 range), the weights of a trunk layer share one scale
(largest |w| -> 448), the last layer has one scale per row.  Bars, about
1.5x the errors measured on He-init maps seeds 0 and 2:
* points: RGB max |err| <= 0.3, mean <= 0.04; density error relative to the
  spread of sigma max <= 1.5, mean <= 0.25;
* rendered rays (seed-0 map, where the density is positive almost
  everywhere): RGB max <= 0.12, mean <= 0.02 on rays whose last-sample
  density is not within the FP8 band of zero (0.6, the largest density error
  seen at points): those rays can absorb or pass the 1e10-long last
  interval depending on rounding, as in the BF16 tests;
* particle ranking: Spearman correlation of log-weights >= 0.93, top-10
  overlap >= 8, the ground-truth particle keeps the largest weight."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import lib, make_scene, run_gpu_update, run_oracle_update

pytestmark = pytest.mark.gpu

FP8_SIGMA_BAND = 0.6


@pytest.fixture(scope="module")
def M():
    return lib()


@pytest.fixture(scope="module")
def gmaps(M):
    maps = {}

    def get(seed):
        if seed not in maps:
            maps[seed] = M.Map(synth.he_init_weights(seed), max_rays=40000, max_samples=192,
                               max_particles=4096)
            assert maps[seed].supports("fp8"), "FP8 tensor-core form unavailable on this GPU"
        return maps[seed]
    yield get
    for m in maps.values():
        m.close()


def spearman(a, b):
    from scipy.stats import spearmanr
    return float(spearmanr(a, b).correlation)


def topk_overlap(a, b, k=10):
    return len(set(np.argsort(-a)[:k]) & set(np.argsort(-b)[:k]))


@pytest.mark.parametrize("seed,n", [(0, 4097), (2, 4097), (2, 129)])
def test_mlp_points_fp8_vs_oracle(M, gmaps, seed, n):
    import torch
    rng = np.random.default_rng(12345 + n)
    x = rng.uniform(-6, 6, size=(n, 3)).astype(np.float32)
    d = rng.normal(size=(n, 3))
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    out = gmaps(seed).query(torch.tensor(x, device="cuda"), torch.tensor(d, device="cuda"),
                            "fp8").cpu().numpy()
    dd = d.astype(np.float64)
    s_ref, rgb_ref = oracle.mlp(synth.he_init_weights(seed), x.astype(np.float64),
                                dd / np.linalg.norm(dd, axis=1, keepdims=True))
    # density scale: spread over a fixed reference sample of the volume
    rs = np.random.default_rng(99)
    xr = rs.uniform(-6, 6, size=(2048, 3))
    dr = rs.normal(size=(2048, 3))
    dr /= np.linalg.norm(dr, axis=1, keepdims=True)
    spread = float(np.std(oracle.mlp(synth.he_init_weights(seed), xr, dr)[0]))
    assert np.all(np.isfinite(out))
    e_rgb = np.abs(out[:, 1:] - rgb_ref)
    e_sig = np.abs(out[:, 0] - s_ref) / spread
    print(f"seed {seed} n={n}: rgb max {e_rgb.max():.3g} mean {e_rgb.mean():.3g}, "
          f"sigma/spread max {e_sig.max():.3g} mean {e_sig.mean():.3g}")
    assert e_rgb.max() <= 0.3 and e_rgb.mean() <= 0.04
    assert e_sig.max() <= 1.5 and e_sig.mean() <= 0.25


def scene(map_seed, *a, **k):
    sc = make_scene(map_seed, *a, **k)
    sc["map_seed"] = map_seed
    return sc


@pytest.mark.parametrize("args", [(0, 32, 8, 100, 100, 138.9, 32, 0, False),
                                  (31, 40, 8, 400, 400, 555.6, 64, 128, True)])
def test_fp8_update_seed0(M, gmaps, args):
    sc = scene(0, *args[:8], add_gt=args[8])
    g = run_gpu_update(M, gmaps(0), sc, precision="fp8")
    r = run_oracle_update(sc)
    flip = (np.abs(r["sigma_last"]) < FP8_SIGMA_BAND) & (r["T_last"] > 1e-3)
    assert flip.mean() <= 0.1, flip.mean()
    e = np.abs(g["rgb"] - r["rgb"])[~flip]
    fin = np.isfinite(r["logw"]) & (r["S"] > 1e-6)
    rho = spearman(g["logw"][fin], r["logw"][fin])
    top = topk_overlap(g["logw"][fin], r["logw"][fin])
    print(f"fp8 update: rgb max {e.max():.3g} mean {e.mean():.3g} flip {flip.mean():.3f} "
          f"spearman {rho:.4f} top10 {top}")
    assert e.max() <= 0.12 and e.mean() <= 0.02
    assert rho >= 0.93 and top >= 8
    assert abs(g["w"].sum() - 1.0) < 1e-12
    if args[8]:
        assert np.argmax(g["w"]) == args[1] and np.argmax(r["w"]) == args[1]


def test_fp8_update_seed2_ranking(M, gmaps):
    """Seed-2 map (density of either sign): many rays end near zero density,
    so only the particle ranking is held to a bar."""
    sc = scene(2, 31, 40, 8, 400, 400, 555.6, 64, 128, add_gt=True)
    g = run_gpu_update(M, gmaps(2), sc, precision="fp8")
    r = run_oracle_update(sc)
    fin = np.isfinite(r["logw"]) & (r["S"] > 1e-6)
    assert spearman(g["logw"][fin], r["logw"][fin]) >= 0.93
    assert topk_overlap(g["logw"][fin], r["logw"][fin]) >= 8
    assert np.argmax(g["w"]) == 40
