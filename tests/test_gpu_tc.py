"""Tensor-core (tcgen05, BF16 operands, FP32 accumulation) form of the NeRF
MLP against the FP64 oracle: the MLP itself at sampled points, then whole
weight updates.

The bars derived from the BF16 format's own error floor (twice the error of
the plain layer structure with BF16-rounded operands, every ray counted) are
in test_gpu_format_floor.py; the checks below are the survey's absolute
bars where that floor allows them (the c1 workload: RGB max 2e-2, mean 5e-3,
Spearman 0.99, top-10 9) and coarser sanity bounds elsewhere.

BF16 bars (stated, not inherited from FP32): BF16 keeps 8 significant bits,
so each of the 63 positional-encoding inputs and 256 activations per layer
carries a relative rounding of up to 2^-9; through nine layers this gives
RGB errors of order 1e-2.  Bars: per-sample RGB max |err| <= 2.5e-2 and mean
<= 5e-3; rendered RGB
max <= 3e-2, mean <= 6e-3 without importance samples, max <= 8e-2, mean
<= 1.5e-2 with them (the inverse-CDF sampler amplifies any MLP difference,
see the FP32 tests), on rays whose last-sample density is not within the
BF16 band of zero (gpu_helpers.bf16_flip_prone, at most 15 % of rays);
particle ranking: Spearman correlation of log-weights >= 0.99 (0.97 with
importance samples) and top-10 overlap >= 9 (8).  Density at points: error
relative to the spread of sigma, max <= 0.1 and mean <= 0.02."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import bf16_flip_prone, lib, make_scene, run_gpu_update, run_oracle_update

pytestmark = pytest.mark.gpu


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
            assert maps[seed].supports("bf16"), "tensor-core form unavailable on this GPU"
        return maps[seed]
    yield get
    for m in maps.values():
        m.close()


def spearman(a, b):
    from scipy.stats import spearmanr
    return float(spearmanr(a, b).correlation)


def topk_overlap(a, b, k=10):
    return len(set(np.argsort(-a)[:k]) & set(np.argsort(-b)[:k]))


_SPREAD = {}


def sigma_spread(seed):
    """Standard deviation of the map's raw density over the sample volume
    (oracle, 2048 seeded points): the scale the density error is judged on."""
    if seed not in _SPREAD:
        rng = np.random.default_rng(12345)
        x = rng.uniform(-6, 6, size=(2048, 3))
        d = rng.normal(size=(2048, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        _SPREAD[seed] = float(np.std(oracle.mlp(synth.he_init_weights(seed), x, d)[0]))
    return _SPREAD[seed]


@pytest.mark.parametrize("n", [1, 127, 128, 129, 256, 4097])
def test_mlp_points_bf16_vs_oracle(M, gmaps, n):
    """Ragged row counts around the 128-row tile and 256-row pair."""
    import torch
    rng = np.random.default_rng(n)
    x = rng.uniform(-6, 6, size=(n, 3)).astype(np.float32)
    d = rng.normal(size=(n, 3))
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    gm = gmaps(2)
    out = gm.query(torch.tensor(x, device="cuda"), torch.tensor(d, device="cuda"), "bf16").cpu().numpy()
    s_ref, rgb_ref = oracle.mlp(synth.he_init_weights(2), x.astype(np.float64),
                                d.astype(np.float64) / np.linalg.norm(d.astype(np.float64), axis=1, keepdims=True))
    assert np.all(np.isfinite(out))
    e_rgb = np.abs(out[:, 1:] - rgb_ref)
    e_sig = np.abs(out[:, 0] - s_ref) / sigma_spread(2)
    print(f"n={n} rgb max {e_rgb.max():.3g} mean {e_rgb.mean():.3g} sigma rel max {e_sig.max():.3g}")
    assert e_rgb.max() <= 2.5e-2 and e_rgb.mean() <= 5e-3
    assert e_sig.max() <= 0.1 and e_sig.mean() <= 0.02


def test_mlp_points_fp32_vs_oracle(M, gmaps):
    import torch
    rng = np.random.default_rng(7)
    n = 3000
    x = rng.uniform(-6, 6, size=(n, 3)).astype(np.float32)
    d = rng.normal(size=(n, 3)).astype(np.float32)
    gm = gmaps(0)
    out = gm.query(torch.tensor(x, device="cuda"), torch.tensor(d, device="cuda"), "fp32").cpu().numpy()
    dd = d.astype(np.float64)
    s_ref, rgb_ref = oracle.mlp(synth.he_init_weights(0), x.astype(np.float64),
                                dd / np.linalg.norm(dd, axis=1, keepdims=True))
    assert np.all(np.abs(out[:, 1:] - rgb_ref) <= 1e-4 * np.abs(rgb_ref) + 1e-6)
    assert np.all(np.abs(out[:, 0] - s_ref) <= 1e-4 * np.abs(s_ref) + 1e-4)


def _bf16_update(M, gmaps, sc, max_abs, mean_abs, rho, topk):
    g = run_gpu_update(M, gmaps(sc["map_seed"]), sc, precision="bf16")
    r = run_oracle_update(sc)
    flip = bf16_flip_prone(r)
    assert flip.mean() <= 0.15, flip.mean()
    e = np.abs(g["rgb"] - r["rgb"])[~flip]
    rep = dict(rgb_max=float(e.max()), rgb_mean=float(e.mean()), flip_rays=int(flip.sum()))
    fin = np.isfinite(r["logw"]) & (r["S"] > 1e-6)
    rep["spearman"] = spearman(g["logw"][fin], r["logw"][fin])
    rep["top10"] = topk_overlap(g["logw"][fin], r["logw"][fin])
    print(rep)
    assert e.max() <= max_abs and e.mean() <= mean_abs, rep
    assert rep["spearman"] >= rho, rep
    assert rep["top10"] >= topk, rep
    assert abs(g["w"].sum() - 1.0) < 1e-12
    return g, r


def scene(map_seed, *a, **k):
    sc = make_scene(map_seed, *a, **k)
    sc["map_seed"] = map_seed
    return sc


def test_bf16_update_c1_workload(M, gmaps):
    sc = scene(0, 0, 32, 8, 100, 100, 138.9, 32, 0, add_gt=False)
    _bf16_update(M, gmaps, sc, 2e-2, 5e-3, 0.99, 9)


def test_bf16_update_hierarchical(M, gmaps):
    sc = scene(2, 31, 40, 8, 400, 400, 555.6, 64, 128, add_gt=True)
    g, r = _bf16_update(M, gmaps, sc, 8e-2, 1.5e-2, 0.97, 8)
    assert np.argmax(g["w"]) == 40 and np.argmax(r["w"]) == 40


def test_bf16_update_ragged(M, gmaps):
    sc = scene(2, 32, 7, 5, 60, 40, 70.0, 17, 33, add_gt=False)
    g = run_gpu_update(M, gmaps(2), sc, precision="bf16")
    r = run_oracle_update(sc)
    flip = bf16_flip_prone(r)
    e = np.abs(g["rgb"] - r["rgb"])[~flip]
    assert np.all(np.isfinite(g["rgb"])) and e.max() <= 8e-2 and e.mean() <= 1.5e-2


def test_bf16_full_c2_against_fp32_form(M, gmaps):
    """Full 600 x 64 update in both forms on the GPU: same ranking of
    particles, RGB close (the oracle check at this size is the sampled test
    below)."""
    sc = scene(0, 9, 600, 64, 400, 400, 555.6, 64, 128, add_gt=False)
    gm = gmaps(0)
    g16 = run_gpu_update(M, gm, sc, precision="bf16")
    g32 = run_gpu_update(M, gm, sc, precision="fp32")
    e = np.abs(g16["rgb"] - g32["rgb"])
    print("bf16 vs fp32 full c2:", e.max(), e.mean(), spearman(g16["logw"], g32["logw"]))
    assert e.mean() <= 1.5e-2
    assert spearman(g16["logw"], g32["logw"]) >= 0.97
    # sampled particles against the oracle
    pick = [5, 300, 598]
    sub = dict(sc)
    sub["P"] = sc["P"][pick]
    r = run_oracle_update(sub)
    rays = np.concatenate([np.arange(i * 64, (i + 1) * 64) for i in pick])
    flip = bf16_flip_prone(r)
    e2 = np.abs(g16["rgb"][rays] - r["rgb"])[~flip]
    assert e2.max() <= 8e-2 and e2.mean() <= 1.5e-2
