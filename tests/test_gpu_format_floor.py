"""Parity bars of the BF16 and FP8 tensor-core forms, derived from each
format's own error floor (tests/format_floor.py): the NeRF MLP on its plain
layer structure with every matrix-product operand rounded to the format and
FP32 accumulation, rendered with the FP64 oracle's pinned pieces.  The floor
is what any kernel that computes with these operand formats carries against
the FP64 oracle; the library's forms round at different points (the linear
feature layer folded into the RGB hidden layer, the density head as an extra
output row, gamma(d) as a per-ray FP32 bias, the RGB output layer in FP32),
so they are held to a stated multiple of the floor rather than to it:

  RGB error (all rays, none excluded):  mean <= K mean_floor,
                                        99th percentile <= K p99_floor,
                                        max <= K max_floor;
  particle ranking:  1 - Spearman <= max(K (1 - Spearman_floor), 2e-3),
                     top-10 overlap >= min(9, top10_floor - 1);
  K = 2.

The floor and the measured errors are printed (the numbers behind the
reduced-precision rows of the design notes)."""
import numpy as np
import pytest

import format_floor
from gpu_helpers import lib, make_scene, run_gpu_update, run_oracle_update

pytestmark = pytest.mark.gpu

K = 2.0
SCENES = {
    "c1 (seed-0 map, 32 coarse)": (0, 0, 32, 8, 100, 100, 138.9, 32, 0, False),
    "hierarchical (seed-2 map, 64+128)": (2, 31, 40, 8, 400, 400, 555.6, 64, 128, True),
    "hierarchical (seed-0 map, 64+128)": (0, 33, 40, 8, 400, 400, 555.6, 64, 128, True),
}
FORMATS = {"bf16": "bf16", "fp8": "e4m3"}


@pytest.fixture(scope="module")
def M():
    return lib()


@pytest.fixture(scope="module")
def maps(M):
    import synth
    cache = {}

    def get(seed):
        if seed not in cache:
            cache[seed] = M.Map(synth.he_init_weights(seed), max_rays=40000, max_samples=192,
                                max_particles=4096)
        return cache[seed]
    yield get
    for m in cache.values():
        m.close()


def _stats(rgb, ref, logw, logw_ref, S_ref):
    from scipy.stats import spearmanr
    e = np.abs(rgb - ref)
    fin = np.isfinite(logw) & np.isfinite(logw_ref) & (S_ref > 1e-6)
    rho = float(spearmanr(logw[fin], logw_ref[fin]).correlation)
    top = len(set(np.argsort(-logw[fin])[:10]) & set(np.argsort(-logw_ref[fin])[:10]))
    return dict(mean=float(e.mean()), p99=float(np.quantile(e, 0.99)), max=float(e.max()),
                spearman=rho, top10=top)


@pytest.mark.parametrize("scene_name", list(SCENES))
@pytest.mark.parametrize("precision", list(FORMATS))
def test_update_error_within_format_floor(M, maps, scene_name, precision):
    a = SCENES[scene_name]
    sc = make_scene(a[0], *a[1:9], add_gt=a[9])
    gm = maps(a[0])
    if not gm.supports(precision):
        pytest.skip(f"{precision} unavailable")
    r = run_oracle_update(sc)
    fl = format_floor.render_scene(sc, FORMATS[precision])
    g = run_gpu_update(M, gm, sc, precision=precision)
    floor = _stats(fl["rgb"], r["rgb"], fl["logw"], r["logw"], r["S"])
    got = _stats(g["rgb"], r["rgb"], g["logw"], r["logw"], r["S"])
    print(f"\n{precision} {scene_name}\n  floor {floor}\n  gpu   {got}\n  ratios mean "
          f"{got['mean'] / floor['mean']:.2f} p99 {got['p99'] / floor['p99']:.2f} max "
          f"{got['max'] / floor['max']:.2f}")
    assert got["mean"] <= K * floor["mean"]
    assert got["p99"] <= K * floor["p99"]
    assert got["max"] <= K * floor["max"]
    assert 1.0 - got["spearman"] <= max(K * (1.0 - floor["spearman"]), 2e-3)
    assert got["top10"] >= min(9, floor["top10"] - 1)
    assert abs(g["w"].sum() - 1.0) < 1e-12


@pytest.mark.parametrize("precision", list(FORMATS))
@pytest.mark.parametrize("seed", [0, 2])
def test_points_error_within_format_floor(M, maps, precision, seed):
    """The MLP alone at 4,097 points of [-6, 6]^3: RGB and density errors
    (density relative to its spread over the volume) against the floor."""
    import torch
    import oracle
    import synth
    gm = maps(seed)
    if not gm.supports(precision):
        pytest.skip(f"{precision} unavailable")
    rng = np.random.default_rng(777 + seed)
    x = rng.uniform(-6, 6, size=(4097, 3)).astype(np.float32).astype(np.float64)
    d = rng.normal(size=(4097, 3))
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32).astype(np.float64)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    blob = synth.he_init_weights(seed)
    s_ref, c_ref = oracle.mlp(blob, x, d)
    s_fl, c_fl = format_floor.mlp_rounded(blob, x, d, FORMATS[precision])
    out = gm.query(torch.tensor(x, dtype=torch.float32, device="cuda"),
                   torch.tensor(d, dtype=torch.float32, device="cuda"), precision).cpu().numpy()
    spread = float(np.std(s_ref))
    res = {}
    for name, s, c in (("floor", s_fl, c_fl), ("gpu", out[:, 0], out[:, 1:])):
        ec = np.abs(c - c_ref)
        es = np.abs(s - s_ref) / spread
        res[name] = dict(rgb_mean=float(ec.mean()), rgb_max=float(ec.max()),
                         sig_mean=float(es.mean()), sig_max=float(es.max()))
    print(f"\n{precision} points seed {seed}: {res}")
    for k in ("rgb_mean", "rgb_max", "sig_mean", "sig_max"):
        assert res["gpu"][k] <= K * res["floor"][k], k
