"""Kernel variants of the tensor-core MLP (epilogue warps per tile, lockstep
or staggered tiles) and the autotuner that picks among them.  The variants
reorder work, not arithmetic: every variant of a precision must give
bit-identical outputs."""
import numpy as np
import pytest

import synth
from gpu_helpers import lib, make_scene, run_gpu_update

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    return lib()


@pytest.fixture(scope="module")
def gm(M):
    m = M.Map(synth.he_init_weights(2), max_rays=40000, max_samples=192, max_particles=4096)
    yield m
    m.close()


def _variants(M, prec):
    return [i for i, v in M.MLP_VARIANT_TABLE.items() if v[0] == prec]


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_variants_bit_identical_points(M, gm, prec):
    import torch
    rng = np.random.default_rng(5)
    n = 3000   # ragged: 11.7 tile pairs
    x = torch.tensor(rng.uniform(-6, 6, size=(n, 3)), dtype=torch.float32, device="cuda")
    d = torch.tensor(rng.normal(size=(n, 3)), dtype=torch.float32, device="cuda")
    outs = []
    for v in _variants(M, prec):
        gm.set_mlp_variant(prec, v)
        outs.append(gm.query(x, d, prec))
    torch.cuda.synchronize()
    assert all(torch.equal(outs[0], o) for o in outs[1:])
    assert torch.isfinite(outs[0]).all()


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_variants_bit_identical_update(M, gm, prec):
    sc = make_scene(2, 31, 40, 8, 400, 400, 555.6, 64, 128, add_gt=True)
    res = []
    for v in _variants(M, prec):
        gm.set_mlp_variant(prec, v)
        res.append(run_gpu_update(M, gm, sc, precision=prec))
    for r in res[1:]:
        for k in ("rgb", "logw", "w", "F"):
            assert np.array_equal(np.nan_to_num(res[0][k], nan=7.0), np.nan_to_num(r[k], nan=7.0)), k


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_autotune_picks_a_variant_of_the_precision(M, gm, prec):
    chosen, ms = gm.autotune(prec, 256 * 152 * 8)
    assert chosen in _variants(M, prec)
    assert set(ms) == set(_variants(M, prec))
    assert all(v > 0 for v in ms.values())
    assert ms[chosen] == min(ms.values())


def test_variant_and_autotune_arguments_checked(M, gm):
    with pytest.raises(M.MclError):
        gm.set_mlp_variant("bf16", 5)       # an FP8 variant
    with pytest.raises(M.MclError):
        gm.autotune("bf16", 10)             # too few rows
    with pytest.raises(M.MclError):
        gm.autotune("fp32", 100000)         # no variants
