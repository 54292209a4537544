"""mcl_resample_noalloc: systematic resampling for callers that cannot
allocate device memory (no map, scratch in a fixed array of the library).
It must return exactly the indices of the map-based mcl_resample, call after
call, since both evaluate the same integer rule.  Collected last on purpose."""
import numpy as np
import pytest

import synth
from gpu_helpers import lib

pytestmark = pytest.mark.gpu


def test_noalloc_matches_map_resample_on_consecutive_calls():
    import torch
    M = lib()
    gm = M.Map(synth.he_init_weights(0), max_rays=64, max_samples=64, max_particles=8000)
    try:
        # a large call, then a smaller one that must not see the first call's
        # leftover scratch, then one with zero weights in it
        for n_in, n_out, seed in ((6000, 6000, 1), (1500, 3000, 2), (700, 65536, 3)):
            w = torch.tensor(synth.random_weights(seed, n_in, zero_frac=0.3), dtype=torch.float64,
                             device="cuda")
            u0 = synth.resample_u0(seed)
            ref = gm.resample(w, n_out, u0).cpu().numpy()
            got = M.resample_noalloc(w, n_out, u0).cpu().numpy()
            torch.cuda.synchronize()
            assert np.array_equal(got, ref)
            assert got.min() >= 0 and got.max() < n_in
    finally:
        gm.close()


def test_noalloc_rejects_oversize_and_flags_degenerate_weights():
    import torch
    M = lib()
    big = torch.ones(M.RESAMPLE_NOALLOC_MAX_IN + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(M.MclError) as e:
        M.resample_noalloc(big, 10, 0.5)
    assert e.value.code == M.MCL_ERR_ARG
    idx = M.resample_noalloc(torch.zeros(16, dtype=torch.float64, device="cuda"), 8, 0.5)
    assert np.all(idx.cpu().numpy() == -1)
    # the next call starts from a clean status and resamples normally
    w = torch.tensor(synth.random_weights(5, 16), dtype=torch.float64, device="cuda")
    assert M.resample_noalloc(w, 8, 0.25).cpu().numpy().min() >= 0
