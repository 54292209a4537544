"""mcl_resample_noalloc: systematic resampling for callers that cannot
allocate device memory (no map; the scratch is a fixed array in the library
image).  It must return exactly the indices of the FP64 oracle's resampling
rule, and of the map-based mcl_resample, call after call.

The file name makes pytest collect it last.  The tests do not depend on what
ran before them (each test makes its own first call, which also performs the
one-time per-device address lookup of the scratch array); the order only
means that, in a run stopped at the first failure, every other test has
already run when one of these fails."""
import ctypes as C

import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import lib

pytestmark = pytest.mark.gpu


def test_noalloc_matches_oracle_and_map_resample_on_consecutive_calls():
    import torch
    M = lib()
    gm = M.Map(synth.he_init_weights(0), max_rays=64, max_samples=64, max_particles=8000)
    try:
        # a large call, then a smaller one that must not see the first call's
        # leftover scratch, then one with zero weights in it
        for n_in, n_out, seed in ((6000, 6000, 1), (1500, 3000, 2), (700, 65536, 3)):
            wh = synth.random_weights(seed, n_in, zero_frac=0.3)
            w = torch.tensor(wh, dtype=torch.float64, device="cuda")
            u0 = synth.resample_u0(seed)
            got = M.resample_noalloc(w, n_out, u0).cpu().numpy()
            ref = gm.resample(w, n_out, u0).cpu().numpy()
            assert np.array_equal(got, oracle.resample(wh, n_out, u0))
            assert np.array_equal(got, ref)
            assert got.min() >= 0 and got.max() < n_in
    finally:
        gm.close()


def test_noalloc_rejects_oversize_host_pointers_and_flags_degenerate_weights():
    import torch
    M = lib()
    L = M.lib()
    big = torch.ones(M.RESAMPLE_NOALLOC_MAX_IN + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(M.MclError) as e:
        M.resample_noalloc(big, 10, 0.5)
    assert e.value.code == M.MCL_ERR_ARG
    # host memory is not device memory of the current device: rejected
    # before anything is launched
    wh = np.ones(16, dtype=np.float64)
    idx = torch.empty(8, dtype=torch.int32, device="cuda")
    rc = L.mcl_resample_noalloc(wh.ctypes.data_as(C.c_void_p), 16, 8, C.c_double(0.5),
                                C.c_void_p(idx.data_ptr()),
                                C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == M.MCL_ERR_ARG and b"not device memory" in L.mcl_last_error()
    # all-zero weights: every index -1
    idx = M.resample_noalloc(torch.zeros(16, dtype=torch.float64, device="cuda"), 8, 0.5)
    assert np.all(idx.cpu().numpy() == -1)
    # the next call resamples normally and clears the error message
    wv = synth.random_weights(5, 16)
    w = torch.tensor(wv, dtype=torch.float64, device="cuda")
    got = M.resample_noalloc(w, 8, 0.25).cpu().numpy()
    assert np.array_equal(got, oracle.resample(wv, 8, 0.25))
    assert L.mcl_last_error() == b""
