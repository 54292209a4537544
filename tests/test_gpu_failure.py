"""Failure detection on the GPU without a fault: the tensor-core MLP's
bounded waits.  mcl_inject_weight_stall holds back the weight stream of the
next MLP launches and shortens their wait limit, so the wait for the first
weight block runs out (nothing is in flight: no copy was issued).  The kernel
must then stop all its warps, release its tensor memory and exit; the map's
status word reports MCL_ERR_TIMEOUT to the host, and the next launches on the
same map and context run normally and give the same results as before."""
import time

import numpy as np
import pytest

import synth
from gpu_helpers import lib

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_expired_wait_reports_timeout_and_next_call_succeeds(precision):
    import torch
    M = lib()
    gm = M.Map(synth.he_init_weights(0), max_rays=4096, max_samples=64)
    try:
        if not gm.supports(precision):
            pytest.skip(f"{precision} not available")
        rng = np.random.default_rng(11)
        n = 3000
        x = torch.tensor(rng.uniform(-1.5, 1.5, size=(n, 3)), dtype=torch.float32, device="cuda")
        d = torch.tensor(rng.normal(size=(n, 3)), dtype=torch.float32, device="cuda")
        ref = gm.query(x, d, precision)
        torch.cuda.synchronize()
        assert gm.read_status()[0] == M.MCL_OK
        gm.inject_weight_stall(1, 2.0)
        t0 = time.perf_counter()
        gm.query(x, d, precision)           # returns OK; the device sees the stall
        torch.cuda.synchronize()
        waited = time.perf_counter() - t0
        assert gm.read_status()[0] == M.MCL_ERR_TIMEOUT
        assert waited < 1.0                 # the 2 ms limit ended the launch
        again = gm.query(x, d, precision)
        torch.cuda.synchronize()
        assert gm.read_status()[0] == M.MCL_OK
        assert torch.equal(again, ref)
    finally:
        gm.close()


def test_stall_hook_rejects_bad_arguments():
    M = lib()
    gm = M.Map(synth.he_init_weights(0), max_rays=64, max_samples=64)
    try:
        for n, ms in ((-1, 1.0), (1, 0.0), (1, 5000.0)):
            with pytest.raises(M.MclError) as e:
                gm.inject_weight_stall(n, ms)
            assert e.value.code == M.MCL_ERR_ARG
        gm.inject_weight_stall(0, 1.0)
    finally:
        gm.close()
