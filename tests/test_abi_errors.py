"""Argument errors at the C boundary, without a GPU: every entry point below
rejects a NULL map or handle, a missing buffer, or a size outside its
documented range with MCL_ERR_ARG before any CUDA call, and leaves a message
naming the call for mcl_last_error (include/mcl.h: "negative MCL_ERR_* code;
mcl_last_error() ...").  Pointers passed are NULL or never dereferenced."""
import ctypes as C

import pytest

import paper_2406_12202_gb300 as M


@pytest.fixture(scope="module")
def L():
    from paper_2406_12202_gb300 import build as B
    B.build()
    return M.lib()


FAKE = C.c_void_p(0x1000)   # non-NULL, never dereferenced: the call fails on another argument


def _cases(L):
    d, ll, i = C.c_double(), C.c_longlong(), C.c_int()
    fit = M.FitCfg()
    return [
        ("mcl_update", lambda: L.mcl_update(None, None, 1, None, None, 0, None, 1, None, None,
                                            None, None, None, None)),
        ("mcl_render", lambda: L.mcl_render(None, None, 1, None, 0, None, 1, None, None, None,
                                            None)),
        ("mcl_resample", lambda: L.mcl_resample(None, None, 1, 1, 0.5, None, None)),
        ("mcl_query", lambda: L.mcl_query(None, None, None, 1, 0, None, None)),
        ("mcl_predict", lambda: L.mcl_predict(None, 1, None, 1, 0.1, 0.1, 0, 0, None, None)),
        ("mcl_predict", lambda: L.mcl_predict(FAKE, 4, None, 8, 0.1, 0.1, 0, 0, FAKE, None)),
        ("mcl_predict", lambda: L.mcl_predict(FAKE, 4, None, 4, -1.0, 0.1, 0, 0, FAKE, None)),
        ("mcl_downscale", lambda: L.mcl_downscale(FAKE, 10, 10, 3, FAKE, None)),
        ("mcl_downscale", lambda: L.mcl_downscale(None, 8, 8, 2, FAKE, None)),
        ("mcl_position_spread", lambda: L.mcl_position_spread(FAKE, 0, FAKE, None)),
        ("mcl_draw_pixels", lambda: L.mcl_draw_pixels(0, 10, 4, 1, 0, FAKE, None)),
        ("mcl_draw_pixels", lambda: L.mcl_draw_pixels(100, 100, 2000, 1, 0, FAKE, None)),
        ("mcl_draw_pixels", lambda: L.mcl_draw_pixels(4, 4, 17, 1, 0, FAKE, None)),
        ("mcl_draw_pixels", lambda: L.mcl_draw_pixels(100, 100, 16, 1, 0, None, None)),
        ("mcl_resample_noalloc", lambda: L.mcl_resample_noalloc(None, 4, 4, 0.5, FAKE, None)),
        ("mcl_resample_noalloc", lambda: L.mcl_resample_noalloc(FAKE, 4, 70000, 0.5, FAKE, None)),
        ("mcl_resample_noalloc", lambda: L.mcl_resample_noalloc(FAKE, 4, 4, 1.0, FAKE, None)),
        ("mcl_read_status", lambda: L.mcl_read_status(None, C.byref(i), None)),
        ("mcl_profile_read", lambda: L.mcl_profile_read(None, C.byref(d), C.byref(ll), 0)),
        ("mcl_set_mlp_variant", lambda: L.mcl_set_mlp_variant(None, 1, 0)),
        ("mcl_autotune", lambda: L.mcl_autotune(None, 1, 100000, None, None, None)),
        ("mcl_inject_weight_stall", lambda: L.mcl_inject_weight_stall(None, 1, 1.0)),
        ("mcl_set_fused_epilogue", lambda: L.mcl_set_fused_epilogue(None, 1)),
        ("mcl_fit_map", lambda: L.mcl_fit_map(None, None, None, None, 1, C.byref(fit), None,
                                              None)),
        ("mcl_get_map_weights", lambda: L.mcl_get_map_weights(None, None, 0)),
        ("mcl_proposal_get", lambda: L.mcl_proposal_get(None, None, 0)),
        ("mcl_probe_mma_rate", lambda: L.mcl_probe_mma_rate(0, 0, 1, C.byref(d), None)),
        ("mcl_probe_mma_rate", lambda: L.mcl_probe_mma_rate(4, 5000, 1, C.byref(d), None)),
    ]


def test_argument_errors_before_any_cuda_call(L):
    for name, call in _cases(L):
        rc = call()
        msg = L.mcl_last_error().decode()
        assert rc == M.MCL_ERR_ARG, (name, rc, msg)
        assert msg, name
        # the message names the failing call (a size message may name only
        # the argument)
        assert name.replace("_odom", "") in msg or any(w in msg for w in ("N ", "n_bins", "N_")), \
            (name, msg)


def test_init_map_rejects_missing_arguments(L):
    out = C.c_void_p()
    assert L.mcl_init_map(None, 0, None, None, C.byref(out)) == M.MCL_ERR_ARG
    assert "mcl_init_map" in L.mcl_last_error().decode()
    assert L.mcl_init_map(None, 0, None, None, None) == M.MCL_ERR_ARG
    assert not out.value
