"""The C-ABI shared library builds, loads without a GPU, and exports every
function that include/*.h declares.  No compute call is made here."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(mcl_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def built_lib():
    from paper_2406_12202_gb300 import build as B
    return B.build()


def test_header_declares_entry_points():
    names = declared_functions()
    for n in ("mcl_init_map", "mcl_update", "mcl_resample"):
        assert n in names


def test_library_exports_every_declared_symbol(built_lib):
    lib = ctypes.CDLL(built_lib)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_declared_symbol():
    import paper_2406_12202_gb300 as M
    assert sorted(M.EXPORTED) == [n for n in declared_functions() if n in M.EXPORTED]
    assert set(declared_functions()) <= set(M.EXPORTED)


def test_last_error_without_gpu(built_lib):
    """A fresh process starts with an empty error message (checked in a
    child process: the message is per thread and earlier tests in this one
    may have set it)."""
    import subprocess
    import sys
    code = ("import ctypes, sys; lib = ctypes.CDLL(sys.argv[1]); "
            "lib.mcl_last_error.restype = ctypes.c_char_p; print(repr(lib.mcl_last_error()))")
    out = subprocess.run([sys.executable, "-c", code, built_lib], capture_output=True, text=True,
                         check=True).stdout.strip()
    assert out == "b''"


def header_defines():
    vals = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        for m in re.finditer(r"^#define\s+(MCL_[A-Z0-9_]+)\s+\(?(-?\d+)\)?", src, flags=re.M):
            vals[m.group(1)] = int(m.group(2))
        for m in re.finditer(r"\b(MCL_PREC_[A-Z0-9]+)\s*=\s*(\d+)", src):
            vals[m.group(1)] = int(m.group(2))
    return vals


def test_binding_constants_match_header():
    """The binding's copies of the header's constants (error codes, sizes,
    the number of MLP kernel variants, the profiled phases) are the
    header's values."""
    import paper_2406_12202_gb300 as M
    d = header_defines()
    for name in ("MCL_OK", "MCL_ERR_ARG", "MCL_ERR_CUDA", "MCL_ERR_NONFINITE", "MCL_ERR_TIMEOUT",
                 "MCL_ERR_UNSUPPORTED", "MCL_ERR_DEGENERATE"):
        assert getattr(M, name) == d[name], name
    assert M.MAX_STAGES == d["MCL_MAX_STAGES"]
    assert M.RESAMPLE_NOALLOC_MAX_IN == d["MCL_RESAMPLE_NOALLOC_MAX_IN"]
    assert M.PROPOSAL_N_WEIGHTS == d["MCL_PROPOSAL_N_WEIGHTS"]
    assert M.N_PHASES == d["MCL_N_PHASES"]
    assert M.MLP_VARIANTS == d["MCL_MLP_VARIANTS"]
    assert sorted(M.MLP_VARIANT_TABLE) == list(range(d["MCL_MLP_VARIANTS"]))
    assert {v[0] for v in M.MLP_VARIANT_TABLE.values()} == {"bf16", "fp8"}
    for prec, code in (("FP32", M.PREC_FP32), ("BF16", M.PREC_BF16), ("FP8", M.PREC_FP8)):
        assert d["MCL_PREC_" + prec] == code


STRUCTS = {"Arch": "mcl_arch", "MapConfig": "mcl_map_config", "Intrinsics": "mcl_intrinsics",
           "Opts": "mcl_opts", "Debug": "mcl_debug", "Schedule": "mcl_schedule",
           "IterRecord": "mcl_iter_record", "TrainCfg": "mcl_train_cfg", "FitCfg": "mcl_fit_cfg"}


def test_struct_layouts_match_binding(tmp_path):
    """Every ctypes structure of the binding has the size, field names and
    field offsets of its C struct in include/mcl.h, as the host C compiler
    lays it out (a plain C program prints sizeof / offsetof)."""
    import ctypes as C
    import shutil
    import subprocess
    import paper_2406_12202_gb300 as M
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "mcl.h"', "int main(void) {"]
    for py, cs in STRUCTS.items():
        lines.append(f'    printf("{py} sizeof %zu\\n", sizeof({cs}));')
        for f in getattr(M, py)._fields_:
            lines.append(f'    printf("{py} {f[0]} %zu\\n", offsetof({cs}, {f[0]}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = {}
    for line in subprocess.check_output([str(exe)], text=True).splitlines():
        py, field, val = line.split()
        got[(py, field)] = int(val)
    for py in STRUCTS:
        cls = getattr(M, py)
        assert got[(py, "sizeof")] == C.sizeof(cls), py
        for f in cls._fields_:
            assert got[(py, f[0])] == getattr(cls, f[0]).offset, (py, f[0])


def test_decode_log_order_and_fields():
    """mcl_localize writes record q * iterations + t for query q, iteration t;
    the binding decodes it into per-query lists with every field."""
    import ctypes as C
    import numpy as np
    import torch
    import paper_2406_12202_gb300 as M
    Q, T = 3, 4
    recs = (M.IterRecord * (Q * T))()
    for q in range(Q):
        for t in range(T):
            r = recs[q * T + t]
            r.stage, r.level, r.n_particles, r.n_pixels = t % 3, (t + 1) % 3, 1000 + q, 16 << q
            r.n_survivors, r.status, r.spread = 900 + t, q, 0.5 ** t
            for i in range(4):
                r.est[i] = q + 0.25 * i - t
            r.t_start_ns = (1 << 40) + 1000 * q + t
    log = torch.from_numpy(np.frombuffer(bytes(recs), dtype=np.uint8).copy())
    out = M.Map.decode_log(log, Q, T)
    assert len(out) == Q and all(len(rows) == T for rows in out)
    for q in range(Q):
        for t in range(T):
            d = out[q][t]
            assert (d["stage"], d["level"], d["n_particles"], d["n_pixels"]) == (t % 3, (t + 1) % 3,
                                                                                  1000 + q, 16 << q)
            assert (d["n_survivors"], d["status"], d["spread"]) == (900 + t, q, 0.5 ** t)
            assert d["est"] == [q + 0.25 * i - t for i in range(4)]
            assert d["t_start_ns"] == (1 << 40) + 1000 * q + t
    assert C.sizeof(M.IterRecord) * Q * T == log.numel()
