"""Python front of the FP64 CPU oracle (``oracle/orc.c``).

TEST INFRASTRUCTURE.  Only the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
GPU library never imports it and shares no code with it; the only module both
sides read is ``synth`` (seeded input generators, none of the method's
arithmetic).

The C file is compiled on first use (``gcc -O2 -fopenmp``) into
``oracle/_build/liborc.so``; ``build()`` does it explicitly.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "orc.c")
_OUT = os.path.join(_HERE, "_build", "liborc.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (plain C, portable flags)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


class Opts(C.Structure):
    """Mirror of orc_opts in orc.c."""
    _fields_ = [("near_z", C.c_double), ("far_z", C.c_double),
                ("alpha", C.c_double), ("tau", C.c_double),
                ("rho", C.c_double), ("s_min", C.c_double),
                ("n_coarse", C.c_int), ("n_fine", C.c_int),
                ("use_rejection", C.c_int), ("pad", C.c_int)]


def make_opts(n_coarse=64, n_fine=128, near=2.0, far=6.0, alpha=0.05,
              tau=0.1, rho=1e-3, s_min=1e-30, use_rejection=True) -> Opts:
    return Opts(near, far, alpha, tau, rho, s_min, n_coarse, n_fine,
                int(bool(use_rejection)), 0)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            fp = C.POINTER(C.c_float)
            ip = C.POINTER(C.c_int)
            L.orc_n_weights.restype = C.c_long
            L.orc_n_weights.argtypes = [ip]
            L.orc_pe.argtypes = [dp, C.c_int, dp]
            L.orc_mlp.argtypes = [fp, ip, C.c_int, dp, dp, dp, dp]
            L.orc_ray.argtypes = [dp] + [C.c_double] * 6 + [dp, dp]
            L.orc_composite.argtypes = [C.c_int, dp, dp, dp, C.c_double, dp, dp, dp]
            L.orc_sample_pdf.argtypes = [C.c_int, dp, dp, C.c_int, dp, dp]
            L.orc_uncertainty.argtypes = [C.c_int, dp, dp, C.c_double, C.c_double,
                                          dp, dp, dp, dp, dp]
            L.orc_render_rays.argtypes = [fp, ip, C.c_int, dp, dp, C.POINTER(Opts),
                                          dp, dp, dp, dp]
            L.orc_downscale.argtypes = [dp, C.c_int, C.c_int, C.c_int, dp]
            L.orc_update.argtypes = [fp, ip, dp, C.c_int, dp, C.c_int, C.c_int, dp,
                                     C.c_int, C.POINTER(C.c_int32), C.c_int,
                                     C.POINTER(Opts), dp, dp, dp, dp, dp, dp, dp,
                                     dp, dp, dp, dp, dp, dp, C.POINTER(C.c_uint8)]
            L.orc_resample.argtypes = [dp, C.c_int, C.c_int, C.c_double,
                                       C.POINTER(C.c_int32)]
            L.orc_splitmix64_next.restype = C.c_uint64
            L.orc_splitmix64_next.argtypes = [C.POINTER(C.c_uint64)]
            L.orc_cbrng.restype = C.c_uint64
            L.orc_cbrng.argtypes = [C.c_uint64] * 3
            L.orc_uniform.restype = C.c_double
            L.orc_uniform.argtypes = [C.c_uint64] * 3
            L.orc_normal.restype = C.c_double
            L.orc_normal.argtypes = [C.c_uint64] * 3
            L.orc_se3_exp.argtypes = [dp, dp, dp]
            L.orc_predict.argtypes = [C.c_int, dp, dp, dp]
            L.orc_predict_odom.argtypes = [C.c_int, dp, dp, dp, dp]
            L.orc_motion_noise.argtypes = [C.c_int, C.c_uint64, C.c_uint64,
                                           C.c_double, C.c_double, dp]
            L.orc_position_spread.argtypes = [C.c_int, dp, dp]
            L.orc_loop_statistics.argtypes = [C.c_int, dp, dp, C.POINTER(C.c_uint8), dp]
            L.orc_loop_schedule.argtypes = [ip, C.c_int, dp, ip, ip, C.c_int, C.c_int,
                                            C.c_double, C.c_int]
            L.orc_num_threads.restype = C.c_int
            L.orc_pixel_set.argtypes = [C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_uint64,
                                        C.POINTER(C.c_int32)]
            L.orc_prop_n_weights.restype = C.c_long
            L.orc_prop_forward.argtypes = [fp, C.c_int, dp, dp]
            L.orc_histogram.argtypes = [C.c_int, dp, dp, C.c_int, C.c_double, C.c_double, dp]
            L.orc_prop_loss_grad.argtypes = [fp, C.c_int, dp, dp, C.c_int, C.c_double, C.c_double,
                                             dp, dp, dp]
            L.orc_prop_weights.argtypes = [fp, C.c_int, dp, dp, C.c_int, C.c_double, C.c_double, dp]
            L.orc_render_rays_proposal.argtypes = [fp, ip, fp, C.c_int, dp, dp, C.POINTER(Opts),
                                                   C.c_int, C.c_int, dp]
            _lib = L
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def _arch(arch):
    a = np.ascontiguousarray(np.asarray(arch, dtype=np.int32))
    return a, a.ctypes.data_as(C.POINTER(C.c_int))


def _blob(blob):
    b = np.ascontiguousarray(blob, dtype=np.float32)
    return b, b.ctypes.data_as(C.POINTER(C.c_float))


DEFAULT_ARCH = (10, 4, 8, 256, 5, 128)


def num_threads() -> int:
    return lib().orc_num_threads()


def n_weights(arch=DEFAULT_ARCH) -> int:
    a, ap = _arch(arch)
    return int(lib().orc_n_weights(ap))


def pe(p, L):
    p, pp = _d(p)
    out = np.zeros(3 + 6 * L)
    lib().orc_pe(pp, L, out.ctypes.data_as(C.POINTER(C.c_double)))
    return out


def mlp(blob, x, dhat, arch=DEFAULT_ARCH):
    """sigma_raw [n], rgb [n,3] of the NeRF MLP at points x [n,3], unit view
    directions dhat [n,3]."""
    b, bp = _blob(blob)
    a, ap = _arch(arch)
    x, xp = _d(np.reshape(x, (-1, 3)))
    dh, dp_ = _d(np.reshape(dhat, (-1, 3)))
    n = x.shape[0]
    s = np.zeros(n)
    rgb = np.zeros((n, 3))
    rc = lib().orc_mlp(bp, ap, n, xp, dp_, s.ctypes.data_as(C.POINTER(C.c_double)),
                       rgb.ctypes.data_as(C.POINTER(C.c_double)))
    assert rc == 0, rc
    return s, rgb


def ray(pose, fx, fy, cx, cy, u, v):
    P, pp = _d(pose)
    o = np.zeros(3)
    d = np.zeros(3)
    lib().orc_ray(pp, fx, fy, cx, cy, float(u), float(v),
                  o.ctypes.data_as(C.POINTER(C.c_double)),
                  d.ctypes.data_as(C.POINTER(C.c_double)))
    return o, d


def composite(z, sigma_raw, rgb, dnorm):
    z, zp = _d(z)
    s, sp = _d(sigma_raw)
    c, cp = _d(np.reshape(rgb, (-1, 3)))
    n = z.shape[0]
    w = np.zeros(n)
    T = np.zeros(n)
    Cc = np.zeros(3)
    lib().orc_composite(n, zp, sp, cp, float(dnorm),
                        w.ctypes.data_as(C.POINTER(C.c_double)),
                        T.ctypes.data_as(C.POINTER(C.c_double)),
                        Cc.ctypes.data_as(C.POINTER(C.c_double)))
    return w, T, Cc


def sample_pdf(z_c, w_c, n_f, u=None):
    z_c, zp = _d(z_c)
    w_c, wp = _d(w_c)
    if u is None:
        u = np.linspace(0.0, 1.0, n_f) if n_f > 1 else np.zeros(n_f)
    u, up = _d(u)
    zf = np.zeros(n_f)
    lib().orc_sample_pdf(z_c.shape[0], zp, wp, n_f, up,
                         zf.ctypes.data_as(C.POINTER(C.c_double)))
    return zf


def uncertainty(z, w, alpha, tau):
    z, zp = _d(z)
    w, wp = _d(w)
    out = np.zeros(5)
    o = out.ctypes.data_as(C.POINTER(C.c_double))
    dp = C.POINTER(C.c_double)
    base = C.addressof(o.contents)
    lib().orc_uncertainty(z.shape[0], zp, wp, float(alpha), float(tau),
                          C.cast(base, dp), C.cast(base + 8, dp),
                          C.cast(base + 16, dp), C.cast(base + 24, dp), C.cast(base + 32, dp))
    return dict(z_trans=out[0], z_opaque=out[1], F=out[2], tie=out[3], step=out[4])


def render_rays(blob, o, d, opts: Opts, uj=None, arch=DEFAULT_ARCH, debug=False):
    """Render rays o, d [n,3].  Returns dict rgb [n,3], z_trans, z_opaque, F,
    tie [n] (and z, w [n, n_c + n_f] with debug=True)."""
    b, bp = _blob(blob)
    a, ap = _arch(arch)
    o, op_ = _d(np.reshape(o, (-1, 3)))
    d, dp_ = _d(np.reshape(d, (-1, 3)))
    n = o.shape[0]
    out = np.zeros((n, 10))
    ns = opts.n_coarse + opts.n_fine
    zd = np.zeros((n, ns)) if debug else None
    wd = np.zeros((n, ns)) if debug else None
    ujp = None
    if uj is not None:
        uj, ujp = _d(np.reshape(uj, (n, opts.n_coarse)))
    P = C.POINTER(C.c_double)
    rc = lib().orc_render_rays(bp, ap, n, op_, dp_, C.byref(opts), ujp,
                               out.ctypes.data_as(P),
                               zd.ctypes.data_as(P) if debug else None,
                               wd.ctypes.data_as(P) if debug else None)
    assert rc == 0, rc
    res = dict(rgb=out[:, :3].copy(), z_trans=out[:, 3].copy(),
               z_opaque=out[:, 4].copy(), F=out[:, 5].copy(), tie=out[:, 6].copy(),
               sigma_last=out[:, 7].copy(), T_last=out[:, 8].copy(), step=out[:, 9].copy())
    if debug:
        res["z"] = zd
        res["w"] = wd
    return res


def downscale(img, factor):
    img, ip = _d(img)
    H, W, _ = img.shape
    out = np.zeros((H // factor, W // factor, 3))
    rc = lib().orc_downscale(ip, W, H, factor, out.ctypes.data_as(C.POINTER(C.c_double)))
    assert rc == 0
    return out


def update(blob, particles, image, K4, factor, pixels, opts: Opts, uj=None,
           arch=DEFAULT_ARCH):
    """One weight update (Alg. 1 with Eq. 6).  Returns a dict of per-ray
    (rgb, E, F, z_trans, z_opaque, tie; shape [N*B]) and per-particle
    (S, logw, w, mask; shape [N]) results."""
    b, bp = _blob(blob)
    a, ap = _arch(arch)
    P, pp = _d(np.reshape(particles, (-1, 12)))
    N = P.shape[0]
    img, imgp = _d(image)
    H, W, _ = img.shape
    K, kp = _d(K4)
    px = np.ascontiguousarray(pixels, dtype=np.int32).reshape(-1, 2)
    B = px.shape[0]
    nr = N * B
    res = {k: np.zeros(nr) for k in ("E", "F", "z_trans", "z_opaque", "tie", "sigma_last",
                                     "T_last", "step")}
    res["rgb"] = np.zeros((nr, 3))
    for k in ("S", "logw", "w"):
        res[k] = np.zeros(N)
    res["mask"] = np.zeros(N, dtype=np.uint8)
    ujp = None
    if uj is not None:
        uj, ujp = _d(np.reshape(uj, (nr, opts.n_coarse)))
    dp = C.POINTER(C.c_double)
    rc = lib().orc_update(bp, ap, pp, N, imgp, W, H, kp, int(factor),
                          px.ctypes.data_as(C.POINTER(C.c_int32)), B, C.byref(opts),
                          ujp, res["rgb"].ctypes.data_as(dp), res["E"].ctypes.data_as(dp),
                          res["F"].ctypes.data_as(dp), res["z_trans"].ctypes.data_as(dp),
                          res["z_opaque"].ctypes.data_as(dp), res["tie"].ctypes.data_as(dp),
                          res["sigma_last"].ctypes.data_as(dp), res["T_last"].ctypes.data_as(dp),
                          res["step"].ctypes.data_as(dp), res["S"].ctypes.data_as(dp), res["logw"].ctypes.data_as(dp),
                          res["w"].ctypes.data_as(dp),
                          res["mask"].ctypes.data_as(C.POINTER(C.c_uint8)))
    if rc != 0:
        raise ValueError(f"orc_update returned {rc}")
    return res


def resample(w, n_out, u0):
    w, wp = _d(w)
    idx = np.zeros(n_out, dtype=np.int32)
    rc = lib().orc_resample(wp, w.shape[0], int(n_out), float(u0),
                            idx.ctypes.data_as(C.POINTER(C.c_int32)))
    if rc != 0:
        raise ValueError(f"orc_resample returned {rc}")
    return idx


# ---------------------------------------------------------------- proposal
def prop_n_weights() -> int:
    return int(lib().orc_prop_n_weights())


def prop_forward(pblob, x):
    b, bp = _blob(pblob)
    x, xp = _d(np.reshape(x, (-1, 3)))
    out = np.zeros(x.shape[0])
    lib().orc_prop_forward(bp, x.shape[0], xp, out.ctypes.data_as(C.POINTER(C.c_double)))
    return out


def histogram(z, w, nb, near, far):
    z, zp = _d(z)
    w, wp = _d(w)
    out = np.zeros(nb)
    lib().orc_histogram(z.shape[0], zp, wp, nb, float(near), float(far),
                        out.ctypes.data_as(C.POINTER(C.c_double)))
    return out


def prop_loss_grad(pblob, o, d, hist, near=2.0, far=6.0, with_grad=True):
    b, bp = _blob(pblob)
    o, op_ = _d(np.reshape(o, (-1, 3)))
    d, dp_ = _d(np.reshape(d, (-1, 3)))
    n = o.shape[0]
    h, hp = _d(np.reshape(hist, (n, -1)))
    nb = h.shape[1]
    loss = np.zeros(1)
    grad = np.zeros(prop_n_weights()) if with_grad else None
    P = C.POINTER(C.c_double)
    lib().orc_prop_loss_grad(bp, n, op_, dp_, nb, float(near), float(far), hp,
                             loss.ctypes.data_as(P), grad.ctypes.data_as(P) if with_grad else None)
    return float(loss[0]), grad


def prop_weights(pblob, o, d, nb, near=2.0, far=6.0):
    b, bp = _blob(pblob)
    o, op_ = _d(np.reshape(o, (-1, 3)))
    d, dp_ = _d(np.reshape(d, (-1, 3)))
    out = np.zeros((o.shape[0], nb))
    lib().orc_prop_weights(bp, o.shape[0], op_, dp_, nb, float(near), float(far),
                           out.ctypes.data_as(C.POINTER(C.c_double)))
    return out


def render_rays_proposal(blob, pblob, o, d, opts: Opts, n_p=64, n_g=32, arch=DEFAULT_ARCH):
    """Render with the proposal sampler (n_p proposal samples, n_g guided
    samples, opts.n_fine importance samples from those)."""
    b, bp = _blob(blob)
    pb, pbp = _blob(pblob)
    a, ap = _arch(arch)
    o, op_ = _d(np.reshape(o, (-1, 3)))
    d, dp_ = _d(np.reshape(d, (-1, 3)))
    n = o.shape[0]
    out = np.zeros((n, 10))
    rc = lib().orc_render_rays_proposal(bp, ap, pbp, n, op_, dp_, C.byref(opts), n_p, n_g,
                                        out.ctypes.data_as(C.POINTER(C.c_double)))
    assert rc == 0, rc
    return dict(rgb=out[:, :3].copy(), z_trans=out[:, 3].copy(), z_opaque=out[:, 4].copy(),
                F=out[:, 5].copy(), tie=out[:, 6].copy(), sigma_last=out[:, 7].copy(),
                T_last=out[:, 8].copy(), step=out[:, 9].copy())


def pixel_set(W, H, B, seed, ctr):
    """B distinct pixels (u, v) of a W x H image drawn by Floyd's algorithm
    from SplitMix64 stream (seed, ctr)."""
    out = np.zeros((B, 2), dtype=np.int32)
    rc = lib().orc_pixel_set(W, H, B, seed, ctr, out.ctypes.data_as(C.POINTER(C.c_int32)))
    if rc != 0:
        raise ValueError(f"orc_pixel_set returned {rc}")
    return out


def splitmix64_stream(seed, n):
    st = C.c_uint64(seed)
    return [int(lib().orc_splitmix64_next(C.byref(st))) for _ in range(n)]


def cbrng(seed, ctr, idx):
    return int(lib().orc_cbrng(seed, ctr, idx))


def uniform(seed, ctr, idx):
    return float(lib().orc_uniform(seed, ctr, idx))


def normal(seed, ctr, m):
    return float(lib().orc_normal(seed, ctr, m))


def se3_exp(rho, omega):
    r, rp = _d(rho)
    w, wp = _d(omega)
    M = np.zeros(12)
    lib().orc_se3_exp(rp, wp, M.ctypes.data_as(C.POINTER(C.c_double)))
    return M.reshape(3, 4)


def predict(poses, noise, odom=None):
    """x_t = x_{t-1} O_t Exp(delta) (odom: 3x4 O_t, default identity)."""
    P, pp = _d(np.reshape(poses, (-1, 12)))
    q, qp = _d(np.reshape(noise, (-1, 4)))
    out = np.zeros_like(P)
    if odom is None:
        lib().orc_predict(P.shape[0], pp, qp, out.ctypes.data_as(C.POINTER(C.c_double)))
    else:
        o, op_ = _d(np.reshape(odom, (12,)))
        lib().orc_predict_odom(P.shape[0], pp, op_, qp, out.ctypes.data_as(C.POINTER(C.c_double)))
    return out


def motion_noise(n, seed, ctr, sigma_t, sigma_yaw):
    out = np.zeros((n, 4))
    lib().orc_motion_noise(n, seed, ctr, sigma_t, sigma_yaw,
                           out.ctypes.data_as(C.POINTER(C.c_double)))
    return out


def position_spread(poses):
    P, pp = _d(np.reshape(poses, (-1, 12)))
    out = np.zeros(4)
    lib().orc_position_spread(P.shape[0], pp, out.ctypes.data_as(C.POINTER(C.c_double)))
    return dict(mean=out[:3].copy(), trace=float(out[3]))


def loop_statistics(poses, w, mask):
    """Weighted mean position, circular weighted yaw, weighted position spread
    and survivor count of one weighted particle set (orc_loop_statistics)."""
    P, pp = _d(np.reshape(poses, (-1, 12)))
    wv, wp = _d(np.reshape(w, -1))
    mk = np.ascontiguousarray(np.reshape(mask, -1), dtype=np.uint8)
    assert wv.shape[0] == P.shape[0] == mk.shape[0]
    out = np.zeros(6)
    lib().orc_loop_statistics(P.shape[0], pp, wp, mk.ctypes.data_as(C.POINTER(C.c_uint8)),
                              out.ctypes.data_as(C.POINTER(C.c_double)))
    return dict(mean=out[:3].copy(), yaw=float(out[3]), spread=float(out[4]),
                n_survivors=int(out[5]))


def loop_schedule(stage, iter_at_stage, n_survivors, spread, refine, iter_cap, n_cap, n_min,
                  stride):
    """Next (stage, iter_at_stage, N) of the coarse-to-fine schedule
    (orc_loop_schedule)."""
    st = np.array([stage, iter_at_stage, 0], dtype=np.int32)
    ns = len(refine)
    rf = np.ascontiguousarray(refine, dtype=np.float64)
    ic = np.ascontiguousarray(iter_cap, dtype=np.int32)
    nc = np.ascontiguousarray(n_cap, dtype=np.int32)
    assert len(ic) == len(nc) == ns
    ip = C.POINTER(C.c_int)
    lib().orc_loop_schedule(st.ctypes.data_as(ip), ns, rf.ctypes.data_as(C.POINTER(C.c_double)),
                            ic.ctypes.data_as(ip), nc.ctypes.data_as(ip), int(n_min), int(stride),
                            float(spread), int(n_survivors))
    return int(st[0]), int(st[1]), int(st[2])


def level_intrinsics(K4, factor):
    """R K of Alg. 1 for R = 1/factor: focal and principal point divided."""
    fx, fy, cx, cy = K4
    return (fx / factor, fy / factor, cx / factor, cy / factor)


def render_observation_pixels(blob, gt_pose, K4, factor, pixels, opts: Opts,
                              arch=DEFAULT_ARCH):
    """Oracle renders of the level-image pixels [B,2] at the ground-truth pose
    (used to build observed images whose sampled pixels match the map)."""
    fx, fy, cx, cy = level_intrinsics(K4, factor)
    os_, ds = [], []
    for u, v in np.asarray(pixels).reshape(-1, 2):
        o, d = ray(gt_pose, fx, fy, cx, cy, u, v)
        os_.append(o)
        ds.append(d)
    return render_rays(blob, np.array(os_), np.array(ds), opts, arch=arch)["rgb"]


def paint_pixels(image, pixels, factor, colours):
    """Set the factor x factor full-resolution block of every level pixel to
    its colour, so that the box-filtered level image holds exactly that colour
    there."""
    img = np.array(image, dtype=np.float64, copy=True)
    for (u, v), c in zip(np.asarray(pixels).reshape(-1, 2), np.asarray(colours).reshape(-1, 3)):
        img[v * factor:(v + 1) * factor, u * factor:(u + 1) * factor, :] = c
    return img
