"""Python binding of the GB300 MCL particle-weight-update library.

Thin argument marshalling over the C ABI of ``include/mcl.h``: every stage of
the update runs in the library's CUDA kernels.  Tensors are torch CUDA
tensors (device memory and the current stream come from PyTorch).  If the
shared library has not been built, every call raises ``RuntimeError``;
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmcl.so")

MCL_OK = 0
MCL_ERR_ARG = -1
MCL_ERR_CUDA = -2
MCL_ERR_NONFINITE = -3
MCL_ERR_TIMEOUT = -4
MCL_ERR_UNSUPPORTED = -5
MCL_ERR_DEGENERATE = -6

PREC_FP32, PREC_BF16, PREC_FP8 = 0, 1, 2
PHASES = ("raygen", "mlp_coarse", "sample", "mlp_fine", "composite", "weights", "resample")
N_PHASES = len(PHASES)
_PREC = {"fp32": PREC_FP32, "bf16": PREC_BF16, "fp8": PREC_FP8}


class MclError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"mcl error {code}: {msg}")
        self.code = code


class Arch(C.Structure):
    _fields_ = [("n_freq_xyz", C.c_int), ("n_freq_dir", C.c_int), ("trunk_depth", C.c_int),
                ("trunk_width", C.c_int), ("skip_layer", C.c_int), ("rgb_width", C.c_int)]


class MapConfig(C.Structure):
    _fields_ = [("max_rays", C.c_int), ("max_samples", C.c_int), ("max_particles", C.c_int),
                ("max_queries", C.c_int)]


MAX_STAGES = 3


class Schedule(C.Structure):
    _fields_ = [("n_stages", C.c_int), ("level", C.c_int * MAX_STAGES),
                ("n_pixels", C.c_int * MAX_STAGES), ("n_cap", C.c_int * MAX_STAGES),
                ("n_min", C.c_int), ("stage_iter_cap", C.c_int * MAX_STAGES),
                ("refine", C.c_double * MAX_STAGES), ("iterations", C.c_int),
                ("sigma_t", C.c_float), ("sigma_yaw", C.c_float)]


class IterRecord(C.Structure):
    _fields_ = [("stage", C.c_int), ("level", C.c_int), ("n_particles", C.c_int),
                ("n_pixels", C.c_int), ("n_survivors", C.c_int), ("status", C.c_int),
                ("spread", C.c_double), ("est", C.c_double * 4), ("t_start_ns", C.c_uint64)]


def schedule(levels, pixels, caps, n_min=64, iter_caps=None, refine=None, iterations=20,
             sigma_t=0.05, sigma_yaw=0.05) -> Schedule:
    n = len(levels)
    pad = lambda v, fill: list(v) + [fill] * (MAX_STAGES - len(v))
    iter_caps = iter_caps or [iterations] * n
    refine = refine or [0.0] * n
    return Schedule(n, (C.c_int * MAX_STAGES)(*pad(levels, 0)),
                    (C.c_int * MAX_STAGES)(*pad(pixels, 1)), (C.c_int * MAX_STAGES)(*pad(caps, 1)),
                    n_min, (C.c_int * MAX_STAGES)(*pad(iter_caps, 1)),
                    (C.c_double * MAX_STAGES)(*pad(refine, 0.0)), iterations, sigma_t, sigma_yaw)


class Intrinsics(C.Structure):
    _fields_ = [("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("width", C.c_int), ("height", C.c_int)]


class Opts(C.Structure):
    _fields_ = [("n_coarse", C.c_int), ("n_fine", C.c_int), ("precision", C.c_int),
                ("use_rejection", C.c_int), ("jitter", C.c_int),
                ("near_z", C.c_float), ("far_z", C.c_float), ("alpha", C.c_float),
                ("tau", C.c_float), ("rho_reject", C.c_double), ("s_min", C.c_double),
                ("seed", C.c_uint64), ("counter", C.c_uint64),
                ("use_proposal", C.c_int), ("n_proposal", C.c_int), ("n_guided", C.c_int)]


class TrainCfg(C.Structure):
    _fields_ = [("epochs", C.c_int), ("batch_rays", C.c_int), ("n_bins", C.c_int),
                ("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float),
                ("eps", C.c_float), ("seed", C.c_uint64), ("lr_end", C.c_float)]


class FitCfg(C.Structure):
    _fields_ = [("steps", C.c_int), ("batch", C.c_int), ("lr", C.c_float), ("beta1", C.c_float),
                ("beta2", C.c_float), ("eps", C.c_float), ("lr_end", C.c_float),
                ("sigma_weight", C.c_float), ("seed", C.c_uint64)]


class Debug(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("rgb", "E", "F", "z_trans", "z_opaque", "S")]


_lock = threading.Lock()
_lib = None


def lib():
    """The loaded shared library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"CUDA library {LIB_PATH} is not built; run "
                    "paper_2406_12202_gb300.build.build() (or __graft_entry__.build()) first")
            L = C.CDLL(LIB_PATH)
            vp, i32, f32, f64, u64 = C.c_void_p, C.c_int, C.c_float, C.c_double, C.c_uint64
            L.mcl_init_map.argtypes = [vp, C.c_size_t, C.POINTER(Arch), C.POINTER(MapConfig),
                                       C.POINTER(vp)]
            L.mcl_destroy_map.argtypes = [vp]
            L.mcl_destroy_map.restype = None
            L.mcl_update.argtypes = [vp, vp, i32, vp, C.POINTER(Intrinsics), i32, vp, i32,
                                     C.POINTER(Opts), vp, vp, vp, C.POINTER(Debug), vp]
            L.mcl_render.argtypes = [vp, vp, i32, C.POINTER(Intrinsics), i32, vp, i32,
                                     C.POINTER(Opts), vp, vp, vp]
            L.mcl_resample.argtypes = [vp, vp, i32, i32, f64, vp, vp]
            L.mcl_predict.argtypes = [vp, i32, vp, i32, f32, f32, u64, u64, vp, vp]
            L.mcl_predict_odom.argtypes = [vp, i32, vp, i32, vp, f32, f32, u64, u64, vp, vp]
            L.mcl_downscale.argtypes = [vp, i32, i32, i32, vp, vp]
            L.mcl_position_spread.argtypes = [vp, i32, vp, vp]
            L.mcl_read_status.argtypes = [vp, C.POINTER(C.c_int), vp]
            L.mcl_map_supports.argtypes = [vp, i32]
            L.mcl_draw_pixels.argtypes = [i32, i32, i32, u64, u64, vp, vp]
            L.mcl_localize.argtypes = [vp, i32, vp, i32, C.POINTER(C.c_int), C.POINTER(vp),
                                       C.POINTER(Intrinsics), C.POINTER(Schedule), C.POINTER(Opts),
                                       vp, vp, i32, vp]
            L.mcl_query.argtypes = [vp, vp, vp, i32, i32, vp, vp]
            L.mcl_resample_noalloc.argtypes = [vp, i32, i32, f64, vp, vp]
            L.mcl_profile_enable.argtypes = [vp, i32]
            L.mcl_profile_read.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_longlong), i32]
            L.mcl_proposal_set.argtypes = [vp, vp, C.c_size_t]
            L.mcl_proposal_get.argtypes = [vp, vp, C.c_size_t]
            L.mcl_render_histogram.argtypes = [vp, vp, i32, C.POINTER(Intrinsics), i32, vp, i32,
                                               C.POINTER(Opts), i32, vp, vp]
            L.mcl_proposal_loss_grad.argtypes = [vp, vp, vp, i32, i32, f32, f32, vp, vp, vp, vp]
            L.mcl_proposal_train.argtypes = [vp, vp, i32, vp, i32, C.POINTER(Intrinsics), i32,
                                             C.POINTER(Opts), C.POINTER(TrainCfg), vp, vp]
            L.mcl_proposal_query.argtypes = [vp, vp, i32, i32, vp, vp]
            L.mcl_autotune.argtypes = [vp, i32, C.c_longlong, C.POINTER(C.c_int),
                                       C.POINTER(C.c_float), vp]
            L.mcl_set_mlp_variant.argtypes = [vp, i32, i32]
            L.mcl_inject_weight_stall.argtypes = [vp, i32, f64]
            L.mcl_set_fused_epilogue.argtypes = [vp, i32]
            L.mcl_fit_map.argtypes = [vp, vp, vp, vp, i32, C.POINTER(FitCfg), vp, vp]
            L.mcl_map_loss_grad.argtypes = [vp, vp, vp, vp, i32, f32, vp, vp, vp]
            L.mcl_get_map_weights.argtypes = [vp, vp, C.c_size_t]
            L.mcl_probe_mma_rate.argtypes = [i32, i32, i32, C.POINTER(C.c_double),
                                             C.POINTER(C.c_double)]
            L.mcl_last_error.restype = C.c_char_p
            L.mcl_last_error.argtypes = []
            _lib = L
    return _lib


def _check(rc):
    if rc != MCL_OK:
        raise MclError(rc, lib().mcl_last_error().decode())


def probe_mma_rate(group: int = 4, gap: int = 0, n_groups: int = 4000):
    """(SM cycles per group of `group` back-to-back BF16 128x256x16 MMAs,
    cycles of the `gap`-long chain between groups) (mcl_probe_mma_rate)."""
    clk, gclk = C.c_double(0.0), C.c_double(0.0)
    _check(lib().mcl_probe_mma_rate(int(group), int(gap), int(n_groups), C.byref(clk), C.byref(gclk)))
    return clk.value, gclk.value


def synth_blob_size(arch) -> int:
    """Floats of a weight blob of architecture arch (the layer table of
    mcl_init_map)."""
    gx, gd = 3 + 6 * arch.n_freq_xyz, 3 + 6 * arch.n_freq_dir
    D, W, skip, Wr = arch.trunk_depth, arch.trunk_width, arch.skip_layer, arch.rgb_width
    n = 0
    for l in range(1, D + 1):
        fi = gx if l == 1 else (W + gx if l == skip + 1 else W)
        n += fi * W + W
    n += W + 1 + W * W + W + (W + gd) * Wr + Wr + Wr * 3 + 3
    return n


def _torch():
    import torch
    return torch


def _stream():
    return _torch().cuda.current_stream().cuda_stream


def _ptr(t, dtype, shape=None, name="tensor"):
    torch = _torch()
    if t is None:
        return None
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t.data_ptr()


@dataclass
class UpdateOptions:
    n_coarse: int = 64
    n_fine: int = 128
    precision: str = "fp32"
    use_rejection: bool = True
    jitter: bool = False
    near: float = 2.0
    far: float = 6.0
    alpha: float = 0.05
    tau: float = 0.1
    rho_reject: float = 1e-3
    s_min: float = 1e-30
    seed: int = 0
    counter: int = 0
    use_proposal: bool = False   # learned proposal sampler (Map.proposal_train)
    n_proposal: int = 64
    n_guided: int = 32

    def c(self) -> Opts:
        return Opts(self.n_coarse, self.n_fine, _PREC[self.precision], int(self.use_rejection),
                    int(self.jitter), self.near, self.far, self.alpha, self.tau,
                    self.rho_reject, self.s_min, self.seed, self.counter,
                    int(self.use_proposal), self.n_proposal, self.n_guided)


def intrinsics(fx, fy, cx, cy, width, height) -> Intrinsics:
    return Intrinsics(fx, fy, cx, cy, width, height)


class Map:
    """A NeRF map uploaded to the GPU with its workspace (mcl_init_map)."""

    def __init__(self, weights: np.ndarray, max_rays: int, max_samples: int = 192,
                 max_particles: int | None = None, max_queries: int = 1,
                 arch=(10, 4, 8, 256, 5, 128)):
        w = np.ascontiguousarray(weights, dtype=np.float32)
        self._arch = Arch(*arch)
        self.cfg = MapConfig(int(max_rays), int(max_samples),
                             int(max_particles if max_particles is not None else max_rays),
                             int(max_queries))
        h = C.c_void_p()
        _check(lib().mcl_init_map(w.ctypes.data, w.size, C.byref(self._arch), C.byref(self.cfg),
                                  C.byref(h)))
        self.handle = h

    def supports(self, precision: str) -> bool:
        return bool(lib().mcl_map_supports(self.handle, _PREC[precision]))

    def close(self):
        if getattr(self, "handle", None):
            lib().mcl_destroy_map(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- update
    def update(self, particles, image, K: Intrinsics, level: int, pixels,
               opts: UpdateOptions, out=None, debug: bool = False):
        """Eq. 6 weights of particles [N,12] against image [H,W,3] at level.
        Returns dict logw [N] f32, w [N] f64, mask [N] u8 (+ per-ray debug)."""
        torch = _torch()
        N = particles.shape[0]
        B = pixels.shape[0]
        dev = particles.device
        if out is None:
            out = dict(logw=torch.empty(N, dtype=torch.float32, device=dev),
                       w=torch.empty(N, dtype=torch.float64, device=dev),
                       mask=torch.empty(N, dtype=torch.uint8, device=dev))
        dbg = None
        if debug:
            nr = N * B
            out.update(rgb=torch.empty(nr, 3, dtype=torch.float32, device=dev),
                       E=torch.empty(nr, dtype=torch.float32, device=dev),
                       F=torch.empty(nr, dtype=torch.float32, device=dev),
                       z_trans=torch.empty(nr, dtype=torch.float32, device=dev),
                       z_opaque=torch.empty(nr, dtype=torch.float32, device=dev),
                       S=torch.empty(N, dtype=torch.float32, device=dev))
            dbg = Debug(*(out[k].data_ptr() for k in ("rgb", "E", "F", "z_trans", "z_opaque", "S")))
        o = opts.c()
        _check(lib().mcl_update(
            self.handle, _ptr(particles, torch.float32, (N, 12), "particles"), N,
            _ptr(image, torch.float32, (K.height, K.width, 3), "image"), C.byref(K), int(level),
            _ptr(pixels, torch.int32, (B, 2), "pixels"), B, C.byref(o),
            _ptr(out["logw"], torch.float32, (N,), "logw"),
            _ptr(out["w"], torch.float64, (N,), "w"),
            _ptr(out["mask"], torch.uint8, (N,), "mask"),
            C.byref(dbg) if dbg is not None else None, _stream()))
        return out

    def query(self, x, dirs, precision: str = "fp32"):
        """(sigma_raw, r, g, b) [n,4] of the map at points x [n,3] seen from
        directions dirs [n,3]."""
        torch = _torch()
        n = x.shape[0]
        out = torch.empty(n, 4, dtype=torch.float32, device=x.device)
        _check(lib().mcl_query(self.handle, _ptr(x, torch.float32, (n, 3), "x"),
                               _ptr(dirs, torch.float32, (n, 3), "dirs"), n, _PREC[precision],
                               out.data_ptr(), _stream()))
        return out

    def render(self, poses, K: Intrinsics, level: int, pixels, opts: UpdateOptions,
               with_F: bool = False):
        """Rendered colours [n*B, 3] (and F [n*B]) of poses x pixels."""
        torch = _torch()
        n, B = poses.shape[0], pixels.shape[0]
        rgb = torch.empty(n * B, 3, dtype=torch.float32, device=poses.device)
        F = torch.empty(n * B, dtype=torch.float32, device=poses.device) if with_F else None
        o = opts.c()
        _check(lib().mcl_render(self.handle, _ptr(poses, torch.float32, (n, 12), "poses"), n,
                                C.byref(K), int(level), _ptr(pixels, torch.int32, (B, 2), "pixels"),
                                B, C.byref(o), rgb.data_ptr(),
                                F.data_ptr() if F is not None else None, _stream()))
        return (rgb, F) if with_F else rgb

    def resample(self, w, n_out: int, u0: float, idx=None):
        torch = _torch()
        n_in = w.shape[0]
        if idx is None:
            idx = torch.empty(n_out, dtype=torch.int32, device=w.device)
        _check(lib().mcl_resample(self.handle, _ptr(w, torch.float64, (n_in,), "w"), n_in,
                                  int(n_out), float(u0), _ptr(idx, torch.int32, (n_out,), "idx"),
                                  _stream()))
        return idx

    def profile(self, enable: bool = True):
        _check(lib().mcl_profile_enable(self.handle, int(enable)))

    def profile_read(self, reset: bool = True):
        """Accumulated GPU ms per phase (dict) and the library's launch count."""
        ms = (C.c_double * N_PHASES)()
        n = C.c_longlong(0)
        _check(lib().mcl_profile_read(self.handle, ms, C.byref(n), int(reset)))
        return dict(zip(PHASES, list(ms))), n.value

    def localize(self, particles, n0, images, K: Intrinsics, sch: Schedule, opts: UpdateOptions,
                 use_graph: bool = True, log=None, final_n=None):
        """Run MCL on the device for len(images) queries (mcl_localize).
        particles: [Q, stride, 12] f32 CUDA tensor (in / out); n0: initial
        counts; images: list of [H,W,3] f32 CUDA tensors.  Returns (log
        ndarray of IterRecord fields [Q, iterations], final counts)."""
        torch = _torch()
        Q, stride, _ = particles.shape
        if log is None:
            log = torch.empty(Q * sch.iterations * C.sizeof(IterRecord), dtype=torch.uint8,
                              device=particles.device)
        if final_n is None:
            final_n = torch.empty(Q, dtype=torch.int32, device=particles.device)
        n0a = (C.c_int * Q)(*[int(v) for v in n0])
        imgs = (C.c_void_p * Q)(*[_ptr(im, torch.float32, (K.height, K.width, 3), "image")
                                  for im in images])
        o = opts.c()
        _check(lib().mcl_localize(self.handle, Q, _ptr(particles, torch.float32, None, "particles"),
                                  stride, n0a, imgs, C.byref(K), C.byref(sch), C.byref(o),
                                  log.data_ptr(), final_n.data_ptr(), int(use_graph), _stream()))
        self._last_log = log
        return log, final_n

    @staticmethod
    def decode_log(log, Q, iterations):
        raw = log.cpu().numpy().tobytes()
        recs = (IterRecord * (Q * iterations)).from_buffer_copy(raw)
        out = []
        for q in range(Q):
            rows = []
            for t in range(iterations):
                r = recs[q * iterations + t]
                rows.append(dict(stage=r.stage, level=r.level, n_particles=r.n_particles,
                                 n_pixels=r.n_pixels, n_survivors=r.n_survivors, status=r.status,
                                 spread=r.spread, est=list(r.est), t_start_ns=r.t_start_ns))
            out.append(rows)
        return out

    # -------------------------------------------------------------- proposal
    def proposal_set(self, weights: np.ndarray):
        w = np.ascontiguousarray(weights, dtype=np.float32)
        _check(lib().mcl_proposal_set(self.handle, w.ctypes.data, w.size))

    def proposal_get(self) -> np.ndarray:
        w = np.zeros(PROPOSAL_N_WEIGHTS, dtype=np.float32)
        _check(lib().mcl_proposal_get(self.handle, w.ctypes.data, w.size))
        return w

    def proposal_query(self, x, precision: str = "fp32"):
        """Raw proposal density at points x [n,3] (mcl_proposal_query)."""
        torch = _torch()
        n = x.shape[0]
        out = torch.empty(n, dtype=torch.float32, device=x.device)
        _check(lib().mcl_proposal_query(self.handle, _ptr(x, torch.float32, (n, 3), "x"), n,
                                        _PREC[precision], out.data_ptr(), _stream()))
        return out

    def render_histogram(self, poses, K: Intrinsics, level: int, pixels, opts: UpdateOptions,
                         n_bins: int):
        """Distillation targets [n*B, n_bins] (mcl_render_histogram)."""
        torch = _torch()
        n, B = poses.shape[0], pixels.shape[0]
        out = torch.empty(n * B, n_bins, dtype=torch.float32, device=poses.device)
        o = opts.c()
        _check(lib().mcl_render_histogram(
            self.handle, _ptr(poses, torch.float32, (n, 12), "poses"), n, C.byref(K), int(level),
            _ptr(pixels, torch.int32, (B, 2), "pixels"), B, C.byref(o), int(n_bins),
            out.data_ptr(), _stream()))
        return out

    def proposal_loss_grad(self, o, d, hist, near: float = 2.0, far: float = 6.0):
        """Mean cross-entropy of the proposal against hist and its gradient
        (mcl_proposal_loss_grad): (loss float, grad [PROPOSAL_N_WEIGHTS] f32)."""
        torch = _torch()
        n, nb = hist.shape
        loss = torch.empty(1, dtype=torch.float64, device=hist.device)
        grad = torch.empty(PROPOSAL_N_WEIGHTS, dtype=torch.float32, device=hist.device)
        _check(lib().mcl_proposal_loss_grad(
            self.handle, _ptr(o, torch.float32, (n, 3), "o"), _ptr(d, torch.float32, (n, 3), "d"),
            n, nb, float(near), float(far), _ptr(hist, torch.float32, (n, nb), "hist"),
            loss.data_ptr(), grad.data_ptr(), _stream()))
        return float(loss.item()), grad

    def proposal_train(self, poses, pixels, K: Intrinsics, level: int, opts: UpdateOptions,
                       epochs: int = 10, batch_rays: int = 4096, n_bins: int = 64,
                       lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999,
                       eps: float = 1e-7, seed: int = 0, lr_end: float = 0.0):
        """Distil the proposal from the full sampler of opts
        (mcl_proposal_train); the rate decays geometrically from lr to
        lr_end (constant if lr_end <= 0).  Returns the mean loss of every
        epoch."""
        torch = _torch()
        n, B = poses.shape[0], pixels.shape[0]
        log = torch.zeros(epochs, dtype=torch.float32, device=poses.device)
        cfg = TrainCfg(int(epochs), int(batch_rays), int(n_bins), lr, beta1, beta2, eps, int(seed),
                       lr_end)
        o = opts.c()
        _check(lib().mcl_proposal_train(
            self.handle, _ptr(poses, torch.float32, (n, 12), "poses"), n,
            _ptr(pixels, torch.int32, (B, 2), "pixels"), B, C.byref(K), int(level), C.byref(o),
            C.byref(cfg), log.data_ptr(), _stream()))
        return log.cpu().numpy()

    def autotune(self, precision: str, rows: int):
        """Time the MLP kernel variants of `precision` on `rows` synthetic
        samples and keep the fastest (mcl_autotune).  Returns (chosen index,
        {index: ms})."""
        ch = C.c_int(-1)
        ms = (C.c_float * MLP_VARIANTS)()
        _check(lib().mcl_autotune(self.handle, _PREC[precision], int(rows), C.byref(ch), ms,
                                  _stream()))
        return ch.value, {i: float(ms[i]) for i in range(MLP_VARIANTS) if ms[i] >= 0}

    # ------------------------------------------------------------ map fitting
    def fit(self, x, dirs, target, steps=2000, batch=16384, lr=1e-3, lr_end=1e-4, beta1=0.9,
            beta2=0.999, eps=1e-8, sigma_weight=1e-2, seed=0):
        """Fit the map's weights to field samples (mcl_fit_map): points x
        [n,3], view directions dirs [n,3], targets [n,4] (density, r, g, b),
        CUDA f32 tensors.  Returns the per-step batch losses [steps]."""
        torch = _torch()
        n = x.shape[0]
        log = torch.empty(steps, dtype=torch.float32, device=x.device)
        cfg = FitCfg(int(steps), int(batch), lr, beta1, beta2, eps, lr_end, sigma_weight, int(seed))
        _check(lib().mcl_fit_map(self.handle, _ptr(x, torch.float32, (n, 3), "x"),
                                 _ptr(dirs, torch.float32, (n, 3), "dirs"),
                                 _ptr(target, torch.float32, (n, 4), "target"), n, C.byref(cfg),
                                 log.data_ptr(), _stream()))
        return log

    def loss_grad(self, x, dirs, target, sigma_weight=1e-2):
        """Fitting loss (mean) and its gradient in the blob layout
        (mcl_map_loss_grad)."""
        torch = _torch()
        n = x.shape[0]
        loss = torch.empty(1, dtype=torch.float64, device=x.device)
        grad = torch.empty(synth_blob_size(self._arch), dtype=torch.float32, device=x.device)
        _check(lib().mcl_map_loss_grad(self.handle, _ptr(x, torch.float32, (n, 3), "x"),
                                       _ptr(dirs, torch.float32, (n, 3), "dirs"),
                                       _ptr(target, torch.float32, (n, 4), "target"), n,
                                       float(sigma_weight), loss.data_ptr(), grad.data_ptr(),
                                       _stream()))
        return float(loss.item()), grad

    def weights(self) -> np.ndarray:
        """The map's FP32 weights in the blob layout (mcl_get_map_weights)."""
        w = np.zeros(synth_blob_size(self._arch), dtype=np.float32)
        _check(lib().mcl_get_map_weights(self.handle, w.ctypes.data, w.size))
        return w

    def set_fused_epilogue(self, enable: bool):
        """Fused ray epilogues of the tensor-core forms on / off
        (mcl_set_fused_epilogue; off by default: the separate kernels are
        faster on GB300)."""
        _check(lib().mcl_set_fused_epilogue(self.handle, int(bool(enable))))

    def set_mlp_variant(self, precision: str, variant: int):
        _check(lib().mcl_set_mlp_variant(self.handle, _PREC[precision], int(variant)))

    def inject_weight_stall(self, n_launches: int, wait_ms: float):
        """Failure-detection test hook (mcl_inject_weight_stall): the next
        n_launches tensor-core MLP launches hold their weight stream, so their
        bounded waits run out after wait_ms and the status word records
        MCL_ERR_TIMEOUT."""
        _check(lib().mcl_inject_weight_stall(self.handle, int(n_launches), float(wait_ms)))

    def read_status(self):
        n = C.c_int(0)
        rc = lib().mcl_read_status(self.handle, C.byref(n), _stream())
        return rc, n.value


RESAMPLE_NOALLOC_MAX_IN = 65536


def resample_noalloc(w, n_out: int, u0: float, idx=None):
    """Systematic resampling without a map and without any device allocation
    in the library (mcl_resample_noalloc).  Same indices as Map.resample for
    the same weights and u0.  The call runs on w's device (made current for
    the call, on that device's current stream); idx must live there too.
    Calls that overlap on the GPU race on the library's fixed scratch, so
    issue them from one stream."""
    torch = _torch()
    if not (isinstance(w, torch.Tensor) and w.is_cuda):
        raise TypeError("w must be a CUDA tensor")
    n_in = w.shape[0]
    with torch.cuda.device(w.device):
        if idx is None:
            idx = torch.empty(n_out, dtype=torch.int32, device=w.device)
        elif not (isinstance(idx, torch.Tensor) and idx.device == w.device):
            raise ValueError(f"idx must be on {w.device}")
        _check(lib().mcl_resample_noalloc(_ptr(w, torch.float64, (n_in,), "w"), n_in, int(n_out),
                                          float(u0), _ptr(idx, torch.int32, (n_out,), "idx"),
                                          _stream()))
    return idx


def draw_pixels(W: int, H: int, B: int, seed: int, counter: int, out=None):
    torch = _torch()
    if out is None:
        out = torch.empty(B, 2, dtype=torch.int32, device="cuda")
    _check(lib().mcl_draw_pixels(W, H, B, int(seed), int(counter),
                                 _ptr(out, torch.int32, (B, 2), "out"), _stream()))
    return out


def predict(poses, idx, n_out: int, sigma_t: float, sigma_yaw: float, seed: int, counter: int,
            out=None, odom=None):
    """x_t = x_{t-1} (O_t) Exp(delta) (mcl_predict / mcl_predict_odom; odom:
    a [12] f32 CUDA tensor, the 3x4 relative motion, or None)."""
    torch = _torch()
    if out is None:
        out = torch.empty(n_out, 12, dtype=torch.float32, device=poses.device)
    args = (_ptr(poses, torch.float32, (poses.shape[0], 12), "poses"), poses.shape[0],
            _ptr(idx, torch.int32, (n_out,), "idx") if idx is not None else None, int(n_out))
    tail = (float(sigma_t), float(sigma_yaw), int(seed), int(counter),
            _ptr(out, torch.float32, (n_out, 12), "out"), _stream())
    if odom is None:
        _check(lib().mcl_predict(*args, *tail))
    else:
        _check(lib().mcl_predict_odom(*args, _ptr(odom, torch.float32, (12,), "odom"), *tail))
    return out


def downscale(image, factor: int, out=None):
    torch = _torch()
    H, W, _ = image.shape
    if out is None:
        out = torch.empty(H // factor, W // factor, 3, dtype=torch.float32, device=image.device)
    _check(lib().mcl_downscale(_ptr(image, torch.float32, (H, W, 3), "image"), W, H, int(factor),
                               _ptr(out, torch.float32, (H // factor, W // factor, 3), "out"),
                               _stream()))
    return out


def position_spread(poses, out=None):
    torch = _torch()
    if out is None:
        out = torch.empty(4, dtype=torch.float64, device=poses.device)
    _check(lib().mcl_position_spread(_ptr(poses, torch.float32, None, "poses"), poses.shape[0],
                                     _ptr(out, torch.float64, (4,), "out"), _stream()))
    return out


EXPORTED = ("mcl_init_map", "mcl_destroy_map", "mcl_update", "mcl_render", "mcl_resample",
            "mcl_predict", "mcl_downscale", "mcl_position_spread", "mcl_read_status",
            "mcl_profile_enable", "mcl_profile_read", "mcl_map_supports", "mcl_last_error",
            "mcl_resample_noalloc", "mcl_query", "mcl_draw_pixels", "mcl_localize",
            "mcl_proposal_set", "mcl_proposal_get", "mcl_render_histogram",
            "mcl_proposal_loss_grad", "mcl_proposal_train", "mcl_proposal_query", "mcl_autotune",
            "mcl_predict_odom",
            "mcl_set_mlp_variant", "mcl_inject_weight_stall", "mcl_set_fused_epilogue",
            "mcl_fit_map", "mcl_map_loss_grad", "mcl_get_map_weights", "mcl_probe_mma_rate")

# Kernel variants of the tensor-core MLP (include/mcl.h, MCL_MLP_VARIANTS):
# (precision, epilogue warps per tile, staggered tiles)
MLP_VARIANTS = 14
# index: (precision, epilogue warps per tile, schedule)
MLP_VARIANT_TABLE = {0: ("bf16", 4, "lockstep"), 1: ("bf16", 8, "lockstep"),
                     2: ("fp8", 4, "lockstep"), 3: ("fp8", 8, "lockstep"),
                     4: ("fp8", 4, "staggered"), 5: ("fp8", 8, "staggered"),
                     6: ("bf16", 4, "split"), 7: ("bf16", 4, "pipelined"),
                     8: ("bf16", 4, "lockstep pair"), 9: ("fp8", 4, "lockstep pair"),
                     10: ("fp8", 4, "staggered pair"), 11: ("bf16", 4, "staggered"),
                     12: ("bf16", 8, "staggered"), 13: ("bf16", 4, "staggered pair")}

# Weights of the learned proposal (gamma(x) with 6 frequencies -> 4 x 64 ReLU
# -> density): 64*39+64 + 3*(64*64+64) + 64+1.
PROPOSAL_N_WEIGHTS = 15105

# Algorithmic multiply-accumulates per sample of the network the tensor-core
# form evaluates (the linear feature layer folded into the RGB hidden layer):
# trunk 63*256 + 4*256^2 + 319*256 + 2*256^2, RGB hidden 256*128, density
# head 256, RGB output 128*3 (the per-ray gamma(d) term is per ray, not per
# sample).  Padding (63 -> 64, 319 -> 320, N 129 -> 144) is not counted.
TC_MAC_PER_SAMPLE = 63 * 256 + 4 * 256 * 256 + 319 * 256 + 2 * 256 * 256 + 256 * 128 + 256 + 384
