"""ctypes binding of libcbp (include/cbp.h), names as in the C ABI.

Argument marshalling only: tensors become ``cbp_frames`` descriptors and raw
pointers, every step of the method runs in the CUDA library.  PyTorch supplies
device memory and streams.  If ``libcbp.so`` is missing, loading raises.
With CBP_LIBRARY=checks in the environment the bounds-checked build
``libcbp_checks.so`` is loaded instead (see cbp_check_words).
"""
from __future__ import annotations

import ctypes
from ctypes import POINTER, byref, c_double, c_int, c_int32, c_int64, c_uint32, c_uint64, c_void_p
import os
from pathlib import Path

import torch

LIB_PATH = Path(__file__).resolve().parent / (
    "libcbp_checks.so" if os.environ.get("CBP_LIBRARY") == "checks" else "libcbp.so")

CBP_OK, CBP_WARN_ILL_CONDITIONED = 0, 1
CBP_ERR_INVALID_ARG, CBP_ERR_SIZE_MISMATCH, CBP_ERR_NOT_COPRIME = -1, -2, -3
CBP_ERR_OOM, CBP_ERR_CUDA, CBP_ERR_BUSY, CBP_ERR_TIMEOUT = -4, -5, -6, -7
CBP_ERR_BUDGET, CBP_ERR_UNSUPPORTED = -8, -9
CBP_F32, CBP_F64 = 0, 1
CBP_PATH_FP64, CBP_PATH_MIXED, CBP_PATH_LEARNED = 0, 1, 2
CBP_FLAG_HOST_IO, CBP_FLAG_KERNELS_IN, CBP_FLAG_SINGLE_KERNEL, CBP_FLAG_KERNELS_F64 = 1, 2, 4, 8
CBP_FLAG_K1_ONLY, CBP_FLAG_SCALE_SUPPORT = 16, 32
CBP_FLAG_OVERLAP_CALLS = 64
PATHS = {"fp64": CBP_PATH_FP64, "mixed": CBP_PATH_MIXED, "learned": CBP_PATH_LEARNED}

# Every symbol include/cbp.h declares (checked by the CPU tests).
EXPORTED = [
    "cbp_create", "cbp_destroy", "cbp_status_string", "cbp_workspace_size",
    "cbp_estimate_kernels", "cbp_deblur_pair", "cbp_forward_blur", "cbp_synth_latent",
    "cbp_stream_submit", "cbp_stream_poll", "cbp_stream_stats", "cbp_profile", "cbp_stage_times",
    "cbp_estimate_kernels_stages", "cbp_estimate_kernels_noalloc", "cbp_cnn_param_count",
    "cbp_cnn_forward", "cbp_cnn_train_step", "cbp_learned_load", "cbp_estimate_size",
    "cbp_truncate_lsb", "cbp_encrypt", "cbp_check_recip", "cbp_check_words",
    "cbp_check_expire_waits",
]
STAGES = ["eval", "sample_solve", "scale_solve", "kernel_spectra", "row_fft", "col_deconv",
          "row_ifft", "h2d", "d2h", "proposal", "gate"]


class cbp_encrypt_params(ctypes.Structure):
    _fields_ = [("t1", c_int32), ("t2", c_int32), ("t3", c_int32), ("t4", c_int32), ("m", c_int32),
                ("max_attempts", c_int32), ("tol", c_double), ("sigma", c_double), ("seed", c_uint64),
                ("frame0", c_int32), ("reserved", c_int32)]


class cbp_size_params(ctypes.Structure):
    _fields_ = [("t_min", c_int32), ("t_max", c_int32), ("tol", c_double)]


class cbp_frames(ctypes.Structure):
    _fields_ = [("data", c_void_p), ("n", c_int32), ("c", c_int32), ("h", c_int32),
                ("w", c_int32), ("dtype", c_int), ("row_stride", c_int64),
                ("chan_stride", c_int64), ("frame_stride", c_int64)]


class cbp_params(ctypes.Structure):
    _fields_ = [("t1", c_int32), ("t2", c_int32), ("m", c_int32), ("path", c_int),
                ("eps", c_double), ("pad_h", c_int32), ("pad_w", c_int32),
                ("accept_rho", c_double), ("flags", c_uint32), ("reserved", c_int32)]


class cbp_stage_out(ctypes.Structure):
    _fields_ = [("p_z2", c_void_p * 2), ("p_z1", c_void_p * 2), ("x_z2", c_void_p), ("x_z1", c_void_p),
                ("sample_diag", c_void_p), ("lifted", c_void_p), ("kernels", c_void_p)]


class cbp_cnn_trace(ctypes.Structure):
    _fields_ = [("input", c_void_p), ("act", c_void_p * 3), ("logits", c_void_p), ("grad", c_void_p)]


class cbp_adamw(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("weight_decay", ctypes.c_float), ("step", c_int32)]


class cbp_diag(ctypes.Structure):
    _fields_ = [("kappa_max", c_double), ("gap_min", c_double), ("sigma_min_max", c_double),
                ("scale_resid", c_double), ("imag_ratio", c_double), ("support_ratio", c_double),
                ("rho", c_double), ("flagged_samples", c_int32), ("used_fallback", c_int32),
                ("pad_h", c_int32), ("pad_w", c_int32), ("status", c_int32),
                ("hard_samples", c_int32), ("gpu_start_ms", c_double), ("gpu_end_ms", c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib() -> ctypes.CDLL:
    """Load libcbp.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not LIB_PATH.exists():
            raise RuntimeError(f"{LIB_PATH.name} not built at {LIB_PATH}; run __graft_entry__.build()")
        L = ctypes.CDLL(str(LIB_PATH))
        fr, pr, dg = POINTER(cbp_frames), POINTER(cbp_params), POINTER(cbp_diag)
        sig = {
            "cbp_create": ([POINTER(c_void_p), c_int, ctypes.c_size_t], c_int),
            "cbp_destroy": ([c_void_p], c_int),
            "cbp_status_string": ([c_int], ctypes.c_char_p),
            "cbp_workspace_size": ([fr, fr, pr, POINTER(ctypes.c_size_t)], c_int),
            "cbp_estimate_kernels": ([c_void_p, fr, fr, pr, c_void_p, c_void_p, dg, c_void_p], c_int),
            "cbp_deblur_pair": ([c_void_p, fr, fr, pr, c_void_p, c_void_p, c_void_p, dg, c_void_p], c_int),
            "cbp_forward_blur": ([c_void_p, c_void_p, c_int32, c_int32, c_int32, c_int32, c_int,
                                  c_void_p, c_int32, c_double, c_uint64, c_void_p, c_void_p], c_int),
            "cbp_synth_latent": ([c_void_p, c_void_p, c_int32, c_int32, c_int32, c_int32, c_int32,
                                  c_int, c_double, c_uint64, c_void_p, c_void_p], c_int),
            "cbp_stream_submit": ([c_void_p, fr, fr, pr, c_void_p, c_void_p, c_void_p,
                                   POINTER(c_uint64)], c_int),
            "cbp_stream_poll": ([c_void_p, c_uint64, c_int32, dg], c_int),
            "cbp_stream_stats": ([c_void_p, POINTER(c_uint64), POINTER(c_double), POINTER(c_double),
                                  c_int32], c_int),
            "cbp_profile": ([c_void_p, c_int32], c_int),
            "cbp_estimate_kernels_noalloc": ([fr, fr, pr, c_void_p, c_void_p, dg, c_void_p], c_int),
            "cbp_estimate_kernels_stages": ([c_void_p, fr, fr, pr, c_void_p, c_void_p, dg,
                                             POINTER(cbp_stage_out), c_void_p], c_int),
            "cbp_stage_times": ([c_void_p, POINTER(c_double), POINTER(c_int64)], c_int),
            "cbp_cnn_param_count": ([], ctypes.c_size_t),
            "cbp_cnn_forward": ([c_void_p, fr, fr, c_void_p, c_void_p, POINTER(cbp_cnn_trace), c_void_p],
                                c_int),
            "cbp_cnn_train_step": ([c_void_p, fr, fr, c_void_p, c_void_p, c_void_p, c_void_p,
                                    POINTER(cbp_adamw), c_void_p, POINTER(cbp_cnn_trace), c_void_p], c_int),
            "cbp_learned_load": ([c_void_p, ctypes.c_char_p], c_int),
            "cbp_truncate_lsb": ([c_void_p, c_void_p, c_int, c_int64, c_int32, c_int32, c_void_p,
                                  c_void_p], c_int),
            "cbp_check_recip": ([c_void_p, c_int64, c_void_p, c_void_p, c_void_p], c_int),
            "cbp_check_words": ([POINTER(c_uint32), c_int32, c_int32], c_int),
            "cbp_check_expire_waits": ([c_int32], c_int),
            "cbp_encrypt": ([c_void_p, c_void_p, c_int32, c_int32, c_int32, c_int32, c_int,
                             POINTER(cbp_encrypt_params), c_void_p, c_void_p, c_void_p, c_void_p,
                             c_void_p, c_void_p, c_void_p, c_void_p, POINTER(c_int32), c_void_p], c_int),
            "cbp_estimate_size": ([c_void_p, fr, fr, POINTER(cbp_size_params), POINTER(c_int32),
                                   POINTER(c_int32), POINTER(c_int32), POINTER(c_double),
                                   POINTER(c_int32), c_void_p], c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


class CbpError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})")


def status_string(s: int) -> str:
    return lib().cbp_status_string(int(s)).decode()


def _check(s: int, what: str) -> int:
    if s < 0:
        raise CbpError(s, what)
    return s


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else None
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def frames(t: torch.Tensor) -> cbp_frames:
    """Descriptor of a (n, c, h, w), (c, h, w) or (h, w) float32/float64 tensor."""
    if t.dtype not in (torch.float32, torch.float64):
        raise TypeError("frames must be float32 or float64")
    v = t
    while v.dim() < 4:
        v = v.unsqueeze(0)
    n, c, h, w = v.shape
    sn, sc, sh, sw = v.stride()
    if sw != 1:
        raise ValueError("frames need unit column stride")
    return cbp_frames(v.data_ptr(), n, c, h, w, CBP_F64 if t.dtype == torch.float64 else CBP_F32,
                      sh, sc, sn)


def params(t1: int, t2: int, m: int = 0, path: str = "fp64", eps: float = 1e-4, pad_h: int = 0,
           pad_w: int = 0, accept_rho: float = 1e-3, flags: int = 0) -> cbp_params:
    return cbp_params(t1, t2, m, PATHS[path], eps, pad_h, pad_w, accept_rho, flags, 0)


def cbp_create(device: int = 0, hbm_budget_bytes: int = 0) -> c_void_p:
    ctx = c_void_p()
    _check(lib().cbp_create(byref(ctx), device, hbm_budget_bytes), "cbp_create")
    return ctx


def cbp_destroy(ctx) -> None:
    _check(lib().cbp_destroy(ctx), "cbp_destroy")


def cbp_workspace_size(b1, b2, prm: cbp_params) -> int:
    out = ctypes.c_size_t()
    _check(lib().cbp_workspace_size(byref(frames(b1)), byref(frames(b2)), byref(prm), byref(out)),
           "cbp_workspace_size")
    return out.value


def _batch(t: torch.Tensor) -> int:
    return t.shape[0] if t.dim() == 4 else 1


def _out(t, shape, dtype, device, what):
    """Allocate an output, or check a caller-supplied one: the library writes
    raw memory and cannot check sizes itself."""
    if t is None:
        pin = device.type == "cpu" and torch.cuda.is_available()
        return torch.empty(shape, dtype=dtype, device=device, pin_memory=pin)
    if tuple(t.shape) != tuple(shape) or t.dtype != dtype or t.device != device or not t.is_contiguous():
        raise ValueError(f"{what}: expected contiguous {tuple(shape)} {dtype} on {device}, got "
                         f"{tuple(t.shape)} {t.dtype} on {t.device}")
    return t


def cbp_estimate_kernels(ctx, b1: torch.Tensor, b2: torch.Tensor, prm: cbp_params, k1=None, k2=None,
                         diag: bool = True, stream=None):
    """Returns (k1, k2, diag list or None, status).  k1: (n, t1, t1) like b1."""
    n = _batch(b1)
    kdt = torch.float64 if prm.flags & CBP_FLAG_KERNELS_F64 else b1.dtype
    k1 = _out(k1, (n, prm.t1, prm.t1), kdt, b1.device, "k1")
    k2 = _out(k2, (n, prm.t2, prm.t2), kdt, b1.device, "k2")
    d = (cbp_diag * n)() if diag else None
    s = lib().cbp_estimate_kernels(ctx, byref(frames(b1)), byref(frames(b2)), byref(prm),
                                   k1.data_ptr(), k2.data_ptr(), d, _stream_ptr(stream))
    _check(s, "cbp_estimate_kernels")
    return k1, k2, d, s


def cbp_deblur_pair(ctx, b1: torch.Tensor, b2: torch.Tensor, prm: cbp_params, k1=None, k2=None,
                    latent=None, diag: bool = True, stream=None):
    """Returns (latent, k1, k2, diag list or None, status).  latent: (n, c, H, W) like b1.

    With CBP_FLAG_HOST_IO in prm.flags every tensor is a host tensor (pinned
    memory keeps the call asynchronous)."""
    v1 = b1
    while v1.dim() < 4:
        v1 = v1.unsqueeze(0)
    n, c, h1, w1 = v1.shape
    hh, ww = h1 - prm.t1 + 1, w1 - prm.t1 + 1
    if (b1.device.type == "cpu") != bool(prm.flags & CBP_FLAG_HOST_IO):
        raise ValueError("host tensors need CBP_FLAG_HOST_IO and device tensors must not set it")
    latent = _out(latent, (n, c, hh, ww), b1.dtype, b1.device, "latent")
    kin = bool(prm.flags & CBP_FLAG_KERNELS_IN)
    kdt = torch.float64 if prm.flags & CBP_FLAG_KERNELS_F64 else b1.dtype
    if kin and (k1 is None or k2 is None):
        raise ValueError("CBP_FLAG_KERNELS_IN needs k1 and k2")
    if k1 is not None or not kin:
        k1 = _out(k1, (n, prm.t1, prm.t1), kdt, b1.device, "k1")
    if k2 is not None or not kin:
        k2 = _out(k2, (n, prm.t2, prm.t2), kdt, b1.device, "k2")
    d = (cbp_diag * n)() if diag else None
    s = lib().cbp_deblur_pair(ctx, byref(frames(b1)), byref(frames(b2)), byref(prm),
                              k1.data_ptr() if k1 is not None else None,
                              k2.data_ptr() if k2 is not None else None,
                              latent.data_ptr(), d, _stream_ptr(stream))
    _check(s, "cbp_deblur_pair")
    return latent, k1, k2, d, s


def cbp_forward_blur(ctx, latent: torch.Tensor, kernels: torch.Tensor, sigma: float = 0.0,
                     seed: int = 0, out=None, stream=None) -> torch.Tensor:
    """Eq. 1 on the device: latent (n, c, h, w), kernels (n, t, t) float64."""
    if not latent.is_contiguous() or latent.dim() != 4:
        raise ValueError("latent must be a contiguous (n, c, h, w) tensor")
    n, c, h, w = latent.shape
    t = kernels.shape[-1]
    kd = kernels.to(torch.float64).contiguous()
    if kd.shape != (n, t, t):
        raise ValueError("kernels must be (n, t, t)")
    out = _out(out, (n, c, h + t - 1, w + t - 1), latent.dtype, latent.device, "out")
    s = lib().cbp_forward_blur(ctx, latent.data_ptr(), n, c, h, w,
                               CBP_F64 if latent.dtype == torch.float64 else CBP_F32,
                               kd.data_ptr(), t, sigma, seed, out.data_ptr(), _stream_ptr(stream))
    _check(s, "cbp_forward_blur")
    return out


def cbp_synth_latent(ctx, blobs: torch.Tensor, n: int, c: int, h: int, w: int,
                     dtype=torch.float32, floor_amp: float = 0.05, seed: int = 0, out=None,
                     stream=None) -> torch.Tensor:
    """Blob latent on the device; blobs (n, c, nblobs, 4) float64 rows (a, sigma, cx, cy)."""
    bl = blobs.to(torch.float64).contiguous()
    nb = bl.shape[-2]
    if tuple(bl.shape) != (n, c, nb, 4):
        raise ValueError("blobs must be (n, c, nblobs, 4)")
    out = _out(out, (n, c, h, w), dtype, bl.device, "out")
    s = lib().cbp_synth_latent(ctx, bl.data_ptr(), nb, n, c, h, w,
                               CBP_F64 if dtype == torch.float64 else CBP_F32, floor_amp, seed,
                               out.data_ptr(), _stream_ptr(stream))
    _check(s, "cbp_synth_latent")
    return out


def cbp_profile(ctx, enable: bool) -> None:
    _check(lib().cbp_profile(ctx, 1 if enable else 0), "cbp_profile")


def cbp_stage_times(ctx) -> dict:
    """{stage: (milliseconds, kernel launches)} accumulated since the last call."""
    ms = (c_double * len(STAGES))()
    nl = (c_int64 * len(STAGES))()
    _check(lib().cbp_stage_times(ctx, ms, nl), "cbp_stage_times")
    return {name: (ms[i], nl[i]) for i, name in enumerate(STAGES)}


def cbp_estimate_kernels_stages(ctx, b1: torch.Tensor, b2: torch.Tensor, prm: cbp_params, stream=None):
    """Kernel estimation plus every intermediate, as complex/real tensors:
    p_z2/p_z1 (lists over the two frames), x_z2, x_z1, sample_diag, lifted, kernels."""
    v1 = b1 if b1.dim() == 4 else b1.reshape((1,) * (4 - b1.dim()) + tuple(b1.shape))
    v2 = b2 if b2.dim() == 4 else b2.reshape((1,) * (4 - b2.dim()) + tuple(b2.shape))
    n, c = v1.shape[0], v1.shape[1]
    m = prm.m or max(prm.t1, prm.t2)
    s = m // 2 + 1
    nn = prm.t1 + prm.t2
    ct = torch.complex128
    dev = b1.device
    out = {
        "p_z2": [torch.empty((n, c, s, v.shape[2]), dtype=ct, device=dev) for v in (v1, v2)],
        "p_z1": [torch.empty((n, c, s, v.shape[3]), dtype=ct, device=dev) for v in (v1, v2)],
        "x_z2": torch.empty((n, s, nn), dtype=torch.complex128, device=dev),
        "x_z1": torch.empty((n, s, nn), dtype=torch.complex128, device=dev),
        "sample_diag": torch.empty((n, 2, s, 4), dtype=torch.float64, device=dev),
        "lifted": torch.empty((n, 4, m, m), dtype=torch.complex128, device=dev),
        "kernels": torch.empty((n, prm.t1 * prm.t1 + prm.t2 * prm.t2), dtype=torch.float64, device=dev),
    }
    so = cbp_stage_out((c_void_p * 2)(*[t.data_ptr() for t in out["p_z2"]]),
                       (c_void_p * 2)(*[t.data_ptr() for t in out["p_z1"]]),
                       out["x_z2"].data_ptr(), out["x_z1"].data_ptr(), out["sample_diag"].data_ptr(),
                       out["lifted"].data_ptr(), out["kernels"].data_ptr())
    kdt = torch.float64 if prm.flags & CBP_FLAG_KERNELS_F64 else b1.dtype
    k1 = torch.empty((n, prm.t1, prm.t1), dtype=kdt, device=dev)
    k2 = torch.empty((n, prm.t2, prm.t2), dtype=kdt, device=dev)
    d = (cbp_diag * n)()
    st = lib().cbp_estimate_kernels_stages(ctx, byref(frames(b1)), byref(frames(b2)), byref(prm),
                                           k1.data_ptr(), k2.data_ptr(), d, byref(so),
                                           _stream_ptr(stream))
    _check(st, "cbp_estimate_kernels_stages")
    out["k1"], out["k2"], out["diag"] = k1, k2, d
    return out


def cbp_encrypt(ctx, latent: torch.Tensor, t1: int, t2: int, seed: int, frame0: int = 0,
                sigma: float = 0.0, cascade: tuple | None = None, m: int = 0, max_attempts: int = 0,
                tol: float = 0.0, stream=None) -> dict:
    """Camera side on the device (Section 3): per-frame coprime kernel pairs,
    the public/private blurred streams and, with cascade = (t3, t4), the
    cascaded pair.  latent: (n, c, h, w) contiguous device tensor.  Returns a
    dict of tensors (k1, k2, b1, b2[, k3, k4, c1, c2]) and `attempts` (list)."""
    if not latent.is_contiguous() or latent.dim() != 4:
        raise ValueError("(n, c, h, w) contiguous latent expected")
    n, c, h, w = latent.shape
    dev, dt = latent.device, latent.dtype
    t3, t4 = cascade if cascade else (0, 0)
    prm = cbp_encrypt_params(t1, t2, t3, t4, m, max_attempts, tol, sigma, seed, frame0, 0)
    out = {"k1": torch.empty((n, t1, t1), dtype=torch.float64, device=dev),
           "k2": torch.empty((n, t2, t2), dtype=torch.float64, device=dev),
           "b1": torch.empty((n, c, h + t1 - 1, w + t1 - 1), dtype=dt, device=dev),
           "b2": torch.empty((n, c, h + t2 - 1, w + t2 - 1), dtype=dt, device=dev)}
    if cascade:
        out["k3"] = torch.empty((n, t3, t3), dtype=torch.float64, device=dev)
        out["k4"] = torch.empty((n, t4, t4), dtype=torch.float64, device=dev)
        out["c1"] = torch.empty((n, c, h + t1 + t3 - 2, w + t1 + t3 - 2), dtype=dt, device=dev)
        out["c2"] = torch.empty((n, c, h + t1 + t4 - 2, w + t1 + t4 - 2), dtype=dt, device=dev)
    att = (c_int32 * (2 * n if cascade else n))()
    ptr = lambda k: out[k].data_ptr() if k in out else None
    _check(lib().cbp_encrypt(ctx, latent.data_ptr(), n, c, h, w,
                             CBP_F64 if dt == torch.float64 else CBP_F32, byref(prm), ptr("k1"), ptr("k2"),
                             ptr("b1"), ptr("b2"), ptr("k3"), ptr("k4"), ptr("c1"), ptr("c2"), att,
                             _stream_ptr(stream)), "cbp_encrypt")
    torch.cuda.synchronize()
    out["attempts"] = list(att)
    return out


def cbp_truncate_lsb(ctx, x: torch.Tensor, bits: int, drop: int, out: torch.Tensor | None = None,
                     stream=None) -> torch.Tensor:
    """The frames `x` (device, float32/float64, contiguous) with the `drop`
    least significant bits of their `bits`-bit codes removed (Section 3)."""
    if not x.is_contiguous():
        raise ValueError("contiguous frames expected")
    out = torch.empty_like(x) if out is None else out
    dt = CBP_F64 if x.dtype == torch.float64 else CBP_F32
    _check(lib().cbp_truncate_lsb(ctx, x.data_ptr(), dt, x.numel(), bits, drop, out.data_ptr(),
                                  _stream_ptr(stream)), "cbp_truncate_lsb")
    return out


def cbp_estimate_size(ctx, b1: torch.Tensor, b2: torch.Tensor, t_min: int = 0, t_max: int = 0,
                      tol: float = 0.0, stream=None):
    """Kernel-size scan of a batch on the device.  Synchronises the stream and
    returns (t1 list, t2 list, found list, ratios as an (n, ncand) float64
    tensor over the candidates t_min.. after the library's caps, -1 marking
    excluded ones)."""
    n = _batch(b1)
    sp = cbp_size_params(t_min, t_max, tol)
    nc = c_int32()
    cap = 64                      # candidates never exceed t1 + t2 <= 64
    t1 = (c_int32 * n)()
    t2 = (c_int32 * n)()
    fd = (c_int32 * n)()
    ratios = torch.empty((n, cap), dtype=torch.float64).pin_memory() if torch.cuda.is_available() \
        else torch.empty((n, cap), dtype=torch.float64)
    rp = ctypes.cast(ratios.data_ptr(), POINTER(c_double))
    _check(lib().cbp_estimate_size(ctx, byref(frames(b1)), byref(frames(b2)), byref(sp), t1, t2, fd,
                                   rp, byref(nc), _stream_ptr(stream)), "cbp_estimate_size")
    torch.cuda.synchronize()
    k = nc.value
    r = ratios.flatten()[:n * k].reshape(n, k).clone()
    return list(t1), list(t2), [bool(x) for x in fd], r


def cbp_estimate_kernels_noalloc(b1: torch.Tensor, b2: torch.Tensor, prm: cbp_params, k1: torch.Tensor,
                                 k2: torch.Tensor, diag: bool = True, stream=None):
    """Kernel estimation in the library's fixed device scratch array, for callers
    that may not allocate device memory: the caller supplies k1, k2; nothing is
    allocated on the device.  Returns (diag list or None, status)."""
    n = _batch(b1)
    kdt = torch.float64 if prm.flags & CBP_FLAG_KERNELS_F64 else b1.dtype
    _out(k1, (n, prm.t1, prm.t1), kdt, b1.device, "k1")
    _out(k2, (n, prm.t2, prm.t2), kdt, b1.device, "k2")
    d = (cbp_diag * n)() if diag else None
    s = lib().cbp_estimate_kernels_noalloc(byref(frames(b1)), byref(frames(b2)), byref(prm),
                                           k1.data_ptr(), k2.data_ptr(), d, _stream_ptr(stream))
    _check(s, "cbp_estimate_kernels_noalloc")
    return d, s


# ---------------------------------------------------------------- serving --
def cbp_stream_submit(ctx, b1: torch.Tensor, b2: torch.Tensor, prm: cbp_params, k1: torch.Tensor,
                      k2: torch.Tensor, latent: torch.Tensor | None = None) -> int:
    """Queue one frame pair (device tensors, batch of one) with the serving
    engine; latent None asks for the kernels only.  Every tensor must stay
    alive until the request completes.  Returns the ticket."""
    if _batch(b1) != 1 or _batch(b2) != 1:
        raise ValueError("a serving request is one frame pair")
    if prm.flags & CBP_FLAG_HOST_IO:
        raise ValueError("the serving engine takes device tensors")
    v1 = b1
    while v1.dim() < 4:
        v1 = v1.unsqueeze(0)
    _, c, h1, w1 = v1.shape
    kdt = torch.float64 if prm.flags & CBP_FLAG_KERNELS_F64 else b1.dtype
    _out(k1, (1, prm.t1, prm.t1), kdt, b1.device, "k1")
    _out(k2, (1, prm.t2, prm.t2), kdt, b1.device, "k2")
    if latent is not None:
        _out(latent, (1, c, h1 - prm.t1 + 1, w1 - prm.t1 + 1), b1.dtype, b1.device, "latent")
    t = c_uint64()
    s = lib().cbp_stream_submit(ctx, byref(frames(b1)), byref(frames(b2)), byref(prm), k1.data_ptr(),
                                k2.data_ptr(), latent.data_ptr() if latent is not None else None,
                                byref(t))
    _check(s, "cbp_stream_submit")
    return t.value


def cbp_stream_poll(ctx, ticket: int, timeout_us: int = -1):
    """(status, diag) of a ticket: the request's status once done (the ticket
    is then released), CBP_ERR_BUSY / CBP_ERR_TIMEOUT while it is not."""
    d = cbp_diag()
    s = lib().cbp_stream_poll(ctx, ticket, int(timeout_us), byref(d))
    return s, d


def cbp_stream_stats(ctx, reset: bool = False) -> dict:
    n, p50, p99 = c_uint64(), c_double(), c_double()
    _check(lib().cbp_stream_stats(ctx, byref(n), byref(p50), byref(p99), int(reset)), "cbp_stream_stats")
    return {"completed": n.value, "p50_ms": p50.value, "p99_ms": p99.value}


# ------------------------------------------------------ learned proposal --
CNN_SIDE, CNN_T = 256, 15


def cbp_cnn_param_count() -> int:
    return int(lib().cbp_cnn_param_count())


def _trace(trace: dict | None):
    if not trace:
        return None
    t = cbp_cnn_trace()
    t.input = trace["input"].data_ptr() if trace.get("input") is not None else None
    for i, a in enumerate(trace.get("act", [None] * 3)):
        t.act[i] = a.data_ptr() if a is not None else None
    t.logits = trace["logits"].data_ptr() if trace.get("logits") is not None else None
    t.grad = trace["grad"].data_ptr() if trace.get("grad") is not None else None
    return byref(t)


def cnn_trace_buffers(n: int, device, grad: bool = False) -> dict:
    f = dict(dtype=torch.float32, device=device)
    tr = {"input": torch.empty((n, 2, CNN_SIDE, CNN_SIDE), **f),
          "act": [torch.empty((n, 32, CNN_SIDE // 2, CNN_SIDE // 2), **f),
                  torch.empty((n, 32, CNN_SIDE // 4, CNN_SIDE // 4), **f),
                  torch.empty((n, 32, CNN_SIDE // 16, CNN_SIDE // 16), **f)],
          "logits": torch.empty((n, 2, CNN_T, CNN_T), **f)}
    if grad:
        tr["grad"] = torch.empty(cbp_cnn_param_count(), **f)
    return tr


def cbp_cnn_forward(ctx, b1: torch.Tensor, b2: torch.Tensor, weights: torch.Tensor | None = None,
                    trace: dict | None = None, stream=None) -> torch.Tensor:
    """Proposed kernels [n][2][15][15] (float32) for n pairs."""
    n = _batch(b1)
    k = torch.empty((n, 2, CNN_T, CNN_T), dtype=torch.float32, device=b1.device)
    if weights is not None:
        _out(weights, (cbp_cnn_param_count(),), torch.float32, b1.device, "weights")
    s = lib().cbp_cnn_forward(ctx, byref(frames(b1)), byref(frames(b2)),
                              weights.data_ptr() if weights is not None else None, k.data_ptr(),
                              _trace(trace), _stream_ptr(stream))
    _check(s, "cbp_cnn_forward")
    return k


def cbp_cnn_train_step(ctx, b1, b2, k_true: torch.Tensor, weights: torch.Tensor, m: torch.Tensor,
                       v: torch.Tensor, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
                       eps: float = 1e-8, weight_decay: float = 1e-4, loss: torch.Tensor | None = None,
                       trace: dict | None = None, stream=None) -> None:
    n = _batch(b1)
    P = cbp_cnn_param_count()
    for t, nm in ((weights, "weights"), (m, "adam_m"), (v, "adam_v")):
        _out(t, (P,), torch.float32, b1.device, nm)
    _out(k_true, (n, 2, CNN_T, CNN_T), torch.float32, b1.device, "k_true")
    hp = cbp_adamw(lr, beta1, beta2, eps, weight_decay, step)
    s = lib().cbp_cnn_train_step(ctx, byref(frames(b1)), byref(frames(b2)), k_true.data_ptr(),
                                 weights.data_ptr(), m.data_ptr(), v.data_ptr(), byref(hp),
                                 loss.data_ptr() if loss is not None else None, _trace(trace),
                                 _stream_ptr(stream))
    _check(s, "cbp_cnn_train_step")


def save_cnn_weights(path, weights) -> None:
    """Write a weight vector in the file format cbp_learned_load reads."""
    import numpy as np
    w = np.asarray(weights.detach().cpu() if hasattr(weights, "detach") else weights, dtype="<f4")
    if w.size != cbp_cnn_param_count():
        raise ValueError("wrong number of weights")
    with open(path, "wb") as f:
        f.write(b"CBPCNN1\0")
        f.write(np.array([CNN_SIDE, w.size], dtype="<i4").tobytes())
        f.write(w.tobytes())


def cbp_learned_load(ctx, path) -> None:
    _check(lib().cbp_learned_load(ctx, str(path).encode()), "cbp_learned_load")


CHECK_WORDS = 6   # source files with checked sites: fft, colpass, eval, solve, cnn, forward


def cbp_check_words(reset: bool = False) -> list:
    """The bounds-checked build's check words (all zero: no failed check);
    raises CbpError(CBP_ERR_UNSUPPORTED) in a normal build."""
    w = (c_uint32 * CHECK_WORDS)()
    _check(lib().cbp_check_words(w, CHECK_WORDS, int(reset)), "cbp_check_words")
    return list(w)


def cbp_check_expire_waits(on: bool) -> None:
    """Checked build only: make the row passes' bulk-copy waits run out
    (CBP_ERR_TIMEOUT) or restore them."""
    _check(lib().cbp_check_expire_waits(int(on)), "cbp_check_expire_waits")
