"""GB300-native inverse and determinant of per-pixel 3x3 Hermitian PolSAR matrices.

Thin Python binding over the C ABI of ``libzinv.so`` (declared in
``include/zinv.h``): each function checks and marshals torch CUDA tensors and
calls the entry point of the same name on the current torch stream.  All
arithmetic runs in the library's CUDA kernels; there is no CPU path, and every
function raises if the library cannot be built or loaded or if a tensor is not
on a CUDA device.

Method: Coelho, Cintra, Frery, Dimitrov, "Fast Matrix Inversion and Determinant
Computation for Polarimetric Synthetic Aperture Radar", arXiv:1807.08084 --
Alg. 2 (adjugate, §3.1) and its baseline Alg. 1 (Cholesky, §2.2).

Packed layout: float32 [9, ...] planes a, Re b, Im b, Re c, Im c, d, Re e,
Im e, f of Z = [[a, b, c], [conj b, d, e], [conj c, conj e, f]] (§2.1).
"""
from __future__ import annotations

import ctypes
import threading

import torch

from . import build as _build

PLAIN = 0
COMPENSATED = 1
FP64_RECOMPUTE = 2
HOST_STAGED = 4
PIX_NOT_PD = 1
PIX_RECOMPUTED = 2
DEFAULT_TAU = 2.0 ** -10

_lib = None
_lock = threading.Lock()

_P = ctypes.c_void_p
_I64 = ctypes.c_int64


def load() -> ctypes.CDLL:
    """Builds libzinv.so in-tree if it is missing or stale, loads it once."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build_lib("libzinv.so")
        lib = ctypes.CDLL(str(path))
        lib.zinv_abi_version.restype = ctypes.c_int
        lib.zinv_status_string.restype = ctypes.c_char_p
        lib.zinv_status_string.argtypes = [ctypes.c_int]
        sig = [_P, _I64, _I64, _P, _P, ctypes.c_uint32, ctypes.c_float, _P, _P, _P]
        for f in ("zinv_det", "chol_zinv_det"):
            getattr(lib, f).argtypes = sig
            getattr(lib, f).restype = ctypes.c_int
        lib.zinv_det_bwd.argtypes = [_P, _P, _I64, _I64, _P, _P, _P, _P, _P]
        lib.zinv_det_bwd.restype = ctypes.c_int
        lib.zinv_det_host_workspace_bytes.argtypes = [_I64]
        lib.zinv_det_host_workspace_bytes.restype = ctypes.c_size_t
        lib.zinv_det_host.argtypes = [_P, _I64, _I64, _P, _P, ctypes.c_uint32, ctypes.c_float,
                                      _P, ctypes.c_size_t, _P]
        lib.zinv_det_host.restype = ctypes.c_int
        _declare_extra(lib)
        if lib.zinv_abi_version() != 1:
            raise RuntimeError("libzinv.so ABI version mismatch")
        _lib = lib
        return lib


def _declare_extra(lib):
    """Signatures of the window, block-diagonal, nonlocal-means and Wishart entry points
    (including the allocation-free Wishart forward)."""
    lib.multilook_zinv_det.argtypes = [_P, _I64, _I64, _I64, ctypes.c_int, _P, _P, _P,
                                       ctypes.c_uint32, ctypes.c_float, _P, _P, _P]
    lib.multilook_zinv_det.restype = ctypes.c_int
    lib.zinv_det_blockdiag.argtypes = [_P, ctypes.c_int, _I64, _I64, _P, _P, ctypes.c_uint32,
                                       ctypes.c_float, _P, _P, _P]
    lib.zinv_det_blockdiag.restype = ctypes.c_int
    lib.nlm_wishart.argtypes = [_P, _I64, _I64, _I64, ctypes.c_int, ctypes.c_float,
                                ctypes.c_float, ctypes.c_int, _P, _P]
    lib.nlm_wishart.restype = ctypes.c_int
    lib.nlm_stochastic.argtypes = [_P, _I64, _I64, _I64, ctypes.c_int, ctypes.c_float,
                                   ctypes.c_float, ctypes.c_int, ctypes.c_float, ctypes.c_int,
                                   _P, _P]
    lib.nlm_stochastic.restype = ctypes.c_int
    lib.wishart_workspace_bytes.argtypes = [_I64, _I64, ctypes.c_int]
    lib.wishart_workspace_bytes.restype = ctypes.c_size_t
    lib.wishart_saved_bytes.argtypes = [_I64, _I64]
    lib.wishart_saved_bytes.restype = ctypes.c_size_t
    lib.wishart_bwd_saved_workspace_bytes.argtypes = [_I64, _I64, ctypes.c_int]
    lib.wishart_bwd_saved_workspace_bytes.restype = ctypes.c_size_t
    lib.wishart_stat_fwd_save.argtypes = [_P, _P, _I64, _I64, _I64, ctypes.c_int, _P, _P, _P,
                                          _P, _P, ctypes.c_size_t, _P]
    lib.wishart_stat_fwd_save.restype = ctypes.c_int
    lib.wishart_stat_bwd_saved.argtypes = [_P, _P, _I64, _I64, _I64, ctypes.c_int, _P, _P, _P,
                                           _P, ctypes.c_size_t, _P]
    lib.wishart_stat_bwd_saved.restype = ctypes.c_int
    lib.wishart_stat_fwd.argtypes = [_P, _P, _I64, _I64, _I64, ctypes.c_int, _P, _P, _P,
                                     _P, ctypes.c_size_t, _P]
    lib.wishart_stat_fwd.restype = ctypes.c_int
    lib.wishart_stat_bwd.argtypes = [_P, _P, _I64, _I64, _I64, ctypes.c_int, _P, _P, _P,
                                     _P, ctypes.c_size_t, _P]
    lib.wishart_stat_bwd.restype = ctypes.c_int
    lib.wishart_stat_fwd_noalloc.argtypes = [_P, _P, _I64, _I64, _I64, ctypes.c_int, _P, _P, _P,
                                             _P]
    lib.wishart_stat_fwd_noalloc.restype = ctypes.c_int


def status_string(code: int) -> str:
    return load().zinv_status_string(code).decode()


def _check(rc: int, fn: str):
    if rc != 0:
        raise RuntimeError(f"{fn} failed: {status_string(rc)} ({rc})")


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(dev) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


def _planes(z: torch.Tensor, name: str = "z", nplanes: int = 9):
    """(n, ld) of a [9, ...] float32 CUDA tensor in the packed layout."""
    if not z.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (there is no CPU path)")
    if z.dtype != torch.float32:
        raise ValueError(f"{name} must be float32")
    if z.dim() < 2 or z.shape[0] != nplanes:
        raise ValueError(f"{name} must have shape [{nplanes}, ...]")
    if z.dim() == 2 and (z.stride(1) == 1 or z.shape[1] <= 1):
        return z.shape[1], max(z.stride(0), z.shape[1])
    if not z.is_contiguous():
        raise ValueError(f"{name} must be contiguous (or a [9, n] view with unit column stride)")
    n = z[0].numel()
    return n, n


def _like(t: torch.Tensor, ref: torch.Tensor, name: str, ref_name: str):
    """t must be a float32 tensor with ref's device, shape and strides."""
    if (t.dtype != torch.float32 or t.device != ref.device or t.shape != ref.shape
            or t.stride() != ref.stride()):
        raise ValueError(f"{name} must be float32 with the device, shape and strides of {ref_name}")
    return t


def _out(t: torch.Tensor, shape, device, name: str):
    """A caller-supplied output: contiguous float32 of `shape` on `device`."""
    if (t.dtype != torch.float32 or t.device != device or tuple(t.shape) != tuple(shape)
            or not t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous float32 tensor of shape {tuple(shape)} "
                         f"on {device}")
    return t


def _flat(x: torch.Tensor | None, n: int, name: str):
    if x is None:
        return None
    if not x.is_cuda or x.dtype != torch.float32 or x.numel() != n or not x.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor of {n} elements")
    return x


def zinv_det(z: torch.Tensor, flags: int = PLAIN, tau: float = DEFAULT_TAU,
             want_status: bool = False, want_counts: bool = False,
             out: tuple | None = None):
    """Alg. 2: (Z^-1 packed like z, det [...]) [+ status uint8] [+ counts int64[2]]."""
    return _inv_det("zinv_det", z, flags, tau, want_status, want_counts, out)


def chol_zinv_det(z: torch.Tensor, want_status: bool = False, want_counts: bool = False,
                  out: tuple | None = None):
    """Alg. 1 (Cholesky route, with the corrected l21): same outputs as zinv_det."""
    return _inv_det("chol_zinv_det", z, PLAIN, 0.0, want_status, want_counts, out)


def _inv_det(fn, z, flags, tau, want_status, want_counts, out):
    lib = load()
    n, ld = _planes(z)
    if out is None:
        zinv = torch.empty_strided(z.shape, z.stride(), dtype=z.dtype, device=z.device)
        det = torch.empty(z.shape[1:], dtype=torch.float32, device=z.device)
    else:
        zinv, det = out
        _like(zinv, z, "zinv", "z")
        _flat(det, n, "det")
    status = torch.empty(z.shape[1:], dtype=torch.uint8, device=z.device) if want_status else None
    counts = torch.empty(2, dtype=torch.int64, device=z.device) if want_counts else None
    with torch.cuda.device(z.device):
        rc = getattr(lib, fn)(_ptr(z), n, ld, _ptr(zinv), _ptr(det), int(flags), float(tau),
                              _ptr(status), _ptr(counts), _stream(z.device))
    _check(rc, fn)
    res = (zinv, det)
    if want_status:
        res += (status,)
    if want_counts:
        res += (counts,)
    return res


def zinv_det_bwd(zinv: torch.Tensor, det: torch.Tensor, g_zinv=None, g_det=None,
                 g_logdet=None, out: torch.Tensor | None = None) -> torch.Tensor:
    """Packed gradient w.r.t. Z from W = Z^-1, det and upstream gradients (any may be None)."""
    lib = load()
    n, ld = _planes(zinv, "zinv")
    _flat(det, n, "det")
    if g_zinv is not None:
        _like(g_zinv, zinv, "g_zinv", "zinv")
    _flat(g_det, n, "g_det")
    _flat(g_logdet, n, "g_logdet")
    if out is None:
        g_z = torch.empty_strided(zinv.shape, zinv.stride(), dtype=zinv.dtype, device=zinv.device)
    else:
        g_z = _like(out, zinv, "out", "zinv")
    with torch.cuda.device(zinv.device):
        rc = lib.zinv_det_bwd(_ptr(zinv), _ptr(det), n, ld, _ptr(g_zinv), _ptr(g_det),
                              _ptr(g_logdet), _ptr(g_z), _stream(zinv.device))
    _check(rc, "zinv_det_bwd")
    return g_z


def _slc(s: torch.Tensor, name: str = "s"):
    """(H, W, plane_ld) of a complex64 [3, H, W] CUDA tensor with contiguous rows."""
    if not s.is_cuda or s.dtype != torch.complex64:
        raise ValueError(f"{name} must be a complex64 CUDA tensor")
    if s.dim() != 3 or s.shape[0] != 3:
        raise ValueError(f"{name} must have shape [3, H, W]")
    H, W = s.shape[1], s.shape[2]
    if s.stride(2) != 1 or (H > 1 and s.stride(1) != W):
        raise ValueError(f"{name} rows must be contiguous ([3, H, W] with strides (plane, W, 1))")
    return H, W, max(s.stride(0), H * W)


def multilook_zinv_det(s: torch.Tensor, win: int = 7, weights: torch.Tensor | None = None,
                       flags: int = PLAIN, tau: float = DEFAULT_TAU, want_status: bool = False,
                       want_counts: bool = False, out: tuple | None = None):
    """Fused multilook (boxcar mean, or the weighted window) + Algorithm 2.

    s: complex64 [3, H, W] single-look vectors; returns (Z^-1 [9, H, W], det [H, W])
    [+ status] [+ counts]; Z itself is never materialised."""
    lib = load()
    H, W, pld = _slc(s)
    if weights is not None:
        if (not weights.is_cuda or weights.dtype != torch.float32 or weights.numel() != win * win
                or not weights.is_contiguous()):
            raise ValueError("weights must be a contiguous float32 CUDA tensor of win*win values")
    if out is None:
        zinv = torch.empty((9, H, W), dtype=torch.float32, device=s.device)
        det = torch.empty((H, W), dtype=torch.float32, device=s.device)
    else:
        zinv = _out(out[0], (9, H, W), s.device, "zinv")
        det = _out(out[1], (H, W), s.device, "det")
    status = torch.empty((H, W), dtype=torch.uint8, device=s.device) if want_status else None
    counts = torch.empty(2, dtype=torch.int64, device=s.device) if want_counts else None
    with torch.cuda.device(s.device):
        rc = lib.multilook_zinv_det(_ptr(s), H, W, pld, int(win), _ptr(weights), _ptr(zinv),
                                    _ptr(det), int(flags), float(tau), _ptr(status), _ptr(counts),
                                    _stream(s.device))
    _check(rc, "multilook_zinv_det")
    res = (zinv, det)
    if want_status:
        res += (status,)
    if want_counts:
        res += (counts,)
    return res


def zinv_det_blockdiag(z: torch.Tensor, flags: int = PLAIN, tau: float = DEFAULT_TAU,
                       want_status: bool = False, want_counts: bool = False):
    """Multifrequency pixels: z float32 [nb, 9, ...] (nb diagonal 3x3 blocks per pixel).
    Returns (the blocks' inverses, shaped like z; det = product over blocks) [+ status]
    [+ counts]."""
    lib = load()
    if not z.is_cuda or z.dtype != torch.float32 or z.dim() < 3 or z.shape[1] != 9:
        raise ValueError("z must be a float32 CUDA tensor of shape [nb, 9, ...]")
    if not z.is_contiguous():
        raise ValueError("z must be contiguous")
    nb = z.shape[0]
    n = z[0, 0].numel()
    zinv = torch.empty_like(z)
    det = torch.empty(z.shape[2:], dtype=torch.float32, device=z.device)
    status = torch.empty(z.shape[2:], dtype=torch.uint8, device=z.device) if want_status else None
    counts = torch.empty(2, dtype=torch.int64, device=z.device) if want_counts else None
    with torch.cuda.device(z.device):
        rc = lib.zinv_det_blockdiag(_ptr(z), nb, n, n, _ptr(zinv), _ptr(det), int(flags),
                                    float(tau), _ptr(status), _ptr(counts), _stream(z.device))
    _check(rc, "zinv_det_blockdiag")
    res = (zinv, det)
    if want_status:
        res += (status,)
    if want_counts:
        res += (counts,)
    return res


NLM_ADJUGATE = 0
NLM_CHOLESKY = 1
NLM_COMPENSATED = 2   # Bhattacharyya and Hellinger: compensated pair determinant


def nlm_wishart(z: torch.Tensor, radius: int = 11, looks: float = 16.0, h: float = 1.0,
                method: int = NLM_ADJUGATE, out: torch.Tensor | None = None) -> torch.Tensor:
    """Nonlocal-means filter of a packed [9, H, W] image with the Wishart
    equal-looks distance over a (2 radius + 1)^2 search window; the per-pair
    determinant by Algorithm 2 (NLM_ADJUGATE), Algorithm 1 (NLM_CHOLESKY) or
    compensated Algorithm 2 on the exact pair sum (NLM_COMPENSATED)."""
    lib = load()
    if z.dim() != 3:
        raise ValueError("z must be [9, H, W]")
    n, ld = _planes(z)
    H, W = z.shape[1], z.shape[2]
    if out is None:
        out = torch.empty((9, H, W), dtype=torch.float32, device=z.device)
    else:
        _out(out, (9, H, W), z.device, "out")
    with torch.cuda.device(z.device):
        rc = lib.nlm_wishart(_ptr(z), H, W, ld, int(radius), float(looks), float(h), int(method),
                             _ptr(out), _stream(z.device))
    _check(rc, "nlm_wishart")
    return out


NLM_BHATTACHARYYA = 0
NLM_HELLINGER = 1
NLM_KULLBACK_LEIBLER = 2
NLM_RENYI = 3


def nlm_stochastic(z: torch.Tensor, radius: int = 11, looks: float = 16.0, h: float = 1.0,
                   distance: int = NLM_BHATTACHARYYA, method: int = NLM_ADJUGATE,
                   out: torch.Tensor | None = None, order: float = 0.5) -> torch.Tensor:
    """Nonlocal-means filter of a packed [9, H, W] image with weights
    exp(-d / h), d the Bhattacharyya, Hellinger, Kullback-Leibler or Renyi
    (of `order` in (0, 1)) distance between the pixels' equal-looks Wishart
    laws; the per-pair determinants by Algorithm 2 (NLM_ADJUGATE) or
    Algorithm 1 (NLM_CHOLESKY), for Bhattacharyya and Hellinger also
    compensated (NLM_COMPENSATED), Kullback-Leibler taking none."""
    lib = load()
    if z.dim() != 3:
        raise ValueError("z must be [9, H, W]")
    n, ld = _planes(z)
    H, W = z.shape[1], z.shape[2]
    if out is None:
        out = torch.empty((9, H, W), dtype=torch.float32, device=z.device)
    else:
        _out(out, (9, H, W), z.device, "out")
    with torch.cuda.device(z.device):
        rc = lib.nlm_stochastic(_ptr(z), H, W, ld, int(radius), float(looks), float(h),
                                int(distance), float(order), int(method), _ptr(out),
                                _stream(z.device))
    _check(rc, "nlm_stochastic")
    return out


def wishart_workspace_bytes(H: int, W: int, win: int) -> int:
    return int(load().wishart_workspace_bytes(int(H), int(W), int(win)))


def _wishart_common(s1, s2, weights, win, ws):
    H, W, pld = _slc(s1, "s1")
    H2, W2, pld2 = _slc(s2, "s2")
    if (H, W) != (H2, W2) or pld != pld2 or s1.device != s2.device:
        raise ValueError("s1 and s2 must have the same shape, plane stride and device")
    if (not weights.is_cuda or weights.dtype != torch.float32 or weights.numel() != win * win
            or not weights.is_contiguous()):
        raise ValueError("weights must be a contiguous float32 CUDA tensor of win*win values")
    need = wishart_workspace_bytes(H, W, win)
    if ws is None:
        ws = torch.empty(need, dtype=torch.uint8, device=s1.device)
    elif not ws.is_cuda or ws.dtype != torch.uint8 or ws.numel() < need:
        raise ValueError(f"ws must be a uint8 CUDA tensor of at least {need} bytes")
    return H, W, pld, ws


def wishart_stat_fwd(s1: torch.Tensor, s2: torch.Tensor, weights: torch.Tensor, win: int = 7,
                     want_map: bool = False, ws: torch.Tensor | None = None):
    """L = sum_p [ln det Z1 + ln det Z2 - 2 ln det((Z1+Z2)/2)] (float64 0-dim tensor)
    [+ the per-pixel q map [H, W]]."""
    lib = load()
    H, W, pld, ws = _wishart_common(s1, s2, weights, win, ws)
    loss = torch.empty((), dtype=torch.float64, device=s1.device)
    q = torch.empty((H, W), dtype=torch.float32, device=s1.device) if want_map else None
    with torch.cuda.device(s1.device):
        rc = lib.wishart_stat_fwd(_ptr(s1), _ptr(s2), H, W, pld, int(win), _ptr(weights),
                                  _ptr(q), _ptr(loss), _ptr(ws), ws.numel(), _stream(s1.device))
    _check(rc, "wishart_stat_fwd")
    return (loss, q) if want_map else loss


def wishart_stat_bwd(s1: torch.Tensor, s2: torch.Tensor, weights: torch.Tensor, win: int = 7,
                     grad_loss: torch.Tensor | None = None, ws: torch.Tensor | None = None):
    """g * dL/dw (float32, shaped like weights); grad_loss a float64 CUDA scalar or None (1)."""
    lib = load()
    H, W, pld, ws = _wishart_common(s1, s2, weights, win, ws)
    if grad_loss is not None:
        grad_loss = grad_loss.to(device=s1.device, dtype=torch.float64).contiguous()
    gw = torch.empty_like(weights)
    with torch.cuda.device(s1.device):
        rc = lib.wishart_stat_bwd(_ptr(s1), _ptr(s2), H, W, pld, int(win), _ptr(weights),
                                  _ptr(grad_loss), _ptr(gw), _ptr(ws), ws.numel(),
                                  _stream(s1.device))
    _check(rc, "wishart_stat_bwd")
    return gw


def wishart_stat_fwd_save(s1: torch.Tensor, s2: torch.Tensor, weights: torch.Tensor,
                          win: int = 7, want_map: bool = False,
                          z_saved: torch.Tensor | None = None, ws: torch.Tensor | None = None):
    """wishart_stat_fwd that also returns both dates' window covariances Z
    ([18, H, W] float32: date 1's packed planes, then date 2's) for
    wishart_stat_bwd_saved: (loss, z_saved) or (loss, z_saved, q)."""
    lib = load()
    H, W, pld, ws = _wishart_common(s1, s2, weights, win, ws)
    if z_saved is None:
        z_saved = torch.empty((18, H, W), dtype=torch.float32, device=s1.device)
    else:
        _out(z_saved, (18, H, W), s1.device, "z_saved")
    loss = torch.empty((), dtype=torch.float64, device=s1.device)
    q = torch.empty((H, W), dtype=torch.float32, device=s1.device) if want_map else None
    with torch.cuda.device(s1.device):
        rc = lib.wishart_stat_fwd_save(_ptr(s1), _ptr(s2), H, W, pld, int(win), _ptr(weights),
                                       _ptr(q), _ptr(loss), _ptr(z_saved), _ptr(ws), ws.numel(),
                                       _stream(s1.device))
    _check(rc, "wishart_stat_fwd_save")
    return (loss, z_saved, q) if want_map else (loss, z_saved)


def wishart_bwd_saved_workspace_bytes(H: int, W: int, win: int) -> int:
    return int(load().wishart_bwd_saved_workspace_bytes(int(H), int(W), int(win)))


def wishart_stat_bwd_saved(s1: torch.Tensor, s2: torch.Tensor, z_saved: torch.Tensor,
                           win: int = 7, grad_loss: torch.Tensor | None = None,
                           ws: torch.Tensor | None = None):
    """g * dL/dw (float32 [win*win]) from the forward's saved Z: the same bits
    as wishart_stat_bwd without recomputing the window sums."""
    lib = load()
    H, W, pld = _slc(s1, "s1")
    if _slc(s2, "s2") != (H, W, pld) or s1.device != s2.device:
        raise ValueError("s1 and s2 must have the same shape, plane stride and device")
    _out(z_saved, (18, H, W), s1.device, "z_saved")
    need = wishart_bwd_saved_workspace_bytes(H, W, win)
    if ws is None:
        ws = torch.empty(need, dtype=torch.uint8, device=s1.device)
    elif not ws.is_cuda or ws.dtype != torch.uint8 or ws.numel() < need:
        raise ValueError(f"ws must be a uint8 CUDA tensor of at least {need} bytes")
    if grad_loss is not None:
        grad_loss = grad_loss.to(device=s1.device, dtype=torch.float64).contiguous()
    gw = torch.empty(win * win, dtype=torch.float32, device=s1.device)
    with torch.cuda.device(s1.device):
        rc = lib.wishart_stat_bwd_saved(_ptr(s1), _ptr(s2), H, W, pld, int(win), _ptr(z_saved),
                                        _ptr(grad_loss), _ptr(gw), _ptr(ws), ws.numel(),
                                        _stream(s1.device))
    _check(rc, "wishart_stat_bwd_saved")
    return gw


class WishartStat(torch.autograd.Function):
    """loss = WishartStat.apply(s1, s2, weights, win, save_z): the change
    statistic with a learnable window; returns the weights' gradient only (the
    images are data).  The backward recomputes Z from s1, s2 in the kernel, or
    with save_z=True reads the Z the forward saved (72 bytes per pixel kept
    between the two passes)."""

    @staticmethod
    def forward(ctx, s1, s2, weights, win: int = 7, save_z: bool = False):
        ctx.win, ctx.save_z = win, save_z
        if save_z:
            loss, z_saved = wishart_stat_fwd_save(s1, s2, weights.contiguous(), win)
            ctx.save_for_backward(s1, s2, weights, z_saved)
            return loss
        ctx.save_for_backward(s1, s2, weights)
        return wishart_stat_fwd(s1, s2, weights.contiguous(), win)

    @staticmethod
    def backward(ctx, g):
        if ctx.save_z:
            s1, s2, weights, z_saved = ctx.saved_tensors
            gw = wishart_stat_bwd_saved(s1, s2, z_saved, ctx.win, g.reshape(()))
        else:
            s1, s2, weights = ctx.saved_tensors
            gw = wishart_stat_bwd(s1, s2, weights.contiguous(), ctx.win, g.reshape(()))
        return None, None, gw.reshape(weights.shape), None, None


def zinv_det_host_workspace_bytes(chunk: int) -> int:
    return int(load().zinv_det_host_workspace_bytes(int(chunk)))


def zinv_det_host(z_host: torch.Tensor, ws: torch.Tensor | None = None, flags: int = PLAIN,
                  tau: float = DEFAULT_TAU, out: tuple | None = None,
                  device: torch.device | None = None):
    """zinv_det over host tensors.  Pinned buffers are processed in place by the
    kernel over the CPU-GPU link; otherwise (or with HOST_STAGED in flags) the
    image streams through the device workspace `ws` (a uint8 CUDA tensor of
    zinv_det_host_workspace_bytes(chunk) bytes).  Asynchronous: synchronize the
    current stream before reading the outputs."""
    lib = load()
    if z_host.is_cuda or z_host.dtype != torch.float32 or z_host.shape[0] != 9:
        raise ValueError("z_host must be a float32 host tensor of shape [9, ...]")
    if not z_host.is_contiguous():
        raise ValueError("z_host must be contiguous")
    n = z_host[0].numel()
    if ws is not None and (not ws.is_cuda or ws.dtype != torch.uint8):
        raise ValueError("ws must be a uint8 CUDA tensor")
    if out is None:
        zinv = torch.empty_like(z_host, pin_memory=True)
        det = torch.empty(z_host.shape[1:], dtype=torch.float32, pin_memory=True)
    else:
        zinv, det = out
        if (zinv.is_cuda or zinv.dtype != torch.float32 or zinv.shape != z_host.shape
                or not zinv.is_contiguous()):
            raise ValueError("zinv must be a contiguous float32 host tensor shaped like z_host")
        if det.is_cuda or det.dtype != torch.float32 or det.numel() != n or not det.is_contiguous():
            raise ValueError(f"det must be a contiguous float32 host tensor of {n} elements")
    dev = (ws.device if ws is not None else torch.device("cuda", torch.cuda.current_device())) \
        if device is None else device
    with torch.cuda.device(dev):
        rc = lib.zinv_det_host(_ptr(z_host), n, n, _ptr(zinv), _ptr(det), int(flags), float(tau),
                               _ptr(ws), 0 if ws is None else ws.numel(), _stream(dev))
    _check(rc, "zinv_det_host")
    return zinv, det


class ZInvDet(torch.autograd.Function):
    """(Z^-1, det) = ZInvDet.apply(z) with the hand-written backward kernel.

    Gradients are real partial derivatives w.r.t. the nine packed reals of z.
    """

    @staticmethod
    def forward(ctx, z, flags: int = PLAIN, tau: float = DEFAULT_TAU):
        zinv, det = zinv_det(z, flags, tau)
        ctx.save_for_backward(zinv, det)
        return zinv, det

    @staticmethod
    def backward(ctx, g_zinv, g_det):
        zinv, det = ctx.saved_tensors
        g_zinv = None if g_zinv is None else g_zinv.contiguous()
        g_det = None if g_det is None else g_det.contiguous()
        return zinv_det_bwd(zinv, det, g_zinv, g_det, None), None, None

