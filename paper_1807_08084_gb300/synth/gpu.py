"""GPU twin of the seeded generators (libzsynth.so, built from synth.cu).

Produces the same bits as the numpy twin in ``synth/__init__.py`` for every
pixel, at full image sizes (a 16384 x 16384 packed image is 9.7 GB), directly
in device memory.  The class tables and block maps are computed once on the
host by the numpy twin and copied to the device, so both sides use the same
values.
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np
import torch

from .. import build as _build
from . import TAG_GRAD, Workload, dlog

_lib = None
_lock = threading.Lock()
_P, _I64, _U32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint32


def load() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(str(_build.build_lib("libzsynth.so")))
            lib.synth_z_wishart.argtypes = [_U32, _I64, _I64, ctypes.c_int, _P, _P, ctypes.c_int,
                                            _P, _I64, _P]
            lib.synth_z_cond.argtypes = [_U32, _I64, ctypes.c_double, _P, _I64, _P]
            lib.synth_z_rrh.argtypes = [_U32, _I64, _P, _I64, _P]
            lib.synth_slc.argtypes = [_U32, _I64, _I64, _P, _P, ctypes.c_int, ctypes.c_int, _P,
                                      _I64, _P]
            lib.synth_uniform.argtypes = [_U32, _U32, _U32, _I64, ctypes.c_double,
                                          ctypes.c_double, _P, _P]
            for f in ("synth_z_wishart", "synth_z_cond", "synth_z_rrh", "synth_slc",
                      "synth_uniform"):
                getattr(lib, f).restype = ctypes.c_int
            _lib = lib
        return _lib


def _stream(dev):
    return ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


def _check(rc, fn):
    if rc != 0:
        raise RuntimeError(f"{fn} failed ({rc})")


def _tables(w: Workload, device, date: int = 0):
    F = np.asarray(w.factors(), dtype=np.complex128).reshape(-1, 3, 3)
    Ft = torch.from_numpy(np.ascontiguousarray(np.stack([F.real, F.imag], axis=-1))).to(device)
    bm = w.block_map(date)
    bmt = None if bm is None else torch.from_numpy(bm.astype(np.int32)).to(device)
    return Ft, bmt


def packed_z(w: Workload, device="cuda", out: torch.Tensor | None = None) -> torch.Tensor:
    """float32 [9, H, W] packed Z of a packed-Z workload, generated on the GPU."""
    lib = load()
    device = torch.device(device)
    z = torch.empty((9, w.H, w.W), dtype=torch.float32, device=device) if out is None else out
    n = w.n
    with torch.cuda.device(device):
        s = _stream(device)
        if w.kind == "wishart":
            Ft, bmt = _tables(w, device)
            rc = lib.synth_z_wishart(w.seed, w.H, w.W, w.N, Ft.data_ptr(),
                                     None if bmt is None else bmt.data_ptr(), max(w.block, 1),
                                     z.data_ptr(), n, s)
            torch.cuda.current_stream(device).synchronize()  # tables die with this frame
        elif w.kind == "cond":
            rc = lib.synth_z_cond(w.seed, n, float(dlog(w.kappa_max)), z.data_ptr(), n, s)
        elif w.kind == "rrh":
            rc = lib.synth_z_rrh(w.seed, n, z.data_ptr(), n, s)
        else:
            raise ValueError(w.kind)
    _check(rc, "synth packed_z")
    return z


def image(w: Workload, date: int = 0, device="cuda") -> torch.Tensor:
    """complex64 [3, H, W] single-look image of one date, generated on the GPU."""
    lib = load()
    device = torch.device(device)
    s = torch.empty((3, w.H, w.W), dtype=torch.complex64, device=device)
    with torch.cuda.device(device):
        Ft, bmt = _tables(w, device, date)
        rc = lib.synth_slc(w.seed, w.H, w.W, Ft.data_ptr(),
                           None if bmt is None else bmt.data_ptr(), max(w.block, 1), date,
                           s.data_ptr(), w.n, _stream(device))
        torch.cuda.current_stream(device).synchronize()
    _check(rc, "synth image")
    return s


def uniform(seed: int, n: int, tag: int = TAG_GRAD, stream: int = 0, lo=-1.0, hi=1.0,
            device="cuda") -> torch.Tensor:
    """float32 [n] uniforms on (lo, hi], matching synth.uniform_f32."""
    lib = load()
    device = torch.device(device)
    out = torch.empty(n, dtype=torch.float32, device=device)
    with torch.cuda.device(device):
        rc = lib.synth_uniform(seed, tag, stream, n, float(lo), float(hi), out.data_ptr(),
                               _stream(device))
    _check(rc, "synth uniform")
    return out
