"""Plain FP64 CPU oracle for the 3x3 Hermitian inverse / determinant path.

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import this
package.  The arithmetic lives in ``oracle.c`` (plain single-threaded C, FP64),
which shares no code with the CUDA library; this module only compiles it with
gcc and marshals numpy arrays through ctypes.  Every input is widened to
float64 exactly before it reaches the C code.

Paper: Coelho, Cintra, Frery, Dimitrov, "Fast Matrix Inversion and Determinant
Computation for Polarimetric Synthetic Aperture Radar", arXiv:1807.08084.
Which section each function follows is stated in ``oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "oracle.c"
BUILD_DIR = HERE / "_build"

_lock = threading.Lock()
_default = None


def compile_oracle(out: Path | None = None, mutant: int = 0) -> Path:
    """Compiles oracle.c into a shared library (mutant > 0 plants a mistake)."""
    BUILD_DIR.mkdir(exist_ok=True)
    if out is None:
        out = BUILD_DIR / ("liboracle.so" if mutant == 0 else f"liboracle_mutant{mutant}.so")
    if out.exists() and out.stat().st_mtime >= SRC.stat().st_mtime:
        return out
    tmp = out.with_suffix(f".tmp{os.getpid()}.so")
    cmd = [
        "gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
        f"-DORACLE_MUTANT={mutant}", str(SRC), "-o", str(tmp), "-lm",
    ]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.c_int64


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=np.float64)


def _slc_f64(s) -> tuple[np.ndarray, int, int]:
    """complex [3, H, W] -> interleaved float64 buffer, H, W."""
    s = np.asarray(s)
    assert s.ndim == 3 and s.shape[0] == 3 and np.iscomplexobj(s)
    buf = np.ascontiguousarray(s.astype(np.complex128)).view(np.float64)
    return np.ascontiguousarray(buf), s.shape[1], s.shape[2]


class Oracle:
    """ctypes handle on one build of oracle.c."""

    def __init__(self, path: Path):
        self.path = Path(path)
        lib = ctypes.CDLL(str(self.path))
        lib.oracle_version.restype = ctypes.c_int
        lib.oracle_zinv_det.argtypes = [_D, _I64, _I64, _D, _D, _D]
        lib.oracle_det_expansions.argtypes = [_D, _I64, _I64, _D]
        lib.oracle_inverse_full.argtypes = [_D, _I64, _I64, ctypes.c_int, _D]
        lib.oracle_eigvals.argtypes = [_D, _I64, _I64, _D]
        lib.oracle_multilook.argtypes = [_D, _I64, _I64, _I64, ctypes.c_int, _D, _D]
        lib.oracle_zinv_det_bwd.argtypes = [_D, _I64, _I64, _D, _D, _D, _D]
        lib.oracle_wishart_fwd.argtypes = [_D, _D, _I64, _I64, _I64, ctypes.c_int, _D, _D, _D]
        lib.oracle_wishart_bwd.argtypes = [_D, _D, _I64, _I64, _I64, ctypes.c_int, _D,
                                           ctypes.c_double, _D]
        lib.oracle_wishart_bwd_rows.argtypes = [_D, _D, _I64, _I64, _I64, ctypes.c_int, _D,
                                                ctypes.c_double, _I64, _I64, _D]
        lib.oracle_wishart_bwd_rows.restype = None
        lib.oracle_zinv_det_blockdiag.argtypes = [_D, ctypes.c_int, _I64, _I64, _D, _D, _D]
        lib.oracle_zinv_det_blockdiag.restype = None
        lib.oracle_pair_distance.argtypes = [_D, _D]
        lib.oracle_pair_distance.restype = ctypes.c_double
        lib.oracle_nlm_wishart.argtypes = [_D, _I64, _I64, ctypes.c_int, ctypes.c_double,
                                           ctypes.c_double, _D]
        lib.oracle_nlm_wishart.restype = None
        lib.oracle_stochastic_distance.argtypes = [_D, _D, ctypes.c_double, ctypes.c_int,
                                                   ctypes.c_double]
        lib.oracle_stochastic_distance.restype = ctypes.c_double
        lib.oracle_nlm_stochastic.argtypes = [_D, _I64, _I64, ctypes.c_int, ctypes.c_double,
                                              ctypes.c_double, ctypes.c_int, ctypes.c_double, _D]
        lib.oracle_nlm_stochastic.restype = None
        for f in ("oracle_zinv_det", "oracle_det_expansions", "oracle_inverse_full",
                  "oracle_eigvals", "oracle_multilook", "oracle_zinv_det_bwd",
                  "oracle_wishart_fwd", "oracle_wishart_bwd"):
            getattr(lib, f).restype = None
        self.lib = lib

    # -- per-pixel inverse and determinant (§2.1, §3.1) -------------------
    def zinv_det(self, z, with_imag: bool = False):
        """z: packed [9, n] (any float dtype). Returns (zinv [9, n], det [n]) in FP64."""
        z = _f64(z).reshape(9, -1)
        n = z.shape[1]
        zinv = np.empty((9, n))
        det = np.empty(n)
        det_im = np.empty(n) if with_imag else None
        self.lib.oracle_zinv_det(_ptr(z), n, n, _ptr(zinv), _ptr(det), _ptr(det_im))
        return (zinv, det, det_im) if with_imag else (zinv, det)

    def det_expansions(self, z) -> np.ndarray:
        """[6, n] complex: det along rows 0..2 then columns 0..2."""
        z = _f64(z).reshape(9, -1)
        n = z.shape[1]
        out = np.empty((12, n))
        self.lib.oracle_det_expansions(_ptr(z), n, n, _ptr(out))
        return out[0::2] + 1j * out[1::2]

    def inverse_full(self, z, method: str = "ge") -> np.ndarray:
        """[n, 3, 3] complex inverse; method 'ge' (Gauss-Jordan) or 'adj' (adj/det)."""
        z = _f64(z).reshape(9, -1)
        n = z.shape[1]
        out = np.empty((18, n))
        self.lib.oracle_inverse_full(_ptr(z), n, n, 1 if method == "adj" else 0, _ptr(out))
        c = out[0::2] + 1j * out[1::2]
        return c.T.reshape(n, 3, 3)

    def eigvals(self, z) -> np.ndarray:
        """[3, n] ascending eigenvalues."""
        z = _f64(z).reshape(9, -1)
        n = z.shape[1]
        lam = np.empty((3, n))
        self.lib.oracle_eigvals(_ptr(z), n, n, _ptr(lam))
        return lam

    def cond(self, z) -> np.ndarray:
        """cond_2 = lmax / lmin; inf where lmin <= 0 (not positive definite)."""
        lam = self.eigvals(z)
        with np.errstate(divide="ignore", invalid="ignore"):
            c = lam[2] / lam[0]
        c[~(lam[0] > 0)] = np.inf
        return c

    # -- multilook (Eq. ZN) ---------------------------------------------
    def multilook(self, s, win: int, weights=None) -> np.ndarray:
        """s: complex [3, H, W]. Returns packed Z [9, H*W] (boxcar mean if weights is None)."""
        buf, H, W = _slc_f64(s)
        w = None if weights is None else _f64(weights).reshape(-1)
        z = np.empty((9, H * W))
        self.lib.oracle_multilook(_ptr(buf), H, W, H * W, int(win), _ptr(w), _ptr(z))
        return z

    # -- backward of the per-pixel inverse / det --------------------------
    def zinv_det_bwd(self, z, g_zinv=None, g_det=None, g_logdet=None) -> np.ndarray:
        z = _f64(z).reshape(9, -1)
        n = z.shape[1]
        gz = None if g_zinv is None else _f64(g_zinv).reshape(9, n)
        gd = None if g_det is None else _f64(g_det).reshape(n)
        gl = None if g_logdet is None else _f64(g_logdet).reshape(n)
        out = np.empty((9, n))
        self.lib.oracle_zinv_det_bwd(_ptr(z), n, n, _ptr(gz), _ptr(gd), _ptr(gl), _ptr(out))
        return out

    # -- multifrequency block-diagonal pixels (§5) ------------------------
    def zinv_det_blockdiag(self, z, nb: int):
        """z: [nb, 9, n] packed blocks -> (zinv [nb, 9, n], det [n], off-block max [n])."""
        z = _f64(z).reshape(nb, 9, -1)
        n = z.shape[2]
        zinv = np.empty((nb, 9, n))
        det = np.empty(n)
        off = np.empty(n)
        self.lib.oracle_zinv_det_blockdiag(_ptr(z), int(nb), n, n, _ptr(zinv), _ptr(det), _ptr(off))
        return zinv, det, off

    # -- nonlocal means with the Wishart equal-looks distance (§1) --------
    def pair_distance(self, zi, zj) -> float:
        a, b = _f64(zi).reshape(9), _f64(zj).reshape(9)
        return float(self.lib.oracle_pair_distance(_ptr(a), _ptr(b)))

    def nlm_wishart(self, z, H: int, W: int, radius: int, looks: float, h: float) -> np.ndarray:
        """z: packed [9, H*W]; returns the filtered packed image [9, H*W]."""
        z = _f64(z).reshape(9, H * W)
        out = np.empty((9, H * W))
        self.lib.oracle_nlm_wishart(_ptr(z), H, W, int(radius), float(looks), float(h), _ptr(out))
        return out

    # -- stochastic distances between equal-looks Wishart laws (§1) ------
    BHATTACHARYYA, HELLINGER, KULLBACK_LEIBLER, RENYI = 0, 1, 2, 3

    def stochastic_distance(self, zi, zj, looks: float, dist: int, order: float = 0.5) -> float:
        a, b = _f64(zi).reshape(9), _f64(zj).reshape(9)
        return float(self.lib.oracle_stochastic_distance(_ptr(a), _ptr(b), float(looks),
                                                         int(dist), float(order)))

    def nlm_stochastic(self, z, H: int, W: int, radius: int, looks: float, h: float,
                       dist: int, order: float = 0.5) -> np.ndarray:
        """z: packed [9, H*W]; weights exp(-d / h) with the distance `dist`
        (`order`: the Renyi order in (0, 1))."""
        z = _f64(z).reshape(9, H * W)
        out = np.empty((9, H * W))
        self.lib.oracle_nlm_stochastic(_ptr(z), H, W, int(radius), float(looks), float(h),
                                       int(dist), float(order), _ptr(out))
        return out

    # -- Wishart change statistic ----------------------------------------
    def wishart_fwd(self, s1, s2, win: int, weights, want_map: bool = False):
        b1, H, W = _slc_f64(s1)
        b2, H2, W2 = _slc_f64(s2)
        assert (H, W) == (H2, W2)
        w = _f64(weights).reshape(-1)
        assert w.size == win * win
        q = np.empty(H * W) if want_map else None
        loss = np.zeros(1)
        self.lib.oracle_wishart_fwd(_ptr(b1), _ptr(b2), H, W, H * W, int(win), _ptr(w),
                                    _ptr(q), _ptr(loss))
        return (float(loss[0]), q) if want_map else float(loss[0])

    def wishart_bwd(self, s1, s2, win: int, weights, g: float = 1.0, rows=None) -> np.ndarray:
        """g dL/dw; rows=(y_lo, y_hi) sums over those output rows only."""
        b1, H, W = _slc_f64(s1)
        b2, _, _ = _slc_f64(s2)
        w = _f64(weights).reshape(-1)
        out = np.empty(win * win)
        if rows is None:
            self.lib.oracle_wishart_bwd(_ptr(b1), _ptr(b2), H, W, H * W, int(win), _ptr(w),
                                        float(g), _ptr(out))
        else:
            self.lib.oracle_wishart_bwd_rows(_ptr(b1), _ptr(b2), H, W, H * W, int(win), _ptr(w),
                                             float(g), int(rows[0]), int(rows[1]), _ptr(out))
        return out


def load(mutant: int = 0) -> Oracle:
    """Builds (if stale) and loads the oracle; mutant > 0 loads a planted-mistake build."""
    global _default
    with _lock:
        if mutant == 0 and _default is not None:
            return _default
        o = Oracle(compile_oracle(mutant=mutant))
        if mutant == 0:
            _default = o
        return o
