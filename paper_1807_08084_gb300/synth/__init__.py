"""Seeded synthetic PolSAR inputs, CPU twin (numpy).

This module generates the inputs that both the FP64 oracle and the CUDA path
consume.  It holds none of the method's arithmetic: no inverse, no determinant,
no cofactor and no window averaging.  The packed-Z workloads are drawn from the
complex Wishart law by the Bartlett decomposition (the law of an N-look sample
covariance, Eq. ZN of the paper, without forming the looks' outer products), or
as U diag(lambda) U^H with a Haar-random unitary U, or as R R^H with uniform R
(the paper's simulated data, §4.2.1).

Bit-identical twin.  ``synth.cu`` computes the same values on the GPU.  Both
sides use

* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
  as 1, 2, 3", SC 2011), counter = (pixel index lo, hi, draw, stream), key =
  (seed, tag), so any pixel can be regenerated alone;
* 53-bit uniforms u = (k + 1) 2^-53 in (0, 1];
* their own log, exp and sin/cos written from series (atanh series for log,
  Taylor series for exp and sin/cos) using only IEEE +, -, *, / and sqrt, which
  are correctly rounded on both sides, evaluated in the same order (the CUDA
  file is compiled with -fmad=false so nothing is fused);
* FP64 throughout, rounded to FP32 (round-to-nearest-even) at the end.

Layouts match the library: packed Z is float32 [9, n] in plane order
a, Re b, Im b, Re c, Im c, d, Re e, Im e, f; single-look data is complex64
[3, H, W] (S_HH, S_HV, S_VV).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# --------------------------------------------------------------------------
# Philox4x32-10
# --------------------------------------------------------------------------
PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
_MASK32 = np.uint64(0xFFFFFFFF)

# tags (second key word): one independent stream family per use
TAG_Z_WISHART = 1
TAG_Z_COND = 2
TAG_Z_RRH = 3
TAG_SLC = 4
TAG_CLASS = 5
TAG_BLOCK_MAP = 6
TAG_CHANGE = 7
TAG_GRAD = 8


def philox4x32_10(c0, c1, c2, c3, k0: int, k1: int):
    """Philox4x32 with 10 rounds; counters are uint32-valued arrays, key two ints."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & _MASK32 for c in (c0, c1, c2, c3))
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    k0 = int(k0) & 0xFFFFFFFF
    k1 = int(k1) & 0xFFFFFFFF
    for r in range(10):
        if r:
            k0 = (k0 + PHILOX_W0) & 0xFFFFFFFF
            k1 = (k1 + PHILOX_W1) & 0xFFFFFFFF
        p0 = PHILOX_M0 * c0
        p1 = PHILOX_M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(k0), lo1, hi0 ^ c3 ^ np.uint64(k1), lo0)
    return c0, c1, c2, c3


def _u53(a, b):
    """Two uint32 words -> uniform double (k + 1) * 2^-53 in (0, 1]."""
    k = ((a >> np.uint64(5)) << np.uint64(26)) | (b >> np.uint64(6))
    return (k + np.uint64(1)).astype(np.float64) * 2.0 ** -53


class Stream:
    """Uniform draws u_0, u_1, ... for a vector of pixel indices.

    Call d of Philox yields u_{2d} (words 0, 1) and u_{2d+1} (words 2, 3).
    """

    def __init__(self, seed: int, tag: int, idx, stream: int = 0):
        self.seed = int(seed)
        self.tag = int(tag)
        self.idx = np.asarray(idx, dtype=np.uint64)
        self.stream = int(stream)
        self._cache: dict[int, tuple[np.ndarray, np.ndarray]] = {}

    def u(self, j: int) -> np.ndarray:
        d = j // 2
        if d not in self._cache:
            lo = self.idx & _MASK32
            hi = self.idx >> np.uint64(32)
            w = philox4x32_10(lo, hi, d, self.stream, self.seed, self.tag)
            self._cache = {d: (_u53(w[0], w[1]), _u53(w[2], w[3]))}
        return self._cache[d][j % 2]


# --------------------------------------------------------------------------
# Deterministic elementary functions (IEEE +, -, *, / and sqrt only)
# --------------------------------------------------------------------------
LN2 = float.fromhex("0x1.62e42fefa39efp-1")
INV_LN2 = float.fromhex("0x1.71547652b82fep+0")
HALF_PI = float.fromhex("0x1.921fb54442d18p+0")
SQRT_HALF = float.fromhex("0x1.6a09e667f3bcdp-1")
# 1/(2k+1), k = 0..12 (atanh series of log)
LOG_C = [float.fromhex(h) for h in (
    "0x1.0000000000000p+0", "0x1.5555555555555p-2", "0x1.999999999999ap-3",
    "0x1.2492492492492p-3", "0x1.c71c71c71c71cp-4", "0x1.745d1745d1746p-4",
    "0x1.3b13b13b13b14p-4", "0x1.1111111111111p-4", "0x1.e1e1e1e1e1e1ep-5",
    "0x1.af286bca1af28p-5", "0x1.8618618618618p-5", "0x1.642c8590b2164p-5",
    "0x1.47ae147ae147bp-5")]
# 1/k!, k = 0..23 (Taylor series of exp, sin, cos)
INV_FACT = [float.fromhex(h) for h in (
    "0x1.0000000000000p+0", "0x1.0000000000000p+0", "0x1.0000000000000p-1",
    "0x1.5555555555555p-3", "0x1.5555555555555p-5", "0x1.1111111111111p-7",
    "0x1.6c16c16c16c17p-10", "0x1.a01a01a01a01ap-13", "0x1.a01a01a01a01ap-16",
    "0x1.71de3a556c734p-19", "0x1.27e4fb7789f5cp-22", "0x1.ae64567f544e4p-26",
    "0x1.1eed8eff8d898p-29", "0x1.6124613a86d09p-33", "0x1.93974a8c07c9dp-37",
    "0x1.ae7f3e733b81fp-41", "0x1.ae7f3e733b81fp-45", "0x1.952c77030ad4ap-49",
    "0x1.6827863b97d97p-53", "0x1.2f49b46814157p-57", "0x1.e542ba4020225p-62",
    "0x1.71b8ef6dcf572p-66", "0x1.0ce396db7f853p-70", "0x1.761b413163819p-75")]


def dlog(x):
    """Natural log of positive finite x: x = m 2^e, log m = 2 atanh((m-1)/(m+1))."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)
    small = m < SQRT_HALF
    m = np.where(small, m * 2.0, m)
    e = np.where(small, e - 1, e).astype(np.float64)
    z = (m - 1.0) / (m + 1.0)
    z2 = z * z
    p = np.full_like(z, LOG_C[12])
    for k in range(11, -1, -1):
        p = p * z2 + LOG_C[k]
    return e * LN2 + (2.0 * z) * p


def dexp(x):
    """exp(x) = 2^k exp(r), k = rint(x / ln 2), Taylor series of exp(r) to r^17."""
    x = np.asarray(x, dtype=np.float64)
    k = np.rint(x * INV_LN2)
    r = x - k * LN2
    p = np.full_like(r, INV_FACT[17])
    for j in range(16, -1, -1):
        p = p * r + INV_FACT[j]
    return np.ldexp(p, k.astype(np.int32))


def dsincos_2pi(u):
    """(sin, cos) of 2 pi u for u in (0, 1], by quadrant and Taylor series."""
    u = np.asarray(u, dtype=np.float64)
    v = u * 4.0
    q = np.floor(v)
    f = v - q
    th = f * HALF_PI
    t2 = th * th
    s = np.full_like(th, -INV_FACT[23])
    for j in range(21, 0, -2):  # odd powers: sign (-1)^((j-1)/2)
        s = s * t2 + (INV_FACT[j] if ((j - 1) // 2) % 2 == 0 else -INV_FACT[j])
    s = s * th
    c = np.full_like(th, -INV_FACT[22])
    for j in range(20, -1, -2):
        c = c * t2 + (INV_FACT[j] if (j // 2) % 2 == 0 else -INV_FACT[j])
    qi = q.astype(np.int64) % 4
    sin = np.select([qi == 0, qi == 1, qi == 2], [s, c, -s], -c)
    cos = np.select([qi == 0, qi == 1, qi == 2], [c, -s, -c], s)
    return sin, cos


def cnormal(u1, u2):
    """Circular complex Gaussian CN(0, 1) (Re, Im ~ N(0, 1/2)) by Box-Muller."""
    r = np.sqrt(-dlog(u1))
    s, c = dsincos_2pi(u2)
    return r * c, r * s


# --------------------------------------------------------------------------
# Small complex helpers on (re, im) pairs, fixed evaluation order
# --------------------------------------------------------------------------
def _cmul(ar, ai, br, bi):
    return ar * br - ai * bi, ar * bi + ai * br


def _cmulc(ar, ai, br, bi):
    """a * conj(b)."""
    return ar * br + ai * bi, ai * br - ar * bi


def gram_schmidt(vr, vi):
    """Haar unitary from three complex Gaussian columns (modified Gram-Schmidt).

    vr, vi: lists [row][col] of arrays.  Returns (qr, qi) in the same layout.
    """
    qr = [[None] * 3 for _ in range(3)]
    qi = [[None] * 3 for _ in range(3)]
    wr = [[vr[i][j] for j in range(3)] for i in range(3)]
    wi = [[vi[i][j] for j in range(3)] for i in range(3)]
    for j in range(3):
        nrm2 = (wr[0][j] * wr[0][j] + wi[0][j] * wi[0][j]) \
            + (wr[1][j] * wr[1][j] + wi[1][j] * wi[1][j]) \
            + (wr[2][j] * wr[2][j] + wi[2][j] * wi[2][j])
        nrm = np.sqrt(nrm2)
        for i in range(3):
            qr[i][j] = wr[i][j] / nrm
            qi[i][j] = wi[i][j] / nrm
        for k in range(j + 1, 3):
            # p = q_j^H w_k
            pr = (qr[0][j] * wr[0][k] + qi[0][j] * wi[0][k]) \
                + (qr[1][j] * wr[1][k] + qi[1][j] * wi[1][k]) \
                + (qr[2][j] * wr[2][k] + qi[2][j] * wi[2][k])
            pi = (qr[0][j] * wi[0][k] - qi[0][j] * wr[0][k]) \
                + (qr[1][j] * wi[1][k] - qi[1][j] * wr[1][k]) \
                + (qr[2][j] * wi[2][k] - qi[2][j] * wr[2][k])
            for i in range(3):
                tr, ti = _cmul(pr, pi, qr[i][j], qi[i][j])
                wr[i][k] = wr[i][k] - tr
                wi[i][k] = wi[i][k] - ti
    return qr, qi


def _pack32(zr, zi):
    """Upper triangle of a Hermitian 3x3 (lists of arrays) -> float32 [9, n]."""
    planes = [zr[0][0], zr[0][1], zi[0][1], zr[0][2], zi[0][2], zr[1][1], zr[1][2], zi[1][2],
              zr[2][2]]
    return np.stack([np.asarray(p, dtype=np.float64) for p in planes]).astype(np.float32)


def _sandwich(Fr, Fi, Br, Bi):
    """Upper triangle of F B F^H for 3x3 complex F (per-pixel arrays or scalars), B Hermitian."""
    Cr = [[None] * 3 for _ in range(3)]
    Ci = [[None] * 3 for _ in range(3)]
    for i in range(3):
        for j in range(3):
            sr, si = _cmul(Fr[i][0], Fi[i][0], Br[0][j], Bi[0][j])
            for k in (1, 2):
                tr, ti = _cmul(Fr[i][k], Fi[i][k], Br[k][j], Bi[k][j])
                sr, si = sr + tr, si + ti
            Cr[i][j], Ci[i][j] = sr, si
    Zr = [[None] * 3 for _ in range(3)]
    Zi = [[None] * 3 for _ in range(3)]
    for i in range(3):
        for j in range(i, 3):
            sr, si = _cmulc(Cr[i][0], Ci[i][0], Fr[j][0], Fi[j][0])
            for k in (1, 2):
                tr, ti = _cmulc(Cr[i][k], Ci[i][k], Fr[j][k], Fi[j][k])
                sr, si = sr + tr, si + ti
            Zr[i][j], Zi[i][j] = sr, si
    return Zr, Zi


# --------------------------------------------------------------------------
# Class covariances and maps (host-side tables, shared by both sides)
# --------------------------------------------------------------------------
def class_factors(seed: int, n_classes: int = 8, lam_lo: float = 0.01, lam_hi: float = 10.0):
    """F_c = U_c diag(sqrt(lambda_c)) with U_c Haar and lambda_c log-uniform in [lo, hi].

    Sigma_c = F_c F_c^H.  Returns (F [C, 3, 3] complex128, lam [C, 3]).
    """
    idx = np.arange(n_classes, dtype=np.uint64)
    st = Stream(seed, TAG_CLASS, idx)
    llo, lhi = float(dlog(lam_lo)), float(dlog(lam_hi))
    lam = np.stack([dexp(llo + st.u(k) * (lhi - llo)) for k in range(3)], axis=1)
    vr = [[None] * 3 for _ in range(3)]
    vi = [[None] * 3 for _ in range(3)]
    j = 3
    for col in range(3):
        for row in range(3):
            vr[row][col], vi[row][col] = cnormal(st.u(j), st.u(j + 1))
            j += 2
    qr, qi = gram_schmidt(vr, vi)
    F = np.empty((n_classes, 3, 3), dtype=np.complex128)
    for i in range(3):
        for k in range(3):
            sq = np.sqrt(lam[:, k])
            F[:, i, k] = qr[i][k] * sq + 1j * (qi[i][k] * sq)
    return F, lam


def cholesky_factor(S) -> np.ndarray:
    """Lower-triangular F with F F^H = S for one fixed Hermitian PD 3x3 (host table).

    Only used to draw CN(0, S) samples for the fixed-covariance workload.
    """
    S = np.asarray(S, dtype=np.complex128)
    L = np.zeros((3, 3), dtype=np.complex128)
    for j in range(3):
        acc = S[j, j].real - sum(abs(L[j, k]) ** 2 for k in range(j))
        L[j, j] = np.sqrt(acc)
        for i in range(j + 1, 3):
            L[i, j] = (S[i, j] - sum(L[i, k] * np.conj(L[j, k]) for k in range(j))) / L[j, j]
    return L


def block_classes(seed: int, n_blocks: int, n_classes: int = 8) -> np.ndarray:
    """Class index of each image block: Philox word mod n_classes."""
    w = philox4x32_10(np.arange(n_blocks, dtype=np.uint64), 0, 0, 0, seed, TAG_BLOCK_MAP)
    return (w[0] % np.uint64(n_classes)).astype(np.int32)


def changed_block_classes(seed: int, cls: np.ndarray, n_changed: int,
                          n_classes: int = 8) -> np.ndarray:
    """Second-date classes: the n_changed blocks with the smallest Philox keys switch
    to a different class (old + 1 + word mod (C - 1)) mod C."""
    nb = cls.size
    w = philox4x32_10(np.arange(nb, dtype=np.uint64), 0, 0, 0, seed, TAG_CHANGE)
    order = np.argsort(w[0].astype(np.int64), kind="stable")
    out = cls.copy()
    ch = order[:n_changed]
    step = 1 + (w[1][ch] % np.uint64(n_classes - 1)).astype(np.int32)
    out[ch] = (cls[ch] + step) % n_classes
    return out


def pixel_class(idx, W: int, block: int, block_cls: np.ndarray) -> np.ndarray:
    idx = np.asarray(idx, dtype=np.int64)
    y, x = idx // W, idx % W
    bx = (W + block - 1) // block
    return block_cls[(y // block) * bx + (x // block)]


# --------------------------------------------------------------------------
# Per-pixel generators (any subset of pixel indices)
# --------------------------------------------------------------------------
def _split_F(F):
    F = np.asarray(F)
    return ([[F[..., i, j].real for j in range(3)] for i in range(3)],
            [[F[..., i, j].imag for j in range(3)] for i in range(3)])


def z_wishart(seed: int, idx, N: int, F, cls=None) -> np.ndarray:
    """Packed Z ~ W_C(N, Sigma)/N with Sigma = F F^H, by the Bartlett decomposition.

    W_C(N, I) = T T^H, T lower triangular, T_ii^2 ~ Gamma(N - i, 1) (i = 0, 1, 2),
    T_ij ~ CN(0, 1) below the diagonal.  Gamma(k, 1) = -log(u_1 ... u_k).
    F: [3, 3] or [C, 3, 3] with cls the class index per pixel.
    Uniform draws per pixel: 3N - 3 for the gammas, then 6 for T_10, T_20, T_21.
    """
    idx = np.asarray(idx, dtype=np.uint64)
    st = Stream(seed, TAG_Z_WISHART, idx)
    j = 0
    Td = []
    for i in range(3):
        prod = np.ones(idx.shape)
        for _ in range(N - i):
            prod = prod * st.u(j)
            j += 1
        Td.append(np.sqrt(-dlog(prod)))
    off = []
    for _ in range(3):
        off.append(cnormal(st.u(j), st.u(j + 1)))
        j += 2
    (t10r, t10i), (t20r, t20i), (t21r, t21i) = off
    zero = np.zeros(idx.shape)
    # B = T T^H (upper triangle and its mirror)
    Br = [[None] * 3 for _ in range(3)]
    Bi = [[None] * 3 for _ in range(3)]
    Br[0][0], Bi[0][0] = Td[0] * Td[0], zero
    Br[0][1], Bi[0][1] = Td[0] * t10r, -(Td[0] * t10i)
    Br[0][2], Bi[0][2] = Td[0] * t20r, -(Td[0] * t20i)
    Br[1][1], Bi[1][1] = (t10r * t10r + t10i * t10i) + Td[1] * Td[1], zero
    b12r, b12i = _cmulc(t10r, t10i, t20r, t20i)
    Br[1][2], Bi[1][2] = b12r + Td[1] * t21r, b12i - Td[1] * t21i
    Br[2][2], Bi[2][2] = ((t20r * t20r + t20i * t20i) + (t21r * t21r + t21i * t21i)) \
        + Td[2] * Td[2], zero
    for i in range(3):
        for k in range(i):
            Br[i][k], Bi[i][k] = Br[k][i], -Bi[k][i]
    F = np.asarray(F)
    if F.ndim == 3:
        F = F[np.asarray(cls)]
    Fr, Fi = _split_F(F)
    Zr, Zi = _sandwich(Fr, Fi, Br, Bi)
    invN = 1.0 / N
    Zr = [[None if Zr[i][k] is None else Zr[i][k] * invN for k in range(3)] for i in range(3)]
    Zi = [[None if Zi[i][k] is None else Zi[i][k] * invN for k in range(3)] for i in range(3)]
    return _pack32(Zr, Zi)


def z_cond(seed: int, idx, kappa_max: float = 1e7) -> np.ndarray:
    """Packed Z = U diag(1, kappa^-v, 1/kappa) U^H, kappa log-uniform in [1, kappa_max],
    v ~ U(0, 1], U Haar per pixel; computed in FP64 then rounded to FP32."""
    idx = np.asarray(idx, dtype=np.uint64)
    st = Stream(seed, TAG_Z_COND, idx)
    lnk = st.u(0) * float(dlog(kappa_max))
    kappa = dexp(lnk)
    lam = [np.ones(idx.shape), dexp(-(st.u(1) * lnk)), 1.0 / kappa]
    vr = [[None] * 3 for _ in range(3)]
    vi = [[None] * 3 for _ in range(3)]
    j = 2
    for col in range(3):
        for row in range(3):
            vr[row][col], vi[row][col] = cnormal(st.u(j), st.u(j + 1))
            j += 2
    qr, qi = gram_schmidt(vr, vi)
    Zr = [[None] * 3 for _ in range(3)]
    Zi = [[None] * 3 for _ in range(3)]
    for i in range(3):
        for k in range(i, 3):
            sr, si = _cmulc(qr[i][0], qi[i][0], qr[k][0], qi[k][0])
            sr, si = lam[0] * sr, lam[0] * si
            for m in (1, 2):
                tr, ti = _cmulc(qr[i][m], qi[i][m], qr[k][m], qi[k][m])
                sr, si = sr + lam[m] * tr, si + lam[m] * ti
            Zr[i][k], Zi[i][k] = sr, si
    return _pack32(Zr, Zi)


def z_rrh(seed: int, idx) -> np.ndarray:
    """Packed A = R R^H with Re, Im of R iid uniform on [-1, 1] (§4.2.1 of the paper)."""
    idx = np.asarray(idx, dtype=np.uint64)
    st = Stream(seed, TAG_Z_RRH, idx)
    Rr = [[None] * 3 for _ in range(3)]
    Ri = [[None] * 3 for _ in range(3)]
    j = 0
    for i in range(3):
        for k in range(3):
            Rr[i][k] = 2.0 * st.u(j) - 1.0
            Ri[i][k] = 2.0 * st.u(j + 1) - 1.0
            j += 2
    Zr = [[None] * 3 for _ in range(3)]
    Zi = [[None] * 3 for _ in range(3)]
    for i in range(3):
        for k in range(i, 3):
            sr, si = _cmulc(Rr[i][0], Ri[i][0], Rr[k][0], Ri[k][0])
            for m in (1, 2):
                tr, ti = _cmulc(Rr[i][m], Ri[i][m], Rr[k][m], Ri[k][m])
                sr, si = sr + tr, si + ti
            Zr[i][k], Zi[i][k] = sr, si
    return _pack32(Zr, Zi)


def slc(seed: int, idx, F, cls=None, date: int = 0) -> np.ndarray:
    """Single-look scattering vectors s = F g, g ~ CN(0, I_3): complex64 [3, len(idx)]."""
    idx = np.asarray(idx, dtype=np.uint64)
    st = Stream(seed, TAG_SLC, idx, stream=date)
    g = [cnormal(st.u(2 * i), st.u(2 * i + 1)) for i in range(3)]
    F = np.asarray(F)
    if F.ndim == 3:
        F = F[np.asarray(cls)]
    Fr, Fi = _split_F(F)
    out = np.empty((3, idx.size), dtype=np.complex64)
    for i in range(3):
        sr, si = _cmul(Fr[i][0], Fi[i][0], g[0][0], g[0][1])
        for k in (1, 2):
            tr, ti = _cmul(Fr[i][k], Fi[i][k], g[k][0], g[k][1])
            sr, si = sr + tr, si + ti
        out[i].real = np.asarray(sr, dtype=np.float64).astype(np.float32)
        out[i].imag = np.asarray(si, dtype=np.float64).astype(np.float32)
    return out


def uniform_f32(seed: int, idx, tag: int = TAG_GRAD, stream: int = 0, lo=-1.0, hi=1.0):
    """float32 uniforms on (lo, hi] per index (e.g. upstream gradients in tests)."""
    st = Stream(seed, tag, idx, stream=stream)
    return (lo + (hi - lo) * st.u(0)).astype(np.float32)


# --------------------------------------------------------------------------
# The synthetic workloads
# --------------------------------------------------------------------------
SEED_BASE = 18070808

# fixed covariance of the small plain workload
SIGMA_FIXED = np.array([[1.0, 0.3 + 0.1j, 0.5],
                        [0.3 - 0.1j, 0.4, 0.05j],
                        [0.5, -0.05j, 0.9]], dtype=np.complex128)


@dataclass
class Workload:
    name: str
    kind: str              # 'wishart' | 'cond' | 'rrh' | 'slc' | 'slc_pair'
    H: int
    W: int
    seed: int
    N: int = 0             # looks (packed-Z Wishart workloads)
    block: int = 0         # class block size (0: fixed covariance)
    n_classes: int = 8
    kappa_max: float = 1e7
    changed_fraction: float = 0.0
    windows: tuple = field(default_factory=tuple)

    @property
    def n(self) -> int:
        return self.H * self.W

    def factors(self):
        if self.block == 0:
            return cholesky_factor(SIGMA_FIXED)
        F, _ = class_factors(self.seed, self.n_classes)
        return F

    def block_map(self, date: int = 0) -> np.ndarray | None:
        if self.block == 0:
            return None
        nb = ((self.H + self.block - 1) // self.block) * ((self.W + self.block - 1) // self.block)
        cls = block_classes(self.seed, nb, self.n_classes)
        if date == 1:
            n_changed = int(round(self.changed_fraction * nb))
            cls = changed_block_classes(self.seed, cls, n_changed, self.n_classes)
        return cls

    def classes(self, idx, date: int = 0):
        bm = self.block_map(date)
        return None if bm is None else pixel_class(idx, self.W, self.block, bm)

    def packed_z(self, idx=None) -> np.ndarray:
        """float32 [9, len(idx)] (all pixels when idx is None)."""
        if idx is None:
            idx = np.arange(self.n, dtype=np.uint64)
        if self.kind == "wishart":
            return z_wishart(self.seed, idx, self.N, self.factors(), self.classes(idx))
        if self.kind == "cond":
            return z_cond(self.seed, idx, self.kappa_max)
        if self.kind == "rrh":
            return z_rrh(self.seed, idx)
        raise ValueError(self.kind)

    def looks(self, idx=None, date: int = 0) -> np.ndarray:
        """complex64 [3, len(idx)] single-look vectors of one date."""
        if idx is None:
            idx = np.arange(self.n, dtype=np.uint64)
        return slc(self.seed, idx, self.factors(), self.classes(idx, date), date)

    def image(self, date: int = 0) -> np.ndarray:
        """complex64 [3, H, W]."""
        return self.looks(None, date).reshape(3, self.H, self.W)


WORKLOADS = {
    # 256 x 256, N = 4 looks, fixed Sigma
    "plain_256": Workload("plain_256", "wishart", 256, 256, SEED_BASE + 1, N=4),
    # 16384 x 16384, N = 16 looks, 8 classes in 512 x 512 blocks
    "scale_16k": Workload("scale_16k", "wishart", 16384, 16384, SEED_BASE + 2, N=16, block=512),
    # 8192 x 8192 single-look, 8 classes in 256 x 256 blocks, windows 3/5/7
    "multilook_8k": Workload("multilook_8k", "slc", 8192, 8192, SEED_BASE + 3, block=256,
                             windows=(3, 5, 7)),
    # 4096 x 4096, cond log-uniform in [1, 1e7], Haar U per pixel
    "precision_4k": Workload("precision_4k", "cond", 4096, 4096, SEED_BASE + 4, kappa_max=1e7),
    # two dates of 4096 x 4096 single-look, 30% of 256 x 256 blocks change class
    "wishart_pair_4k": Workload("wishart_pair_4k", "slc_pair", 4096, 4096, SEED_BASE + 5,
                                block=256, changed_fraction=0.3, windows=(7,)),
    # the paper's simulated workload: 5,469,354 matrices A = R R^H
    "paper_sim": Workload("paper_sim", "rrh", 1, 5469354, SEED_BASE + 6),
    # shaped like the paper's AIRSAR scene (450 x 600), classes as scale_16k, N = 4
    "paper_meas_shaped": Workload("paper_meas_shaped", "wishart", 450, 600, SEED_BASE + 7, N=4,
                                  block=64),
}


def scaled(w: Workload, H: int, W: int, name: str | None = None) -> Workload:
    """Same generator and seed, another image size (small parity cases)."""
    from dataclasses import replace
    return replace(w, H=H, W=W, name=name or f"{w.name}@{H}x{W}")
