"""Pins of the FP64 oracle to things other than itself (CPU only).

Each ``check_*`` takes an oracle build and raises AssertionError when it does
not agree with what the paper and the mathematics fix:

* exact rational arithmetic (sympy) on the fixed covariance of the plain
  workload;
* numpy.linalg (LAPACK: LU inverse, LU determinant, Hermitian eigenvalues) on
  random matrices, an independent library route;
* Z Z^-1 = I, a Hermitian inverse, a real positive determinant equal to the
  product of the eigenvalues, agreement of all row and column cofactor
  expansions (§3.1), det(Z^-1) = 1/det Z, Hadamard det <= a d f;
* the closed forms of diagonal, block-diagonal (§5) and scalar Z, and of
  U diag(l) U^H with known l;
* brute-force Python loops for the window covariance (Eq. ZN);
* central finite differences through numpy.linalg for the gradients;
* q <= 0, q(Z, Z) = 0, Euler homogeneity and date-swap symmetry for the Wishart
  change statistic;
* Monte Carlo estimates, from sampled complex Wishart matrices, of the integrals
  that define the Bhattacharyya, Kullback-Leibler and Renyi distances, and the
  closed forms, limits and invariances of those distances.

``test_mutants_are_caught`` builds the oracle with each planted mistake and
requires that at least one check fails for each.
"""
import itertools

import numpy as np
import pytest

from helpers import pack, random_pd, unpack

import oracle
from paper_1807_08084_gb300 import synth


# --------------------------------------------------------------------------
# the checks
# --------------------------------------------------------------------------
def check_sigma_exact(o):
    """Fixed Sigma of the plain workload vs exact rational arithmetic."""
    sympy = pytest.importorskip("sympy")
    R, Ii = sympy.Rational, sympy.I
    b = R(3, 10) + R(1, 10) * Ii
    c = R(1, 2)
    e = R(1, 20) * Ii
    S = sympy.Matrix([[1, b, c], [sympy.conjugate(b), R(2, 5), e],
                      [sympy.conjugate(c), sympy.conjugate(e), R(9, 10)]])
    det_exact = S.det()
    inv_exact = S.inv()
    assert det_exact == R(13, 80)
    z = pack(synth.SIGMA_FIXED[None])
    zinv, det, det_im = o.zinv_det(z, with_imag=True)
    assert abs(det[0] - 13 / 80) <= 1e-15 * 13 / 80 * 50
    assert abs(det_im[0]) <= 1e-16
    ref = pack(np.array(inv_exact.evalf(30).tolist(), dtype=np.complex128)[None])
    np.testing.assert_allclose(zinv[:, 0], ref[:, 0], rtol=0, atol=1e-13)
    lam = o.eigvals(z)[:, 0]
    # characteristic-polynomial invariants: trace, sum of principal 2x2 minors, det
    tr = float(sympy.re(S.trace()))
    m2 = float(sympy.re(sum(S.extract([i, j], [i, j]).det()
                           for i, j in itertools.combinations(range(3), 2))))
    assert abs(lam.sum() - tr) < 1e-13
    assert abs(lam[0] * lam[1] + lam[0] * lam[2] + lam[1] * lam[2] - m2) < 1e-13
    assert abs(lam.prod() - 13 / 80) < 1e-13


def check_random_vs_numpy(o):
    rng = np.random.default_rng(11)
    A = random_pd(rng, 2000, cond_max=1e4)
    z = pack(A)
    zinv, det = o.zinv_det(z)
    ref_inv = np.linalg.inv(A)
    ref_det = np.linalg.det(A).real
    lam_ref = np.linalg.eigvalsh(A)
    cond = lam_ref[:, 2] / lam_ref[:, 0]
    np.testing.assert_array_less(np.abs(det - ref_det) / ref_det, 1e-13 * cond)
    scale = np.abs(pack(ref_inv)).max(axis=0)
    np.testing.assert_array_less(np.abs(zinv - pack(ref_inv)).max(axis=0) / scale, 1e-13 * cond)
    lam = o.eigvals(z)
    np.testing.assert_array_less(np.abs(lam - lam_ref.T).max(axis=0) / lam_ref[:, 2], 1e-13)


def check_identity_and_hermitian(o):
    rng = np.random.default_rng(12)
    z = pack(random_pd(rng, 1000, cond_max=1e5))
    A = unpack(z)  # exactly Hermitian
    zinv, _ = o.zinv_det(z)
    W = unpack(zinv)
    lam = np.linalg.eigvalsh(A)
    cond = lam[:, 2] / lam[:, 0]
    err = np.abs(A @ W - np.eye(3)).max(axis=(1, 2))
    np.testing.assert_array_less(err, 1e-12 * cond)
    X = o.inverse_full(z, "ge")
    herm = np.abs(X - np.conj(np.transpose(X, (0, 2, 1)))).max(axis=(1, 2))
    np.testing.assert_array_less(herm / np.abs(X).max(axis=(1, 2)), 1e-13 * cond)
    # the packed output is the upper triangle of the full inverse
    np.testing.assert_allclose(pack(X), zinv, rtol=0, atol=0)
    # two derivations of the inverse agree (GE vs adj/det, Eq. inv_adjoint)
    Y = o.inverse_full(z, "adj")
    np.testing.assert_array_less(np.abs(X - Y).max(axis=(1, 2)) / np.abs(X).max(axis=(1, 2)),
                                 1e-13 * cond)


def check_det_properties(o):
    rng = np.random.default_rng(13)
    A = random_pd(rng, 1000, cond_max=1e3)
    z = pack(A)
    _, det, det_im = o.zinv_det(z, with_imag=True)
    assert np.all(det > 0)
    lam_np = np.linalg.eigvalsh(unpack(z))
    cond = lam_np[:, 2] / lam_np[:, 0]
    # det is real (§3.1): the imaginary part is rounding, relative to the terms' size
    np.testing.assert_array_less(np.abs(det_im) / det, 1e-14 * cond)
    ex = o.det_expansions(z)  # six expansions (§3.1: any row or column)
    np.testing.assert_array_less(np.abs(ex - det).max(axis=0) / det, 1e-13 * cond)
    lam = o.eigvals(z)
    np.testing.assert_array_less(np.abs(lam.prod(axis=0) - det) / det, 1e-13 * cond)
    # det(Z^-1) = 1 / det Z
    zinv, _ = o.zinv_det(z)
    dW = np.linalg.det(unpack(zinv)).real
    np.testing.assert_array_less(np.abs(dW * det - 1), 1e-13 * cond)
    # Hadamard: det <= a d f for PD
    assert np.all(det <= z[0] * z[5] * z[8] * (1 + 1e-14))


def check_closed_forms(o):
    rng = np.random.default_rng(14)
    n = 200
    # diagonal: W = diag(1/a, 1/d, 1/f), det = a d f
    a, d, f = (rng.uniform(0.01, 10, n) for _ in range(3))
    z = np.zeros((9, n))
    z[0], z[5], z[8] = a, d, f
    zinv, det = o.zinv_det(z)
    np.testing.assert_allclose(det, a * d * f, rtol=1e-15)
    np.testing.assert_allclose(zinv[[0, 5, 8]], np.stack([1 / a, 1 / d, 1 / f]), rtol=1e-15)
    assert np.all(zinv[[1, 2, 3, 4, 6, 7]] == 0)
    # block-diagonal (b = c = 0, §5): det = a (d f - |e|^2), blockwise inverse
    e = (rng.uniform(-1, 1, n) + 1j * rng.uniform(-1, 1, n)) * np.sqrt(d * f) * 0.9
    z = np.zeros((9, n))
    z[0], z[5], z[8], z[6], z[7] = a, d, f, e.real, e.imag
    zinv, det = o.zinv_det(z)
    m = d * f - np.abs(e) ** 2
    np.testing.assert_allclose(det, a * m, rtol=1e-12)
    np.testing.assert_allclose(zinv[0], 1 / a, rtol=1e-14)
    np.testing.assert_allclose(zinv[5], f / m, rtol=1e-11)
    np.testing.assert_allclose(zinv[8], d / m, rtol=1e-11)
    np.testing.assert_allclose(zinv[6] + 1j * zinv[7], -e / m, rtol=1e-11)
    assert np.all(np.abs(zinv[[1, 2, 3, 4]]) <= 1e-15 * np.abs(zinv[0]))
    # scalar c I
    c = rng.uniform(0.01, 100, n)
    z = np.zeros((9, n))
    z[0] = z[5] = z[8] = c
    zinv, det = o.zinv_det(z)
    np.testing.assert_allclose(det, c ** 3, rtol=1e-15)
    np.testing.assert_allclose(zinv[[0, 5, 8]], np.stack([1 / c] * 3), rtol=1e-15)
    # Z = U diag(l) U^H with known l: spectrum, det, cond, inverse
    G = rng.standard_normal((n, 3, 3)) + 1j * rng.standard_normal((n, 3, 3))
    U, _ = np.linalg.qr(G)
    lam = np.sort(np.exp(rng.uniform(np.log(1e-2), np.log(1e2), (n, 3))), axis=1)
    A = (U * lam[:, None, :]) @ np.conj(np.transpose(U, (0, 2, 1)))
    z = pack(A)
    np.testing.assert_allclose(o.eigvals(z), lam.T, rtol=1e-11)
    np.testing.assert_allclose(o.cond(z), lam[:, 2] / lam[:, 0], rtol=1e-10)
    zinv, det = o.zinv_det(z)
    np.testing.assert_allclose(det, lam.prod(axis=1), rtol=1e-11)
    Winv = (U / lam[:, None, :]) @ np.conj(np.transpose(U, (0, 2, 1)))
    np.testing.assert_allclose(zinv, pack(Winv), rtol=0, atol=1e-10 * np.abs(pack(Winv)).max())


def check_ill_conditioned_det(o):
    """Z = U diag(1, l, l) U^H with l down to 1e-7: the oracle's det and inverse
    against exact rational arithmetic on the very FP64 matrix it receives (two
    small eigenvalues are where a floating-point cofactor expansion breaks down)."""
    sympy = pytest.importorskip("sympy")
    rng = np.random.default_rng(18)
    n = 12
    G = rng.standard_normal((n, 3, 3)) + 1j * rng.standard_normal((n, 3, 3))
    U, _ = np.linalg.qr(G)
    lam = np.stack([np.ones(n), np.logspace(-1, -7, n), np.logspace(-1, -7, n) * 0.5], axis=1)
    z = pack((U * lam[:, None, :]) @ np.conj(np.transpose(U, (0, 2, 1))))
    zinv, det = o.zinv_det(z)
    A = unpack(z)
    for p in range(n):
        M = sympy.Matrix(3, 3, lambda i, j: sympy.Rational(float(A[p, i, j].real))
                         + sympy.I * sympy.Rational(float(A[p, i, j].imag)))
        d_exact = complex(sympy.N(M.det(), 30))
        assert abs(d_exact.imag) < 1e-30
        assert abs(det[p] - d_exact.real) <= 1e-7 * abs(d_exact.real), p
        Minv = M.inv()
        wa = float(sympy.re(sympy.N(Minv[0, 0], 30)))
        wb = complex(sympy.N(Minv[0, 1], 30))
        assert abs(zinv[0, p] - wa) <= 1e-6 * abs(wa), p
        assert abs(zinv[1, p] + 1j * zinv[2, p] - wb) <= 1e-6 * np.sqrt(abs(wa) * abs(
            float(sympy.re(sympy.N(Minv[1, 1], 30))))), p


def _brute_window(s, win, w):
    """Window covariance by explicit loops (clamp-to-edge addressing)."""
    _, H, W = s.shape
    r = (win - 1) // 2
    out = np.zeros((H * W, 3, 3), dtype=np.complex128)
    for y in range(H):
        for x in range(W):
            acc = np.zeros((3, 3), dtype=np.complex128)
            for dy in range(-r, r + 1):
                for dx in range(-r, r + 1):
                    yy = min(max(y + dy, 0), H - 1)
                    xx = min(max(x + dx, 0), W - 1)
                    v = s[:, yy, xx].astype(np.complex128)
                    wk = 1.0 / (win * win) if w is None else float(w[(dy + r) * win + dx + r])
                    for i in range(3):
                        for j in range(3):
                            acc[i, j] += wk * v[i] * np.conj(v[j])
            out[y * W + x] = acc
    return out


def check_multilook_brute(o):
    rng = np.random.default_rng(15)
    s = (rng.standard_normal((3, 6, 7)) + 1j * rng.standard_normal((3, 6, 7))).astype(np.complex64)
    for win in (1, 3, 5):
        ref = pack(_brute_window(s, win, None))
        np.testing.assert_allclose(o.multilook(s, win), ref, rtol=1e-13, atol=1e-14)
    w = rng.uniform(0.1, 1.0, 9).astype(np.float32)
    ref = pack(_brute_window(s, 3, w))
    np.testing.assert_allclose(o.multilook(s, 3, w), ref, rtol=1e-13, atol=1e-14)
    # a constant image gives the rank-one S S^H everywhere (boxcar mean, Eq. ZN)
    c = np.broadcast_to(s[:, :1, :1], s.shape).copy()
    v = s[:, 0, 0].astype(np.complex128)
    ref = pack(np.outer(v, np.conj(v))[None])
    np.testing.assert_allclose(o.multilook(c, 5), np.repeat(ref, 42, axis=1), rtol=1e-13,
                               atol=1e-14)


def _loss_numpy(z, gW, gdet, glog):
    A = unpack(z)
    W = pack(np.linalg.inv(A))
    det = np.linalg.det(A).real
    return np.sum(gW * W) + np.sum(gdet * det) + np.sum(glog * np.log(det))


def check_bwd_finite_differences(o):
    rng = np.random.default_rng(16)
    n = 40
    z = pack(random_pd(rng, n, cond_max=30))
    gW = rng.uniform(-1, 1, (9, n))
    gdet = rng.uniform(-1, 1, n)
    glog = rng.uniform(-1, 1, n)
    for args in ((gW, None, None), (None, gdet, None), (None, None, glog), (gW, gdet, glog)):
        g = o.zinv_det_bwd(z, *args)
        a = [np.zeros((9, n)) if args[0] is None else args[0],
             np.zeros(n) if args[1] is None else args[1],
             np.zeros(n) if args[2] is None else args[2]]
        fd = np.empty((9, n))
        for k in range(9):
            h = 1e-6 * np.abs(z).max(axis=0)
            for p in range(n):
                zp, zm = z.copy(), z.copy()
                zp[k, p] += h[p]
                zm[k, p] -= h[p]
                sel = (slice(None), slice(p, p + 1))
                fd[k, p] = (_loss_numpy(zp[sel], a[0][sel], a[1][p:p + 1], a[2][p:p + 1])
                            - _loss_numpy(zm[sel], a[0][sel], a[1][p:p + 1], a[2][p:p + 1])) / (2 * h[p])
        scale = np.abs(fd).max(axis=0) + 1e-30
        np.testing.assert_array_less(np.abs(g - fd).max(axis=0) / scale, 1e-6)


def _wishart_numpy(s1, s2, win, w):
    Z1 = _brute_window(s1, win, w)
    Z2 = _brute_window(s2, win, w)
    l1 = np.linalg.slogdet(Z1)[1]
    l2 = np.linalg.slogdet(Z2)[1]
    lm = np.linalg.slogdet((Z1 + Z2) / 2)[1]
    return l1 + l2 - 2 * lm


def check_wishart(o):
    rng = np.random.default_rng(17)
    H, W, win = 5, 6, 3
    s1 = (rng.standard_normal((3, H, W)) + 1j * rng.standard_normal((3, H, W))).astype(np.complex64)
    s2 = (rng.standard_normal((3, H, W)) + 1j * rng.standard_normal((3, H, W))).astype(np.complex64)
    w = rng.uniform(0.5, 1.5, win * win)
    loss, q = o.wishart_fwd(s1, s2, win, w, want_map=True)
    qref = _wishart_numpy(s1, s2, win, w)
    np.testing.assert_allclose(q, qref, rtol=1e-10, atol=1e-11)
    assert abs(loss - qref.sum()) < 1e-10 * max(1, abs(loss))
    assert np.all(q <= 1e-12)
    # no change: q = 0
    l0, q0 = o.wishart_fwd(s1, s1, win, w, want_map=True)
    assert np.all(np.abs(q0) < 1e-12)
    # swapping the dates leaves L and its gradient unchanged
    assert abs(o.wishart_fwd(s2, s1, win, w) - loss) < 1e-12 * abs(loss)
    g = o.wishart_bwd(s1, s2, win, w, 1.0)
    np.testing.assert_allclose(o.wishart_bwd(s2, s1, win, w, 1.0), g, rtol=1e-10, atol=1e-12)
    # Euler: L is homogeneous of degree 0 in w
    assert abs(np.dot(w, g)) < 1e-9 * np.abs(g).max() * np.abs(w).max()
    # central finite differences through numpy
    fd = np.empty(win * win)
    for k in range(win * win):
        h = 1e-6 * max(1.0, abs(w[k]))
        wp, wm = w.copy(), w.copy()
        wp[k] += h
        wm[k] -= h
        fd[k] = (_wishart_numpy(s1, s2, win, wp).sum() - _wishart_numpy(s1, s2, win, wm).sum()) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-6 * np.abs(fd).max())
    # upstream scalar
    np.testing.assert_allclose(o.wishart_bwd(s1, s2, win, w, -2.5), -2.5 * g, rtol=1e-14)


def check_blockdiag(o):
    """Block-diagonal multifrequency pixels (§5): the oracle's full-matrix GE
    against numpy.linalg on the assembled 3nb x 3nb matrix."""
    rng = np.random.default_rng(20)
    n, nb = 200, 3
    blocks = np.stack([pack(random_pd(rng, n, cond_max=1e3)) for _ in range(nb)])
    zinv, det, off = o.zinv_det_blockdiag(blocks, nb)
    full = np.zeros((n, 3 * nb, 3 * nb), dtype=np.complex128)
    for b in range(nb):
        full[:, 3 * b:3 * b + 3, 3 * b:3 * b + 3] = unpack(blocks[b])
    inv = np.linalg.inv(full)
    np.testing.assert_allclose(det, np.linalg.det(full).real, rtol=1e-10)
    for b in range(nb):
        ref = pack(inv[:, 3 * b:3 * b + 3, 3 * b:3 * b + 3])
        np.testing.assert_allclose(zinv[b], ref, rtol=0, atol=1e-9 * np.abs(ref).max())
    assert np.all(off <= 1e-12 * np.abs(zinv).max())
    # det of the whole = product of the blocks' dets (§5)
    prod = np.prod([np.linalg.det(unpack(blocks[b])).real for b in range(nb)], axis=0)
    np.testing.assert_allclose(det, prod, rtol=1e-10)


def check_nlm(o):
    from paper_1807_08084_gb300 import synth as S
    rng = np.random.default_rng(19)
    H, W, rad, L = 7, 9, 2, 4.0
    z = S.scaled(S.WORKLOADS["paper_meas_shaped"], H, W).packed_z().astype(np.float64)
    A = unpack(z)
    # distance: d >= 0, d(i, i) = 0, symmetric, against numpy slogdet
    for _ in range(20):
        i, j = rng.integers(0, H * W, 2)
        d = o.pair_distance(z[:, i], z[:, j])
        ref = (np.linalg.slogdet((A[i] + A[j]) / 2)[1]
               - 0.5 * (np.linalg.slogdet(A[i])[1] + np.linalg.slogdet(A[j])[1]))
        assert abs(d - ref) < 1e-12 and d >= -1e-14
        assert abs(o.pair_distance(z[:, j], z[:, i]) - d) < 1e-14
        assert abs(o.pair_distance(z[:, i], z[:, i])) < 1e-14
    # brute force with numpy on a tiny image
    out = o.nlm_wishart(z, H, W, rad, L, 0.7)
    ld = np.linalg.slogdet(A)[1]
    ref = np.empty_like(out)
    for y in range(H):
        for x in range(W):
            i = y * W + x
            acc, ws = np.zeros(9), 0.0
            for yy in range(max(0, y - rad), min(H, y + rad + 1)):
                for xx in range(max(0, x - rad), min(W, x + rad + 1)):
                    j = yy * W + xx
                    d = np.linalg.slogdet((A[i] + A[j]) / 2)[1] - 0.5 * (ld[i] + ld[j])
                    wgt = np.exp(-L * d / 0.7)
                    acc += wgt * z[:, j]
                    ws += wgt
            ref[:, i] = acc / ws
    np.testing.assert_allclose(out, ref, rtol=1e-11, atol=1e-13)
    # constant image: unchanged
    zc = np.repeat(z[:, :1], H * W, axis=1)
    np.testing.assert_allclose(o.nlm_wishart(zc, H, W, rad, L, 1.0), zc, rtol=1e-13)
    # h -> infinity: plain mean over the in-image search window
    big = o.nlm_wishart(z, H, W, rad, L, 1e30)
    zi = z.reshape(9, H, W)
    for (y, x) in [(0, 0), (3, 4), (6, 8)]:
        win = zi[:, max(0, y - rad):y + rad + 1, max(0, x - rad):x + rad + 1].reshape(9, -1)
        np.testing.assert_allclose(big[:, y * W + x], win.mean(axis=1), rtol=1e-12)
    # h -> 0: only the pixel itself keeps weight (distinct neighbours)
    np.testing.assert_allclose(o.nlm_wishart(z, H, W, rad, L, 1e-9), z, rtol=1e-12)


def _wishart_samples(rng, S, L, n):
    """n draws of Z = (1/L) sum_l s_l s_l^H, s_l ~ CN(0, S): the complex
    Wishart law W(S, L) of an L-look covariance (E[Z] = S)."""
    C = np.linalg.cholesky(S)
    g = (rng.standard_normal((n, L, 3)) + 1j * rng.standard_normal((n, L, 3))) / np.sqrt(2)
    s = g @ C.T                                   # rows s_l = C g_l
    return np.einsum("nli,nlj->nij", s, s.conj()) / L


def check_stochastic_distances(o):
    """Stochastic distances between equal-looks Wishart laws (§1's list), pinned
    to the density they are defined from and to the mathematics, not to their
    closed forms alone."""
    from paper_1807_08084_gb300 import synth as S
    B, HL, KL, RY = o.BHATTACHARYYA, o.HELLINGER, o.KULLBACK_LEIBLER, o.RENYI
    rng = np.random.default_rng(23)
    L = 4.0
    Z = pack(random_pd(rng, 40, cond_max=1e2))
    A = unpack(Z)

    def renyi_z_form(Si, Sj, b):
        """(D_b(i||j) + D_b(j||i)) / 2 through det((1-b) S_x + b S_y) (numpy)."""
        ldi, ldj = np.linalg.slogdet(Si)[1], np.linalg.slogdet(Sj)[1]
        dij = np.linalg.slogdet((1 - b) * Si + b * Sj)[1] - (1 - b) * ldi - b * ldj
        dji = np.linalg.slogdet((1 - b) * Sj + b * Si)[1] - (1 - b) * ldj - b * ldi
        return L / (1 - b) * 0.5 * (dij + dji)
    for k in range(0, 40, 2):
        zi, zj = Z[:, k], Z[:, k + 1]
        dB, dH, dK = (o.stochastic_distance(zi, zj, L, d) for d in (B, HL, KL))
        # Bhattacharyya through the inverses equals the log-det of the mean:
        # S_i^-1 + S_j^-1 = S_i^-1 (S_i + S_j) S_j^-1
        assert abs(dB - L * o.pair_distance(zi, zj)) < 1e-12 * max(1.0, dB)
        assert abs(dH - (1 - np.exp(-dB))) < 1e-14
        # symmetric, >= 0, zero on the diagonal
        for d, v in ((B, dB), (HL, dH), (KL, dK)):
            assert v > 0 and abs(o.stochastic_distance(zj, zi, L, d) - v) < 1e-12 * max(1.0, v)
            assert abs(o.stochastic_distance(zi, zi, L, d)) < 1e-12
        # invariant under a common congruence S -> T S T^H (T invertible, complex)
        T = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
        ti, tj = pack(T @ A[k] @ T.conj().T), pack(T @ A[k + 1] @ T.conj().T)
        for d, v in ((B, dB), (HL, dH), (KL, dK)):
            assert abs(o.stochastic_distance(ti, tj, L, d) - v) < 1e-8 * max(1.0, v)
        # Renyi: order 1/2 is twice Bhattacharyya, order -> 1 tends to KL, the
        # inverse form (the oracle) equals the Z form (numpy), symmetric,
        # invariant, zero on the diagonal
        assert abs(o.stochastic_distance(zi, zj, L, RY, 0.5) - 2 * dB) < 1e-11 * max(1.0, dB)
        # D_b = D_KL + c1 (1 - b) + c2 (1 - b)^2 + ...: one Richardson step
        # removes the linear term (c2 reaches ~5e7 for the most distant pair)
        ext = (2 * o.stochastic_distance(zi, zj, L, RY, 1 - 1e-7)
               - o.stochastic_distance(zi, zj, L, RY, 1 - 2e-7))
        assert abs(ext - dK) < 1e-6 * max(1.0, dK)
        for b in (0.2, 0.75):
            v = o.stochastic_distance(zi, zj, L, RY, b)
            assert v > 0 and abs(v - renyi_z_form(A[k], A[k + 1], b)) < 1e-10 * max(1.0, v)
            assert abs(o.stochastic_distance(zj, zi, L, RY, b) - v) < 1e-12 * max(1.0, v)
            assert abs(o.stochastic_distance(zi, zi, L, RY, b)) < 1e-12
            assert abs(o.stochastic_distance(ti, tj, L, RY, b) - v) < 1e-8 * max(1.0, v)
        # KL against numpy: traces of S_i^-1 S_j
        ref = L * (0.5 * (np.trace(np.linalg.solve(A[k], A[k + 1]))
                          + np.trace(np.linalg.solve(A[k + 1], A[k]))).real - 3)
        assert abs(dK - ref) < 1e-10 * max(1.0, ref)
    # closed forms: S_j = c S_i, and diagonal pairs (per-component sums)
    for c in (0.25, 0.9, 3.0):
        zi = Z[:, 0]
        dB = 3 * L * np.log((np.sqrt(c) + 1 / np.sqrt(c)) / 2)
        assert abs(o.stochastic_distance(zi, c * zi, L, B) - dB) < 1e-12
        assert abs(o.stochastic_distance(zi, c * zi, L, HL) - (1 - np.exp(-dB))) < 1e-12
        assert abs(o.stochastic_distance(zi, c * zi, L, KL) - 3 * L * ((c + 1 / c) / 2 - 1)) < 1e-12
        for b in (0.3, 0.75):
            dij = 3 * (np.log(1 - b + b * c) - b * np.log(c))
            dji = 3 * (np.log(1 - b + b / c) + b * np.log(c))
            assert abs(o.stochastic_distance(zi, c * zi, L, RY, b)
                       - L / (1 - b) * 0.5 * (dij + dji)) < 1e-12
    a, b = np.array([1.0, 0.3, 7.0]), np.array([2.0, 0.3, 0.5])
    za, zb = np.zeros(9), np.zeros(9)
    za[[0, 5, 8]], zb[[0, 5, 8]] = a, b
    assert abs(o.stochastic_distance(za, zb, L, KL) - L * ((a / b + b / a) / 2 - 1).sum()) < 1e-12
    assert abs(o.stochastic_distance(za, zb, L, B)
               - L * np.log((np.sqrt(a / b) + np.sqrt(b / a)) / 2).sum()) < 1e-12
    # Monte Carlo from the Wishart density: with Z ~ W(S_i, L),
    #   f_j / f_i (Z) = (det S_i / det S_j)^L exp(-L tr((S_j^-1 - S_i^-1) Z)),
    # E_i[sqrt(f_j / f_i)] = exp(-d_B) and E_i[ln(f_i / f_j)] = D(i || j).
    Li = 4
    Si = A[2]
    Sj = Si + 0.15 * np.diag(np.diag(Si).real) + 0.05 * A[3]
    zi, zj = pack(Si[None])[:, 0], pack(Sj[None])[:, 0]
    n = 200_000
    lr = {}
    for (P, Q), key in (((Si, Sj), "ij"), ((Sj, Si), "ji")):
        Zs = _wishart_samples(rng, P, Li, n)
        D = np.linalg.inv(Q) - np.linalg.inv(P)
        tr = np.einsum("ab,nba->n", D, Zs).real
        lr[key] = Li * (np.log(np.linalg.det(P).real / np.linalg.det(Q).real) - tr)  # ln f_Q/f_P
    bc = np.exp(0.5 * lr["ij"])
    d_mc = -np.log(bc.mean())
    se = bc.std() / np.sqrt(n) / bc.mean()
    assert abs(o.stochastic_distance(zi, zj, Li, B) - d_mc) < 5 * se + 1e-3 * d_mc
    kl = 0.5 * (np.mean(-lr["ij"]) + np.mean(-lr["ji"]))
    se_kl = 0.5 * (lr["ij"].std() + lr["ji"].std()) / np.sqrt(n)
    assert abs(o.stochastic_distance(zi, zj, Li, KL) - kl) < 5 * se_kl
    # Renyi: the integral of f_i^b f_j^(1-b) is E_i[(f_j / f_i)^(1-b)]
    b = 0.7
    ry, var = 0.0, 0.0
    for key in ("ij", "ji"):
        m = np.exp((1 - b) * lr[key])
        ry += 0.5 * np.log(m.mean()) / (b - 1)
        var += (0.5 / (1 - b) * m.std() / m.mean()) ** 2 / n
    assert abs(o.stochastic_distance(zi, zj, Li, RY, b) - ry) < 5 * np.sqrt(var) + 1e-3 * ry
    # the filters: Bhattacharyya weights are the log-det filter's; Hellinger
    # and Kullback-Leibler against a numpy brute force on a tiny image
    H, W, rad, h = 6, 7, 2, 0.8
    z = S.scaled(S.WORKLOADS["paper_meas_shaped"], H, W).packed_z().astype(np.float64)
    np.testing.assert_allclose(o.nlm_stochastic(z, H, W, rad, L, h, B),
                               o.nlm_wishart(z, H, W, rad, L, h), rtol=1e-11,
                               atol=1e-13 * np.abs(z).max())
    Az = unpack(z)
    inv = np.linalg.inv(Az)
    ld = np.linalg.slogdet(Az)[1]
    for dist in (HL, KL, RY):
        out = o.nlm_stochastic(z, H, W, rad, L, h, dist, 0.7)
        ref = np.empty_like(out)
        for y in range(H):
            for x in range(W):
                i = y * W + x
                acc, ws = np.zeros(9), 0.0
                for yy in range(max(0, y - rad), min(H, y + rad + 1)):
                    for xx in range(max(0, x - rad), min(W, x + rad + 1)):
                        j = yy * W + xx
                        if dist == KL:
                            d = L * (0.5 * np.trace(inv[i] @ Az[j] + inv[j] @ Az[i]).real - 3)
                        elif dist == RY:
                            d = renyi_z_form(Az[i], Az[j], 0.7)
                        else:
                            d = 1 - np.exp(-L * (np.linalg.slogdet((inv[i] + inv[j]) / 2)[1]
                                                 + 0.5 * (ld[i] + ld[j])))
                        wgt = np.exp(-d / h)
                        acc += wgt * z[:, j]
                        ws += wgt
                ref[:, i] = acc / ws
        np.testing.assert_allclose(out, ref, rtol=1e-11, atol=1e-13 * np.abs(z).max())


CHECKS = [check_sigma_exact, check_random_vs_numpy, check_identity_and_hermitian,
          check_det_properties, check_closed_forms, check_ill_conditioned_det,
          check_multilook_brute,
          check_bwd_finite_differences, check_wishart, check_nlm, check_blockdiag,
          check_stochastic_distances]


@pytest.mark.parametrize("check", CHECKS, ids=lambda c: c.__name__)
def test_oracle_pin(orc, check):
    check(orc)


# mutant id -> what it plants (see ORACLE_MUTANT in oracle.c)
MUTANTS = {
    1: "cofactor sign ignores the column",
    2: "lower triangle not conjugated on unpack",
    3: "packs the lower triangle of the inverse",
    4: "window covariance drops the conjugate",
    5: "wrong clamp bound at the bottom edge",
    6: "packed gradient drops the factor 2",
    7: "Wishart statistic drops the 1/2 in the pooled matrix",
    8: "Wishart gradient drops the factor 2 on W_12",
    9: "Jacobi rotation loses the sign of tau",
    10: "gradient sign of the W G W term",
    11: "elimination det ignores the permutation sign",
    12: "nonlocal means drops the 1/2 of the pair mean",
    13: "trace of a product takes the second factor untransposed",
    14: "Hellinger distance from the square root of the Bhattacharyya coefficient",
    15: "Renyi divergence weights both inverses by the order",
}


@pytest.mark.parametrize("mutant", sorted(MUTANTS), ids=lambda m: f"m{m}")
def test_mutants_are_caught(mutant):
    o = oracle.load(mutant=mutant)
    failed = []
    for check in CHECKS:
        try:
            with np.errstate(all="ignore"):
                check(o)
        except (AssertionError, FloatingPointError, ValueError):
            failed.append(check.__name__)
    assert failed, f"no pin catches mutant {mutant}: {MUTANTS[mutant]}"


def test_row_bands_reproduce_the_full_image_oracle(orc):
    """The banded evaluation the full-size GPU test uses (sub-images with r halo
    rows, cut at the border) gives the full-image oracle's loss and weight
    gradient: a halo or band-offset slip would change both."""
    from oracle_bands import wishart_by_bands
    from paper_1807_08084_gb300 import synth as S
    import tempfile
    import os
    w = S.scaled(S.WORKLOADS["wishart_pair_4k"], 37, 29)
    s1, s2 = w.image(0), w.image(1)
    wt = np.random.default_rng(4).uniform(0.5, 1.5, 25) / 25
    with tempfile.TemporaryDirectory() as d:
        p1, p2 = os.path.join(d, "a.npy"), os.path.join(d, "b.npy")
        np.save(p1, s1)
        np.save(p2, s2)
        loss, grad = wishart_by_bands(p1, p2, w.H, 5, wt, band_rows=6, processes=2)
    ref_loss = orc.wishart_fwd(s1, s2, 5, wt)
    ref_grad = orc.wishart_bwd(s1, s2, 5, wt, 1.0)
    assert abs(loss - ref_loss) <= 1e-12 * abs(ref_loss) * 37
    np.testing.assert_allclose(grad, ref_grad, rtol=1e-12, atol=1e-12 * np.abs(ref_grad).max())
