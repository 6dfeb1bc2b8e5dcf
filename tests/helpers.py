"""numpy helpers for the tests: packed <-> full Hermitian, error metrics."""
import numpy as np


def pack(A) -> np.ndarray:
    """[..., 3, 3] complex Hermitian -> packed [9, ...] (upper triangle, plane order
    a, Re b, Im b, Re c, Im c, d, Re e, Im e, f)."""
    A = np.asarray(A)
    return np.stack([A[..., 0, 0].real, A[..., 0, 1].real, A[..., 0, 1].imag,
                     A[..., 0, 2].real, A[..., 0, 2].imag, A[..., 1, 1].real,
                     A[..., 1, 2].real, A[..., 1, 2].imag, A[..., 2, 2].real])


def unpack(z) -> np.ndarray:
    """packed [9, n] -> [n, 3, 3] complex128 Hermitian."""
    z = np.asarray(z, dtype=np.float64).reshape(9, -1)
    n = z.shape[1]
    A = np.empty((n, 3, 3), dtype=np.complex128)
    A[:, 0, 0] = z[0]
    A[:, 0, 1] = z[1] + 1j * z[2]
    A[:, 0, 2] = z[3] + 1j * z[4]
    A[:, 1, 1] = z[5]
    A[:, 1, 2] = z[6] + 1j * z[7]
    A[:, 2, 2] = z[8]
    A[:, 1, 0] = np.conj(A[:, 0, 1])
    A[:, 2, 0] = np.conj(A[:, 0, 2])
    A[:, 2, 1] = np.conj(A[:, 1, 2])
    return A


def random_pd(rng, n: int, cond_max: float = 1e3) -> np.ndarray:
    """[n, 3, 3] Hermitian PD with log-uniform spectra (numpy's own generator)."""
    G = rng.standard_normal((n, 3, 3)) + 1j * rng.standard_normal((n, 3, 3))
    Q, R = np.linalg.qr(G)
    Q = Q * (np.diagonal(R, axis1=1, axis2=2) / np.abs(np.diagonal(R, axis1=1, axis2=2)))[:, None, :]
    lam = np.exp(rng.uniform(0, np.log(cond_max), (n, 3)))
    lam *= rng.uniform(0.1, 10, (n, 1))
    return (Q * lam[:, None, :]) @ np.conj(np.transpose(Q, (0, 2, 1)))


def inv_err(zinv_test, zinv_ref) -> np.ndarray:
    """Per-pixel max error of a packed inverse: diagonal |dW_ii| / W_ii, off-diagonal
    |dW_ij| / sqrt(W_ii W_jj) (|W_ij| <= sqrt(W_ii W_jj) for PD W)."""
    t = np.asarray(zinv_test, dtype=np.float64).reshape(9, -1)
    r = np.asarray(zinv_ref, dtype=np.float64).reshape(9, -1)
    d = np.abs(t - r)
    wa, wd, wf = r[0], r[5], r[8]
    e = np.stack([
        d[0] / wa, d[5] / wd, d[8] / wf,
        np.hypot(d[1], d[2]) / np.sqrt(wa * wd),
        np.hypot(d[3], d[4]) / np.sqrt(wa * wf),
        np.hypot(d[6], d[7]) / np.sqrt(wd * wf),
    ])
    return e.max(axis=0)


def det_err(det_test, det_ref) -> np.ndarray:
    r = np.asarray(det_ref, dtype=np.float64)
    return np.abs(np.asarray(det_test, dtype=np.float64) - r) / np.abs(r)
