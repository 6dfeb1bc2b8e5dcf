"""The seeded input generators (CPU twin): published known answers, accuracy of the
deterministic elementary functions, index-addressable reproducibility, and the
distributions the workloads promise."""
import numpy as np
import pytest

from helpers import unpack

from paper_1807_08084_gb300 import synth as S


def test_philox_known_answers():
    # Random123 known-answer vectors for philox4x32, 10 rounds (Salmon et al. 2011)
    cases = [
        ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
        ((0xFFFFFFFF,) * 4, (0xFFFFFFFF, 0xFFFFFFFF),
         (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
        ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
         (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
    ]
    for ctr, key, want in cases:
        got = S.philox4x32_10(*[np.uint64(c) for c in ctr], *key)
        assert tuple(int(g) for g in got) == want


def test_elementary_functions():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.uniform(1e-300, 1, 10000), rng.uniform(1, 1e6, 10000),
                        [2.0 ** -53, 1.0, 0.5, 2.0]])
    assert np.max(np.abs(S.dlog(x) - np.log(x)) / np.maximum(1, np.abs(np.log(x)))) < 1e-15
    y = rng.uniform(-40, 40, 10000)
    assert np.max(np.abs(S.dexp(y) - np.exp(y)) / np.exp(y)) < 1e-14
    u = np.concatenate([rng.uniform(0, 1, 10000), [1.0, 0.25, 0.5, 0.75, 2.0 ** -53]])
    s, c = S.dsincos_2pi(u)
    assert np.max(np.abs(s - np.sin(2 * np.pi * u))) < 1e-14
    assert np.max(np.abs(c - np.cos(2 * np.pi * u))) < 1e-14
    assert np.max(np.abs(s * s + c * c - 1)) < 1e-14


def test_uniforms_in_range_and_moments():
    st = S.Stream(1, S.TAG_GRAD, np.arange(200000, dtype=np.uint64))
    u = np.concatenate([st.u(0), st.u(1)])
    assert u.min() > 0 and u.max() <= 1
    assert abs(u.mean() - 0.5) < 3e-3 and abs(u.var() - 1 / 12) < 2e-3
    re, im = S.cnormal(st.u(0), st.u(1))
    assert abs(re.var() - 0.5) < 1e-2 and abs(im.var() - 0.5) < 1e-2
    assert abs(np.mean(re * im)) < 1e-2


@pytest.mark.parametrize("name", ["plain_256", "scale_16k", "precision_4k", "paper_sim"])
def test_pixels_are_index_addressable(name):
    """Any subset of pixels regenerates bit-identically (counter-based generator)."""
    w = S.WORKLOADS[name]
    idx = np.arange(1000, 1500, dtype=np.uint64)
    full = w.packed_z(idx)
    sub = np.array([3, 77, 499], dtype=np.uint64)
    np.testing.assert_array_equal(w.packed_z(idx[sub]), full[:, sub])
    assert full.dtype == np.float32 and full.shape == (9, 500)


def test_wishart_mean_is_sigma():
    w = S.WORKLOADS["plain_256"]
    Z = unpack(w.packed_z())
    se = 1 / np.sqrt(w.N * Z.shape[0])
    assert np.abs(Z.mean(axis=0) - S.SIGMA_FIXED).max() < 6 * se
    # the per-pixel law has N looks: the diagonal's relative variance is 1/N
    a = Z[:, 0, 0].real
    assert abs(a.var() / a.mean() ** 2 - 1 / w.N) < 0.02


def test_class_covariances_and_maps():
    w = S.WORKLOADS["scale_16k"]
    F, lam = S.class_factors(w.seed)
    assert F.shape == (8, 3, 3)
    assert lam.min() >= 0.01 and lam.max() <= 10
    for c in range(8):
        Sg = F[c] @ F[c].conj().T
        np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(Sg)), np.sort(lam[c]), rtol=1e-12)
    bm = w.block_map()
    assert bm.shape == (32 * 32,) and set(np.unique(bm)) <= set(range(8))
    p = S.WORKLOADS["wishart_pair_4k"]
    b0, b1 = p.block_map(0), p.block_map(1)
    assert b0.size == 256 and np.sum(b0 != b1) == 77


def test_cond_workload_spans_range():
    w = S.WORKLOADS["precision_4k"]
    Z = unpack(w.packed_z(np.arange(20000, dtype=np.uint64)))
    lam = np.linalg.eigvalsh(Z)
    cond = lam[:, 2] / lam[:, 0]
    ok = lam[:, 0] > 0
    assert np.percentile(cond[ok], 5) < 3 and np.percentile(cond[ok], 95) > 1e6
    assert np.all(np.abs(lam[:, 2] - 1) < 1e-5)   # largest eigenvalue is 1


def test_slc_has_class_covariance():
    w = S.scaled(S.WORKLOADS["multilook_8k"], 256, 256)
    idx = np.arange(w.n, dtype=np.uint64)
    s = w.looks(idx).astype(np.complex128)
    cls = w.classes(idx)
    F = w.factors()
    c = np.bincount(cls).argmax()
    v = s[:, cls == c]
    emp = v @ v.conj().T / v.shape[1]
    Sg = F[c] @ F[c].conj().T
    assert np.abs(emp - Sg).max() < 0.05 * np.abs(Sg).max()
