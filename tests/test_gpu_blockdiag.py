"""GPU parity of multifrequency block-diagonal pixels (zinv_det_blockdiag, §5)
against the oracle's Gauss-Jordan inverse of the full 3nb x 3nb matrix."""
import numpy as np
import pytest
import torch

from helpers import det_err, inv_err

from paper_1807_08084_gb300 import synth as S

pytestmark = pytest.mark.gpu


def bands(nb, n, seed=0):
    """nb bands of the class-covariance workload (different seeds per band)."""
    from dataclasses import replace
    w = S.WORKLOADS["scale_16k"]
    return np.stack([replace(w, seed=w.seed + 17 * b + seed).packed_z(np.arange(n, dtype=np.uint64))
                     for b in range(nb)])


@pytest.mark.parametrize("nb", [1, 2, 3, 8])
@pytest.mark.parametrize("n", [1, 5, 4099])
@pytest.mark.parametrize("flags", [0, 1, 2])
def test_blockdiag_vs_full_matrix_oracle(zlib, orc, nb, n, flags):
    z_np = bands(nb, n)
    z = torch.from_numpy(z_np).cuda()
    zinv, det, st = zlib.zinv_det_blockdiag(z, flags, want_status=True)
    torch.cuda.synchronize()
    ref_inv, ref_det, off = orc.zinv_det_blockdiag(z_np, nb)
    cond = np.max(np.stack([orc.cond(z_np[b]) for b in range(nb)]), axis=0)
    zi = zinv.cpu().numpy()
    for b in range(nb):
        assert np.all(inv_err(zi[b], ref_inv[b]) <= 1e-5 * cond)
    # det of the product: relative errors of the factors add up
    assert np.all(det_err(det.cpu().numpy(), ref_det) <= nb * 1e-5 * cond)
    assert not (st.cpu().numpy() & 1).any()


def test_blockdiag_one_block_equals_zinv_det(zlib):
    z_np = bands(1, 10001)
    z = torch.from_numpy(z_np).cuda()
    a_inv, a_det = zlib.zinv_det_blockdiag(z)
    b_inv, b_det = zlib.zinv_det(z[0])
    torch.cuda.synchronize()
    assert torch.equal(a_inv[0], b_inv) and torch.equal(a_det, b_det)


def test_blockdiag_flags_bad_block(zlib):
    z_np = bands(3, 64)
    z_np[1, :, 7] = 0.0  # band 1 of pixel 7 singular
    z = torch.from_numpy(z_np).cuda()
    _, det, st, cnt = zlib.zinv_det_blockdiag(z, 0, want_status=True, want_counts=True)
    torch.cuda.synchronize()
    s = st.cpu().numpy()
    assert (s[7] & 1) and int(cnt[0]) == 1 and int((s & 1).sum()) == 1


def test_blockdiag_full_size_sampled(zlib, orc):
    """Three bands of 8192 x 8192 pixels built as the benchmark builds them, in
    its launch configuration; 60k sampled pixels against the oracle's inverse of
    the full 9 x 9 matrix, on inputs regenerated by the numpy twin."""
    from dataclasses import replace
    from paper_1807_08084_gb300.synth import gpu as G
    wb = S.scaled(S.WORKLOADS["scale_16k"], 8192, 8192)
    ws = [replace(wb, seed=wb.seed + 17 * b) for b in range(3)]
    zb = torch.stack([G.packed_z(w) for w in ws])
    zinv, det = zlib.zinv_det_blockdiag(zb)
    torch.cuda.synchronize()
    rng = np.random.default_rng(17)
    idx = np.unique(np.concatenate([rng.integers(0, wb.n, 60000), [0, wb.n - 1]]))
    it = torch.from_numpy(idx).cuda()
    z_np = np.stack([w.packed_z(idx.astype(np.uint64)) for w in ws])
    np.testing.assert_array_equal(zb.reshape(3, 9, -1)[:, :, it].cpu().numpy(), z_np)
    ref_inv, ref_det, _ = orc.zinv_det_blockdiag(z_np, 3)
    cond = np.max(np.stack([orc.cond(z_np[b]) for b in range(3)]), axis=0)
    zi = zinv.reshape(3, 9, -1)[:, :, it].cpu().numpy()
    for b in range(3):
        assert np.all(inv_err(zi[b], ref_inv[b]) <= 1e-5 * cond)
    assert np.all(det_err(det.reshape(-1)[it].cpu().numpy(), ref_det) <= 3e-5 * cond)
