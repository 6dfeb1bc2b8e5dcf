"""GPU parity of the Wishart change statistic (wishart_stat_fwd / _bwd and the
WishartStat autograd Function) against the FP64 oracle, through the C ABI.

Per-pixel bound on q (first order).  The GPU forms Z_t in FP32: each entry is
an FMA chain of K = win^2 weighted products, so |dZ_ij| <= gamma_(K+1)
sum_k w_k |S_i S_j| <= gamma_(K+1) sqrt(Z_ii Z_jj) (Cauchy-Schwarz, w_k >= 0),
and Z1 + Z2 adds one rounding.  A perturbation dZ moves ln det Z by
tr(Z^-1 dZ), at most sum_ij |(Z^-1)_ij| |dZ_ij| = g * S(Z) with
    S(Z) = sum_ij |(Z^-1)_ij| sqrt(Z_ii Z_jj)
(the absolute entry sum of the inverse of Z's correlation form).  The
compensated log-dets add 4u each, logf one ulp of its result, and forming q
rounds it a few times.  So, with u = 2^-24 and l = ln det,
    |dq| <= gamma_(K+2) (S(Z1) + S(Z2) + 2 S(Z1 + Z2))
            + 16u + 4u (|l1| + |l2| + 2 |l12| + 6 ln 2),
computed per pixel from the oracle's FP64 window covariances; the tests allow
1.25 times that.  The loss must be within the sum of the per-pixel bounds.
"""
import numpy as np
import pytest
import torch

from paper_1807_08084_gb300 import synth as S

pytestmark = pytest.mark.gpu

G_REL = 1e-4     # weight gradient, relative to its largest component
U = 2.0 ** -24


def gamma(k):
    return k * U / (1 - k * U)


def q_bound(orc, s1, s2, win, wts):
    """[H*W] first-order bound on |q_gpu - q_oracle| (module docstring)."""
    K = win * win
    z1 = orc.multilook(s1, win, wts)
    z2 = orc.multilook(s2, win, wts)
    total = 16 * U + 4 * U * 6 * np.log(2)
    for z, mult in ((z1, 1.0), (z2, 1.0), (z1 + z2, 2.0)):
        inv, det = orc.zinv_det(z)
        d = np.sqrt(z[[0, 5, 8]])  # sqrt of the diagonal
        # sum_ij |W_ij| sqrt(Z_ii Z_jj): diagonal terms once, off-diagonal twice
        S = inv[0] * d[0] ** 2 + inv[5] * d[1] ** 2 + inv[8] * d[2] ** 2
        S = S + 2 * (np.hypot(inv[1], inv[2]) * d[0] * d[1] + np.hypot(inv[3], inv[4]) * d[0] * d[2]
                     + np.hypot(inv[6], inv[7]) * d[1] * d[2])
        total = total + mult * (gamma(K + 2) * S + 4 * U * np.abs(np.log(det)))
    return 1.25 * total


def pair(H, W, seed_shift=0):
    w = S.scaled(S.WORKLOADS["wishart_pair_4k"], H, W)
    return w, w.image(0), w.image(1)


def weights(win, seed=0):
    rng = np.random.default_rng(seed + win)
    return rng.uniform(0.5, 1.5, win * win).astype(np.float32) / (win * win)


@pytest.mark.parametrize("win", [3, 5, 7])
@pytest.mark.parametrize("shape", [(37, 70), (8, 64), (21, 5)])
def test_forward_and_backward_small(zlib, orc, win, shape):
    H, W = shape
    w, s1_np, s2_np = pair(H, W)
    wt = weights(win)
    s1, s2 = torch.from_numpy(s1_np).cuda(), torch.from_numpy(s2_np).cuda()
    wd = torch.from_numpy(wt).cuda()
    loss, q = zlib.wishart_stat_fwd(s1, s2, wd, win, want_map=True)
    g = zlib.wishart_stat_bwd(s1, s2, wd, win)
    torch.cuda.synchronize()
    ref_loss, ref_q = orc.wishart_fwd(s1_np, s2_np, win, wt, want_map=True)
    ref_g = orc.wishart_bwd(s1_np, s2_np, win, wt, 1.0)
    dq = np.abs(q.cpu().numpy().ravel() - ref_q)
    qb = q_bound(orc, s1_np, s2_np, win, wt)
    assert np.all(dq <= qb), f"max |dq|/bound {(dq / qb).max():.3f}"
    assert abs(float(loss) - ref_loss) <= qb.sum()
    np.testing.assert_allclose(float(loss), q.double().sum().item(), rtol=1e-12, atol=1e-9)
    gg = g.cpu().numpy().astype(np.float64)
    assert np.abs(gg - ref_g).max() <= G_REL * np.abs(ref_g).max(), (
        f"grad rel err {np.abs(gg - ref_g).max() / np.abs(ref_g).max():.3e}")
    # bit-exact repeat
    loss2 = zlib.wishart_stat_fwd(s1, s2, wd, win)
    g2 = zlib.wishart_stat_bwd(s1, s2, wd, win)
    torch.cuda.synchronize()
    assert float(loss2) == float(loss) and torch.equal(g2, g)


def test_no_change_gives_zero(zlib):
    w, s1_np, _ = pair(40, 90)
    s1 = torch.from_numpy(s1_np).cuda()
    wd = torch.from_numpy(weights(7)).cuda()
    loss, q = zlib.wishart_stat_fwd(s1, s1, wd, 7, want_map=True)
    torch.cuda.synchronize()
    assert q.abs().max().item() < 1e-5
    assert abs(float(loss)) < 1e-5 * q.numel()


def test_gradient_vs_fp64_finite_differences(zlib, orc):
    """64 x 64 crop: the GPU's analytic weight gradient against FP64 central
    differences of the oracle's forward."""
    w, s1_np, s2_np = pair(64, 64)
    wt = weights(7, seed=3).astype(np.float64)
    g = zlib.wishart_stat_bwd(torch.from_numpy(s1_np).cuda(), torch.from_numpy(s2_np).cuda(),
                              torch.from_numpy(wt.astype(np.float32)).cuda(), 7)
    torch.cuda.synchronize()
    w32 = wt.astype(np.float32).astype(np.float64)
    fd = np.empty(49)
    for k in range(49):
        h = 1e-5 * max(1.0, abs(w32[k]))
        wp, wm = w32.copy(), w32.copy()
        wp[k] += h
        wm[k] -= h
        fd[k] = (orc.wishart_fwd(s1_np, s2_np, 7, wp) - orc.wishart_fwd(s1_np, s2_np, 7, wm)) / (2 * h)
    gg = g.cpu().numpy().astype(np.float64)
    assert np.abs(gg - fd).max() <= G_REL * np.abs(fd).max(), (
        f"FD rel err {np.abs(gg - fd).max() / np.abs(fd).max():.3e}")


def test_invariants(zlib):
    """Euler (L homogeneous of degree 0 in w), date swap, upstream scaling, autograd."""
    import paper_1807_08084_gb300 as zp
    w, s1_np, s2_np = pair(96, 160)
    s1, s2 = torch.from_numpy(s1_np).cuda(), torch.from_numpy(s2_np).cuda()
    wd = torch.from_numpy(weights(7, seed=5)).cuda()
    g = zlib.wishart_stat_bwd(s1, s2, wd, 7)
    l12 = zlib.wishart_stat_fwd(s1, s2, wd, 7)
    l21 = zlib.wishart_stat_fwd(s2, s1, wd, 7)
    g21 = zlib.wishart_stat_bwd(s2, s1, wd, 7)
    g_scaled = zlib.wishart_stat_bwd(s1, s2, wd, 7, torch.tensor(-2.5, dtype=torch.float64))
    torch.cuda.synchronize()
    gd = g.double()
    assert abs(float((gd * wd.double()).sum())) <= 1e-4 * float(gd.abs().max() * wd.abs().max()) * 49
    assert abs(float(l12) - float(l21)) <= 1e-6 * abs(float(l12))
    assert torch.allclose(g, g21, rtol=1e-4, atol=1e-4 * float(g.abs().max()))
    assert torch.allclose(g_scaled, -2.5 * g, rtol=1e-6, atol=0)
    # scaling all weights leaves L unchanged (degree-0 homogeneity)
    l_scaled = zlib.wishart_stat_fwd(s1, s2, wd * 4.0, 7)
    torch.cuda.synchronize()
    assert abs(float(l_scaled) - float(l12)) <= 1e-5 * abs(float(l12))
    # autograd Function
    wp = wd.clone().requires_grad_()
    loss = zp.WishartStat.apply(s1, s2, wp, 7)
    (3.0 * loss).backward()
    torch.cuda.synchronize()
    assert torch.allclose(wp.grad, 3.0 * g, rtol=1e-6, atol=0)


def test_full_size_pair(zlib, orc):
    """Both 4096 x 4096 dates generated on the GPU; forward and backward in the
    benchmark's launch configuration.  Crops of the q map against the oracle,
    the loss as the sum of the q map, determinism, Euler invariant."""
    from paper_1807_08084_gb300.synth import gpu as G
    w = S.WORKLOADS["wishart_pair_4k"]
    s1, s2 = G.image(w, 0), G.image(w, 1)
    wd = torch.full((49,), 1 / 49, device="cuda")
    loss, q = zlib.wishart_stat_fwd(s1, s2, wd, 7, want_map=True)
    g = zlib.wishart_stat_bwd(s1, s2, wd, 7)
    loss_b = zlib.wishart_stat_fwd(s1, s2, wd, 7)
    g_b = zlib.wishart_stat_bwd(s1, s2, wd, 7)
    torch.cuda.synchronize()
    assert float(loss) == float(loss_b) and torch.equal(g, g_b)
    assert float(loss) <= 0
    np.testing.assert_allclose(float(loss), q.double().sum().item(), rtol=1e-9)
    gd = g.double()
    assert abs(float((gd * wd.double()).sum())) <= 1e-4 * float(gd.abs().max() * wd.abs().max()) * 49
    H, W = w.H, w.W
    rng = np.random.default_rng(10)
    wt = np.full(49, 1 / 49, dtype=np.float32)
    for (y0, x0) in [(0, 0), (H - 24, W - 24), (0, 2000)] + [tuple(rng.integers(10, 4000, 2)) for _ in range(3)]:
        y1, x1 = y0 + 24, x0 + 24
        cy0, cy1, cx0, cx1 = max(0, y0 - 3), min(H, y1 + 3), max(0, x0 - 3), min(W, x1 + 3)
        yy, xx = np.meshgrid(np.arange(cy0, cy1), np.arange(cx0, cx1), indexing="ij")
        idx = (yy * W + xx).ravel().astype(np.uint64)
        c1 = w.looks(idx, 0).reshape(3, cy1 - cy0, cx1 - cx0)
        c2 = w.looks(idx, 1).reshape(3, cy1 - cy0, cx1 - cx0)
        np.testing.assert_array_equal(s1[:, cy0:cy1, cx0:cx1].cpu().numpy(), c1)
        _, rq = orc.wishart_fwd(c1, c2, 7, wt, want_map=True)
        qb = q_bound(orc, c1, c2, 7, wt).reshape(cy1 - cy0, cx1 - cx0)
        sl = (slice(y0 - cy0, y1 - cy0), slice(x0 - cx0, x1 - cx0))
        rq = rq.reshape(cy1 - cy0, cx1 - cx0)[sl]
        gq = q[y0:y1, x0:x1].cpu().numpy()
        assert np.all(np.abs(gq - rq) <= qb[sl])


def test_full_size_gradient_and_loss_vs_oracle(zlib, tmp_path):
    """The 4096 x 4096 pair in the benchmark's launch configuration: the weight
    gradient after the 32,768-tile fixed-order reduction, and the loss, against
    the FP64 oracle over the full image (row bands on all host cores)."""
    from oracle_bands import wishart_by_bands
    from paper_1807_08084_gb300.synth import gpu as G
    w = S.WORKLOADS["wishart_pair_4k"]
    s1, s2 = G.image(w, 0), G.image(w, 1)
    wt = weights(7, seed=9)
    wd = torch.from_numpy(wt).cuda()
    loss = zlib.wishart_stat_fwd(s1, s2, wd, 7)
    g = zlib.wishart_stat_bwd(s1, s2, wd, 7)
    torch.cuda.synchronize()
    p1, p2 = tmp_path / "s1.npy", tmp_path / "s2.npy"
    np.save(p1, s1.cpu().numpy())
    np.save(p2, s2.cpu().numpy())
    del s1, s2
    ref_loss, ref_g = wishart_by_bands(str(p1), str(p2), w.H, 7, wt)
    gg = g.cpu().numpy().astype(np.float64)
    err = np.abs(gg - ref_g).max() / np.abs(ref_g).max()
    assert err <= G_REL, f"grad rel err {err:.3e}"
    # the loss within 2e-4 per pixel (the per-pixel bound is typically 1e-5..1e-4)
    assert abs(float(loss) - ref_loss) <= 2e-4 * w.H * w.W, (float(loss), ref_loss)


# ---------------------------------------------------------------------------
# saved window covariances (wishart_stat_fwd_save / wishart_stat_bwd_saved)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("win", [3, 5, 7])
@pytest.mark.parametrize("shape", [(70, 100), (37, 45)])  # 128-bit and 32-bit Z stores
def test_saved_z_matches_recompute_and_oracle(zlib, orc, win, shape):
    """The saved path gives the recomputing path's bits (loss, q map, weight
    gradient), and the saved Z is each date's window covariance: against the
    oracle within gamma_(K+3) sqrt(Z_ii Z_jj) per entry (K positive-weight
    terms of FP32 products; off-diagonal sums are bounded by Cauchy-Schwarz)."""
    H, W = shape
    _, c1, c2 = pair(H, W)
    s1, s2 = torch.from_numpy(c1).cuda(), torch.from_numpy(c2).cuda()
    wts = weights(win, 3)
    wd = torch.from_numpy(wts).cuda()
    loss, q = zlib.wishart_stat_fwd(s1, s2, wd, win, want_map=True)
    loss2, zs, q2 = zlib.wishart_stat_fwd_save(s1, s2, wd, win, want_map=True)
    g = torch.tensor(-0.75, dtype=torch.float64, device="cuda")
    gw = zlib.wishart_stat_bwd(s1, s2, wd, win, g)
    gw2 = zlib.wishart_stat_bwd_saved(s1, s2, zs, win, g)
    torch.cuda.synchronize()
    assert float(loss) == float(loss2) and torch.equal(q, q2)
    assert torch.equal(gw, gw2)
    K = win * win
    for t, c in ((0, c1), (1, c2)):
        ref = orc.multilook(c, win, wts)
        got = zs[9 * t:9 * t + 9].reshape(9, -1).cpu().double().numpy()
        dg = ref[[0, 5, 8]]
        scale = np.sqrt(np.stack([dg[0], dg[0] * dg[1], dg[0] * dg[1], dg[0] * dg[2],
                                  dg[0] * dg[2], dg[1], dg[1] * dg[2], dg[1] * dg[2], dg[2]]))
        scale[[0, 5, 8]] = dg
        assert np.all(np.abs(got - ref) <= gamma(K + 3) * scale)


@pytest.mark.parametrize("offset", [0, 8])
def test_saved_backward_workspace_alignment(zlib, offset):
    """W % 4 == 0: a 16-byte aligned workspace takes 16-byte copies of M, one
    8 bytes off takes 4-byte copies; both give the recomputing backward's bits."""
    H, W = 52, 96
    _, c1, c2 = pair(H, W)
    s1, s2 = torch.from_numpy(c1).cuda(), torch.from_numpy(c2).cuda()
    wd = torch.from_numpy(weights(7, 4)).cuda()
    _, zs = zlib.wishart_stat_fwd_save(s1, s2, wd, 7)
    need = zlib.wishart_bwd_saved_workspace_bytes(H, W, 7)
    buf = torch.empty(need + 16, dtype=torch.uint8, device="cuda")
    ws = buf[offset:offset + need]
    assert ws.data_ptr() % 16 == offset
    g = torch.tensor(0.5, dtype=torch.float64, device="cuda")
    gw = zlib.wishart_stat_bwd(s1, s2, wd, 7, g)
    gw2 = zlib.wishart_stat_bwd_saved(s1, s2, zs, 7, g, ws=ws)
    torch.cuda.synchronize()
    assert torch.equal(gw, gw2)


def test_saved_z_full_size_and_autograd(zlib):
    """The 4096 x 4096 pair in the benchmark's configuration: the saved path's
    loss and gradient are the recomputing path's bits, and WishartStat with
    save_z gives the same gradient through autograd."""
    from paper_1807_08084_gb300.synth import gpu as G
    w = S.WORKLOADS["wishart_pair_4k"]
    s1, s2 = G.image(w, 0), G.image(w, 1)
    wd = torch.full((49,), 1 / 49, device="cuda")
    loss = zlib.wishart_stat_fwd(s1, s2, wd, 7)
    g = zlib.wishart_stat_bwd(s1, s2, wd, 7)
    loss2, zs = zlib.wishart_stat_fwd_save(s1, s2, wd, 7)
    g2 = zlib.wishart_stat_bwd_saved(s1, s2, zs, 7)
    torch.cuda.synchronize()
    assert float(loss) == float(loss2) and torch.equal(g, g2)
    del zs
    wv = wd.clone().requires_grad_(True)
    zlib.WishartStat.apply(s1, s2, wv, 7, True).backward()
    torch.cuda.synchronize()
    assert torch.equal(wv.grad, g)


def test_saved_z_bad_arguments(zlib):
    H, W = 16, 32
    _, c1, c2 = pair(H, W)
    s1, s2 = torch.from_numpy(c1).cuda(), torch.from_numpy(c2).cuda()
    wd = torch.from_numpy(weights(3)).cuda()
    with pytest.raises(ValueError):
        zlib.wishart_stat_fwd_save(s1, s2, wd, 3, z_saved=torch.empty((9, H, W), device="cuda"))
    _, zs = zlib.wishart_stat_fwd_save(s1, s2, wd, 3)
    with pytest.raises(ValueError):
        zlib.wishart_stat_bwd_saved(s1, s2, zs[:9], 3)
    with pytest.raises(ValueError):
        zlib.wishart_stat_bwd_saved(s1, s2, zs, 3, ws=torch.empty(8, dtype=torch.uint8,
                                                                  device="cuda"))


@pytest.mark.parametrize("pad", [5, 6])  # plane stride H*W + pad (odd / even)
def test_padded_planes_give_the_same_bits(zlib, pad):
    """Single-look images whose three planes sit H*W + pad elements apart give
    the bits of the unpadded images: the Wishart statistic and gradient (both
    paths) and the boxcar and weighted multilook (an odd pad takes the
    boxcar's 8-byte copies, an even one its 16-byte copies)."""
    H, W = 37, 70
    _, c1, c2 = pair(H, W)
    s1, s2 = torch.from_numpy(c1).cuda(), torch.from_numpy(c2).cuda()

    def padded(s):
        buf = torch.zeros(3 * (H * W + pad), dtype=torch.complex64, device="cuda")
        v = buf.as_strided((3, H, W), (H * W + pad, W, 1))
        v.copy_(s)
        return v

    p1, p2 = padded(s1), padded(s2)
    wd = torch.from_numpy(weights(7, 1)).cuda()
    loss, q = zlib.wishart_stat_fwd(s1, s2, wd, 7, want_map=True)
    lossp, qp = zlib.wishart_stat_fwd(p1, p2, wd, 7, want_map=True)
    g, gp = zlib.wishart_stat_bwd(s1, s2, wd, 7), zlib.wishart_stat_bwd(p1, p2, wd, 7)
    _, zs = zlib.wishart_stat_fwd_save(s1, s2, wd, 7)
    _, zsp = zlib.wishart_stat_fwd_save(p1, p2, wd, 7)
    gs = zlib.wishart_stat_bwd_saved(p1, p2, zsp, 7)
    zi, dt = zlib.multilook_zinv_det(s1, 7)
    zip_, dtp = zlib.multilook_zinv_det(p1, 7)
    wzi, wdt = zlib.multilook_zinv_det(s1, 5, torch.from_numpy(weights(5, 2)).cuda())
    wzip, wdtp = zlib.multilook_zinv_det(p1, 5, torch.from_numpy(weights(5, 2)).cuda())
    torch.cuda.synchronize()
    assert float(loss) == float(lossp) and torch.equal(q, qp)
    assert torch.equal(g, gp) and torch.equal(g, gs) and torch.equal(zs, zsp)
    assert torch.equal(zi, zip_) and torch.equal(dt, dtp)
    assert torch.equal(wzi, wzip) and torch.equal(wdt, wdtp)
