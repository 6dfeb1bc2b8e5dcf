"""GPU parity of the fused multilook + inverse (multilook_zinv_det) against the
FP64 oracle (window covariance by Eq. ZN with clamp-to-edge addressing, then
Gauss-Jordan inverse and det), through the C ABI.

Z is accumulated in FP32 on chip: a perturbation of order u trace(Z), so the
inverse carries ~c u cond on top of the per-pixel route's own error.  Modes with
the FP64 recompute or compensation must meet 1e-5 cond; the plain adjugate the
derived bound (1e-5 + 64 u lmax/lmid) cond (see test_gpu_zinv).
"""
import numpy as np
import pytest
import torch

from helpers import det_err, inv_err

from paper_1807_08084_gb300 import synth as S

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def reference(orc, s_np, win, weights=None):
    z = orc.multilook(s_np, win, weights)
    inv, det = orc.zinv_det(z)
    cond = orc.cond(z)
    lam = orc.eigvals(z)
    return inv, det, cond, lam[2] / lam[1]


def check(zinv, det, ref, mode, tol=1e-5, sel=None):
    inv, rdet, cond, spread = ref
    zi = zinv.reshape(9, -1).cpu().numpy()
    dt = det.reshape(-1).cpu().numpy()
    if sel is not None:
        zi, dt = zi[:, sel], dt[sel]
        inv, rdet, cond, spread = inv[:, sel], rdet[sel], cond[sel], spread[sel]
    pd = np.isfinite(cond) & (rdet > 0)
    bound = tol + (64 * U32 * np.maximum(spread, 1) if mode == "plain" else 0)
    e = np.maximum(inv_err(zi, inv), det_err(dt, rdet))
    bad = pd & ~(e <= bound * cond)
    assert not bad.any(), f"{mode}: {bad.sum()} pixels out, worst err/cond {np.max(e[pd] / cond[pd]):.3e}"


MODES = {"plain": 0, "compensated": 1, "plain_fp64": 2, "compensated_fp64": 3}


@pytest.mark.parametrize("win", [3, 5, 7])
@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("shape", [(37, 131), (70, 64), (16, 64)])
def test_boxcar_small_images(zlib, orc, win, mode, shape):
    """Several tiles with ragged right/bottom edges, every pixel against the oracle."""
    H, W = shape
    w = S.scaled(S.WORKLOADS["multilook_8k"], H, W)
    s_np = w.image()
    s = torch.from_numpy(s_np).cuda()
    zinv, det, st, cnt = zlib.multilook_zinv_det(s, win, None, MODES[mode], want_status=True,
                                                 want_counts=True)
    torch.cuda.synchronize()
    check(zinv, det, reference(orc, s_np, win), mode)
    assert int(cnt[0]) == int((st & 1).sum().item())
    zinv2, det2 = zlib.multilook_zinv_det(s, win, None, MODES[mode])
    assert torch.equal(zinv, zinv2) and torch.equal(det, det2)


@pytest.mark.parametrize("mode", list(MODES))
def test_power_of_two_scaling(zlib, orc, mode):
    """Single-look data scaled by 2^j gives window covariances scaled by 2^2j:
    Z^-1 comes out scaled by 2^-2j bit for bit while det stays a normal float
    (j = +-8).  At j = +-30 det leaves the FP32 range; the FP64-recompute
    modes take every pixel to FP64 and match the oracle there."""
    w = S.scaled(S.WORKLOADS["multilook_8k"], 37, 131)
    s_np = w.image()
    base_inv, base_det = (t.cpu().numpy() for t in zlib.multilook_zinv_det(
        torch.from_numpy(s_np).cuda(), 5, None, MODES[mode]))
    for j in (-8, 8):
        sj = (s_np * np.float32(2.0 ** j)).astype(np.complex64)
        inv, det = (t.cpu().numpy() for t in zlib.multilook_zinv_det(
            torch.from_numpy(sj).cuda(), 5, None, MODES[mode]))
        assert np.array_equal(inv.view(np.uint32),
                              np.ldexp(base_inv, -2 * j).astype(np.float32).view(np.uint32))
        assert np.array_equal(det.view(np.uint32),
                              np.ldexp(base_det, 6 * j).astype(np.float32).view(np.uint32))
    if not MODES[mode] & 2:
        return
    for j in (-30, 30):
        sj = (s_np * np.float32(2.0 ** j)).astype(np.complex64)
        inv, det, st = (t.cpu().numpy() for t in zlib.multilook_zinv_det(
            torch.from_numpy(sj).cuda(), 5, None, MODES[mode], want_status=True))
        assert np.all(st == 2)
        assert np.all(det == 0) if j < 0 else np.all(np.isinf(det))
        ref_inv, _, cond, _ = reference(orc, sj, 5)
        # Z itself is accumulated in FP32 on chip: the usual 1e-5 cond
        assert np.all(inv_err(inv.reshape(9, -1), ref_inv) <= 1e-5 * cond)


@pytest.mark.parametrize("shape", [(1, 1), (1, 9), (9, 1), (3, 2), (5, 200)])
def test_degenerate_shapes(zlib, orc, shape):
    """Images smaller than the window: clamp-to-edge everywhere."""
    H, W = shape
    rng = np.random.default_rng(H * 1000 + W)
    s_np = (rng.standard_normal((3, H, W)) + 1j * rng.standard_normal((3, H, W))).astype(np.complex64)
    s = torch.from_numpy(s_np).cuda()
    for win in (3, 7):
        zinv, det, st = zlib.multilook_zinv_det(s, win, None, 2, want_status=True)
        torch.cuda.synchronize()
        ref = reference(orc, s_np, win)
        # windows with fewer than three distinct looks are (numerically) rank
        # deficient: no assertion beyond "no fault"; the rest must match
        ok = np.isfinite(ref[2]) & (ref[2] < 1e6)
        if ok.any():
            check(zinv, det, ref, "plain_fp64", sel=ok)


@pytest.mark.parametrize("win", [1, 3, 5, 7, 9])
@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("shape", [(45, 70), (32, 64), (5, 3), (17, 33)])
def test_weighted_window(zlib, orc, win, mode, shape):
    """General (non-separable) taps: 3 x 3 to 7 x 7 on the tiled window kernel,
    other sizes on the simpler one; ragged tiles, exact tile multiples (32 x 16
    tiles), images smaller than the window, every mode, against the oracle."""
    H, W = shape
    w = S.scaled(S.WORKLOADS["wishart_pair_4k"], H, W)
    s_np = w.image(0)
    rng = np.random.default_rng(win)
    wts = rng.uniform(0.2, 1.0, win * win).astype(np.float32)
    s = torch.from_numpy(s_np).cuda()
    zinv, det = zlib.multilook_zinv_det(s, win, torch.from_numpy(wts).cuda(), MODES[mode])
    zinv2, det2 = zlib.multilook_zinv_det(s, win, torch.from_numpy(wts).cuda(), MODES[mode])
    torch.cuda.synchronize()
    assert torch.equal(zinv, zinv2) and torch.equal(det, det2)
    if win == 1:  # single look: rank one, det 0
        return
    check(zinv, det, reference(orc, s_np, win, wts), mode)


def test_weighted_equals_boxcar(zlib, orc):
    """The weighted path with w = 1/N is the boxcar up to summation order: each
    is within 1e-5 cond of the oracle, so they are within 2e-5 cond of each other."""
    w = S.scaled(S.WORKLOADS["multilook_8k"], 64, 96)
    s_np = w.image()
    s = torch.from_numpy(s_np).cuda()
    a_inv, a_det = zlib.multilook_zinv_det(s, 5, None, 3)
    b_inv, b_det = zlib.multilook_zinv_det(s, 5, torch.full((25,), 1 / 25, device="cuda"), 3)
    torch.cuda.synchronize()
    cond = orc.cond(orc.multilook(s_np, 5))
    ad, bd = a_det.reshape(-1).cpu().numpy(), b_det.reshape(-1).cpu().numpy()
    assert np.all(np.abs(ad - bd) <= 2e-5 * cond * np.abs(ad))


def test_argument_errors(zlib):
    s = torch.zeros((3, 8, 8), dtype=torch.complex64, device="cuda")
    for bad in (2, 4, 9):
        with pytest.raises(RuntimeError):
            zlib.multilook_zinv_det(s, bad)


def test_full_size_crops(zlib, orc):
    """8192 x 8192 generated on the GPU, the three boxcar windows and two
    weighted ones (the benchmark's 7 x 7 Gaussian taps, random 5 x 5 taps) in
    the launch configuration of the full image; 12 crops (corners, edges,
    interior) against the oracle on inputs regenerated by the numpy twin."""
    from paper_1807_08084_gb300.synth import gpu as G
    w = S.WORKLOADS["multilook_8k"]
    s = G.image(w)
    H, W = w.H, w.W
    rng = np.random.default_rng(9)
    boxes = [(0, 0), (0, W - 48), (H - 48, 0), (H - 48, W - 48), (0, 4000), (4000, 0),
             (H - 48, 5000), (6000, W - 48)] + [tuple(rng.integers(100, 8000, 2)) for _ in range(4)]
    g = np.exp(-0.5 * (np.arange(-3, 4) / 1.5) ** 2)
    gauss7 = (np.outer(g, g) / np.outer(g, g).sum()).astype(np.float32)  # the bench's taps
    rand5 = np.random.default_rng(5).uniform(0.2, 1.0, 25).astype(np.float32)
    for win, wts in ((3, None), (5, None), (7, None), (7, gauss7), (5, rand5)):
        r = (win - 1) // 2
        wt = None if wts is None else torch.from_numpy(wts.ravel()).cuda()
        zinv, det = zlib.multilook_zinv_det(s, win, wt, 2)
        torch.cuda.synchronize()
        for (y0, x0) in boxes:
            y1, x1 = y0 + 48, x0 + 48
            cy0, cy1 = max(0, y0 - r), min(H, y1 + r)
            cx0, cx1 = max(0, x0 - r), min(W, x1 + r)
            yy, xx = np.meshgrid(np.arange(cy0, cy1), np.arange(cx0, cx1), indexing="ij")
            idx = (yy * W + xx).ravel().astype(np.uint64)
            crop = w.looks(idx).reshape(3, cy1 - cy0, cx1 - cx0)
            got_in = s[:, cy0:cy1, cx0:cx1].cpu().numpy()
            np.testing.assert_array_equal(got_in, crop)
            ref = reference(orc, crop, win, None if wts is None else wts.ravel())
            ch, cw = cy1 - cy0, cx1 - cx0
            inner = np.zeros((ch, cw), bool)
            inner[y0 - cy0:y1 - cy0, x0 - cx0:x1 - cx0] = True
            sel = inner.ravel()
            zc = zinv[:, cy0:cy1, cx0:cx1].reshape(9, -1)
            dc = det[cy0:cy1, cx0:cx1].reshape(-1)
            check(zc, dc, ref, "plain_fp64", sel=sel)
        del zinv, det


@pytest.mark.parametrize("win", [3, 7])
@pytest.mark.parametrize("mode", ["plain", "compensated_fp64"])
def test_weighted_larger_ragged_image(zlib, orc, win, mode):
    """An 811 x 1000 image: 1632 tiles of 32 x 16 with ragged right and bottom
    tiles.  Every pixel against the oracle, the status plane against the
    counters, and the same bits on a repeat."""
    H, W = 811, 1000
    w = S.scaled(S.WORKLOADS["wishart_pair_4k"], H, W)
    s_np = w.image(1)
    wts = np.random.default_rng(40 + win).uniform(0.2, 1.0, win * win).astype(np.float32)
    s = torch.from_numpy(s_np).cuda()
    wt = torch.from_numpy(wts).cuda()
    zinv, det, st, cnt = zlib.multilook_zinv_det(s, win, wt, MODES[mode], want_status=True,
                                                 want_counts=True)
    zinv2, det2 = zlib.multilook_zinv_det(s, win, wt, MODES[mode])
    torch.cuda.synchronize()
    assert torch.equal(zinv, zinv2) and torch.equal(det, det2)
    check(zinv, det, reference(orc, s_np, win, wts), mode)
    stn = st.cpu().numpy()
    assert int(cnt[0]) == int((stn & 1).sum()) and int(cnt[1]) == int(((stn & 2) > 0).sum())
