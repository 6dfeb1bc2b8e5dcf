"""GPU parity of the per-pixel kernels (zinv_det in every mode, chol_zinv_det,
zinv_det_bwd, zinv_det_host) against the FP64 oracle, through the C ABI.

Tolerance (stated for FP32 inverse and det): per pixel, max relative entrywise
error <= 1e-5 * cond_2(Z), where the diagonal error is |dW_ii|/W_ii, the
off-diagonal error |dW_ij|/sqrt(W_ii W_jj) (a bound on |W_ij| for positive
definite W), and cond_2 comes from the oracle on the FP32 input.  Repeated GPU
runs must agree bit for bit.
"""
import numpy as np
import pytest
import torch

from helpers import det_err, inv_err, unpack

from paper_1807_08084_gb300 import synth as S

pytestmark = pytest.mark.gpu

TOL = 1e-5
MODES = {
    "plain": ("zinv_det", 0),
    "compensated": ("zinv_det", 1),
    "plain_fp64": ("zinv_det", 2),
    "compensated_fp64": ("zinv_det", 3),
    "cholesky": ("chol_zinv_det", 0),
}


def strided(a, ld: int) -> torch.Tensor:
    """[9, n] CUDA view with plane stride ld (>= n) holding a copy of a."""
    a = torch.as_tensor(a).cuda()
    n = a.shape[1]
    t = torch.as_strided(torch.zeros(9 * ld, device="cuda"), (9, n), (ld, 1))
    t.copy_(a)
    return t


def odd_ld(n: int) -> int:
    return n + 1 if (n + 1) % 4 else n + 2


def run_mode(zp, z, mode, **kw):
    fn, flags = MODES[mode]
    if fn == "chol_zinv_det":
        return zp.chol_zinv_det(z, **kw)
    return zp.zinv_det(z, flags, **kw)


def check_parity(orc, z_np, zinv_gpu, det_gpu, tol=TOL, mask=None):
    ref_inv, ref_det = orc.zinv_det(z_np)
    cond = orc.cond(z_np)
    pd = np.isfinite(cond) & (ref_det > 0)
    if mask is not None:
        pd &= mask
    ei = inv_err(zinv_gpu, ref_inv)
    ed = det_err(det_gpu, ref_det)
    bad = pd & ~((ei <= tol * cond) & (ed <= tol * cond))
    assert not bad.any(), (
        f"{bad.sum()} of {pd.sum()} pixels out of tolerance; worst inv err/cond "
        f"{np.nanmax(ei[pd] / cond[pd]):.3e}, det err/cond {np.nanmax(ed[pd] / cond[pd]):.3e}")
    return ei[pd], ed[pd], cond[pd]


@pytest.mark.parametrize("mode", list(MODES))
def test_plain_workload_full(zlib, orc, mode):
    """256 x 256, N = 4 looks of the fixed Sigma: every pixel against the oracle."""
    w = S.WORKLOADS["plain_256"]
    z_np = w.packed_z()
    z = torch.from_numpy(z_np).cuda().reshape(9, w.H, w.W)
    zinv, det, status, counts = run_mode(zlib, z, mode, want_status=True, want_counts=True)
    torch.cuda.synchronize()
    check_parity(orc, z_np, zinv.cpu().numpy().reshape(9, -1), det.cpu().numpy().ravel())
    assert int(counts[0]) == 0 and int((status & 1).sum()) == 0
    # bit-exact repeat
    zinv2, det2 = run_mode(zlib, z, mode)
    assert torch.equal(zinv, zinv2) and torch.equal(det, det2)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 255, 1023, 4097, 65537])
@pytest.mark.parametrize("mode", ["plain", "compensated", "cholesky"])
def test_ragged_sizes_and_both_paths(zlib, orc, n, mode):
    """Tails that do not fill a float4, the 128-bit path (ld % 4 == 0) and the
    one-pixel path (ld % 4 != 0) give the same bits and match the oracle."""
    w = S.WORKLOADS["paper_sim"]
    z_np = w.packed_z(np.arange(n, dtype=np.uint64))
    z_vec = strided(z_np, (n + 3) // 4 * 4)
    z_sca = strided(z_np, odd_ld(n))
    a_inv, a_det = run_mode(zlib, z_vec, mode)
    b_inv, b_det = run_mode(zlib, z_sca, mode)
    torch.cuda.synchronize()
    assert torch.equal(a_inv.contiguous(), b_inv.contiguous()) and torch.equal(a_det, b_det)
    check_parity(orc, z_np, a_inv.cpu().numpy(), a_det.cpu().numpy())


def test_empty_input(zlib):
    z = torch.empty((9, 0), device="cuda")
    zinv, det, counts = zlib.zinv_det(z, want_counts=True)
    torch.cuda.synchronize()
    assert zinv.shape == (9, 0) and det.shape == (0,) and counts.tolist() == [0, 0]


def test_in_place(zlib, orc):
    w = S.WORKLOADS["plain_256"]
    z_np = w.packed_z(np.arange(10001, dtype=np.uint64))
    z = torch.from_numpy(z_np).cuda()
    ref_inv, ref_det = zlib.zinv_det(z.clone())
    det = torch.empty(z.shape[1], device="cuda")
    zlib.zinv_det(z, out=(z, det))
    torch.cuda.synchronize()
    assert torch.equal(z, ref_inv) and torch.equal(det, ref_det)


def test_not_pd_and_non_finite_pixels(zlib):
    """Bad pixels are flagged in the status plane and counted; nothing traps."""
    rows = [
        [1, 0, 0, 0, 0, 1, 0, 0, 1],          # identity (good)
        [0, 0, 0, 0, 0, 0, 0, 0, 0],          # zero matrix
        [1, 2, 0, 0, 0, 1, 0, 0, 1],          # indefinite (det < 0)
        [-1, 0, 0, 0, 0, -1, 0, 0, 1],        # det > 0 but not PD (two negative eigenvalues)
        [float("nan")] + [0] * 8,             # NaN
        [float("inf"), 0, 0, 0, 0, 1, 0, 0, 1],
        [1, 1, 0, 0, 0, 1, 0, 0, 1],          # singular (det = 0)
    ]
    z_np = np.array(rows, dtype=np.float32).T.copy()
    z = torch.from_numpy(z_np).cuda()
    for mode in MODES:
        zinv, det, st, cnt = run_mode(zlib, z, mode, want_status=True, want_counts=True)
        torch.cuda.synchronize()
        st = st.cpu().numpy()
        not_pd = (st & 1).astype(bool)
        assert not not_pd[0]
        assert not_pd[[1, 2, 4, 5, 6]].all(), (mode, st)
        assert int(cnt[0]) == int(not_pd.sum())
        if mode.endswith("fp64"):
            assert int(cnt[1]) == int(((st & 2) > 0).sum()) >= 5
        # a det > 0 matrix with two negative eigenvalues passes the det test of the
        # adjugate route (Eq. det cannot see it); the Cholesky route fails on it
        if mode == "cholesky":
            assert not_pd[3]


def test_fp64_flag_and_counts(zlib, orc):
    """Pixels with det <= tau * a d f are recomputed in FP64 and counted; the
    recomputed ones match the oracle to FP32 rounding."""
    w = S.WORKLOADS["precision_4k"]
    idx = np.arange(200000, dtype=np.uint64)
    z_np = w.packed_z(idx)
    z = torch.from_numpy(z_np).cuda()
    tau = 2.0 ** -10
    zinv, det, st, cnt = zlib.zinv_det(z, 2, tau, want_status=True, want_counts=True)
    torch.cuda.synchronize()
    st = st.cpu().numpy()
    rec = (st & 2) > 0
    ref_inv, ref_det = orc.zinv_det(z_np)
    # the flag decision, re-taken in FP32 exactly as the kernel does, on the kernel's det
    plain_inv, plain_det = zlib.zinv_det(z, 0)
    pdet = plain_det.cpu().numpy()
    adf = (z_np[0] * z_np[5]).astype(np.float32) * z_np[8]
    expect = ~(pdet > np.float32(tau) * adf)
    assert np.array_equal(rec, expect)
    assert int(cnt[1]) == int(rec.sum()) > 0
    # NOT_PD in FP64 mode is the FP64 sign of det, as the oracle's
    not_pd = (st & 1) > 0
    assert np.array_equal(not_pd, ~(ref_det > 0))
    # recomputed pixels: compensated FP64, then one FP32 rounding of each output
    good = rec & (ref_det > 0)
    ei = inv_err(zinv.cpu().numpy()[:, good], ref_inv[:, good])
    ed = det_err(det.cpu().numpy()[good], ref_det[good])
    assert ei.max() < 4 * 2.0 ** -24 and ed.max() < 4 * 2.0 ** -24


@pytest.mark.parametrize("density", [0.0, 0.01, 0.5, 1.0])
@pytest.mark.parametrize("flags", [2, 3])
def test_fp64_queue_is_position_independent(zlib, orc, density, flags):
    """The FP64 variants queue flagged pixels per warp and recompute them 32 at
    a time.  A pixel's outputs must not depend on where it sits, on how many of
    its neighbours are flagged, on the layout (128-bit path, unaligned plane
    stride on the one-pixel path, in place) or on the run: every arrangement
    gives the same bits, and the flagged pixels match the oracle to FP32
    rounding."""
    rng = np.random.default_rng(11 + int(100 * density) + flags)
    n = 40001  # a ragged tail after the last float4 group
    well = S.WORKLOADS["scale_16k"].packed_z(np.arange(n, dtype=np.uint64))
    ill = S.WORKLOADS["precision_4k"].packed_z(np.arange(n, dtype=np.uint64))
    # precision_4k pixels with det/(adf) far below tau are flagged; scale_16k's are not
    pick = rng.random(n) < density
    z_np = np.where(pick[None, :], ill, well).astype(np.float32)
    tau = 2.0 ** -10
    z = torch.from_numpy(z_np).cuda()
    zinv, det, st, cnt = zlib.zinv_det(z, flags, tau, want_status=True, want_counts=True)
    perm = rng.permutation(n)
    zp_, dp_, sp_ = zlib.zinv_det(z[:, perm].contiguous(), flags, tau, want_status=True)
    inv_perm = np.argsort(perm)
    zu = strided(z_np, odd_ld(n))  # one-pixel path, FP64 inline
    zu_inv, zu_det, zu_st = zlib.zinv_det(zu, flags, tau, want_status=True)
    zi = z.clone()
    d_ip = torch.empty(n, device="cuda")
    zlib.zinv_det(zi, flags, tau, out=(zi, d_ip))
    again = zlib.zinv_det(z, flags, tau, want_status=True)
    torch.cuda.synchronize()
    a_inv, a_det, a_st = zinv.cpu().numpy(), det.cpu().numpy(), st.cpu().numpy()
    for other_inv, other_det in ((zp_.cpu().numpy()[:, inv_perm], dp_.cpu().numpy()[inv_perm]),
                                 (zu_inv.cpu().numpy(), zu_det.cpu().numpy()),
                                 (zi.cpu().numpy(), d_ip.cpu().numpy()),
                                 (again[0].cpu().numpy(), again[1].cpu().numpy())):
        assert np.array_equal(a_inv.view(np.uint32), other_inv.view(np.uint32))
        assert np.array_equal(a_det.view(np.uint32), other_det.view(np.uint32))
    assert np.array_equal(a_st, sp_.cpu().numpy()[inv_perm])
    assert np.array_equal(a_st, zu_st.cpu().numpy())
    rec = (a_st & 2) > 0
    assert int(cnt[1]) == int(rec.sum()) and int(cnt[0]) == int(((a_st & 1) > 0).sum())
    if density == 0.0:
        assert not rec.any()
    if density == 1.0:
        assert rec.mean() > 0.4
    ref_inv, ref_det = orc.zinv_det(z_np)
    assert np.array_equal((a_st & 1) > 0, ~(ref_det > 0))
    good = rec & (ref_det > 0)
    if good.any():
        ei = inv_err(a_inv[:, good], ref_inv[:, good])
        ed = det_err(a_det[good], ref_det[good])
        assert ei.max() < 4 * 2.0 ** -24 and ed.max() < 4 * 2.0 ** -24


@pytest.mark.parametrize("flags", [0, 1, 2, 3])
def test_power_of_two_scaling(zlib, orc, flags):
    """Algorithm 2 is homogeneous and power-of-two scaling is exact, so Z 2^j
    gives Z^-1 2^-j and det 2^3j bit for bit while det stays a normal float
    (j = +-20).  det scales with the cube of the entries: at 2^+-36 and 2^+-60
    det leaves the band [2^-100, 2^100) and the FP64-recompute modes take those
    pixels to FP64, whose range covers them: Z^-1 within FP32 rounding of the
    oracle, det the FP32 rounding of the exact det (0 or inf where that is out
    of range), the pixels positive definite."""
    w = S.WORKLOADS["plain_256"]
    n = 4099
    z_np = w.packed_z(np.arange(n, dtype=np.uint64))
    base_inv, base_det, base_st = (t.cpu().numpy() for t in zlib.zinv_det(
        torch.from_numpy(z_np).cuda(), flags, want_status=True))
    for j in (-20, 20):
        zj = np.ldexp(z_np, j).astype(np.float32)
        assert np.array_equal(np.ldexp(zj, -j), z_np)  # the scaled input is exact
        inv, det, st = (t.cpu().numpy() for t in zlib.zinv_det(
            torch.from_numpy(zj).cuda(), flags, want_status=True))
        assert np.array_equal(inv.view(np.uint32),
                              np.ldexp(base_inv, -j).astype(np.float32).view(np.uint32))
        assert np.array_equal(det.view(np.uint32),
                              np.ldexp(base_det, 3 * j).astype(np.float32).view(np.uint32))
        assert np.array_equal(st, base_st)
    if not flags & 2:
        return
    assert np.all((base_st == 0) | (base_st == 2))
    for j in (-60, -36, 36, 60):
        zj = np.ldexp(z_np, j).astype(np.float32)
        inv, det, st = (t.cpu().numpy() for t in zlib.zinv_det(
            torch.from_numpy(zj).cuda(), flags, want_status=True))
        # det of Z 2^j is base_det 2^3j: out of [2^-100, 2^100) -> FP64
        scaled = np.ldexp(base_det.astype(np.float64), 3 * j)
        out = ~((scaled >= 2.0 ** -100) & (scaled < 2.0 ** 100))
        assert np.all((st == 0) | (st == 2)) and np.all(st[out] == 2)
        assert np.all(st[base_st == 2] == 2)
        if abs(j) == 60:
            assert out.all()
        keep = st == 0  # the FP32 route in range: exactly the scaled bits
        assert np.array_equal(inv[:, keep].view(np.uint32),
                              np.ldexp(base_inv[:, keep], -j).astype(np.float32).view(np.uint32))
        assert np.array_equal(det[keep].view(np.uint32), scaled[keep].astype(np.float32).view(np.uint32))
        out = st == 2  # recomputed in FP64: FP32 rounding of the exact result
        ref_inv, ref_det = orc.zinv_det(zj)
        assert np.all(inv_err(inv[:, out], ref_inv[:, out]) < 4 * 2.0 ** -24)
        with np.errstate(over="ignore"):  # dets beyond FP32 become inf
            e32 = ref_det.astype(np.float32)
        normal = out & np.isfinite(e32) & (e32 >= np.float32(2.0 ** -126))
        assert np.all(det_err(det[normal], ref_det[normal]) < 4 * 2.0 ** -24)
        assert np.all(np.isinf(det[out & np.isinf(e32)]))
        sub = out & np.isfinite(e32) & (e32 < np.float32(2.0 ** -126))
        assert np.all(np.abs(det[sub].astype(np.float64) - e32[sub]) <= 2.0 ** -149)


U32 = 2.0 ** -24


@pytest.mark.parametrize("mode", list(MODES))
def test_precision_workload_tolerance(zlib, orc, mode):
    """cond log-uniform in [1, 1e7] (Z = U diag(1, kappa^-v, 1/kappa) U^H).

    Compensated, FP64-recompute and Cholesky modes: every positive-definite pixel
    within 1e-5 cond.  The plain FP32 adjugate is not backward stable: its
    cofactors carry absolute errors ~u lmax^2, so det (and with it Z^-1) is off
    by ~c u cond (lmax/lmid), c ~ 6 measured, up to u cond^2 when two eigenvalues
    are small.  It meets 1e-5 cond where lmax/lmid <= 16 and the derived bound
    64 u cond (lmax/lmid) everywhere.
    """
    w = S.WORKLOADS["precision_4k"]
    z_np = w.packed_z(np.arange(100000, dtype=np.uint64))
    z = torch.from_numpy(z_np).cuda()
    zinv, det = run_mode(zlib, z, mode)
    torch.cuda.synchronize()
    if mode != "plain":
        ei, ed, cond = check_parity(orc, z_np, zinv.cpu().numpy(), det.cpu().numpy())
        if mode.startswith("compensated"):
            # compensation removes the cond-proportional term for moderate cond
            m = cond < 1e4
            assert np.max(ei[m]) < 1e-5 and np.max(ed[m]) < 1e-5
        return
    lam = orc.eigvals(z_np)
    spread = lam[2] / lam[1]
    check_parity(orc, z_np, zinv.cpu().numpy(), det.cpu().numpy(), mask=spread <= 16)
    check_parity(orc, z_np, zinv.cpu().numpy(), det.cpu().numpy(),
                 tol=64 * U32 * np.maximum(spread, 1.0))


def test_generator_twin_bit_exact(zlib):
    """The GPU generator reproduces the numpy twin bit for bit at sampled pixels."""
    from paper_1807_08084_gb300.synth import gpu as G
    rng = np.random.default_rng(5)
    for name in ("plain_256", "precision_4k", "paper_sim", "paper_meas_shaped"):
        w = S.WORKLOADS[name]
        if w.n > 5_000_000:
            w = S.scaled(w, 1, 2_000_000)
        zg = G.packed_z(w).reshape(9, -1)
        idx = np.unique(rng.integers(0, w.n, 3000)).astype(np.uint64)
        got = zg[:, torch.from_numpy(idx.astype(np.int64)).cuda()].cpu().numpy()
        np.testing.assert_array_equal(got, w.packed_z(idx), err_msg=name)
    for name in ("multilook_8k", "wishart_pair_4k"):
        w = S.scaled(S.WORKLOADS[name], 512, 384)
        for date in (0, 1):
            sg = G.image(w, date).reshape(3, -1)
            idx = np.unique(rng.integers(0, w.n, 3000)).astype(np.uint64)
            got = sg[:, torch.from_numpy(idx.astype(np.int64)).cuda()].cpu().numpy()
            np.testing.assert_array_equal(got, w.looks(idx, date), err_msg=f"{name} {date}")
    u = G.uniform(7, 1000).cpu().numpy()
    np.testing.assert_array_equal(u, S.uniform_f32(7, np.arange(1000, dtype=np.uint64)))


def test_scale_workload_full_size_sampled(zlib, orc):
    """16384 x 16384 (268M pixels) generated on the GPU, inverted in the launch
    configuration the benchmark times; 200k sampled pixels against the oracle on
    inputs regenerated by the numpy twin."""
    from paper_1807_08084_gb300.synth import gpu as G
    w = S.WORKLOADS["scale_16k"]
    z = G.packed_z(w)
    rng = np.random.default_rng(6)
    idx = np.unique(rng.integers(0, w.n, 200000))
    it = torch.from_numpy(idx).cuda()
    z_np = w.packed_z(idx.astype(np.uint64))
    np.testing.assert_array_equal(z.reshape(9, -1)[:, it].cpu().numpy(), z_np)
    for mode in ("plain", "compensated", "plain_fp64", "cholesky"):
        zinv, det = run_mode(zlib, z, mode)
        torch.cuda.synchronize()
        check_parity(orc, z_np, zinv.reshape(9, -1)[:, it].cpu().numpy(),
                     det.reshape(-1)[it].cpu().numpy())
        del zinv, det
    # the last pixel (a ragged-free size, but the final group of the grid-stride loop)
    last = np.array([w.n - 1], dtype=np.uint64)
    zinv, det = zlib.zinv_det(z)
    ref_inv, ref_det = orc.zinv_det(w.packed_z(last))
    assert det_err(det.reshape(-1)[-1:].cpu().numpy(), ref_det)[0] < 1e-3


def test_paper_sim_full_size_sampled(zlib, orc):
    """The paper's simulated set (its Table 2: 5,469,354 matrices A = R R^H)
    generated on the GPU as one row, in the benchmark's launch configuration
    (a plane stride that is not a multiple of four: the one-pixel kernel);
    100k sampled pixels and the last one against the oracle, both routes."""
    from paper_1807_08084_gb300.synth import gpu as G
    w = S.WORKLOADS["paper_sim"]
    z = G.packed_z(w)
    rng = np.random.default_rng(8)
    idx = np.unique(np.concatenate([rng.integers(0, w.n, 100000), [w.n - 1]]))
    it = torch.from_numpy(idx).cuda()
    z_np = w.packed_z(idx.astype(np.uint64))
    np.testing.assert_array_equal(z.reshape(9, -1)[:, it].cpu().numpy(), z_np)
    for mode in ("plain", "cholesky"):
        zinv, det = run_mode(zlib, z, mode)
        torch.cuda.synchronize()
        check_parity(orc, z_np, zinv.reshape(9, -1)[:, it].cpu().numpy(),
                     det.reshape(-1)[it].cpu().numpy())


def _bwd_tol_check(orc, z_np, gz_gpu, gW, gd, gl, tol=TOL):
    ref = orc.zinv_det_bwd(z_np, gW, gd, gl)
    W, det = orc.zinv_det(z_np)
    cond = orc.cond(z_np)
    Wn = np.abs(unpack(W)).max(axis=(1, 2))
    s = np.zeros(z_np.shape[1])
    if gd is not None:
        s += np.abs(gd) * np.abs(det)
    if gl is not None:
        s += np.abs(gl)
    scale = Wn * Wn * (0 if gW is None else np.abs(gW).max(axis=0)) + s * Wn
    err = np.abs(gz_gpu - ref).max(axis=0) / scale
    assert np.all(err <= tol * cond), f"worst bwd err/cond {np.max(err / cond):.3e}"


@pytest.mark.parametrize("which", ["W", "det", "logdet", "all"])
def test_bwd_parity(zlib, orc, which):
    w = S.WORKLOADS["plain_256"]
    n = 50001
    idx = np.arange(n, dtype=np.uint64)
    z_np = w.packed_z(idx)
    z = torch.from_numpy(z_np).cuda()
    zinv, det = zlib.zinv_det(z)
    gW = np.stack([S.uniform_f32(11, idx, stream=k) for k in range(9)])
    gd = S.uniform_f32(12, idx)
    gl = S.uniform_f32(13, idx)
    use = {"W": (gW, None, None), "det": (None, gd, None), "logdet": (None, None, gl),
           "all": (gW, gd, gl)}[which]
    args = [None if a is None else torch.from_numpy(a).cuda() for a in use]
    gz = zlib.zinv_det_bwd(zinv, det, *args)
    torch.cuda.synchronize()
    _bwd_tol_check(orc, z_np, gz.cpu().numpy(), *use)
    # one-pixel path (ld % 4 != 0) gives the same bits
    ld = odd_ld(n)
    a2 = [None if a is None else (a.clone() if a.dim() == 1 else strided(a, ld)) for a in args]
    gz2 = zlib.zinv_det_bwd(strided(zinv, ld), det, *a2)
    torch.cuda.synchronize()
    assert torch.equal(gz2.contiguous(), gz)


def test_autograd_function(zlib):
    import paper_1807_08084_gb300 as zp
    w = S.WORKLOADS["plain_256"]
    z = torch.from_numpy(w.packed_z(np.arange(4096, dtype=np.uint64))).cuda().requires_grad_()
    gW = torch.randn(9, 4096, device="cuda")
    gd = torch.randn(4096, device="cuda")
    zinv, det = zp.ZInvDet.apply(z)
    (zinv * gW).sum().add_((det * gd).sum()).backward()
    direct = zp.zinv_det_bwd(zinv.detach(), det.detach(), gW, gd, None)
    torch.cuda.synchronize()
    assert torch.equal(z.grad, direct)


def test_host_streaming_matches_device(zlib):
    w = S.WORKLOADS["paper_sim"]
    n = 1_000_003
    z = torch.from_numpy(w.packed_z(np.arange(n, dtype=np.uint64)))
    z_pin = z.pin_memory()
    ref_inv, ref_det = zlib.zinv_det(z.cuda())
    for chunk in (4096, 100_000, n + 10):
        ws = torch.empty(zlib.zinv_det_host_workspace_bytes(chunk), dtype=torch.uint8,
                         device="cuda")
        zinv_h, det_h = zlib.zinv_det_host(z_pin, ws, zlib.HOST_STAGED)
        torch.cuda.synchronize()
        assert torch.equal(zinv_h, ref_inv.cpu()) and torch.equal(det_h, ref_det.cpu())
    # pinned buffers without a workspace: the kernel works on host memory directly
    zinv_h, det_h = zlib.zinv_det_host(z_pin)
    torch.cuda.synchronize()
    assert torch.equal(zinv_h, ref_inv.cpu()) and torch.equal(det_h, ref_det.cpu())
    # pageable input cannot be read by the kernel: it needs the staged way
    with pytest.raises(RuntimeError):
        zlib.zinv_det_host(z.clone())


def test_host_streaming_fp64_recompute(zlib):
    """The FP64-recompute variant queues flagged pixels and parks their inputs
    in the outputs: through the staged path (in place in device chunks) and the
    direct path (the kernel on pinned host memory) it gives the device result
    bit for bit on an image where half the pixels are flagged."""
    w = S.WORKLOADS["precision_4k"]
    n = 300_007
    z = torch.from_numpy(w.packed_z(np.arange(n, dtype=np.uint64)))
    z_pin = z.pin_memory()
    flags = zlib.COMPENSATED | zlib.FP64_RECOMPUTE
    ref_inv, ref_det, st, cnt = zlib.zinv_det(z.cuda(), flags, want_status=True,
                                              want_counts=True)
    assert int(cnt[1]) > n // 3
    ws = torch.empty(zlib.zinv_det_host_workspace_bytes(65536), dtype=torch.uint8,
                     device="cuda")
    for args in ((ws, flags | zlib.HOST_STAGED), (None, flags)):
        zinv_h, det_h = zlib.zinv_det_host(z_pin, *args)
        torch.cuda.synchronize()
        assert torch.equal(zinv_h, ref_inv.cpu()) and torch.equal(det_h, ref_det.cpu())
