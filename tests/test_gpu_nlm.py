"""GPU parity of the nonlocal-means filter (nlm_wishart) against the FP64 oracle.

Tolerance, derived per output pixel i and packed channel c (first order).  The
kernel forms w_ij = 2^(-p t_ij), p = L/h, t_ij = log2 D_ij - 3 - h_i - h_j with
D_ij = det(Z_i + Z_j) in FP32 (Algorithm 2 or Algorithm 1) and h = log2(det)/2
(compensated).  An error e_ij in t gives w_ij a relative error
    delta_ij = p ln2 e_ij + eta      (eta: the exp2 rounding, <= 2^-22),
and the filtered value Z'_i = sum_j w_ij Z_j / sum_j w_ij moves by
    |dZ'_ic| <= max_j |delta_ij| * max_j |Z_jc - Z'_ic|,
plus the FP32 rounding of the two weighted sums over n_i <= (2r+1)^2 terms,
    <= 2 gamma_(n_i + 2) max_j |Z_jc|,   gamma_k = k u / (1 - k u), u = 2^-24.
The FP32 determinant of the pair sum has relative error <= gamma_16 E_ij / D_ij,
where E_ij is its cofactor expansion with every term taken in magnitude
(E >= a d f, so this also bounds the Cholesky route's pivots); the log2
approximation errs by <= 2^-21 absolute, and rounding t and its terms by
<= 4u (|log2 D_ij| + 3 + |h_i| + |h_j|), so
    e_ij <= gamma_16 E_ij / (D_ij ln2) + 2^-21 + 4u (|log2 D_ij| + 3 + |h_i| + |h_j|).
The test bound is 1.25 times that sum, computed from the oracle's inputs."""
import numpy as np
import pytest
import torch

from paper_1807_08084_gb300 import synth as S

pytestmark = pytest.mark.gpu
U = 2.0 ** -24


def gamma(k):
    return k * U / (1 - k * U)


def det3(s):
    """det of packed Hermitian 3x3 matrices [9, ...] (FP64, cofactor expansion)."""
    a, br, bi, cr, ci, d, er, ei, f = s
    return (a * (d * f - er * er - ei * ei) - br * (br * f - (cr * er + ci * ei))
            - bi * (bi * f - (ci * er - cr * ei)) - cr * (cr * d - (br * er - bi * ei))
            - ci * (ci * d - (br * ei + bi * er)))


def nlm_bound(z, H, W, radius, p, ref):
    """[9, H*W] first-order error bound of the FP32 filter at every pixel
    (see the module docstring); z: packed input, ref: the oracle's output."""
    Z = np.asarray(z, dtype=np.float64).reshape(9, H, W)
    R = np.asarray(ref, dtype=np.float64).reshape(9, H, W)
    hz = np.abs(np.log2(det3(Z))) / 2
    e_max = np.zeros((H, W))
    spread = np.zeros((9, H, W))
    mag = np.zeros((9, H, W))
    count = np.zeros((H, W))
    for dy in range(-radius, radius + 1):
        for dx in range(-radius, radius + 1):
            ys = slice(max(0, -dy), min(H, H - dy))
            xs = slice(max(0, -dx), min(W, W - dx))
            yj = slice(max(0, dy), min(H, H + dy))
            xj = slice(max(0, dx), min(W, W + dx))
            zi, zj = Z[:, ys, xs], Z[:, yj, xj]
            s = zi + zj
            a, br, bi, cr, ci, d, er, ei, f = s
            det = det3(s)
            ab, ac, ae = np.abs(br) + np.abs(bi), np.abs(cr) + np.abs(ci), np.abs(er) + np.abs(ei)
            E = a * (d * f + ae * ae) + ab * (ac * ae + ab * f) + ac * (ab * ae + ac * d)
            e = (gamma(16) * E / (det * np.log(2)) + 2.0 ** -21
                 + 4 * U * (np.abs(np.log2(det)) + 3 + hz[ys, xs] + hz[yj, xj]))
            e_max[ys, xs] = np.maximum(e_max[ys, xs], e)
            spread[:, ys, xs] = np.maximum(spread[:, ys, xs], np.abs(zj - R[:, ys, xs]))
            mag[:, ys, xs] = np.maximum(mag[:, ys, xs], np.abs(zj))
            count[ys, xs] += 1
    delta = p * np.log(2) * e_max + 2.0 ** -22
    b = delta[None] * spread + 2 * gamma(count + 2)[None] * mag
    return 1.25 * b.reshape(9, -1)


def check(out, ref, bound, where=""):
    err = np.abs(np.asarray(out, dtype=np.float64) - ref)
    bad = err > bound
    assert not bad.any(), (f"{where}{bad.sum()} entries over the bound; worst err/bound "
                           f"{(err / bound).max():.3f}")
    return (err / bound).max()


@pytest.mark.parametrize("radius", [1, 3, 11])
@pytest.mark.parametrize("method", [0, 1])
def test_nlm_vs_oracle(zlib, orc, radius, method):
    H, W = 37, 70
    w = S.scaled(S.WORKLOADS["scale_16k"], H, W)
    z_np = w.packed_z()
    z = torch.from_numpy(z_np).cuda().reshape(9, H, W)
    out = zlib.nlm_wishart(z, radius, 16.0, 1.0, method)
    torch.cuda.synchronize()
    ref = orc.nlm_wishart(z_np, H, W, radius, 16.0, 1.0)
    check(out.reshape(9, -1).cpu().numpy(), ref, nlm_bound(z_np, H, W, radius, 16.0, ref))


def test_methods_agree_and_repeat(zlib):
    """Repeated runs give the same bits; the two determinant methods agree to
    twice the bound (each is within one bound of the exact filter; the bound's
    scale is taken from the adjugate output)."""
    H, W = 96, 128
    w = S.scaled(S.WORKLOADS["scale_16k"], H, W)
    z_np = w.packed_z()
    z = torch.from_numpy(z_np).cuda().reshape(9, H, W)
    a = zlib.nlm_wishart(z, 11, 16.0, 1.0, 0)
    b = zlib.nlm_wishart(z, 11, 16.0, 1.0, 1)
    a2 = zlib.nlm_wishart(z, 11, 16.0, 1.0, 0)
    torch.cuda.synchronize()
    assert torch.equal(a, a2)
    an = a.reshape(9, -1).cpu().double().numpy()
    check(b.reshape(9, -1).cpu().numpy(), an, 2 * nlm_bound(z_np, H, W, 11, 16.0, an))


def test_constant_image_is_fixed_point(zlib):
    w = S.scaled(S.WORKLOADS["plain_256"], 1, 1)
    z1 = torch.from_numpy(w.packed_z()).cuda()
    z = z1.reshape(9, 1, 1).expand(9, 20, 30).contiguous()
    for method in (0, 1):
        out = zlib.nlm_wishart(z, 5, 4.0, 1.0, method)
        torch.cuda.synchronize()
        # the output is a ratio of two <= 121-term FP32 sums of one value with
        # equal weights: <= 2 gamma_123 relative
        assert torch.allclose(out, z, rtol=2 * gamma(123), atol=0)


def test_bad_arguments(zlib):
    z = torch.zeros((9, 8, 8), device="cuda")
    for kw in ({"radius": 4}, {"looks": 0.0}, {"h": -1.0}, {"method": 2}):
        args = {"radius": 3, "looks": 4.0, "h": 1.0, "method": 0}
        args.update(kw)
        with pytest.raises(RuntimeError):
            zlib.nlm_wishart(z, args["radius"], args["looks"], args["h"], args["method"])


@pytest.mark.parametrize("method", [0, 1])
def test_full_size_sampled(zlib, orc, method):
    """The benchmark's 1024 x 1024 image, radius 11 (23 x 23 window), in its
    launch configuration.  A pixel's output depends only on its search window,
    so corner, edge and interior pixels are checked against the oracle run on a
    crop holding that window (clipped by the image as the full image clips it)."""
    from paper_1807_08084_gb300.synth import gpu as G
    R, N = 11, 1024
    w = S.scaled(S.WORKLOADS["scale_16k"], N, N)
    z = G.packed_z(w)
    out = zlib.nlm_wishart(z, R, 16.0, 1.0, method).reshape(9, N, N)
    torch.cuda.synchronize()
    rng = np.random.default_rng(23)
    pts = [(0, 0), (0, N - 1), (N - 1, 0), (N - 1, N - 1), (5, 500), (700, N - 3)]
    pts += [tuple(int(v) for v in rng.integers(R, N - R, 2)) for _ in range(6)]
    for (y, x) in pts:
        y0, y1, x0, x1 = max(0, y - R), min(N, y + R + 1), max(0, x - R), min(N, x + R + 1)
        yy, xx = np.meshgrid(np.arange(y0, y1), np.arange(x0, x1), indexing="ij")
        crop = w.packed_z((yy * N + xx).ravel().astype(np.uint64))
        ch, cw = y1 - y0, x1 - x0
        ref_all = orc.nlm_wishart(crop, ch, cw, R, 16.0, 1.0)
        k = (y - y0) * cw + (x - x0)
        bound = nlm_bound(crop, ch, cw, R, 16.0, ref_all)[:, k]
        check(out[:, y, x].cpu().numpy(), ref_all[:, k], bound, f"pixel {(y, x)}: ")
