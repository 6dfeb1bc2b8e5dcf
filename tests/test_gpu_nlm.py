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
    for kw in ({"radius": 4}, {"looks": 0.0}, {"h": -1.0}, {"method": 3}):
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


# ---------------------------------------------------------------------------
# nlm_stochastic: Hellinger and Kullback-Leibler weights
# ---------------------------------------------------------------------------
BHATTACHARYYA, HELLINGER, KULLBACK_LEIBLER, RENYI = 0, 1, 2, 3


def inv3_with_magnitudes(Z):
    """Exact (FP64) packed inverse of packed Z [9, ...], the magnitude sums S_k
    of the three products in each cofactor of the compensated inverse (same
    packed order), and the det with its expansion's magnitude sum E."""
    a, br, bi, cr, ci, d, er, ei, f = Z
    cof = np.stack([d * f - er * er - ei * ei, cr * er + ci * ei - br * f,
                    ci * er - cr * ei - bi * f, br * er - bi * ei - cr * d,
                    br * ei + bi * er - ci * d, a * f - cr * cr - ci * ci,
                    cr * br + ci * bi - a * er, ci * br - cr * bi - a * ei,
                    a * d - br * br - bi * bi])
    A = np.abs
    S = np.stack([A(d * f) + er * er + ei * ei, A(cr * er) + A(ci * ei) + A(br * f),
                  A(ci * er) + A(cr * ei) + A(bi * f), A(br * er) + A(bi * ei) + A(cr * d),
                  A(br * ei) + A(bi * er) + A(ci * d), A(a * f) + cr * cr + ci * ci,
                  A(cr * br) + A(ci * bi) + A(a * er), A(ci * br) + A(cr * bi) + A(a * ei),
                  A(a * d) + br * br + bi * bi])
    det = det3(Z)
    ab, ac, ae = A(br) + A(bi), A(cr) + A(ci), A(er) + A(ei)
    E = a * (d * f + ae * ae) + ab * (ac * ae + ab * f) + ac * (ab * ae + ac * d)
    return cof / det, S, det, E


def _expansion_magnitude(m):
    """The cofactor expansion of det over packed entries taken in magnitude
    (packed [9, ...] of nonnegative entry magnitudes; complex entries as
    |Re| + |Im|)."""
    a, ab, ac, d, ae, f = m[0], m[1] + m[2], m[3] + m[4], m[5], m[6] + m[7], m[8]
    return a * (d * f + ae * ae) + ab * (ac * ae + ab * f) + ac * (ab * ae + ac * d)


def stochastic_bound(z, H, W, radius, L, h, dist, ref, order=0.5, method=0):
    """[9, H*W] first-order error bound of the FP32 filter with weights
    w_ij = exp(-d_ij / h).  A relative error delta_ij of w_ij moves
    Z'_i = sum_j w_ij Z_j / sum_j w_ij by at most
        sum_j w_ij delta_ij |Z_jc - Z'_ic| / sum_j w_ij
    (the exact weights from the FP64 distances), plus the FP32 rounding of the
    two weighted sums, 2 gamma_(n_i + 2) max_j |Z_jc|.  Per pair:
      Bhattacharyya   delta = (L/h) ln2 e + 2^-22, e the error of t as for nlm_wishart;
      Hellinger       w = 2^(-(log2 e / h)(1 - x)), x = 2^(-L t) <= 1; over the
                      interval t +- e the derivative of x is at most
                      L ln2 x_m, x_m = min(1, x 2^(L e)), so
                      delta = min(1, x_m (L ln2 e + d_B u + 2^-22) + 3u) / h + 2^-22;
      Kullback-Leibler  t = (tr(I_i Z_j) + tr(I_j Z_i)) / 2 - 3 with I the
                      compensated inverse, |dI_k| <= 6u |I_k| + 2 gamma_3^2 (S_k + E |I_k|) / det
                      (Dot2 cofactors and det), each trace a 9-term FP32 FMA chain
                      (error <= sum c_k |dI_k| |Z_k| + gamma_9 sum c_k |I_k| |Z_k|,
                      c_k = 2 off the diagonal), t rounded once more:
                      e <= (dtr1 + dtr2 + u |tr1 + tr2|) / 2 + u |t|,
                      delta = (L/h)(e + 2u t) + 2^-22;
      Renyi (order b) M1 = (1-b) Z_i + b Z_j, M2 = b Z_i + (1-b) Z_j, each entry
                      within 3u of its magnitude m (1 - b, the product and the
                      FMA rounded), so det M_k errs by <= gamma_16 E(M_k)
                      + 9u E(m_k) (E: the expansion in magnitudes);
                      e = (e1 + e2)/2 + 4u (|log2 D1 + log2 D2|/2 + |h_i| + |h_j|),
                      e_k = that / (D_k ln2) + 2^-21, delta = p ln2 (e + u t) + 2^-22
                      with p = L / ((1-b) h);
      compensated pair det (method 2, Bhattacharyya and Hellinger): the pair sum
                      is exact (hi + lo); det(hi) by Dot2 (cofactors of three
                      products, then about ten products with their low parts)
                      errs by <= u D + 2 gamma_10^2 E, the first-order lo term
                      by O(u^2 E) more, so
                      e = (u + 2 gamma_10^2 E / D) / ln2 + 4u (|log2 D| + 3 + |h_i| + |h_j|)
                      + 2^-21 (the fast log2 and the lo / hi term), then delta as above.
    The half log-dets h of the determinant-based distances come from the same
    compensated route on each pixel: each adds (u + 2 gamma_10^2 E_z / D_z) / (2 ln2)
    to e (negligible beside the plain routes' pair det, not beside method 2's).
    The test bound is 1.25 times the total."""
    Z = np.asarray(z, dtype=np.float64).reshape(9, H, W)
    R = np.asarray(ref, dtype=np.float64).reshape(9, H, W)
    hz = np.abs(np.log2(det3(Z))) / 2
    ldz = np.log(det3(Z))
    eh = (U + 2 * gamma(10) ** 2 * _expansion_magnitude(np.abs(Z)) / det3(Z)) / (2 * np.log(2))
    if dist == KULLBACK_LEIBLER:
        I, S, dz, Ez = inv3_with_magnitudes(Z)
        dI = 6 * U * np.abs(I) + 2 * gamma(3) ** 2 * (S + Ez * np.abs(I)) / dz
        ck = np.array([1, 2, 2, 2, 2, 1, 2, 2, 1], dtype=np.float64)[:, None, None]
    num = np.zeros((9, H, W))
    den = np.zeros((H, W))
    mag = np.zeros((9, H, W))
    count = np.zeros((H, W))
    for dy in range(-radius, radius + 1):
        for dx in range(-radius, radius + 1):
            ys = slice(max(0, -dy), min(H, H - dy))
            xs = slice(max(0, -dx), min(W, W - dx))
            yj = slice(max(0, dy), min(H, H + dy))
            xj = slice(max(0, dx), min(W, W + dx))
            zi, zj = Z[:, ys, xs], Z[:, yj, xj]
            if dist == RENYI:
                b, b1 = order, 1 - order
                pr = L / (b1 * h)
                t = -(0.5 * (ldz[ys, xs] + ldz[yj, xj])) / np.log(2)
                ek = 0.0
                lsum = 0.0
                for (ca, cb) in ((b1, b), (b, b1)):
                    M = ca * zi + cb * zj
                    D = det3(M)
                    mag_m = ca * np.abs(zi) + cb * np.abs(zj)
                    ek = ek + 0.5 * ((gamma(16) * _expansion_magnitude(np.abs(M))
                                      + 9 * U * _expansion_magnitude(mag_m)) / (D * np.log(2))
                                     + 2.0 ** -21)
                    lsum = lsum + np.log2(D)
                    t = t + 0.5 * np.log2(D)
                e = ek + 4 * U * (np.abs(lsum) / 2 + hz[ys, xs] + hz[yj, xj])
                t = np.maximum(t, 0)
                delta = pr * np.log(2) * (e + U * t) + 2.0 ** -22
                d = pr * h * np.log(2) * t
            elif dist == KULLBACK_LEIBLER:
                Ii, Ij = I[:, ys, xs], I[:, yj, xj]
                tr1 = (ck * Ii * zj).sum(axis=0)
                tr2 = (ck * Ij * zi).sum(axis=0)
                dtr1 = (ck * dI[:, ys, xs] * np.abs(zj)).sum(axis=0) \
                    + gamma(9) * (ck * np.abs(Ii * zj)).sum(axis=0)
                dtr2 = (ck * dI[:, yj, xj] * np.abs(zi)).sum(axis=0) \
                    + gamma(9) * (ck * np.abs(Ij * zi)).sum(axis=0)
                t = 0.5 * (tr1 + tr2) - 3
                e = 0.5 * (dtr1 + dtr2 + U * np.abs(tr1 + tr2)) + U * np.abs(t)
                delta = (L / h) * (e + 2 * U * np.abs(t)) + 2.0 ** -22
                d = L * np.maximum(t, 0)
            else:
                s = zi + zj
                a, br, bi, cr, ci, dd, er, ei, f = s
                det = det3(s)
                ab, ac, ae = np.abs(br) + np.abs(bi), np.abs(cr) + np.abs(ci), np.abs(er) + np.abs(ei)
                E = a * (dd * f + ae * ae) + ab * (ac * ae + ab * f) + ac * (ab * ae + ac * dd)
                if method == 2:
                    e = ((U + 2 * gamma(10) ** 2 * E / det) / np.log(2) + 2.0 ** -21
                         + 4 * U * (np.abs(np.log2(det)) + 3 + hz[ys, xs] + hz[yj, xj]))
                else:
                    e = (gamma(16) * E / (det * np.log(2)) + 2.0 ** -21
                         + 4 * U * (np.abs(np.log2(det)) + 3 + hz[ys, xs] + hz[yj, xj]))
                e = e + eh[ys, xs] + eh[yj, xj]
                dB = L * np.maximum(np.log(det / 8) - 0.5 * (ldz[ys, xs] + ldz[yj, xj]), 0)
                if dist == HELLINGER:
                    xm = np.minimum(1.0, np.exp(-dB) * 2.0 ** np.minimum(L * e, 60.0))
                    dh = np.minimum(1.0, xm * (L * np.log(2) * e + dB * U + 2.0 ** -22) + 3 * U)
                    delta = dh / h + 2.0 ** -22
                    d = 1 - np.exp(-dB)
                else:
                    delta = (L / h) * np.log(2) * e + 2.0 ** -22
                    d = dB
            w = np.exp(-d / h)
            num[:, ys, xs] += (w * delta)[None] * np.abs(zj - R[:, ys, xs])
            den[ys, xs] += w
            mag[:, ys, xs] = np.maximum(mag[:, ys, xs], np.abs(zj))
            count[ys, xs] += 1
    b = num / den[None] + 2 * gamma(count + 2)[None] * mag
    return 1.25 * b.reshape(9, -1)


def test_renyi_order_one_half_is_bhattacharyya_with_half_h(zlib, orc):
    """d_R(1/2) = 2 d_B, so Renyi of order 1/2 with h is the Bhattacharyya
    filter with h/2: the two kernels (two pair determinants vs one) agree
    within both bounds."""
    H, W = 37, 70
    w = S.scaled(S.WORKLOADS["scale_16k"], H, W)
    z_np = w.packed_z()
    z = torch.from_numpy(z_np).cuda().reshape(9, H, W)
    a = zlib.nlm_stochastic(z, 3, 16.0, 2.0, RENYI, 0, order=0.5)
    b = zlib.nlm_wishart(z, 3, 16.0, 1.0, 0)
    torch.cuda.synchronize()
    ref = orc.nlm_stochastic(z_np, H, W, 3, 16.0, 1.0, BHATTACHARYYA)
    bound = (stochastic_bound(z_np, H, W, 3, 16.0, 2.0, RENYI, ref, 0.5)
             + stochastic_bound(z_np, H, W, 3, 16.0, 1.0, BHATTACHARYYA, ref))
    check(a.reshape(9, -1).cpu().numpy(), b.reshape(9, -1).cpu().double().numpy(), bound)


def test_bhattacharyya_is_the_log_det_filter(zlib):
    """nlm_stochastic with the Bhattacharyya distance runs nlm_wishart's kernel."""
    H, W = 40, 75
    w = S.scaled(S.WORKLOADS["scale_16k"], H, W)
    z = torch.from_numpy(w.packed_z()).cuda().reshape(9, H, W)
    for method in (0, 1):
        a = zlib.nlm_wishart(z, 7, 16.0, 1.0, method)
        b = zlib.nlm_stochastic(z, 7, 16.0, 1.0, BHATTACHARYYA, method)
        torch.cuda.synchronize()
        assert torch.equal(a, b)


@pytest.mark.parametrize("radius", [1, 3, 11])
@pytest.mark.parametrize("dist,method,h", [(HELLINGER, 0, 0.25), (HELLINGER, 1, 0.25),
                                           (KULLBACK_LEIBLER, 0, 4.0), (RENYI, 0, 2.0),
                                           (RENYI, 1, 2.0)])
def test_stochastic_vs_oracle(zlib, orc, radius, dist, method, h):
    """Every output pixel of a ragged 37 x 70 image (two partial tiles in x, a
    ragged row pair) against the FP64 oracle under the derived bound.  The
    Hellinger distance lies in [0, 1), so its h is smaller; both h move the
    outputs by 10-20% of their scale (the filter does work)."""
    H, W = 37, 70
    w = S.scaled(S.WORKLOADS["scale_16k"], H, W)
    z_np = w.packed_z()
    z = torch.from_numpy(z_np).cuda().reshape(9, H, W)
    out = zlib.nlm_stochastic(z, radius, 16.0, h, dist, method, order=0.7)
    torch.cuda.synchronize()
    ref = orc.nlm_stochastic(z_np, H, W, radius, 16.0, h, dist, 0.7)
    check(out.reshape(9, -1).cpu().numpy(), ref,
          stochastic_bound(z_np, H, W, radius, 16.0, h, dist, ref, 0.7))


@pytest.mark.parametrize("dist,h,method", [(HELLINGER, 0.25, 0), (KULLBACK_LEIBLER, 4.0, 0),
                                           (RENYI, 2.0, 0), (RENYI, 2.0, 1)])
def test_stochastic_full_size_sampled(zlib, orc, dist, h, method):
    """The benchmark's 1024 x 1024 image, radius 11, in its launch
    configuration: corner, edge and interior pixels against the oracle run on a
    crop holding the pixel's search window."""
    from paper_1807_08084_gb300.synth import gpu as G
    R, N = 11, 1024
    w = S.scaled(S.WORKLOADS["scale_16k"], N, N)
    z = G.packed_z(w)
    out = zlib.nlm_stochastic(z, R, 16.0, h, dist, method, order=0.7).reshape(9, N, N)
    torch.cuda.synchronize()
    rng = np.random.default_rng(29)
    pts = [(0, 0), (0, N - 1), (N - 1, 0), (N - 1, N - 1), (11, 511), (1012, 3)]
    pts += [tuple(int(v) for v in rng.integers(R, N - R, 2)) for _ in range(6)]
    for (y, x) in pts:
        y0, y1, x0, x1 = max(0, y - R), min(N, y + R + 1), max(0, x - R), min(N, x + R + 1)
        yy, xx = np.meshgrid(np.arange(y0, y1), np.arange(x0, x1), indexing="ij")
        crop = w.packed_z((yy * N + xx).ravel().astype(np.uint64))
        ch, cw = y1 - y0, x1 - x0
        ref_all = orc.nlm_stochastic(crop, ch, cw, R, 16.0, h, dist, 0.7)
        k = (y - y0) * cw + (x - x0)
        bound = stochastic_bound(crop, ch, cw, R, 16.0, h, dist, ref_all, 0.7)[:, k]
        check(out[:, y, x].cpu().numpy(), ref_all[:, k], bound, f"pixel {(y, x)}: ")


@pytest.mark.parametrize("dist", [HELLINGER, KULLBACK_LEIBLER, RENYI])
def test_stochastic_constant_image_is_fixed_point(zlib, dist):
    w = S.scaled(S.WORKLOADS["plain_256"], 1, 1)
    z1 = torch.from_numpy(w.packed_z()).cuda()
    z = z1.reshape(9, 1, 1).expand(9, 20, 30).contiguous()
    out = zlib.nlm_stochastic(z, 5, 4.0, 0.5, dist, 0, order=0.7)
    torch.cuda.synchronize()
    # equal weights up to rounding of d near 0: the output is a weighted mean
    # of one value, within 2 gamma_123 of it
    assert torch.allclose(out, z, rtol=2 * gamma(123), atol=0)


def test_stochastic_bad_arguments(zlib):
    z = torch.zeros((9, 8, 8), device="cuda")
    for dist, method in ((4, 0), (-1, 0), (KULLBACK_LEIBLER, 1), (HELLINGER, 3),
                         (RENYI, 2)):
        with pytest.raises(RuntimeError):
            zlib.nlm_stochastic(z, 3, 4.0, 1.0, dist, method)
    for order in (0.0, 1.0, -0.5, float("inf")):
        with pytest.raises(RuntimeError):
            zlib.nlm_stochastic(z, 3, 4.0, 1.0, RENYI, 0, order=order)


def ill_conditioned_image(H, W, cond=1e3, looks=16, seed=31):
    """[9, H*W] FP32 sample covariances of `looks` looks of one Sigma =
    U diag(1, cond^-1/2, 1/cond) U^H (U a seeded Haar matrix): neighbours are
    close in the Wishart sense, every pixel is ill-conditioned."""
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
    Q, R = np.linalg.qr(G)
    Q = Q * (np.diag(R) / np.abs(np.diag(R)))
    Sig = (Q * np.array([1.0, cond ** -0.5, 1.0 / cond])) @ Q.conj().T
    C = np.linalg.cholesky(Sig)
    g = (rng.standard_normal((H * W, looks, 3)) + 1j * rng.standard_normal((H * W, looks, 3))) / np.sqrt(2)
    s = g @ C.T
    Z = np.einsum("nli,nlj->nij", s, s.conj()) / looks
    return np.stack([Z[:, 0, 0].real, Z[:, 0, 1].real, Z[:, 0, 1].imag, Z[:, 0, 2].real,
                     Z[:, 0, 2].imag, Z[:, 1, 1].real, Z[:, 1, 2].real, Z[:, 1, 2].imag,
                     Z[:, 2, 2].real]).astype(np.float32)


@pytest.mark.parametrize("dist,method,h,order", [(BHATTACHARYYA, 0, 1.0, 0.5),
                                                 (BHATTACHARYYA, 1, 1.0, 0.5),
                                                 (HELLINGER, 0, 0.25, 0.5),
                                                 (KULLBACK_LEIBLER, 0, 4.0, 0.5),
                                                 (RENYI, 0, 2.0, 0.1), (RENYI, 1, 2.0, 0.1),
                                                 (RENYI, 0, 8.0, 0.95)])
def test_stochastic_ill_conditioned_vs_oracle(zlib, orc, dist, method, h, order):
    """Every pixel of a 24 x 40 image of 16-look covariances of one Sigma with
    cond 1e3 against the oracle under the derived bounds (the determinants'
    and traces' cond-dependent terms are the ones exercised), for every
    distance and Renyi orders near 0 and 1.  From cond ~1e4 the bounds of the
    determinant-based distances exceed the data's scale: rounding the FP32
    pair sum alone moves det(Z_i + Z_j) by up to u E / D relative."""
    H, W = 24, 40
    z_np = ill_conditioned_image(H, W)
    z = torch.from_numpy(z_np).cuda().reshape(9, H, W)
    out = zlib.nlm_stochastic(z, 3, 16.0, h, dist, method, order=order)
    torch.cuda.synchronize()
    ref = orc.nlm_stochastic(z_np, H, W, 3, 16.0, h, dist, order)
    assert np.median(np.abs(ref - z_np).max(axis=0) / np.abs(ref).max(axis=0)) > 1e-3  # it filters
    check(out.reshape(9, -1).cpu().numpy(), ref,
          stochastic_bound(z_np, H, W, 3, 16.0, h, dist, ref, order))


@pytest.mark.parametrize("dist,method,h", [(BHATTACHARYYA, 0, 1.0), (BHATTACHARYYA, 1, 1.0),
                                           (KULLBACK_LEIBLER, 0, 4.0), (RENYI, 0, 2.0)])
def test_largest_radius_vs_oracle(zlib, orc, dist, method, h):
    """Radius 15 (31 x 31 windows; Kullback-Leibler's 16-row tiles) on the
    ragged 37 x 70 image: every output against the oracle."""
    H, W = 37, 70
    w = S.scaled(S.WORKLOADS["scale_16k"], H, W)
    z_np = w.packed_z()
    z = torch.from_numpy(z_np).cuda().reshape(9, H, W)
    out = zlib.nlm_stochastic(z, 15, 16.0, h, dist, method, order=0.7)
    torch.cuda.synchronize()
    ref = orc.nlm_stochastic(z_np, H, W, 15, 16.0, h, dist, 0.7)
    check(out.reshape(9, -1).cpu().numpy(), ref,
          stochastic_bound(z_np, H, W, 15, 16.0, h, dist, ref, 0.7))


COMPENSATED = 2


@pytest.mark.parametrize("cond", [1e5, 1e6])
@pytest.mark.parametrize("dist,h", [(BHATTACHARYYA, 1.0), (HELLINGER, 0.25)])
def test_compensated_ill_conditioned_vs_oracle(zlib, orc, cond, dist, h):
    """The compensated pair determinant on 16-look covariances of one Sigma
    with cond 1e5 and 1e6, where the plain route's bounds exceed the data's
    scale: every output against the oracle under the derived bound."""
    H, W = 24, 40
    z_np = ill_conditioned_image(H, W, cond=cond)
    z = torch.from_numpy(z_np).cuda().reshape(9, H, W)
    out = zlib.nlm_stochastic(z, 3, 16.0, h, dist, COMPENSATED)
    torch.cuda.synchronize()
    ref = orc.nlm_stochastic(z_np, H, W, 3, 16.0, h, dist)
    assert np.median(np.abs(ref - z_np).max(axis=0) / np.abs(ref).max(axis=0)) > 1e-3
    bound = stochastic_bound(z_np, H, W, 3, 16.0, h, dist, ref, method=COMPENSATED)
    assert np.median(bound.max(axis=0) / np.abs(ref).max(axis=0)) < 1e-2  # a real constraint
    check(out.reshape(9, -1).cpu().numpy(), ref, bound)


@pytest.mark.parametrize("radius", [1, 11])
@pytest.mark.parametrize("dist,h", [(BHATTACHARYYA, 1.0), (HELLINGER, 0.25)])
def test_compensated_vs_oracle(zlib, orc, radius, dist, h):
    """The compensated pair determinant on the ragged 37 x 70 class image."""
    H, W = 37, 70
    w = S.scaled(S.WORKLOADS["scale_16k"], H, W)
    z_np = w.packed_z()
    z = torch.from_numpy(z_np).cuda().reshape(9, H, W)
    out = zlib.nlm_stochastic(z, radius, 16.0, h, dist, COMPENSATED)
    torch.cuda.synchronize()
    ref = orc.nlm_stochastic(z_np, H, W, radius, 16.0, h, dist)
    check(out.reshape(9, -1).cpu().numpy(), ref,
          stochastic_bound(z_np, H, W, radius, 16.0, h, dist, ref, method=COMPENSATED))


def test_compensated_through_nlm_wishart(zlib):
    """nlm_wishart's method 2 is nlm_stochastic's compensated Bhattacharyya
    filter; the other distances refuse method 2."""
    H, W = 40, 75
    w = S.scaled(S.WORKLOADS["scale_16k"], H, W)
    z = torch.from_numpy(w.packed_z()).cuda().reshape(9, H, W)
    a = zlib.nlm_wishart(z, 5, 16.0, 1.0, COMPENSATED)
    b = zlib.nlm_stochastic(z, 5, 16.0, 1.0, BHATTACHARYYA, COMPENSATED)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    for dist in (KULLBACK_LEIBLER, RENYI):
        with pytest.raises(RuntimeError):
            zlib.nlm_stochastic(z, 5, 16.0, 1.0, dist, COMPENSATED)

