"""GPU parity of the nonlocal-means filter (nlm_wishart) against the FP64 oracle.

Weights exp(-L d / h) amplify errors of the pair log-determinants by L/h; the
FP32 routes compute them with relative error ~u cond (Cholesky) to ~u cond
(lmax/lmid) (plain cofactors), so the filtered output is compared with a
tolerance of 2e-3 relative to sqrt(Z'_ii Z'_jj), and the two methods must agree
with each other to the same bound.
"""
import numpy as np
import pytest
import torch

from paper_1807_08084_gb300 import synth as S

pytestmark = pytest.mark.gpu
TOL = 2e-3


def rel_err(out, ref):
    r = ref
    d = np.abs(out - r)
    sc = [r[0], None, None, None, None, r[5], None, None, r[8]]
    pairs = {1: (0, 5), 2: (0, 5), 3: (0, 8), 4: (0, 8), 6: (5, 8), 7: (5, 8)}
    e = [d[k] / (sc[k] if sc[k] is not None else np.sqrt(r[pairs[k][0]] * r[pairs[k][1]]))
         for k in range(9)]
    return np.max(np.stack(e), axis=0)


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
    e = rel_err(out.reshape(9, -1).cpu().numpy(), ref)
    assert e.max() <= TOL, f"max rel err {e.max():.3e}"


def test_methods_agree_and_repeat(zlib):
    w = S.scaled(S.WORKLOADS["scale_16k"], 96, 128)
    z = torch.from_numpy(w.packed_z()).cuda().reshape(9, 96, 128)
    a = zlib.nlm_wishart(z, 11, 16.0, 1.0, 0)
    b = zlib.nlm_wishart(z, 11, 16.0, 1.0, 1)
    a2 = zlib.nlm_wishart(z, 11, 16.0, 1.0, 0)
    torch.cuda.synchronize()
    assert torch.equal(a, a2)
    e = rel_err(a.reshape(9, -1).cpu().double().numpy(), b.reshape(9, -1).cpu().double().numpy())
    assert e.max() <= 2 * TOL


def test_constant_image_is_fixed_point(zlib):
    w = S.scaled(S.WORKLOADS["plain_256"], 1, 1)
    z1 = torch.from_numpy(w.packed_z()).cuda()
    z = z1.reshape(9, 1, 1).expand(9, 20, 30).contiguous()
    out = zlib.nlm_wishart(z, 5, 4.0, 1.0, 0)
    torch.cuda.synchronize()
    # the output is a ratio of two 121-term FP32 sums: <= 2 * 121 * 2^-24 relative
    assert torch.allclose(out, z, rtol=2 * 121 * 2.0 ** -24, atol=0)


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
        ref = orc.nlm_wishart(crop, ch, cw, R, 16.0, 1.0)[:, (y - y0) * cw + (x - x0)]
        got = out[:, y, x].cpu().numpy()
        assert rel_err(got[:, None], ref[:, None]).max() <= TOL, (y, x)
