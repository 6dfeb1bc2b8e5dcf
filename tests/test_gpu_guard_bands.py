"""Out-of-bounds write checks (guard bands) for every entry point's outputs.

No device memory checker runs with these tests, so each output is placed in a
larger buffer whose words before and after it, and between its planes when the
plane stride ld exceeds the pixel count, hold a sentinel bit pattern (a NaN no
kernel computes; 0xA5 for status bytes, which hold 0..3).  After the call every
sentinel word outside the output must be intact, and every word inside it must
have been written.  Shapes are ragged -- pixel counts that are not multiples of
four, images cut through tiles, strips and strip segments, planes padded apart,
workspaces sized exactly -- so the kernels' tails and borders are the code
under test, on both the 128-bit and the one-pixel paths.  Calls go through the
C ABI with raw pointers.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1807_08084_gb300 import synth as S

pytestmark = pytest.mark.gpu

GUARD = 64                   # sentinel words on each side (keeps 16-byte alignment)
SENT32 = 0x7FA5A5A5          # float32 words
SENT64 = 0x7FA5A5A5A5A5A5A5  # int64 / float64 words
SENT8 = 0xA5                 # status bytes
KINDS = {"f32": (torch.int32, SENT32), "f64": (torch.int64, SENT64),
         "i64": (torch.int64, SENT64), "u8": (torch.uint8, SENT8)}


class Out:
    """`planes` planes of `n` words, `ld` apart, inside a sentinel-filled buffer."""

    def __init__(self, n, kind="f32", planes=1, ld=None, host=False):
        ld = n if ld is None else ld
        dtype, self.sent = KINDS[kind]
        total = GUARD + (planes - 1) * ld + n + GUARD
        buf = torch.full((total,), self.sent, dtype=dtype)
        self.buf = buf.pin_memory() if host else buf.cuda()
        self.used = torch.zeros(total, dtype=torch.bool)
        for k in range(planes):
            self.used[GUARD + k * ld:GUARD + k * ld + n] = True
        self.ptr = self.buf.data_ptr() + GUARD * self.buf.element_size()

    def check(self, what, written=True):
        torch.cuda.synchronize()
        b = self.buf.cpu()
        assert bool((b[~self.used] == self.sent).all()), f"{what}: write outside the output"
        if written:
            assert bool((b[self.used] != self.sent).all()), f"{what}: output word not written"


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _packed(n, ld, workload="scale_16k", planes=9, seed_shift=0):
    """[planes][ld] device floats: n seeded pixels per block of nine planes, zero padding."""
    from dataclasses import replace
    w = S.WORKLOADS[workload]
    z = np.zeros((planes, ld), dtype=np.float32)
    for b in range(planes // 9):
        wb = replace(w, seed=w.seed + 17 * b + seed_shift)
        z[9 * b:9 * b + 9, :n] = wb.packed_z(np.arange(n, dtype=np.uint64))
    return torch.from_numpy(z).cuda()


@pytest.mark.parametrize("ld_extra", [5, 4])  # ld % 4 != 0 (one pixel) and == 0 (128-bit)
@pytest.mark.parametrize("route", ["plain", "comp", "comp_fp64", "chol"])
def test_zinv_det_outputs(zlib, route, ld_extra):
    lib = zlib.load()
    n = 4099
    ld = n + ld_extra
    z = _packed(n, ld)
    zi, dt = Out(n, planes=9, ld=ld), Out(n)
    st, cnt = Out(n, "u8"), Out(2, "i64")
    flags = {"plain": 0, "comp": 1, "comp_fp64": 3, "chol": 0}[route]
    fn = lib.chol_zinv_det if route == "chol" else lib.zinv_det
    assert fn(z.data_ptr(), n, ld, zi.ptr, dt.ptr, flags, 2.0 ** -10, st.ptr, cnt.ptr,
              _stream()) == 0
    for o, what in ((zi, "zinv"), (dt, "det"), (st, "status"), (cnt, "counts")):
        o.check(f"{route} {what}")


@pytest.mark.parametrize("ld_extra", [5, 4])
def test_zinv_det_bwd_output(zlib, ld_extra):
    lib = zlib.load()
    n = 4099
    ld = n + ld_extra
    z = _packed(n, ld)
    w = torch.empty_like(z)
    det = torch.empty(n, device="cuda")
    assert lib.zinv_det(z.data_ptr(), n, ld, w.data_ptr(), det.data_ptr(), 0, 0.0, None, None,
                        _stream()) == 0
    g = torch.rand((9, ld), device="cuda")
    gd, gl = torch.rand(n, device="cuda"), torch.rand(n, device="cuda")
    gz = Out(n, planes=9, ld=ld)
    assert lib.zinv_det_bwd(w.data_ptr(), det.data_ptr(), n, ld, g.data_ptr(), gd.data_ptr(),
                            gl.data_ptr(), gz.ptr, _stream()) == 0
    gz.check("g_z")


@pytest.mark.parametrize("ld_extra", [5, 4])
@pytest.mark.parametrize("nblocks", [1, 3])
def test_blockdiag_outputs(zlib, nblocks, ld_extra):
    lib = zlib.load()
    n = 4099
    ld = n + ld_extra
    z = _packed(n, ld, planes=9 * nblocks)
    zi, dt = Out(n, planes=9 * nblocks, ld=ld), Out(n)
    st, cnt = Out(n, "u8"), Out(2, "i64")
    assert lib.zinv_det_blockdiag(z.data_ptr(), nblocks, n, ld, zi.ptr, dt.ptr, 0, 0.0, st.ptr,
                                  cnt.ptr, _stream()) == 0
    for o, what in ((zi, "zinv"), (dt, "det"), (st, "status"), (cnt, "counts")):
        o.check(f"blockdiag {what}")


# 37 x 45 cuts every tile, strip and warp row; 300 x 130 adds a second strip
# segment (256 rows) and a 2-column last strip
@pytest.mark.parametrize("shape", [(37, 45), (300, 130)])
@pytest.mark.parametrize("win,weighted", [(3, False), (5, False), (7, False), (3, True),
                                          (5, True), (7, True), (9, True)])
def test_multilook_outputs(zlib, shape, win, weighted):
    lib = zlib.load()
    H, W = shape
    n = H * W
    s = torch.from_numpy(S.scaled(S.WORKLOADS["multilook_8k"], H, W).image()).cuda()
    wts = None
    if weighted:
        rng = np.random.default_rng(win)
        wts = torch.from_numpy(rng.uniform(0.5, 1.5, win * win).astype(np.float32)).cuda()
    zi, dt = Out(n, planes=9), Out(n)
    st, cnt = Out(n, "u8"), Out(2, "i64")
    assert lib.multilook_zinv_det(s.data_ptr(), H, W, n, win,
                                  None if wts is None else wts.data_ptr(), zi.ptr, dt.ptr, 1,
                                  2.0 ** -10, st.ptr, cnt.ptr, _stream()) == 0
    for o, what in ((zi, "zinv"), (dt, "det"), (st, "status"), (cnt, "counts")):
        o.check(f"multilook {what}")


@pytest.mark.parametrize("method", [0, 1])
@pytest.mark.parametrize("radius", [2, 11])
def test_nlm_output(zlib, radius, method):
    lib = zlib.load()
    H, W = 37, 45
    n = H * W
    z = _packed(n, n + 3)
    out = Out(n, planes=9)
    assert lib.nlm_wishart(z.data_ptr(), H, W, n + 3, radius, 16.0, 1.0, method, out.ptr,
                           _stream()) == 0
    out.check(f"nlm radius {radius} method {method}")


@pytest.mark.parametrize("dist,method", [(0, 2), (1, 0), (1, 1), (1, 2), (2, 0), (3, 0), (3, 1)])
@pytest.mark.parametrize("radius", [2, 11, 15])
def test_nlm_stochastic_output(zlib, radius, dist, method):
    """Hellinger, Kullback-Leibler and Renyi weights, and the compensated pair
    determinant; Kullback-Leibler runs 32-row tiles up to radius 11 and 16-row
    tiles at 15, both cut by 37 rows."""
    lib = zlib.load()
    H, W = 37, 45
    n = H * W
    z = _packed(n, n + 3)
    out = Out(n, planes=9)
    assert lib.nlm_stochastic(z.data_ptr(), H, W, n + 3, radius, 16.0, 0.5, dist, 0.7, method,
                              out.ptr, _stream()) == 0
    out.check(f"nlm_stochastic radius {radius} distance {dist} method {method}")


@pytest.mark.parametrize("shape", [(37, 45), (70, 100)])
@pytest.mark.parametrize("win", [3, 5, 7])
def test_wishart_outputs_and_workspace(zlib, shape, win):
    lib = zlib.load()
    H, W = shape
    n = H * W
    w = S.scaled(S.WORKLOADS["wishart_pair_4k"], H, W)
    s1, s2 = (torch.from_numpy(w.image(d)).cuda() for d in (0, 1))
    rng = np.random.default_rng(40 + win)
    wts = torch.from_numpy(rng.uniform(0.5, 1.5, win * win).astype(np.float32) / win**2).cuda()
    ws_bytes = lib.wishart_workspace_bytes(H, W, win)
    assert ws_bytes % 8 == 0
    # the workspace is scratch: only writes past its end are wrong
    ws = Out(ws_bytes // 8, "f64")
    q, loss = Out(n), Out(1, "f64")
    assert lib.wishart_stat_fwd(s1.data_ptr(), s2.data_ptr(), H, W, n, win, wts.data_ptr(), q.ptr,
                                loss.ptr, ws.ptr, ws_bytes, _stream()) == 0
    q.check("q_map")
    loss.check("loss")
    ws.check("workspace (forward)", written=False)
    g = torch.full((1,), 0.5, dtype=torch.float64, device="cuda")
    grad = Out(win * win)
    assert lib.wishart_stat_bwd(s1.data_ptr(), s2.data_ptr(), H, W, n, win, wts.data_ptr(),
                                g.data_ptr(), grad.ptr, ws.ptr, ws_bytes, _stream()) == 0
    grad.check("grad_weights")
    ws.check("workspace (backward)", written=False)
    # saved window covariances: the forward writes exactly the 18 planes of
    # z_saved; the backward reads them and keeps to its larger workspace
    zs = Out(n, planes=18)
    assert lib.wishart_stat_fwd_save(s1.data_ptr(), s2.data_ptr(), H, W, n, win, wts.data_ptr(),
                                     q.ptr, loss.ptr, zs.ptr, ws.ptr, ws_bytes, _stream()) == 0
    zs.check("z_saved")
    ws.check("workspace (forward, saving)", written=False)
    wsb_bytes = lib.wishart_bwd_saved_workspace_bytes(H, W, win)
    assert wsb_bytes % 8 == 0 and wsb_bytes >= ws_bytes + 72 * n
    wsb = Out(wsb_bytes // 8, "f64")
    grad2 = Out(win * win)
    assert lib.wishart_stat_bwd_saved(s1.data_ptr(), s2.data_ptr(), H, W, n, win, zs.ptr,
                                      g.data_ptr(), grad2.ptr, wsb.ptr, wsb_bytes, _stream()) == 0
    grad2.check("grad_weights (saved Z)")
    wsb.check("workspace (backward, saved Z)", written=False)
    zs.check("z_saved after the backward")


@pytest.mark.parametrize("staged", [False, True])
def test_host_streaming_outputs(zlib, staged):
    """Host buffers: the direct kernel writes host memory itself; the staged way
    copies chunk by chunk (a workspace of 1000 pixels leaves a ragged last chunk)."""
    lib = zlib.load()
    n = 4099
    ld = n + 5
    z = _packed(n, ld).cpu().pin_memory()
    zi, dt = Out(n, planes=9, ld=ld, host=True), Out(n, host=True)
    ws_bytes = lib.zinv_det_host_workspace_bytes(1000)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    flags = 4 if staged else 0
    assert lib.zinv_det_host(z.data_ptr(), n, ld, zi.ptr, dt.ptr, flags, 0.0,
                             ws.data_ptr() if staged else None, ws_bytes if staged else 0,
                             _stream()) == 0
    zi.check("host zinv")
    dt.check("host det")
