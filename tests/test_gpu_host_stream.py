"""Oracle parity of zinv_det_host, the host-buffer path of §4.3 (an image that
does not fit is streamed through the GPU in pieces), through the C ABI.

The other host tests compare this path with the device kernel; these compare
it with the FP64 oracle, so a slip that only the host path can make -- a
chunk landing at the wrong host offset, a plane stride taken as n instead of
ld -- fails here.  Host buffers have plane stride ld > n with ld % 4 != 0, the
workspace holds three chunks of a few thousand pixels (the image is dozens of
chunks, the last one ragged), and the words between the planes hold a sentinel
that must survive.  Every pixel is checked against the oracle at 1e-5 cond,
so the first and last pixel of every chunk are among them.  Both ways are run:
the staged one (copies through the workspace on three streams; forced with
HOST_STAGED, or because the buffers are pageable) and the direct one (the
kernel reads and writes page-locked host memory).
"""
import ctypes

import numpy as np
import pytest
import torch

from helpers import det_err, inv_err

from paper_1807_08084_gb300 import synth as S

pytestmark = pytest.mark.gpu

TOL = 1e-5
SENT = 0x7FA5A5A5  # a NaN bit pattern no kernel writes


def host_planes(z_np, ld, pinned):
    """[9 * ld] float32 host buffer: plane k at k * ld, sentinel words between planes."""
    n = z_np.shape[1]
    buf = torch.full((9 * ld,), SENT, dtype=torch.int32).view(torch.float32)
    buf = buf.pin_memory() if pinned else buf.clone()
    for k in range(9):
        buf[k * ld:k * ld + n] = torch.from_numpy(np.ascontiguousarray(z_np[k]))
    return buf


def sentinel_buf(words, pinned):
    buf = torch.full((words,), SENT, dtype=torch.int32).view(torch.float32)
    return buf.pin_memory() if pinned else buf.clone()


def planes_of(buf, n, ld):
    return buf.view(9, ld)[:, :n].numpy().astype(np.float64)


def gaps_intact(buf, n, ld):
    gaps = buf.view(torch.int32).view(9, ld)[:, n:]
    return bool((gaps == SENT).all())


def run_host(zlib, z_np, ld, flags, chunk, pinned, direct=False):
    """One zinv_det_host call through the C ABI; returns (zinv [9, n], det [n])
    after checking that nothing outside the outputs was written."""
    lib = zlib.load()
    n = z_np.shape[1]
    z_h = host_planes(z_np, ld, pinned)
    zinv_h = sentinel_buf(9 * ld, pinned)
    det_h = sentinel_buf(n + 8, pinned)
    ws = None
    if not direct:
        ws = torch.empty(lib.zinv_det_host_workspace_bytes(chunk), dtype=torch.uint8,
                         device="cuda")
    P = ctypes.c_void_p
    stream = P(torch.cuda.current_stream().cuda_stream)
    rc = lib.zinv_det_host(P(z_h.data_ptr()), n, ld, P(zinv_h.data_ptr()), P(det_h.data_ptr()),
                           flags, zlib.DEFAULT_TAU, None if ws is None else P(ws.data_ptr()),
                           0 if ws is None else ws.numel(), stream)
    assert rc == 0, zlib.status_string(rc)
    torch.cuda.synchronize()
    assert gaps_intact(zinv_h, n, ld), "a write landed between the output planes"
    assert bool((det_h.view(torch.int32)[n:] == SENT).all()), "a write landed after det"
    assert torch.equal(z_h.view(torch.int32).view(9, ld)[:, n:],
                       torch.full((9, ld - n), SENT, dtype=torch.int32)), "input modified"
    return planes_of(zinv_h, n, ld), det_h[:n].numpy().astype(np.float64)


def check_oracle(orc, z_np, zinv, det):
    ref_inv, ref_det = orc.zinv_det(z_np)
    cond = orc.cond(z_np)
    pd = np.isfinite(cond) & (ref_det > 0)
    assert pd.all()
    ei = inv_err(zinv, ref_inv)
    ed = det_err(det, ref_det)
    bad = ~((ei <= TOL * cond) & (ed <= TOL * cond))
    assert not bad.any(), (f"{bad.sum()} of {bad.size} pixels out of tolerance; first at "
                           f"{np.flatnonzero(bad)[:8]}")


# (workload, flags): the Wishart image of the fixed Sigma in plain FP32, and the
# cond-controlled image (cond up to 1e7, half the pixels flagged) with the
# compensated route and the FP64 recompute, which meet 1e-5 cond on every pixel.
CASES = {
    "plain": ("plain_256", 0),
    "compensated_fp64": ("precision_4k", 3),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("way", ["staged_pinned", "staged_pageable", "direct"])
def test_host_stream_matches_oracle(zlib, orc, case, way):
    workload, flags = CASES[case]
    n = 200_003
    ld = n + 2                           # ld > n, ld % 4 == 1
    assert ld % 4 != 0
    chunk = 4099                         # the library rounds it down to 4096: 49 chunks
    w = S.WORKLOADS[workload]
    z_np = w.packed_z(np.arange(n, dtype=np.uint64))
    if way == "staged_pinned":
        zinv, det = run_host(zlib, z_np, ld, flags | zlib.HOST_STAGED, chunk, pinned=True)
    elif way == "staged_pageable":
        zinv, det = run_host(zlib, z_np, ld, flags, chunk, pinned=False)
    else:
        zinv, det = run_host(zlib, z_np, ld, flags, chunk, pinned=True, direct=True)
    check_oracle(orc, z_np, zinv, det)


def test_host_stream_image_much_larger_than_workspace(zlib, orc):
    """A 2,000,001-pixel image (72 MB of input) through a workspace of three
    1,000-pixel chunks (0.12 MB): 2,000 chunks, the last of one pixel.  Every
    pixel against the oracle, and the staged result equals the direct one bit
    for bit."""
    n = 2_000_001
    ld = n + 3
    w = S.WORKLOADS["scale_16k"]
    from paper_1807_08084_gb300.synth import gpu as G
    from dataclasses import replace
    # the first n pixels of a scale_16k-style image, generated on the GPU twin
    z_dev = G.packed_z(S.scaled(replace(w), 2048, 1024))
    z_np = z_dev.reshape(9, -1)[:, :n].cpu().numpy()
    zinv_s, det_s = run_host(zlib, z_np, ld, zlib.HOST_STAGED, 1000, pinned=True)
    zinv_d, det_d = run_host(zlib, z_np, ld, 0, 0, pinned=True, direct=True)
    assert np.array_equal(zinv_s, zinv_d) and np.array_equal(det_s, det_d)
    check_oracle(orc, z_np, zinv_s, det_s)
