"""The allocation-free Wishart forward (wishart_stat_fwd_noalloc).

It serves callers that cannot give the library device scratch memory, such as
a plugin inside an application that owns all device allocations, or a loop
that must not allocate once running.  Its partial sums live in a fixed array
inside libzinv.so instead of a caller workspace.  This file is collected last
so that a run stopping at the first failure has already run every other test;
it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1807_08084_gb300 import synth as S

pytestmark = pytest.mark.gpu

Q_ABS = 2e-4  # per-pixel q between the two entry points (same kernel and reduction: same bits in practice)


def _entry(zp):
    lib = zp.load()
    f = lib.wishart_stat_fwd_noalloc
    P = ctypes.c_void_p
    f.argtypes = [P, P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, P, P, P, P]
    f.restype = ctypes.c_int
    return f


def test_noalloc_matches_workspace_entry(zlib):
    f = _entry(zlib)
    w = S.scaled(S.WORKLOADS["wishart_pair_4k"], 300, 700)
    s1 = torch.from_numpy(w.image(0)).cuda()
    s2 = torch.from_numpy(w.image(1)).cuda()
    rng = np.random.default_rng(21)
    wts = torch.from_numpy(rng.uniform(0.5, 1.5, 49).astype(np.float32) / 49).cuda()
    ref_loss, ref_q = zlib.wishart_stat_fwd(s1, s2, wts, 7, want_map=True)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):  # two calls in a row share the fixed scratch
        loss = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
        q = torch.full((w.H, w.W), float("nan"), device="cuda")
        rc = f(s1.data_ptr(), s2.data_ptr(), w.H, w.W, w.H * w.W, 7, wts.data_ptr(),
               q.data_ptr(), loss.data_ptr(), stream)
        assert rc == 0
        torch.cuda.synchronize()
        assert (q - ref_q).abs().max().item() <= Q_ABS
        assert abs(float(loss) - float(ref_loss)) <= Q_ABS * w.n
    # without the optional q map
    loss = torch.zeros((), dtype=torch.float64, device="cuda")
    assert f(s1.data_ptr(), s2.data_ptr(), w.H, w.W, w.H * w.W, 7, wts.data_ptr(), None,
             loss.data_ptr(), stream) == 0
    torch.cuda.synchronize()
    assert abs(float(loss) - float(ref_loss)) <= Q_ABS * w.n


def test_noalloc_rejects_images_beyond_its_scratch(zlib):
    f = _entry(zlib)
    s = torch.zeros((3, 1, 1), dtype=torch.complex64, device="cuda")
    wts = torch.full((49,), 1 / 49, device="cuda")
    loss = torch.zeros((), dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # 8200 x 8192 needs 513 x 256 tiles > 131072: refused before any device work
    H, W = 8200, 8192
    assert f(s.data_ptr(), s.data_ptr(), H, W, H * W, 7, wts.data_ptr(), None, loss.data_ptr(),
             stream) == -1


def test_noalloc_at_its_maximum_size(zlib):
    """8192 x 8192 pixels take all 131072 tiles of the fixed scratch: the largest
    image the entry point accepts.  Same kernel and the same fixed-order reduction
    as wishart_stat_fwd, so the loss and the q map are the same bits."""
    from paper_1807_08084_gb300.synth import gpu as G
    f = _entry(zlib)
    w = S.scaled(S.WORKLOADS["wishart_pair_4k"], 8192, 8192)
    s1, s2 = G.image(w, 0), G.image(w, 1)
    wts = torch.full((49,), 1 / 49, device="cuda")
    ref_loss, ref_q = zlib.wishart_stat_fwd(s1, s2, wts, 7, want_map=True)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    loss = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
    q = torch.full((w.H, w.W), float("nan"), device="cuda")
    assert f(s1.data_ptr(), s2.data_ptr(), w.H, w.W, w.H * w.W, 7, wts.data_ptr(), q.data_ptr(),
             loss.data_ptr(), stream) == 0
    torch.cuda.synchronize()
    assert float(loss) == float(ref_loss)
    assert torch.equal(q, ref_q)
