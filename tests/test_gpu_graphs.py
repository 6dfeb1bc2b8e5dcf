"""The entry points inside CUDA graphs: each family is captured in one graph
(torch's default, global capture mode), replayed twice, and must give the bits
of the eager calls.  Launch-bound loops (the 256 x 256 latency workload) rely
on this."""
import numpy as np
import pytest
import torch

from paper_1807_08084_gb300 import synth as S

pytestmark = pytest.mark.gpu


def _inputs():
    from paper_1807_08084_gb300.synth import gpu as G
    wz = S.scaled(S.WORKLOADS["scale_16k"], 96, 128)
    z = G.packed_z(wz)
    wp = S.scaled(S.WORKLOADS["wishart_pair_4k"], 48, 80)
    s1, s2 = G.image(wp, 0), G.image(wp, 1)
    blocks = torch.stack([G.packed_z(S.scaled(S.WORKLOADS["scale_16k"], 64, 64))] * 3)
    wts = torch.from_numpy(np.random.default_rng(5).uniform(0.5, 1.5, 25).astype(np.float32)
                           / 25).cuda()
    g = torch.rand((9, 96, 128), device="cuda")
    return z, s1, s2, blocks, wts, g


def _run(zlib, z, s1, s2, blocks, wts, g):
    """One pass over the entry point families; returns every output."""
    out = []
    zinv, det, st, cnt = zlib.zinv_det(z, zlib.COMPENSATED | zlib.FP64_RECOMPUTE,
                                       want_status=True, want_counts=True)
    out += [zinv, det, st, cnt]
    out += list(zlib.chol_zinv_det(z))
    out.append(zlib.zinv_det_bwd(zinv, det, g_zinv=g))
    out += list(zlib.zinv_det_blockdiag(blocks))[:2]
    out += list(zlib.multilook_zinv_det(s1, 7))[:2]
    out += list(zlib.multilook_zinv_det(s1, 5, wts))[:2]
    out.append(zlib.nlm_wishart(z, 3, 16.0, 1.0, zlib.NLM_ADJUGATE))
    out.append(zlib.nlm_stochastic(z, 3, 16.0, 4.0, zlib.NLM_KULLBACK_LEIBLER))
    out.append(zlib.nlm_stochastic(z, 3, 16.0, 2.0, zlib.NLM_RENYI, order=0.7))
    out.append(zlib.nlm_stochastic(z, 3, 16.0, 1.0, zlib.NLM_BHATTACHARYYA,
                                   zlib.NLM_COMPENSATED))
    loss, q = zlib.wishart_stat_fwd(s1, s2, wts, 5, want_map=True)
    out += [loss, q, zlib.wishart_stat_bwd(s1, s2, wts, 5)]
    loss2, zs = zlib.wishart_stat_fwd_save(s1, s2, wts, 5)
    out += [loss2, zs, zlib.wishart_stat_bwd_saved(s1, s2, zs, 5)]
    return out


def test_graph_replay_gives_the_eager_bits(zlib):
    args = _inputs()
    # the first allocation-free call on a device must come before any capture
    H, W = args[1].shape[1:]
    d_loss = torch.empty((), dtype=torch.float64, device="cuda")
    assert zlib.load().wishart_stat_fwd_noalloc(args[1].data_ptr(), args[2].data_ptr(), H, W,
                                                H * W, 5, args[4].data_ptr(), None,
                                                d_loss.data_ptr(), None) == 0
    eager = _run(zlib, *args)
    torch.cuda.synchronize()
    eager = [t.clone() for t in eager]
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        _run(zlib, *args)  # warm-up on the capture stream
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        captured = _run(zlib, *args)
        noalloc = torch.empty((), dtype=torch.float64, device="cuda")
        assert zlib.load().wishart_stat_fwd_noalloc(
            args[1].data_ptr(), args[2].data_ptr(), H, W, H * W, 5, args[4].data_ptr(), None,
            noalloc.data_ptr(), torch.cuda.current_stream().cuda_stream) == 0
    for _ in range(2):
        for t in captured:
            t.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert len(captured) == len(eager)
        for k, (a, b) in enumerate(zip(captured, eager)):
            assert torch.equal(a, b), f"output {k} differs after replay"
        assert torch.equal(noalloc, d_loss)
