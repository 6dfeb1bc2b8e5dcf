"""The C ABI without a GPU: the library loads, exports every symbol that
include/*.h declares, and rejects bad arguments on the host before touching a
device.  (No compute call is made here.)"""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
DECL = re.compile(r"^\s*(?:int64_t|int|size_t|const\s+char\s*\*)\s+(\w+)\s*\(", re.M)


def declared(header: Path):
    return DECL.findall(header.read_text())


def test_headers_declare_entry_points():
    names = [n for h in sorted((ROOT / "include").glob("*.h")) for n in declared(h)]
    for must in ("zinv_det", "chol_zinv_det", "zinv_det_bwd", "zinv_abi_version",
                 "zinv_status_string", "zinv_det_host"):
        assert must in names


def test_library_exports_every_declared_symbol():
    import paper_1807_08084_gb300 as zp
    lib = zp.load()
    missing = [n for h in sorted((ROOT / "include").glob("*.h")) for n in declared(h)
               if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"
    assert lib.zinv_abi_version() == 1
    assert zp.status_string(0) == "ok"
    assert "argument" in zp.status_string(-1)


def test_binding_declares_every_entry_point():
    """load() gives every declared entry point that takes arguments a ctypes
    signature, so no call goes out with ctypes' default int conversions (which
    would truncate 64-bit sizes and pointers)."""
    import paper_1807_08084_gb300 as zp
    lib = zp.load()
    undeclared = [n for h in sorted((ROOT / "include").glob("*.h")) for n in declared(h)
                  if n != "zinv_abi_version" and getattr(lib, n).argtypes is None]
    assert not undeclared, f"no argtypes for: {undeclared}"


def test_synth_library_loads():
    from paper_1807_08084_gb300.synth import gpu
    lib = gpu.load()
    for n in ("synth_z_wishart", "synth_z_cond", "synth_z_rrh", "synth_slc", "synth_uniform"):
        assert hasattr(lib, n)


def _call(fn, z, n, ld, zinv, det, flags=0, tau=0.001, status=None, counts=None):
    P = ctypes.c_void_p
    return fn(P(z), n, ld, P(zinv), P(det), flags, tau, P(status), P(counts), None)


def test_host_argument_checks():
    """Argument errors come back as ZINV_ERR_ARG before any device work; valid
    arguments on a machine without a GPU come back as ZINV_ERR_DEVICE."""
    import torch
    import paper_1807_08084_gb300 as zp
    lib = zp.load()
    if torch.cuda.is_available():
        pytest.skip("host-only check")
    fake = 0x10000  # never dereferenced: the call must fail before any access
    for fn in (lib.zinv_det, lib.chol_zinv_det):
        assert _call(fn, fake, -1, 0, fake, fake) == -1            # n < 0
        assert _call(fn, fake, 10, 5, fake, fake) == -1            # ld < n
        assert _call(fn, None, 10, 10, fake, fake) == -1           # null input
        assert _call(fn, fake, 10, 10, None, fake) == -1           # null output
        assert _call(fn, fake + 2, 10, 10, fake, fake) == -1       # misaligned
        assert _call(fn, fake, 10, 10, fake, fake, tau=float("nan")) == -1
        assert _call(fn, fake, 10, 10, fake, fake, tau=-1.0) == -1
        assert _call(fn, fake, 10, 10, fake, fake, counts=fake + 4) == -1
        assert _call(fn, fake, 10, 10, fake, fake) == -3           # valid, no device
    assert _call(lib.zinv_det, fake, 10, 10, fake, fake, flags=4) == -1  # unknown flag
    assert _call(lib.chol_zinv_det, fake, 10, 10, fake, fake, flags=1) == -1
    P = ctypes.c_void_p
    assert lib.zinv_det_bwd(P(fake), P(fake), 10, 5, None, None, None, P(fake), None) == -1
    assert lib.zinv_det_bwd(P(fake), None, 10, 10, None, P(fake), None, P(fake), None) == -1
    assert lib.zinv_det_bwd(P(fake), P(fake), 10, 10, P(fake), None, None, P(fake), None) == -3
    assert lib.zinv_det_host(P(fake), 10, 10, P(fake), P(fake), 0, 0.0, P(fake + 16), 1 << 20,
                             None) == -1  # workspace not 256-byte aligned
    z9 = P(fake)
    # unknown distance, KL with Cholesky, unknown method, Renyi order outside (0, 1)
    for dist, order, method in ((4, 0.5, 0), (-1, 0.5, 0), (2, 0.5, 1), (1, 0.5, 3),
                                (2, 0.5, 2), (3, 0.5, 2), (3, 0.0, 0), (3, 1.0, 0),
                                (3, float("nan"), 1)):
        assert lib.nlm_stochastic(z9, 10, 10, 100, 3, 4.0, 1.0, dist, order, method, z9,
                                  None) == -1
    assert lib.nlm_stochastic(z9, 10, 10, 100, 4, 4.0, 1.0, 0, 0.5, 0, z9, None) == -1  # radius
    for dist, method in ((0, 0), (1, 1), (2, 0), (3, 1), (0, 2), (1, 2)):
        assert lib.nlm_stochastic(z9, 10, 10, 100, 3, 4.0, 1.0, dist, 0.5, method, z9,
                                  None) == -3
    # saved window covariances of the Wishart statistic
    assert lib.wishart_saved_bytes(0, 5) == 0 and lib.wishart_saved_bytes(1 << 30, 1 << 30) == 0
    assert lib.wishart_saved_bytes(4, 8) == 18 * 32 * 4
    need = lib.wishart_bwd_saved_workspace_bytes(40, 70, 7)
    assert need >= lib.wishart_workspace_bytes(40, 70, 7) + 72 * 40 * 70 and need % 8 == 0
    f = P(fake)
    assert lib.wishart_stat_fwd_save(f, f, 40, 70, 2800, 7, f, None, f, None, f, 1 << 30,
                                     None) == -1                      # no z_saved
    assert lib.wishart_stat_fwd_save(f, f, 40, 70, 2800, 7, f, None, f, f, f, 1 << 30,
                                      None) == -3
    assert lib.wishart_stat_bwd_saved(f, f, 40, 70, 2800, 7, f, None, f, f, need - 8,
                                      None) == -1                     # workspace too small
    assert lib.wishart_stat_bwd_saved(f, f, 40, 70, 2800, 7, None, None, f, f, need,
                                      None) == -1                     # no z_saved
    assert lib.wishart_stat_bwd_saved(f, f, 40, 70, 2800, 6, f, None, f, f, need,
                                      None) == -1                     # window
    assert lib.wishart_stat_bwd_saved(f, f, 40, 70, 2800, 7, f, None, f, f, need, None) == -3
    assert lib.zinv_det_host_workspace_bytes(0) == 0
    assert lib.zinv_det_host_workspace_bytes(1024) >= 3 * 40 * 1024


def test_binding_rejects_bad_tensors():
    """The Python binding refuses CPU tensors for device entry points and
    mis-shaped host outputs before the library is called."""
    import torch
    import paper_1807_08084_gb300 as zp
    z = torch.zeros(9, 8)
    with pytest.raises(ValueError):
        zp.zinv_det(z)                       # there is no CPU path
    with pytest.raises(ValueError):
        zp.chol_zinv_det(z)
    bad = torch.zeros(9, 7)                  # one pixel short
    det = torch.zeros(8)
    with pytest.raises(ValueError):
        zp.zinv_det_host(z, out=(bad, det))
    with pytest.raises(ValueError):
        zp.zinv_det_host(z, out=(torch.zeros(9, 8), torch.zeros(7)))
    with pytest.raises(ValueError):
        zp.zinv_det_host(z, out=(torch.zeros(9, 8, dtype=torch.float64), det))


def test_binding_rejects_mismatched_outputs():
    """Caller-supplied outputs and gradients of the wrong dtype or shape are
    refused in Python (a smaller buffer would otherwise be overrun)."""
    import torch
    import paper_1807_08084_gb300 as zp
    z = torch.zeros(9, 8)
    with pytest.raises(ValueError):
        zp._like(torch.zeros(9, 8, dtype=torch.float16), z, "out", "z")
    with pytest.raises(ValueError):
        zp._like(torch.zeros(9, 4), z, "out", "z")
    with pytest.raises(ValueError):
        zp._like(torch.zeros(8, 9).t(), z, "out", "z")     # same shape, other strides
    assert zp._like(torch.zeros(9, 8), z, "out", "z").shape == z.shape
    with pytest.raises(ValueError):
        zp._out(torch.zeros(9, 4, 4, dtype=torch.float64), (9, 4, 4), z.device, "out")
    with pytest.raises(ValueError):
        zp._out(torch.zeros(9, 4, 5), (9, 4, 4), z.device, "out")


C_PROGRAM = r"""
#include <stdio.h>
#include "zinv.h"

int main(void) {
    static float buf[64];
    /* argument errors come back before any device work */
    int bad = zinv_det(buf, -1, 0, buf, buf, ZINV_PLAIN, 0.0f, NULL, NULL, NULL);
    int bad_nlm = nlm_stochastic(buf, 4, 4, 16, 3, 4.0f, 1.0f, ZINV_NLM_KULLBACK_LEIBLER,
                                 0.5f, ZINV_NLM_CHOLESKY, buf, NULL);
    size_t ws = wishart_workspace_bytes(16, 32, 3);
    printf("%d %d %d %s %zu\n", zinv_abi_version(), bad, bad_nlm, zinv_status_string(bad), ws);
    return 0;
}
"""


def test_header_is_plain_c_and_links(tmp_path):
    """include/zinv.h compiles as C11 and a C program links against libzinv.so
    and calls it: the boundary has no C++ or torch types in it."""
    import subprocess
    import paper_1807_08084_gb300 as zp
    lib = Path(zp.load()._name)
    src = tmp_path / "use_zinv.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "use_zinv"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-I", str(ROOT / "include"),
                    str(src), "-o", str(exe), "-L", str(lib.parent), "-l:" + lib.name,
                    "-Wl,-rpath," + str(lib.parent)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    assert out[0] == "1" and out[1] == "-1" and out[2] == "-1"
    assert "argument" in " ".join(out[3:-1])
    assert int(out[-1]) == 1 * 9 * 8  # one 32 x 16 tile, 9 taps, one double each
