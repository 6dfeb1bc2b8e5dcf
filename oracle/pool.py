"""The unmodified FP64 oracle timed on every host core: one worker process per core.

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only ``bench.py``'s CPU-baseline
leg and its reference arm use this module.  The oracle stays plain
single-threaded C; this runs one copy of it per core on disjoint data, which
is how the paper's per-pixel problem parallelises on a CPU (every matrix is
independent).  Nothing of the oracle's arithmetic is changed or tuned here.

Workers are separate interpreters (``python -m oracle.pool``) that import only
numpy and the oracle, so starting them needs no fork of a process that holds a
GPU context.  Protocol, one line each way: a worker loads its data, prints
``ready``; on ``go`` it runs its route once over its data and prints the item
count and the seconds the oracle took; on ``quit`` (or end of input) it exits.

Routes:
    ge       oracle.zinv_det: Gauss-Jordan inverse and det (per matrix)
    adj      oracle.inverse_full(method="adj"): the cofactor route, Z^-1 = adj/det
             with det by the first-column expansion (per matrix)
    wishart  oracle.wishart_fwd then oracle.wishart_bwd (7 x 7, uniform taps) on
             a band of output rows of a pair of single-look images (per pixel)
"""
from __future__ import annotations

import json
import os
import subprocess
import sys
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent.parent


class OraclePool:
    """`workers` oracle processes, each holding its share of the data.

    matrices: path of a .npy [9, m] packed sample (routes ge, adj); each worker
    takes the slice [i*m/N, (i+1)*m/N) -- or all of it with share=False.
    images: (path1, path2) of .npy [3, H, W] single-look dates (route wishart);
    worker i takes output rows [i*H/N, (i+1)*H/N) with the window's halo."""

    def __init__(self, route: str, data, workers: int | None = None, share: bool = True):
        self.n = workers or os.cpu_count() or 1
        self.procs = []
        env = dict(os.environ, PYTHONPATH=str(ROOT) + os.pathsep + os.environ.get("PYTHONPATH", ""),
                   OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1")
        paths = [str(p) for p in (data if isinstance(data, (tuple, list)) else (data,))]
        for i in range(self.n):
            cmd = [sys.executable, "-m", "oracle.pool", route, str(i), str(self.n),
                   "1" if share else "0", *paths]
            self.procs.append(subprocess.Popen(cmd, stdin=subprocess.PIPE, stdout=subprocess.PIPE,
                                               text=True, cwd=str(ROOT), env=env))
        for p in self.procs:
            line = p.stdout.readline().strip()
            if line != "ready":
                self.close()
                raise RuntimeError(f"oracle worker failed to start: {line!r}")

    def step(self):
        """All workers run once, together.  Returns (items, wall seconds, the
        slowest worker's oracle seconds)."""
        t0 = time.perf_counter()
        for p in self.procs:
            p.stdin.write("go\n")
            p.stdin.flush()
        items, slowest = 0, 0.0
        for p in self.procs:
            r = json.loads(p.stdout.readline())
            items += r["items"]
            slowest = max(slowest, r["seconds"])
        return items, time.perf_counter() - t0, slowest

    def close(self):
        for p in self.procs:
            try:
                p.stdin.write("quit\n")
                p.stdin.flush()
            except (BrokenPipeError, ValueError):
                pass
        for p in self.procs:
            try:
                p.wait(timeout=30)
            except subprocess.TimeoutExpired:
                p.kill()
        self.procs = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _split(total: int, i: int, n: int) -> tuple[int, int]:
    return total * i // n, total * (i + 1) // n


def _worker(argv):
    route, i, n, share = argv[0], int(argv[1]), int(argv[2]), argv[3] == "1"
    paths = argv[4:]
    import oracle
    o = oracle.load()
    if route in ("ge", "adj"):
        z = np.load(paths[0], mmap_mode="r")
        lo, hi = _split(z.shape[1], i, n) if share else (0, z.shape[1])
        z = np.ascontiguousarray(z[:, lo:hi], dtype=np.float64)
        items = z.shape[1]
        run = (lambda: o.zinv_det(z)) if route == "ge" else (lambda: o.inverse_full(z, "adj"))
    elif route == "wishart":
        s1 = np.load(paths[0], mmap_mode="r")
        s2 = np.load(paths[1], mmap_mode="r")
        H, W = s1.shape[1], s1.shape[2]
        win, r = 7, 3
        y_lo, y_hi = _split(H, i, n) if share else (0, H)
        h0, h1 = max(0, y_lo - r), min(H, y_hi + r)
        b1 = np.ascontiguousarray(s1[:, h0:h1])
        b2 = np.ascontiguousarray(s2[:, h0:h1])
        wts = np.full(win * win, 1.0 / (win * win))
        items = (y_hi - y_lo) * W

        def run():
            o.wishart_fwd(b1, b2, win, wts)
            o.wishart_bwd(b1, b2, win, wts, 1.0, rows=(y_lo - h0, y_hi - h0))
    else:
        raise SystemExit(f"unknown route {route}")
    print("ready", flush=True)
    for line in sys.stdin:
        cmd = line.strip()
        if cmd == "quit":
            break
        if cmd == "go":
            t = time.perf_counter()
            run()
            print(json.dumps({"items": items, "seconds": time.perf_counter() - t}), flush=True)


if __name__ == "__main__":
    _worker(sys.argv[1:])
