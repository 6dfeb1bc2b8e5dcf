"""Throughput of the per-pixel 3x3 Hermitian inverse + determinant on a GB300.

Workload (default): the 16384 x 16384 packed-FP32 image (268,435,456 matrices,
N = 16 looks, 8 class covariances in 512 x 512 blocks), generated on the GPU
from the seeded generator.  One step = one launch of zinv_det (Alg. 2 of the
paper, plain FP32) over the whole image: 36 B read and 40 B written per matrix,
20.4 GB per step, so every step streams well past the 126 MB L2.

The JSON line carries the headline (adjugate Gmatrices/s), the same launch for
the Cholesky baseline (Alg. 1), the compensated and FP64-recompute variants,
the backward, the end-to-end number through the host-buffer entry point, the
roofline of the dominant kernel, the FP64 oracle timed on the host cores, and
the SM clocks sampled during the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) each rank runs the same per-GPU workload on its own
synthetic image (weak scaling, no data-path collective); the time is the max
over ranks and the value the matrices of all ranks over that time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import statistics
import subprocess
import sys
import threading
import time
from pathlib import Path

import numpy as np
import torch

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "Gmatrices/s and HBM GB/s (% of peak) for 3x3 inv+det: adjugate vs Cholesky; fwd+bwd"
UNIT = "Gmatrices/s"
BYTES_FWD = 76     # 9 planes in + 9 planes + det out, FP32
BYTES_BWD = 116    # W, det, g_W, g_det in; g_Z out
L2_BYTES = 126 * 2**20  # GB300 L2
HBM_SPEC_GBS = 7900.0  # GB300 nominal HBM3e bandwidth (context beside the measured copy)


def peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def sm_max_mhz() -> float:
    """Maximum SM clock: the measured figure if present, else nvidia-smi."""
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        if d.get("sm_max_mhz"):
            return float(d["sm_max_mhz"])
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(torch.cuda.current_device()),
                              "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits"],
                             capture_output=True, text=True, timeout=10).stdout
        return float(out.strip().splitlines()[0])
    except (OSError, subprocess.SubprocessError, ValueError, IndexError):
        return 2070.0


def source_hash(files) -> str:
    h = hashlib.sha256()
    for f in files:
        h.update((ROOT / "paper_1807_08084_gb300" / "csrc" / f).read_bytes())
    return h.hexdigest()[:16]


def traffic_record(kernel: str):
    """DRAM bytes per full-size launch from the committed ncu summary
    (profiles/traffic.json), or None once the kernel's sources have changed
    since the counters were taken."""
    p = ROOT / "profiles" / "traffic.json"
    if not p.exists():
        return None
    d = json.loads(p.read_text()).get(kernel)
    if not d or d.get("source_hash") != source_hash(d["sources"]):
        return None
    return float(d["bytes_per_launch"])


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 100 ms in the background."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.samples = []
        self.proc = None
        uuid = None
        try:
            uuid = str(torch.cuda.get_device_properties(device_index).uuid)
        except Exception:
            pass
        self.target = (["-i", uuid if uuid.startswith("GPU-") else f"GPU-{uuid}"]
                       if uuid else ["-i", str(device_index)])

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", *self.target, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except FileNotFoundError:
            self.proc = None
            return
        self.t0 = time.time()
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), line.strip()))

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        return self.summary()

    def summary(self, t_from=None, t_to=None):
        rows = []
        for t, line in self.samples:
            if t_from is not None and not (t_from <= t <= t_to):
                continue
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[4:8]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r)
                          if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    from paper_1807_08084_gb300 import shard
    shard.barrier()


def max_over_ranks(x: float, world: int) -> float:
    from paper_1807_08084_gb300 import shard
    return shard.max_over_ranks(x, device="cuda")


def timed(fn, steps: int, warmup: int, world: int) -> float:
    """Average ms per call: CUDA events on the launching stream, barrier and
    synchronize on both sides, max over ranks."""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    barrier(world)
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(steps):
        fn()
    e1.record(s)
    torch.cuda.synchronize()
    barrier(world)
    return max_over_ranks(e0.elapsed_time(e1) / steps, world)


def timed_stats(fn, steps: int, warmup: int, world: int) -> dict:
    """As timed(), plus the fastest and the median single call: an event is
    recorded between consecutive calls (max over ranks of each statistic)."""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    barrier(world)
    s = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    ev[0].record(s)
    for i in range(steps):
        fn()
        ev[i + 1].record(s)
    torch.cuda.synchronize()
    barrier(world)
    per = sorted(ev[i].elapsed_time(ev[i + 1]) for i in range(steps))
    return {"mean": max_over_ranks(ev[0].elapsed_time(ev[steps]) / steps, world),
            "min": max_over_ranks(per[0], world),
            "median": max_over_ranks(per[steps // 2], world)}


def timed_device(fn, steps: int, warmup: int, world: int) -> float:
    """Median device time of single calls (ms) for launches shorter than the
    host's cost of issuing them: before each call a short GPU spin
    (torch.cuda._sleep) lets the host queue the start event, the call and the
    end event, so the events bracket the kernel, not the host."""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    barrier(world)
    s = torch.cuda.current_stream()
    per = []
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda._sleep(200_000)
        e0.record(s)
        fn()
        e1.record(s)
        e1.synchronize()
        per.append(e0.elapsed_time(e1))
    barrier(world)
    return max_over_ranks(sorted(per)[steps // 2], world)


def host_cpu() -> str:
    """CPU model and core count of this host, as the OS reports them."""
    model = platform.machine()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return f"{model}, {os.cpu_count()} cores"


def _pool_rate(route, data, workers, budget_s, share=True):
    """Items per second of the oracle over `workers` processes: whole steps
    (every worker once over its data) until budget_s of wall time."""
    from oracle.pool import OraclePool
    with OraclePool(route, data, workers, share=share) as pool:
        pool.step()  # warm-up: page in the data and the code
        items, wall = 0, 0.0
        while wall < budget_s:
            it, t, _ = pool.step()
            items += it
            wall += t
    return items / wall, pool.n


def cpu_oracle_baseline(images: dict, budget_s: float = 2.0):
    """The unmodified FP64 oracle on the host cores: one thread, and one process
    per core on disjoint shares of the data (oracle.pool), for the Gauss-Jordan
    and the cofactor (adjugate) routes on samples of the 16384 x 16384 and the
    cond-controlled 4096 x 4096 images, and the Wishart forward + backward on a
    band of rows of the 4096 x 4096 pair.  The headline value is the
    Gauss-Jordan route on all cores on the 16384 x 16384 sample."""
    import tempfile
    cores = os.cpu_count() or 1
    per_worker = 1 << 19
    out = {"host": host_cpu(), "routes": {}}
    with tempfile.TemporaryDirectory() as d:
        for key, z_dev in (("scale_16k", images["scale_16k"]),
                           ("precision_4k", images["precision_4k"])):
            zf = z_dev.reshape(9, -1)
            m_all = min(zf.shape[1], cores * per_worker)
            all_path, one_path = f"{d}/{key}_all.npy", f"{d}/{key}_one.npy"
            np.save(all_path, zf[:, :m_all].cpu().numpy())
            np.save(one_path, zf[:, :2 * per_worker].cpu().numpy())
            for route in ("ge", "adj"):
                r1, _ = _pool_rate(route, one_path, 1, budget_s)
                rn, used = _pool_rate(route, all_path, cores, budget_s)
                out["routes"][f"{key}/{route}"] = {
                    "gmat_s_1_thread": r1 / 1e9, "gmat_s_all_cores": rn / 1e9, "cores": used,
                    "matrices_all_cores": m_all, "matrices_1_thread": 2 * per_worker}
        s1, s2 = images["wishart_pair_4k"]
        rows_per = 32
        rows_all = min(s1.shape[1], cores * rows_per)
        paths = {}
        for name, rows in (("one", rows_per), ("all", rows_all)):
            pa, pb = f"{d}/w1_{name}.npy", f"{d}/w2_{name}.npy"
            np.save(pa, s1[:, :rows].cpu().numpy())
            np.save(pb, s2[:, :rows].cpu().numpy())
            paths[name] = (pa, pb)
        r1, _ = _pool_rate("wishart", paths["one"], 1, budget_s)
        rn, used = _pool_rate("wishart", paths["all"], cores, budget_s)
        out["routes"]["wishart_pair_4k/fwd+bwd"] = {
            "gpix_s_1_thread": r1 / 1e9, "gpix_s_all_cores": rn / 1e9, "cores": used,
            "sample": f"the first {rows_all} rows of both 4096-wide dates, 7 x 7 uniform taps, "
                      f"{rows_all // used} output rows per process (forward over the band "
                      "plus its 3-row halo, backward over the band)"}
    head = out["routes"]["scale_16k/ge"]
    return {"value": head["gmat_s_all_cores"], "unit": UNIT, "cores": head["cores"],
            "kind": "oracle",
            "sample": f"the first {head['matrices_all_cores']} matrices of the same 16384 x 16384 "
                      f"image, one process per core ({head['matrices_all_cores'] // head['cores']} "
                      "matrices each), FP64 Gauss-Jordan inverse and det of the oracle as it "
                      f"stands, repeated for ~{budget_s:.0f} s",
            "single_thread": head["gmat_s_1_thread"], **out}


def fp32_peak_tflops() -> float:
    """FP32 FMA peak of this GPU: SMs (read from the device) x 128 FP32 lanes x
    2 flops x the maximum SM clock (152 x 128 x 2 x 2.07 GHz = 80.5 TFLOP/s on
    a GB300)."""
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return sms * 128 * 2 * sm_max_mhz() * 1e6 / 1e12


def workload_config(H: int, W: int, world: int) -> dict:
    """The `config` of both arms' JSON lines: the scale_16k workload."""
    n = H * W
    return {"workload": f"scale_16k: {H}x{W} packed FP32 Hermitian Z ({n:,} matrices), "
                        "N=16 looks, 8 class covariances in 512x512 blocks",
            "matrices_per_gpu": n, "bytes_per_step_per_gpu": BYTES_FWD * n,
            "l2": f"inputs larger than L2 ({BYTES_FWD * n / 1e9:.1f} GB streamed per step)",
            "parallelism": f"replicas x{world}"}


def run_reference(args, world, rank):
    """The FP64 oracle timed on the host cores (the reference arm): one process
    per core, each running the unmodified oracle over the same seeded sample of
    the workload every step."""
    if rank != 0:
        return
    import tempfile
    from oracle.pool import OraclePool
    from paper_1807_08084_gb300 import synth as S
    w = S.WORKLOADS["scale_16k"]
    m = 1 << 18
    z = w.packed_z(np.arange(m, dtype=np.uint64))   # numpy twin, CPU only
    with tempfile.TemporaryDirectory() as d:
        path = f"{d}/sample.npy"
        np.save(path, z)
        with OraclePool("ge", path, share=False) as pool:
            for _ in range(args.warmup):
                pool.step()
            items, wall = 0, 0.0
            for _ in range(args.steps):
                it, t, _ = pool.step()
                items += it
                wall += t
            cores = pool.n
    value = items / wall / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": workload_config(w.H, w.W, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "host": host_cpu(),
                             "sample": f"per step, each of {cores} processes (one per core) "
                                       f"runs the oracle's FP64 Gauss-Jordan inverse and det "
                                       f"over the first {m} matrices of the {w.H}x{w.W} image"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def build_parser() -> argparse.ArgumentParser:
    """The command line (also used to check the commands quoted in profiles/)."""
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--sub-steps", type=int, default=50, help="steps per secondary path")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--multilook", type=int, default=1, help="also time the fused multilook")
    ap.add_argument("--ml-rows", type=int, default=8192, help="multilook image height")
    ap.add_argument("--wishart", type=int, default=1, help="also time the Wishart statistic")
    ap.add_argument("--nlm", type=int, default=1, help="also time the nonlocal-means filter")
    ap.add_argument("--blockdiag", type=int, default=1, help="also time 3-band block-diagonal pixels")
    ap.add_argument("--precision", type=int, default=1,
                    help="also time the precision modes on the cond-controlled workload")
    ap.add_argument("--nlm-rows", type=int, default=1024, help="nonlocal-means image side")
    ap.add_argument("--paper", type=int, default=1,
                    help="also time the paper's own workload sizes (its Table 2)")
    ap.add_argument("--ws-rows", type=int, default=4096, help="Wishart image height")
    ap.add_argument("--plain256", type=int, default=1,
                    help="also time single launches on the 256 x 256 latency workload")
    ap.add_argument("--cpu-baseline", type=int, default=1,
                    help="time the FP64 oracle on the host cores (rank 0, one GPU only)")
    ap.add_argument("--rows", type=int, default=16384,
                    help="image height (16384 = the full workload; smaller for profiling)")
    return ap


def main():
    ap = build_parser()
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        # host-only: rank 0 times the oracle, the other ranks exit without work
        run_reference(args, int(os.environ.get("WORLD_SIZE", "1")),
                      int(os.environ.get("RANK", "0")))
        return
    world, rank, local = dist_setup(args)

    import paper_1807_08084_gb300 as zp
    from paper_1807_08084_gb300 import synth as S
    from paper_1807_08084_gb300.synth import gpu as G

    zp.load()
    w = S.WORKLOADS["scale_16k"]
    if args.rows != w.H:
        w = S.scaled(w, args.rows, w.W)
    if world > 1:
        from dataclasses import replace
        from paper_1807_08084_gb300 import shard
        w = replace(w, seed=shard.rank_seed(w.seed, rank))
    n = w.n
    z = G.packed_z(w)
    zinv = torch.empty_like(z)
    det = torch.empty((w.H, w.W), device="cuda")
    hbm_peak, peak_kind = peaks()

    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    # --- headline: adjugate (Alg. 2), plain FP32 -----------------------------
    t_from = time.time()
    ms = timed(lambda: zp.zinv_det(z, zp.PLAIN, out=(zinv, det)), args.steps, args.warmup, world)
    t_to = time.time()
    clocks = sampler.summary(t_from, t_to)

    def path(ms_):
        gbs = BYTES_FWD * n / (ms_ * 1e-3) / 1e9
        return {"gmat_s": n / (ms_ * 1e-3) / 1e9, "ms": ms_, "gbs": gbs,
                "frac_hbm": gbs / hbm_peak, "frac_hbm_spec": gbs / HBM_SPEC_GBS}

    paths = {"adjugate": path(ms)}
    sub = args.sub_steps
    # single-launch statistics of the two routes (events between launches)
    st_adj = timed_stats(lambda: zp.zinv_det(z, zp.PLAIN, out=(zinv, det)), sub, args.warmup,
                         world)
    st_chol = timed_stats(lambda: zp.chol_zinv_det(z, out=(zinv, det)), sub, args.warmup, world)
    paths["adjugate"].update({"ms_min": st_adj["min"], "ms_median": st_adj["median"]})
    paths["cholesky"] = path(st_chol["mean"])
    paths["cholesky"].update({"ms_min": st_chol["min"], "ms_median": st_chol["median"]})
    paths["compensated"] = path(timed(lambda: zp.zinv_det(z, zp.COMPENSATED, out=(zinv, det)),
                                      sub, args.warmup, world))
    counts = zp.zinv_det(z, zp.FP64_RECOMPUTE, want_counts=True, out=(zinv, det))[2]
    paths["fp64_recompute"] = path(timed(
        lambda: zp.zinv_det(z, zp.FP64_RECOMPUTE, out=(zinv, det)), sub, args.warmup, world))
    paths["fp64_recompute"]["flagged_fraction"] = int(counts[1]) / n
    paths["compensated_fp64"] = path(timed(
        lambda: zp.zinv_det(z, zp.COMPENSATED | zp.FP64_RECOMPUTE, out=(zinv, det)), sub,
        args.warmup, world))
    # backward from saved (W, det) with upstream gradients of W and det
    zp.zinv_det(z, zp.PLAIN, out=(zinv, det))
    g_w = G.uniform(w.seed, 9 * n, stream=1).reshape(9, w.H, w.W)
    g_det = G.uniform(w.seed, n, stream=2).reshape(w.H, w.W)
    g_z = torch.empty_like(z)
    ms_bwd = timed(lambda: zp.zinv_det_bwd(zinv, det, g_w, g_det, None, out=g_z), sub,
                   args.warmup, world)
    gbs_bwd = BYTES_BWD * n / (ms_bwd * 1e-3) / 1e9
    paths["backward"] = {"gmat_s": n / (ms_bwd * 1e-3) / 1e9, "ms": ms_bwd, "gbs": gbs_bwd,
                         "frac_hbm": gbs_bwd / hbm_peak}
    paths["fwd_plus_bwd"] = {"gmat_s": n / ((ms + ms_bwd) * 1e-3) / 1e9, "ms": ms + ms_bwd}
    scale = n / float(1 << 28)
    for key, kern in (("adjugate", "zinv_det_plain_vec4"), ("cholesky", "chol_zinv_det_vec4"),
                      ("backward", "zinv_det_bwd_vec4")):
        t = traffic_record(kern)
        paths[key]["dram_bytes_ncu"] = None if t is None else t * scale
    del g_w, g_det, g_z
    sampler.stop()

    cpu_inputs = {"scale_16k": z}  # device images the host-core oracle timing samples

    # --- plain_256 (256 x 256, N = 4 looks of one fixed Sigma): launch latency --
    plain256 = {}
    if args.plain256:
        wq = S.WORKLOADS["plain_256"]
        zq = G.packed_z(wq)
        zqi = torch.empty_like(zq)
        dq = torch.empty((wq.H, wq.W), device="cuda")
        t_a = timed_device(lambda: zp.zinv_det(zq, zp.PLAIN, out=(zqi, dq)), sub, args.warmup,
                           world)
        t_c = timed_device(lambda: zp.chol_zinv_det(zq, out=(zqi, dq)), sub, args.warmup, world)
        t_b = timed(lambda: zp.zinv_det(zq, zp.PLAIN, out=(zqi, dq)), 10 * sub, args.warmup,
                    world)
        # device-side rate of back-to-back launches: 100 launches captured in a
        # CUDA graph and replayed, so the binding's per-call host cost drops out
        t_g = None
        try:
            graph = torch.cuda.CUDAGraph()
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                zp.zinv_det(zq, zp.PLAIN, out=(zqi, dq))  # warm on the capture stream
            torch.cuda.current_stream().wait_stream(side)
            with torch.cuda.graph(graph, capture_error_mode="relaxed"):
                for _ in range(100):
                    zp.zinv_det(zq, zp.PLAIN, out=(zqi, dq))
            t_g = timed(graph.replay, max(3, sub // 5), args.warmup, world) / 100
        except RuntimeError as exc:  # capture not available: report the reason
            t_g = None
            graph_error = str(exc)[:200]
        plain256 = {"matrices": wq.n, "adjugate_us": t_a * 1e3, "cholesky_us": t_c * 1e3,
                    "adjugate_back_to_back_us": t_b * 1e3,
                    "adjugate_back_to_back_gmat_s": wq.n / (t_b * 1e-3) / 1e9,
                    "adjugate_graph_us": None if t_g is None else t_g * 1e3,
                    "adjugate_graph_gmat_s": None if t_g is None else wq.n / (t_g * 1e-3) / 1e9,
                    "l2": "L2-resident (5.0 MB per launch): no flush; *_us are the median device "
                          "time of single launches, back_to_back the mean of consecutive calls "
                          "through the Python binding (host-bound), graph the mean of 100 "
                          "launches replayed from a CUDA graph (the device rate)",
                    "workload": "256x256 packed Z, N = 4 looks of the fixed Sigma "
                                "(Bartlett-sampled complex Wishart)"}
        if t_g is None:
            plain256["graph_error"] = graph_error
        del zq, zqi, dq

    # --- fused multilook (8192 x 8192 single-look, boxcar 3/5/7) ---------------
    multilook = {}
    if args.multilook:
        wl = S.WORKLOADS["multilook_8k"]
        if args.ml_rows != wl.H:
            wl = S.scaled(wl, args.ml_rows, wl.W)
        sl = G.image(wl)
        ml_inv = torch.empty((9, wl.H, wl.W), device="cuda")
        ml_det = torch.empty((wl.H, wl.W), device="cuda")
        for win in wl.windows:
            t = timed(lambda: zp.multilook_zinv_det(sl, win, None, zp.PLAIN, out=(ml_inv, ml_det)),
                      sub, args.warmup, world)
            gbs = 64 * wl.n / (t * 1e-3) / 1e9
            multilook[f"win{win}"] = {"gpix_s": wl.n / (t * 1e-3) / 1e9, "ms": t, "gbs": gbs,
                                      "frac_hbm": gbs / hbm_peak}
        # learnable 7 x 7 window (general weights: 441 window FMAs per pixel)
        g = np.exp(-0.5 * (np.arange(-3, 4) / 1.5) ** 2)
        wts = torch.from_numpy((np.outer(g, g) / np.outer(g, g).sum()).astype(np.float32)).cuda()
        t = timed(lambda: zp.multilook_zinv_det(sl, 7, wts, zp.PLAIN, out=(ml_inv, ml_det)),
                  sub, args.warmup, world)
        gbs = 64 * wl.n / (t * 1e-3) / 1e9
        tflops = 2 * 9 * 49 * wl.n / (t * 1e-3) / 1e12
        multilook["weighted7"] = {"gpix_s": wl.n / (t * 1e-3) / 1e9, "ms": t, "gbs": gbs,
                                  "frac_hbm": gbs / hbm_peak, "window_tflops": tflops,
                                  "frac_alu": tflops / fp32_peak_tflops(),
                                  "weights": "7 x 7 Gaussian, sigma 1.5, normalised"}
        del sl, ml_inv, ml_det

    # --- multifrequency: three bands, block-diagonal pixels (8192 x 8192) -------
    blockdiag = {}
    if args.blockdiag:
        from dataclasses import replace as _replace
        wb = S.scaled(S.WORKLOADS["scale_16k"], 8192, 8192)
        zb = torch.stack([G.packed_z(_replace(wb, seed=wb.seed + 17 * b)) for b in range(3)])
        t = timed(lambda: zp.zinv_det_blockdiag(zb), sub, args.warmup, world)
        gbs = (3 * 72 + 4) * wb.n / (t * 1e-3) / 1e9
        blockdiag = {"ms": t, "gpix_s": wb.n / (t * 1e-3) / 1e9, "gbs": gbs,
                     "frac_hbm": gbs / hbm_peak,
                     "workload": "8192x8192 pixels x 3 bands of packed Z (scale_16k generator)"}
        del zb

    # --- precision modes where the FP64 recompute has work: the cond-controlled
    # 4096 x 4096 workload (cond log-uniform in [1, 1e7]) ----------------------
    precision = {}
    if args.precision:
        wp = S.WORKLOADS["precision_4k"]
        zp4 = G.packed_z(wp)
        zi4 = torch.empty_like(zp4)
        d4 = torch.empty((wp.H, wp.W), device="cuda")
        for name, flags in (("plain", zp.PLAIN), ("compensated", zp.COMPENSATED),
                            ("plain_fp64", zp.FP64_RECOMPUTE),
                            ("compensated_fp64", zp.COMPENSATED | zp.FP64_RECOMPUTE)):
            t = timed(lambda: zp.zinv_det(zp4, flags, out=(zi4, d4)), sub, args.warmup, world)
            gbs = BYTES_FWD * wp.n / (t * 1e-3) / 1e9
            precision[name] = {"ms": t, "gmat_s": wp.n / (t * 1e-3) / 1e9, "gbs": gbs,
                               "frac_hbm": gbs / hbm_peak}
        cnt = zp.zinv_det(zp4, zp.FP64_RECOMPUTE, want_counts=True, out=(zi4, d4))[2]
        precision["flagged_fraction"] = int(cnt[1]) / wp.n
        precision["workload"] = ("4096x4096 packed Z = U diag(1, k^-v, 1/k) U^H, k log-uniform "
                                 "in [1, 1e7], tau = 2^-10")
        cpu_inputs["precision_4k"] = zp4
        del zi4, d4

    # --- the paper's own workload sizes (its Table 2): context, not the headline --
    paper = {}
    if args.paper:
        for key, wname, (adj_ms, chol_ms), note in (
                ("simulated", "paper_sim", (231.51, 507.54),
                 "5,469,354 matrices A = R R^H, Re/Im R ~ U[-1, 1]; 416 MB, HBM-bound"),
                ("measured_shaped", "paper_meas_shaped", (12.98, 28.35),
                 "450 x 600 matrices (stand-in for the AIRSAR scene); 20.5 MB, L2-resident; "
                 "median device time of single launches")):
            wq = S.WORKLOADS[wname]
            zq = G.packed_z(wq)
            zqi = torch.empty_like(zq)
            dq = torch.empty((wq.H, wq.W), device="cuda")
            tfn = timed if wq.n * BYTES_FWD > 2 * L2_BYTES else timed_device
            t_a = tfn(lambda: zp.zinv_det(zq, zp.PLAIN, out=(zqi, dq)), sub, args.warmup, world)
            t_c = tfn(lambda: zp.chol_zinv_det(zq, out=(zqi, dq)), sub, args.warmup, world)
            paper[key] = {"matrices": wq.n, "adjugate_ms": t_a, "cholesky_ms": t_c,
                          "adjugate_gmat_s": wq.n / (t_a * 1e-3) / 1e9,
                          "speedup_adjugate_vs_cholesky": t_c / t_a,
                          "paper_table2_avg_ms": {"adjugate": adj_ms, "cholesky": chol_ms,
                                                  "hardware": "GeForce 940M, OpenCL"},
                          "workload": note}
            del zq, zqi, dq

    # --- nonlocal means, 23 x 23 search window: arithmetic-bound per-pair dets --
    nlm = {}
    if args.nlm:
        wn = S.scaled(S.WORKLOADS["scale_16k"], args.nlm_rows, args.nlm_rows)
        zn = G.packed_z(wn)
        zo = torch.empty_like(zn)
        pairs = wn.n * 23 * 23
        for name, meth in (("adjugate", zp.NLM_ADJUGATE), ("cholesky", zp.NLM_CHOLESKY)):
            t = timed(lambda: zp.nlm_wishart(zn, 11, 16.0, 1.0, meth, out=zo), max(3, sub // 5),
                      args.warmup, world)
            nlm[name] = {"ms": t, "gpairs_s": pairs / (t * 1e-3) / 1e9}
        nlm["speedup_adjugate_vs_cholesky"] = nlm["cholesky"]["ms"] / nlm["adjugate"]["ms"]
        t = timed(lambda: zp.nlm_wishart(zn, 11, 16.0, 1.0, zp.NLM_COMPENSATED, out=zo),
                  max(3, sub // 5), args.warmup, world)
        nlm["compensated"] = {"ms": t, "gpairs_s": pairs / (t * 1e-3) / 1e9,
                              "note": "pair sum kept exact, Dot2 det + first-order term"}
        nlm["workload"] = (f"{wn.H}x{wn.W} packed Z (scale_16k generator), radius 11 "
                           "(23 x 23 window), L = 16, h = 1")
        # the other stochastic distances (nlm_stochastic): Hellinger shares the
        # per-pair determinant; Kullback-Leibler takes two traces with the
        # per-pixel inverses instead; Renyi two determinants per pair
        hel = {}
        for name, meth in (("adjugate", zp.NLM_ADJUGATE), ("cholesky", zp.NLM_CHOLESKY)):
            t = timed(lambda: zp.nlm_stochastic(zn, 11, 16.0, 0.25, zp.NLM_HELLINGER, meth,
                                                out=zo), max(3, sub // 5), args.warmup, world)
            hel[name] = {"ms": t, "gpairs_s": pairs / (t * 1e-3) / 1e9}
        hel["speedup_adjugate_vs_cholesky"] = hel["cholesky"]["ms"] / hel["adjugate"]["ms"]
        hel["h"] = 0.25
        nlm["hellinger"] = hel
        t = timed(lambda: zp.nlm_stochastic(zn, 11, 16.0, 4.0, zp.NLM_KULLBACK_LEIBLER,
                                            zp.NLM_ADJUGATE, out=zo), max(3, sub // 5),
                  args.warmup, world)
        nlm["kullback_leibler"] = {"ms": t, "gpairs_s": pairs / (t * 1e-3) / 1e9, "h": 4.0}
        ren = {}
        for name, meth in (("adjugate", zp.NLM_ADJUGATE), ("cholesky", zp.NLM_CHOLESKY)):
            t = timed(lambda: zp.nlm_stochastic(zn, 11, 16.0, 2.0, zp.NLM_RENYI, meth, out=zo,
                                                order=0.7), max(3, sub // 5), args.warmup, world)
            ren[name] = {"ms": t, "gpairs_s": pairs / (t * 1e-3) / 1e9}
        ren["speedup_adjugate_vs_cholesky"] = ren["cholesky"]["ms"] / ren["adjugate"]["ms"]
        ren["h"], ren["order"] = 2.0, 0.7
        nlm["renyi"] = ren
        del zn, zo

    # --- Wishart change statistic (two 4096 x 4096 dates, 7 x 7 window) -------
    wishart = {}
    if args.wishart:
        ww = S.WORKLOADS["wishart_pair_4k"]
        if args.ws_rows != ww.H:
            ww = S.scaled(ww, args.ws_rows, ww.W)
        s1, s2 = G.image(ww, 0), G.image(ww, 1)
        wts = torch.full((49,), 1.0 / 49.0, device="cuda")
        ws_buf = torch.empty(zp.wishart_workspace_bytes(ww.H, ww.W, 7), dtype=torch.uint8,
                             device="cuda")
        g1 = torch.ones((), dtype=torch.float64, device="cuda")
        t_f = timed(lambda: zp.wishart_stat_fwd(s1, s2, wts, 7, ws=ws_buf), sub, args.warmup, world)
        t_b = timed(lambda: zp.wishart_stat_bwd(s1, s2, wts, 7, g1, ws=ws_buf), sub, args.warmup,
                    world)
        # algorithmic FP32 work: the window sums, 2 dates x 49 taps x 9 channels FMA
        # per pixel forward; the backward recomputes them and correlates as many
        fl_f, fl_b = 2 * 2 * 49 * 9, 2 * 2 * 2 * 49 * 9
        alu_peak = fp32_peak_tflops()
        for name, t, fl in (("forward", t_f, fl_f), ("backward", t_b, fl_b)):
            tf = fl * ww.n / (t * 1e-3) / 1e12
            wishart[name] = {"gpix_s": ww.n / (t * 1e-3) / 1e9, "ms": t, "tflops": tf,
                             "frac_alu": tf / alu_peak,
                             "gbs": 48 * ww.n / (t * 1e-3) / 1e9}
        wishart["alu_peak_tflops"] = alu_peak
        # saved window covariances: the forward also writes both dates' Z
        # (72 B/pixel); the backward forms M point-wise and only correlates
        zs = torch.empty((18, ww.H, ww.W), dtype=torch.float32, device="cuda")
        wsb = torch.empty(zp.wishart_bwd_saved_workspace_bytes(ww.H, ww.W, 7), dtype=torch.uint8,
                          device="cuda")
        t_fs = timed(lambda: zp.wishart_stat_fwd_save(s1, s2, wts, 7, z_saved=zs, ws=ws_buf), sub,
                     args.warmup, world)
        t_bs = timed(lambda: zp.wishart_stat_bwd_saved(s1, s2, zs, 7, g1, ws=wsb), sub,
                     args.warmup, world)
        tf_corr = 2 * 2 * 49 * 9 * ww.n / (t_bs * 1e-3) / 1e12  # the correlation's FMAs
        wishart["saved_z"] = {"forward_ms": t_fs, "backward_ms": t_bs,
                              "fwd_plus_bwd_ms": t_fs + t_bs,
                              "recompute_fwd_plus_bwd_ms": t_f + t_b,
                              "saved_bytes": 72 * ww.n,
                              "backward_tflops": tf_corr, "backward_frac_alu": tf_corr / alu_peak}
        del zs, wsb
        if ww.H == 4096:
            cpu_inputs["wishart_pair_4k"] = (s1, s2)
        del ws_buf

    # --- end to end through the host-buffer entry point -----------------------
    e2e = None
    if args.e2e_steps > 0:
        z_host = torch.empty(z.shape, dtype=torch.float32, pin_memory=True)
        z_host.copy_(z)
        zinv_h = torch.empty(z.shape, dtype=torch.float32, pin_memory=True)
        det_h = torch.empty((w.H, w.W), dtype=torch.float32, pin_memory=True)
        chunk = 1 << 24
        ws = torch.empty(zp.zinv_det_host_workspace_bytes(chunk), dtype=torch.uint8,
                         device="cuda")
        ms_e2e = timed(lambda: zp.zinv_det_host(z_host, ws, zp.PLAIN, out=(zinv_h, det_h)),
                       args.e2e_steps, 1, world)
        ms_staged = timed(lambda: zp.zinv_det_host(z_host, ws, zp.PLAIN | zp.HOST_STAGED,
                                                   out=(zinv_h, det_h)), args.e2e_steps, 1, world)
        e2e = {"value": world * n / (ms_e2e * 1e-3) / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": 36 * n, "d2h_bytes_per_step": 40 * n,
               "ms_per_step": ms_e2e,
               "api": "zinv_det_host on pinned host buffers (the kernel reads and writes "
                      "host memory over the CPU-GPU link)",
               "staged": {"value": world * n / (ms_staged * 1e-3) / 1e9, "ms_per_step": ms_staged,
                          "api": f"zinv_det_host with HOST_STAGED (chunks of {chunk} matrices "
                                 "through device memory, 3 streams)"}}
        del z_host, zinv_h, det_h, ws

    cpu = None
    if args.cpu_baseline and rank == 0 and world == 1:
        if "precision_4k" not in cpu_inputs:
            cpu_inputs["precision_4k"] = G.packed_z(S.WORKLOADS["precision_4k"])
        if "wishart_pair_4k" not in cpu_inputs:
            wpair = S.WORKLOADS["wishart_pair_4k"]
            cpu_inputs["wishart_pair_4k"] = (G.image(wpair, 0), G.image(wpair, 1))
        cpu = cpu_oracle_baseline(cpu_inputs)
    del cpu_inputs
    traffic = traffic_record("zinv_det_plain_vec4")
    if traffic is not None:
        traffic *= n / float(1 << 28)
    achieved = BYTES_FWD * n / (ms * 1e-3) / 1e9
    if rank == 0:
        line = {
            "metric": METRIC, "value": world * n / (ms * 1e-3) / 1e9, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": workload_config(w.H, w.W, world),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak,
                         "unit": "GB/s", "frac": achieved / hbm_peak,
                         "traffic": traffic, "peak_kind": peak_kind,
                         "peak_spec": HBM_SPEC_GBS, "frac_spec": achieved / HBM_SPEC_GBS,
                         "note": "peak/frac: the measured HBM copy (MEASURED_PEAKS.json); "
                                 "peak_spec/frac_spec: the GB300 nominal HBM3e bandwidth",
                         "kernel": "k_inv_det_vec4<plain>",
                         "algorithmic_bytes_per_launch": BYTES_FWD * n},
            "tolerance_note": "plain FP32 (the headline kernel) meets 1e-5 cond on the plain_256 "
                              "and scale_16k workloads; on the cond-controlled precision_4k "
                              "workload (cond up to 1e7) it needs COMPENSATED or FP64_RECOMPUTE",
            "paths": paths,
            "plain_256": plain256 or None,
            "multilook_8k": multilook or None,
            "wishart_pair_4k": wishart or None,
            "nlm_23x23": nlm or None,
            "blockdiag_3band": blockdiag or None,
            "precision_4k": precision or None,
            "paper_workloads": paper or None,
            "speedup_vs_cholesky": paths["cholesky"]["ms"] / ms,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "gpu_launches": args.steps,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
