"""Benchmark: least-squares time-to-1e-12 backward error and QR TFLOP/s on one GB300.

Workload (one step = one full solve of the hot path): A is 32768 x 4096 FP32,
A = U diag(sigma) V^T with Haar U, V and a geometric spectrum from 1 to 1/kappa
(kappa = 1e3, seed 2), x_true ~ N(0, I), b = A x_true + e with e orthogonal to range(A),
||e|| = 1e-6 ||A x_true||. Recursive Gram-Schmidt QR with FP16 tensor-core products,
then R-preconditioned CGLS to the FP64 target (eta_est <= 1e-12, confirmed on a fresh
residual). Inputs are generated on the device in FP64 and rounded to FP32.

Prints ONE JSON line (rank 0). `value` is the mean device time per solve in ms
(lower is better); `qr_tflops` is (2 m n^2 - 2/3 n^3) / QR time. `--impl reference`
times the CPU oracle (FP64 Householder, Alg. 1) instead, on the same problem.

Multi-GPU: the path solves one independent problem per GPU (replicas, no collective);
`value` is then the max-over-ranks time per solve and `problems_per_s` counts all ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LLS time-to-1e-12 backward error & QR TFLOP/s vs plain FP64 Householder, GB300"


def qr_flops(m, n):
    return 2.0 * m * n * n - 2.0 / 3.0 * n ** 3


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    # (torch.distributed.run would read an abbreviated "--m" as one of its own options)
    ap.add_argument("--rows", "--m", dest="m", type=int, default=32768)
    ap.add_argument("--cols", "--n", dest="n", type=int, default=4096)
    ap.add_argument("--kind", default="geometric")
    ap.add_argument("--kappa", type=float, default=1e3)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--prec", default="fp16")
    ap.add_argument("--target", default="fp64")
    ap.add_argument("--krylov", default="cgls", choices=["cgls", "lsqr"])
    ap.add_argument("--reorth", type=int, default=0, choices=[0, 1])
    ap.add_argument("--pw", type=int, default=0, help="panel width (0 = library default)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-householder", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip the autotuner (the library's default settings, or the ones cached)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other workload configurations (small solve, spectrum sweep, large QR, "
                         "batched, differentiable)")
    return ap.parse_args()


def dist_setup(backend):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group(backend=backend)
    return rank, ws


class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        with open(self.f.name) as fh:
            lines = fh.readlines()
        os.unlink(self.f.name)
        return summarize_clocks(lines)


def summarize_clocks(lines):
    """Median SM clock under load, the maximum clock and the throttle reasons seen, from
    nvidia-smi lines in ClockSampler.FIELDS order (csv, no header, no units). Samples below
    half the maximum clock count as idle when loaded samples exist; fields that are not
    numbers ("[N/A]") are skipped."""
    rows = []
    for line in lines:
        parts = [x.strip() for x in line.split(",")]
        if len(parts) >= 9:
            rows.append(parts)
    if not rows:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
    sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
    mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
    loaded = [s for s in sm if mx and s >= 0.5 * max(mx)] or sm
    return {"sm_mhz": statistics.median(loaded) if loaded else None,
            "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), or None."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def oracle_threads():
    """Threads the C oracle's OpenMP loops use (OMP_NUM_THREADS, else every core)."""
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v and v.isdigit() else os.cpu_count()


def cpu_baseline(A32_dev, b_dev, m, n):
    """The oracle (FP64 Householder least squares, Alg. 1) on the same A and b, one full solve,
    timed on the host's cores. No sampling and no scaling: the value is that solve's time."""
    from oracle import direct
    A = A32_dev.cpu().numpy()
    b = b_dev.cpu().numpy()
    direct.lib()
    t0 = time.perf_counter()
    direct.lls(A, b)
    dt = time.perf_counter() - t0
    return {"value": dt * 1e3, "unit": "ms", "cores": oracle_threads(), "cpu_model": cpu_model(),
            "kind": "oracle",
            "sample": f"one full FP64 Householder solve (unblocked, OpenMP over the trailing columns) of the "
                      f"same {m}x{n} problem, A and b as the GPU solves them"}


def run_reference(args):
    """The reference arm: the CPU oracle, as it stands, on the same problem as the GPU arm
    (the same generator, seed and sizes). Warm-up steps solve the small 1024 x 128 problem of
    the same family (they load the library and start the threads); each timed step is one full
    solve of the benchmark problem. Timed steps stop early once 240 s have been spent, and the
    line reports the number actually timed."""
    rank, ws = dist_setup("gloo")
    if rank != 0:
        return
    import torch
    from oracle import direct
    from paper_1912_05508_gb300 import synth
    m, n = args.m, args.n
    if torch.cuda.is_available():
        dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
        A_d, b_d = make_inputs(args, m, n, 0, dev)
        A, b = A_d.cpu().numpy(), b_d.cpu().numpy()
        del A_d, b_d
        torch.cuda.empty_cache()
        gen = "generated on the GPU as in the GPU arm"
    else:
        p = synth.svd_lls(m, n, args.kind, args.kappa, seed=args.seed)
        A, b = p.A, p.b
        gen = "generated on the CPU (no GPU present): same family and seed, different random stream"
    small = synth.svd_lls(1024, 128, args.kind, args.kappa, seed=1)
    direct.lib()
    for _ in range(args.warmup):
        direct.lls(small.A, small.b)
    times = []
    budget_s = 240.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        direct.lls(A, b)
        times.append(time.perf_counter() - t0)
        if sum(times) > budget_s:
            break
    ms = statistics.mean(times) * 1e3
    sample = (f"{len(times)} full FP64 Householder solves of the {m}x{n} problem ({gen}); warm-up: "
              f"{args.warmup} solves of the 1024x128 problem of the same family")
    cfg = {"workload": f"single LLS {m}x{n} FP32, {args.kind} kappa={args.kappa:g}", "m": m, "n": n,
           "kind": args.kind, "kappa": args.kappa, "seed": args.seed, "sample": sample}
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": ms, "unit": "ms",
                      "n_gpus": args.gpus, "steps": len(times), "steps_requested": args.steps,
                      "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
                      "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
                      "steps_ms": [round(t * 1e3, 1) for t in times],
                      "cpu_baseline": {"value": ms, "unit": "ms", "cores": oracle_threads(), "cpu_model": cpu_model(),
                                       "kind": "oracle", "sample": sample},
                      "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0,
                              "d2h_bytes_per_step": 0}}))


# ncu DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of each kernel, from
# the captures summarised under profiles/, each with the SHA-256 (first 16 hex digits) of the
# kernel's source file at the time of the capture. A kernel whose source has changed since
# reports null until it is captured again. tc_projection is the product kernel alone (the
# split-K reduce is a separate, small launch).
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one ncu capture per kernel
# (summaries under profiles/), valid only while the kernel's source is the captured one:
# key -> (captured bytes, captured units, source file, sha256 prefix of that file). The bench
# scales the bytes by its own units over the captured units, since every term of the traffic
# grows in proportion: block launches of the same shape; the products' rows m (the capture
# runs m = 16384, half the bench's top node); the Krylov phase's algorithmic bytes (the capture
# runs 16384 x 4096 for 6 iterations: 15 passes over A and 14 triangular products).
NCU_TRAFFIC = {"block": (54.846992e9 * 79.264e-6, 1.0, "panel_flat.cu", "d9c64e926cb88eff"),
               "tc_projection": (134252288 + 3640064, 16384, "gemm_persist.cu", "e6322d58344b9a4e"),
               "tc_update": (209890560 + 82324480, 16384, "gemm_persist.cu", "e6322d58344b9a4e"),
               "cgls": (4120058000 + 62745344, 15 * 4.0 * 16384 * 4096 + 14 * 4.0 * 4096 * 4097 / 2,
                        "krylov.cu", "8a52e08a690e00b6")}


def source_digest(name):
    import hashlib
    path = os.path.join(ROOT, "paper_1912_05508_gb300", "csrc", name)
    try:
        with open(path, "rb") as fh:
            return hashlib.sha256(fh.read()).hexdigest()[:16]
    except OSError:
        return None


def ncu_traffic(key, units=1.0):
    """DRAM bytes per launch of a kernel, from its capture scaled to `units` (see NCU_TRAFFIC),
    or None when there is no capture of the kernel as its source stands."""
    rec = NCU_TRAFFIC.get(key)
    if rec is None:
        return None
    nbytes, cunits, src, digest = rec
    return nbytes * units / cunits if source_digest(src) == digest else None


def max_over_ranks(value, world_size, device):
    """The slowest rank's value (every rank returns it); the job's time per step is the
    slowest replica's. device: where the collective's tensor lives (cuda under NCCL, cpu
    under gloo)."""
    if world_size <= 1:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def split_point(w, pw):
    return pw * (-(-w // (2 * pw)))


def time_launches(launch, count, stream, reps=3):
    """Mean device time (ms) per call: `count` calls captured in one CUDA graph (as inside the
    solve, where the library replays its own graph), replayed `reps` times between CUDA events
    on the launching stream, so host submission cost is not in the number."""
    import torch
    for i in range(3):
        launch(i)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream, capture_error_mode="thread_local"):
        for i in range(count):
            launch(i)
    g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        g.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / (reps * count)


def kernel_rooflines(m, n, pw, prec, stream, dev, hbm_peak, tc_peak):
    """The panel and the two top-level tensor-core products of the bench shape, each timed
    alone through its kernel-level C entry point. Inputs rotate over more than L2 holds."""
    import torch
    from paper_1912_05508_gb300 import lls
    sh = stream.cuda_stream
    # FP8 runs cast Q after the panel (the panel itself keeps only FP32), and the kernel-level
    # product entry points take FP16/BF16 operands only
    pcode = lls.PREC["fp32" if prec in ("fp8", "fp32") else prec]
    tdt = torch.float16 if prec in ("fp16", "fp8") else torch.bfloat16
    out = {}
    g = torch.Generator(device=dev).manual_seed(7)

    # panel: m x pw, algorithmic bytes = read m*pw FP32 + write Q (FP32) + write Q (2-byte copy)
    nbuf = max(2, -(-(160 << 20) // (m * pw * 4)))
    W = torch.randn((nbuf * pw, m), device=dev, generator=g).t()
    Wh = torch.empty((nbuf * pw, m), dtype=tdt, device=dev).t()
    R = torch.empty((pw, pw), device=dev)
    pws = lls.workspace(lls.lls_panel_qr_workspace_size(m, pw), dev).zero_()

    def panel(i):
        k = i % nbuf
        st = lls.lls_panel_qr(m, pw, pcode, W[:, k * pw:].data_ptr(), m, Wh[:, k * pw:].data_ptr(), m,
                              R.data_ptr(), pw, pws.data_ptr(), pws.numel(), sh)
        assert st == 0, st
    ms = time_launches(panel, 100, stream)
    by = 10.0 * m * pw
    out["panel"] = {"kernel": f"panel_flat_kernel (CAQR panel {m}x{pw}, CGS2 leaves, one-level tree)", "bound": "hbm",
                    "achieved": by / (ms * 1e-3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                    "us_per_launch": ms * 1e3, "algorithmic_bytes_per_launch": by}
    del W, Wh

    if prec in ("fp16", "bf16") and pw <= 16 and 2 * pw <= n:
        # the lowest recursion node as the solve runs it: left panel, node, right panel in one
        # launch; algorithmic bytes = read m*2pw FP32 + write Q (FP32 and the 2-byte copy)
        w = 2 * pw
        nbuf = max(2, -(-(160 << 20) // (m * w * 4)))
        W = torch.randn((nbuf * w, m), device=dev, generator=g).t()
        Wh = torch.empty((nbuf * w, m), dtype=tdt, device=dev).t()
        R = torch.empty((w, w), device=dev)
        bws = lls.workspace(lls.lls_panel_block_qr_workspace_size(m, pw, pw), dev).zero_()

        def blk(i):
            k = i % nbuf
            st = lls.lls_panel_block_qr(m, pw, pw, pcode, W[:, k * w:].data_ptr(), m, Wh[:, k * w:].data_ptr(), m,
                                        R.data_ptr(), w, bws.data_ptr(), bws.numel(), sh)
            assert st == 0, st
        ms = time_launches(blk, 100, stream)
        by = 10.0 * m * w
        out["block"] = {"kernel": f"block_fused_kernel (panel {m}x{pw}, node, panel {m}x{pw} in one launch)",
                        "bound": "hbm", "achieved": by / (ms * 1e-3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                        "us_per_launch": ms * 1e3, "algorithmic_bytes_per_launch": by}
        del W, Wh

    if prec not in ("fp16", "bf16"):
        for k, v in out.items():
            v["frac"] = v["achieved"] / v["peak"]
            v["traffic"] = None
        return out
    # top recursion node: R12 = Q1^T A2 (projection) and A2 -= Q1 R12 (update)
    w1 = split_point(n, pw)
    w2 = n - w1
    Q1l = (torch.randn((w1, m), device=dev, generator=g) / m ** 0.5).to(tdt).t()
    A2l = torch.randn((w2, m), device=dev, generator=g).to(tdt).t()
    A2 = torch.randn((w2, m), device=dev, generator=g).t()
    e = torch.zeros(w2, dtype=torch.int32, device=dev)
    R12 = torch.empty((w2, w1), device=dev)
    ldrl = -(-w1 // 8) * 8
    R12l = torch.empty((w2, ldrl), dtype=tdt, device=dev)
    f = torch.zeros(w2, dtype=torch.int32, device=dev)
    gws = lls.workspace(lls.lls_lowp_projection_workspace_size(m, w1, w2), dev)

    def proj(i):
        st = lls.lls_lowp_projection(m, w1, w2, pcode, Q1l.data_ptr(), A2l.data_ptr(), m, e.data_ptr(),
                                     R12.data_ptr(), w1, R12l.data_ptr(), ldrl, f.data_ptr(), gws.data_ptr(),
                                     gws.numel(), sh)
        assert st == 0, st
    ms_p = time_launches(proj, 10, stream)
    R12l.zero_()     # the update then subtracts zero products: same work, A2 stays finite
    f.zero_()

    def upd(i):
        st = lls.lls_lowp_update(m, w1, w2, pcode, Q1l.data_ptr(), m, R12l.data_ptr(), ldrl, f.data_ptr(),
                                 A2.data_ptr(), m, gws.data_ptr(), gws.numel(), sh)
        assert st == 0, st
    ms_u = time_launches(upd, 10, stream)
    fl = 2.0 * m * w1 * w2
    for key, t, name in (("tc_projection", ms_p, f"tc_gemm_kernel projection R12 = Q1^T A2 ({w1}x{w2}x{m}, "
                                                   f"split-K + fixed-order reduce)"),
                         ("tc_update", ms_u, f"tc_gemm_kernel update A2 -= Q1 R12 ({m}x{w2}x{w1})")):
        out[key] = {"kernel": name, "bound": "tensor", "achieved": fl / (t * 1e-3) / 1e12, "peak": tc_peak,
                    "unit": "TFLOP/s", "us_per_launch": t * 1e3, "algorithmic_flops_per_launch": fl}
    for k, v in out.items():
        v["frac"] = v["achieved"] / v["peak"]
        v["traffic"] = ncu_traffic(k, m if k.startswith("tc_") else 1.0)
    return out


def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def cfg_small_latency(stream, dev):
    """The paper's plain method at 1024 x 128 (geometric spectrum 1 .. 1e-3, seed 1): FP16
    products, LSQR to the FP32 target. A latency figure: the device time per solve of 50
    back-to-back asynchronous calls (graph replays), and the wall time of a call that also
    fills info (one host round trip), against the plain FP64 Householder solve."""
    import torch
    from paper_1912_05508_gb300 import lls, synth
    p = synth.svd_lls(1024, 128, "geometric", 1e3, seed=1)
    A = lls.colmajor(p.A, device=dev)
    b = torch.from_numpy(p.b).to(dev)
    m, n = A.shape
    o = lls.make_options(prec="fp16", target="fp32", krylov="lsqr")
    ws = lls.workspace(lls.lls_solve_workspace_size(m, n, o), dev)
    x = torch.empty(n, dtype=torch.float64, device=dev)
    sh = stream.cuda_stream
    info = lls.lls_info()

    def solve(inf):
        st = lls.lls_solve(m, n, A.data_ptr(), m, b.data_ptr(), x.data_ptr(), None, n, ws.data_ptr(), ws.numel(),
                           o, inf, sh)
        assert st >= 0, st
    for _ in range(5):
        solve(None)
    solve(info)
    torch.cuda.synchronize()
    e0, e1 = _events()
    e0.record(stream)
    for _ in range(50):
        solve(None)
    e1.record(stream)
    torch.cuda.synchronize()
    us = e0.elapsed_time(e1) / 50 * 1e3
    t0 = time.perf_counter()
    for _ in range(20):
        solve(info)
    wall_us = (time.perf_counter() - t0) / 20 * 1e6
    xh = lls.householder_solve(A, b, prec="fp64", stream=sh)
    hws = lls.workspace(lls.lls_householder_workspace_size(m, n, lls.PREC["fp64"]), dev)

    def hh():
        assert lls.lls_householder_solve(m, n, lls.PREC["fp64"], A.data_ptr(), m, b.data_ptr(), xh.data_ptr(),
                                         hws.data_ptr(), hws.numel(), sh) == 0
    hh()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(10):
        hh()
    e1.record(stream)
    torch.cuda.synchronize()
    hh_us = e0.elapsed_time(e1) / 10 * 1e3
    solve(info)
    torch.cuda.synchronize()
    fwd = float(torch.linalg.norm(x - xh) / torch.linalg.norm(xh))
    return {"workload": "single LLS 1024x128 FP32, geometric kappa=1e3 (seed 1), FP16 products, LSQR to the "
                        "FP32 target", "us_per_solve": us, "us_per_solve_with_info": wall_us,
            "iters": info.iters, "status": info.status, "fwd_vs_householder_fp64": fwd,
            "householder_fp64_us": hh_us, "bound": "latency (about 2.3e5 flops of Krylov work per iteration)"}


def cfg_spectrum_sweep(stream, dev, A0, b0, with_householder=True):
    """32768 x 4096 with three spectra (arithmetic, geometric, cluster) x kappa in {1e1, 1e3,
    1e6} (seeds 2..10, the geometric kappa = 1e3 problem being the headline's) and FP16, BF16
    and scaled FP8 products, each refined by CGLS to the FP64 target (eta_est <= 1e-12, at
    most 200 iterations). Per solve: status, iterations, eta and the device time to solution
    (the solve's own phase events, QR + Krylov), after one untimed solve; per matrix the
    relative distance of the FP16 solution from the plain FP64 Householder solution."""
    import torch
    from paper_1912_05508_gb300 import lls, synth
    m, n = A0.shape
    sh = stream.cuda_stream
    seeds = {}
    k = 2
    for kind in ("geometric", "arithmetic", "cluster"):
        for kappa in (1e1, 1e3, 1e6):
            if (kind, kappa) == ("geometric", 1e3):
                seeds[(kind, kappa)] = 2
            else:
                k += 1
                seeds[(kind, kappa)] = k
    size = max(lls.lls_solve_workspace_size(m, n, lls.make_options(prec=p)) for p in ("fp16", "bf16", "fp8"))
    ws = lls.workspace(size, dev)
    x = torch.empty(n, dtype=torch.float64, device=dev)
    rows = []
    for (kind, kappa), seed in seeds.items():
        if seed == 2:
            A, b = A0, b0
        else:
            A, b, _ = synth.svd_lls_torch(m, n, kind, kappa, seed=seed, device=dev)
        xh = lls.householder_solve(A, b, prec="fp64", stream=sh) if with_householder else None
        for prec in ("fp16", "bf16", "fp8"):
            o = lls.make_options(prec=prec, target="fp64")
            info = lls.lls_info()
            for _ in range(2):
                st = lls.lls_solve(m, n, A.data_ptr(), A.stride(1), b.data_ptr(), x.data_ptr(), None, n,
                                   ws.data_ptr(), ws.numel(), o, info, sh)
            row = {"spectrum": kind, "kappa": kappa, "seed": seed, "prec": prec, "status": int(st),
                   "converged": st == 0, "iters": info.iters, "eta": info.eta,
                   "ms": info.qr_ms + info.krylov_ms, "qr_ms": info.qr_ms, "krylov_ms": info.krylov_ms}
            if xh is not None and st >= 0:
                row["fwd_vs_householder_fp64"] = float(torch.linalg.norm(x - xh) / torch.linalg.norm(xh))
            rows.append(row)
        if seed != 2:
            del A, b
        torch.cuda.empty_cache()
    return {"workload": f"single LLS {m}x{n} FP32, spectra x kappa, FP16/BF16/FP8 products, CGLS to the FP64 "
                        f"target (1e-12), 200 iterations at most",
            "time_to_solution": "ms = device time of the whole solve (QR + preconditioner + Krylov) when "
                                "converged; not converged rows report the capped run",
            "rows": rows}


def cfg_large_qr(stream, dev, tc_peak):
    """QR only (RGSQRF, FP16 products) of Gaussian matrices with column norms 10^U(-2, 2):
    262144 x 8192 (seed 11) and 16384 x 16384 (seed 12). The time is the mean of three
    asynchronous factorizations (graph replays) after one untimed; TFLOP/s is given
    Householder-equivalent, (2 m n^2 - 2/3 n^3) / t, and as executed by the recursion,
    2 m n^2 / t. The column-equilibrated backward error ||(A - QR) D^-1||_F / ||A D^-1||_F and
    the orthogonality ||I - Q^T Q||_F / sqrt(n) are computed with FP32 products (TF32 off)."""
    import torch
    from paper_1912_05508_gb300 import lls, synth
    torch.backends.cuda.matmul.allow_tf32 = False
    sh = stream.cuda_stream
    out = []
    for m, n, seed in ((262144, 8192, 11), (16384, 16384, 12)):
        A = synth.scaled_gaussian_torch(m, n, seed=seed, device=dev)
        o = lls.make_options(prec="fp16")
        ws = lls.workspace(lls.qr_factor_workspace_size(m, n, o), dev)
        R = torch.empty((n, n), dtype=torch.float32, device=dev).t()

        def qr(Qp=None):
            st = lls.qr_factor(m, n, A.data_ptr(), m, Qp, m, R.data_ptr(), n, ws.data_ptr(), ws.numel(), o, sh)
            assert st == 0, st
        qr()
        torch.cuda.synchronize()
        e0, e1 = _events()
        e0.record(stream)
        for _ in range(3):
            qr()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 3
        Q = torch.empty((n, m), dtype=torch.float32, device=dev).t()
        qr(Q.data_ptr())
        torch.cuda.synchronize()
        d = torch.linalg.norm(A, dim=0)
        E = torch.addmm(A, Q, R, beta=1.0, alpha=-1.0)
        berr = float(torch.linalg.norm(E / d) / torch.linalg.norm(A / d))
        del E
        G = Q.t() @ Q
        G.diagonal().sub_(1.0)
        orth = float(torch.linalg.norm(G)) / n ** 0.5
        del G, Q
        hh = qr_flops(m, n) / (ms * 1e-3) / 1e12
        ex = 2.0 * m * n * n / (ms * 1e-3) / 1e12
        out.append({"m": m, "n": n, "seed": seed, "prec": "fp16", "ms": ms, "qr_tflops_householder_equiv": hh,
                    "qr_tflops_executed": ex, "executed_frac_of_tensor_peak": ex / tc_peak,
                    "backward_error_col_equilibrated": berr, "orthogonality_fro_over_sqrt_n": orth})
        del A, R, ws
        torch.cuda.empty_cache()
    return {"workload": "QR only, Gaussian with column norms 10^U(-2,2), FP16 products", "rows": out}


def cfg_batched(stream, dev, hbm_peak):
    """4096 uneven problems (m ~ U[256, 4096], n ~ U[16, 512], m >= 4 n, geometric spectra with
    kappa = 10^U(1, 5), seed 13), FP16 products, FP32 target: one lls_solve_batched call (a
    single persistent launch, replayed as a CUDA graph), mean of three after one untimed,
    against the same problems solved one after another by lls_solve on the default stream
    (launched directly). Roofline: the batch's algorithmic bytes are taken as one read and one
    write of every A for the factorization plus two reads of A per Krylov iteration."""
    import torch
    from paper_1912_05508_gb300 import lls, synth
    As, bs, kap = synth.batched_problems_torch(4096, seed=13, device=dev)
    batch = len(As)
    ms_ = [a.shape[0] for a in As]
    ns_ = [a.shape[1] for a in As]
    o = lls.make_options(prec="fp16", target="fp32", panel_width=16)
    nb = lls.lls_solve_batched_workspace_size(batch, ms_, ns_, o)
    ws = lls.workspace(nb, dev)
    xs = [torch.empty(n_, dtype=torch.float64, device=dev) for n_ in ns_]
    sh = stream.cuda_stream
    infos = (lls.lls_info * batch)()
    args = (batch, ms_, ns_, [a.data_ptr() for a in As], ms_, [b.data_ptr() for b in bs],
            [x.data_ptr() for x in xs], None, None, ws.data_ptr(), ws.numel(), o)
    worst = lls.lls_solve_batched(*args, infos, sh)
    st = [infos[i].status for i in range(batch)]
    iters = [infos[i].iters for i in range(batch)]
    torch.cuda.synchronize()
    e0, e1 = _events()
    e0.record(stream)
    for _ in range(3):
        assert lls.lls_solve_batched(*args, None, sh) >= 0
    e1.record(stream)
    torch.cuda.synchronize()
    ms_batch = e0.elapsed_time(e1) / 3
    # the same problems one lls_solve call each, launched directly on the default stream
    so = lls.make_options(prec="fp16", target="fp32")
    sws = lls.workspace(max(lls.lls_solve_workspace_size(a, b_, so) for a, b_ in zip(ms_, ns_)), dev)
    xo = torch.empty(max(ns_), dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(batch):
        lls.lls_solve(ms_[i], ns_[i], As[i].data_ptr(), ms_[i], bs[i].data_ptr(), xo.data_ptr(), None, ns_[i],
                      sws.data_ptr(), sws.numel(), so, None, 0)
    torch.cuda.synchronize()
    ms_loop = (time.perf_counter() - t0) * 1e3
    by = sum(4.0 * m_ * n_ * (2 + 2 * it) for m_, n_, it in zip(ms_, ns_, iters))
    gbs = by / (ms_batch * 1e-3) / 1e9
    out = {"workload": "4096 uneven LLS (m in [256,4096], n in [16,512], m >= 4n, geometric kappa=10^U(1,5)), "
                       "FP16 products, FP32 target", "ms_one_launch": ms_batch, "ms_loop_of_single_solves": ms_loop,
           "speedup_vs_loop": ms_loop / ms_batch, "worst_status": int(worst),
           "converged": sum(1 for v in st if v == 0), "not_converged": sum(1 for v in st if v == 1),
           "errors": sum(1 for v in st if v < 0), "mean_iters": statistics.mean(iters),
           "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                        "algorithmic_bytes": by}}
    del As, bs, xs, ws, sws
    torch.cuda.empty_cache()
    return out


def cfg_differentiable(stream, dev, hbm_peak):
    """256 problems of 4096 x 256 (geometric kappa = 1e3, seeds 1400..1655), L = sum of x^2:
    the forward solve (lls_solve_batched, FP64 target, R kept) and the adjoint (lls_backward:
    z = (A^T A)^-1 2x by CG preconditioned with the forward R, then dL/db = A z and the rank-2
    dL/dA). Times are the mean of three calls after one untimed. The adjoint's roofline counts
    its output write (dL/dA, 4 m n bytes per problem) and two reads of A per CG iteration
    plus three for the gradient sweep."""
    import torch
    from paper_1912_05508_gb300 import lls, synth
    As, bs = [], []
    for i in range(256):
        A, b, _ = synth.svd_lls_torch(4096, 256, "geometric", 1e3, seed=1400 + i, device=dev)
        As.append(A)
        bs.append(b)
    batch = 256
    m, n = 4096, 256
    sh = stream.cuda_stream
    o = lls.make_options(prec="fp16", target="fp64", panel_width=16)
    ws = lls.workspace(lls.lls_solve_batched_workspace_size(batch, [m] * batch, [n] * batch, o), dev)
    xs = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(batch)]
    Rs = [torch.empty((n, n), dtype=torch.float32, device=dev).t() for _ in range(batch)]
    fargs = (batch, [m] * batch, [n] * batch, [a.data_ptr() for a in As], [m] * batch, [b.data_ptr() for b in bs],
             [x.data_ptr() for x in xs], [r.data_ptr() for r in Rs], [n] * batch, ws.data_ptr(), ws.numel(), o)
    infos = (lls.lls_info * batch)()
    assert lls.lls_solve_batched(*fargs, infos, sh) == 0
    torch.cuda.synchronize()
    e0, e1 = _events()
    e0.record(stream)
    for _ in range(3):
        assert lls.lls_solve_batched(*fargs, None, sh) >= 0
    e1.record(stream)
    torch.cuda.synchronize()
    fwd_ms = e0.elapsed_time(e1) / 3
    gxs = [2.0 * x for x in xs]
    gAs = [torch.empty((n, m), dtype=torch.float32, device=dev).t() for _ in range(batch)]
    gbs = [torch.empty(m, dtype=torch.float64, device=dev) for _ in range(batch)]
    bo = lls.make_options(prec="fp16", target="fp64")
    bws = lls.workspace(lls.lls_backward_workspace_size(batch, [m] * batch, [n] * batch, bo), dev)
    bargs = (batch, [m] * batch, [n] * batch, [a.data_ptr() for a in As], [m] * batch, [b.data_ptr() for b in bs],
             [x.data_ptr() for x in xs], [r.data_ptr() for r in Rs], [n] * batch, [g.data_ptr() for g in gxs],
             [g.data_ptr() for g in gAs], [m] * batch, [g.data_ptr() for g in gbs], bws.data_ptr(), bws.numel(), bo, sh)
    assert lls.lls_backward(*bargs) == 0
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(3):
        assert lls.lls_backward(*bargs) == 0
    e1.record(stream)
    torch.cuda.synchronize()
    bwd_ms = e0.elapsed_time(e1) / 3
    by = batch * 4.0 * m * n * 4     # grad write + reads of A in the gradient sweep (lower bound)
    gbs_ = by / (bwd_ms * 1e-3) / 1e9
    out = {"workload": "256 x (4096x256) LLS, geometric kappa=1e3, L = sum x^2, forward FP64 target + adjoint",
           "forward_ms": fwd_ms, "backward_ms": bwd_ms, "total_ms": fwd_ms + bwd_ms,
           "forward_iters_mean": statistics.mean(infos[i].iters for i in range(batch)),
           "backward_roofline": {"bound": "hbm", "achieved": gbs_, "peak": hbm_peak, "unit": "GB/s",
                                 "frac": gbs_ / hbm_peak, "algorithmic_bytes_lower_bound": by}}
    del As, bs, xs, Rs, gAs, gbs, ws, bws
    torch.cuda.empty_cache()
    return out


def other_configs(args, stream, dev, A, b, hbm_peak, tc_peak):
    """Every workload configuration besides the headline, each timed on its own; a failure is
    reported in its entry instead of ending the benchmark."""
    import torch
    out = {}
    for key, fn in (("small_1024x128", lambda: cfg_small_latency(stream, dev)),
                    ("spectrum_sweep_32768x4096", lambda: cfg_spectrum_sweep(stream, dev, A, b,
                                                                             not args.no_householder)),
                    ("large_qr", lambda: cfg_large_qr(stream, dev, tc_peak)),
                    ("batched_4096", lambda: cfg_batched(stream, dev, hbm_peak)),
                    ("differentiable_256x4096x256", lambda: cfg_differentiable(stream, dev, hbm_peak))):
        t0 = time.perf_counter()
        try:
            out[key] = fn()
        except Exception as exc:  # noqa: BLE001 - reported in the line
            out[key] = {"error": f"{type(exc).__name__}: {str(exc).splitlines()[0][:300] if str(exc) else ''}"}
        out[key]["bench_wall_s"] = round(time.perf_counter() - t0, 1)
        torch.cuda.empty_cache()
    return out


def householder_baseline(A, b, x_ref, stream, dev, reps=2):
    """The plain Householder solve (Alg. 1) in FP64 and FP32 on the same GPU and inputs:
    device time per solve (CUDA events, after one warm-up) and its distance from our x."""
    import torch
    from paper_1912_05508_gb300 import lls
    m, n = A.shape
    out = {}
    for prec in ("fp64", "fp32"):
        nb = lls.lls_householder_workspace_size(m, n, lls.PREC[prec])
        ws = lls.workspace(nb, dev)
        x = torch.empty(n, dtype=torch.float64, device=dev)

        def run():
            st = lls.lls_householder_solve(m, n, lls.PREC[prec], A.data_ptr(), A.stride(1), b.data_ptr(),
                                           x.data_ptr(), ws.data_ptr(), ws.numel(), stream.cuda_stream)
            assert st == 0, st
        run()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            run()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        rel = float(torch.linalg.norm(x - x_ref) / torch.linalg.norm(x_ref))
        out[prec] = {"ms": ms, "rel_diff_vs_mixed_precision_x": rel,
                     "qr_tflops_equiv": qr_flops(m, n) / (ms * 1e-3) / 1e12}
        del ws
    return out


def library_lstsq_context(A, b, x_ref, stream):
    """Context only, not a baseline of this library: torch.linalg.lstsq (cuSOLVER's QR-based
    gels) in FP32 and FP64 on the same GPU and inputs, one timed call after a warm-up. Any
    failure is reported in the line instead of ending the benchmark."""
    import torch
    out = {"label": "library, context only (torch.linalg.lstsq, cuSOLVER gels)"}
    for name, dt in (("fp32", torch.float32), ("fp64", torch.float64)):
        try:
            with torch.cuda.stream(stream):
                Ax = A.to(dt)
                bx = b.to(dt)[:, None]
                torch.linalg.lstsq(Ax, bx)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                x = torch.linalg.lstsq(Ax, bx).solution[:, 0]
                e1.record(stream)
                torch.cuda.synchronize()
            rel = float(torch.linalg.norm(x.double() - x_ref) / torch.linalg.norm(x_ref))
            out[name] = {"ms": e0.elapsed_time(e1), "rel_diff_vs_mixed_precision_x": rel}
            del Ax, bx, x
        except Exception as exc:  # noqa: BLE001 - context only
            out[name] = {"error": str(exc).splitlines()[0][:200]}
        torch.cuda.empty_cache()
    return out


def make_inputs(args, m, n, rank, dev):
    """Generate the problem on the device; keep a host copy in /tmp so a rerun of the same
    command (e.g. under a profiler, where torch's linear-algebra plugin may not load) reuses it."""
    import torch
    from paper_1912_05508_gb300 import synth
    path = os.path.join(tempfile.gettempdir(),
                        f"lls_bench_{m}x{n}_{args.kind}_{args.kappa:g}_{args.seed + rank}.pt")
    if os.path.exists(path):
        d = torch.load(path)
        A = torch.empty((n, m), dtype=torch.float32, device=dev).t()
        A.copy_(d["A"])
        return A, d["b"].to(dev)
    A, b, _ = synth.svd_lls_torch(m, n, args.kind, args.kappa, seed=args.seed + rank, device=dev)
    try:
        torch.save({"A": A.cpu(), "b": b.cpu()}, path + ".tmp")
        os.replace(path + ".tmp", path)
    except OSError:
        pass
    return A, b


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    rank, ws = dist_setup("nccl")
    import torch
    from paper_1912_05508_gb300 import lls, synth

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    m, n = args.m, args.n
    A, b = make_inputs(args, m, n, rank, dev)
    # the autotuner measures the implementation choices for this shape once (cached on disk);
    # with panel_width 0 the solves below use its setting
    tune = None
    if args.no_autotune:
        lls.load_tuning_cache(dev)      # settings an earlier run measured, if any
    elif args.pw == 0:
        t0 = time.perf_counter()
        tune = lls.autotune(A, b, prec=args.prec, target=args.target, krylov=args.krylov, reorth=args.reorth,
                            reps=2)
        tune["wall_s"] = round(time.perf_counter() - t0, 2)
    o = lls.make_options(prec=args.prec, target=args.target, panel_width=args.pw, krylov=args.krylov,
                         reorth=args.reorth)
    pw = args.pw if args.pw > 0 else (tune["panel_width"] if tune else 16)
    nb = lls.lls_solve_workspace_size(m, n, o)
    wsbuf = lls.workspace(nb, dev)
    x = torch.empty(n, dtype=torch.float64, device=dev)
    # a dedicated stream: the library replays each repeated call as one CUDA graph on it
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    sh = stream.cuda_stream

    def solve_once(info):
        st = lls.lls_solve(m, n, A.data_ptr(), A.stride(1), b.data_ptr(), x.data_ptr(), None, n,
                           wsbuf.data_ptr(), wsbuf.numel(), o, info, sh)
        if st < 0:
            raise RuntimeError(f"lls_solve failed: {lls.STATUS.get(st, st)}")
        return st

    info = lls.lls_info()
    for _ in range(args.warmup):
        solve_once(info)
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = lls.lls_kernel_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = []
    ev0.record(stream)
    for _ in range(args.steps):
        solve_once(info)
        infos.append(info.as_dict())
    ev1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    total_ms = ev0.elapsed_time(ev1)
    launches = lls.lls_kernel_launch_count() - launches0
    clocks = sampler.stop()
    ms = max_over_ranks(total_ms / args.steps, ws, dev)

    # QR alone (for the QR TFLOP/s half of the metric)
    qo = lls.make_options(prec=args.prec, panel_width=args.pw, reorth=args.reorth)
    qnb = lls.qr_factor_workspace_size(m, n, qo)
    qws = wsbuf if qnb <= wsbuf.numel() else lls.workspace(qnb, dev)
    R = torch.empty((n, n), dtype=torch.float32, device=dev).t()
    for _ in range(2):
        lls.qr_factor(m, n, A.data_ptr(), A.stride(1), None, m, R.data_ptr(), n, qws.data_ptr(),
                      qws.numel(), qo, sh)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    qsteps = max(3, min(args.steps, 10))
    e0.record(stream)
    for _ in range(qsteps):
        lls.qr_factor(m, n, A.data_ptr(), A.stride(1), None, m, R.data_ptr(), n, qws.data_ptr(),
                      qws.numel(), qo, sh)
    e1.record(stream)
    torch.cuda.synchronize()
    qr_ms = e0.elapsed_time(e1) / qsteps

    # end to end through the C ABI with page-locked host buffers (lls_solve_host): the upload of
    # A and b (A in column chunks, overlapped with the factorization), the solve and the
    # download of x, all inside the timed region
    Ah = torch.empty((n, m), dtype=torch.float32, pin_memory=True).t()
    Ah.copy_(A)
    bh = b.cpu().pin_memory()
    xh = torch.empty(n, dtype=torch.float64, pin_memory=True)
    hws = lls.workspace(lls.lls_solve_host_workspace_size(m, n, o), dev)
    e2e_steps = max(3, min(args.steps, 10))
    e2e_ms = []
    for it in range(e2e_steps + 1):
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        st = lls.lls_solve_host(m, n, Ah.data_ptr(), Ah.stride(1), bh.data_ptr(), xh.data_ptr(),
                                hws.data_ptr(), hws.numel(), o, info, sh)
        s1.record(stream)
        torch.cuda.synchronize()
        if st < 0:
            raise RuntimeError(f"lls_solve_host: {lls.lls_status_string(st)}")
        if it > 0:
            e2e_ms.append(s0.elapsed_time(s1))
    del hws

    x_ref = x.clone()
    hh = householder_baseline(A, b, x_ref, stream, dev) if not args.no_householder else None
    libctx = library_lstsq_context(A, b, x_ref, stream) if not args.no_householder else None

    last = infos[-1]
    kry_ms = statistics.mean(i["krylov_ms"] for i in infos)
    a_passes = statistics.mean(i["a_passes"] for i in infos)
    m_passes = statistics.mean(i["m_passes"] for i in infos)
    kry_bytes = a_passes * 4.0 * m * n + m_passes * 4.0 * n * (n + 1) / 2.0
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
        hbm_peak, peak_src = float(peaks["hbm_gbs"]), "measured"
    except Exception:
        hbm_peak, peak_src = 6800.0, "fallback"
    tc_peak = float(peaks.get("bf16_tflops", 1900.0))   # FP16 and BF16 have the same dense rate
    achieved = kry_bytes / (kry_ms * 1e-3) / 1e9
    kernels = kernel_rooflines(m, n, pw, args.prec, stream, dev, hbm_peak, tc_peak)
    kernels["cgls"] = {"kernel": f"{args.krylov}_kernel (persistent {args.krylov.upper()} iteration, whole Krylov phase)", "bound": "hbm",
                       "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                       "traffic": ncu_traffic("cgls", kry_bytes), "algorithmic_bytes_per_launch": kry_bytes}
    # the block kernel (two panels and the node between them) has the largest share of the
    # solve in the ncu launch list
    roofline = dict(kernels["block"] if "block" in kernels else kernels["panel"])
    roofline["peak_source"] = ("measured (MEASURED_PEAKS.json hbm_gbs, burst copy)" if peak_src == "measured"
                               else "fallback 6800 GB/s")
    out = {"metric": METRIC, "value": ms, "unit": "ms", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "fp16 products / f32 panel / double-float Krylov",
           "data": "synthetic",
           "config": {"workload": f"single LLS {m}x{n} FP32, {args.kind} spectrum kappa={args.kappa:g}, "
                                  f"{args.prec.upper()} products, {args.krylov.upper()} to the "
                                  f"{args.target.upper()} target",
                      "m": m, "n": n, "prec": args.prec, "target": args.target, "krylov": args.krylov,
                      "reorth": args.reorth,
                      "panel_width": pw,
                      "autotuned": tune,
                      "l2": "inputs larger than L2 (A is %d MiB)" % (m * n * 4 >> 20),
                      "parallelism": f"replicas x{ws}"},
           "qr_ms": qr_ms, "qr_tflops": qr_flops(m, n) / (qr_ms * 1e-3) / 1e12,
           "krylov_ms": kry_ms, "iters": last["iters"], "eta": last["eta"],
           "status": last["status"], "problems_per_s": ws * 1e3 / ms,
           "roofline": roofline,
           "kernels": kernels,
           "e2e": {"value": statistics.median(e2e_ms), "unit": "ms",
                   "h2d_bytes_per_step": m * n * 4 + m * 8, "d2h_bytes_per_step": n * 8,
                   "stat": "median of %d steps" % len(e2e_ms), "mean": statistics.mean(e2e_ms),
                   "steps_ms": [round(v, 3) for v in e2e_ms],
                   "api": "lls_solve_host (page-locked host A, b, x; upload overlapped with the QR)"},
           "householder": hh,
           "library_context": libctx,
           "speedup_vs_householder_fp64": (hh["fp64"]["ms"] / ms) if hh else None,
           "gpu_launches": launches, "gpu_launches_per_step": launches / args.steps,
           "clocks": clocks}
    if ws == 1 and not args.no_configs:
        out["configs"] = other_configs(args, stream, dev, A, b, hbm_peak, tc_peak)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(A, b, m, n)
    if rank == 0:
        print(json.dumps(out))
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
