"""Benchmark: tensor GB/s sketched + decomposed (randomized TR-ALS), mixed
precision vs plain FP32, on one GB300 per rank.

Workload (one step): an order-4 200x200x200x200 float32 tensor (6.4 GB) made
from TR ranks 10 with N(0,1) cores plus Gaussian noise at 30 dB, K_n = 25,
R_n = 10, 30 ALS sweeps: sketch (Algorithm 1 steps 4-5), QR and the
mode-product chain (steps 6-7), TR-ALS (step 9), back-projection (step 11)
and the RSE identity.  The input is synthetic, built on the GPU from seeded
cores; it is larger than L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--prec bf16|fp32|fp8] [--size S] [--no-cpu-baseline]

Multi-GPU: replicas only (each rank decomposes its own tensor, no collective
on the data path); value = all ranks' bytes / max-over-ranks time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "tensor GB/s sketched+decomposed at rel err <=1e-3: mixed vs plain FP32, same GB300"
WORKLOAD = "rTR-ALS order-4 200^4 fp32 (6.4 GB), TR rank 10 + 30 dB noise, K=25, R=10, 30 sweeps"
FP64_TFLOPS = 1.25       # GB300 nominal dense FP64 rate (the float64 sketch's roofline)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default=None, choices=["bf16", "fp32", "fp8"],
                    help="sketch/chain arithmetic (default: bf16 for c2, the workload's own for c1/c3)")
    ap.add_argument("--size", type=int, default=200, help="mode length (200 = the named workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-parity", action="store_true", help="skip the reduced-tensor parity check vs the oracle")
    ap.add_argument("--pair", action="store_true",
                    help="BF16: sketch the last two modes in one pass over X (RTR_PARAM_PAIR)")
    ap.add_argument("--inflight", type=int, default=6,
                    help="tensors in flight: consecutive steps on this many streams, each with its own plan, so that "
                         "the latency-bound TR-ALS runs of several tensors overlap one another and the HBM-bound "
                         "passes of the others (1 = one step after the other; at most steps - 1 are used)")
    ap.add_argument("--workload", default="c2", choices=["c2", "batch256", "c1", "c3"],
                    help="c2 = the 200^4 tensor (default); batch256 = 256 uneven image-like tensors; "
                         "c1 = FP64 60^4 TR-ALS; c3 = hyperspectral-shaped 1024x1024x256 TR-SVD")
    ap.add_argument("--streams", type=int, default=16, help="worker streams of the batched form")
    ap.add_argument("--batch-count", type=int, default=256, help="tensors of the batched workload (256 = the named workload)")
    ap.add_argument("--no-graph", action="store_true", help="batched form: eager runs, no CUDA graph")
    ap.add_argument("--batch-inflight", type=int, default=2,
                    help="batched form: batches in flight (each its own batch object, graph and stream), so that "
                         "one batch's grouped TR-ALS overlaps the next one's sketches")
    return ap.parse_args()


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples (SM clock, throttle reasons) during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- GPU arm

def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "of measured"
    except Exception:
        return 6800.0, "of fallback"


def ncu_traffic(kernel_key):
    """Per-launch DRAM bytes of the dominant kernel from the committed ncu
    summary (profiles/traffic.txt: "<key> <bytes>" lines), else None."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        for line in open(p):
            parts = line.split()
            if len(parts) == 2 and parts[0] == kernel_key:
                return int(parts[1])
    except Exception:
        pass
    return None


def build_input(dims, rank, snr_db, seed, device):
    import torch
    from paper_1901_01652_gb300 import rtr, workloads
    N = len(dims)
    R = [rank] * N
    cores = [torch.from_numpy(c).to(device) for c in workloads.tr_cores(dims, R, seed)]
    X = torch.empty(dims, dtype=torch.float32, device=device)
    work = torch.empty(rtr.rtr_reconstruct_work_bytes(dims, R), dtype=torch.uint8, device=device)
    rtr.rtr_reconstruct(dims, R, cores, "fp32", X, work)
    del work
    nrm = float(torch.linalg.vector_norm(X, dtype=torch.float64))
    sigma = workloads.snr_sigma(nrm, X.numel(), snr_db)
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    flat = X.view(-1)
    chunk = 1 << 28
    for i in range(0, flat.numel(), chunk):
        n = min(chunk, flat.numel() - i)
        flat[i:i + n].add_(torch.randn(n, generator=g, device=device, dtype=torch.float32), alpha=sigma)
    torch.cuda.synchronize()
    return X


class Pipeline:
    def __init__(self, dims, K, R, sweeps, prec, seed, device, pair=False):
        import torch
        from paper_1901_01652_gb300 import workloads
        from paper_1901_01652_gb300.api import RTRD
        self.eng = RTRD(dims, K, R, prec, seed, sweeps, device=device, pair=pair)
        Ke = self.eng.plan.K
        self.init = [torch.from_numpy(z).to(device) for z in workloads.als_init(Ke, R, seed)]
        self.ev = None

    def step(self, X, stream, events=None):
        from paper_1901_01652_gb300 import rtr
        e = self.eng
        for z, i in zip(e.Z, self.init):
            z.copy_(i, non_blocking=True)
        rec = (lambda i: events[i].record(stream)) if events is not None else (lambda i: None)
        rec(0)
        rtr.rtr_sketch(e.plan, X, e.Y, stream)
        rec(1)
        rtr.rtr_project(e.plan, X, e.Y, e.Q, e.P, stream)
        rec(2)
        rtr.rtr_als(e.plan, e.P, e.Z, True, e.err, stream)
        rec(3)
        rtr.rtr_backproject(e.plan, e.Z, e.Q, e.G, None, stream)
        rtr.rtr_rse(e.plan, e.P, e.Z, e.rse, None, stream)
        rec(4)


PARITY_DIMS = (8, 200, 200, 200)


def parity_vs_oracle(precs, device, seed=1903):
    """The GPU path against the FP64 oracle on an 8 x 200 x 200 x 200 tensor of
    the benchmark's recipe (TR rank 10 + 30 dB, K = 25, R = 10, 30 sweeps, the
    same start cores on both sides).  Its mode views run the benchmark's
    kernels at the 200^4 launch configurations (mode 1: TMA sketch with two M
    tiles and 64-wide chunks, as modes 0 and 1 of 200^4; mode 2: 64-wide
    chunks with a ragged tail, as mode 2 of 200^4; mode 3: the last-mode sketch and the first,
    tensor-core mode product at I = 200, K = 25; mode 0, I = 8 < K, is kept
    whole).  Returns
    {prec: ||Xhat_gpu - Xhat_oracle|| / ||Xhat_oracle||} with the distance
    taken by TR inner products of the back-projected cores."""
    import torch
    from oracle import rtrd as orc
    from oracle import tensor as ot
    from paper_1901_01652_gb300 import workloads
    from paper_1901_01652_gb300.api import RTRD
    dims, K, R, sweeps = PARITY_DIMS, (25,) * 4, (10,) * 4, 30
    S = ot.tr_full_unfolded(workloads.tr_cores(dims, R, seed))
    X32 = (S + workloads.snr_sigma(ot.fro(S), S.size, 30.0) * workloads.unit_noise(dims, seed)).astype(np.float32)
    del S
    init = workloads.als_init(orc.effective_K(dims, K), R, seed)
    order = orc.default_chain_order(dims, K)
    refs = {}
    out = {}
    Xd = torch.from_numpy(X32).to(device)
    for prec in precs:
        table = "fp8" if prec == "fp8" else "bf16"       # FP32 and BF16 plans draw the bfloat16 table
        if table not in refs:
            refs[table] = orc.rtrd(X32.astype(np.float64), K, R, "als", seed=seed, prec=table, sweeps=sweeps,
                                   init=init, order=order)["G"]
        Go = refs[table]
        eng = RTRD(dims, K, R, prec, seed, sweeps, device=device)
        eng.run(Xd, "als", init=[torch.from_numpy(z) for z in init])
        Gg = [g.cpu().numpy() for g in eng.cores()]
        d2 = ot.tr_inner(Gg, Gg) - 2.0 * ot.tr_inner(Gg, Go) + ot.tr_inner(Go, Go)
        out[prec] = float(np.sqrt(max(d2, 0.0) / ot.tr_inner(Go, Go)))
        del eng
    return out


def pipeline_bytes(dims, K, order, elem=4):
    """Algorithmic bytes of the sketch-and-projection phase (Algorithm 1 steps
    5-7): (strict, per_mode).  Every Y_n is needed before any Q_n and one
    Q_n before the chain starts, so at least two reads of X; the chain then
    writes and reads each intermediate once and writes P.  The per-mode
    accounting reads X once per projected mode and once more for the first
    product."""
    numel = int(np.prod(dims))
    cur = list(dims)
    inter = 0
    for i, n in enumerate(order):
        cur[n] = min(K[n], dims[n])
        t = int(np.prod(cur))
        inter += t * elem * (1 if i == len(order) - 1 else 2)
    nproj = sum(1 for k, d in zip(K, dims) if k < d)
    return 2 * numel * elem + inter, (nproj + 1) * numel * elem + inter


def time_steps_inflight(pipes, streams, X, steps, warmup, dist_max):
    """K steps with step i on streams[i % len(streams)] (its own plan), so that
    up to len(streams) tensors are in flight; every step runs the whole path.
    Returns (max-over-ranks ms for the K steps, kernel launches)."""
    import torch
    from paper_1901_01652_gb300 import rtr
    main = torch.cuda.current_stream()

    def run(n):
        for s in streams:
            s.wait_stream(main)
        for i in range(n):
            k = i % len(pipes)
            with torch.cuda.stream(streams[k]):
                pipes[k].step(X, streams[k])
        for s in streams:
            main.wait_stream(s)

    run(warmup)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dist_barrier()
    torch.cuda.synchronize()
    l0 = rtr.rtr_kernel_launches()
    t0.record(main)
    run(steps)
    t1.record(main)
    torch.cuda.synchronize()
    l1 = rtr.rtr_kernel_launches()
    dist_barrier()
    return dist_max(t0.elapsed_time(t1)), l1 - l0


def time_steps(pipe, X, steps, warmup, stream, dist_max):
    import torch
    from paper_1901_01652_gb300 import rtr
    for _ in range(warmup):
        pipe.step(X, stream)
    torch.cuda.synchronize()
    sk_events = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dist_barrier()
    torch.cuda.synchronize()
    l0 = rtr.rtr_kernel_launches()
    t0.record(stream)
    for i in range(steps):
        pipe.step(X, stream, sk_events[i])
    t1.record(stream)
    torch.cuda.synchronize()
    l1 = rtr.rtr_kernel_launches()
    dist_barrier()
    ms = t0.elapsed_time(t1)
    phases = [sum(ev[i].elapsed_time(ev[i + 1]) for ev in sk_events) / steps for i in range(4)]
    return dist_max(ms), phases, l1 - l0


_DIST = {"on": False}


def dist_barrier():
    if _DIST["on"]:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, device):
    """The maximum of x over the ranks of the process group (x itself when
    there is none): a step's time is the slowest rank's."""
    if not _DIST["on"]:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t[0])


def whole_job_gbps(world, bytes_per_rank, steps, ms):
    """Whole-job throughput in GB/s: every rank's bytes over `steps` steps
    divided by the max-over-ranks time `ms` (weak scaling: each rank
    decomposes its own tensor)."""
    return world * bytes_per_rank * steps / (ms * 1e-3) / 1e9


def run_ours(args):
    import torch
    from paper_1901_01652_gb300 import build, rtr
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
        _DIST["on"] = True
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    if rank == 0:
        build.build()
    if world > 1:
        dist_barrier()
    rtr.lib()

    def dist_max(x):
        return max_over_ranks(x, device)

    S = args.size
    dims, K, R, sweeps, snr, seed = (S, S, S, S), (25,) * 4, (10,) * 4, 30, 30.0, 1903 + rank
    X = build_input(dims, 10, snr, seed, device)
    xbytes = X.numel() * 4
    stream = torch.cuda.current_stream(device)

    # more tensors in flight than the timed steps can fill would time mostly the fill and drain
    inflight = max(1, min(args.inflight, max(2, args.steps - 1)))
    pipes = [Pipeline(dims, K, R, sweeps, args.prec, 1903, device, args.pair) for _ in range(inflight)]
    pipe = pipes[0]
    with ClockSampler(local) as clk:
        if inflight > 1:
            streams = [torch.cuda.Stream(device) for _ in range(inflight)]
            ms, launches = time_steps_inflight(pipes, streams, X, args.steps, args.warmup, dist_max)
        else:
            ms, phases, launches = time_steps(pipe, X, args.steps, args.warmup, stream, dist_max)
    if inflight > 1:
        # phase times and the sketch's roofline from steps run one after the other
        _, phases, _ = time_steps(pipe, X, max(2, args.steps // 2), 1, stream, dist_max)
    sk_ms = phases[0]
    clocks = clk.summary()
    ms_step = ms / args.steps
    value = whole_job_gbps(world, xbytes, args.steps, ms)
    torch.cuda.synchronize()
    rse_mixed = float(pipe.eng.rse.cpu()[0])

    out = {
        "metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"bf16": "bf16", "fp32": "f32", "fp8": "fp8-e4m3 sketch, bf16 chain"}[args.prec], "data": "synthetic",
        "config": {"workload": WORKLOAD if S == 200 else f"rTR-ALS order-4 {S}^4 fp32 (reduced)",
                   "dims": list(dims), "K": list(K), "R": list(R), "sweeps": sweeps, "snr_db": snr,
                   "prec": args.prec, "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas{world}",
                   "inflight": inflight, "sketch_pair": bool(args.pair)},
        "rse": rse_mixed,
        "phases_ms": {"sketch": round(phases[0], 4), "project": round(phases[1], 4), "als": round(phases[2], 4),
                      "backproject_rse": round(phases[3], 4)},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    # roofline of the dominant kernels: the sketch's passes over X, each reading
    # X once (|X| * 4 bytes of algorithmic traffic): one per projected mode, the
    # last two modes of a BF16 plan sharing one
    peak, peak_kind = measured_peak()
    nproj = sum(1 for k, d in zip(K, dims) if k < d)
    passes = rtr.rtr_plan_sketch_passes(pipe.eng.plan)
    per_launch_ms = sk_ms / passes
    achieved = xbytes / (per_launch_ms * 1e-3) / 1e9
    key = f"sketch_{args.prec}_{S}x4"
    strict, per_mode = pipeline_bytes(dims, K, list(pipe.eng.plan.order))
    ph_ms = phases[0] + phases[1]
    out["roofline"] = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                       "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                       "traffic": ncu_traffic(key), "kernel": key,
                       "sketch_passes": passes, "sketch_ms_per_pass": round(per_launch_ms, 4),
                       "sketch_ms_per_mode": round(sk_ms / nproj, 4),
                       "pipeline_bytes_per_step": strict, "pipeline_bytes_per_mode_accounting": per_mode,
                       "pipeline_ms": round(ph_ms, 4),
                       "pipeline_frac_strict": round(strict / (ph_ms * 1e-3) / 1e9 / peak, 4),
                       "pipeline_frac_per_mode": round(per_mode / (ph_ms * 1e-3) / 1e9 / peak, 4)}
    # plain FP32 arm on the same tensor
    if not args.no_plain and args.prec != "fp32":
        plains = [Pipeline(dims, K, R, sweeps, "fp32", 1903, device) for _ in range(inflight)]
        plain = plains[0]
        psteps = max(2, args.steps // 2)
        if inflight > 1:
            pms, _ = time_steps_inflight(plains, streams, X, psteps, inflight, dist_max)
            _, pph, _ = time_steps(plain, X, 1, 0, stream, dist_max)
        else:
            pms, pph, _ = time_steps(plain, X, psteps, 1, stream, dist_max)
        psk = pph[0]
        torch.cuda.synchronize()
        rse_plain = float(plain.eng.rse.cpu()[0])
        Xm = pipe.eng.reconstruct("fp32")
        Xp = plain.eng.reconstruct("fp32")
        diff = float(torch.linalg.vector_norm(Xm - Xp, dtype=torch.float64) /
                     torch.linalg.vector_norm(Xp, dtype=torch.float64))
        del Xm, Xp
        out["plain_fp32"] = {"value": round(world * xbytes * psteps / (pms * 1e-3) / 1e9, 3),
                             "ms_per_step": round(pms / psteps, 4), "rse": rse_plain,
                             "sketch_ms_per_mode": round(psk / nproj, 4),
                             "phases_ms": {"sketch": round(pph[0], 4), "project": round(pph[1], 4),
                                           "als": round(pph[2], 4), "backproject_rse": round(pph[3], 4)}}
        out["mixed_vs_plain_rel_diff"] = diff
        del plain, plains
    # end to end through the public API with host buffers: a stream of host
    # tensors, `inflight` of them in flight (copies overlap the other's compute)
    if not args.no_e2e:
        from paper_1901_01652_gb300.api import decompose_stream
        Xh = X.cpu().pin_memory()
        del X
        torch.cuda.empty_cache()
        ek = max(2 * inflight, min(args.steps, 6))
        engs = [p.eng for p in pipes]
        decompose_stream([Xh] * inflight, K, R, "als", args.prec, 1903, sweeps, init=pipe.init, engines=engs)
        torch.cuda.synchronize()
        t = time.perf_counter()
        res = decompose_stream([Xh] * ek, K, R, "als", args.prec, 1903, sweeps, init=pipe.init, engines=engs)
        el = time.perf_counter() - t
        d2h = sum(g.numel() * 8 for g in res[-1][0]) + 8
        out["e2e"] = {"value": round(world * xbytes * ek / el / 1e9, 3), "unit": "GB/s",
                      "h2d_bytes_per_step": int(xbytes), "d2h_bytes_per_step": int(d2h),
                      "ms_per_step": round(el / ek * 1e3, 3), "inflight": inflight}
        del Xh
        X = None
    parity = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle leg: the oracle timed on the host cores, and the 1e-3 gate
        # of the metric checked against it on a tensor that runs the same kernels
        X = None
        torch.cuda.empty_cache()
        out["cpu_baseline"] = cpu_baseline()
        if not args.no_parity:
            arms = [args.prec] + ([] if args.no_plain or args.prec == "fp32" else ["fp32"])
            parity = parity_vs_oracle(arms, device)
    if parity is not None:
        out["parity_vs_oracle"] = {"workload": "x".join(map(str, PARITY_DIMS)) + " tensor of the same recipe "
                                   "(TR rank 10 + 30 dB, K=25, R=10, 30 sweeps), the benchmark's kernel "
                                   "configurations; ||Xhat_gpu - Xhat_oracle|| / ||Xhat_oracle||",
                                   "rel": {k: float(f"{v:.3e}") for k, v in parity.items()}, "gate": 1e-3}
        bad = {k: v for k, v in parity.items() if not v <= 1e-3}
        if bad:
            out["rejected"] = f"parity vs the oracle above the 1e-3 gate: {bad}"
            out["value"] = None
    if rank == 0:
        print(json.dumps(out), flush=True)
    if _DIST["on"]:
        import torch.distributed as dist
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- oracle arms

SAMPLE_SIDE = 120        # the 200^4 workload's recipe on a 120^4 slice (about 25 s of oracle work)
REF_SAMPLE_SIDE = 48     # the reference arm's per-step sample (a bounded --steps/--warmup run)


def blas_threads():
    """Threads the oracle's BLAS runs with (threadpoolctl when present, else
    the thread-count variables, else the library default = all cores)."""
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        if info:
            return max(int(i.get("num_threads", 0)) for i in info)
    except Exception:
        pass
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(v, "").isdigit():
            return int(os.environ[v])
    return os.cpu_count()


def oracle_sample_step(side, seed):
    """One step of the same workload recipe on a bounded side^4 sample, run
    by the FP64 oracle; returns (bytes of X as float32, seconds)."""
    from oracle import rtrd as orc
    from oracle import tensor as ot
    from paper_1901_01652_gb300 import workloads
    dims, K, R = (side,) * 4, (25,) * 4, (10,) * 4
    S = ot.tr_full_unfolded(workloads.tr_cores(dims, R, seed))
    X = (S + workloads.snr_sigma(ot.fro(S), S.size, 30.0) * workloads.unit_noise(dims, seed)).astype(np.float32)
    X = X.astype(np.float64)
    init = workloads.als_init(orc.effective_K(dims, K), R, seed)
    t = time.perf_counter()
    out = orc.rtrd(X, K, R, "als", seed=seed, prec="fp32", sweeps=30, init=init)
    orc.rse_identity(ot.fro(X) ** 2, out["P"], out["Z"])
    return X.size * 4, time.perf_counter() - t


def cpu_baseline():
    b, s = oracle_sample_step(SAMPLE_SIDE, 1903)
    return {"value": round(b / s / 1e9, 6), "unit": "GB/s", "cores": blas_threads(), "kind": "oracle",
            "sample": f"{SAMPLE_SIDE}^4 slice of the same recipe (K=25, R=10, 30 sweeps), FP64 NumPy oracle "
                      f"({os.cpu_count()} host cores, BLAS threads {blas_threads()}), {s:.1f} s"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # untimed warm-up of the interpreter and BLAS on a small sample (each
    # timed step's cost is mostly the TR-ALS on P = 25^4, whatever the sample)
    for _ in range(args.warmup):
        oracle_sample_step(12, 1903)
    tot_b, tot_s = 0, 0.0
    for i in range(args.steps):
        b, s = oracle_sample_step(REF_SAMPLE_SIDE, 1903)
        tot_b += b
        tot_s += s
    v = tot_b / tot_s / 1e9
    out = {"metric": METRIC, "value": round(v, 6), "unit": "GB/s", "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(tot_s / args.steps * 1e3, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": WORKLOAD, "sample": f"{REF_SAMPLE_SIDE}^4 per step"},
           "cpu_baseline": {"value": round(v, 6), "unit": "GB/s", "cores": blas_threads(), "kind": "oracle",
                            "sample": f"{REF_SAMPLE_SIDE}^4 tensor of the same recipe per step"},
           "e2e": {"value": round(v, 6), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------------------- batched form

BATCH_WORKLOAD = ("256 image-like order-4 fp32 tensors, modes U{32..96}, TR rank r ~ U{4..12} (smoothed spatial "
                  "cores, 0..255 integer pixels), K_n = min(I_n, 2r), R_n = r, 20 sweeps")


def batch_inputs(device, count=256):
    """The batched workload on the device: per tensor t, smoothed TR cores
    (seed 1905 + 31 t) expanded by the library's reconstruct, mapped to pixels."""
    import torch
    from paper_1901_01652_gb300 import rtr, workloads
    cfg = workloads.CONFIGS["c4_batch256"]
    shapes = workloads.batch_shapes(count, cfg["lo"], cfg["hi"], cfg["rlo"], cfg["rhi"], cfg["seed"])
    Xs, Ks, Rs = [], [], []
    for t, (dims, r) in enumerate(shapes):
        cores = [torch.from_numpy(c).to(device) for c in workloads.smoothed_tr_cores(dims, r, cfg["seed"] + 31 * t)]
        X = torch.empty(dims, dtype=torch.float32, device=device)
        R = [r] * 4
        work = torch.empty(rtr.rtr_reconstruct_work_bytes(dims, R), dtype=torch.uint8, device=device)
        rtr.rtr_reconstruct(dims, R, cores, "fp32", X, work)
        Xs.append(workloads.to_pixels(X))
        K, Rr = workloads.batch_ranks(dims, r)
        Ks.append(K)
        Rs.append(Rr)
    torch.cuda.synchronize()
    return [s[0] for s in shapes], Xs, Ks, Rs, cfg


def batch_cpu_baseline(shapes, Ks, Rs, cfg, budget_s=15.0):
    """The FP64 oracle on the first tensors of the batch, one by one, until
    about budget_s seconds of work; returns GB/s of float32 input."""
    from oracle import rtrd as orc
    from oracle import tensor as ot
    from paper_1901_01652_gb300 import workloads
    tot_b, tot_s, n = 0, 0.0, 0
    for t, dims in enumerate(shapes):
        X = workloads.to_pixels(ot.tr_full(workloads.smoothed_tr_cores(dims, Rs[t][0], cfg["seed"] + 31 * t)))
        X = X.astype(np.float32).astype(np.float64)
        t0 = time.perf_counter()
        out = orc.rtrd(X, Ks[t], Rs[t], "als", seed=cfg["seed"] + t, prec="bf16", sweeps=cfg["sweeps"])
        orc.rse_identity(ot.fro(X) ** 2, out["P"], out["Z"])
        tot_s += time.perf_counter() - t0
        tot_b += X.size * 4
        n += 1
        if tot_s >= budget_s:
            break
    return {"value": round(tot_b / tot_s / 1e9, 6), "unit": "GB/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"first {n} tensors of the batch ({tot_b / 1e9:.2f} GB fp32), FP64 NumPy oracle, {tot_s:.1f} s"}


def run_batch(args):
    import torch
    from paper_1901_01652_gb300 import build, rtr
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    build.build()
    rtr.lib()
    shapes, Xs, Ks, Rs, cfg = batch_inputs(device, args.batch_count)
    N = 4
    xbytes = sum(X.numel() * 4 for X in Xs)
    # per-mode accounting: every projected mode's sketch reads X once, the
    # first mode product reads it once more
    mode_bytes = sum(X.numel() * 4 * (1 + sum(1 for k, d in zip(K, X.shape) if k < d)) for X, K in zip(Xs, Ks))
    params = rtr.make_params(cfg["prec"], cfg["seed"], cfg["sweeps"])
    if args.no_graph:
        params.flags = rtr.PARAM_NO_GRAPH
    # batches in flight: step i runs batch object i % nbf on its own stream, so
    # that one batch's grouped TR-ALS overlaps the next one's sketches
    nbf = max(1, min(args.batch_inflight, args.steps))
    batches, Gs, rses = [], [], []
    for _ in range(nbf):
        batches.append(rtr.rtr_batch_create(shapes, Ks, Rs, params, args.streams))
        Gs.append([[torch.empty(Rs[t][n] * shapes[t][n] * Rs[t][(n + 1) % N], dtype=torch.float64, device=device)
                    for n in range(N)] for t in range(len(shapes))])
        rses.append(torch.empty(len(shapes), dtype=torch.float64, device=device))
    b, G, rse = batches[0], Gs[0], rses[0]
    stream = torch.cuda.current_stream(device)
    bstreams = [torch.cuda.Stream(device) for _ in range(nbf)]
    t_first = time.perf_counter()
    rtr.rtr_batch_run(b, Xs, G, rse, stream)            # eager run, tuning, capture
    torch.cuda.synchronize()
    t_first = time.perf_counter() - t_first

    def run_steps(n):
        for st in bstreams:
            st.wait_stream(stream)
        for i in range(n):
            k = i % nbf
            rtr.rtr_batch_run(batches[k], Xs, Gs[k], rses[k], bstreams[k])
        for st in bstreams:
            stream.wait_stream(st)

    run_steps(max(nbf, args.warmup - 1))                 # every batch object captured and replayed once
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        run_steps(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    value = world * xbytes * args.steps / (ms * 1e-3) / 1e9
    r = rse.cpu().numpy()
    peak, peak_kind = measured_peak()
    achieved = mode_bytes * args.steps / (ms * 1e-3) / 1e9
    out = {
        "metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": BATCH_WORKLOAD if len(shapes) == 256 else f"first {len(shapes)} tensors of: " + BATCH_WORKLOAD,
                   "tensors": len(shapes), "total_gb": round(xbytes / 1e9, 3),
                   "streams": args.streams, "graph": not args.no_graph, "batches_in_flight": nbf,
                   "prec": cfg["prec"], "l2": "inputs larger than L2 (no flush)",
                   "parallelism": f"replicas{world}"},
        "rse": {"mean": float(r.mean()), "max": float(r.max())},
        "first_run_s": round(t_first, 3),
        "gpu_launches": rtr.rtr_batch_graph_kernels(b) * args.steps,
        "clocks": clk.summary(),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "peak_kind": peak_kind, "traffic": None,
                     "kernel": "whole batched step (one graph), per-mode accounting of X reads"},
    }
    if not args.no_e2e:
        Xh = [X.cpu().pin_memory() for X in Xs]
        Gh = [[torch.empty(g.shape, dtype=torch.float64).pin_memory() for g in gt] for gt in G]
        ek = max(1, min(args.steps, 3))
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(ek):
            for xd, xh in zip(Xs, Xh):
                xd.copy_(xh, non_blocking=True)
            rtr.rtr_batch_run(b, Xs, G, rse, stream)
            for gt, ght in zip(G, Gh):
                for g, gh in zip(gt, ght):
                    gh.copy_(g, non_blocking=True)
            torch.cuda.synchronize()
        el = time.perf_counter() - t
        d2h = sum(g.numel() * 8 for gt in G for g in gt)
        out["e2e"] = {"value": round(world * xbytes * ek / el / 1e9, 3), "unit": "GB/s",
                      "h2d_bytes_per_step": int(xbytes), "d2h_bytes_per_step": int(d2h),
                      "ms_per_step": round(el / ek * 1e3, 3)}
        del Xh, Gh
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = batch_cpu_baseline(shapes, Ks, Rs, cfg)
    if rank == 0:
        print(json.dumps(out), flush=True)
    for bb in batches:
        bb.close()


# ----------------------------------------------------------------------------- other single-tensor workloads

SINGLE = {
    "c1": dict(workload="rTR-ALS order-4 60^4 fp64 (104 MB), TR rank 5 + 40 dB noise, K=15, R=5, 20 sweeps",
               dims=(60, 60, 60, 60), K=(15,) * 4, R=(5,) * 4, prec="fp64", method="als", sweeps=20,
               eps=None, seed=1902, sample=(60, 60, 60, 60)),
    "c3": dict(workload="rTR-SVD hyperspectral-shaped 1024x1024x256 fp32 (1.07 GB), 20 abundance maps x 20 "
                        "spectra + 1% noise, K=(60,60,30), eps=1e-2, block-scaled FP8 sketch",
               dims=(1024, 1024, 256), K=(60, 60, 30), R=(16, 16, 16), prec="fp8", method="svd", sweeps=1,
               eps=1e-2, seed=1904, sample=(512, 512, 256),
               # the last (spectral) mode first: its product reads X once on the
               # tensor cores and does half the work of the 1024-long modes; then
               # mode 0, whose view of the intermediate has the longest contiguous runs
               chain_order=(2, 0, 1)),
}


def single_input(name, dims, seed, device, host=False):
    """The named workload's tensor (CUDA tensor, or float64 NumPy on the host
    for the oracle's sample)."""
    import torch
    from paper_1901_01652_gb300 import rtr, workloads
    if name == "c1":
        cores = workloads.tr_cores(dims, 5, seed)
        if host:
            from oracle import tensor as ot
            S = ot.tr_full(cores)
            return S + workloads.snr_sigma(ot.fro(S), S.size, 40.0) * workloads.unit_noise(dims, seed)
        R = [5] * len(dims)
        X = torch.empty(dims, dtype=torch.float64, device=device)
        work = torch.empty(rtr.rtr_reconstruct_work_bytes(dims, R), dtype=torch.uint8, device=device)
        rtr.rtr_reconstruct(dims, R, [torch.from_numpy(c).to(device) for c in cores], "fp64", X, work)
        nrm = float(torch.linalg.vector_norm(X))
        g = torch.Generator(device=device)
        g.manual_seed(seed)
        X.add_(torch.randn(dims, generator=g, device=device, dtype=torch.float64),
               alpha=workloads.snr_sigma(nrm, X.numel(), 40.0))
        return X
    H, W, B = dims
    A, Sg = workloads.hsi_factors(H, W, B, n_sig=20, n_bumps=40, seed=seed)
    if host:
        X = np.einsum("hws,bs->hwb", A, Sg)
        return X + 0.01 * np.linalg.norm(X) / np.sqrt(X.size) * workloads.unit_noise(X.shape, seed)
    X = (torch.from_numpy(A.reshape(-1, A.shape[-1])).to(device) @ torch.from_numpy(Sg.T).to(device))
    X = X.reshape(dims)
    nrm = float(torch.linalg.vector_norm(X))
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    X.add_(torch.randn(dims, generator=g, device=device, dtype=torch.float64), alpha=0.01 * nrm / X.numel() ** 0.5)
    return X.float().contiguous()


def single_step(eng, X, spec, stream, ranks=None):
    eng.sketch(X, stream)
    eng.project(X, stream)
    if spec["method"] == "als":
        eng.als(None, stream)
    else:
        eng.svd(spec["eps"], ranks, stream)
    eng.backproject(stream)
    eng.compute_rse(stream)


def run_single(args):
    import torch
    from paper_1901_01652_gb300 import build, rtr
    from paper_1901_01652_gb300.api import RTRD, decompose
    spec = dict(SINGLE[args.workload])
    if args.prec is not None and spec["prec"] != "fp64":
        spec["prec"] = args.prec
    local = int(os.environ.get("LOCAL_RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    build.build()
    rtr.lib()
    X = single_input(args.workload, spec["dims"], spec["seed"], device)
    xbytes = X.numel() * X.element_size()
    eng = RTRD(spec["dims"], spec["K"], spec["R"], spec["prec"], spec["seed"], spec["sweeps"],
               spec["eps"] or 1e-2, chain_order=spec.get("chain_order"), device=device)
    stream = torch.cuda.current_stream(device)
    # tensors in flight, one plan and stream each: tensor i + depth's passes
    # over X are enqueued before tensor i's decomposition, whose latency-bound
    # kernels then run beside them (TR-SVD reads its chosen ranks back on the
    # host, so the next tensor's work has to be in the queues before it)
    nf = max(1, min(args.inflight, max(2, args.steps - 1)))
    engs = [eng] + [RTRD(spec["dims"], spec["K"], spec["R"], spec["prec"], spec["seed"], spec["sweeps"],
                         spec["eps"] or 1e-2, chain_order=spec.get("chain_order"), device=device)
                    for _ in range(nf - 1)]
    streams = [torch.cuda.Stream(device) for _ in engs]

    def front(i):
        k = i % nf
        with torch.cuda.stream(streams[k]):
            engs[k].sketch(X, streams[k])
            engs[k].project(X, streams[k])

    def back(i):
        k = i % nf
        e, st = engs[k], streams[k]
        with torch.cuda.stream(st):
            if spec["method"] == "als":
                e.als(None, st)
            else:
                e.svd(spec["eps"], None, st)
            e.backproject(st)
            e.compute_rse(st)

    def run_steps(n):
        depth = max(1, nf - 1)
        for st in streams:
            st.wait_stream(stream)
        for i in range(min(depth, n)):
            front(i)
        for i in range(n):
            if i + depth < n:
                front(i + depth)
            back(i)
        for st in streams:
            stream.wait_stream(st)

    run_steps(max(args.warmup, nf))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = rtr.rtr_kernel_launches()
    with ClockSampler(local) as clk:
        e0.record(stream)
        run_steps(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
    launches = rtr.rtr_kernel_launches() - l0
    ms = e0.elapsed_time(e1)
    value = world * xbytes * args.steps / (ms * 1e-3) / 1e9
    # sketch alone (one launch set per step) for the roofline of the sketch kernels
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for _ in range(args.steps):
        eng.sketch(X, stream)
    s1.record(stream)
    torch.cuda.synchronize()
    nproj = sum(1 for k, d in zip(eng.plan.K, spec["dims"]) if k < d)
    # time per pass over X (one per projected mode, the last two modes of a
    # BF16 plan sharing one)
    sk_ms = s0.elapsed_time(s1) / args.steps / max(rtr.rtr_plan_sketch_passes(eng.plan), 1)
    peak, peak_kind = measured_peak()
    achieved = xbytes / (sk_ms * 1e-3) / 1e9
    out = {
        "metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "f32", "bf16": "bf16", "fp8": "fp8-e4m3 sketch, bf16 chain"}[spec["prec"]],
        "data": "synthetic",
        "config": {"workload": spec["workload"], "dims": list(spec["dims"]), "K": list(spec["K"]),
                   "prec": spec["prec"], "method": spec["method"], "l2": "inputs larger than L2 (no flush)"
                   if xbytes > 129e6 else "input smaller than L2 (resident between steps)",
                   "parallelism": f"replicas{world}"},
        "rse": float(eng.rse.cpu()[0]), "ranks": list(eng.ranks), "inflight": nf,
        "gpu_launches": int(launches), "clocks": clk.summary(),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1),
                     "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                     "traffic": None, "kernel": f"sketch_{spec['prec']}_{args.workload} (mean per mode)",
                     "sketch_ms_per_mode": round(sk_ms, 4)},
    }
    if spec["prec"] == "fp64":
        # the float64 sketch is bound by the FP64 pipe: 2 |X| K_n flops per mode
        # against GB300's nominal dense FP64 rate (no measured FP64 peak exists)
        kmean = sum(k for k, d in zip(eng.plan.K, spec["dims"]) if k < d) / max(nproj, 1)
        tflops = 2.0 * X.numel() * kmean / (sk_ms * 1e-3) / 1e12
        out["roofline"] = {"bound": "alu", "achieved": round(tflops, 4), "peak": FP64_TFLOPS, "unit": "TFLOP/s",
                           "frac": round(tflops / FP64_TFLOPS, 4), "peak_kind": "of nominal (FP64 dense)",
                           "traffic": None, "kernel": f"sketch_fp64_{args.workload} (mean per mode)",
                           "sketch_ms_per_mode": round(sk_ms, 4), "hbm_GBps": round(achieved, 1)}
    if not args.no_plain and spec["prec"] not in ("fp64", "fp32"):
        # plain FP32 arm on the same tensor, and how far the two reconstructions
        # are apart; TR-SVD ranks forced to the mixed arm's choice (equal ranks)
        plain = RTRD(spec["dims"], spec["K"], spec["R"], "fp32", spec["seed"], spec["sweeps"],
                     spec["eps"] or 1e-2, device=device)
        fr = list(eng.ranks) if spec["method"] == "svd" else None
        single_step(plain, X, spec, stream, fr)
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        psteps = max(1, args.steps // 2)
        p0.record(stream)
        for _ in range(psteps):
            single_step(plain, X, spec, stream, fr)
        p1.record(stream)
        torch.cuda.synchronize()
        pms = p0.elapsed_time(p1) / psteps
        Xm = eng.reconstruct("fp32")
        Xp = plain.reconstruct("fp32")
        out["plain_fp32"] = {"value": round(world * xbytes / (pms * 1e-3) / 1e9, 3), "ms_per_step": round(pms, 4),
                             "rse": float(plain.rse.cpu()[0]), "ranks": list(plain.ranks)}
        out["mixed_vs_plain_rel_diff"] = float(torch.linalg.vector_norm(Xm - Xp, dtype=torch.float64) /
                                               torch.linalg.vector_norm(Xp, dtype=torch.float64))
        del Xm, Xp, plain
    if not args.no_e2e:
        Xh = X.cpu().pin_memory()
        decompose(Xh, spec["K"], spec["R"], spec["method"], spec["prec"], spec["seed"], spec["sweeps"],
                  spec["eps"] or 1e-2, engine=eng)
        torch.cuda.synchronize()
        t = time.perf_counter()
        ek = max(1, min(args.steps, 3))
        for _ in range(ek):
            G, _, _ = decompose(Xh, spec["K"], spec["R"], spec["method"], spec["prec"], spec["seed"],
                                spec["sweeps"], spec["eps"] or 1e-2, engine=eng)
        el = time.perf_counter() - t
        out["e2e"] = {"value": round(world * xbytes * ek / el / 1e9, 3), "unit": "GB/s",
                      "h2d_bytes_per_step": int(xbytes), "d2h_bytes_per_step": int(sum(g.numel() * 8 for g in G) + 8),
                      "ms_per_step": round(el / ek * 1e3, 3)}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import rtrd as orc
        from oracle import tensor as ot
        Xs = single_input(args.workload, spec["sample"], spec["seed"], None, host=True)
        if spec["prec"] != "fp64":
            Xs = Xs.astype(np.float32).astype(np.float64)
        t = time.perf_counter()
        ref = orc.rtrd(Xs, spec["K"], spec["R"], spec["method"], seed=spec["seed"], prec=spec["prec"],
                       sweeps=spec["sweeps"], eps=spec["eps"])
        if spec["method"] == "als":
            orc.rse_identity(ot.fro(Xs) ** 2, ref["P"], ref["Z"])
        el = time.perf_counter() - t
        b = Xs.size * (8 if spec["prec"] == "fp64" else 4)
        out["cpu_baseline"] = {"value": round(b / el / 1e9, 6), "unit": "GB/s", "cores": os.cpu_count(),
                               "kind": "oracle", "sample": f"{'x'.join(map(str, spec['sample']))} tensor of the same "
                                                            f"recipe, FP64 NumPy oracle, {el:.1f} s"}
    if rank == 0:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "batch256":
        run_batch(a)
    elif a.workload in SINGLE:
        run_single(a)
    else:
        a.prec = a.prec or "bf16"
        run_ours(a)
