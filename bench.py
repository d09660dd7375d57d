#!/usr/bin/env python
"""Benchmark: DoF x V-cycles per second of the variable V-cycle (Sec. 3.2 of
arXiv:1602.04858) on the 256x256 RT_1 channelised-permeability workload.

Workload (synthetic, seeded; the paper's own fields are not available):
2-D unit square, 256x256 cells, levels 4x4 -> 256x256 (7 levels), RT_1 x Q_1,
Brinkman mu = 0.01, 20 random-walk channels two cells wide with c = 1
(permeability 1) in a c = 1e6 background (contrast 1e6); variable V-cycle with
m(J) = 2 and the symmetric multiplicative vertex-patch Schwarz smoother.

One step = one V-cycle B_J r (all levels: smoothing, residual, transfers,
coarse solve) on a seeded residual vector resident in HBM.  `value` is for
the mixed-precision V-cycle (FP32 vectors and patch inverses), the mode the
FP64 flexible GMRES uses as its preconditioner; the FP64 and BF16-inverse
V-cycles and the time to a 1e-8 relative residual of each mode are reported
beside it.  The finest-level patch inverses alone (416 MB in FP32) exceed the
L2 cache, so every V-cycle streams them from HBM.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With N > 1 (torchrun), each rank runs an independent replica on its own GPU
(a single solve has no data-parallel split: it would need a halo exchange
after every colour pass) and value sums the ranks' DoF x V-cycles over the
slowest rank's time.
"""
from __future__ import annotations

import os

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import json
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DoF·V-cycles/s and time-to-1e-8 residual (mixed/batched/learned vs FP64)"
UNIT = "DoF·V-cycles/s"
WORKLOAD = "channels_256"


def workload_config():
    if WORKLOAD == "lognormal_3d_64":
        return {"workload": "3-D 64^3 cells, 6 levels (2^3->64^3), RT_0 x Q_0, Darcy mu=0, c = exp(G), "
                            "G ~ GRF(sigma=3, 8 cells), variable V-cycle m(J)=2, symmetric multiplicative "
                            "vertex-patch Schwarz",
                "levels": 6, "n_fine": 64, "degree": 0, "mu": 0.0, "cycle": "variable, m(J)=2",
                "l2": "inputs larger than L2 (finest patch inverses 400 MB FP32 / 800 MB FP64 streamed per sweep)"}
    if WORKLOAD == "channels_256_rt2":
        return {"workload": "2-D 256x256 cells, 7 levels (4x4->256x256), RT_2 x Q_2, Brinkman mu=0.01, "
                            "20 random-walk channels (c=1) in c=1e6 background, variable V-cycle m(J)=2, "
                            "symmetric multiplicative vertex-patch Schwarz",
                "levels": 7, "n_fine": 256, "degree": 2, "mu": 0.01, "cycle": "variable, m(J)=2",
                "l2": "inputs larger than L2 (finest patch inverses 2.4 GB FP32 / 4.8 GB FP64 streamed per sweep)"}
    return {"workload": "2-D 256x256 cells, 7 levels (4x4->256x256), RT_1 x Q_1, Brinkman mu=0.01, "
                        "20 random-walk channels (c=1) in c=1e6 background, variable V-cycle m(J)=2, "
                        "symmetric multiplicative vertex-patch Schwarz",
            "levels": 7, "n_fine": 256, "degree": 1, "mu": 0.01, "cycle": "variable, m(J)=2",
            "l2": "inputs larger than L2 (finest patch inverses 416 MB FP32 / 832 MB FP64 streamed per V-cycle)"}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id=None):
        self.proc = None
        # raw samples (the summary goes into the JSON line); MG_CLOCKS_DIR picks the folder
        self.path = os.path.join(os.environ.get("MG_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"clocks_bench_{os.getpid()}.csv")
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200"]
        if gpu_id:
            cmd += ["-i", gpu_id]
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [s.strip() for s in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


def gpu_uuid(torch, dev):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


def _oracle_worker(seconds, seed, barrier, queue):
    """One oracle replica (single-threaded NumPy/SciPy): set-up, then FP64
    V-cycles of the full workload for `seconds` once every replica is set up."""
    from oracle import multigrid as mg
    from paper_1602_04858_gb300 import inputs
    w = inputs.workload(WORKLOAD)
    t0 = time.perf_counter()
    H = mg.Hierarchy(w["d"], w["n_coarse"], w["n_levels"], w["degree"], w["mu"], w["c"])
    setup_s = time.perf_counter() - t0
    LJ = H.levels[-1]
    r = np.random.default_rng(seed).standard_normal(LJ.S.ndof)
    barrier.wait()
    n = 0
    t0 = time.perf_counter()
    while True:
        mg.vcycle(H, r, m_fine=2, variable=True)
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    queue.put((n, el, setup_s, LJ.S.ndof))


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def available_memory_bytes():
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) * 1024
    except Exception:
        pass
    return None


def run_cpu_baseline(seconds=15.0, workers=None):
    """The FP64 oracle as it stands (plain NumPy/SciPy, single-threaded) on all
    host cores: one independent replica per core (each ~3.3 GB), the same
    replicas-only split as the GPU side, processes started with spawn.  value =
    the DoF x V-cycles of all replicas over the slowest replica's time."""
    import multiprocessing as mp
    cores = host_cores()
    if workers is None:
        workers = cores
        mem = available_memory_bytes()
        if mem is not None:
            workers = max(1, min(workers, int(mem // (4.5 * 2 ** 30))))
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(workers)
    queue = ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=(seconds, 7 + i, barrier, queue)) for i in range(workers)]
    for pr in procs:
        pr.start()
    res = [queue.get() for _ in procs]
    for pr in procs:
        pr.join()
    ndof = res[0][3]
    total = sum(n for n, _, _, _ in res)
    span = max(el for _, el, _, _ in res)
    per = [ndof * n / el for n, el, _, _ in res]
    return {"value": ndof * total / span, "unit": UNIT, "cores": workers, "host_cores": cores, "kind": "oracle",
            "per_core_value": float(np.mean(per)),
            "sample": f"{workers} single-threaded oracle replicas (one per core, NumPy/SciPy with BLAS threads = 1), "
                      f"{total} FP64 V-cycles of the full workload in {span:.1f} s after a "
                      f"{max(s for _, _, s, _ in res):.0f} s oracle set-up"}


def reference_arm(args, rank):
    if rank != 0:
        return
    from oracle import multigrid as mg
    from paper_1602_04858_gb300 import inputs
    w = inputs.workload(WORKLOAD)
    H = mg.Hierarchy(w["d"], w["n_coarse"], w["n_levels"], w["degree"], w["mu"], w["c"])
    LJ = H.levels[-1]
    r = np.random.default_rng(7).standard_normal(LJ.S.ndof)
    for _ in range(args.warmup):
        mg.vcycle(H, r)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        mg.vcycle(H, r)
    el = time.perf_counter() - t0
    value = LJ.S.ndof * args.steps / el
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"each step one FP64 oracle V-cycle of the full workload (single thread)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def aggregate_throughput(dofs, steps, local_ms, dist=None, device="cpu"):
    """Whole-job DoF x V-cycles/s over N independent replicas: the DoF-cycles of
    all ranks divided by the slowest rank's time (max over ranks)."""
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    world = 1
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        world = dist.get_world_size()
    ms_max = float(t.item())
    return dofs * steps * world / (ms_max / 1e3), ms_max


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the FP32 colour pass on the finest level of a workload, by workload and
# kernel, from an ncu capture of the kernel as it stands; each has to be taken
# again whenever its kernel changes (a workload without an entry reports null).
FINEST_PASS_DRAM_BYTES = {("channels_256", "warp"): 51.033344e6 + 0.011776e6,
                          # 64^3 RT_0: 9,261 patches of 20 dofs per colour
                          ("lognormal_3d_64", "warp"): 20.315392e6 + 0.0,
                          # RT_2 on the 256^2 mesh: the persistent block kernel
                          ("channels_256_rt2", "persistent blocks"): 277.022976e6 + 3.764992e6}


def vcycle_model(levels, d, prec, l2_bytes, m_fine=2, variable=True):
    """Algorithmic bytes and smoother FLOPs of one V-cycle (the hot path's
    per-V-cycle roofline): per level j >= 1 with N_j dofs and P_j patches of
    n_v dofs (nnz_j operator entries in a patch's rows),
        bytes_j = S_j + 2 m(j) (2C - 1)/C (3 N_j s_v) + 6 N_j s_v,
        S_j = P_j n_v^2 s_inv, counted once per V-cycle if it fits the L2
              cache, else 2 m(j) (2C - 1)/C times (one sweep per smoothing
              step and direction, C = 3^d colours),
        flops_j = 2 m(j) (2C - 1)/C P_j (2 n_v^2 + 2 nnz_j).
    s_v: bytes per vector entry (4, FP64: 8); s_inv: bytes per stored inverse
    entry (4, FP64: 8, BF16 inverses on the finest level: 2).
    levels: list of (N_j, P_j, n_v, nnz_j) for j = 1..J."""
    C = 3 ** d
    J = len(levels)
    total_b = total_f = 0.0
    for j, (N, P, nv, nnz) in enumerate(levels, start=1):
        s_v = 8 if prec == "fp64" else 4
        s_inv = 8 if prec == "fp64" else (2 if (prec == "fp32_bf16inv" and j == J) else 4)
        m = m_fine * (2 ** (J - j) if variable else 1)
        sweeps = 2 * m * (2 * C - 1) / C
        inv = P * nv * nv * s_inv
        total_b += (inv if inv <= l2_bytes else sweeps * inv) + sweeps * 3 * N * s_v + 6 * N * s_v
        total_f += sweeps * P * (2 * nv * nv + 2 * nnz)
    return total_b, total_f


def colour_pass_bytes(count, nv, s_inv, s_v):
    """Algorithmic bytes of one colour pass: each patch streams its n_v x n_v
    inverse once and reads b_v, x_v and writes x_v (3 n_v vector entries)."""
    return count * (nv * nv * s_inv + 3 * nv * s_v)


def end_to_end(args, make, rh, N, barrier, dist, dev, world):
    """The same metric through the C interface with host (pinned) buffers:
    every step copies r host->device and z device->host inside mg_vcycle."""
    import torch
    G = make("fp32")
    rp = torch.empty(N, dtype=torch.float64, pin_memory=True)
    rp.copy_(torch.as_tensor(rh))
    zp = torch.empty(N, dtype=torch.float64, pin_memory=True)
    for _ in range(2):
        G.vcycle(rp, zp)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        G.vcycle(rp, zp)
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_value, _ = aggregate_throughput(N, args.steps, 1e3 * e2e_s, dist, dev)

    return e2e_value


def batched_workload(per_size=16, sizes=(64, 128, 256, 512), pass_kernel=0):
    """64 independent problems: per_size each of 64^2, 128^2, 256^2, 512^2 cells (coarsest 4^2), RT_1,
    mu = 0.01, c = exp(G) with G ~ GRF(sigma_i, n/16), sigma_i ~ U[1, 3] (seed 4000 + i; i counts the
    problems of all four sizes, so a subset of the sizes keeps the same problems)."""
    from paper_1602_04858_gb300 import inputs
    probs = []
    i = 0
    for n in (64, 128, 256, 512):
        for _ in range(per_size):
            if n in sizes:
                sig = float(inputs.rng(4000 + i).uniform(1.0, 3.0))
                c = inputs.lognormal_c(n, 2, sig, n / 16.0, 4000 + i)
                probs.append(dict(dim=2, n_coarse=4, n_levels=int(np.log2(n // 4)) + 1, degree=1, mu=0.01, c=c,
                                  precision="fp32", pass_kernel=pass_kernel))
            i += 1
    return probs


def batched_figures(args, steps, warmup, solve=True):
    """Batched V-cycle (all problems, 4 right-hand sides) with CUDA events, and
    the batched FP64 FGMRES(20) time to 1e-8 on random load vectors (no
    divergence source, no-slip walls)."""
    import torch
    from paper_1602_04858_gb300 import mgdarcy
    sizes = tuple(int(v) for v in args.batch_sizes.split(","))
    probs = batched_workload(args.batch_per_size, sizes, args.pass_kernel)
    for p in probs:
        p["c"] = torch.as_tensor(p["c"], device="cuda")
    t0 = time.perf_counter()
    B = mgdarcy.Batch(probs, nrhs=4)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    total = B.total()
    rng = np.random.default_rng(17)
    r = torch.as_tensor(rng.standard_normal(total), device="cuda")
    z = torch.zeros_like(r)
    for _ in range(warmup):
        B.vcycle(r, z)
    torch.cuda.synchronize()
    l0 = B.launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler()
    torch.cuda.nvtx.range_push("timed_vcycles")   # lets profilers select the timed region
    e0.record()
    for _ in range(steps):
        B.vcycle(r, z)
    e1.record()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    launches = B.launches() - l0
    status = B.sync(check=False)
    stats = []
    if solve:
        # right-hand sides: random loads in the free velocity rows
        b = rng.standard_normal(total)
        for p in range(len(probs)):
            nd, off, _ = B.layout(p)
            n = probs[p]["c"].shape[0]
            N = 2 * n
            nu = 2 * (N + 1) * N
            for rr in range(4):
                seg = b[off + rr * nd: off + (rr + 1) * nd]
                seg[nu:] = 0.0
                ux = seg[:(N + 1) * N].reshape(N, N + 1)
                ux[:, 0] = ux[:, -1] = 0.0
                uy = seg[(N + 1) * N:nu].reshape(N + 1, N)
                uy[0, :] = uy[-1, :] = 0.0
        x = torch.zeros_like(r)
        stats, status = B.solve(torch.as_tensor(b, device="cuda"), x, tol=1e-8, maxit=400, restart=20, check=False)
    its = [s_.iterations for s_ in stats] or [0]
    # colour-pass choice per level of the first problem of each size: (kernel, right-hand sides per S_v load)
    names = {1: "warp", 2: "block", 3: "persistent blocks"}
    choice, seen = {}, set()
    for p_, pr in enumerate(probs):
        n = pr["c"].shape[0]
        if n in seen:
            continue
        seen.add(n)
        choice[f"{n}^2"] = {}
        for j in range(1, pr["n_levels"]):
            k, g, t = B.level_choice(p_, j)
            choice[f"{n}^2"][str(j)] = f"{names[k]}, {g} rhs per inverse load" + (f", {t} threads per row" if k == 2 else "")
    desc = (f"batched: {len(probs)} 2-D problems ({args.batch_per_size} each of "
            + ", ".join(f"{n}^2" for n in sizes) + " cells), RT_1, mu=0.01, lognormal c with sigma in [1,3], "
            "4 right-hand sides each, one CUDA graph per batched V-cycle, FP32 smoother")
    return {"workload": desc, "dofs_times_rhs": total, "vcycle_ms": ms / steps,
            "value": total * steps / (ms / 1e3), "unit": "DoF x rhs x V-cycles/s", "gpu_launches_per_vcycle":
                int(launches // max(1, steps)), "setup_s": setup_s, "clocks": clocks, "pass_choice": choice,
            "time_to_1e-8": {"ms": stats[0].solve_ms if stats else None, "converged": bool(status == 0),
                             "systems": len(stats), "iterations_max": int(max(its)),
                             "iterations_mean": float(np.mean(its)), "restart": 20} if solve else None}


def bench_batched(args):
    """The batched workload as the timed step (--workload batched)."""
    f = batched_figures(args, args.steps, args.warmup, solve=not args.no_companions)
    line = {"metric": METRIC, "value": f["value"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": f["vcycle_ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f["workload"], "dofs_times_rhs": f["dofs_times_rhs"], "l2": "inputs larger than L2",
                       "pass_kernel": args.pass_kernel, "pass_choice": f["pass_choice"]},
            "gpu_launches": f["gpu_launches_per_vcycle"] * args.steps, "clocks": f["clocks"], "setup_s": f["setup_s"],
            "time_to_1e-8": f["time_to_1e-8"]}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--workload", default="channels", choices=["channels", "batched", "rt2", "3d"],
                    help="channels: the 256^2 RT_1 benchmark; rt2: the same with RT_2 (no CPU baseline: the oracle's "
                         "RT_2 hierarchy needs about 6 GB per replica); 3d: 64^3 RT_0 Darcy on a lognormal field "
                         "(no CPU baseline); batched: 64 problems x 4 right-hand sides")
    ap.add_argument("--batch-per-size", type=int, default=16)
    ap.add_argument("--batch-sizes", default="64,128,256,512", help="batched: the mesh sizes taken (one group each)")
    ap.add_argument("--pass-kernel", type=int, default=0,
                    help="mg_problem.pass_kernel of every problem (0: each level's kernel timed at setup; 5: the "
                         "fixed rule, the same choice on the timed levels of the default workload, for runs under a "
                         "profiler, whose serialised launches change the timed choice)")
    ap.add_argument("--no-companions", action="store_true",
                    help="skip the FP64/BF16 V-cycles, the solves and the end-to-end pass (profiling runs)")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched companion figures")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank)
        return
    if args.workload == "batched":
        bench_batched(args)
        return
    if args.workload in ("rt2", "3d"):
        global WORKLOAD
        WORKLOAD = "channels_256_rt2" if args.workload == "rt2" else "lognormal_3d_64"
        args.no_cpu_baseline = True

    import torch
    from paper_1602_04858_gb300 import inputs, mgdarcy

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
            torch.cuda.synchronize()

    w = inputs.workload(WORKLOAD)
    dev = torch.device("cuda", local)
    cdev = torch.as_tensor(w["c"], device=dev)
    stream = torch.cuda.current_stream(dev)

    def make(prec, variable=True):
        return mgdarcy.Multigrid(w["d"], w["n_coarse"], w["n_levels"], w["degree"], w["mu"], cdev,
                                 precision=prec, m_fine=2, variable_cycle=variable, stream=stream.cuda_stream,
                                 pass_kernel=args.pass_kernel)

    torch.cuda.synchronize()
    t_setup = time.perf_counter()
    G = make("fp32")
    setup_s = time.perf_counter() - t_setup
    names = {1: "warp", 2: "block", 3: "persistent blocks"}
    pass_kernels = {j: names[G.pass_kernel(j)] + (f" ({G.row_threads(j)} threads per row)" if G.pass_kernel(j) == 2
                                                   else "") for j in range(1, w["n_levels"])}
    nu, npr = G.sizes()
    N = nu + npr
    # per level j >= 1: (dofs, patches, n_v, nonzeros of a patch's rows) for the V-cycle model
    J = w["n_levels"] - 1
    C = 3 ** w["d"]
    level_info = []
    for j in range(1, J + 1):
        cnts = [G.patch_info(j, col) for col in range(C)]
        level_info.append((sum(G.sizes(j)), sum(cn for cn, _ in cnts), cnts[0][1], G.patch_nnz(j)))
    l2_bytes = torch.cuda.get_device_properties(dev).L2_cache_size
    rng = np.random.default_rng(11 + rank)
    rh = rng.standard_normal(N)
    r = torch.as_tensor(rh, device=dev)
    z = torch.zeros_like(r)

    def time_vcycles(Gh, steps, warmup):
        for _ in range(warmup):
            Gh.vcycle(r, z)
        barrier()
        l0 = Gh.launches()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            Gh.vcycle(r, z)
        e1.record(stream)
        barrier()
        return e0.elapsed_time(e1), Gh.launches() - l0

    # --- timed region: the headline mixed-precision V-cycle ---------------------
    for _ in range(args.warmup):
        G.vcycle(r, z)
    barrier()
    # The timed region lasts well under the 200 ms sampling interval of
    # nvidia-smi, so the sampler runs from 0.6 s of untimed V-cycles (the same
    # load) through the end of the timed region.
    sampler = ClockSampler(gpu_uuid(torch, dev))
    t_load = time.perf_counter()
    while time.perf_counter() - t_load < 0.6:
        for _ in range(20):
            G.vcycle(r, z)
        torch.cuda.synchronize()
    barrier()
    torch.cuda.nvtx.range_push("timed_vcycles")   # lets profilers select the timed region
    ms, launches = time_vcycles(G, args.steps, 0)
    torch.cuda.nvtx.range_pop()
    clocks = sampler.stop()
    if clocks is not None:
        clocks["window"] = "0.6 s of untimed V-cycles, then the timed region"
    value, ms_max = aggregate_throughput(N, args.steps, ms, dist, dev)

    # --- dominant kernel: finest-level colour pass ---------------------------------
    # In the V-cycle the 2C - 1 passes of a symmetric smoothing step run back to
    # back (programmatic dependent launch overlaps each pass's prologue with
    # the previous pass), so the average launch duration is taken over whole
    # steps: CUDA events on the launching stream around each step of 2C - 1 passes.
    # Events around every single pass break that overlap; that (pessimistic)
    # figure is reported beside it as isolated_launch_ms.
    J = w["n_levels"] - 1
    C = 3 ** w["d"]
    order = list(range(C)) + list(range(C - 2, -1, -1))
    step_bytes = sum(colour_pass_bytes(*G.patch_info(J, col), 4, 4) for col in order)
    G.level_load(J, torch.zeros_like(r), r)
    reps = max(4, args.steps // 2)
    steps_ev = []
    for rep in range(reps + 1):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for col in order:
            G.colour_pass(J, col)
        b.record(stream)
        if rep > 0:
            steps_ev.append((a, b))
    iso = []
    for col in order:
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        G.colour_pass(J, col)
        b.record(stream)
        iso.append((a, b))
    torch.cuda.synchronize()
    tot_ms = sum(a.elapsed_time(b) for a, b in steps_ev)
    npasses = len(order) * len(steps_ev)
    hbm, peak_kind = peaks()
    achieved = step_bytes * len(steps_ev) / (tot_ms / 1e3) / 1e9
    avg_launch_ms = tot_ms / npasses
    per_launch_bytes = step_bytes / len(order)
    isolated_launch_ms = sum(a.elapsed_time(b) for a, b in iso) / len(iso)

    # --- where the V-cycle's time goes: per level, the pass time (graph of two
    # symmetric steps, mg_time_passes) x the passes a V-cycle runs there
    # (pre- and post-smoothing of m(j) steps, 2C - 1 passes for the first step
    # and 2C - 2 for each further one, C = 3^d colours; levels folded into the
    # dense sub-cycle run none)
    Ls = G.dense_level()
    level_breakdown = {}
    for j in range(Ls + 1, J + 1):
        m = 2 * 2 ** (J - j)
        C = 3 ** w["d"]
        passes = 2 * ((2 * C - 1) + (2 * C - 2) * (m - 1))
        us = G.time_passes(j)
        level_breakdown[str(j)] = {"n": w["n_coarse"] << j, "kernel": pass_kernels[j], "us_per_pass": us,
                                   "passes_per_vcycle": passes, "ms_per_vcycle": us * passes / 1e3}

    # --- companions: FP64 and BF16-inverse V-cycles, time to 1e-8 ----------------
    extra = {}
    vc_ms = {"fp32": ms_max / args.steps}
    solves = {}
    e2e_value = None
    bsol = rng.standard_normal(N)
    # random load in the velocity rows, no divergence source, boundary normal dofs zero
    b_host = torch.as_tensor(bsol)
    f = torch.as_tensor(bsol[:nu], device=dev)
    g = torch.zeros(npr, dtype=torch.float64, device=dev)
    for prec, Gh in (() if args.no_companions else (("fp32", G),)):
        x = torch.zeros_like(r)
        st, status = Gh.solve(f, g, x, tol=1e-8, maxit=400, check=False)
        solves[prec] = {"ms": st.solve_ms, "iterations": st.iterations, "rel_residual": st.rel_residual,
                        "converged": bool(st.converged)}
    del G
    torch.cuda.empty_cache()
    # (the standard V(2,2) cycle beside the paper's variable cycle: fewer
    # latency-bound coarse passes per preconditioner application)
    for prec, variable in (() if args.no_companions else (("fp64", True), ("fp32_bf16inv", True),
                                                          ("fp32", False))):
        Gh = make(prec, variable)
        key = prec if variable else prec + "_V(2,2)"
        ksteps = max(3, args.steps // 2)
        torch.cuda.nvtx.range_push("timed_vcycles_" + key)   # lets profilers select this mode's V-cycles
        ms_p, _ = time_vcycles(Gh, ksteps, 2)
        torch.cuda.nvtx.range_pop()
        extra[key] = N * ksteps / (ms_p / 1e3)
        vc_ms[key] = ms_p / ksteps
        x = torch.zeros_like(r)
        st, status = Gh.solve(f, g, x, tol=1e-8, maxit=400, check=False)
        solves[key] = {"ms": st.solve_ms, "iterations": st.iterations, "rel_residual": st.rel_residual,
                       "converged": bool(st.converged)}
        del Gh
        torch.cuda.empty_cache()

    # --- end to end through the C interface with host buffers ------------------
    if not args.no_companions:
        e2e_value = end_to_end(args, make, rh, N, barrier, dist, dev, world)

    # --- per-V-cycle roofline of every mode; ALU roofline of the FP64 mode -----------
    peaks_alu = {}
    if not args.no_companions:
        for kind in ("fp64", "fp32", "fp32x2"):
            try:
                peaks_alu[kind + "_tflops"] = mgdarcy.measure_fma_peak(kind)
            except Exception as ex:  # reported, not required
                peaks_alu[kind + "_tflops"] = None
                peaks_alu["error"] = str(ex)
    # --- cost of one ordering point between colour passes: grid barrier vs dependent launch ---
    sync_costs = None
    if not args.no_companions:
        sync_costs = {"unit": "us per ordering point", "grid_barrier": {}, "dependent_launch": {},
                      "note": "grid barrier: one cooperative launch, blocks of 160 threads; dependent launch: "
                              "a graph of launches with programmatic dependent launch, as the V-cycle runs"}
        nsm = torch.cuda.get_device_properties(dev).multi_processor_count
        try:
            for nb in (nsm, 2 * nsm, 4 * nsm):
                sync_costs["grid_barrier"][str(nb)] = mgdarcy.measure_sync_cost("grid_barrier", nb)
            for nb in (nsm, 441, 1800):
                sync_costs["dependent_launch"][str(nb)] = mgdarcy.measure_sync_cost("dependent_launch", nb)
        except Exception as ex:  # reported, not required
            sync_costs["error"] = str(ex)
    rv = {}
    for key, t in vc_ms.items():
        prec = key.split("_V(")[0]
        nbytes, flops = vcycle_model(level_info, w["d"], prec, l2_bytes, 2, "V(2,2)" not in key)
        ent = {"bytes": nbytes, "ms": t, "achieved_gbs": nbytes / (t / 1e3) / 1e9,
               "frac": nbytes / (t / 1e3) / 1e9 / hbm, "flops": flops,
               "achieved_tflops": flops / (t / 1e3) / 1e12}
        if prec == "fp64" and peaks_alu.get("fp64_tflops"):
            ent["alu_frac"] = ent["achieved_tflops"] / peaks_alu["fp64_tflops"]
        rv[key] = ent
    batched = None
    if not args.no_companions and not args.no_batched and world == 1:
        try:
            batched = batched_figures(args, 3, 1, solve=True)
        except Exception as ex:  # reported, not required
            batched = {"error": str(ex)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            cpu = run_cpu_baseline(args.cpu_seconds)
        except Exception as ex:  # the baseline is reported, not required
            cpu = {"value": None, "unit": UNIT, "cores": host_cores(), "kind": "oracle", "sample": f"failed: {ex}"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": dict(workload_config(), pass_kernel_by_level=pass_kernels),
                "e2e": ({"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * N, "d2h_bytes_per_step": 8 * N}
                        if e2e_value is not None else None),
                "gpu_launches": int(launches),
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                             "frac": achieved / hbm,
                             "traffic": FINEST_PASS_DRAM_BYTES.get((WORKLOAD, pass_kernels[J])),
                             "kernel": {"warp": "k_colour_pass", "block": "k_colour_pass_cta",
                                        "persistent blocks": "k_colour_pass_ctap"}[pass_kernels[J].split(" (")[0]]
                                       + "<%d,%d,float,float> (finest level)" % (w["d"], w["degree"]),
                             "peak_kind": peak_kind, "avg_launch_ms": avg_launch_ms,
                             "bytes_per_launch": per_launch_bytes, "isolated_launch_ms": isolated_launch_ms,
                             "timing": f"CUDA events around back-to-back symmetric steps ({len(order)} passes) on the "
                                       "launching stream, as the passes run inside the V-cycle"},
                "clocks": clocks,
                "roofline_vcycle": {"model": "algorithmic bytes of one V-cycle: per level the patch inverses once "
                                             "if the level's set fits the L2 cache, else once per sweep, plus the "
                                             "vector traffic of the sweeps, residual and transfers; achieved = bytes "
                                             "/ CUDA-event time of a V-cycle; frac against the measured HBM copy "
                                             "bandwidth (peak above); FP64 also against the measured FP64 FMA peak",
                                    "l2_bytes": l2_bytes, "modes": rv},
                "level_breakdown": {"dense_fold_level": Ls, "levels": level_breakdown},
                "alu_peaks": peaks_alu or None,
                "sync_costs": sync_costs,
                "setup_s": setup_s,
                "batched": batched,
                "cpu_baseline": cpu,
                "dofs": N,
                "fp64_value": extra.get("fp64"), "bf16inv_value": extra.get("fp32_bf16inv"),
                "fp32_v22_value": extra.get("fp32_V(2,2)"),
                "time_to_1e-8": solves}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
