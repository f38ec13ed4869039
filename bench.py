#!/usr/bin/env python
"""Benchmark of the PCG + aggregation-AMG pressure solve on one GB300.

Workload: the Q1 trilinear hex Laplacian on 128^3 nodes (2,097,152 dofs,
55.3M stored entries), z graded geometrically by 1.04 from a Dirichlet wall,
b = A x* with seeded x* ~ N(0,1), x0 = 0, rtol 1e-8 on ||r|| / ||b||.
A step is one complete solve (every V-cycle, Krylov update and true-residual
check until convergence) of one right-hand side; four seeded right-hand sides
are used in turn. The headline is the float32-V-cycle / float64-FCG(1) solve;
the plain float64 PCG solve is measured the same way beside it.

Prints one JSON line (rank 0). ``--impl reference`` times the CPU oracle on
the host instead (bounded sample, scaled to solves/s).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "solves/s + p50/p99 latency at rel.res 1e-8, mixed vs FP64 PCG-AMG; HBM GB/s"
UNIT = "solves/s"


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--N", type=int, default=128)
    ap.add_argument("--ratio", type=float, default=1.04)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--maxit", type=int, default=500)
    ap.add_argument("--nrhs", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--multi-k", type=int, default=32, help="right-hand sides of the multi-column form (0: skip)")
    ap.add_argument("--multi-N", type=int, default=160, help="mesh of the multi-column form (N^3 nodes)")
    ap.add_argument("--serve-sweep", action="store_true",
                    help="instead of the default run: arrival-rate sweep of the mixed and plain float64 servers "
                         "(--sweep-count requests per rate) and an 8 GB admission run")
    ap.add_argument("--sweep-count", type=int, default=2000)
    ap.add_argument("--large", action="store_true",
                    help="instead of the default run: one 320^3 mesh, 8 right-hand sides, per-level rates")
    ap.add_argument("--multi-reps", type=int, default=3)
    ap.add_argument("--batch-count", type=int, default=48, help="independent systems of the batched form (0: skip)")
    ap.add_argument("--serve-count", type=int, default=160,
                    help="requests per serving run over resident 64^3/128^3/192^3 meshes (0: skip)")
    ap.add_argument("--serve-sizes", type=int, nargs="+", default=[64, 128, 192])
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-engines", type=int, default=2)
    ap.add_argument("--serve-chunk", type=int, default=4)
    ap.add_argument("--serve-batch-min", type=int, default=3)
    ap.add_argument("--serve-no-solo", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the fixed sweep launch shapes")
    ap.add_argument("--no-refresh", action="store_true", help="skip the partial-reuse (amg_refresh) measurement")
    ap.add_argument("--gs-nu", type=int, default=4, help="sweeps of the hybrid Gauss-Seidel comparison (0: skip)")
    ap.add_argument("--gs-blocks", type=int, default=65536, help="row blocks per level of the Gauss-Seidel smoother")
    ap.add_argument("--no-smoothed", action="store_true", help="skip the smoothed-aggregation comparison")
    return ap.parse_args(argv)


# ----------------------------------------------------------------- ranks
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def init_dist(world, backend):
    if world <= 1:
        return None
    import torch.distributed as dist
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group(backend=backend)
    return dist


def max_over_ranks(value: float, dist, device=None) -> float:
    """Largest value over all ranks (the job's time is its slowest rank's)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, dist, device=None) -> float:
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (every 200 ms) while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ----------------------------------------------------------------- roofline
def algorithmic_bytes(kind: str, mode: str, n0: int, nnz0: int, n1: int, ib: int = 4,
                      flexible: bool = False, stored: int = 0, pat_entries: int = 0) -> float:
    """Compulsory DRAM bytes of one launch of a level-0 kernel (each array once).

    Matrix: a value per nonzero; a column (ib = 2 bytes for int16 offsets,
    else 4) per nonzero of the slices stored without a shared offset
    pattern, and for the slices with one (``pat_entries`` of the ``stored``
    entries) the pattern itself, ib per entry column, plus one pattern flag
    (ib) per slice; one int32 slice pointer per 32 rows. Vectors as the
    kernels read/write them (gathered vectors counted once). A vector the
    kernel launched just before wrote and this one reads (xp between the
    prolongation and the post sweep, 8-17 MB at 128^3) is served by the L2
    and not counted. ``flexible``: the FCG(1) beta in float64 too (the
    iterative coarsest solve), so the post sweep also reads q_old.
    """
    sptr = 4 * (n0 // 32 + 1)
    if pat_entries and stored:
        uf = pat_entries / stored
        idx = nnz0 * (1 - uf) * ib + ib * (pat_entries / 32 + (n0 + 31) // 32)
    else:
        idx = nnz0 * ib
    vb = 4 if mode == "fcg32" else 8          # V-cycle value / vector bytes
    remit = 12 if mode == "fcg32" else 16     # r32 + xpre32 written, dinv32 read | xpre64 written, dinv read
    if kind == "spmv":      # p read, q written; float64 A
        return nnz0 * 8 + idx + n0 * 16 + sptr
    if kind == "axpy":      # z, p read; p written
        return n0 * 24
    if kind == "update":    # x, p, r, q read; x, r written; + the V-cycle's copy of r
        return n0 * (48 + remit)
    if kind == "residual":  # b, x read; r written; + the V-cycle's copy of r (columns entry by entry)
        return nnz0 * (8 + ib) + n0 * (24 + remit) + sptr
    if kind == "down0":     # xpre, b (r32 / r), p read; t written
        return nnz0 * vb + idx + n0 * 4 * vb + sptr
    if kind == "prolong0":  # xpre, p, agg read, x_1 gathered, xp written
        return n0 * (3 * vb + 4) + n1 * vb
    if kind == "post0":     # b (r32 | r), dinv read, z (float64) written; xp from L2
        post = nnz0 * vb + idx + n0 * (2 * vb + 8) + sptr
        if mode == "fcg32":
            post += n0 * 8                   # float64 r for r.z
        if mode == "fcg32" or flexible:
            post += n0 * 8                   # q_old for z.q_old
        return post
    raise KeyError(kind)


def kernel_source(kernel: str) -> str:
    """Text of a kernel's definition in solve.cu (template line to closing brace)."""
    src = open(os.path.join(ROOT, "paper_2210_16660_gb300", "csrc", "solve.cu")).read()
    m = re.search(r"(^template <[^\n]*\n)?^__global__[^\n]*?\b" + re.escape(kernel) + r"\(", src, flags=re.M)
    if not m:
        return ""
    end = src.find("\n}\n", m.start())
    return src[m.start(): end + 3]


def kernel_sha(kernel: str) -> str:
    """Hash of what decides a kernel's memory traffic: its own source and the
    sliced-ELL row helper it inlines."""
    h = hashlib.sha256(kernel_source(kernel).encode())
    with open(os.path.join(ROOT, "paper_2210_16660_gb300", "csrc", "sell_row.cuh"), "rb") as fh:
        h.update(fh.read())
    return h.hexdigest()[:16]


def committed_traffic(kernel: str, mode: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernel's
    source is still the one the counters were taken on."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        data = json.load(open(path))
    except (OSError, ValueError):
        return None
    ent = data.get("kernels", {}).get(f"{kernel}:{mode}")
    if not ent or ent.get("kernel_sha") != kernel_sha(kernel):
        return None
    return ent.get("dram_bytes_per_launch_full_size")


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# ----------------------------------------------------------------- oracle
def host_cpu() -> dict:
    """Host core count (threads the CPU baseline uses) and the CPU model."""
    cores = os.cpu_count() or 1
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    return {"cores": cores, "model": model}


def headline_config(args, n: int, nnz: int) -> dict:
    """The headline workload, printed identically by both arms."""
    return {"workload": f"q1_hex_{args.N}^3_zgrade{args.ratio}", "n": n, "nnz": nnz, "rtol": args.rtol,
            "mode": "fcg32 (float32 V-cycle in float64 FCG(1))", "n_pass": 2, "coarse_max": 200,
            "nrhs_cycled": args.nrhs,
            "l2": "inputs larger than L2 (level-0 values read per pass: 0.44 GB float64, 0.22 GB float32)",
            "parallelism": "replicas x1" if args.gpus <= 1 else f"replicas x{args.gpus}"}


def oracle_round(h, rhs, threads: int, rtol: float, maxit: int, offset: int = 0):
    """`threads` complete oracle solves (float32 V-cycle FCG(1), x0 = 0) run
    at once, one per host thread, right-hand sides cycled; the oracle's C
    calls release the interpreter lock, so they run on separate cores.
    Returns (wall seconds, iterations, largest true relative residual)."""
    from concurrent.futures import ThreadPoolExecutor

    def one(k):
        r = h.solve(rhs[(offset + k) % len(rhs)], rtol=rtol, maxit=maxit, mode="fcg32")
        if r["status"] != 0:
            raise RuntimeError(f"oracle solve status {r['status']}")
        return r["iters"], r["true_rel"]

    t = time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        res = list(ex.map(one, range(threads)))
    return time.perf_counter() - t, [r[0] for r in res], max(r[1] for r in res)


def run_reference(args):
    """The CPU oracle on the host cores, on the headline workload: every step
    is one complete solve per core, all cores at once (measured, not scaled)."""
    world, rank, local = dist_env()
    if rank != 0:
        return 0
    from paper_2210_16660_gb300 import workloads as W
    import oracle as O
    prob = W.make_problem(args.N, args.ratio, seed=args.seed)
    extra_b, _ = W.make_rhs(prob, args.nrhs - 1, seed=args.seed + 1000)
    rhs = [prob.b] + [np.ascontiguousarray(extra_b[:, c]) for c in range(args.nrhs - 1)]
    cpu = host_cpu()
    threads = cpu["cores"]
    h = O.Hierarchy(prob.A, n_pass=2)
    times, iters, worst = [], [], 0.0
    for s in range(args.warmup + args.steps):
        dt, its, tr = oracle_round(h, rhs, threads, args.rtol, args.maxit, offset=s)
        if s >= args.warmup:
            times.append(dt)
            iters += its
            worst = max(worst, tr)
    total = sum(times)
    value = threads * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": headline_config(args, prob.A.n, prob.A.nnz),
        "iters": {"median": statistics.median(iters), "min": min(iters), "max": max(iters)},
        "true_rel_max": worst,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "cpu_model": cpu["model"],
                         "kind": "oracle",
                         "sample": f"each step: {threads} complete solves of the 128^3 system at once, one per "
                                   f"host thread (right-hand sides cycled), measured end to end"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- ours
def timed_solves(amg, bs, x, steps, warmup, rtol, maxit, torch, stream, dist, device, profile=False):
    n_rhs = len(bs)
    for s in range(warmup):
        x.zero_()
        amg.solve(bs[s % n_rhs], x, rtol=rtol, maxit=maxit, stream=stream, hist=False)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    if profile:
        amg.profile(True)
        amg.profile_read()
        amg.profile_levels()
    launches0 = amg.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    iters = []
    t_all0 = torch.cuda.Event(enable_timing=True)
    t_all1 = torch.cuda.Event(enable_timing=True)
    t_all0.record(stream)
    for s in range(steps):
        ev[s][0].record(stream)
        x.zero_()
        res = amg.solve(bs[s % n_rhs], x, rtol=rtol, maxit=maxit, stream=stream, hist=False)
        ev[s][1].record(stream)
        if res.status != 0:
            raise RuntimeError(f"solve failed: {res.message}")
        iters.append(res.iters)
    t_all1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    launches = amg.launch_count() - launches0
    prof = amg.profile_read() if profile else None
    lev_prof = amg.profile_levels() if profile else None
    if profile:
        amg.profile(False)
    lat = [a.elapsed_time(b) for a, b in ev]
    total_ms = t_all0.elapsed_time(t_all1)
    return {"total_ms": total_ms, "lat_ms": lat, "iters": iters, "launches": launches, "prof": prof,
            "levels": lev_prof, "true_rel": res.true_rel}


def level_table(amg, lev_prof, mode: str, peak: float) -> list:
    """Per-level V-cycle time and HBM rate from a profiled pass.

    Algorithmic bytes per V-cycle of level l (each array once, gathered
    vectors once; vb = value bytes of the V-cycle precision, ib = column
    bytes, matrices as stored with their slice padding):
      down (l >= 1): matrix nnz_l (vb + ib) + xpre, b, p, t n_l vb;
      restriction l -> l+1: t n_l vb + member lists 4 (n_l + n_{l+1})
        + b, xpre, dinv of l+1 (float64 b on the coarsest);
      up (l >= 1): prolongation xpre, p, xp n_l vb + agg 4 n_l + x_{l+1};
        post: matrix nnz_l (vb + ib) + xp, b, dinv, x n_l vb;
      coarsest: the dense inverse 8 n_L^2 + b_L, x_L.
    """
    ms, cnt = lev_prof
    info = amg.info()
    L = len(info) - 1
    vb = 4 if mode == "fcg32" else 8
    # the coarsest span sits on the first level of the shared-memory tail
    # (when there is one): that level's time covers the tail levels below it
    tail = next((lvl for lvl in range(L + 1) if cnt[lvl][2] > 0), L)
    coarse_kind = amg.coarse_info().get("kind")
    out = []
    for lvl in range(L + 1):
        n = info[lvl][0]
        lay = amg.level_layout(lvl)
        z, ib = lay["stored"], lay["index_bytes"]
        pe = amg.level_pattern(lvl)["entries"]
        # one sweep's matrix: the values, and a column per entry of the slices
        # without a shared offset pattern (the pattern itself per entry column
        # and a flag per slice for the others)
        mat = z * vb + (ib * (z - pe) + ib * (pe / 32 + (n + 31) // 32) if pe else ib * z)
        nc = info[lvl + 1][0] if lvl < L else 0
        down = up = 0.0
        if lvl < L:
            restr = n * vb + 4 * (n + nc) + (nc * 8 if lvl + 1 == L else 3 * nc * vb)
            down = restr + (mat + 4 * n * vb if lvl > 0 else 0)
            up = (3 * n * vb + 4 * n + nc * vb + mat + 4 * n * vb) if lvl > 0 else 0
        elif coarse_kind == "iter":
            down = None  # FCG + block-Jacobi ILU(1): its inner iteration count varies per V-cycle
        else:
            down = 8 * n * n + 16 * n
        t = ms[lvl][0] / max(cnt[lvl][0], 1) + ms[lvl][1] / max(cnt[lvl][1], 1) + ms[lvl][2] / max(cnt[lvl][2], 1)
        byt = None if down is None else down + up
        row = {"level": lvl, "n": n, "stored": z, "us_per_vcycle": 1e3 * t,
               "algorithmic_bytes": byt, "gbs": byt / (t * 1e-3) / 1e9 if t > 0 and byt else None,
               "frac_of_hbm": byt / (t * 1e-3) / 1e9 / peak if t > 0 and byt else None}
        if down is None:
            row["note"] = "iterative coarsest solve (FCG + block-Jacobi ILU(1), at most the configured inner iterations)"
        if tail < L and lvl == tail:
            row["note"] = f"time of the shared-memory cluster tail, levels {tail}..{L}"
        elif lvl > tail:
            row["note"] = f"inside the cluster tail of level {tail}"
        out.append(row)
    return out


def pct(v, q):
    return float(np.percentile(np.asarray(v), q))


def serving_summary(serving: dict) -> dict | None:
    """Saturated solves/s and p50/p99 at the common rate for each server, in a
    few keys (the full record is under "serving")."""
    if not serving:
        return None
    out = {"common_rate_per_s": serving.get("common_rate")}
    for name in ("mixed", "fp64", "fp64_plain"):
        rec = serving.get(name)
        if not isinstance(rec, dict) or "saturated" not in rec:
            continue
        row = {"saturated_solves_per_s": rec["saturated"].get("solves_per_s")}
        common = rec.get("at_common_rate") or {}
        if common:
            row["p50_ms"] = common.get("p50_ms")
            row["p99_ms"] = common.get("p99_ms")
            row["all_ok"] = bool(common.get("all_ok")) and bool(rec["saturated"].get("all_ok"))
        out[name] = row
    return out


def run_ours(args):
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = init_dist(world, "nccl")
    device = torch.device("cuda", local)
    from paper_2210_16660_gb300 import binding as B
    from paper_2210_16660_gb300 import workloads as W
    B.load()
    prob = W.make_problem(args.N, args.ratio, seed=args.seed)
    extra_b, _ = W.make_rhs(prob, args.nrhs - 1, seed=args.seed + 1000)
    rhs = [prob.b] + [np.ascontiguousarray(extra_b[:, c]) for c in range(args.nrhs - 1)]
    stream = torch.cuda.current_stream()
    amg = B.AMG.from_csr(prob.A, mode="fcg32", stream=stream)
    setup = amg.setup_times()
    tune = {"enabled": not args.no_autotune}
    if not args.no_autotune:
        t0 = time.perf_counter()
        tune["changed"] = amg.autotune(reps=10, stream=stream)
        tune["ms"] = 1e3 * (time.perf_counter() - t0)
        tune["shapes"] = [amg.level_shape(lvl) for lvl in range(len(amg.info()))]
    levels = amg.info()
    bs = [torch.from_numpy(b).to(device) for b in rhs]
    x = torch.zeros(prob.A.n, dtype=torch.float64, device=device)

    sampler = ClockSampler(local)
    out, prof = {}, {}
    for mode in ("fcg32", "pcg64"):
        amg.set_mode(mode)
        if mode == "fcg32":
            sampler.start()
        # timed region: whole-solve graphs, no instrumentation
        out[mode] = timed_solves(amg, bs, x, args.steps, args.warmup, args.rtol, args.maxit, torch, stream,
                                 dist, device, profile=False)
        if mode == "fcg32":
            clocks = sampler.stop()
        # same solves again with CUDA events around every level-0 kernel
        prof[mode] = timed_solves(amg, bs, x, args.steps, 1, args.rtol, args.maxit, torch, stream, dist,
                                  device, profile=True)
    amg.set_mode("fcg32")

    # multi right-hand-side form: k columns of the same system in one solve
    multi = {}
    if args.multi_k > 0:
        r_m = args.ratio
        mprob = prob if args.multi_N == args.N else W.make_problem(args.multi_N, r_m, seed=4)
        mamg = amg if mprob is prob else B.AMG.from_csr(mprob.A, mode="fcg32", stream=stream)
        if mamg is not amg and not args.no_autotune:
            mamg.autotune(reps=10, stream=stream)
        Bm, _ = W.make_rhs(mprob, args.multi_k, seed=args.seed + 2000)
        Bd = torch.from_numpy(Bm).to(device)
        Xd = torch.zeros_like(Bd)
        multi["workload"] = f"q1_hex_{args.multi_N}^3_zgrade{r_m}"
        multi["n"] = mprob.A.n
        for mode in ("fcg32", "pcg64"):
            mamg.set_mode(mode)
            for _ in range(max(1, min(args.warmup, 2))):
                Xd.zero_()
                mamg.solve_multi(Bd, Xd, rtol=args.rtol, maxit=args.maxit, stream=stream, hist=False)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = args.multi_reps
            its = []
            e0.record(stream)
            for _ in range(reps):
                Xd.zero_()
                st, it, _, sts, tr = mamg.solve_multi(Bd, Xd, rtol=args.rtol, maxit=args.maxit, stream=stream,
                                                     hist=False)
                if st != 0:
                    raise RuntimeError(f"multi solve failed: {sts}")
                its.append(int(it.max()))
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            # the same right-hand sides one at a time (whole-solve graphs)
            xs = torch.zeros(mprob.A.n, dtype=torch.float64, device=device)
            cols = [Bd[:, c].contiguous() for c in range(min(args.multi_k, 4))]
            mamg.solve(cols[0], xs, rtol=args.rtol, maxit=args.maxit, stream=stream, hist=False)
            e0.record(stream)
            for col in cols:
                xs.zero_()
                mamg.solve(col, xs, rtol=args.rtol, maxit=args.maxit, stream=stream, hist=False)
            e1.record(stream)
            torch.cuda.synchronize()
            ms1 = e0.elapsed_time(e1) / len(cols)
            multi[mode] = {"k": args.multi_k, "ms_per_multi_solve": ms,
                           "solves_per_s": args.multi_k / (ms / 1e3), "max_iters": max(its),
                           "max_true_rel": float(np.max(tr)), "single_solves_per_s": 1e3 / ms1}
        mamg.set_mode("fcg32")
        if mamg is not amg:
            mamg.close()
        del Bd, Xd

    # batched form: independent graded systems of uneven size, one launch
    batch = {}
    if args.batch_count > 0:
        sizes = W.batch_sizes(args.batch_count, 24, 112, seed=3)
        bprobs = [W.make_problem(Nn, args.ratio, seed=3000 + k) for k, Nn in enumerate(sizes)]
        bamgs = [B.AMG.from_csr(p.A, mode="fcg32", stream=stream) for p in bprobs]
        if not args.no_autotune:
            for a in bamgs:
                a.autotune(reps=10, stream=stream)
        bb = [torch.from_numpy(p.b).to(device) for p in bprobs]
        bx = [torch.zeros_like(v) for v in bb]
        bt = B.Batch(bamgs)
        for _ in range(2):
            for v in bx:
                v.zero_()
            bt.solve(bb, bx, rtol=args.rtol, maxit=args.maxit, stream=stream)
        torch.cuda.synchronize()
        reps = args.multi_reps
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            for v in bx:
                v.zero_()
            st, bit, bsts = bt.solve(bb, bx, rtol=args.rtol, maxit=args.maxit, stream=stream)
            if st != 0:
                raise RuntimeError(f"batch solve failed: {bsts}")
        e1.record(stream)
        torch.cuda.synchronize()
        ms_batch = e0.elapsed_time(e1) / reps
        # the same systems one after another (each its own whole-solve graph)
        e0.record(stream)
        for k in range(len(bamgs)):
            bx[k].zero_()
            bamgs[k].solve(bb[k], bx[k], rtol=args.rtol, maxit=args.maxit, stream=stream, hist=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_seq = e0.elapsed_time(e1)
        batch = {"systems": len(sizes), "dofs": int(sum(Nn ** 3 for Nn in sizes)), "mode": "fcg32",
                 "ms_per_batch": ms_batch, "solves_per_s": len(sizes) / (ms_batch / 1e3),
                 "sequential_ms": ms_seq, "sequential_solves_per_s": len(sizes) / (ms_seq / 1e3),
                 "max_iters": int(bit.max())}
        bt.close()
        for a in bamgs:
            a.close()

    # serving: Poisson streams of warm-started solves over resident meshes;
    # the batching server (mixed and float64) against the plain float64
    # solver serving one request at a time, saturated and at a common rate
    serving = {}
    if args.serve_count > 0:
        from paper_2210_16660_gb300 import serving as SV
        meshes = SV.prepare_meshes(tuple(args.serve_sizes), ratio=args.ratio, seed=5, pool=4, device=device)
        if not args.no_autotune:
            for mm in meshes:
                mm.amg.autotune(reps=10, stream=stream)
        kw = dict(slots=args.serve_slots, max_engines=args.serve_engines, chunk=args.serve_chunk,
                  rtol=args.rtol, maxit=args.maxit, solo=not args.serve_no_solo, batch_min=args.serve_batch_min)
        srv = SV.make_server(meshes, "fcg32", **kw)
        plan = [dict(zip(("engines", "slots", "engine_bytes", "resident_bytes"), srv.mesh_info(i)))
                for i in range(len(meshes))]
        srv.close()
        res = SV.serve_modes(meshes, args.serve_count, load_fraction=0.7, seed=5, **kw)
        serving = {"meshes": [{"name": mm.name, "n": mm.problem.A.n, **pl} for mm, pl in zip(meshes, plan)],
                   "requests_per_run": args.serve_count, "arrivals": "Poisson, mesh uniform, seed 5",
                   "warm_start": "x0 = previous step's x*, x*_t = x*_{t-1} + 0.01 rms(x*_{t-1}) xi_t",
                   "server": {"slots": args.serve_slots, "max_engines": args.serve_engines,
                              "chunk": args.serve_chunk, "solo": not args.serve_no_solo,
                              "batch_min": args.serve_batch_min}, **res}
        for mm in meshes:
            mm.amg.close()
        del meshes

    # partial reuse (Sec. 4): the same mesh with new coefficients D A D; the
    # hierarchy keeps its aggregates and rebuilds its coarse operators,
    # smoothers and coarsest inverse, against a fresh setup of the new matrix
    refresh = {}
    if not args.no_refresh:
        A2 = W.rescaled(prob.A, seed=args.seed + 2000)
        b2 = torch.from_numpy(W.spmv(A2, W.normals(args.seed + 2001, prob.A.n))).to(device)
        ra = B.AMG.from_csr(prob.A, mode="fcg32", stream=stream)
        times = []
        for k in range(3):
            ra.refresh(A2 if k % 2 == 0 else prob.A, stream=stream)
            times.append(ra.refresh_ms())
        ra.refresh(A2, stream=stream)
        times.append(ra.refresh_ms())
        fresh = B.AMG.from_csr(A2, mode="fcg32", stream=stream)
        row = {"workload": f"{prob.name} with coefficients (d_i d_j) a_ij, d = 1 + 0.5 u",
               "refresh_ms": statistics.median(times), "setup_ms": fresh.setup_times()["total_ms"]}
        for name, h in (("refreshed", ra), ("fresh", fresh)):
            xr = torch.zeros_like(b2)
            h.solve(b2, xr, rtol=args.rtol, maxit=args.maxit, stream=stream, hist=False)   # graph capture
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            xr.zero_()
            e0.record(stream)
            r = h.solve(b2, xr, rtol=args.rtol, maxit=args.maxit, stream=stream, hist=False)
            e1.record(stream)
            torch.cuda.synchronize()
            if r.status != 0:
                raise RuntimeError(f"refresh check solve failed: {r.message}")
            row[name] = {"iters": r.iters, "solve_ms": e0.elapsed_time(e1), "true_rel": r.true_rel}
        refresh = row
        ra.close()
        fresh.close()

    # the paper's smoother (Sec. 3.1): nu = 4 sweeps of l1 hybrid Gauss-Seidel
    # over 65,536 row blocks per level, against the default one-sweep l1-Jacobi
    smoother = {}
    if args.gs_nu > 0:
        ga = B.AMG.from_csr(prob.A, mode="fcg32", stream=stream)
        smoother = {"workload": prob.name, "nu": args.gs_nu, "blocks_per_level": args.gs_blocks,
                    "rows_per_block_level0": -(-prob.A.n // args.gs_blocks)}
        for sm in ("l1_jacobi", "hybrid_gs"):
            if sm == "hybrid_gs":
                ga.set_smoother(args.gs_nu, args.gs_blocks, stream=stream)
            row = {}
            for mode in ("fcg32", "pcg64"):
                ga.set_mode(mode)
                m = timed_solves(ga, bs, x, 3, 1, args.rtol, args.maxit, torch, stream, None, device)
                row[mode] = {"iters": statistics.median(m["iters"]), "ms_per_solve": m["total_ms"] / 3,
                             "solves_per_s": 3e3 / m["total_ms"], "kernels_per_solve": m["launches"] / 3}
            smoother[sm] = row
        ga.close()

    # smoothed aggregation (Sec. 3.1): P = (I - omega D^-1 A) P_hat on every
    # level against the tentative P_hat, same system and right-hand sides
    smoothed = {}
    if not args.no_smoothed:
        smoothed = {"workload": prob.name,
                    "note": "tentative n_pass = 2 (the default) against smoothed aggregation with the paper's "
                            "aggregate sizes |G| <= 8 (n_pass = 3, MLVSMATCH3) and |G| <= 16 (n_pass = 4, "
                            "MLVSMATCH4); l1-Jacobi smoothing in all three"}
        cands = [("tentative_npass2", amg, False)]
        for npass in (3, 4):
            t0 = time.perf_counter()
            sa = B.AMG.from_csr(prob.A, mode="fcg32", stream=stream, smoothed=True, n_pass=npass)
            torch.cuda.synchronize()
            cands.append((f"smoothed_npass{npass}", sa, True))
        for name, h, is_sa in cands:
            info = h.info()
            vb = {"fcg32": 4, "pcg64": 8}
            row = {"levels": len(info), "rows_nnz": info,
                   "operator_complexity": sum(z for _, z in info) / info[0][1]}
            for mode in ("fcg32", "pcg64"):
                h.set_mode(mode)
                m = timed_solves(h, bs, x, 3, 1, args.rtol, args.maxit, torch, stream, None, device)
                # V-cycle bytes: two sweeps of every level's matrix as stored
                # (values + columns) plus the transfers (aggregate maps, or P
                # and P^T as CSR: value + column per entry, twice)
                byt = 0
                for l in range(len(info) - 1):
                    lay = h.level_layout(l)
                    byt += 2 * lay["stored"] * (vb[mode] + lay["index_bytes"])
                    if is_sa:
                        byt += 2 * len(h.prolongator(l)[1]) * (vb[mode] + 4)
                    else:
                        byt += 2 * info[l][0] * (vb[mode] + 4)
                its = statistics.median(m["iters"])
                row[mode] = {"iters": its, "ms_per_solve": m["total_ms"] / 3, "solves_per_s": 3e3 / m["total_ms"],
                             "vcycle_bytes": byt, "vcycle_bytes_x_iters": byt * its}
            h.set_mode("fcg32")
            row["setup_ms"] = h.setup_times()["total_ms"]
            smoothed[name] = row
        for name, h, is_sa in cands:
            if is_sa:
                h.close()

    # end to end through the C ABI with host buffers (pinned), copies inside the call
    pin_b = [torch.from_numpy(b).pin_memory().numpy() for b in rhs]
    pin_x = torch.zeros(prob.A.n, dtype=torch.float64).pin_memory().numpy()
    for s in range(args.warmup):
        pin_x[:] = 0.0
        amg.solve(pin_b[s % len(pin_b)], pin_x, rtol=args.rtol, maxit=args.maxit, stream=stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    e2e_iters = []
    for s in range(args.steps):
        pin_x[:] = 0.0
        res = amg.solve(pin_b[s % len(pin_b)], pin_x, rtol=args.rtol, maxit=args.maxit, stream=stream)
        e2e_iters.append(res.iters)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    if dist is not None:
        dist.barrier()

    # whole-job aggregation (replicas: every rank solves its own copy)
    m = out["fcg32"]
    tot_ms = max_over_ranks(m["total_ms"], dist, device)
    solves = sum_over_ranks(float(args.steps), dist, device)
    value = solves / (tot_ms / 1e3)
    f64 = out["pcg64"]
    f64_ms = max_over_ranks(f64["total_ms"], dist, device)
    e2e_s = max_over_ranks(e2e_s, dist, device)
    e2e_value = solves / e2e_s

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as O
        hc = host_cpu()
        t0 = time.perf_counter()
        ho = O.Hierarchy(prob.A, n_pass=2)
        setup_s = time.perf_counter() - t0
        dt, its, tr = oracle_round(ho, rhs, hc["cores"], args.rtol, args.maxit)
        cpu = {"value": hc["cores"] / dt, "unit": UNIT, "cores": hc["cores"], "cpu_model": hc["model"],
               "kind": "oracle",
               "sample": f"{hc['cores']} complete 128^3 solves (float32 V-cycle FCG(1)) at once, one per host "
                         f"thread, measured end to end ({dt:.1f} s; oracle setup {setup_s:.1f} s not counted)",
               "iters": statistics.median(its), "true_rel_max": tr}
        ho.close()

    # roofline of the dominant level-0 kernel in the headline mode
    peaks = measured_peaks()
    n0, nnz0 = levels[0]
    n1 = levels[1][0] if len(levels) > 1 else 0
    ib0 = amg.level_layout(0)["index_bytes"]
    stored0 = amg.level_layout(0)["stored"]
    pat0 = amg.level_pattern(0)
    peak = peaks.get("hbm_gbs")
    peak_src = "measured"
    if not peak:
        peak, peak_src = 6800.0, "fallback"
    kernel_names = {"down0": "k_down", "post0": "k_post", "prolong0": "k_prolong", "spmv": "k_spmv",
                    "update": "k_update", "residual": "k_residual", "axpy": "k_axpy_p"}

    def kernel_table(mode):
        pr = prof[mode]["prof"]
        table = {}
        for k, (ms, cnt) in pr.items():
            if cnt == 0:
                continue
            entry = {"avg_ms": ms / cnt, "launches": cnt, "share_of_profiled": ms / prof[mode]["total_ms"]}
            if k == "residual":
                entry["note"] = "runs a full sweep only when the recursive residual met rtol; other launches exit"
            elif k != "coarse_levels":
                bl = algorithmic_bytes(k, mode, n0, nnz0, n1, ib0, stored=stored0, pat_entries=pat0["entries"])
                entry["algorithmic_bytes"] = bl
                entry["gbs"] = bl / (ms / cnt * 1e-3) / 1e9
                entry["frac_of_hbm"] = entry["gbs"] / peak
            table[k] = entry
        return table

    per_kernel = kernel_table("fcg32")
    per_kernel64 = kernel_table("pcg64")
    levels32 = level_table(amg, prof["fcg32"]["levels"], "fcg32", peak)
    levels64 = level_table(amg, prof["pcg64"]["levels"], "pcg64", peak)
    cand = {k: v for k, v in per_kernel.items() if k not in ("coarse_levels", "residual")}
    dom = max(cand, key=lambda k: cand[k]["avg_ms"] * cand[k]["launches"])
    roofline_hbm = {"kernel": kernel_names[dom], "bound": "hbm", "achieved": cand[dom]["gbs"], "peak": peak,
                "unit": "GB/s", "frac": cand[dom]["gbs"] / peak, "peak_source": peak_src,
                "traffic": committed_traffic(kernel_names[dom], "fcg32"),
                "algorithmic_bytes_per_launch": cand[dom]["algorithmic_bytes"],
                "avg_launch_ms": cand[dom]["avg_ms"],
                "timing": "CUDA events around each launch in a profiled pass of the same steps"}

    # the same kernel against the float64 pipe: one FMA per stored entry plus
    # the p.q dot, at 2 FP64 FMA per clock per SM (1.25 TFLOP/s nominal at the
    # 2070 MHz clock GB300 reports)
    sp_entries = amg.level_layout(0)["stored"] + n0
    fp64_peak = 152 * 2 * 2 * 2.070e9 / 1e9
    roofline_fp64 = None
    if "spmv" in per_kernel:
        gf = 2 * sp_entries / (per_kernel["spmv"]["avg_ms"] * 1e-3) / 1e9
        roofline_fp64 = {"kernel": "k_spmv", "bound": "alu", "achieved": gf, "peak": fp64_peak, "unit": "GFLOP/s",
                         "frac": gf / fp64_peak, "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2070 MHz",
                         "flops_per_launch": 2 * sp_entries}
    # the dominant kernel's binding limit: k_spmv does one float64 FMA per stored
    # entry and is held by GB300's float64 pipe (ncu: 91% active at 0.51 of peak
    # DRAM throughput), so its roofline is the float64 one, its HBM view beside it
    roofline = roofline_hbm
    if kernel_names[dom] == "k_spmv" and roofline_fp64:
        roofline = dict(roofline_fp64, traffic=roofline_hbm["traffic"], avg_launch_ms=roofline_hbm["avg_launch_ms"],
                        algorithmic_bytes_per_launch=roofline_hbm["algorithmic_bytes_per_launch"],
                        timing=roofline_hbm["timing"],
                        hbm={"achieved": roofline_hbm["achieved"], "peak": peak, "unit": "GB/s",
                             "frac": roofline_hbm["frac"]})

    if rank == 0:
        h2d = 16 * n0
        d2h = 8 * n0 + 8 * (int(statistics.median(e2e_iters)) + 1)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
            "config": headline_config(args, n0, nnz0),
            "serving_summary": serving_summary(serving),
            "hierarchy": {"levels": len(levels), "rows_nnz": levels, "coarse": amg.coarse_info(),
                          "layout": [amg.level_layout(l) for l in range(len(levels))],
                          "level0_patterns": pat0},
            "iters": {"median": statistics.median(m["iters"]), "min": min(m["iters"]), "max": max(m["iters"])},
            "latency_ms": {"p50": pct(m["lat_ms"], 50), "p99": pct(m["lat_ms"], 99)},
            "true_rel": m["true_rel"],
            "multi_rhs": multi,
            "batch": batch,
            "serving": serving,
            "refresh": refresh,
            "smoother": smoother,
            "smoothed": smoothed,
            "fp64": {"value": solves / (f64_ms / 1e3), "unit": UNIT, "ms_per_step": f64_ms / args.steps,
                     "latency_ms": {"p50": pct(f64["lat_ms"], 50), "p99": pct(f64["lat_ms"], 99)},
                     "iters": statistics.median(f64["iters"]), "gpu_launches": f64["launches"]},
            "setup_ms": setup,
            "autotune": tune,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "roofline": roofline,
            "roofline_hbm": roofline_hbm,
            "roofline_fp64_pipe": roofline_fp64,
            "kernels": per_kernel,
            "kernels_fp64": per_kernel64,
            "levels": levels32,
            "levels_fp64": levels64,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "gpu_launches": m["launches"],
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    amg.close()
    return 0


def run_large(args):
    """One 320^3 mesh (32.8M dofs) with z graded at ratio 1.02 and a 4:1
    x-stretch, 8 right-hand sides in one multi-column solve and one at a
    time, both modes, with per-level V-cycle rates from a profiled pass. Its
    coarsening stalls above the dense limit, so the hierarchy uses the
    iterative coarsest solve."""
    import torch
    from paper_2210_16660_gb300 import binding as B
    from paper_2210_16660_gb300 import workloads as W
    torch.cuda.set_device(0)
    device = torch.device("cuda", 0)
    N, k = 320, 8
    r, lx = 1.02, 4.0
    t0 = time.perf_counter()
    prob = W.make_problem(N, r, seed=6, lx=lx)
    Bm, _ = W.make_rhs(prob, k, seed=1006)
    gen_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    amg = B.AMG.from_csr(prob.A, mode="fcg32", stream=stream)
    setup = amg.setup_times()
    if not args.no_autotune:
        amg.autotune(reps=10, stream=stream)
    info = amg.info()
    Bd = torch.from_numpy(Bm).to(device)
    Xd = torch.zeros_like(Bd)
    peak = measured_peaks().get("hbm_gbs") or 6800.0
    out = {}
    sampler = ClockSampler(0)
    sampler.start()
    for mode in ("fcg32", "pcg64"):
        amg.set_mode(mode)
        Xd.zero_()
        amg.solve_multi(Bd, Xd, rtol=args.rtol, maxit=args.maxit, stream=stream, hist=False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        Xd.zero_()
        e0.record(stream)
        st, it, _, sts, tr = amg.solve_multi(Bd, Xd, rtol=args.rtol, maxit=args.maxit, stream=stream, hist=False)
        e1.record(stream)
        torch.cuda.synchronize()
        if st != 0:
            raise RuntimeError(f"multi solve failed: {sts}")
        ms_multi = e0.elapsed_time(e1)
        cols = [Bd[:, c].contiguous() for c in range(k)]
        x = torch.zeros(prob.A.n, dtype=torch.float64, device=device)
        single = timed_solves(amg, cols, x, k, 1, args.rtol, args.maxit, torch, stream, None, device)
        prof = timed_solves(amg, cols, x, 2, 1, args.rtol, args.maxit, torch, stream, None, device, profile=True)
        out[mode] = {"multi": {"k": k, "ms": ms_multi, "solves_per_s": k / (ms_multi / 1e3),
                               "max_iters": int(it.max()), "max_true_rel": float(np.max(tr))},
                     "single": {"solves_per_s": k / (single["total_ms"] / 1e3),
                                "iters": statistics.median(single["iters"]), "true_rel": single["true_rel"]},
                     "levels": level_table(amg, prof["levels"], mode, peak)}
    clocks = sampler.stop()
    line = {"metric": "solves/s at rel.res 1e-8 (8 right-hand sides), mixed vs FP64; HBM GB/s per V-cycle level",
            "config": {"workload": f"q1_hex_{N}^3_zgrade{r}_xstretch{lx:g}", "n": prob.A.n, "nnz": prob.A.nnz,
                       "rhs": k, "coarse": amg.coarse_info(),
                       "levels": len(info), "generation_s": gen_s},
            "setup_ms": setup, "mixed": out["fcg32"], "fp64": out["pcg64"], "clocks": clocks,
            "peak_hbm_gbs": peak}
    print(json.dumps(line), flush=True)
    amg.close()
    return 0


def run_serve_sweep(args):
    """Serving over the resident 64^3 / 128^3 / 192^3 meshes (r = 1.04, warm
    starts): saturated rates, an arrival-rate sweep with p50/p99 latency per
    rate for the mixed batching server and the plain float64 server, and an
    admission run under an 8 GB device budget."""
    import torch
    from paper_2210_16660_gb300 import serving as SV
    torch.cuda.set_device(0)
    device = torch.device("cuda", 0)
    meshes = SV.prepare_meshes(tuple(args.serve_sizes), ratio=args.ratio, seed=5, pool=4, device=device)
    if not args.no_autotune:
        for mm in meshes:
            mm.amg.autotune(reps=10)
    kw = dict(slots=args.serve_slots, max_engines=args.serve_engines, chunk=args.serve_chunk, rtol=args.rtol,
              maxit=args.maxit, solo=not args.serve_no_solo, batch_min=args.serve_batch_min)
    sampler = ClockSampler(0)
    sampler.start()
    res = SV.serve_sweep(meshes, count=args.sweep_count, **kw)
    clocks = sampler.stop()
    line = {"metric": "serving: solves/s and p50/p99 latency (ms) per arrival rate, mixed batching server vs "
                      "plain FP64 pcg_solve, rel.res 1e-8",
            "config": {"meshes": [{"name": mm.name, "n": mm.problem.A.n, "coarse": mm.amg.coarse_info()["kind"]}
                                  for mm in meshes],
                       "arrivals": "Poisson, mesh uniform", "server": kw},
            "clocks": clocks, **res}
    print(json.dumps(line), flush=True)
    for mm in meshes:
        mm.amg.close()
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.serve_sweep:
        return run_serve_sweep(args)
    if args.large:
        return run_large(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
