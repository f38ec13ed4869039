"""Request streams for the serving runtime (``amg_server_*``).

Each mesh's hierarchy is built once and stays resident; a request is one
time step's pressure solve on a mesh, warm-started from the previous step's
solution (arxiv 2210.16660, Sec. 4 and Sec. 5). Requests arrive as a Poisson
stream, each for a mesh drawn uniformly; the server batches whatever is in
flight. Latency is measured from a request's scheduled arrival to the moment
its result is read back on the host.

Usage as a load generator::

    python -m paper_2210_16660_gb300.serving --sizes 64 128 192 --count 400
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import time

import numpy as np

from . import binding as B
from . import workloads as W


@dataclasses.dataclass
class Mesh:
    """One resident mesh: its problem, hierarchy and a pool of time steps
    ``(b_t, x0_t)`` on the device (requests cycle through the pool)."""
    name: str
    problem: W.Problem
    amg: B.AMG
    steps: list


def prepare_meshes(sizes=(64, 128, 192), ratio: float = 1.04, seed: int = 5, pool: int = 4,
                   device: str = "cuda", lx: float = 1.0, coarse: str = "auto", coarse_max: int = 200) -> list[Mesh]:
    """Meshes N^3 with z graded by ``ratio`` (x stretched to ``lx``), each
    with its hierarchy (coarsest solver ``coarse``: a mesh whose coarsening
    stalls above 4096 rows gets the iterative coarsest solve under "auto")
    and a chain of ``pool`` time steps."""
    import torch
    meshes = []
    for idx, N in enumerate(sizes):
        prob = W.make_problem(N, ratio, seed=seed + idx, lx=lx, name=f"q1_{N}cube_r{ratio}")
        _, xs0 = W.make_rhs(prob, 1, seed + 100 + idx)
        chain = W.time_steps(prob, np.ascontiguousarray(xs0[:, 0]), pool, seed + 200 + idx)
        amg = B.AMG.from_csr(prob.A, mode="fcg32", coarse=coarse, coarse_max=coarse_max)
        steps = [(torch.from_numpy(b).to(device), torch.from_numpy(np.ascontiguousarray(x0)).to(device))
                 for b, x0, _ in chain]
        meshes.append(Mesh(prob.name, prob, amg, steps))
    return meshes


def make_server(meshes: list[Mesh], mode: str, slots: int = 4, max_engines: int = 2, chunk: int = 4,
                hbm_budget: int = 0, queue_cap: int = 1 << 20, rtol: float = 1e-8, maxit: int = 1000,
                solo: bool = True, batch_min: int = 3, lane_priority: bool = False) -> B.Server:
    loads = [float(m.problem.A.n) for m in meshes]
    return B.Server([m.amg for m in meshes], mode=mode, slots=slots, max_engines=max_engines, chunk=chunk,
                    queue_cap=queue_cap, rtol=rtol, maxit=maxit, hbm_budget=hbm_budget, loads=loads, solo=solo,
                    batch_min=batch_min, lane_priority=lane_priority)


def run_stream(server: B.Server, meshes: list[Mesh], rate: float, count: int, seed: int = 5) -> dict:
    """Serve ``count`` requests arriving at ``rate`` per second (inf: all at
    once). Returns throughput, latency percentiles and per-request outcomes."""
    import torch
    arrivals = W.poisson_arrivals(rate, count, seed)
    which = W.uniform_choices(count, len(meshes), seed)
    used = [0] * len(meshes)
    outstanding: dict[int, tuple[int, float]] = {}
    lat, iters, rels, statuses, queue_ms, lanes = [], [], [], [], [], []
    rejected = 0
    nxt = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    t_first_done = None
    t_last = t0
    while nxt < count or outstanding:
        now = time.perf_counter() - t0
        while nxt < count and arrivals[nxt] <= now:
            m = int(which[nxt])
            b, x0 = meshes[m].steps[used[m] % len(meshes[m].steps)]
            used[m] += 1
            x = torch.empty_like(b)
            st, t = server.submit(m, b, x0, x)
            if st == B.OK:
                outstanding[t] = (nxt, float(arrivals[nxt]))
            else:
                rejected += 1
            nxt += 1
        if server.progress(wait=False) == 0:
            continue
        tnow = time.perf_counter()
        for t in list(outstanding):
            r = server.result(t)
            if r is None:
                continue
            _, arr = outstanding.pop(t)
            lat.append(1e3 * (tnow - t0 - arr))
            iters.append(r.iters)
            rels.append(r.true_rel)
            statuses.append(r.status)
            queue_ms.append(r.queue_ms)
            lanes.append(r.lane)
            t_last = tnow
            if t_first_done is None:
                t_first_done = tnow
    span = t_last - t0
    done = len(lat)
    lat_a = np.asarray(lat) if lat else np.zeros(1)
    return {
        "rate": None if not np.isfinite(rate) else rate,
        "requests": count,
        "completed": done,
        "rejected": rejected,
        "span_s": span,
        "solves_per_s": done / span if span > 0 else 0.0,
        "p50_ms": float(np.percentile(lat_a, 50)),
        "p99_ms": float(np.percentile(lat_a, 99)),
        "mean_queue_ms": float(np.mean(queue_ms)) if queue_ms else 0.0,
        "in_lane": int(len(lanes) - sum(lanes)),
        "mean_iters": float(np.mean(iters)) if iters else 0.0,
        "max_true_rel": float(np.max(rels)) if rels else 0.0,
        "all_ok": bool(statuses) and all(s == B.OK for s in statuses),
    }


def run_sequential(meshes: list[Mesh], mode: str, rate: float, count: int, seed: int = 5,
                   rtol: float = 1e-8, maxit: int = 1000) -> dict:
    """The same request stream served one request at a time by pcg_solve
    (first come, first served, no batching): the plain solver as a server."""
    import torch
    arrivals = W.poisson_arrivals(rate, count, seed)
    which = W.uniform_choices(count, len(meshes), seed)
    used = [0] * len(meshes)
    for m in meshes:
        m.amg.set_mode(mode)
    lat, iters, rels = [], [], []
    ok = True
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    try:
        for k in range(count):
            while time.perf_counter() - t0 < arrivals[k]:
                pass
            m = int(which[k])
            b, x0 = meshes[m].steps[used[m] % len(meshes[m].steps)]
            used[m] += 1
            x = x0.clone()
            r = meshes[m].amg.solve(b, x, rtol=rtol, maxit=maxit, hist=False)
            lat.append(1e3 * (time.perf_counter() - t0 - arrivals[k]))
            iters.append(r.iters)
            rels.append(r.true_rel)
            ok = ok and r.status == B.OK
    finally:
        for m in meshes:
            m.amg.set_mode("fcg32")
    span = time.perf_counter() - t0
    lat_a = np.asarray(lat)
    return {"rate": None if not np.isfinite(rate) else rate, "requests": count, "completed": count,
            "span_s": span, "solves_per_s": count / span, "p50_ms": float(np.percentile(lat_a, 50)),
            "p99_ms": float(np.percentile(lat_a, 99)), "mean_iters": float(np.mean(iters)),
            "max_true_rel": float(np.max(rels)), "all_ok": ok}


def serve_modes(meshes: list[Mesh], count: int, load_fraction: float = 0.7, seed: int = 5, **server_kw) -> dict:
    """Three servers on the same request streams:

    * ``fp64_plain``: one request at a time through pcg_solve in float64 PCG;
    * ``fp64``: the batching server in float64 PCG;
    * ``mixed``: the batching server with the float32 V-cycle in FCG(1).

    Each is run saturated (every request queued at t = 0: throughput), at a
    common arrival rate of ``load_fraction`` times the plain server's
    saturated throughput (latency, all three stable), and the batching
    servers also at ``load_fraction`` of their own saturated throughput."""
    rtol = server_kw.get("rtol", 1e-8)
    maxit = server_kw.get("maxit", 1000)
    run_sequential(meshes, "pcg64", float("inf"), max(8, count // 8), seed + 1, rtol, maxit)   # warm-up
    plain_sat = run_sequential(meshes, "pcg64", float("inf"), count, seed, rtol, maxit)
    common = load_fraction * plain_sat["solves_per_s"]
    out = {"common_rate": common,
           "fp64_plain": {"saturated": plain_sat,
                          "at_common_rate": run_sequential(meshes, "pcg64", common, count, seed + 2, rtol, maxit)}}
    for name, mode in (("mixed", "fcg32"), ("fp64", "pcg64")):
        srv = make_server(meshes, mode, **server_kw)
        try:
            run_stream(srv, meshes, float("inf"), max(8, count // 8), seed + 1)       # warm-up
            sat = run_stream(srv, meshes, float("inf"), count, seed)
            at_common = run_stream(srv, meshes, common, count, seed + 2)
            at_own = run_stream(srv, meshes, load_fraction * sat["solves_per_s"], count, seed + 3)
        finally:
            srv.close()
        out[name] = {"saturated": sat, "at_common_rate": at_common, "at_own_load": at_own}
    return out


def serve_sweep(meshes: list[Mesh], count: int = 2000, start_fraction: float = 0.35, factor: float = 1.5,
                seed: int = 7, budget_bytes: int = 8 << 30, **server_kw) -> dict:
    """Arrival-rate sweep of the mixed batching server and the plain float64
    server (pcg_solve, one request at a time) on the same streams.

    Each server's saturated rate is measured first (``count // 4`` requests
    queued at once). Rates then grow geometrically by ``factor`` from
    ``start_fraction`` times the plain server's saturated rate; a server is
    run at every rate below its own saturated rate (above it its queue only
    grows), ``count`` requests per rate. Then one run of the mixed server with
    an ``budget_bytes`` device budget for hierarchies and engines: meshes that
    do not fit are not admitted and their requests are refused."""
    rtol = server_kw.get("rtol", 1e-8)
    maxit = server_kw.get("maxit", 1000)
    run_sequential(meshes, "pcg64", float("inf"), 16, seed + 1, rtol, maxit)    # warm-up
    plain_sat = run_sequential(meshes, "pcg64", float("inf"), max(64, count // 4), seed, rtol, maxit)
    srv = make_server(meshes, "fcg32", **server_kw)
    try:
        run_stream(srv, meshes, float("inf"), 16, seed + 1)                       # warm-up
        mixed_sat = run_stream(srv, meshes, float("inf"), max(64, count // 4), seed)
        rates = []
        r = start_fraction * plain_sat["solves_per_s"]
        while r < mixed_sat["solves_per_s"]:
            rates.append(r)
            r *= factor
        mixed_rows = [run_stream(srv, meshes, rate, count, seed + 10 + k) for k, rate in enumerate(rates)]
    finally:
        srv.close()
    plain_rows = [run_sequential(meshes, "pcg64", rate, count, seed + 10 + k, rtol, maxit)
                  for k, rate in enumerate(rates) if rate < plain_sat["solves_per_s"]]
    kw = dict(server_kw)
    kw["hbm_budget"] = budget_bytes
    small = make_server(meshes, "fcg32", **kw)
    try:
        admitted = [small.mesh_info(i)[0] > 0 for i in range(len(meshes))]
        budget_run = run_stream(small, meshes, 0.7 * mixed_sat["solves_per_s"], max(64, count // 4), seed + 99)
        used = small.info()
    finally:
        small.close()
    return {"requests_per_rate": count, "rates": rates,
            "mixed": {"saturated": mixed_sat, "sweep": mixed_rows},
            "fp64_plain": {"saturated": plain_sat, "sweep": plain_rows},
            "budget": {"bytes": budget_bytes, "admitted": admitted, "run": budget_run, "info": used}}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--sizes", type=int, nargs="+", default=[64, 128, 192])
    ap.add_argument("--count", type=int, default=400)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--engines", type=int, default=2)
    ap.add_argument("--chunk", type=int, default=4)
    ap.add_argument("--budget-gb", type=float, default=0.0)
    ap.add_argument("--no-solo", action="store_true", help="engines only, no whole-solve lanes")
    ap.add_argument("--batch-min", type=int, default=3)
    ap.add_argument("--rates", type=float, nargs="*", default=[],
                    help="arrival rates to sweep (per s); default: saturation and 70%% of it")
    a = ap.parse_args(argv)
    meshes = prepare_meshes(tuple(a.sizes))
    kw = dict(slots=a.slots, max_engines=a.engines, chunk=a.chunk, hbm_budget=int(a.budget_gb * 2 ** 30),
              solo=not a.no_solo, batch_min=a.batch_min)
    if not a.rates:
        print(json.dumps(serve_modes(meshes, a.count, **kw)))
        return
    for mode in ("fcg32", "pcg64"):
        for rate in a.rates:
            print(json.dumps({"mode": mode, "server": "plain", **run_sequential(meshes, mode, rate, a.count)}))
        srv = make_server(meshes, mode, **kw)
        try:
            for rate in a.rates:
                r = run_stream(srv, meshes, rate, a.count)
                print(json.dumps({"mode": mode, **r}))
        finally:
            srv.close()


if __name__ == "__main__":
    main()
