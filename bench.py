"""LAMG benchmark: one step = lamg_setup + lamg_solve to relative residual 1e-8
on a device-resident synthetic graph (default: the 256^3 7-point grid with
weights 1/1/0.01, n = 16.8M, FP32 cycles inside FP64 iterative refinement),
timed with CUDA events.  Prints one JSON line; the Chung-Lu n = 1M workload is
measured too and reported under "secondary".

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--workload grid256|chung_lu1m|grid64|grid1024|...] [--precision fp32ir|fp64] [--elim]

Multi-GPU: the solve of one graph does not shard (each relaxation sweep would
need a halo exchange); N GPUs run N independent replicas of the step.  The
batched workloads are many independent problems and shard: the right-hand
sides (rgg2m_b64) or the graphs (er500, balanced by size) are split over the
ranks.  Either way there is no collective on the data path, and value = all
ranks' units / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOADS = {
    # name: (graph, precision default, description)
    "chung_lu1m": ("chung_lu1m", "fp32ir",
                   "Chung-Lu n=1M beta=2.5 mean degree 10 (LCC), w~U[0.5,2] FP32; FP32 cycles in FP64 IR to 1e-8"),
    "grid256": ("grid256", "fp32ir",
                "256^3 7-point grid, weights 1/1/0.01; FP32 cycles in FP64 IR to 1e-8"),
    "grid128": ("grid128", "fp32ir",
                "128^3 7-point grid, weights 1/1/0.01 (the profiling case of the 256^3 family); FP32 cycles in "
                "FP64 IR to 1e-8"),
    "grid64": ("grid64", "fp64", "64x64 5-point grid, unit weights; FP64 to 1e-10"),
    "grid1024": ("grid1024", "fp32ir", "1024x1024 5-point grid, unit weights; FP32 cycles in FP64 IR to 1e-8"),
    "grid1024_13pt": ("grid1024_13pt", "fp32ir",
                      "1024x1024 13-point 4th-order grid (negative weights, Sec. 5 grid table (b)); FP32 cycles "
                      "in FP64 IR to 1e-8"),
    "grid1024_rot_c": ("grid1024_rot_c", "fp32ir",
                       "1024x1024 anisotropic-rotated grid, agnostic cross term (negative weights, Sec. 5 grid "
                       "table (c)); FP32 cycles in FP64 IR to 1e-8"),
    "torus1024_lgmg": ("torus1024", "fp32ir",
                       "1024x1024 periodic 5-point grid, unit weights; Lean Geometric MG (Sec. 6): 2x2 aggregates, "
                       "red-black GS, gamma 1.5 at every level, flat mu 2; FP32 cycles in FP64 IR to 1e-8"),
}
TOL = {"chung_lu1m": 1e-8, "grid256": 1e-8, "grid128": 1e-8, "grid1024_13pt": 1e-8, "grid1024_rot_c": 1e-8, "grid64": 1e-10, "grid1024": 1e-8, "torus1024_lgmg": 1e-8}
# The DRAM bytes (read + write) of one engine launch come from the committed
# ncu summary of the workload, profiles/k_engine_<workload>_<precision>.md,
# which records them with a hash of the engine's sources at capture time; when
# the sources have changed since, the figure is stale and reported as null.
ENGINE_SOURCES = ("cycle.cu", "engine.cuh", "solve_rows.cuh", "solve.cu")


def engine_sources_sha():
    h = hashlib.sha256()
    for f in ENGINE_SOURCES:
        with open(os.path.join(ROOT, "paper_1108_1310_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload, prec_name):
    """(bytes per engine launch, source) from the committed capture, or (None, why)."""
    p = os.path.join(ROOT, "profiles", f"k_engine_{workload}_{prec_name}.md")
    if not os.path.exists(p):
        return None, "no ncu capture of this workload"
    with open(p) as f:
        txt = f.read()
    m_sha = re.search(r"engine_sources_sha256_16:\s*`?([0-9a-f]{16})", txt)
    m_tr = re.search(r"traffic_bytes_per_launch:\s*`?([0-9.eE+]+)", txt)
    if not (m_sha and m_tr):
        return None, "capture without a traffic line"
    if m_sha.group(1) != engine_sources_sha():
        return None, "engine sources changed since the capture"
    return float(m_tr.group(1)), f"profiles/{os.path.basename(p)}"


def host_cpu():
    """Model name and logical core count of this host (the CPU baseline's machine)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"model": model, "nproc": os.cpu_count()}
# batched forms (many right-hand sides on one hierarchy; many graphs as one union)
ADJOINT = {
    "knn500k_adjoint": "kNN graph n=500k, k=10, 16-D Gaussian-mixture points, Gaussian weights FP32, all components "
                       "as one union; semi-supervised solve (1% labelled sources, zero-sum per component) to 1e-8 "
                       "plus the adjoint: lambda and dL/dw for every edge",
}
BATCHED = {
    "rgg2m_b64": "64 zero-sum Gaussian RHS on a 2M-node 2-D RGG (mean degree 12, w = exp(-d^2/r^2), FP32); "
                 "FP32 cycles in FP64 IR to 1e-8, lamg_solve_batched",
    "er500": "500 Erdos-Renyi graphs (LCC), n uniform in [1k, 200k], mean degree 8, unit weights, one zero-sum "
             "RHS each, as one block-diagonal union (lamg_setup_graphs); FP32 cycles in FP64 IR to 1e-8 per graph",
}
CPU_SAMPLE = {"chung_lu1m": ("chung_lu", 1_000_000), "grid256": ("grid3d", 96), "grid128": ("grid3d", 64),
              "grid1024_13pt": ("stencil:13pt", 256), "grid1024_rot_c": ("stencil:rot_c", 128), "grid64": ("grid2d", 64),
              "grid1024": ("grid2d", 256),
              "torus1024_lgmg": ("torus", 1024)}


# Per-workload settings of the method's options (each also a command-line flag,
# which overrides it; the library's defaults are the paper's printed values):
# - gamma_coarse_max 1 on the 3-D grids and the power-law graph: the same cycle
#   counts as the printed 2 at a tenth of the colour phases on the 3-D grids;
# - gamma 1.2 (fine-level cap; printed 1.5) on the 3-D grids: each coarse level
#   is visited 5 times per cycle instead of 8, for 27/27, 29/29 and 28/30 cycles
#   (printed cap / 1.2) on the oracle's 96^3, 64^3 and 128^3 grids; on the GPU
#   at 256^3, 32 cycles in 621 ms against 30 in 752 ms;
# - elimination (Sec. 3.2) on the power-law graph, where its degree-1..4 nodes
#   are many (on 3-D grids no node qualifies);
# - on the 1024^2 grids the printed cap 2 with mu_adaptive 1.2: with mu 1 the
#   adaptive cycle stalls there (5-point: with cap 1 too; 13-point: 0.997 per
#   cycle, against 16 cycles at 0.31 with mu 1.2, the oracle on the same grid);
# - the other workloads run the library's defaults (cap 1 slows RGGs, 11 -> 18
#   cycles on a 200k-node one, and can stall them).
WORKLOAD_OPTS = {
    "grid256": {"gamma": 1.2, "gamma_coarse_max": 1.0, "colour_rule": 1, "sb_work32": 65536},
    "grid128": {"gamma": 1.2, "gamma_coarse_max": 1.0, "colour_rule": 1, "sb_work32": 65536},
    "chung_lu1m": {"gamma_coarse_max": 1.0, "elim": 1},
    "grid1024": {"gamma_coarse_max": 2.0, "mu_adaptive": 1.2},
    "grid1024_13pt": {"negative_weights": 1, "mu_adaptive": 1.2},
    "grid1024_rot_c": {"negative_weights": 1, "recomb_finest": 0},
}


def method_opts(workload, n):
    """Options of the method for a workload of n nodes, the same for the library and
    the oracle, and whether the solve is adaptive.  The geometric workloads run Lean
    Geometric MG (Sec. 6) in flat mode with mu = 2 on the grid of side sqrt(n)."""
    if workload.endswith("_lgmg"):
        return {"lgmg_nx": int(round(n ** 0.5)), "mu_flat": 2.0}, False
    return dict(WORKLOAD_OPTS.get(workload, {})), True


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def sample_graph(workload):
    import workloads as W
    kind, size = CPU_SAMPLE[workload]
    if kind == "chung_lu":
        return W.chung_lu(size, 2.5, 10.0, seed=2), f"Chung-Lu n={size} (same family and seed rule)"
    if kind == "grid3d":
        return W.grid3d(size, size, size, 1.0, 1.0, 0.01), f"{size}^3 7-point grid, weights 1/1/0.01"
    if kind == "torus":
        return W.grid2d_periodic(size), f"{size}x{size} periodic 5-point grid, Lean Geometric MG"
    if kind.startswith("stencil:"):
        st = kind.split(":")[1]
        return W.grid2d_stencil(size, st), f"{size}x{size} grid, stencil {st}"
    return W.grid2d(size, size), f"{size}x{size} 5-point grid"


def method_options(args, workload, n):
    """The method's options of this run, shared by the library and the oracle, and
    whether the solve is adaptive: the workload's settings, then any flag given."""
    opts, adaptive = method_opts(workload, n)
    for k in ("gamma", "gamma_coarse_max", "elim", "agg_rule", "recomb_finest", "n_coarsest", "mu_adaptive",
              "colour_rule"):
        v = getattr(args, k)
        if v is not None:
            opts[k] = v
    return opts, adaptive


def cpu_oracle_step(g, b, tol, opts, adaptive):
    """The oracle as it stands: FP64 setup + solve on one host core."""
    import oracle
    # the method's options (performance knobs of the GPU engine are not the oracle's)
    mopts = {k: v for k, v in opts.items() if k in dict(oracle.Opts._fields_)}
    t0 = time.perf_counter()
    h = oracle.Hierarchy(g.n, g.rp, g.col, g.w, **mopts)
    x, hist = h.solve(b, tol=tol, max_cycles=500, adaptive=adaptive)
    t = time.perf_counter() - t0
    return t, len(hist) - 1


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p is not None:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            parts = [t.strip() for t in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def run_reference(args):
    """--impl reference: the CPU oracle, timed on this host, on a bounded sample."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import workloads as W
    g, desc = sample_graph(args.workload)
    b = W.zero_sum_rhs(g.n, 2)
    tol = TOL[args.workload]
    opts, adaptive = method_options(args, args.workload, g.n)
    for _ in range(min(args.warmup, 1)):
        cpu_oracle_step(g, b, tol, opts, adaptive)
    ts, cyc = [], []
    for _ in range(args.steps):
        t, c = cpu_oracle_step(g, b, tol, opts, adaptive)
        ts.append(t)
        cyc.append(c)
    tmean = sum(ts) / len(ts)
    value = g.m * (sum(cyc) / len(cyc)) / tmean
    line = {
        "impl": "reference", "metric": "edges*cycles/s (LAMG setup + solve to tol)", "value": value,
        "unit": "edges*cycles/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": min(args.warmup, 1),
        "ms_per_step": tmean * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "sample": desc, "n": g.n, "m": g.m, "tol": tol, **opts},
        "cpu_baseline": {"value": value, "unit": "edges*cycles/s", "cores": 1, "kind": "oracle",
                         "sample": desc, "host": host_cpu()},
        "e2e": {"value": value, "unit": "edges*cycles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def slowest_rank_ms(ms, dist, device):
    """Max over ranks of a per-rank step time (replicas: the job ends with its slowest rank)."""
    if not dist:
        return ms
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, units_per_rank_step, ms):
    """Whole-job throughput: every rank processes the same units per step (weak scaling)."""
    return world * units_per_rank_step / (ms / 1e3)


def total_units(units, dist, device):
    """Sum over ranks of the units each rank processed (a sharded job: one host-side
    reduction of the counts after the timed region, nothing on the data path)."""
    if not dist:
        return units
    import torch
    t = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def shard_block(count, world, rank):
    """Contiguous share [c0, c1) of `count` independent items (right-hand sides) for
    one rank; the shares differ in size by at most one."""
    base, extra = divmod(count, world)
    c0 = rank * base + min(rank, extra)
    return c0, c0 + base + (1 if rank < extra else 0)


def shard_lpt(loads, world):
    """Independent problems of the given loads (graph sizes) dealt to `world` ranks,
    largest first, each to the least-loaded rank so far (ties: lower rank; equal
    loads: lower index).  Returns each rank's problem indices in increasing order."""
    order = sorted(range(len(loads)), key=lambda k: (-loads[k], k))
    total = [0] * world
    share = [[] for _ in range(world)]
    for k in order:
        r = min(range(world), key=lambda q: (total[q], q))
        share[r].append(k)
        total[r] += loads[k]
    return [sorted(s) for s in share]


def run_adjoint(args, L, W, torch, dev, stream, rank, world, dist=None):
    """One step = setup + forward solve + adjoint (lambda and the gradient for every edge), FP32 in FP64 IR."""
    tol = 1e-8
    # all 500k points: the kNN graph of a 10-cluster mixture falls into components,
    # solved together as one block-diagonal union (lamg_setup_graphs)
    g, gptr, _, _ = W.knn_gmm(500_000, dim=16, k=10, seed=6, device=str(dev), components=True)
    rng = np.random.default_rng(6)
    perm = rng.permutation(g.n)
    lab, held = perm[: g.n // 100], perm[g.n // 100: g.n // 100 + g.n // 20]
    y = rng.integers(0, 2, g.n).astype(np.float64)
    b_host = np.zeros(g.n)
    labelled = np.zeros(g.n, dtype=bool)
    labelled[lab] = True
    for c in range(len(gptr) - 1):   # zero-sum sources on every component
        idx = np.arange(gptr[c], gptr[c + 1])[labelled[gptr[c]:gptr[c + 1]]]
        if idx.size >= 2:
            b_host[idx] = y[idx] - y[idx].mean()
    gx_host = np.zeros(g.n)
    gx_host[held] = 1.0
    eu, ev, _ = g.edges()
    rp = torch.tensor(g.rp, device=dev)
    col = torch.tensor(g.col, device=dev)
    w = torch.tensor(g.w, device=dev).to(torch.float32)
    b = torch.tensor(b_host, device=dev)
    gx = torch.tensor(gx_host, device=dev)
    eut = torch.tensor(eu, device=dev)
    evt = torch.tensor(ev, device=dev)
    x = torch.zeros_like(b)
    lam = torch.zeros_like(b)
    dw = torch.zeros(eu.size, dtype=torch.float64, device=dev)
    mopts, _ = method_options(args, args.workload, g.n)
    opt = L.lamg_default_options(validate=1, max_cycles=2000, **mopts)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    prof = {"ms": 0.0, "n": 0, "bytes": 0}

    def step(prec=L.LAMG_FP32_IR, profile=False):
        h = L.lamg_setup_graphs(gptr, rp, col, w, opt, stream)
        if profile:
            L.lamg_profile(h, True)
        x.zero_()
        st = L.lamg_solve(h, b, x, tol, prec, stream)
        sa = L.lamg_adjoint(h, x, gx, lam, eut, evt, dw, tol=tol, precision=prec, stream=stream)
        if profile:
            ms, n, byt = L.lamg_profile(h, False)
            prof["ms"] += ms * n
            prof["n"] += n
            prof["bytes"] = byt
        L.lamg_free(h)
        return st, sa

    for _ in range(args.warmup):
        step()
        flush.fill_(1.0)
    torch.cuda.synchronize()
    times, res = [], []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = L.lamg_launch_count()
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        for _ in range(args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res.append(step(profile=True))
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            flush.fill_(1.0)
    launches = L.lamg_launch_count() - launches0
    if dist:
        dist.barrier()
    ms = slowest_rank_ms(sum(times) / len(times), dist, dev)
    cyc = sum(r[0].cycles + r[1].cycles for r in res) / len(res)
    roof = roofline_line(prof, "knn500k_adjoint", "fp32ir",
                         "cycle engine k_engine (forward and adjoint refinement steps: ir_inner FP32 cycles + FP64 "
                         "update, projection and residual)")
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_adjoint(W, mopts, tol)
    # forward and adjoint solves timed alone on one hierarchy, FP32 IR and plain FP64
    h = L.lamg_setup_graphs(gptr, rp, col, w, opt, stream)
    cmp = {}
    for name, prec in (("fp32ir", L.LAMG_FP32_IR), ("fp64", L.LAMG_FP64)):
        for what in ("forward", "adjoint"):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            x.zero_()
            if what == "adjoint":
                L.lamg_solve(h, b, x, tol, prec, stream)
            e0.record(stream)
            if what == "forward":
                st = L.lamg_solve(h, b, x, tol, prec, stream)
            else:
                st = L.lamg_adjoint(h, x, gx, lam, eut, evt, dw, tol=tol, precision=prec, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            cmp[f"{what}_ms_{name}"] = e0.elapsed_time(e1)
            cmp[f"{what}_cycles_{name}"] = st.cycles
            cmp[f"{what}_rel_res_{name}"] = st.rel_res
    L.lamg_free(h)
    line = {
        "metric": "edges*cycles/s (LAMG setup + solve to tol)",
        "value": job_value(world, g.m * cyc, ms), "unit": "edges*cycles/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": args.workload, "desc": ADJOINT[args.workload], "n": g.n, "m": g.m, "tol": tol,
                   "graphs": len(gptr) - 1, **mopts,
                   "levels": res[-1][0].levels, "cycles_forward_plus_adjoint": cyc,
                   "l2": "flushed between steps (512 MB write)", "parallelism": f"replicas{world}"},
        "fp64_vs_ir": cmp, "e2e": None, "roofline": roof, "cpu_baseline": cpu,
        "clocks": clk.summary(), "gpu_launches": launches,
    }
    if rank == 0:
        print(json.dumps(line))


def roofline_line(prof, workload, prec_name, kernel):
    """The roofline object of an engine: model bytes per launch over its average
    CUDA-event time, against the HBM peak; traffic from the committed capture."""
    if not prof["n"]:
        return None
    peak, peak_kind = load_peaks()
    avg = prof["ms"] / prof["n"]
    achieved = prof["bytes"] / (avg / 1e3) / 1e9
    traffic, tsrc = profiled_traffic(workload, prec_name)
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "traffic_source": tsrc, "kernel": kernel, "bytes_per_launch": prof["bytes"],
            "avg_ms": avg, "launches": prof["n"], "peak_kind": f"{peak_kind} hbm_gbs (burst copy)"}


def cpu_baseline_adjoint(W, mopts, tol):
    """The oracle's forward solve and adjoint on a 150k-point sample of the kNN family."""
    import oracle
    g, gptr, _, _ = W.knn_gmm(150_000, dim=16, k=10, seed=6, components=True)
    rng = np.random.default_rng(6)
    b = np.zeros(g.n)
    lab = rng.permutation(g.n)[: g.n // 100]
    b[lab] = rng.normal(size=lab.size)
    for c in range(len(gptr) - 1):
        sl = slice(gptr[c], gptr[c + 1])
        b[sl] -= b[sl].mean()
    gx = rng.normal(size=g.n)
    eu, ev, _ = g.edges()
    om = {k: v for k, v in mopts.items() if k in dict(oracle.Opts._fields_)}
    t0 = time.perf_counter()
    h = oracle.Hierarchy(g.n, g.rp, g.col, g.w, gptr=gptr, **om)
    x, hist = h.solve(b, tol=tol, max_cycles=500)
    lam, dw = h.adjoint(x, gx, eu, ev, tol=tol, max_cycles=500)
    t = time.perf_counter() - t0
    cyc = len(hist) - 1
    return {"value": g.m * cyc * 2 / t, "unit": "edges*cycles/s", "cores": 1, "kind": "oracle",
            "sample": f"kNN n={g.n} (150k points of the same mixture), setup + forward solve + adjoint to {tol:g}, "
                      f"{t:.1f} s; forward cycles counted twice", "host": host_cpu()}


def cpu_baseline_batched(W, workload, mopts, tol):
    """The oracle on a sample of a batched workload: 2 columns on a 200k-node RGG, or a
    union of 8 Erdos-Renyi graphs of the same size distribution."""
    import oracle
    om = {k: v for k, v in mopts.items() if k in dict(oracle.Opts._fields_)}
    t0 = time.perf_counter()
    if workload == "rgg2m_b64":
        g = W.rgg2d(200_000, 12.0, seed=4)
        B = W.zero_sum_rhs(g.n, 3, count=2)
        h = oracle.Hierarchy(g.n, g.rp, g.col, g.w, **om)
        cyc = 0
        for c in range(B.shape[1]):
            _, hist = h.solve(np.ascontiguousarray(B[:, c]), tol=tol, max_cycles=500)
            cyc += len(hist) - 1
        desc = "200k-node RGG of the same family, 2 right-hand sides"
    else:
        g, gptr = W.er_batch(8, 1000, 200_000, seed=7)
        b = W.zero_sum_rhs_graphs(gptr, 3)
        h = oracle.Hierarchy(g.n, g.rp, g.col, g.w, gptr=gptr, **om)
        _, hist = h.solve(b, tol=tol, max_cycles=500)
        cyc = len(hist) - 1
        desc = "union of the first 8 Erdos-Renyi graphs of the same generator"
    t = time.perf_counter() - t0
    return {"value": g.m * cyc / t, "unit": "edges*cycles/s", "cores": 1, "kind": "oracle",
            "sample": f"{desc}, setup + solve to {tol:g}, {cyc} cycles in {t:.1f} s", "host": host_cpu()}


def run_batched(args, L, W, torch, dev, stream, rank, world, dist=None):
    """One step = setup + solve of every right-hand side / every graph to 1e-8.
    The job is fixed (64 right-hand sides, 500 graphs) and shards over the ranks
    with no collective on the data path: rank r takes a contiguous block of the
    columns (each rank builds the hierarchy of the one matrix), or its share of
    the graphs balanced by size; value = all ranks' units / the slowest rank."""
    tol = 1e-8
    if args.workload == "rgg2m_b64":
        g, gptr, R_all = W.config_graph("rgg2m"), None, 64
        c0, c1 = shard_block(R_all, world, rank)
        R, G_all, G = c1 - c0, 1, 1
        Bh = np.ascontiguousarray(W.zero_sum_rhs(g.n, 3, count=R_all)[:, c0:c1])
        B = torch.tensor(Bh[:, 0].copy() if R == 1 else Bh, device=dev)
    else:
        G_all = 500
        mine = shard_lpt(W.er_batch_sizes(G_all, 1000, 200_000, seed=7).tolist(), world)[rank]
        (g, gptr), R, R_all, G = W.er_batch(G_all, 1000, 200_000, seed=7, only=mine), 1, 1, len(mine)
        B = torch.tensor(W.zero_sum_rhs_graphs(gptr, 3), device=dev)
    rp = torch.tensor(g.rp, device=dev)
    col = torch.tensor(g.col, device=dev)
    w = torch.tensor(g.w, device=dev).to(torch.float32)
    X = torch.zeros_like(B)
    mopts, _ = method_options(args, args.workload, g.n)
    opt = L.lamg_default_options(validate=1, max_cycles=2000, **mopts)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    tuned = {}

    def setup():
        if gptr is None:
            h = L.lamg_setup(g.n, rp, col, w, opt, stream)
            if R > 1:
                # column chunk of the batched engine: tuned once on the first hierarchy
                if "cols" not in tuned:
                    tuned["cols"], tuned["ms"] = L.lamg_autotune_batched(h, R, L.LAMG_FP32_IR, stream)
                L.lamg_set_batch_cols(h, tuned["cols"])
            return h
        return L.lamg_setup_graphs(gptr, rp, col, w, opt, stream)

    def solve(h, prec):
        X.zero_()
        if R > 1:
            sts = L.lamg_solve_batched(h, B, X, tol, prec, stream)
            return sum(s.cycles for s in sts), max(s.rel_res for s in sts), sts[0].levels
        st = L.lamg_solve(h, B, X, tol, prec, stream)
        return st.cycles, st.rel_res, st.levels

    prof = {"ms": 0.0, "n": 0, "bytes": 0}

    def step(profile=False):
        h = setup()
        if profile:
            L.lamg_profile(h, True)
        r = solve(h, L.LAMG_FP32_IR)
        if profile:
            ms_, n_, byt = L.lamg_profile(h, False)
            prof["ms"] += ms_ * n_
            prof["n"] += n_
            prof["bytes"] = byt
        L.lamg_free(h)
        return r

    for _ in range(args.warmup):
        step()
        flush.fill_(1.0)
    torch.cuda.synchronize()
    times, res = [], []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = L.lamg_launch_count()
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        for _ in range(args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res.append(step(profile=True))
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            flush.fill_(1.0)
    launches = L.lamg_launch_count() - launches0
    if dist:
        dist.barrier()
    ms = slowest_rank_ms(sum(times) / len(times), dist, dev)
    cyc = sum(r[0] for r in res) / len(res)
    roof = roofline_line(prof, args.workload, "fp32ir",
                         "batched cycle engine k_engine4 (one launch = one refinement step of a column chunk)"
                         if R > 1 else "cycle engine k_engine on the union (one launch = one refinement step)")
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_batched(W, args.workload, mopts, tol)
    units = total_units(g.m * cyc, dist, dev)     # edges*cycles of all ranks' shares per step

    def timed(fn):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), r

    # the same solves in plain FP64, and (many RHS) one right-hand side alone, on one hierarchy
    h = setup()
    t32, r32 = timed(lambda: solve(h, L.LAMG_FP32_IR))
    t64, r64 = timed(lambda: solve(h, L.LAMG_FP64))
    cmp = {"solve_ms_fp32ir": t32, "cycles_fp32ir": r32[0], "rel_res_fp32ir": r32[1],
           "solve_ms_fp64": t64, "cycles_fp64": r64[0], "rel_res_fp64": r64[1]}
    if R > 1:
        b1 = B[:, 0].contiguous()
        x1 = torch.zeros_like(b1)
        t1, st1 = timed(lambda: L.lamg_solve(h, b1, x1, tol, L.LAMG_FP32_IR, stream))
        t1d, st1d = timed(lambda: L.lamg_solve(h, b1, x1.zero_(), tol, L.LAMG_FP64, stream))
        cmp.update({"single_rhs_ms_fp32ir": t1, "single_rhs_ms_fp64": t1d,
                    "batched_ms_per_rhs_fp32ir": t32 / R, "batched_ms_per_rhs_fp64": t64 / R})
    L.lamg_free(h)
    line = {
        "metric": "edges*cycles/s (LAMG setup + solve to tol)",
        "value": units / (ms / 1e3), "unit": "edges*cycles/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": args.workload, "desc": BATCHED[args.workload], "n": g.n, "m": g.m,
                   "rhs": R_all, "rhs_rank0": R, "graphs": G_all, "graphs_rank0": G, "tol": tol, **mopts,
                   "batch_cols": tuned.get("cols"), "autotune_ms_16_32_64_128": tuned.get("ms"),
                   "levels": res[-1][2], "cycles_all_columns": cyc, "max_rel_res": res[-1][1],
                   "l2": "flushed between steps (512 MB write)", "parallelism": f"shard{world}"},
        "fp64_vs_ir": cmp, "e2e": None, "roofline": roof, "cpu_baseline": cpu,
        "clocks": clk.summary(), "gpu_launches": launches,
    }
    if rank == 0:
        print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu")
    ap.add_argument("--workload", default="grid256", choices=list(WORKLOADS) + list(BATCHED) + list(ADJOINT))
    ap.add_argument("--precision", default=None, choices=["fp32ir", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the Chung-Lu n = 1M measurement that the default run adds")
    ap.add_argument("--op-times", default=None, metavar="PATH",
                    help="after the timed region, time one more solve with the engine's op timer "
                         "(lamg_op_times) and write its table to PATH")
    # the method's options: unset flags keep the workload's setting (WORKLOAD_OPTS),
    # else the library's default
    ap.add_argument("--elim", type=int, default=None, choices=[0, 1],
                    help="low-degree elimination levels (Sec. 3.2)")
    ap.add_argument("--gamma", type=float, default=None,
                    help="cap of the cycle index at the fine levels (Sec. 4.1 prints 1.5)")
    ap.add_argument("--gamma-coarse-max", type=float, default=None,
                    help="cap of the cycle index at the coarse levels (Eq. (4.1) prints 2)")
    ap.add_argument("--mu-adaptive", type=float, default=None,
                    help="restriction factor under recombination (reading R15: 1)")
    ap.add_argument("--agg-rule", type=int, default=None, choices=[0, 1, 2],
                    help="aggregation stages: 2 the paper's scan in hashed order (default), 1 in index order, "
                         "0 the parallel handshake")
    ap.add_argument("--recomb-finest", type=int, default=None, choices=[0, 1],
                    help="1: the adaptive cycle recombines at the finest level too (default)")
    ap.add_argument("--n-coarsest", type=int, default=None,
                    help="coarsening stops below this many nodes (Sec. 4.1: 150)")
    ap.add_argument("--colour-rule", type=int, default=None, choices=[0, 1],
                    help="JP priority: 0 degree then hash (default), 1 degree then index (red-black on grids)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    from paper_1108_1310_gb300 import build
    build.build()
    from paper_1108_1310_gb300 import lamg as L
    import workloads as W

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    if args.workload in BATCHED:
        return run_batched(args, L, W, torch, dev, stream, rank, world, dist)
    if args.workload in ADJOINT:
        return run_adjoint(args, L, W, torch, dev, stream, rank, world, dist)
    line = run_single(args, args.workload, L, W, torch, dev, stream, rank, world, local, dist, full=True)
    if rank == 0 and args.workload == "grid256" and not args.no_secondary:
        # the power-law workload of the same metric, measured the same way (fewer steps)
        sec = run_single(args, "chung_lu1m", L, W, torch, dev, stream, rank, world, local, dist, full=False,
                         cpu=True)
        line["secondary"] = {"chung_lu1m": {k: sec[k] for k in ("value", "unit", "ms_per_step", "steps", "warmup")}
                             | {k: sec["config"][k] for k in ("levels", "cycles", "acf", "rel_res", "setup_s_host",
                                                              "solve_s_host", "gamma_coarse_max", "elim")}
                             | {"roofline_frac": (sec["roofline"] or {}).get("frac"),
                                "fp64_vs_ir": sec["fp64_vs_ir"], "cpu_baseline": sec["cpu_baseline"]}}
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def run_single(args, workload, L, W, torch, dev, stream, rank, world, local, dist, full, cpu=None):
    """One graph: setup + solve to tol per step.  full: also the end-to-end form
    and the CPU baseline; otherwise only the device-timed steps and the FP64
    comparison (a secondary workload of the same run), and the CPU baseline if
    cpu is set."""
    cpu_leg = full if cpu is None else cpu
    gname, pdef, desc = WORKLOADS[workload]
    prec_name = (args.precision if full else None) or pdef
    prec = L.LAMG_FP32_IR if prec_name == "fp32ir" else L.LAMG_FP64
    tol = TOL[workload]
    steps, warmup = (args.steps, args.warmup) if full else (min(args.steps, 3), 3)
    g = W.config_graph(gname)
    b_host = W.zero_sum_rhs(g.n, 2)
    w_dtype = torch.float32 if workload == "chung_lu1m" else torch.float64
    rp = torch.tensor(g.rp, device=dev)
    col = torch.tensor(g.col, device=dev)
    w = torch.tensor(g.w, device=dev).to(w_dtype)
    b = torch.tensor(b_host, device=dev)
    x = torch.zeros_like(b)
    mopts, adaptive = method_options(args, workload, g.n)
    opt = L.lamg_default_options(validate=1, max_cycles=2000, adaptive=int(adaptive), **mopts)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 512 MB > L2

    def step():
        h = L.lamg_setup(g.n, rp, col, w, opt, stream)
        # CUDA events around the engine launches only (two per launch, on this stream)
        L.lamg_profile(h, True)
        x.zero_()
        st = L.lamg_solve(h, b, x, tol, prec, stream)
        prof = L.lamg_profile(h, False)
        L.lamg_free(h)
        return st, prof

    for _ in range(warmup):
        step()
        flush.fill_(1.0)
    torch.cuda.synchronize()
    # timed region: each step bracketed by CUDA events; L2 flushed between steps
    evs, stats = [], []
    prof_ms, prof_cnt, prof_bytes = 0.0, 0, 0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = L.lamg_launch_count()
    with ClockSampler(local) as clk:
        for _ in range(steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st, prof = step()
            e1.record(stream)
            evs.append((e0, e1))
            stats.append(st)
            prof_ms += prof[0] * prof[1]
            prof_cnt += prof[1]
            prof_bytes = prof[2]
            flush.fill_(1.0)
        torch.cuda.synchronize()
    launches = L.lamg_launch_count() - launches0
    if dist:
        dist.barrier()
    times = [a.elapsed_time(bb) for a, bb in evs]
    ms = slowest_rank_ms(sum(times) / len(times), dist, dev)
    cycles = sum(s.cycles for s in stats) / len(stats)
    value = job_value(world, g.m * cycles, ms)

    # plain FP64 on the same workload, same accuracy (context for the IR form)
    fp64 = None
    if prec == L.LAMG_FP32_IR:
        h = L.lamg_setup(g.n, rp, col, w, opt, stream)
        res = {}
        for name, p in (("fp64", L.LAMG_FP64), ("fp32ir", prec)):
            x.zero_()
            L.lamg_solve(h, b, x, tol, p, stream)  # warm
            x.zero_()
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            stp = L.lamg_solve(h, b, x, tol, p, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            res[name] = (e0.elapsed_time(e1), stp)
        fp64 = {"solve_ms_fp64": res["fp64"][0], "cycles_fp64": res["fp64"][1].cycles,
                "solve_ms_fp32ir": res["fp32ir"][0], "cycles_fp32ir": res["fp32ir"][1].cycles,
                "rel_res_fp64": res["fp64"][1].rel_res, "rel_res_fp32ir": res["fp32ir"][1].rel_res}
        L.lamg_free(h)

    if full and args.op_times and rank == 0:
        # one more solve with the engine's op timer (outside the timed region)
        h = L.lamg_setup(g.n, rp, col, w, opt, stream)
        x.zero_()
        L.lamg_solve(h, b, x, tol, prec, stream)
        L.lamg_op_times(h, 1)
        x.zero_()
        sto = L.lamg_solve(h, b, x, tol, prec, stream)
        rows = L.lamg_op_times(h, 0)
        L.lamg_op_times(h, -1)
        lv = [L.lamg_level_info(h, l) for l in range(sto.levels)]
        L.lamg_free(h)
        with open(args.op_times, "w") as f:
            f.write(f"# engine op times: {workload}, {prec_name}, {sto.cycles} cycles, block 0's clock\n")
            for l, i in enumerate(lv):
                f.write(f"# level {l}: n {i['n']} nnz {i['nnz']} colours {i['ncolours']} gamma {i['gamma']:.3f}\n")
            f.write("level\top\tsingle_block\tcount\ttotal_ms\tper_us\n")
            for r in sorted(rows, key=lambda r: -r[4]):
                f.write(f"{r[0]}\t{r[1]}\t{r[2]}\t{r[3]}\t{r[4]:.3f}\t{1e3 * r[4] / r[3]:.2f}\n")

    # end to end through the host-array API, the same K steps: the graph and b from
    # pinned host memory, setup, solve, x back to the host; mean over the steps
    e2e = None
    if full and not args.no_e2e:
        rp_h = torch.tensor(g.rp).pin_memory()
        col_h = torch.tensor(g.col).pin_memory()
        w_h = torch.tensor(g.w).to(w_dtype).pin_memory()
        b_h = torch.tensor(b_host).pin_memory()
        x_h = torch.zeros(g.n, dtype=torch.float64).pin_memory()
        rp_d, col_d, w_d = torch.empty_like(rp), torch.empty_like(col), torch.empty_like(w)
        h2d = rp_h.numel() * 8 + col_h.numel() * 4 + w_h.numel() * w_h.element_size() + b_h.numel() * 8
        d2h = x_h.numel() * 8
        tt, cyc_e = [], []
        for it in range(warmup + steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rp_d.copy_(rp_h, non_blocking=True)
            col_d.copy_(col_h, non_blocking=True)
            w_d.copy_(w_h, non_blocking=True)
            h = L.lamg_setup(g.n, rp_d, col_d, w_d, opt, stream)
            x_h.zero_()
            st = L.lamg_solve_host(h, b_h.numpy(), x_h.numpy(), tol, prec, stream)
            torch.cuda.synchronize()
            L.lamg_free(h)
            if it >= warmup:
                tt.append(time.perf_counter() - t0)
                cyc_e.append(st.cycles)
        te = sum(tt) / len(tt)
        e2e = {"value": world * g.m * (sum(cyc_e) / len(cyc_e)) / te, "unit": "edges*cycles/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "ms_per_step": te * 1e3,
               "steps": steps, "statistic": "mean over the timed steps"}

    peak, peak_kind = load_peaks()
    roof = None
    if prof_cnt:
        avg = prof_ms / prof_cnt
        achieved = prof_bytes / (avg / 1e3) / 1e9
        traffic, tsrc = profiled_traffic(workload, prec_name)
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "traffic_source": tsrc,
                "kernel": "cycle engine k_engine (one launch = one refinement step: ir_inner FP32 cycles + FP64 "
                          "update, projection and residual)" if prec == L.LAMG_FP32_IR else
                          "cycle engine k_engine (one launch = one FP64 cycle + residual)",
                "bytes_per_launch": prof_bytes, "avg_ms": avg, "launches": prof_cnt,
                "peak_kind": f"{peak_kind} hbm_gbs (burst copy)"}

    cpu = None
    if cpu_leg and rank == 0 and world == 1 and not args.no_cpu_baseline:
        sg, sdesc = sample_graph(workload)
        sb = W.zero_sum_rhs(sg.n, 2)
        sopts, sadaptive = method_options(args, workload, sg.n)
        t, c = cpu_oracle_step(sg, sb, tol, sopts, sadaptive)
        same = sg.n == g.n and sg.m == g.m
        cpu = {"value": sg.m * c / t, "unit": "edges*cycles/s", "cores": 1, "kind": "oracle",
               "sample": f"{sdesc}, FP64 setup + solve to {tol:g} with the same options: {c} cycles in {t:.1f} s"
                         + ("" if same else "; rate per edge*cycle extrapolated to the full workload"),
               "host": host_cpu()}

    s0 = stats[-1]
    return {
        "metric": "edges*cycles/s (LAMG setup + solve to tol)",
        "value": value, "unit": "edges*cycles/s", "n_gpus": world, "steps": steps,
        "warmup": warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if prec == L.LAMG_FP32_IR else "f64", "data": "synthetic",
        "config": {"workload": workload, "desc": desc, "n": g.n, "m": g.m, "tol": tol,
                   "precision": prec_name, **mopts, "levels": s0.levels, "cycles": cycles, "acf": s0.acf,
                   "rel_res": s0.rel_res, "time_to_tol_s": ms / 1e3,
                   "setup_s_host": s0.t_setup_s, "solve_s_host": s0.t_solve_s,
                   "model_bytes_per_cycle": s0.bytes_per_cycle32 if prec == L.LAMG_FP32_IR else s0.bytes_per_cycle,
                   "l2": "flushed between steps (512 MB write)", "parallelism": f"replicas{world}"},
        "fp64_vs_ir": fp64,
        "e2e": e2e,
        "roofline": roof,
        "cpu_baseline": cpu,
        "clocks": clk.summary(),
        "gpu_launches": launches,
    }


if __name__ == "__main__":
    main()
