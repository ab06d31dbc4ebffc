"""Benchmark: SpHcurlAMG setup + solve to a 1e-8 relative residual on one synthetic eddy-current
system per GPU (replicas; no data exchange between ranks).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload kuhn128] [--impl mine|reference]

One step = sphc_setup (the whole hierarchy: nodal operator, colourings, aggregation, P_n, D_H,
pattern, least-norm initial guess, learned warm start of P_e, energy minimisation, Galerkin
operators, coarse factor, V-cycle operators) + sphc_solve (FP32 V-cycle inside FP64 CG, x0 = 0,
tol 1e-8) + sphc_destroy, with the inputs already resident in device memory.  The plain FP32
and plain FP64 GPU paths are timed after it on the same GPU and reported under `comparators`.  `value` is seconds per
system (lower is better); with N ranks it is the slowest rank's time divided by the systems all
ranks processed.  `e2e` repeats the step through the same C ABI with pinned host buffers, the
host-to-device input copies and the device-to-host copy of x inside the timed region.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD_TEXT = {
    "kuhn128": "128^3-cell Kuhn-tet unit cube, 14,532,992 interior-edge unknowns (236,921,168 nnz), interior nodes "
               "jittered uniform +-0.2h (seed 4), per-tet log10 sigma ~ N(0, 2^2) clipped to [-6, 2] (seed 5), "
               "tangential Dirichlet edges eliminated, RHS uniform[-1,1] (seed 6)",
    "kuhn48": "48^3-cell Kuhn-tet unit cube, 753,552 unknowns, +-0.2h jitter (seed 2), sigma 1 inside [0.25,0.75]^3 "
              "else 1e-3, RHS seed 3",
    "kuhn8": "8^3-cell Kuhn-tet unit cube, 3,032 unknowns, no jitter, sigma 1, RHS seed 1",
}
WORKLOAD_TEXT["batch64"] = ("64 independent Kuhn-tet systems, cells per axis n_s uniform in 12..64 (splitmix64 seed 200+s), "
                            "+-0.2h jitter (seed 200+s), per-tet log10 sigma ~ N(0, 2^2) clipped to [-6, 2] "
                            "(seed 300+s), 4 RHS uniform[-1,1] each (seeds 400+4s..403+4s)")
CPU_SAMPLE = "kuhn32"   # oracle sample for the CPU baseline (about 10 s of single-threaded work)


def batch64_specs():
    """The 64 systems of the batched workload: (MeshSpec, first RHS seed) per system."""
    import meshgen
    M = (1 << 64) - 1

    def splitmix64(seed, counter):
        z = (seed + (counter + 1) * 0x9E3779B97F4A7C15) & M
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        return z ^ (z >> 31)

    out = []
    for sidx in range(64):
        n = 12 + splitmix64(200 + sidx, 0) % 53
        out.append((meshgen.MeshSpec(int(n), jitter=0.2, seed_jitter=200 + sidx, sigma="lognormal", sigma_in=2.0,
                                     seed_sigma=300 + sidx), 400 + 4 * sidx))
    return out


PAPER3D = {9: (5859, [4, 9, 11, 12, 12], 1.13), 27: (144423, [5, 12, 12, 13, 13], 1.11),
           81: (3779379, [9, 12, 13, 13, 11], 1.10)}
PAPER3D_SIGMA = [1e2, 1e1, 1.0, 1e-1, 1e-2]


def run_paper3d(args, rank, local):
    """The paper's 3D tetrahedral table (Sec. 6.1): natural BCs, unjittered Kuhn meshes with 10^3,
    28^3 and 82^3 nodes, constant sigma, FP64 V-cycle in PCG, tolerance 1e-8 capped at
    kappa_1(D^-1 A) / 1e16 (kappa by the library's Hager estimate).  One JSON line: CG iterations,
    operator complexity and setup + solve seconds beside the paper's counts (Matlab, hardware not
    stated).  Context, not a bench value: the headline is the default workload."""
    import numpy as np
    import torch

    import meshgen
    import paper_2506_08284_gb300 as pkg
    if rank != 0:
        return
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    dev = lambda a: torch.from_numpy(a).cuda()
    rows = []
    for n, (edges, paper, oc_paper) in PAPER3D.items():
        for sigma, its_paper in zip(PAPER3D_SIGMA, paper):
            p = meshgen.generate(meshgen.MeshSpec(n, natural=True, sigma="const", sigma_in=sigma),
                                 nthreads=min(os.cpu_count() or 1, 32))
            assert p.n_edges == edges
            A = (p.n_edges, p.n_edges, dev(p.A_rowptr), dev(p.A_col), dev(p.A_val))
            D = (p.n_edges, p.n_nodes, dev(p.D_rowptr), dev(p.D_col), dev(p.D_val))
            b = dev(meshgen.rhs(1, p.n_edges))
            x = torch.zeros_like(b)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h = pkg.sphc.setup(A, D, opts=pkg.sphc.default_opts(vcycle_fp32=0, pn_alg1=args.pn_alg1,
                                                                sa_theta=args.sa_theta), stream=stream)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            kappa, _, _ = h.cond_estimate(5, stream=stream)
            tol = max(1e-8, kappa / 1e16)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            rc, it, rr = h.solve(b, x, tol=tol, stream=stream)
            torch.cuda.synchronize()
            t3 = time.perf_counter()
            st = h.stats()
            h.destroy()
            rows.append({"nodes": f"{n + 1}^3", "edges": p.n_edges, "sigma": sigma, "iters": it[0],
                         "paper_iters": its_paper, "status": rc, "relres": rr[0], "tol": tol, "kappa1_est": kappa,
                         "levels": st["n_levels"], "op_complexity": round(st["operator_complexity"], 3),
                         "paper_op_complexity": oc_paper, "setup_s": t1 - t0, "solve_s": t3 - t2})
    line = {"metric": "paper 3D tet table: CG iterations (context)", "impl": "mine", "unit": "iterations",
            "higher_is_better": False, "rows": rows, "pn_alg1": args.pn_alg1, "sa_theta": args.sa_theta,
            "note": "paper: Matlab, hardware not stated; aggregates differ from the paper's (MIS-2 rather than "
                    "MueLu's phases)" + ("; D_H from Alg. 1" if args.pn_alg1 else
                                         "; D_H from the tentative P-bar instead of Alg. 1")}
    print(json.dumps(line), flush=True)


def run_learned96(args, rank, local):
    """Config 4: the learned warm start on the 96^3 test mesh (jitter 0.2h, log-normal sigma) against
    plain energy minimisation with 1 and 4 steps: setup time, CG iterations (FP32 V-cycle),
    A-energy trace(P_e^T A P_e) per level and the V-cycle convergence factor (30 stationary
    iterations from a random x with b = 0, geometric mean of the last 10 A-norm ratios)."""
    import torch

    import meshgen
    import paper_2506_08284_gb300 as pkg
    from paper_2506_08284_gb300 import learned
    if rank != 0:
        return
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    spec, seed = meshgen.workload("kuhn96")
    p = meshgen.generate(spec, nthreads=min(os.cpu_count() or 1, 32))
    dev = lambda a: torch.from_numpy(a).cuda()
    A = (p.n_edges, p.n_edges, dev(p.A_rowptr), dev(p.A_col), dev(p.A_val))
    D = (p.n_edges, p.n_nodes, dev(p.D_rowptr), dev(p.D_col), dev(p.D_val))
    coords, sig, b = dev(p.coords), dev(p.sigma_edge), dev(meshgen.rhs(seed, p.n_edges))
    w = learned.load_weights()
    arms = [("plain, 1 step", dict(emin_iters=1)), ("plain, 4 steps", dict(emin_iters=4)),
            ("plain, projected CG 2 steps", dict(emin_method=1, emin_iters=2)),
            ("learned, 0 steps", dict(learned=1, learned_emin_iters=0, mlp_params=w)),
            ("learned, 1 step", dict(learned=1, learned_emin_iters=1, mlp_params=w))]
    rows = []
    for name, kw in arms:
        o = pkg.sphc.default_opts(vcycle_fp32=1, emin_fp32=1, **kw)
        for rep in range(2):                      # the second setup is timed (memory pool warm)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h = pkg.sphc.setup(A, D, coords, sig, o, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            setup_ms = e0.elapsed_time(e1)
            if rep == 0:
                h.destroy()
        x = torch.zeros_like(b)
        rc, it, rr = h.solve(b, x, stream=stream)
        st = h.stats()
        energies = [h.energy(l, stream=stream) for l in range(st["n_levels"] - 1)]
        factor = h.vcycle_factor(30, 10, seed=1, stream=stream)
        rows.append({"arm": name, "setup_ms": setup_ms, "solve_ms": st["solve_ms"], "iters": it[0], "status": rc,
                     "energy_per_level": energies, "vcycle_factor": factor})
        h.destroy()
    line = {"metric": "learned warm start vs plain energy minimisation (context)", "impl": "mine",
            "config": {"workload": "kuhn96: 96^3-cell Kuhn-tet cube, 6,110,496 unknowns, +-0.2h jitter, log10 sigma ~ "
                                   "N(0, 2^2) clipped to [-6, 2]"}, "rows": rows}
    print(json.dumps(line), flush=True)


def run_batch64(args, rank, world, local):
    """Config 5: all 64 systems set up (concurrently, host threads on their own streams) and solved
    for 4 right-hand sides each through one CUDA graph per right-hand side whose branches run every
    system's whole CG.  One step = sphc_setup_batched + sphc_solve_batched (4 RHS) +
    sphc_batch_destroy, inputs resident on the device.  value = systems per second (all ranks)."""
    import numpy as np
    import torch

    import meshgen
    import paper_2506_08284_gb300 as pkg
    from paper_2506_08284_gb300 import learned

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    weights = learned.load_weights() if os.path.exists(learned.WEIGHTS) else None
    dev = lambda a: torch.from_numpy(a).cuda()
    systems, bs, xs, n_unknowns = [], [], [], 0
    for spec, rseed in batch64_specs():
        p = meshgen.generate(spec, nthreads=min(os.cpu_count() or 1, 32))
        systems.append(((p.n_edges, p.n_edges, dev(p.A_rowptr), dev(p.A_col), dev(p.A_val)),
                        (p.n_edges, p.n_nodes, dev(p.D_rowptr), dev(p.D_col), dev(p.D_val)), dev(p.coords),
                        dev(p.sigma_edge)))
        bs.append(dev(meshgen.rhs(rseed, p.n_edges, nrhs=4)))
        xs.append(torch.zeros_like(bs[-1]))
        n_unknowns += p.n_edges
    stream = torch.cuda.current_stream()

    def step(opts):
        B = pkg.sphc.setup_batched(systems, opts, stream)
        rc, it, rr = B.solve(bs, xs, nrhs=4, stream=stream)
        B.destroy()
        return rc, it, rr

    def timed(opts, steps, warmup):
        for _ in range(warmup):
            step(opts)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        launches0 = pkg.sphc.launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = [step(opts) for _ in range(steps)]
        e1.record(stream)
        torch.cuda.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
        return ms, pkg.sphc.launch_count() - launches0, res[-1]

    clk = ClockSampler(local)
    head = make_opts(pkg, "headline", weights, 0, True)
    clk.start()
    ms, launches, (rc, it, rr) = timed(head, args.steps, args.warmup)
    clocks = clk.stop()
    fp64_ms, _, (rc64, it64, rr64) = timed(make_opts(pkg, "fp64_plain", weights, 0, True), max(1, min(args.steps, 2)), 1)
    fp64_steps = max(1, min(args.steps, 2))
    value = 64 * args.steps * world / (ms / 1e3)
    if rank == 0:
        line = {"metric": "systems/s, setup+solve to 1e-8 residual (batched uneven systems, 4 RHS each)",
                "value": value, "unit": "systems/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64 CG / f32 V-cycle", "data": "synthetic",
                "config": {"workload": f"batch64: {WORKLOAD_TEXT['batch64']}", "unknowns_total": n_unknowns,
                           "solver": "FP32 V-cycle + learned warm start in FP64 CG, one graph per RHS",
                           "l2": "inputs exceed the 129 MB L2; no flush", "parallelism": f"replicas x{world}"},
                "status": rc, "iters_max": int(np.max(it)), "iters_mean": float(np.mean(it)),
                "relres_max": float(np.max(rr)), "gpu_launches": int(launches), "clocks": clocks,
                "comparators": {"fp64_plain": {"systems_per_s": 64 * fp64_steps * world / (fp64_ms / 1e3),
                                               "status": rc64, "iters_max": int(np.max(it64))},
                                "speedup_vs_fp64_plain": (64 * args.steps / (ms / 1e3)) /
                                                         (64 * fp64_steps / (fp64_ms / 1e3))}}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="kuhn128")
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--no-block", action="store_true", help="skip the block-of-16-right-hand-sides leg")
    ap.add_argument("--pn-alg1", type=int, default=0, help="paper3d: D_H from Alg. 1 on the smoothed P_n")
    ap.add_argument("--sa-theta", type=float, default=0.0, help="paper3d: SA drop tolerance")
    ap.add_argument("--oracle-check", action="store_true",
                    help="also run the OpenMP oracle once on the full workload: its time, and the GPU headline "
                         "solution against its solution")
    ap.add_argument("--block-rhs", type=int, default=16)
    ap.add_argument("--no-graph", action="store_true",
                    help="run CG with a host loop instead of the CUDA graph (same kernels; for profilers "
                         "that cannot see kernels inside graphs with conditional nodes)")
    return ap.parse_args()


# ---- aggregation over ranks (one replica system per rank, no data exchange)
def max_over_ranks(value, dist, device):
    """The largest of every rank's value (the slowest rank sets the job's time); value as is
    without a process group."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def seconds_per_system(ms_slowest, steps, world):
    """Whole-job seconds per system: every rank solves `steps` systems in the slowest rank's time."""
    return ms_slowest / 1e3 / (steps * world)


def pinned_h2d_gbs(stream, nbytes=1 << 30, reps=3):
    """This machine's host-to-device rate for one plain copy of a pinned buffer (best of `reps`, CUDA
    events on `stream`), outside the timed steps: the end-to-end figure moves with it.  None when
    the buffers cannot be had."""
    import torch
    try:
        h = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
        d = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        best = None
        with torch.cuda.stream(stream):
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                d.copy_(h, non_blocking=True)
                e1.record(stream)
                e1.synchronize()
                ms = e0.elapsed_time(e1)
                best = ms if best is None else min(best, ms)
        del h, d
        return nbytes / (best / 1e3) / 1e9 if best else None
    except Exception:
        return None


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "sgs_level0_traffic_kuhn128.txt")


def sweep_traffic():
    """DRAM bytes of one level-0 forward + backward sweep from the committed ncu capture, or None
    when the kernel source has changed since the counters were taken."""
    import hashlib
    try:
        fields = {}
        for line in open(TRAFFIC_FILE):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                fields[k.strip()] = v.strip()
        h = hashlib.sha1()
        for name in ("sell.cuh", "solve.cu"):            # the sweep kernel and its helpers
            h.update(open(os.path.join(ROOT, "paper_2506_08284_gb300", "csrc", name), "rb").read())
        if fields.get("sweep_src_sha1") != h.hexdigest():
            return None
        return float(fields["dram_bytes_per_sweep"])
    except Exception:
        return None


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks during the timed region
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
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
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        sm = sorted(r[0] for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[2][i].lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


# ------------------------------------------------------------------ CPU oracle baseline
def _oracle_openmp():
    """Import the oracle in its OpenMP build (row-parallel loops only, bit-identical results),
    which then runs on every host core."""
    os.environ["SPHC_ORACLE_OPENMP"] = "1"
    import oracle
    return oracle


def cpu_baseline(target_edges, steps=1):
    """The oracle (FP64 C, OpenMP build on all host cores) on a bounded sample: the workload's
    recipe at 32^3 cells, scaled to the workload by the number of unknowns (AMG setup and solve
    are linear in the unknowns)."""
    import meshgen
    oracle = _oracle_openmp()

    spec, seed = meshgen.workload(CPU_SAMPLE)
    p = meshgen.generate(spec)
    b = meshgen.rhs(seed, p.n_edges)
    ts = []
    its = None
    for _ in range(steps):
        t0 = time.perf_counter()
        h = oracle.setup_problem(p, sa_theta=SA_THETA)
        r = h.solve(b, tol=1e-8)
        ts.append(time.perf_counter() - t0)
        its = r["iters"]
        del h
    t = sum(ts) / len(ts)
    scale = target_edges / p.n_edges
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": t * scale, "unit": "s", "cores": cores, "kind": "oracle",
            "sample": f"{CPU_SAMPLE} (the same recipe at 32^3 cells, {p.n_edges:,} unknowns): setup+solve {t:.2f} s "
                      f"({its} CG iterations) with the OpenMP oracle on {cores} cores, scaled x{scale:.1f} by "
                      f"unknowns to the workload"}


def bench_config(args, world, learned_weights):
    """The workload description shared by both arms (the reference arm times the oracle on a
    bounded sample of this workload, named in its cpu_baseline)."""
    return {"workload": f"{args.workload}: {WORKLOAD_TEXT.get(args.workload, '')}",
            "solver": "SpHcurlAMG V-cycle (1 pre + 1 post symmetric Hiptmair) in FP64 CG, FP32 V-cycle, "
                      + ("learned warm start of P_e + 1 energy-minimisation step" if learned_weights
                         else "least-norm P0 + 1 energy-minimisation step (no MLP weights found)"),
            "rhs": 1, "tol": args.tol, "l2": "inputs (A_e 2.8 GB FP64) exceed the 129 MB L2; no flush",
            "parallelism": f"replicas x{world}",
            **({"sa_theta": args.sa_theta} if args.sa_theta > 0 else {})}


def workload_edges(name):
    import meshgen
    return meshgen.counts(meshgen.workload(name)[0])["n_edges"]


def run_reference(args, rank):
    if rank != 0:
        return
    from paper_2506_08284_gb300 import learned
    target = workload_edges(args.workload)
    for _ in range(args.warmup):
        cpu_baseline(target, 1)
    t0 = time.perf_counter()
    vals = [cpu_baseline(target, 1) for _ in range(args.steps)]
    wall = time.perf_counter() - t0
    v = sum(x["value"] for x in vals) / len(vals)
    cb = dict(vals[-1])
    cb["value"] = v
    line = {"metric": "setup+solve s to 1e-8 residual", "value": v, "unit": "s", "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall / args.steps * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": bench_config(args, args.gpus, os.path.exists(learned.WEIGHTS)),
            "cpu_baseline": cb, "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
SA_THETA = 0.0      # drop tolerance of every GPU arm (--sa-theta)


def make_opts(pkg, variant, weights, profile, graph=True):
    o = _make_opts(pkg, variant, weights, profile)
    o.cg_graph = 1 if graph else 0
    o.sa_theta = SA_THETA
    return o


def _make_opts(pkg, variant, weights, profile):
    """headline: FP32 V-cycle + learned warm start (one energy-minimisation step after it, its masked
    product accumulated in FP32); fp32_plain: FP32 V-cycle, plain least-norm P0 + one step (FP32
    product); fp64_plain: everything in FP64."""
    if variant == "headline" and weights is not None:
        return pkg.sphc.default_opts(vcycle_fp32=1, emin_fp32=1, learned=1, learned_emin_iters=1, mlp_params=weights,
                                     profile=profile)
    if variant in ("headline", "fp32_plain"):
        return pkg.sphc.default_opts(vcycle_fp32=1, emin_fp32=1, profile=profile)
    return pkg.sphc.default_opts(vcycle_fp32=0, emin_fp32=0, profile=profile)


def main():
    global SA_THETA
    args = parse_args()
    SA_THETA = args.sa_theta
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.workload == "batch64":
        run_batch64(args, rank, world, local)
        return
    if args.workload == "paper3d":
        run_paper3d(args, rank, local)
        return
    if args.workload == "learned96":
        run_learned96(args, rank, local)
        return

    import numpy as np
    import torch

    import meshgen
    import paper_2506_08284_gb300 as pkg
    from paper_2506_08284_gb300 import learned

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    spec, seed = meshgen.workload(args.workload)
    p = meshgen.generate(spec, nthreads=min(os.cpu_count() or 1, 32))
    b = meshgen.rhs(seed, p.n_edges)
    weights = learned.load_weights() if os.path.exists(learned.WEIGHTS) else None
    dev = lambda a: torch.from_numpy(a).cuda()
    A = (p.n_edges, p.n_edges, dev(p.A_rowptr), dev(p.A_col), dev(p.A_val))
    D = (p.n_edges, p.n_nodes, dev(p.D_rowptr), dev(p.D_col), dev(p.D_val))
    coords, sig = dev(p.coords), dev(p.sigma_edge)
    bd = dev(b)
    xd = torch.zeros_like(bd)
    stream = torch.cuda.current_stream()

    def step(opts, A_, D_, c_, s_, b_, x_):
        h = pkg.sphc.setup(A_, D_, c_, s_, opts, stream)
        rc, it, rr = h.solve(b_, x_, tol=args.tol, stream=stream)
        prof = h.profile() if opts.profile else {}
        st = h.stats()
        info = [h.level_info(l) for l in range(st["n_levels"])]
        h.destroy()
        return rc, it[0], rr[0], prof, st, info

    def timed(opts, steps, warmup, sample_clocks=False):
        for _ in range(warmup):
            step(opts, A, D, coords, sig, bd, xd)
        torch.cuda.synchronize()
        clk = ClockSampler(local) if sample_clocks else None
        if clk:
            clk.start()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        launches0 = pkg.sphc.launch_count()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        t0 = time.perf_counter()
        res = [step(opts, A, D, coords, sig, bd, xd) for _ in range(steps)]
        ev1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        if dist:
            dist.barrier()
        launches = pkg.sphc.launch_count() - launches0
        clocks = clk.stop() if clk else None
        ms = max_over_ranks(ev0.elapsed_time(ev1), dist, "cuda")
        return ms, wall, launches, clocks, res

    # headline: FP32 V-cycle + learned warm start
    opts = make_opts(pkg, "headline", weights, 1, not args.no_graph)
    ms, wall, launches, clocks, results = timed(opts, args.steps, args.warmup, sample_clocks=True)
    sec_per_system = seconds_per_system(ms, args.steps, world)
    rc, iters, relres, prof, st, info = results[-1]

    # comparators on the same GPU: plain FP32 and plain FP64 GPU paths (outside the timed steps)
    comparators = {}
    if not args.no_compare:
        for name in ("fp32_plain", "fp64_plain"):
            cms, _, _, _, cres = timed(make_opts(pkg, name, weights, 0, not args.no_graph), max(1, min(args.steps, 2)), 1)
            c_rc, c_it, c_rr, _, c_st, _ = cres[-1]
            comparators[name] = {"s": seconds_per_system(cms, max(1, min(args.steps, 2)), world), "iters": c_it,
                                 "relres": c_rr, "status": c_rc, "setup_ms": c_st["setup_ms"],
                                 "solve_ms": c_st["solve_ms"]}
        comparators["speedup_vs_fp64_plain"] = comparators["fp64_plain"]["s"] / sec_per_system

    # block of right-hand sides on one hierarchy (config 3: seeds 6..21): one CG per column, every
    # operator row read once per block; setup excluded, solve timed with CUDA events
    block = None
    if not args.no_block and args.block_rhs >= 2:
        nb = args.block_rhs
        Bd = dev(meshgen.rhs(seed, p.n_edges, nrhs=nb))
        Xd = torch.zeros_like(Bd)
        ob = make_opts(pkg, "headline", weights, 0, not args.no_graph)
        hb = pkg.sphc.setup(A, D, coords, sig, ob, stream)
        hb.solve(Bd, Xd, tol=args.tol, nrhs=nb, stream=stream)          # warm-up (allocates the block work)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        brc, bit, brr = hb.solve(Bd, Xd, tol=args.tol, nrhs=nb, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        bms = e0.elapsed_time(e1)
        bst = hb.stats()
        # the single-right-hand-side solve on the same hierarchy, for the per-RHS comparison
        x1 = torch.zeros_like(bd)
        e0.record(stream)
        hb.solve(bd, x1, tol=args.tol, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        one_ms = e0.elapsed_time(e1)
        hb.destroy()
        block = {"nrhs": nb, "status": brc, "solve_ms": bms, "ms_per_rhs": bms / nb, "single_rhs_solve_ms": one_ms,
                 "speedup_per_rhs": one_ms / (bms / nb), "iters": bit, "max_relres": max(brr),
                 "setup_ms": bst["setup_ms"]}
        del Bd, Xd

    # end-to-end: the same call with pinned host buffers (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(a).pin_memory()
        Ah = (p.n_edges, p.n_edges, pin(p.A_rowptr), pin(p.A_col), pin(p.A_val))
        Dh = (p.n_edges, p.n_nodes, pin(p.D_rowptr), pin(p.D_col), pin(p.D_val))
        ch, sh, bh = pin(p.coords), pin(p.sigma_edge), pin(b)
        xh = torch.zeros(p.n_edges, dtype=torch.float64).pin_memory()
        o2 = make_opts(pkg, "headline", weights, 0, not args.no_graph)
        step(o2, Ah, Dh, ch, sh, bh, xh)
        torch.cuda.synchronize()
        eclk = ClockSampler(local)
        eclk.start()
        t1 = time.perf_counter()
        eres = [step(o2, Ah, Dh, ch, sh, bh, xh) for _ in range(args.steps)]
        torch.cuda.synchronize()
        te = max_over_ranks((time.perf_counter() - t1) / args.steps, dist, "cuda")
        eclocks = eclk.stop()
        h2d = sum(a.nbytes for a in (p.A_rowptr, p.A_col, p.A_val, p.D_rowptr, p.D_col, p.D_val, p.coords,
                                     p.sigma_edge, b))
        e_st = eres[-1][4]
        e2e = {"value": te / world, "unit": "s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(b.nbytes),
               "last_step_setup_ms": e_st["setup_ms"], "last_step_solve_ms": e_st["solve_ms"], "clocks": eclocks,
               "h2d_copy_gbs": pinned_h2d_gbs(stream)}

    peak, peak_kind = peaks()
    roof = None
    name = "sgs_A_level0"
    if name in prof and prof[name]["calls"] > 0:
        t_call = prof[name]["ms"] / prof[name]["calls"] / 1e3
        achieved = prof[name]["bytes_per_call"] / t_call / 1e9
        roof = {"bound": "hbm", "kernel": "k_sell_sgs<float> (level-0 forward+backward multicolour SGS sweep, "
                                          "SELL-32, one launch per colour and direction, the repeated "
                                          "middle colour left out)",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_kind": f"{peak_kind} HBM copy", "traffic": sweep_traffic(),
                "algorithmic_bytes_per_launch": prof[name]["bytes_per_call"], "ms_per_launch": t_call * 1e3}
        sp = prof.get("spmv_A_fp64")
        if sp and sp["calls"] > 0:
            tsp = sp["ms"] / sp["calls"] / 1e3
            roof["cg_spmv_fp64"] = {"achieved": sp["bytes_per_call"] / tsp / 1e9,
                                    "frac": sp["bytes_per_call"] / tsp / 1e9 / peak, "ms_per_launch": tsp * 1e3}
    # setup steps on the roofline: algorithmic bytes (each operand read once, the result written
    # once) over the section's CUDA-event time, against the same measured HBM peak
    setup_roof = {}
    for key, what in (("emin_level_l0", "energy-minimisation step of eq. (9), level 0: masked product + FP64 row projection"),
                      ("rap_level_l0", "Galerkin product P_e^T (A P_e), level 0"),
                      ("rap_AP_l0", "A P_e, level 0"), ("rap_PtAP_l0", "P_e^T (A P_e), upper triangle mirrored, level 0"),
                      ("setup_nodal_AD", "A_e D_h (nodal operator), level 0")):
        t = prof.get(key)
        if t and t["calls"] > 0 and t["bytes_per_call"] > 0:
            sec = t["ms"] / t["calls"] / 1e3
            ach = t["bytes_per_call"] / sec / 1e9
            setup_roof[key] = {"what": what, "ms": t["ms"] / t["calls"], "algorithmic_bytes": t["bytes_per_call"],
                               "achieved_gbs": ach, "frac": ach / peak}
    if roof is not None:
        roof["setup_steps"] = setup_roof
    oracle_check = None
    if args.oracle_check and rank == 0:
        # the headline arm once more on this process, then the oracle on the same inputs
        hc = pkg.sphc.setup(A, D, coords, sig, make_opts(pkg, "headline", weights, 0, not args.no_graph), stream)
        xc = torch.zeros_like(bd)
        crc, cit, crr = hc.solve(bd, xc, tol=args.tol, stream=stream)
        torch.cuda.synchronize()
        xg = xc.cpu().numpy()
        hc.destroy()
        oracle = _oracle_openmp()
        import platform
        t0 = time.perf_counter()
        ho = oracle.setup_problem(p)
        t1 = time.perf_counter()
        ro = ho.solve(b, tol=args.tol)
        t2 = time.perf_counter()
        err = float(np.linalg.norm(xg - ro["x"]) / np.linalg.norm(ro["x"]))
        mem = None
        try:
            mem = int(open("/proc/meminfo").read().split("MemTotal:")[1].split()[0]) // 1024
        except Exception:
            pass
        cpu_model = platform.processor() or platform.machine()
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith(("model name", "cpu part")):
                    cpu_model = ln.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
        oracle_check = {"oracle_setup_s": t1 - t0, "oracle_solve_s": t2 - t1, "oracle_iters": ro["iters"],
                        "oracle_relres": ro["relres"], "cores": os.cpu_count(), "cpu": cpu_model, "ram_mib": mem,
                        "gpu_iters": cit[0], "gpu_relres": crr[0],
                        "x_rel_err_vs_oracle": err}
        del ho
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(p.n_edges)

    if rank == 0:
        line = {
            "metric": "setup+solve s to 1e-8 residual", "value": sec_per_system, "unit": "s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64 CG / f32 V-cycle", "data": "synthetic",
            "config": bench_config(args, world, weights is not None),
            "iters": iters, "relres": relres, "status": rc, "wall_s_per_step": wall / args.steps,
            "setup_ms": st["setup_ms"], "solve_ms": st["solve_ms"], "levels": st["n_levels"],
            "operator_complexity": st["operator_complexity"], "gpu_launches": int(launches),
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "comparators": comparators,
            "speedup_vs_fp64_plain": comparators.get("speedup_vs_fp64_plain"), "rhs_block": block,
            "oracle_check": oracle_check,
            "profile": {k: {kk: round(vv, 4) if isinstance(vv, float) else vv for kk, vv in v.items()}
                        for k, v in prof.items()},
            "level_edges": [li["n_edges"] for li in info],
            "level_colours": [[li["n_colors_edge"], li["n_colors_node"], li["colour_rounds_edge"], li["colour_rounds_node"]]
                              for li in info],
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
