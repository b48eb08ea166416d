"""Benchmark: AP-Cloud electrostatic solves per second on GB300.

One step is one pass of the whole hot path on one synthetic beam-with-halo
particle set resident in HBM: octree build, stencils (neighbour search + WLS),
deposit and density solve, GMRES Poisson solve to rtol 1e-10, and the gather
of phi and E back to the particles.

Workload (default): 1e7 particles, octree depth 10, refinement constant
tuned to ~1e6 nodes, FP64 throughout.  With --gpus N (launched under
torchrun) every rank solves its own independent beam (seed 1 + rank): the
problems do not share data, so there is no collective on the data path and
the scaling is weak.  --impl reference times the CPU oracle instead.

Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "GFD Poisson solves/sec and nodes·iters/sec at rel-L2 ≤1e-6 vs FP64; % roofline"
WORKLOADS = {
    # name: (particles, max_depth, c_refine)
    "beam_halo_1e7_depth10": (10_000_000, 10, 0.043),
    "beam_halo_1e5_depth6": (100_000, 6, 1.0),
}
BATCH_WORKLOADS = {
    # name: (beams, max_depth, c_refine); particle counts log-uniform in [1e4, 1e6]
    "beam_batch_64_depth9": (64, 9, 0.05),
}


def make_problem(workload, seed):
    """(x, y, z, q, offsets or None, max_depth, c_refine, solves per step)"""
    from paper_1603_04039_gb300 import inputs
    if workload in BATCH_WORKLOADS:
        nb, depth, c = BATCH_WORKLOADS[workload]
        x, y, z, q, offs, _ = inputs.beam_batch(nb, seed)
        return x, y, z, q, offs, depth, c, nb
    npart, depth, c = WORKLOADS[workload]
    x, y, z, q = inputs.beam_with_halo(npart, seed)
    return x, y, z, q, None, depth, c, 1
RTOL = 1e-10
MAX_ITER = 200000


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _ncu_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` on `workload` from a committed ncu summary
    (a line 'traffic: kernel=... workload=... bytes_per_launch=...'), else None."""
    d = os.path.join(ROOT, "profiles")
    try:
        names = sorted(os.listdir(d))
    except OSError:
        return None
    for fn in names:
        if not fn.endswith(".md"):
            continue
        for line in open(os.path.join(d, fn)):
            if not line.startswith("traffic:"):
                continue
            kv = dict(t.split("=", 1) for t in line.split()[1:] if "=" in t)
            if kv.get("kernel") == kernel and kv.get("workload") == workload:
                return {"file": "profiles/" + fn, "bytes_per_launch": float(kv["bytes_per_launch"]),
                        "algorithmic_bytes_per_working_launch": float(kv["algorithmic_bytes_per_working_launch"])}
    return None


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [t.strip() for t in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------- our GPU path
def run_ours(args, ws, rank, local):
    import torch
    import torch.distributed as dist

    from paper_1603_04039_gb300 import APCloud, inputs
    from paper_1603_04039_gb300._binding import kernel_names, measure_fma_peak

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    fp64_peak, fp32_peak = measure_fma_peak()
    seed = 1 + rank
    x, y, z, q, offs, depth, c, nsolve = make_problem(args.workload, seed)
    npart = len(x)
    tx, ty, tz, tq = (torch.from_numpy(a).to(dev) for a in (x, y, z, q))

    def build(a):
        if offs is None:
            return a.build_octree(tx, ty, tz)
        return a.build_octree_batched(tx, ty, tz, offs)
    form = dict(max_depth=depth, c_refine=c, restart=30, precision=args.precision, poly_degree=args.poly_degree,
                poly_omega=args.poly_omega, device=dev)
    ap = APCloud(**form)
    out = tuple(torch.empty(npart, dtype=torch.float64, device=dev) for _ in range(4))
    stream = ap.stream
    info = {}

    def step():
        ni, nb = build(ap)
        ap.stencils()
        _, ir = ap.deposit(q=tq, rtol=RTOL, max_iter=MAX_ITER)
        _, ip = ap.solve(rtol=RTOL, max_iter=MAX_ITER)
        ap.gather_field(out)
        info.update(n_int=ni, n_bnd=nb, iters_rho=ir["iters"], iters_phi=ip["iters"], relres_phi=ip["relres"],
                    status=max(ir["status"], ip["status"]))

    def barrier():
        if ws > 1:
            dist.barrier()

    # launch shapes: the autotuner times them on this workload's node set (untimed)
    build(ap)
    ap.stencils()
    tuned = ap.autotune()
    # warm-up; the last warm-up step times every kernel kind to find the dominant one
    for w in range(args.warmup):
        if w == args.warmup - 1:
            ap.set_timing((1 << len(kernel_names())) - 1)
        step()
    torch.cuda.synchronize()
    all_kinds = ap.get_timing(reset=True)
    ap.set_timing(0)
    solve_kinds = {k: v for k, v in all_kinds.items() if v[1] > 0}
    dominant = max(solve_kinds, key=lambda k: solve_kinds[k][0])
    dom_bit = kernel_names().index(dominant)

    # timed region: inputs resident (positions and charges, 320 MB > L2), no
    # per-kernel timers (their event nodes would slow the step)
    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    torch.cuda.synchronize()
    launches0 = ap.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    iters_total = 0
    for _ in range(args.steps):
        step()
        iters_total += info["iters_phi"] + info["iters_rho"]
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms_total = e0.elapsed_time(e1)
    launches = ap.launch_count() - launches0
    # roofline region: the same K steps again with CUDA events around every
    # launch of the dominant kernel kind
    ap.set_timing(1 << dom_bit)
    r0 = torch.cuda.Event(enable_timing=True)
    r1 = torch.cuda.Event(enable_timing=True)
    r0.record(stream)
    for _ in range(args.steps):
        step()
    r1.record(stream)
    torch.cuda.synchronize()
    ms_timed_steps = r0.elapsed_time(r1)
    dom = ap.get_timing(reset=True)[dominant]
    ap.set_timing(0)
    clocks = sampler.stop()
    ms_step = ms_total / args.steps
    if ws > 1:
        t = torch.tensor([ms_step], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step = float(t.item())
    n_nodes = info["n_int"] + info["n_bnd"]
    sz = ap.sizes()

    # end to end through the host-buffer entry point (pinned host memory)
    hx, hy, hz, hq = (torch.from_numpy(a).pin_memory() for a in (x, y, z, q))
    hout = tuple(torch.empty(npart, dtype=torch.float64).pin_memory() for _ in range(4))
    ap_e2e = APCloud(**form)
    ap_e2e.set_launch_shape(spmv_block=tuned["spmv_block"], wls_warps=tuned["wls_warps"],
                            spmv_unroll=tuned["spmv_unroll"], sweep_sorted=tuned["sweep_sorted"])
    ap_e2e.field_host(hx, hy, hz, q=hq, rtol=RTOL, max_iter=MAX_ITER, out=hout, offsets=offs)   # warm-up
    barrier()
    e2e_steps = max(1, min(args.steps, 3))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ap_e2e.field_host(hx, hy, hz, q=hq, rtol=RTOL, max_iter=MAX_ITER, out=hout, offsets=offs)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    if ws > 1:
        t = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    ap_e2e.close()

    # the plain FP64 form (GMRES(30) + Jacobi) on the same particles: its fields are
    # the reference for this form's error, its step time the reference for the
    # speedup, and its iteration count is what the CPU oracle (same algorithm) needs
    ap64 = APCloud(max_depth=depth, c_refine=c, restart=30, precision="fp64", device=dev)
    ref = tuple(torch.empty(npart, dtype=torch.float64, device=dev) for _ in range(4))
    plain = {}
    for rep in range(2):
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(ap64.stream)
        build(ap64)
        ap64.stencils()
        _, pr = ap64.deposit(q=tq, rtol=RTOL, max_iter=MAX_ITER)
        _, pp = ap64.solve(rtol=RTOL, max_iter=MAX_ITER)
        ap64.gather_field(ref)
        f1.record(ap64.stream)
        torch.cuda.synchronize()
        plain = {"ms_per_step": round(f0.elapsed_time(f1), 2), "iters_phi": pp["iters"], "iters_rho": pr["iters"],
                 "relres_phi": pp["relres"]}
    if offs is None:
        errs = [float(torch.linalg.norm(a - b) / torch.linalg.norm(b)) for a, b in zip(out, ref)]
    else:   # the worst beam
        errs = [float(torch.linalg.norm(a[s:e] - b[s:e]) / torch.linalg.norm(b[s:e]))
                for a, b in zip(out, ref) for s, e in zip(offs[:-1], offs[1:]) if e > s]
    rel_l2 = max(errs) if (args.precision != "fp64" or args.poly_degree > 1) else 0.0
    ap64.close()
    unbatched = None
    if offs is not None:
        # the same form solving the beams one at a time (one context, same stream)
        ap1 = APCloud(**form)
        u0 = torch.cuda.Event(enable_timing=True)
        u1 = torch.cuda.Event(enable_timing=True)
        views = [(tx[s:e], ty[s:e], tz[s:e], tq[s:e]) for s, e in zip(offs[:-1], offs[1:])]
        per_beam = []
        for rep in range(2):
            per_beam = []
            u0.record(ap1.stream)
            for bx, by, bz, bq in views:
                ap1.build_octree(bx, by, bz)
                ap1.stencils()
                ap1.deposit(q=bq, rtol=RTOL, max_iter=MAX_ITER)
                _, ib = ap1.solve(rtol=RTOL, max_iter=MAX_ITER)
                ap1.gather_field()
                per_beam.append((ap1.n_nodes, ib["iters"]))
            u1.record(ap1.stream)
            torch.cuda.synchronize()
        ms_u = u0.elapsed_time(u1)
        # Arnoldi work (rows x steps) of the beams solved alone against the batch's
        work_alone = sum(nn * it for nn, it in per_beam)
        unbatched = {"ms_per_batch": round(ms_u, 2), "solves_per_s": round(nsolve * 1000.0 / ms_u, 4),
                     "speedup_of_batching": round(ms_u / ms_step, 2),
                     "poisson_steps_alone": {"min": min(it for _, it in per_beam),
                                             "max": max(it for _, it in per_beam),
                                             "node_weighted_mean": round(work_alone / sum(nn for nn, _ in per_beam), 1)},
                     "row_steps_alone_over_batch": round(work_alone / max(1, n_nodes * info["iters_phi"]), 3)}
        ap1.close()

    # roofline of the dominant kernel, measured live in the timed region
    peaks = _measured_peaks()
    ms_k, nl_k, by_k, fl_k = dom
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    gbs = by_k / (ms_k * 1e-3) / 1e9 if ms_k > 0 else 0.0
    tfs = fl_k / (ms_k * 1e-3) / 1e12 if ms_k > 0 else 0.0
    # the kernel's arithmetic type sets its ALU peak: in the mixed form the Krylov
    # iterations and the stencil factorisations run in FP32, everything else FP64
    fp32_kinds = {"spmv", "precond_sweep", "gmres_dots", "gmres_update_dots", "gmres_update_norm",
                  "gmres_cycle_end", "ring_select_wls"}
    alu_peak = fp32_peak if (args.precision == "mixed" and dominant in fp32_kinds) else fp64_peak
    alu_name = "FP32" if alu_peak == fp32_peak else "FP64"
    # work per byte decides the bound: above ALU peak / HBM peak the ALU limits
    if fl_k > 0 and fl_k / max(by_k, 1.0) > alu_peak * 1e12 / (hbm * 1e9):
        roof = {"bound": "alu", "achieved": round(tfs, 4), "peak": round(alu_peak, 4), "unit": "TFLOP/s",
                "frac": round(tfs / alu_peak, 4), "alu": alu_name}
    else:
        roof = {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s", "frac": round(gbs / hbm, 4),
                "alu": alu_name}
    roof.update({"kernel": dominant, "traffic": None, "launches": nl_k,
                 "algorithmic_bytes_per_launch": by_k / max(nl_k, 1),
                 "algorithmic_flops_per_launch": fl_k / max(nl_k, 1),
                 "share_of_step": round(ms_k / ms_timed_steps, 4),
                 "region": "a second pass of the K timed steps with CUDA events around every launch of this "
                           "kind (%.1f ms/step there, %.1f ms/step without the events)"
                           % (ms_timed_steps / args.steps, ms_step),
                 "peak_source": "measured: hbm_gbs of MEASURED_PEAKS.json; FP64/FP32 FMA chains on all SMs "
                                "(apcloud_measure_fma_peak) in this run",
                 "fp64_peak_tflops": round(fp64_peak, 4), "fp32_peak_tflops": round(fp32_peak, 3)})
    tr = _ncu_traffic(dominant, args.workload)
    if tr:
        roof["traffic"] = tr["bytes_per_launch"]
        roof["traffic_note"] = ("DRAM read + write of one working launch from an ncu capture (%s); "
                                "algorithmic bytes of a working launch %.4g; the per-launch average above also "
                                "counts launches that exit at once after convergence" %
                                (tr["file"], tr["algorithmic_bytes_per_working_launch"]))
    solves = ws * nsolve * 1000.0 / ms_step
    line = {
        "metric": METRIC, "value": round(solves, 4), "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
        "data": "synthetic", "rel_l2_vs_fp64": rel_l2,
        "config": {"workload": args.workload, "particles": npart, "beams": nsolve, "max_depth": depth, "c_refine": c,
                   "n_nodes": n_nodes, "n_interior": info["n_int"], "precision": args.precision,
                   "solver": ("GMRES(30), right preconditioner " +
                              ("Jacobi" if args.poly_degree <= 1 else
                               "Jacobi-Neumann polynomial, degree %d, omega %g" % (args.poly_degree, args.poly_omega)) +
                              ("" if args.precision == "fp64" else "; FP32 cycles inside FP64 iterative refinement")),
                   "rtol": RTOL,
                   "fp64_stencils": sz["fp64_stencils"],
                   "gmres_iters_phi": info["iters_phi"], "gmres_iters_rho": info["iters_rho"],
                   "relres_phi": info["relres_phi"], "l2": "inputs 320 MB > L2, no flush",
                   "nnz": sz["nnz"], "ell_fill": round(sz["nnz"] / max(1, sz["ell_entries"]), 4),
                   "parallelism": "independent beam per GPU" if ws > 1 else "single GPU",
                   "autotuned": tuned, "cuda_graphs": ap.graph_stats()},
        "nodes_iters_per_s": round(ws * n_nodes * (iters_total / args.steps) / (ms_step * 1e-3), 1),
        "e2e": {"value": round(ws * nsolve / e2e_s, 4), "unit": "solves/s", "h2d_bytes_per_step": 32 * npart,
                "d2h_bytes_per_step": 32 * npart},
        "roofline": roof, "gpu_launches": int(launches), "clocks": clocks,
        "plain_fp64_form": dict(plain, solves_per_s=round(nsolve * 1000.0 / plain["ms_per_step"], 4),
                                speedup_of_this_form=round(plain["ms_per_step"] / ms_step, 2)),
        "unbatched_same_form": unbatched,
        "stage_ms_by_kernel": {k: round(v[0] / 1, 3) for k, v in solve_kinds.items()},
    }
    return line


# ---------------------------------------------------------------- oracle
def oracle_sample(workload, seed=1, gmres_sample=10, gmres_iters_hint=None):
    """Times the CPU oracle on the workload: the tree, stencils, deposit and
    gather in full, and `gmres_sample` GMRES iterations of each system, scaled
    to the iteration counts of a converged solve.  Returns (seconds per solve,
    description)."""
    import oracle
    x, y, z, q, offs, depth, c, nsolve = make_problem(workload, seed)
    if offs is not None:
        return oracle_batch_sample(workload, x, y, z, q, offs, depth, c)
    o = oracle.Oracle(max_depth=depth, c_refine=c)
    t = {}
    t0 = time.perf_counter(); o.build(x, y, z); t["build"] = time.perf_counter() - t0
    t0 = time.perf_counter(); o.stencils(); t["stencils"] = time.perf_counter() - t0
    t0 = time.perf_counter(); rhs, _, _ = o.density_rhs(q); t["deposit"] = time.perf_counter() - t0
    # without a GPU measurement: GMRES(30) + Jacobi needed 3176-3393 iterations on this
    # workload in FP64 on GB300 (8 for the density system)
    it_r, it_p = gmres_iters_hint or (8, 3300)
    t0 = time.perf_counter()
    rho, k_r, _, _ = o.solve_density(rhs, rtol=RTOL, max_iter=min(gmres_sample, it_r))
    t_r = time.perf_counter() - t0
    t0 = time.perf_counter()
    phi, k_p, _, _ = o.solve_poisson(rho, rtol=RTOL, max_iter=gmres_sample)
    t_p = time.perf_counter() - t0
    t["solve_rho"] = t_r / max(k_r, 1) * it_r
    t["solve_phi"] = t_p / max(k_p, 1) * it_p
    t0 = time.perf_counter(); o.gather(phi); t["gather"] = time.perf_counter() - t0
    total = sum(t.values())
    desc = ("oracle on %s seed %d: tree, stencils, deposit and gather in full; %d+%d GMRES iterations timed and "
            "scaled to %d+%d (a converged solve)" % (workload, seed, k_r, k_p, it_r, it_p))
    return total, desc, {k: round(v, 3) for k, v in t.items()}


def oracle_batch_sample(workload, x, y, z, q, offs, depth, c, n_sample=3):
    """Batch workload: full oracle solves (GMRES to convergence) of the
    n_sample smallest beams, scaled to the whole batch by particle count.  The
    oracle's cost grows faster than the particle count (more nodes need more
    iterations), so this underestimates its time on the larger beams."""
    import oracle
    sizes = np.diff(offs)
    pick = np.argsort(sizes, kind="stable")[:n_sample]
    t = {"build": 0.0, "stencils": 0.0, "deposit": 0.0, "solve_rho": 0.0, "solve_phi": 0.0, "gather": 0.0}
    for b in pick:
        s, e = offs[b], offs[b + 1]
        o = oracle.Oracle(max_depth=depth, c_refine=c)
        bx, by, bz, bq = (np.ascontiguousarray(a[s:e]) for a in (x, y, z, q))
        t0 = time.perf_counter(); o.build(bx, by, bz); t["build"] += time.perf_counter() - t0
        t0 = time.perf_counter(); o.stencils(); t["stencils"] += time.perf_counter() - t0
        t0 = time.perf_counter(); rhs, _, _ = o.density_rhs(bq); t["deposit"] += time.perf_counter() - t0
        t0 = time.perf_counter(); rho, _, _, _ = o.solve_density(rhs, rtol=RTOL); t["solve_rho"] += time.perf_counter() - t0
        t0 = time.perf_counter(); phi, _, _, _ = o.solve_poisson(rho, rtol=RTOL); t["solve_phi"] += time.perf_counter() - t0
        t0 = time.perf_counter(); o.gather(phi); t["gather"] += time.perf_counter() - t0
    scale = float(sizes.sum()) / float(sizes[pick].sum())
    total = sum(t.values()) * scale
    desc = ("oracle on %s: full solves of the %d smallest beams (%d particles), scaled by particle count to the "
            "batch's %d particles (%d beams)" % (workload, n_sample, int(sizes[pick].sum()), int(sizes.sum()),
                                                 len(sizes)))
    return total / len(sizes), desc, {k: round(v * scale, 3) for k, v in t.items()}


def run_reference(args, ws, rank):
    if rank != 0:
        return None
    times = []
    for w in range(args.warmup + args.steps):
        tot, desc, stages = oracle_sample(args.workload, gmres_sample=5)
        if w >= args.warmup:
            times.append(tot)
    sec = float(np.mean(times))
    val = 1.0 / sec
    return {"metric": METRIC, "value": round(val, 6), "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(sec * 1e3, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload}, "stage_s": stages,
            "cpu_baseline": {"value": round(val, 6), "unit": "solves/s", "cores": 1, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": round(val, 6), "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_vp(args):
    """Time-dependent workload: leapfrog steps with a full rebuild and solve each
    step (1e7 particles, thermal velocities sigma_v = 0.01, dt = 1e-3), warm
    start from the previous potential.  Reports steps/s, the drift of the total
    (field + kinetic) energy, and a 10-step comparison with the FP64 oracle on
    a bounded sample (2e5 particles of the same law)."""
    import torch

    from paper_1603_04039_gb300 import VlasovPoisson, inputs
    dev = torch.device("cuda", 0)
    npart, depth, c = WORKLOADS["beam_halo_1e7_depth10"]
    x, y, z, q = inputs.beam_with_halo(npart, 1)
    vel = inputs.thermal_velocities(npart, 1, 0.01)
    t = [torch.from_numpy(a).to(dev) for a in (x, y, z) + vel]
    form = dict(max_depth=depth, c_refine=c, precision=args.precision, poly_degree=args.poly_degree,
                poly_omega=args.poly_omega)
    net, t_train = None, 0.0
    if args.learned:
        net, t_train, _ = train_mpnn(args.train_systems)
    vp = VlasovPoisson(*t, qm=1.0, rtol=RTOL, net=net, **form)
    dt = 1e-3
    for _ in range(args.warmup):
        vp.step(dt)
    w0, k0 = vp.energies()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    iters = 0
    for _ in range(args.steps):
        vp.step(dt)
        iters += vp.info["iters_phi"]
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    w1, k1 = vp.energies()
    # bounded oracle comparison: 10 steps on 2e5 particles, GPU vs oracle-driven leapfrog
    import oracle
    ns, ds, cs = 200000, 7, 0.2
    xs, ys, zs, _ = inputs.beam_with_halo(ns, 2)
    vs = inputs.thermal_velocities(ns, 2, 0.01)
    ts = [torch.from_numpy(a.copy()).to(dev) for a in (xs, ys, zs) + vs]
    vps = VlasovPoisson(*ts, qm=1.0, rtol=RTOL, max_depth=ds, c_refine=cs, precision=args.precision,
                        poly_degree=args.poly_degree, poly_omega=args.poly_omega)
    ws_gpu = [vps.energies()[0]]
    for _ in range(10):
        vps.step(dt)
        ws_gpu.append(vps.energies()[0])
    px, py, pz, pvx, pvy, pvz = (a.copy() for a in (xs, ys, zs) + vs)

    def oracle_field():
        o = oracle.Oracle(max_depth=ds, c_refine=cs)
        r = o.run(px, py, pz, q_uniform=1.0 / ns, rtol=RTOL)
        h = 2.0 / 2.0 ** o.nodes()["level"][: o.n_int].astype(float)
        return (r["ex"], r["ey"], r["ez"]), 0.5 * float(((r["dphi"][:, :3] ** 2).sum(1) * h ** 3).sum())

    t_or = time.perf_counter()
    E, w = oracle_field()
    ws_ref = [w]
    for _ in range(10):                       # velocity Verlet, specular walls
        for v, e in zip((pvx, pvy, pvz), E):
            v += 0.5 * dt * e
        for p_, v in zip((px, py, pz), (pvx, pvy, pvz)):
            p_ += dt * v
            hi, lo = p_ > 1.0, p_ < -1.0
            p_[hi] = 2.0 - p_[hi]; v[hi] = -v[hi]
            p_[lo] = -2.0 - p_[lo]; v[lo] = -v[lo]
        E, w = oracle_field()
        ws_ref.append(w)
        for v, e in zip((pvx, pvy, pvz), E):
            v += 0.5 * dt * e
    t_or = time.perf_counter() - t_or
    dw = np.max(np.abs(np.array(ws_gpu) - np.array(ws_ref)) / np.abs(ws_ref))
    return {"metric": "Vlasov-Poisson leapfrog steps/sec (rebuild + solve every step)",
            "value": round(args.steps / el, 4), "unit": "steps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1e3 * el / args.steps, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
            "data": "synthetic",
            "config": {"workload": "vp_beam_halo_1e7_depth10", "particles": npart, "dt": dt, "sigma_v": 0.01,
                       "precision": args.precision, "poly_degree": args.poly_degree,
                       "learned_preconditioner": (None if net is None else
                                                  {"train_systems": args.train_systems, "use": "column scaling",
                                                   "train_seconds": round(t_train, 1)}),
                       "mean_gmres_iters": iters / args.steps},
            "energy": {"field_start": w0, "kinetic_start": k0, "field_end": w1, "kinetic_end": k1,
                       "total_drift_rel": (w1 + k1 - w0 - k0) / (w0 + k0)},
            "oracle_10_steps": {"particles": ns, "max_rel_field_energy_diff": float(dw),
                                "oracle_seconds": round(t_or, 1)}}


TRAIN_SIZES = ((20000, 6, 0.3), (100000, 8, 0.15))


def train_mpnn(n_systems, seed0=10000, lr=2e-3, net_seed=7):
    """Trains the learned preconditioner on the GPU: one Adam step on each of
    n_systems fresh systems from the beam-with-halo law (seeds seed0, seed0 +
    1, ...), alternating 2e4 particles at depth 6 and 1e5 at depth 8.
    Returns the network, seconds spent and the loss curve."""
    import torch
    from paper_1603_04039_gb300 import APCloud, MPNN, inputs
    dev = torch.device("cuda", 0)
    net = MPNN(seed=net_seed)
    aps = [APCloud(max_depth=d, c_refine=cc, device=dev) for _, d, cc in TRAIN_SIZES]
    curve = []
    t0 = time.perf_counter()
    for k in range(n_systems):
        npart = TRAIN_SIZES[k % len(TRAIN_SIZES)][0]
        ap = aps[k % len(TRAIN_SIZES)]
        x, y, z, q = inputs.beam_with_halo(npart, seed0 + k)
        tx, ty, tz, tq = (torch.from_numpy(a).to(dev) for a in (x, y, z, q))
        ap.build_octree(tx, ty, tz)
        ap.stencils()
        ap.deposit(q=tq, rtol=1e-10)
        lo = net.loss(ap, backward=True)
        net.adam(ap, lr=lr)
        if k % max(1, n_systems // 20) == 0 or k == n_systems - 1:
            curve.append((k, round(lo["L"], 5), round(lo["Lp"], 5), round(lo["Lg"], 5)))
    return net, time.perf_counter() - t0, curve


def run_learned(args):
    """Learned preconditioner: trained on the GPU on args.train_systems
    beam-with-halo systems, evaluated on held-out seeds of the 1e7-particle
    depth-10 workload: GMRES iterations and solve time to rtol 1e-10 with
    Jacobi alone, with the network's column scaling (and guess), and with the
    closed-form diagonal of the same objective, in the plain FP64 form; and
    in the mixed form with the degree-16 polynomial."""
    import torch
    from paper_1603_04039_gb300 import APCloud, inputs
    dev = torch.device("cuda", 0)
    net, t_train, curve = train_mpnn(args.train_systems)
    npart, depth, c = WORKLOADS["beam_halo_1e7_depth10"]
    forms = {"fp64_jacobi": (dict(precision="fp64", poly_degree=1), (1, 3, 4)),
             "mixed_poly16": (dict(precision="mixed", poly_degree=16, poly_omega=1.0), (1, 2, 4))}
    names = {0: "jacobi", 1: "learned_scaling", 2: "learned_guess", 3: "learned_scaling_guess",
             4: "closed_form_scaling"}
    rows = []
    for seed in args.eval_seeds:
        x, y, z, q = inputs.beam_with_halo(npart, seed)
        tx, ty, tz, tq = (torch.from_numpy(a).to(dev) for a in (x, y, z, q))
        for fname, (form, uses) in forms.items():
            ap = APCloud(max_depth=depth, c_refine=c, device=dev, **form)
            ap.build_octree(tx, ty, tz)
            ap.stencils()
            ap.deposit(q=tq, rtol=RTOL, max_iter=MAX_ITER)
            lo = net.loss(ap)
            res = {}
            for use in (0,) + uses:
                best = None
                for rep in range(2):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(ap.stream)
                    phi, info = ap.solve_learned(net, use=use, rtol=RTOL, max_iter=args.learned_max_iter)
                    e1.record(ap.stream)
                    torch.cuda.synchronize()
                    ms = e0.elapsed_time(e1)
                    best = ms if best is None else min(best, ms)
                res[names[use]] = {"iters": info["iters"], "ms": round(best, 2), "relres": info["relres"],
                                   "status": info["status"], "phi": phi}
            ref = res["jacobi"]["phi"]
            for r in res.values():
                r["rel_l2_phi_vs_jacobi"] = float(torch.linalg.norm(r.pop("phi") - ref) / torch.linalg.norm(ref))
                r["speedup"] = round(res["jacobi"]["ms"] / r["ms"], 3)
            rows.append({"seed": seed, "form": fname, "n_nodes": ap.n_nodes, "loss_learned": lo, **res})
            ap.close()
    mx = [r for r in rows if r["form"] == "mixed_poly16"]
    speed = float(np.mean([r["learned_scaling"]["speedup"] for r in mx]))
    return {"metric": "Poisson solve time to rtol 1e-10 on held-out seeds, without / with the learned column "
                      "scaling (mixed form, polynomial degree 16)",
            "value": round(speed, 3), "unit": "x", "n_gpus": 1, "steps": len(args.eval_seeds), "warmup": 1,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16+f64",
            "data": "synthetic",
            "config": {"workload": "learned_preconditioner_beam_halo_1e7_depth10", "train_systems": args.train_systems,
                       "train_law": "beam with halo, alternating 2e4 particles depth 6 c 0.3 and 1e5 "
                                    "particles depth 8 c 0.15, seeds 10000..",
                       "eval_seeds": args.eval_seeds, "net": "3 x 64 message passing, BF16 tcgen05 layers",
                       "ilu0": "bench.py --ilu (same seeds)"},
            "train_seconds": round(t_train, 1), "loss_curve": curve, "eval": rows}


def run_ilu(args):
    """ILU(0) against Jacobi on the held-out seeds of the learned-preconditioner
    comparison (1e7-particle depth-10 workload, FP64 GMRES(30), rtol 1e-10).
    The Jacobi solve of the deposited system gives phi; both preconditioners
    then solve A x = A phi (the same operator and, up to the solve tolerance,
    the same right-hand side) from zero."""
    import torch
    from paper_1603_04039_gb300 import APCloud, inputs
    dev = torch.device("cuda", 0)
    npart, depth, c = WORKLOADS["beam_halo_1e7_depth10"]
    rows = []

    def timed(f):
        best, out = None, None
        for rep in range(2):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(ap.stream)
            out = f()
            e1.record(ap.stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        return out, best

    for seed in args.eval_seeds:
        x, y, z, q = inputs.beam_with_halo(npart, seed)
        tx, ty, tz, tq = (torch.from_numpy(a).to(dev) for a in (x, y, z, q))
        ap = APCloud(max_depth=depth, c_refine=c, device=dev, precision="fp64", poly_degree=1)
        ap.build_octree(tx, ty, tz)
        ap.stencils()
        ap.deposit(q=tq, rtol=RTOL, max_iter=MAX_ITER)
        phi, _ = ap.solve(rtol=RTOL, max_iter=MAX_ITER)
        b = ap.matvec("A", phi)
        (xj, ij), msj = timed(lambda: ap.solve_system("A", b, rtol=RTOL, max_iter=MAX_ITER))
        (xi, ii), msi = timed(lambda: ap.solve_system_ilu0("A", b, rtol=RTOL, max_iter=args.ilu_max_iter))
        rows.append({"seed": seed, "n_nodes": ap.n_nodes,
                     "jacobi": {"iters": ij["iters"], "ms": round(msj, 2), "relres": ij["relres"],
                                "status": ij["status"]},
                     "ilu0": {"iters": ii["iters"], "ms": round(msi, 2), "relres": ii["relres"], "status": ii["status"],
                              "host_setup_ms": round(ii["setup_ms"], 1), "levels_lower": ii["levels_lower"],
                              "levels_upper": ii["levels_upper"], "nnz": ii["nnz"],
                              "rel_l2_x_vs_jacobi": float(torch.linalg.norm(xi - xj) / torch.linalg.norm(xj))}})
        ap.close()
    speed = float(np.mean([r["jacobi"]["ms"] / r["ilu0"]["ms"] for r in rows]))
    return {"metric": "Poisson solve time to rtol 1e-10 on held-out seeds, ILU(0) against Jacobi (FP64 GMRES(30))",
            "value": round(speed, 3), "unit": "x", "n_gpus": 1, "steps": len(args.eval_seeds), "warmup": 1,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "ilu0_beam_halo_1e7_depth10", "eval_seeds": args.eval_seeds,
                       "ilu0": "factorised on the host, level-scheduled triangular sweeps on the GPU"},
            "eval": rows}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="beam_halo_1e7_depth10", choices=sorted(WORKLOADS) + sorted(BATCH_WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--poly-degree", type=int, default=16, help="1 = Jacobi")
    ap.add_argument("--poly-omega", type=float, default=1.0)
    ap.add_argument("--vp", action="store_true", help="Vlasov-Poisson leapfrog workload instead of single solves")
    ap.add_argument("--learned", action="store_true",
                    help="train the learned preconditioner and compare it with Jacobi on held-out seeds "
                         "(with --vp: use its column scaling in the leapfrog solves)")
    ap.add_argument("--train-systems", type=int, default=10000)
    ap.add_argument("--eval-seeds", type=int, nargs="+", default=[90001, 90002])
    ap.add_argument("--learned-max-iter", type=int, default=100000)
    ap.add_argument("--ilu", action="store_true", help="ILU(0) against Jacobi on the learned comparison's seeds")
    ap.add_argument("--ilu-max-iter", type=int, default=3000)
    args = ap.parse_args()
    if args.vp:
        print(json.dumps(run_vp(args)))
        return
    if args.learned:
        print(json.dumps(run_learned(args)))
        return
    if args.ilu:
        print(json.dumps(run_ilu(args)))
        return
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    ws, rank, local = _dist()
    if ws != args.gpus and ws > 1:
        print("warning: --gpus %d but WORLD_SIZE %d" % (args.gpus, ws), file=sys.stderr)
    if args.impl == "reference":
        line = run_reference(args, ws, rank)
        if line is not None:
            print(json.dumps(line))
        return
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    line = run_ours(args, ws, rank, local)
    if rank == 0:
        if ws == 1 and not args.no_cpu_baseline:
            # the oracle runs GMRES(30) + Jacobi: scale its sampled iterations to the
            # count that algorithm needs on this workload (measured above in FP64 on the GPU)
            pl = line["plain_fp64_form"]
            tot, desc, stages = oracle_sample(args.workload, gmres_sample=10,
                                              gmres_iters_hint=(pl["iters_rho"], pl["iters_phi"]))
            line["cpu_baseline"] = {"value": round(1.0 / tot, 6), "unit": "solves/s", "cores": 1, "kind": "oracle",
                                    "sample": desc, "stage_s": stages}
        else:
            line["cpu_baseline"] = None
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
