"""Benchmark: input Mfaces/s simplified to the target face count.

Workload: the bumped level-8 icosphere (1,310,720 faces, 32 seeded Gaussian
bumps) simplified to 1 % (13,107 faces) -- a synthetic stand-in with the
paper's scale for its Thingi10K meshes.  One step = one full simplification
(Algorithm 1 from the input mesh to the target) through the C ABI.

  value   device-resident input, CUDA events per step on the launching
          stream, L2 flushed (256 MiB write) between steps outside the timing;
          each step one plain pamo_simplify call (one graph replay per round)
  e2e     the same call with host buffers (pamo_simplify_host): host->device
          copy of the input and device->host copy of the output inside timing
  roofline  the class of the dominant kernel (k_traverse, the check):
          algorithmic bytes / its CUDA-event time per launch, from as many
          profiled steps right after the timed ones; class_share gives every
          class's share; roofline_cost the same for k_edge_cost (Eq. 1 flops)
  cpu_baseline  the CPU oracle (test infrastructure) on a bounded sample

Multi-GPU: a single mesh does not shard (every round needs global 2-hop
minima and a global intersection check), so N ranks run N independent
replicas (weak scaling, no collective on the data path).
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

METRIC = "input Mfaces/s simplified to target, plain vs batched/learned; % HBM roofline"
WORKLOAD = "bumped_icosphere_l8"
CLASS_NAMES = ("adjacency", "cost", "select", "collapse", "bvh", "query", "commit", "other")


# float64 FMA peak: 152 SMs x 2 FMA/clock/SM x 2 flop x 2.07 GHz (ncu reports a
# float64 FMA peak of 304 thread-instructions per cycle on this GPU;
# pamo_measure_fp64 measures it live next to the division and root rates)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12

# float64 operations of the edge-cost source (Eq. 1): per dirty edge, the
# quadric sum, the 3x3 Cramer solve, the quadric at the placement, the edge
# length and the cost (additions, multiplies, FMAs, min/max and compares: 85,
# plus 3 divisions and 1 square root); per produced triangle, the quality term
# (edge differences, cross product, squared lengths, sums: 32, plus 1 division
# and 1 square root).  The kernel runs the triangle terms as certified
# float-float arithmetic on the float32 pipe; only the edges whose key the
# bound leaves open take them in float64.  Certifying a key costs 8 float64
# operations per edge (4 directed additions, 2 FMAs, 2 conversions).
COST_OPS_EDGE, COST_DIV_EDGE, COST_SQRT_EDGE = 85, 3, 1
COST_OPS_TRI, COST_DIV_TRI, COST_SQRT_TRI = 32, 1, 1
COST_OPS_CERT = 8
# algorithmic flops (FMA = 2, division and root = 1) per dirty edge and per
# produced triangle; the library's class_flops use the same counts
COST_FLOPS_EDGE, COST_FLOPS_TRI = 114.0, 45.0

# k_edge_cost DRAM bytes per evaluated edge, from one ncu capture of the current kernel on
# round 0 of the level-7 sphere (491,520 edges, all evaluated); the traffic of a launch grows
# with the edges it evaluates, so a launch's traffic is this times its edge count.  None
# (traffic reported as null) while no capture of the current kernel exists.
COST_DRAM_BYTES_PER_EDGE = 36.49e6 / 491520
COST_FP64_PIPE_BUSY = 0.610  # same capture
# the kernel the roofline describes: k_traverse has the largest share of the
# ncu launch list of the level-8 run (22.5 %, then k_edge_cost 18 %); its class
# (the check: k_traverse, k_pairs and the small kernels around them) is timed
# with CUDA events.  The cost class (k_edge_reuse + k_edge_cost) is reported
# beside it under roofline_cost.
ROOFLINE_CLASS = "query"


def cost_roofline(c_ms, c_launch, c_flops, cost_edges, cost_f64, fp64):
    """ALU roofline of the cost class (k_edge_reuse + k_edge_cost): the
    algorithmic float64 operations of Eq. 1 for the evaluated edges per launch
    (the method's count; the kernel certifies the triangle terms in
    float-float on the float32 pipe and needs the float64 pipe only for the
    rest, see pipe_model) over the class's CUDA-event time."""
    avg_launch_ms = c_ms / max(c_launch, 1)
    flops_per_launch = c_flops / max(c_launch, 1)
    achieved = flops_per_launch / (avg_launch_ms * 1e-3) / 1e12 if avg_launch_ms > 0 else 0.0
    # two launches per round in this class (reuse + cost): edges per k_edge_cost launch
    edges_per_launch = cost_edges / max(c_launch / 2, 1)
    f64_edges_per_launch = cost_f64 / max(c_launch / 2, 1)
    # produced triangles per launch, from the flop model
    flops_cost = flops_per_launch * 2  # the reuse launch has no flops
    tris_per_launch = max(flops_cost - COST_FLOPS_EDGE * edges_per_launch, 0.0) / COST_FLOPS_TRI
    f64_tris_per_launch = tris_per_launch * f64_edges_per_launch / max(edges_per_launch, 1e-9)
    # peak: the float64 FMA rate measured on this GPU just before the timed
    # region (independent FMA chains over one full wave); the nominal figure
    # from the unit count and clock when no measurement exists
    if fp64 is not None:
        peak = 2 * fp64["fma_per_s"] / 1e12
        peak_source = "measured live: pamo_measure_fp64, independent float64 FMA chains"
    else:
        peak, peak_source = FP64_PEAK_TFLOPS, "derived: float64 FMA units x clock"
    roof = {"bound": "alu", "kernel_class": "cost", "kernel": "k_edge_cost",
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "achieved_note": ("Eq. 1 float64 operations per second; the triangle terms run "
                              "as certified float-float on the float32 pipe"),
            "traffic": (COST_DRAM_BYTES_PER_EDGE * edges_per_launch
                        if COST_DRAM_BYTES_PER_EDGE else None),
            "traffic_note": "ncu DRAM bytes per edge (L7 round-0 capture) x edges per launch",
            "ncu_fp64_pipe_busy": COST_FP64_PIPE_BUSY,
            "peak_source": peak_source, "peak_nominal": FP64_PEAK_TFLOPS,
            "launch_ms": avg_launch_ms}
    if fp64 is not None:
        # the float64 pipe time of the float64 operations the kernel still runs
        # (per edge, the certification, and the triangles of the edges the bound
        # left open) at the measured rates, against the event-timed class time
        # of a round (k_edge_reuse + k_edge_cost: two launches)
        t_model = (((COST_OPS_EDGE + COST_OPS_CERT) * edges_per_launch
                    + COST_OPS_TRI * f64_tris_per_launch) / fp64["fma_per_s"]
                   + (COST_DIV_EDGE * edges_per_launch + COST_DIV_TRI * f64_tris_per_launch)
                   / max(fp64["div_per_s"], 1.0)
                   + (COST_SQRT_EDGE * edges_per_launch + COST_SQRT_TRI * f64_tris_per_launch)
                   / max(fp64["sqrt_per_s"], 1.0))
        roof["fp64_measured"] = {"fma_tflops": 2 * fp64["fma_per_s"] / 1e12,
                                 "div_per_s": fp64["div_per_s"],
                                 "sqrt_per_s": fp64["sqrt_per_s"]}
        roof["pipe_model"] = {"edges_per_launch": edges_per_launch,
                              "tris_per_launch": tris_per_launch,
                              "f64_fallback_edges_per_launch": f64_edges_per_launch,
                              "model_ms": t_model * 1e3,
                              "frac": t_model * 1e3 / (2 * avg_launch_ms) if avg_launch_ms else 0.0}
    return roof


def max_over_ranks(x, device=None):
    """Max of a float over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(faces_per_rank, world, ms_per_step):
    """Whole-job throughput in Mfaces/s: every rank simplifies its own replica,
    the job takes as long as the slowest rank."""
    return world * faces_per_rank / (ms_per_step * 1e-3) / 1e6


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) > 8 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 8 and r[2].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for r in self.rows if len(r) > 8
                          for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(sm)}


def make_workload(level=8):
    import meshgen
    cache = os.environ.get("PAMO_BENCH_CACHE", f"/tmp/pamo_bench_l{level}.npz")
    if os.path.exists(cache):
        d = np.load(cache)
        return d["V"], d["F"], int(d["target"])
    if level == 8:
        V, F, target = meshgen.mesh_config(WORKLOAD)
    else:
        V, F = meshgen.bumped_icosphere(level, 0)
        target = len(F) // 100
    try:
        np.savez(cache, V=V, F=F, target=target)
    except OSError:
        pass
    return V, F, target


def host_cpu():
    """Model name (lscpu) and core count of the host the oracle runs on."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    try:
        nproc = len(os.sched_getaffinity(0))
    except Exception:
        nproc = os.cpu_count()
    return {"cpu_model": model, "nproc": nproc}


def _oracle_run(level, config=None):
    """One oracle simplification (single-threaded); returns (seconds, faces in,
    faces out, rounds).  level: icosphere level of the benchmark mesh, or
    config: a named input recipe."""
    import meshgen
    import oracle
    if config is not None:
        V, F, target = meshgen.mesh_config(config)
    else:
        V, F, target = make_workload(level)
    t = time.perf_counter()
    r = oracle.simplify(V, F, target, keep_pairs=False)
    return time.perf_counter() - t, len(F), len(r.F), len(r.rounds)


def cpu_oracle_sample(level=8):
    """The oracle (as it stands) on the benchmark workload itself: one
    simplification of the level-8 sphere to 1 %, single-threaded."""
    dt, nf, nout, rounds = _oracle_run(level)
    return {"value": nf / dt / 1e6, "unit": "Mfaces/s", "cores": 1, "kind": "oracle",
            "sample": f"the benchmark workload itself: bumped icosphere level {level} ({nf} "
                      f"faces) -> {nout} faces, {rounds} rounds in {dt:.1f} s, one thread",
            **host_cpu()}


def run_reference(args, rank, world):
    """The oracle as the reference arm: every step is one full simplification
    of the benchmark workload (level-8 sphere to 1 %), single-threaded; the
    steps run side by side in worker processes, one per host core, and the
    value is the steps' faces over the wall time of all of them.  Warm-up
    steps (untimed) load the library in every worker on the level-6 sphere."""
    if rank != 0:
        return
    import multiprocessing as mp
    import oracle  # noqa: F401  (build happens on import)
    level = args.level
    V, F, target = make_workload(level)  # the cached input file the workers read
    cpu = host_cpu()
    procs = max(1, min(cpu["nproc"] or 1, args.steps))
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        pool.map(_oracle_run, [min(level, 6)] * max(args.warmup, procs))
        t0 = time.perf_counter()
        runs = pool.map(_oracle_run, [level] * args.steps, chunksize=1)
        wall = time.perf_counter() - t0
    nf = runs[0][1]
    v = args.steps * nf / wall / 1e6
    per_run = statistics.mean(r[0] for r in runs)
    sample = (f"{args.steps} full simplifications of the benchmark workload (bumped icosphere "
              f"level {level}, {nf} faces -> {runs[0][2]} faces, {runs[0][3]} rounds), one per "
              f"worker process on {procs} host cores, {per_run:.1f} s each on average, "
              f"{wall:.1f} s wall")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Mfaces/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": wall / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(level), "faces_in": int(nf),
                       "target": int(target), "faces_out": int(runs[0][2]),
                       "rounds": int(runs[0][3]),
                       "parallelism": f"one simplification per host core x{procs}"},
            "cpu_baseline": {"kind": "oracle", "cores": procs, "sample": sample, "value": v,
                             **cpu},
            "e2e": {"value": v, "unit": "Mfaces/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    if level == 8:
        # the near-contact configuration (nested shells level 8 to 0.1 %), once, end to end
        dt3, nf3, nout3, rounds3 = _oracle_run(None, "nested_shells_l8")
        line["oracle_nested_shells_l8"] = {
            "value": nf3 / dt3 / 1e6, "unit": "Mfaces/s", "seconds": round(dt3, 1), "cores": 1,
            "extrapolated": False,
            "sample": f"nested shells level 8 ({nf3} faces) -> {nout3} faces, {rounds3} rounds, "
                      "end to end"}
    print(json.dumps(line), flush=True)


def workload_name(level):
    return WORKLOAD if level == 8 else f"bumped_icosphere_l{level}"


def min_angles_deg(V, F):
    """Smallest interior angle of every triangle, in degrees (float64)."""
    P = np.asarray(V, np.float64)[np.asarray(F)]
    out = np.full(len(F), 180.0)
    for i in range(3):
        u = P[:, (i + 1) % 3] - P[:, i]
        w = P[:, (i + 2) % 3] - P[:, i]
        den = np.linalg.norm(u, axis=1) * np.linalg.norm(w, axis=1)
        cos = np.einsum("ij,ij->i", u, w) / np.where(den > 0, den, 1.0)
        ang = np.degrees(np.arccos(np.clip(cos, -1.0, 1.0)))
        out = np.minimum(out, np.where(den > 0, ang, 0.0))
    return out


ABLATION = {"full": (0.001, 0.005), "no_ce": (0.0, 0.005), "no_cs": (0.001, 0.0),
            "no_ce_cs": (0.0, 0.0)}
ALPHAS = (10.0, 5.0, 1.0)


def run_ablation(args):
    """Edge-cost ablation (the paper's bad-triangle study): each Eq. 1 term
    switched off in turn, bad-triangle ratio (min angle below 10/5/1 degrees)
    of the output on synthetic meshes, on the GPU path."""
    import torch
    import meshgen
    import paper_2509_05595_gb300 as pamo
    cases = []
    Vb, Fb = meshgen.box_grid(32)
    cases.append(("box_grid_32 to 10%", Vb, Fb, len(Fb) // 10))
    Vt, Ft = meshgen.torus()
    cases.append(("torus_64x32 to 10%", Vt, Ft, len(Ft) // 10))
    Vs, Fs = meshgen.bumped_icosphere(7, 0)
    cases.append(("bumped_icosphere_l7 to 1%", Vs, Fs, len(Fs) // 100))
    res = {}
    for name, V, F, target in cases:
        Vd, Fd = torch.from_numpy(V).cuda(), torch.from_numpy(F).cuda()
        res[name] = {}
        for var, (w_e, w_s) in ABLATION.items():
            opts = pamo.Options(w_e=w_e, w_s=w_s, validate_input=0)
            pamo.pamo_simplify(Vd, Fd, target, options=opts)  # warm-up
            Vo, Fo, st, status = pamo.pamo_simplify(Vd, Fd, target, options=opts)
            m = min_angles_deg(Vo.cpu().numpy(), Fo.cpu().numpy())
            res[name][var] = {"bad_pct": [round(100.0 * float((m < a).mean()), 3) for a in ALPHAS],
                              "faces_out": int(len(Fo)), "status": status,
                              "rounds": st["rounds"], "ms": round(st["ms_total"], 3)}
    print(json.dumps({"ablation": "edge_cost_terms", "alpha_deg": list(ALPHAS),
                      "data": "synthetic", "cases": res}), flush=True)


def make_batch(count=256):
    """The batch workload: seeded tori (r ~ U(0.2, 0.5)) and bumped icospheres
    with log-uniform face counts in [2k, 500k], each simplified to 1 %."""
    import meshgen
    import paper_2509_05595_gb300 as pamo
    cache = os.environ.get("PAMO_BATCH_CACHE", f"/tmp/pamo_batch_{count}.npz")
    if os.path.exists(cache):
        d = np.load(cache)
        return d["V"], d["voff"], d["F"], d["foff"], d["targets"]
    meshes = meshgen.batch_meshes(count=count)
    V, voff, F, foff = pamo.concat_meshes(meshes)
    targets = np.array([len(f) // 100 for _, f in meshes], np.int64)
    try:
        np.savez(cache, V=V, voff=voff, F=F, foff=foff, targets=targets)
    except OSError:
        pass
    return V, voff, F, foff, targets


def run_batch_bench(args, world, rank, emit=True):
    """Many meshes per pass: the batched path against the same meshes run one
    call at a time through the plain path (both device-resident, CUDA events).
    emit=False returns the line instead of printing it."""
    import torch
    import paper_2509_05595_gb300 as pamo
    V, voff, F, foff, targets = make_batch(args.batch_count)
    M = len(targets)
    Vd, Fd = torch.from_numpy(V).cuda(), torch.from_numpy(F).cuda()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    base = pamo.Options(validate_input=0)
    # the project's autotuner picks the speed-only knobs on this batch
    opts, trials = pamo.pamo_autotune_batch(Vd, voff, Fd, foff, targets, options=base)
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()  # before the warm-up, as in the plain bench
    for _ in range(args.warmup):
        pamo.pamo_simplify_batch(Vd, voff, Fd, foff, targets, options=opts)
    torch.cuda.synchronize()
    times, launches = [], 0
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        Vo, vo, Fo, fo, status, rounds, st = pamo.pamo_simplify_batch(Vd, voff, Fd, foff, targets,
                                                                      options=opts)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        launches += st["launches"]
    clk = clocks.stop()
    ms = max_over_ranks(sum(times), device="cuda") / args.steps
    value = weak_value(len(F), world, ms)
    # the same meshes one call at a time (plain path), one timed pass
    views = [(Vd[voff[m]:voff[m + 1]], Fd[foff[m]:foff[m + 1]]) for m in range(M)]
    for m in range(min(M, 8)):
        pamo.pamo_simplify(views[m][0], views[m][1], int(targets[m]), options=opts)
    flush.fill_(1)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for m in range(M):
        pamo.pamo_simplify(views[m][0], views[m][1], int(targets[m]), options=opts)
    e1.record(stream)
    e1.synchronize()
    seq_ms = e0.elapsed_time(e1)
    line = {"metric": METRIC, "value": value, "unit": "Mfaces/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"batch_{M}: seeded tori and bumped icospheres, "
                                   "log-uniform 2k-500k faces, each to 1%",
                       "meshes": M, "faces_in": int(len(F)), "faces_out": int(fo[-1]),
                       "stalled": int(sum(s != "PAMO_OK" for s in status)),
                       "rounds_max": int(max(rounds)), "batch_rounds": st["rounds"],
                       "l2": "flushed between steps (256 MiB write, outside the timed span)",
                       "parallelism": f"replicas x{world}"},
            "plain_one_at_a_time": {"value": len(F) / (seq_ms * 1e-3) / 1e6, "unit": "Mfaces/s",
                                    "ms": seq_ms},
            "speedup_vs_plain": seq_ms / ms,
            "autotune": {"resort_percent": opts.resort_percent,
                         "grid_blocks_per_sm": opts.grid_blocks_per_sm,
                         "trials_ms": [round(t, 2) for t in trials],
                         "trials": "resort 25/50/75/100 at 6 blocks/SM, then 4 and 8 blocks/SM"},
            "clocks": clk,
            "gpu_launches": int(launches)}
    if rank == 0 and emit:
        print(json.dumps(line), flush=True)
    return line


def one_sided_hausdorff(Vo, Fo, V, F, k=16, tree=None, T=None):
    """max over the output's vertices and face centroids of the distance to
    the input surface (exact point-to-triangle distance to the k input faces
    whose centroids are nearest; float64).  tree, T: a kd-tree of the input's
    face centroids and its corner array, built once by the caller."""
    from scipy.spatial import cKDTree
    Vo = np.asarray(Vo, np.float64)
    Q = np.concatenate([Vo, Vo[np.asarray(Fo)].mean(1)])
    if T is None:
        T = np.asarray(V, np.float64)[np.asarray(F)]
    if tree is None:
        tree = cKDTree(T.mean(1))
    _, cand = tree.query(Q, k=min(k, len(T)))
    A, B, C = T[cand, 0], T[cand, 1], T[cand, 2]
    P = Q[:, None, :]
    # closest point on triangle (Ericson, Real-Time Collision Detection, 5.1.5)
    ab, ac, ap = B - A, C - A, P - A
    d1, d2 = (ab * ap).sum(-1), (ac * ap).sum(-1)
    bp = P - B
    d3, d4 = (ab * bp).sum(-1), (ac * bp).sum(-1)
    cp = P - C
    d5, d6 = (ab * cp).sum(-1), (ac * cp).sum(-1)
    va, vb, vc = d3 * d6 - d5 * d4, d5 * d2 - d1 * d6, d1 * d4 - d3 * d2
    den = np.where(va + vb + vc == 0, 1.0, va + vb + vc)
    v, w = vb / den, vc / den
    X = A + ab * v[..., None] + ac * w[..., None]
    def put(mask, val):
        X[mask] = val[mask]
    e_ab = (vc <= 0) & (d1 >= 0) & (d3 <= 0)
    t = d1 / np.where(d1 - d3 == 0, 1.0, d1 - d3)
    put(e_ab, A + ab * t[..., None])
    e_ac = (vb <= 0) & (d2 >= 0) & (d6 <= 0)
    t = d2 / np.where(d2 - d6 == 0, 1.0, d2 - d6)
    put(e_ac, A + ac * t[..., None])
    e_bc = (va <= 0) & ((d4 - d3) >= 0) & ((d5 - d6) >= 0)
    t = (d4 - d3) / np.where((d4 - d3) + (d5 - d6) == 0, 1.0, (d4 - d3) + (d5 - d6))
    put(e_bc, B + (C - B) * t[..., None])
    put((d1 <= 0) & (d2 <= 0), A)
    put((d3 >= 0) & (d4 <= d3), B)
    put((d6 >= 0) & (d5 <= d6), C)
    dist = np.linalg.norm(X - P, axis=-1).min(1)
    return float(dist.max())


def _shells_vertices(args):
    """Worker: the vertices of one near-contact mesh (the faces are the same
    for every seed of a level)."""
    import meshgen
    level, seed = args
    V, _ = meshgen.nested_shells_seeded(level, seed)
    return V


def _shells_stream(level, seeds, procs):
    """(seed, V, F) for each seed, generated by `procs` worker processes."""
    import multiprocessing as mp
    import meshgen
    _, F = meshgen.nested_shells(level, check=False)  # shared connectivity
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        for seed, V in zip(seeds, pool.imap(_shells_vertices, [(level, s) for s in seeds])):
            yield seed, V, F


class _Hausdorff:
    """One-sided Hausdorff distance of outputs to one input mesh (kd-tree of
    the input's face centroids built once, reused for every arm)."""

    def __init__(self, V, F):
        from scipy.spatial import cKDTree
        self.V = np.asarray(V, np.float64)
        self.T = self.V[np.asarray(F)]
        self.tree = cKDTree(self.T.mean(1))

    def __call__(self, Vo, Fo):
        return one_sided_hausdorff(Vo, Fo, self.V, None, tree=self.tree, T=self.T)


def run_learned_bench(args, world, rank):
    """The learned proposal against the plain method, and the bound on any
    such proposal: labels logged by the plain method on the near-contact
    family (nested shells, seeds 1000..), negatives subsampled, the network
    trained by the library's kernels; then, on held-out seeds (2000..), the
    plain method, the perfect predictor (deferring exactly the winners the
    plain run undid: the plain output with no undo iteration) and the network
    at several thresholds: Mfaces/s, undo work, faces, self-intersections and
    the one-sided Hausdorff distance to the input."""
    import torch
    import paper_2509_05595_gb300 as pamo
    from paper_2509_05595_gb300 import proposal
    procs = max(1, min(16, (host_cpu()["nproc"] or 2) - 1))
    rng = np.random.default_rng(12345)
    t0 = time.perf_counter()
    Xs, ys, n_all, n_pos = [], [], 0, 0
    for seed, V, F in _shells_stream(args.train_level, range(1000, 1000 + args.train_meshes),
                                     procs):
        X, y = proposal.log_winners(V, F, len(F) // 100)
        n_all += len(y)
        n_pos += int(y.sum().item())
        # every undone winner, a fixed fraction of the standing ones
        keep = (y > 0.5) | torch.as_tensor(rng.random(len(y)) < args.neg_rate, device=y.device)
        Xs.append(X[keep])
        ys.append(y[keep])
    X, y = torch.cat(Xs), torch.cat(ys)
    del Xs, ys
    t_log = time.perf_counter() - t0
    t0 = time.perf_counter()
    # negatives subsampled at rate r: positives weigh r so the probabilities
    # stay calibrated (a threshold is a probability of an undo)
    model, info = proposal.train(X, y, steps=args.train_steps, batch=8192, lr=2e-3,
                                 pos_weight=args.neg_rate,
                                 log_every=max(1, args.train_steps // 10))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    thresholds = [float(t) for t in args.thresholds.split(",")]
    arms = ["plain", "ceiling"] + [f"learned@{t:g}" for t in thresholds]
    res = {name: [] for name in arms}

    def timed_run(make, target):
        """One simplification on a context from make() (created, and for the
        perfect predictor given its schedule, outside the timed span): CUDA
        events around Ctx.run only, after one warm-up run."""
        for _ in range(2):
            c = make()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st, status = c.run(target)
            e1.record(stream)
            e1.synchronize()
            Vo, Fo = c.export()
            c.close()
        return e0.elapsed_time(e1), (Vo, Fo, st, status)

    from tests.meshcheck import is_closed_manifold
    for seed, V, F in _shells_stream(args.eval_level, range(2000, 2000 + args.eval_meshes), procs):
        Vd, Fd = torch.from_numpy(V).cuda(), torch.from_numpy(F).cuda()
        target = len(F) // 100
        hd = _Hausdorff(V, F)
        # the plain run's undone pairs per round: the perfect predictor's schedule
        rc = pamo.Ctx(Vd, Fd, validate_input=0, record_rounds=1)
        rc.run(target)
        undone = [rc.round_pairs(r, 2) for r in range(rc.rounds()[0])]
        rc.close()

        def ceiling_ctx():
            c = pamo.Ctx(Vd, Fd, validate_input=0)
            c.set_deferrals(undone)
            return c

        for name in arms:
            if name == "plain":
                make = lambda: pamo.Ctx(Vd, Fd, validate_input=0)  # noqa: E731
            elif name == "ceiling":
                make = ceiling_ctx
            else:
                thr = float(name.split("@")[1])
                make = lambda thr=thr: pamo.Ctx(  # noqa: E731
                    Vd, Fd, validate_input=0, proposal=model, proposal_threshold=thr)
            ms, (Vo, Fo, st, status) = timed_run(make, target)
            nint, _ = pamo.pamo_check_self_intersections(Vo, Fo)
            Vh, Fh = Vo.cpu().numpy(), Fo.cpu().numpy()
            res[name].append(dict(ms=ms, faces_in=len(F), faces=len(Fh), status=status,
                                  rounds=st["rounds"], undone=st["undone"] - st["deferred"],
                                  deferred=st["deferred"],
                                  undo_iters=sum(i * n for i, n in
                                                 enumerate(st["undo_iters_hist"])),
                                  intersections=int(nint),
                                  manifold=bool(is_closed_manifold(Fh, len(Vh))),
                                  hausdorff=hd(Vh, Fh)))

    def agg(rows):
        ms = sum(r["ms"] for r in rows)
        return {"mfaces_s": sum(r["faces_in"] for r in rows) / (ms * 1e-3) / 1e6, "ms": ms,
                "undo_iters": sum(r["undo_iters"] for r in rows),
                "undone_by_check": sum(r["undone"] for r in rows),
                "deferred": sum(r["deferred"] for r in rows),
                "rounds": sum(r["rounds"] for r in rows),
                "faces_out": sum(r["faces"] for r in rows),
                "stalled": sum(r["status"] != "PAMO_OK" for r in rows),
                "intersections": sum(r["intersections"] for r in rows),
                "manifold": all(r["manifold"] for r in rows),
                "hausdorff_mean": float(np.mean([r["hausdorff"] for r in rows])),
                "hausdorff_max": float(np.max([r["hausdorff"] for r in rows]))}
    summary = {name: agg(rows) for name, rows in res.items()}
    for name in arms[1:]:
        hdr = [l["hausdorff"] / max(p["hausdorff"], 1e-30) for p, l in zip(res["plain"], res[name])]
        summary[name]["hausdorff_ratio_mean"] = float(np.mean(hdr))
        summary[name]["hausdorff_ratio_max"] = float(np.max(hdr))
        summary[name]["speedup_vs_plain"] = summary["plain"]["ms"] / summary[name]["ms"]
    best = max(arms[2:], key=lambda a: summary[a]["mfaces_s"])
    line = {"metric": METRIC, "value": summary[best]["mfaces_s"], "unit": "Mfaces/s",
            "n_gpus": world, "steps": args.eval_meshes, "warmup": 1,
            "ms_per_step": summary[best]["ms"] / args.eval_meshes,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"learned proposal: nested shells L{args.eval_level} "
                                   f"(seeds 2000..{2000 + args.eval_meshes - 1}) to 1%, one "
                                   "context per mesh, the rounds (Ctx.run) timed",
                       "train": f"{args.train_meshes} nested shells L{args.train_level} "
                                f"(seeds 1000..{1000 + args.train_meshes - 1}) to 1%: "
                                f"{n_all} winners logged, {n_pos} undone; all undone and "
                                f"{args.neg_rate:g} of the standing kept ({info['samples']} "
                                f"samples); {args.train_steps} Adam steps",
                       "best_learned_arm": best, "log_s": round(t_log, 1),
                       "train_s": round(t_train, 1),
                       "loss_first_last": [info["losses"][0], info["losses"][-1]]},
            "arms": summary}
    if rank == 0:
        print(json.dumps(line), flush=True)


def host_leg(pamo, torch, V, F, target, steps, world=1, barrier=lambda: None):
    """pamo_simplify_host from pinned host arrays: copies inside the timing.
    Every rank runs its own replica; the whole-job value uses the slowest
    rank's time, like the device-resident value."""
    hV = torch.from_numpy(V).pin_memory().numpy()
    hF = torch.from_numpy(F).pin_memory().numpy()
    for _ in range(2):
        pamo.pamo_simplify_host(hV, hF, target, validate_input=0)
    torch.cuda.synchronize()
    barrier()
    ts = []
    for _ in range(steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Vh, Fh, _, _ = pamo.pamo_simplify_host(hV, hF, target, validate_input=0)
        ts.append(time.perf_counter() - t0)
    barrier()
    # mean of the timed calls, like the device-resident value
    ms = max_over_ranks(sum(ts) / steps * 1e3, device="cuda")
    return {"value": weak_value(len(F), world, ms), "unit": "Mfaces/s",
            "h2d_bytes_per_step": int(V.nbytes + F.nbytes),
            "d2h_bytes_per_step": int(Vh.nbytes + Fh.nbytes)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched leg of the default line")
    ap.add_argument("--train-meshes", type=int, default=512)
    ap.add_argument("--train-level", type=int, default=8)
    ap.add_argument("--train-steps", type=int, default=4000)
    ap.add_argument("--neg-rate", type=float, default=0.05,
                    help="fraction of the standing winners kept as training negatives")
    ap.add_argument("--eval-meshes", type=int, default=64)
    ap.add_argument("--eval-level", type=int, default=8)
    ap.add_argument("--thresholds", default="0.5,0.7,0.9")
    ap.add_argument("--workload", default="plain", choices=["plain", "batch", "learned"],
                    help="plain: the L8 sphere (default); batch: many meshes per pass")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--ablation", action="store_true",
                    help="edge-cost ablation (bad-triangle ratios) instead of the benchmark")
    ap.add_argument("--level", type=int, default=8,
                    help="icosphere level of the workload (8 = the benchmark; smaller "
                         "levels only for profiling captures)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.ablation:
        if rank == 0:
            run_ablation(args)
        return

    import torch
    import torch.distributed as dist
    import paper_2509_05595_gb300 as pamo

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if args.workload in ("batch", "learned"):
        (run_batch_bench if args.workload == "batch" else run_learned_bench)(args, world, rank)
        if world > 1:
            dist.destroy_process_group()
        return
    V, F, target = make_workload(args.level)
    workload = workload_name(args.level)
    Vd = torch.from_numpy(V).cuda()
    Fd = torch.from_numpy(F).cuda()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()

    # rounds and their device times (one recorded run): the latency-bound tail
    rc = pamo.Ctx(Vd, Fd, validate_input=0, record_rounds=1)
    st_rec, _ = rc.run(target)
    n_rounds, _ = rc.rounds()
    per_round = [rc.round_info(r) for r in range(n_rounds)]
    rc.close()
    round_us = [r["us"] for r in per_round]
    tail = [r for r in per_round if r["nF"] < 100000]
    rounds_info = {"rounds": n_rounds, "round0_ms": round_us[0] / 1e3 if round_us else 0.0,
                   # device time of the rounds against the whole recorded run: the rest
                   # is host time between rounds (one synchronisation per round)
                   "rounds_device_ms": sum(round_us) / 1e3, "recorded_run_ms": st_rec["ms_total"],
                   "tail_rounds_below_100k_faces": len(tail),
                   "tail_ms": sum(r["us"] for r in tail) / 1e3,
                   "tail_share": sum(r["us"] for r in tail) / max(sum(round_us), 1)}
    # every class's share: one profiled warm-up run with every class timed
    opts = pamo.Options(validate_input=0, profile=0xFF)
    _, _, st_prof, _ = pamo.pamo_simplify(Vd, Fd, target, options=opts)
    dom = CLASS_NAMES.index(ROOFLINE_CLASS)
    ic = CLASS_NAMES.index("cost")
    prof_opts = pamo.Options(validate_input=0, profile=(1 << dom) | (1 << ic))
    # the timed steps: plain calls, without the class events
    plain_opts = pamo.Options(validate_input=0)
    # float64 rates of this GPU (before the timed region)
    fp64 = pamo.pamo_measure_fp64()
    # the clock sampler starts before the warm-up steps: nvidia-smi's start-up
    # (NVML initialisation) then never lands in a timed step
    clocks = ClockSampler(local)
    clocks.start()
    for _ in range(args.warmup):
        pamo.pamo_simplify(Vd, Fd, target, options=plain_opts)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    times, launches = [], 0
    out = None
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        Vo, Fo, st, status = pamo.pamo_simplify(Vd, Fd, target, options=plain_opts)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        launches += st["launches"]
        out = (Vo, Fo, st, status)
    torch.cuda.synchronize()
    barrier()
    # the roofline class per launch: the same number of steps right after,
    # with CUDA events around the class
    dom_ms, dom_launch, dom_bytes, bytes_alg, cost_edges = 0.0, 0, 0.0, 0.0, 0
    c_ms, c_launch, c_flops, cost_f64 = 0.0, 0, 0.0, 0
    for _ in range(args.steps):
        flush.fill_(1)
        _, _, stp, _ = pamo.pamo_simplify(Vd, Fd, target, options=prof_opts)
        dom_ms += stp["class_ms"][dom]
        dom_launch += stp["class_launches"][dom]
        dom_bytes += stp["class_bytes"][dom]
        c_ms += stp["class_ms"][ic]
        c_launch += stp["class_launches"][ic]
        c_flops += stp["class_flops"][ic]
        bytes_alg += stp["bytes_model"]
        cost_edges += stp["cost_edges"]
        cost_f64 += stp["cost_f64"]
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = max_over_ranks(sum(times), device="cuda")
    ms_per_step = total_ms / args.steps
    value = weak_value(len(F), world, ms_per_step)

    # end to end through the host-buffer entry point
    e2e = None
    if not args.no_e2e:
        e2e = host_leg(pamo, torch, V, F, target, args.steps, world, barrier)
    share = {CLASS_NAMES[i]: round(st_prof["class_ms"][i] / max(sum(st_prof["class_ms"]), 1e-9), 4)
             for i in range(7)}
    # the dominant kernel's class: latency-bound node and pair gathers, set
    # against HBM by its algorithmic bytes (the check's reads and writes per
    # launch, pamo_stats.class_bytes) over its CUDA-event time
    peak, peak_kind = peaks()
    avg_launch_ms = dom_ms / max(dom_launch, 1)
    bytes_per_launch = dom_bytes / max(dom_launch, 1)
    achieved = bytes_per_launch / (avg_launch_ms * 1e-3) / 1e9 if avg_launch_ms > 0 else 0.0
    roof = {"bound": "hbm", "kernel_class": CLASS_NAMES[dom], "kernel": "k_traverse",
            "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": None,
            "traffic_note": ("bound by dependent node loads, not bytes (DRAM 1.7 % of peak "
                             "under ncu); a launch's traffic is not tracked"),
            "peak_source": peak_kind, "launch_ms": avg_launch_ms, "class_share": share}
    roof_cost = cost_roofline(c_ms, c_launch, c_flops, cost_edges, cost_f64, fp64)
    Vo, Fo, st, status = out
    # the whole pipeline against HBM: algorithmic bytes of every round / wall
    hbm_peak, hbm_kind = peaks()
    pipe_gbs = bytes_alg / args.steps / (ms_per_step * 1e-3) / 1e9
    pipeline = {"bytes_alg_per_step": bytes_alg / args.steps, "achieved_gbs": pipe_gbs,
                "peak_gbs": hbm_peak, "frac": pipe_gbs / hbm_peak, "peak_source": hbm_kind}
    line = {"metric": METRIC, "value": value, "unit": "Mfaces/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload, "faces_in": int(len(F)), "target": int(target),
                       "faces_out": int(len(Fo)), "rounds": st["rounds"], "status": status,
                       "undo_iters_hist": st["undo_iters_hist"][:4],
                       "round_times": rounds_info,
                       "l2": "flushed between steps (256 MiB write, outside the timed span)",
                       "parallelism": f"replicas x{world}"},
            "roofline": roof, "roofline_cost": roof_cost, "pipeline_hbm": pipeline, "clocks": clk, "e2e": e2e,
            "gpu_launches": int(launches)}
    if not args.no_batch and args.level == 8:
        # the batched path (many meshes per pass) on its own workload, beside
        # the plain number: its throughput, the same meshes one call at a
        # time, and the speed-up
        b = run_batch_bench(args, world, rank, emit=False)
        line["batch"] = {"value": b["value"], "unit": b["unit"], "ms_per_step": b["ms_per_step"],
                         "steps": b["steps"], "workload": b["config"]["workload"],
                         "meshes": b["config"]["meshes"], "faces_in": b["config"]["faces_in"],
                         "stalled": b["config"]["stalled"],
                         "plain_one_at_a_time": b["plain_one_at_a_time"],
                         "speedup_vs_plain": b["speedup_vs_plain"], "autotune": b["autotune"],
                         "clocks": b["clocks"], "gpu_launches": b["gpu_launches"]}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_oracle_sample(args.level)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
