"""Benchmark of the GB300 GSPM step: GSPM steps/s on the 3M-node void + cuboids mesh.

One "step" = one full GSPM time step (volume averages, both RHS assemblies, magnetostatic and
mechanical CG, strain/field recovery, seven GSPM CG solves, projection) through the C ABI.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --contract [--contract-cells 128,128,32] [--contract-steps 1000]

Prints one JSON line (rank 0).  N > 1 (torchrun) runs independent replicas of the single-mesh
step, one per GPU (the single-mesh path has no independent units to shard).  --contract runs the
mixed-precision contract instead: the sphere-inclusion workload stepped in mixed precision and in
FP64 from the same state, with the angle and field errors between the two trajectories.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GSPM steps/s at 3M nodes, mixed+learned vs plain FP64 on 1 GB300; % HBM peak"
WEIGHTS = os.path.join(ROOT, "paper_2510_09812_gb300", "weights", "warmstart_mpnn.npy")
FALLBACK_HBM = 6800.0
FULL_CELLS = (228, 228, 57)
ORACLE_CELLS = (40, 40, 10)
X0_NAMES = ("prev", "zero", "extrapolate", "learned")


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM, "fallback"


def _workload(args):
    from paper_2510_09812_gb300 import synth
    if args.cells:
        c = tuple(int(v) for v in args.cells.split(","))
        h = 1024.0 / 228.0
        return synth.void_cuboids_box(n_cells=c, box=tuple(v * h for v in c))
    return synth.void_cuboids_box()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while active."""

    def __init__(self, index, enabled=True):
        self.index = index
        self.enabled = enabled
        self.proc = None
        self.path = None

    def __enter__(self):
        if not self.enabled:
            return self
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.proc or not self.path or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nme, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nme)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _kernel_src_hash():
    with open(os.path.join(ROOT, "paper_2510_09812_gb300", "csrc", "kernels.cu"), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def _traffic(kernel):
    """DRAM bytes per launch of `kernel` at the 3M-node mesh from a committed ncu summary taken on
    the current kernel source (a line `dram_bytes_per_launch_full[<kernel>]: <bytes>` next to
    `kernels_sha256: <hash>`), else None."""
    d = os.path.join(ROOT, "profiles")
    if not os.path.isdir(d):
        return None
    pat = re.compile(r"dram_bytes_per_launch_full\[" + re.escape(kernel) + r"\]:\s*([0-9.eE+]+)")
    for fn in sorted(os.listdir(d)):
        txt = open(os.path.join(d, fn)).read()
        h = re.search(r"kernels_sha256:\s*([0-9a-f]+)", txt)
        b = pat.search(txt)
        if h and b and h.group(1) == _kernel_src_hash():
            return float(b.group(1))
    return None


# ------------------------------------------------------------------------------------------
# CPU oracle baseline
# ------------------------------------------------------------------------------------------

def cpu_oracle_sample(steps=None, warmup=1, wall_budget=20.0, cells=ORACLE_CELLS):
    """Time the CPU oracle (as it stands) on the benchmark recipe at `cells` cubes (same h,
    jitter and void + cuboids generator): whole steps, then a fixed number of its own CG
    iterations on each system to separate the iteration cost from the rest of the step."""
    from paper_2510_09812_gb300 import synth
    from oracle.gspm import System
    from oracle.mesh import WrappedMesh
    from oracle.solvers import cg
    h = 1024.0 / 228.0
    cfg = synth.void_cuboids_box(n_cells=cells, box=tuple(v * h for v in cells))
    wm = WrappedMesh.from_synth(cfg["mesh"])
    s = System(wm, cfg["material"], cfg["dt"], cfg["alpha"])
    m = np.array(cfg["m0"])
    m[~s.mag] = 0.0
    U, u = np.zeros(wm.n), np.zeros((wm.n, 3))
    for _ in range(warmup):
        m, U, u, _ = s.step(m, U, u, cfg["H"])
    it = {"ms": 0, "mech": 0, "gs": 0}
    t0 = time.perf_counter()
    k = 0
    while True:
        m, U, u, info = s.step(m, U, u, cfg["H"])
        it["ms"] += info["it_ms"]
        it["mech"] += info["it_mech"]
        it["gs"] += int(np.sum(info["it_gs"]))
        k += 1
        el = time.perf_counter() - t0
        if (steps is not None and k >= steps) or (steps is None and (el > wall_budget or k >= 20)):
            break
    per = el / k
    # seconds per CG iteration of each system (the oracle's CG with a zero tolerance runs the
    # requested number of iterations)
    rng = np.random.default_rng(0)
    t_it = {}
    for name, A in (("ms", s.K_ms), ("mech", s.K_mech), ("gs", s.A_eps)):
        b = rng.standard_normal(A.shape[0])
        best = float("inf")
        for _ in range(3):
            t1 = time.perf_counter()
            cg(A, b, np.zeros_like(b), 0.0, 20)
            best = min(best, (time.perf_counter() - t1) / 20)
        t_it[name] = best
    return {"nodes": int(wm.n), "tets": int(cfg["mesh"].n_tets), "cells": list(cells),
            "steps": k, "warmup": warmup, "s_per_step": per,
            "it_per_step": {key: v / k for key, v in it.items()}, "s_per_iteration": t_it}


def cpu_oracle_child(steps=None, warmup=1, threads=1, cells=ORACLE_CELLS):
    """cpu_oracle_sample in a fresh child process with `threads` BLAS / OpenMP threads."""
    env = dict(os.environ, OMP_NUM_THREADS=str(threads), OPENBLAS_NUM_THREADS=str(threads),
               MKL_NUM_THREADS=str(threads), CUDA_VISIBLE_DEVICES="")
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.cpu_oracle_sample(steps=%r, warmup=%r, cells=%r)))"
            % (ROOT, steps, warmup, tuple(cells)))
    return subprocess.Popen([sys.executable, "-c", code], env=env, cwd=ROOT,
                            stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)


def _child_result(p):
    out, err = p.communicate()
    if p.returncode != 0:
        raise RuntimeError("oracle sample failed: " + err[-2000:])
    return json.loads(out.strip().splitlines()[-1])


def oracle_full_size_model(sample, full_nodes, full_cells, it_full=None):
    """Oracle seconds per step at the full mesh from a sample: the work outside the CG loops
    scales with the nodes; a CG iteration costs the sample's measured time per iteration scaled
    by the nodes; the iteration counts of the plain CG on K^ms and K^mech grow with the mesh's
    linear size in cells (sqrt of the condition number of a Laplacian-type operator), those of
    the GSPM solves (M + c eps K) do not.  it_full: measured full-size counts of the same
    algorithm (pinned systems, plain CG), used instead of the growth law when given."""
    scale = full_nodes / sample["nodes"]
    ips, spi = sample["it_per_step"], sample["s_per_iteration"]
    t_cg = sum(ips[k] * spi[k] for k in ("ms", "mech", "gs"))
    other = max(sample["s_per_step"] - t_cg, 0.0)
    growth = max(full_cells) / max(sample["cells"])
    its = dict(it_full) if it_full else {"ms": ips["ms"] * growth, "mech": ips["mech"] * growth,
                                         "gs": ips["gs"]}
    t = other * scale + sum(its[k] * spi[k] * scale for k in ("ms", "mech", "gs"))
    return t, its, ("measured at full size (same algorithm on the GPU)" if it_full else
                    f"sample counts x {growth:.2f} (linear mesh size) for K^ms and K^mech")


def cpu_baseline_block(sample, full_nodes, it_full=None, cores=1, kind="oracle"):
    t, its, how = oracle_full_size_model(sample, full_nodes, FULL_CELLS, it_full)
    return {"value": 1.0 / t, "unit": "steps/s", "cores": cores, "kind": kind,
            "sample": (f"oracle (NumPy/SciPy) GSPM steps on the same recipe at "
                       f"{'x'.join(map(str, sample['cells']))} cubes ({sample['nodes']} nodes), "
                       f"{sample['steps']} timed after {sample['warmup']} warm-up, plus 3 x 20 CG "
                       f"iterations per system (best); full-size step time = non-CG time x nodes ratio "
                       f"+ CG iterations per step ({how}) x time per iteration x nodes ratio"),
            "measured_at_sample": {"nodes": sample["nodes"],
                                   "steps_per_s": 1.0 / sample["s_per_step"],
                                   "node_updates_per_s": sample["nodes"] / sample["s_per_step"],
                                   "cg_iterations_per_step": sample["it_per_step"],
                                   "s_per_cg_iteration": sample["s_per_iteration"]},
            "cg_iterations_per_step_full": its}


def cpu_all_cores(cells=ORACLE_CELLS, steps=3):
    """The oracle sample run as independent single-thread replicas, one per host core: the
    oracle's sparse products run on one thread, so this is the host's whole-CPU throughput of
    the oracle as it stands (node updates/s summed over the replicas)."""
    ncores = os.cpu_count() or 1
    procs = [cpu_oracle_child(steps=steps, warmup=1, threads=1, cells=cells)
             for _ in range(ncores)]
    res = [_child_result(p) for p in procs]
    nu = sum(r["nodes"] / r["s_per_step"] for r in res)
    return {"cores": ncores, "replicas": ncores, "node_updates_per_s": nu,
            "steps_per_s_each_mean": float(np.mean([1.0 / r["s_per_step"] for r in res])),
            "nodes": res[0]["nodes"], "steps": steps}


def run_cpu_scale(args):
    """Check of the oracle's full-size model against a measurement: the oracle timed on the
    benchmark recipe at --cpu-scale-cells cubes (one warm-up step and --cpu-scale-steps timed
    steps, one thread), next to the model's prediction for that size from the usual 16,000-node
    sample (and from the same sample with the measured iteration counts)."""
    cells = tuple(int(v) for v in args.cpu_scale_cells.split(","))
    t0 = time.perf_counter()
    sample = _child_result(cpu_oracle_child())
    big = _child_result(cpu_oracle_child(steps=args.cpu_scale_steps, warmup=1, cells=cells))
    t_model, its_model, how = oracle_full_size_model(sample, big["nodes"], cells)
    t_model_its, _, _ = oracle_full_size_model(sample, big["nodes"], cells, big["it_per_step"])
    print(json.dumps({"cpu_scale": {
        "sample": {"nodes": sample["nodes"], "s_per_step": sample["s_per_step"],
                   "it_per_step": sample["it_per_step"]},
        "measured": {"nodes": big["nodes"], "cells": list(cells), "steps": big["steps"],
                     "s_per_step": big["s_per_step"], "it_per_step": big["it_per_step"],
                     "s_per_iteration": big["s_per_iteration"]},
        "model": {"s_per_step": t_model, "it_per_step": its_model, "how": how},
        "model_with_measured_iterations": {"s_per_step": t_model_its},
        "cores": 1, "wall_s": round(time.perf_counter() - t0, 1)}}), flush=True)


# ------------------------------------------------------------------------------------------
# helpers on contexts
# ------------------------------------------------------------------------------------------

def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _snapshot(gspm, torch, ctx, fields=None):
    n = ctx.n
    fields = fields or (gspm.FIELD_M, gspm.FIELD_U, gspm.FIELD_DISP, gspm.FIELD_DISP_PREV)
    snap = {f: torch.empty((n, gspm.FIELD_NCOMP[f]) if gspm.FIELD_NCOMP[f] > 1 else (n,),
                           dtype=torch.float64, device="cuda") for f in fields}
    for f, t in snap.items():
        ctx.get_field(f, t)
    torch.cuda.synchronize()
    return snap


def _restore(torch, ctx, snap):
    for f, t in snap.items():
        ctx.set_field(f, t)
    torch.cuda.synchronize()


def _fields(gspm, ctx):
    return {name: ctx.get_field(f) for name, f in (("m", gspm.FIELD_M), ("U", gspm.FIELD_U),
                                                    ("u", gspm.FIELD_DISP), ("E", gspm.FIELD_STRAIN),
                                                    ("h_d", gspm.FIELD_HD), ("h", gspm.FIELD_H))}


def _max_angle(a, b):
    na, nb = np.linalg.norm(a, axis=1), np.linalg.norm(b, axis=1)
    ok = (na > 0.5) & (nb > 0.5)
    c = np.clip((a[ok] * b[ok]).sum(1) / (na[ok] * nb[ok]), -1.0, 1.0)
    return float(np.arccos(c).max()) if ok.any() else 0.0


def field_errors(test, ref):
    """Max angle between the m fields (rad) and, for every other field, max |test - ref| / max
    |ref| (U and u are both zero at the pinned node, so they compare directly)."""
    out = {"m_max_angle_rad": _max_angle(test["m"], ref["m"])}
    for k in ("U", "u", "E", "h_d", "h"):
        d = np.abs(np.asarray(test[k]) - np.asarray(ref[k])).max()
        out[f"{k}_rel_err"] = float(d / max(np.abs(ref[k]).max(), 1e-300))
    return out


# ------------------------------------------------------------------------------------------
# secondary workloads
# ------------------------------------------------------------------------------------------

def run_batch(gspm, torch, args, barrier):
    """64 independent meshes of log-uniform size 2k-200k nodes, each with its own inclusion and
    applied field, stepped together (mixed precision) by gspm_batch_step with graph replay (and
    with direct launches from the same state for comparison); compared with the same meshes
    stepped one after another in their own contexts (first 16 meshes)."""
    from paper_2510_09812_gb300 import synth
    from paper_2510_09812_gb300.shard import batch_shard, max_over_ranks, sum_over_ranks
    ws, rank, _ = _dist()
    every = [synth.batch_member(i) for i in range(args.batch_meshes)]
    # N GPUs: each rank steps its own share of the meshes (no data-path collective)
    mine = batch_shard([c["mesh"].n_unique for c in every], rank, ws)
    members = [every[i] for i in mine]
    meshes = [c["mesh"] for c in members]
    H = np.array([c["H"] for c in members])
    t0 = time.perf_counter()
    ctx = gspm.Context(meshes, members[0]["material"], members[0]["dt"], members[0]["alpha"],
                       precision="mixed", rtol_gs=1e-7, rtol_ms=1e-7, rtol_mech=1e-7,
                       coarse_nodes=args.batch_coarse_nodes)
    t_load = time.perf_counter() - t0
    m_all = np.concatenate([c["m0"] for c in members])
    ctx.set_field(gspm.FIELD_M, m_all)
    info = ctx.info()
    ctx.batch_step(2, H, stats=False)
    snap = _snapshot(gspm, torch, ctx, (gspm.FIELD_M, gspm.FIELD_U, gspm.FIELD_DISP))
    kb = max(1, args.batch_steps)
    kd = min(kb, 20)  # the direct-launch comparison: a shorter run from the same state

    def timed_batch(graph, k):
        # the graph is captured by an untimed step; every pass starts from the same state
        ctx.set_graph(graph)
        ctx.batch_step(1, H, stats=False)
        _restore(torch, ctx, snap)
        l0 = ctx.launch_count()
        barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        st = ctx.batch_step(k, H)
        ev1.record()
        barrier()
        return ev0.elapsed_time(ev1), ctx.launch_count() - l0, st

    ms_direct, _, st_direct = timed_batch(False, kd)
    ms_g20, _, st_g20 = timed_batch(True, kd)
    same = all(a["it_mech"] == b["it_mech"] for a, b in zip(st_g20, st_direct))
    ms, launches, st = timed_batch(True, kb)
    ctx.close()
    dev = torch.device("cuda", torch.cuda.current_device())
    ms_direct = max_over_ranks(ms_direct, dev)
    ms = max_over_ranks(ms, dev)
    nodes_all = sum_over_ranks(info["n_unique"], dev)
    nmag_all = sum_over_ranks(info["n_magnetic_nodes"], dev)
    if ws > 1:
        return {"meshes": len(every), "meshes_per_rank": len(members), "nodes": int(nodes_all),
                "steps": kb, "ms_per_batch_step": ms / kb,
                "batch_steps_per_s": kb / (ms / 1000.0),
                "node_updates_per_s": nmag_all * kb / (ms / 1000.0), "graph_replay": True,
                "ms_per_batch_step_direct": ms_direct / kd, "scaling": "weak"}
    # the same first 16 meshes, one context each, stepped one after another
    k16 = min(16, len(members))
    seq_ctx = []
    for c in members[:k16]:
        x = gspm.Context(c["mesh"], c["material"], c["dt"], c["alpha"], precision="mixed",
                         rtol_gs=1e-7, rtol_ms=1e-7, rtol_mech=1e-7)
        x.set_field(gspm.FIELD_M, c["m0"])
        x.step(2, c["H"], stats=False)
        seq_ctx.append(x)
    bctx = gspm.Context(meshes[:k16], members[0]["material"], members[0]["dt"],
                        members[0]["alpha"], precision="mixed", rtol_gs=1e-7, rtol_ms=1e-7,
                        rtol_mech=1e-7)
    bctx.set_field(gspm.FIELD_M, np.concatenate([c["m0"] for c in members[:k16]]))
    bctx.batch_step(2, H[:k16], stats=False)
    barrier()
    t0 = time.perf_counter()
    for x, c in zip(seq_ctx, members[:k16]):
        x.step(1, c["H"], stats=False)
    barrier()
    t_seq = time.perf_counter() - t0
    t0 = time.perf_counter()
    bctx.batch_step(1, H[:k16], stats=False)
    barrier()
    t_bat = time.perf_counter() - t0
    for x in seq_ctx:
        x.close()
    bctx.close()
    return {"meshes": len(members), "nodes": int(nodes_all),
            "min_nodes": min(m.n_unique for m in meshes), "max_nodes": max(m.n_unique for m in meshes),
            "steps": kb, "ms_per_batch_step": ms / kb, "batch_steps_per_s": kb / (ms / 1000.0),
            "node_updates_per_s": nmag_all * kb / (ms / 1000.0),
            "graph_replay": True, "direct_steps": kd, "ms_per_batch_step_direct": ms_direct / kd,
            "ms_per_batch_step_graph_same_steps": ms_g20 / kd,
            "graph_and_direct_same_iterations": same,
            "gpu_launches_per_batch_step": launches / kb, "load_s": round(t_load, 1),
            "item_slices": info["item_slices"],
            "first16_batched_vs_sequential_ms": [round(1000 * t_bat, 1), round(1000 * t_seq, 1)],
            "mech_it_per_mesh_last_step": [s_["it_mech_last"] for s_ in st]}


def run_small(gspm, torch, barrier, steps=200):
    """The 1024-node Fe box (16x16x4 cubes): kernels of a few microseconds, so the host's
    launches and synchronisations dominate; direct launches against graph replay, same state
    (fixed SpMV schedule, so both contexts round alike and take the same iterations)."""
    from paper_2510_09812_gb300 import synth
    cfg = synth.fe_box_17x17x5()
    out = {"workload": cfg["name"], "steps": steps}
    for graph in (False, True):
        ctx = gspm.Context(cfg["mesh"], cfg["material"], cfg["dt"], cfg["alpha"],
                           precision="mixed", rtol_gs=1e-7, rtol_ms=1e-7, rtol_mech=1e-7,
                           graph=graph, autotune=False)
        ctx.set_field(gspm.FIELD_M, cfg["m0"])
        ctx.step(3, cfg["H"], stats=False)
        barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        st = ctx.step(steps, cfg["H"])
        ev1.record()
        barrier()
        ms = ev0.elapsed_time(ev1)
        key = "graph" if graph else "direct"
        out[key] = {"steps_per_s": steps / (ms / 1000.0), "ms_per_step": ms / steps,
                    "cg_iterations_per_step": (st["it_ms"] + st["it_mech"] + st["it_gs"]) / steps}
        ctx.close()
    return out


# ------------------------------------------------------------------------------------------
# reference arm: the CPU oracle
# ------------------------------------------------------------------------------------------

def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return
    # each requested step is one oracle step of the bounded sample (a fixed mesh of the recipe)
    sample = _child_result(cpu_oracle_child(steps=args.steps, warmup=args.warmup))
    n_full = FULL_CELLS[0] * FULL_CELLS[1] * FULL_CELLS[2]
    cpu = cpu_baseline_block(sample, n_full)
    rate = cpu["value"]
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": "steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 / rate, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "void_cuboids_1024x1024x256nm_2963088n", "precision": "f64",
                       "solver": "CPU oracle (NumPy/SciPy, one thread): pinned systems, plain CG"},
            "cpu_baseline": cpu,
            "e2e": {"value": rate, "unit": "steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------
# mixed-precision contract run (separate invocation)
# ------------------------------------------------------------------------------------------

def run_contract(args):
    """The sphere-inclusion workload (512x512x128 nm, 0.5M nodes, dt 5 ps) stepped for
    --contract-steps steps (graph replay) from its own start (m = e1 in 200 A/m along e1) and
    from a seeded random m, in four ways from the same state: mixed precision and FP64 at the
    paper's tolerance 1e-7, FP64 at 1e-10 (the reference), and FP64 at 1e-7 from the start
    rotated by about 1e-9 rad per node.  Reported at checkpoints: the largest angle of m and the
    relative errors of U, u, E, h~_d and h of each run against the reference and of mixed
    against FP64 at the same tolerance, plus true residuals and step rates.  The FP64 runs show
    how far the trajectory itself amplifies a change of the solver tolerance or of the start,
    against which the mixed-precision difference is read."""
    import torch
    from paper_2510_09812_gb300 import build
    from paper_2510_09812_gb300 import gspm, synth
    build.build()
    torch.cuda.set_device(0)
    cells = tuple(int(v) for v in args.contract_cells.split(","))
    box = tuple(4.0 * c for c in cells)
    cfg = synth.sphere_inclusion_box(n_cells=cells, box=box, radius=60.0 * cells[2] / 32)
    K = args.contract_steps
    n = cfg["mesh"].n_unique
    checkpoints = sorted({c for c in (1, 10, 100, K // 2, K) if 0 < c <= K})
    starts = {"uniform_e1_200Apm": (cfg["m0"], cfg["H"]),
              "random_m_zero_field": (synth.random_unit_m(n, 11), np.zeros(3))}
    rot = synth.normal(synth.substream(12, 1), 3 * n).reshape(n, 3) * 1e-9
    out = {"workload": cfg["name"], "nodes": n, "dt_s": cfg["dt"], "alpha": cfg["alpha"],
           "steps": K, "starts": {}}
    runs = {"mixed_1e-7": ("mixed", 1e-7, False), "f64_1e-7": ("f64", 1e-7, False),
            "f64_1e-10": ("f64", 1e-10, False), "f64_1e-7_perturbed": ("f64", 1e-7, True)}
    ctxs = {}
    for name, (prec, rt, _) in runs.items():
        ctxs[name] = gspm.Context(cfg["mesh"], cfg["material"], cfg["dt"], cfg["alpha"],
                                  precision=prec, rtol_gs=rt, rtol_ms=rt, rtol_mech=rt,
                                  graph=True)
        ctxs[name].set_true_residual(True)
    for sname, (m0, H) in starts.items():
        fields, res = {}, {"checkpoints": {}}
        for name, (prec, rt, perturbed) in runs.items():
            ctx = ctxs[name]
            mi = np.array(m0, dtype=np.float64)
            if perturbed:
                mi = mi + np.cross(rot, mi)
                mi /= np.linalg.norm(mi, axis=1, keepdims=True)
            ctx.set_field(gspm.FIELD_M, mi)
            ctx.set_field(gspm.FIELD_U, np.zeros(n))
            for f in (gspm.FIELD_DISP, gspm.FIELD_DISP_PREV):
                ctx.set_field(f, np.zeros((n, 3)))
            done, ms, its = 0, 0.0, {"it_ms": 0, "it_mech": 0, "it_gs": 0}
            fields[name] = {}
            for c in checkpoints:
                torch.cuda.synchronize()
                ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                ev0.record()
                st = ctx.step(c - done, H)
                ev1.record()
                torch.cuda.synchronize()
                ms += ev0.elapsed_time(ev1)
                for key in its:
                    its[key] += st[key]
                done = c
                fields[name][c] = _fields(gspm, ctx)
            res[name] = {"steps_per_s": K / (ms / 1000.0),
                         "cg_iterations_per_step": {k: v / K for k, v in its.items()},
                         "last_step": {"res_ms": st["res_ms_last"], "res_mech": st["res_mech_last"],
                                       "true_res_ms": st["true_res_ms_last"],
                                       "true_res_mech": st["true_res_mech_last"],
                                       "dm": st["dm_last"], "noconv": st["noconv"]}}
        for c in checkpoints:
            ref = fields["f64_1e-10"][c]
            row = {f"{name}_vs_f64_1e-10": field_errors(fields[name][c], ref)
                   for name in runs if name != "f64_1e-10"}
            row["mixed_vs_f64_1e-7"] = field_errors(fields["mixed_1e-7"][c], fields["f64_1e-7"][c])
            res["checkpoints"][str(c)] = row
        fin = res["checkpoints"][str(K)]
        res["final_max_angle_rad"] = {k: v["m_max_angle_rad"] for k, v in fin.items()}
        out["starts"][sname] = res
    for c in ctxs.values():
        c.close()
    print(json.dumps({"contract": out}), flush=True)


# ------------------------------------------------------------------------------------------
# time-step study (separate invocation)
# ------------------------------------------------------------------------------------------

def run_dt_sweep(args):
    """The time-step study of Sec. 4 (Fig. 4) on the structured hexahedral cuboid-defect
    workload: for every dt, GSPM steps in FP64 from m = e1 until <|m^n - m^(n-1)|> < 5e-10 over
    the magnetic nodes, in two forms: the library's default (consistent singular systems,
    two-level preconditioned CG for K^ms / K^mech, Jacobi-preconditioned GSPM solves) and the
    paper's (pinned systems, plain CG).  Every CG runs to --sweep-rtol (default 1e-10: at 1e-7 the
    solves' own error leaves <|dm|> on a floor of about 1e-9, above the criterion).  Steps go
    in chunks of 100 (graph replay); the chunk whose last step meets the criterion is replayed
    step by step from its start to find the first step that does.  A run whose <|dm|> climbs
    1000-fold above its smallest value (and above 1e-6), or is still above 1e-3 after 500
    steps, has lost stability and stops.  Reported
    per dt and form: N_LLG (or the step of the loss of stability, or the cap), mean CG
    iterations per step of K^ms and K^mech and per GSPM solve, and the wall time."""
    import torch
    from paper_2510_09812_gb300 import build
    from paper_2510_09812_gb300 import gspm, synth
    build.build()
    torch.cuda.set_device(0)
    cells = tuple(int(v) for v in args.sweep_cells.split(","))
    cfg = synth.cuboid_defect_hex_box(n_cells=cells)
    dts = [float(v) * 1e-12 for v in args.sweep_dt_ps.split(",")]
    cap, chunk, tol, rt = args.sweep_cap, 100, cfg["dm_tol"], args.sweep_rtol
    n = cfg["mesh"].n_unique
    out = {"workload": cfg["name"], "nodes": n, "alpha": cfg["alpha"], "dm_tol": tol,
           "precision": "f64", "rtol": rt, "cap": cap, "Nd": cfg["material"]["Nd"], "runs": []}

    def reset(ctx):
        ctx.set_field(gspm.FIELD_M, cfg["m0"])
        ctx.set_field(gspm.FIELD_U, np.zeros(n))
        for f in (gspm.FIELD_DISP, gspm.FIELD_DISP_PREV):
            ctx.set_field(f, np.zeros((n, 3)))

    def relax(ctx):
        reset(ctx)
        done, its = 0, {"it_ms": 0, "it_mech": 0, "it_gs": 0}
        hist, dm, state, dmin = [], float("nan"), "cap", float("inf")
        t0 = time.perf_counter()
        while done < cap:
            k = min(chunk, cap - done)
            snap = _snapshot(gspm, torch, ctx)
            st = ctx.step(k, cfg["H"])
            if st["dm_last"] < tol:
                _restore(torch, ctx, snap)
                for j in range(k):
                    st = ctx.step(1, cfg["H"])
                    for key in its:
                        its[key] += st[key]
                    if st["dm_last"] < tol:
                        done += j + 1
                        break
                dm = st["dm_last"]
                hist.append([done, dm])
                state = "converged"
                break
            for key in its:
                its[key] += st[key]
            done += k
            dm = st["dm_last"]
            dmin = min(dmin, dm)
            if done % 500 == 0:
                hist.append([done, dm])
            # lost stability: <|dm|> climbed 1000-fold from its smallest value, or never fell
            # (still above 1e-3 after 500 steps, where a stable relaxation is below 1e-4)
            if not np.isfinite(dm) or (dm > 1e-6 and dm > 1e3 * dmin) or (done >= 500 and dm > 1e-3):
                hist.append([done, dm])
                state = "unstable"
                break
        return {"steps": done, "state": state, "dm_last": dm, "dm_min": dmin,
                "cg_per_step": {"ms": its["it_ms"] / done, "mech": its["it_mech"] / done,
                                "gs_per_solve": its["it_gs"] / (7.0 * done)},
                "wall_s": round(time.perf_counter() - t0, 2), "dm_history": hist}

    for dt in dts:
        row = {"dt_ps": round(dt * 1e12, 6),
               "dtau": dt * cfg["material"]["Ms"] * cfg["material"]["gamma0"]}
        forms = {"library_form": {}, "paper_form": {"pinned_cg": True, "plain_cg": True}}
        for name, kw in forms.items():
            if name == "paper_form" and args.sweep_skip_paper_form:
                continue
            ctx = gspm.Context(cfg["mesh"], cfg["material"], dt, cfg["alpha"], precision="f64",
                               rtol_gs=rt, rtol_ms=rt, rtol_mech=rt, graph=True, **kw)
            row[name] = relax(ctx)
            ctx.close()
        out["runs"].append(row)
        print(json.dumps({"dt_sweep_row": row}), flush=True)
    print(json.dumps({"dt_sweep": out}), flush=True)


# ------------------------------------------------------------------------------------------
# the headline
# ------------------------------------------------------------------------------------------

def run_ours(args):
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    from paper_2510_09812_gb300 import build
    build.build()
    from paper_2510_09812_gb300 import gspm
    from paper_2510_09812_gb300.shard import max_over_ranks

    cfg = _workload(args)
    mesh = cfg["mesh"]
    H = cfg["H"]
    peak, peak_kind = _peaks()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    weights = np.load(WEIGHTS) if os.path.exists(WEIGHTS) else None
    x0_code = {"prev": gspm.X0_PREV, "zero": gspm.X0_ZERO, "extrapolate": gspm.X0_EXTRAPOLATE,
               "learned": gspm.X0_LEARNED}
    x0 = args.x0 if args.x0 != "auto" else ("learned" if weights is not None else "prev")
    if x0 == "learned" and weights is None:
        raise SystemExit(f"--x0 learned needs trained weights at {WEIGHTS}")

    def make(prec, mode="prev", pinned=False, plain=False):
        t0 = time.perf_counter()
        ctx = gspm.Context(mesh, cfg["material"], cfg["dt"], cfg["alpha"], precision=prec,
                           ordering=args.ordering, rtol_gs=1e-7, rtol_ms=1e-7, rtol_mech=1e-7,
                           pinned_cg=pinned, plain_cg=plain, coarse_nodes=args.coarse_nodes)
        ctx.set_field(gspm.FIELD_M, cfg["m0"])
        if weights is not None:
            ctx.mpnn_set_params(weights)
        ctx.set_x0_mode(x0_code[mode])
        return ctx, time.perf_counter() - t0

    def timed(ctx, k, profile=(), clocks=False):
        """k steps in one gspm_step call between CUDA events (with per-class events when
        `profile` names kernel classes)."""
        if profile:
            ctx.profile_enable(profile)
        l0 = ctx.launch_count()
        barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local, enabled=clocks and not args.no_clocks) as clk:
            ev0.record()
            st = ctx.step(k, H)
            ev1.record()
            barrier()
        ms = ev0.elapsed_time(ev1)
        launches = ctx.launch_count() - l0
        prof = {c: ctx.profile_read(c) for c in profile}
        if profile:
            ctx.profile_enable(())
        return ms, st, launches, prof, clk.summary()

    def its(st, k):
        return {"it_ms": st["it_ms"] / k, "it_mech": st["it_mech"] / k, "it_gs": st["it_gs"] / k}

    precision = args.precision
    ctx, t_load = make(precision, x0, pinned=args.pinned_cg, plain=args.plain_cg)
    info = ctx.info()
    n = info["n_unique"]
    for _ in range(args.warmup):
        ctx.step(1, H, stats=False)
    # every measured pass starts from the state after warm-up, so all passes do identical work
    snap = _snapshot(gspm, torch, ctx)
    K = args.steps

    # headline: graph replay (each step one CUDA graph launch, CG loops as device-side WHILE
    # nodes), K steps in one call; the graph is captured by an untimed step first
    if not args.direct:
        ctx.set_graph(True)
        ctx.step(1, H, stats=False)
    _restore(torch, ctx, snap)
    ms, st, launches, _, clocks = timed(ctx, K, clocks=True)
    t_max = max_over_ranks(ms, torch.device("cuda", local))
    value = ws * K / (t_max / 1000.0)
    headline_mode = "direct launches" if args.direct else "CUDA graph replay"

    # the same steps with direct launches (host-sequenced CG loops)
    other_mode = None
    if not args.direct:
        ctx.set_graph(False)
        _restore(torch, ctx, snap)
        ms_d, st_d, l_d, _, _ = timed(ctx, K)
        other_mode = {"mode": "direct launches", "value": ws * K / (ms_d / 1000.0),
                      "ms_per_step": ms_d / K, "gpu_launches": l_d,
                      "same_iterations": st_d["it_mech"] == st["it_mech"]
                      and st_d["it_ms"] == st["it_ms"] and st_d["it_gs"] == st["it_gs"]}
    ctx.set_graph(False)

    # kernel pass (separate, from the same state): CUDA events around every launch of the
    # mechanical SpMV and of the four assembly / recovery row kernels
    w = 4 if precision == "mixed" else 8
    E, S = info["sell_entries"], (n + 31) // 32
    kern = {  # algorithmic bytes per launch: values + columns + slice headers + vectors
        "spmv_mech": ("k_cg_spmv<B=9> (3x3-block SELL SpMV + p.q)", E * (9 * w + 4) + S * 12 + 6 * n * w),
        "rhs_ms": ("k_fdiv (b^ms = F^ms m)", E * (3 * w + 4) + S * 12 + 3 * n * w + n * w),
        "grad_ms": ("k_fgrad (h~_d = -grad U)", E * (3 * w + 4) + S * 12 + n * w + 8 * n + 3 * n * w),
        "rhs_mech": ("k_gdiv (b^mech = F^mech E0)", E * (3 * w + 4) + S * 12 + 6 * n * w + 3 * n * w),
        "strain": ("k_fstrain (E = E_bar + sym grad u)", E * (3 * w + 4) + S * 12 + 3 * n * w + 8 * n + 6 * n * w),
    }
    _restore(torch, ctx, snap)
    kp = max(1, min(K, 5))
    _, st_k, _, prof, _ = timed(ctx, kp, tuple(kern))
    rooflines = {}
    for c, (desc, nbytes) in kern.items():
        t_ms, cnt = prof[c]
        gbs = nbytes * cnt / (t_ms / 1000.0) / 1e9 if t_ms > 0 else None
        rooflines[c] = {"kernel": desc, "bytes_per_launch": int(nbytes), "launches": cnt,
                        "us_per_launch": 1000.0 * t_ms / cnt if cnt else None,
                        "achieved_gbs": gbs, "frac": gbs / peak if gbs else None,
                        "traffic": _traffic(c) if args.cells is None else None}
    sp = rooflines["spmv_mech"]
    roofline = {"bound": "hbm", "kernel": sp["kernel"], "achieved": sp["achieved_gbs"],
                "peak": peak, "unit": "GB/s", "frac": sp["frac"], "traffic": sp["traffic"],
                "peak_kind": peak_kind, "bytes_per_launch": sp["bytes_per_launch"],
                "launches_timed": sp["launches"], "timed_in": f"separate pass of {kp} steps"}

    # per-class breakdown (separate pass from the same state)
    classes = ["spmv_mech", "spmv_gs", "spmv_ms", "cg_vec", "cg_init", "rhs_ms", "grad_ms",
               "rhs_mech", "strain", "pointwise", "learned"]
    kb = max(1, min(2, K))
    _restore(torch, ctx, snap)
    bms, _, _, bprof, _ = timed(ctx, kb, classes)
    breakdown = {c: round(bprof[c][0] / kb, 3) for c in classes}
    breakdown["total_ms_per_step"] = round(bms / kb, 3)

    # end to end through the C ABI with pinned host buffers, from the same state: every step
    # copies m host->device, steps (graph replay), and copies m device->host
    if not args.direct:
        ctx.set_graph(True)
    _restore(torch, ctx, snap)
    mh = snap[gspm.FIELD_M].cpu().pin_memory()
    mo = torch.empty_like(mh).pin_memory()
    barrier()
    t0 = time.perf_counter()
    for _ in range(K):
        ctx.set_field(gspm.FIELD_M, mh)
        ctx.step(1, H, stats=False)
        ctx.get_field(gspm.FIELD_M, mo)
        mh, mo = mo, mh
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": ws * K / e2e_s, "unit": "steps/s", "h2d_bytes_per_step": n * 3 * 8,
           "d2h_bytes_per_step": n * 3 * 8}
    ctx.set_graph(False)

    # precision: the FP64 path in the same solver form (graph replay), timed from the same
    # state, then both precisions stepped from that state with true residuals on: max angle of m
    # and the relative errors of every exported field after the same steps
    precision_cmp, f64_form = None, None
    if precision == "mixed" and not args.skip_plain:
        ctx64, t_load64 = make("f64", x0, pinned=args.pinned_cg, plain=args.plain_cg)
        ctx64.set_graph(True)
        ctx64.step(1, H, stats=False)
        _restore(torch, ctx64, snap)
        k64 = max(1, min(K, 10))
        ms64, st64, _, _, _ = timed(ctx64, k64)
        f64_form = {"value": k64 / (ms64 / 1000.0), "unit": "steps/s", "steps": k64,
                    "ms_per_step": ms64 / k64, "cg_iterations_per_step": its(st64, k64),
                    "mesh_load_s": round(t_load64, 2), "mode": "CUDA graph replay"}
        kc = max(1, min(K, 10))
        res = {}
        for name, c in (("mixed", ctx), ("f64", ctx64)):
            c.set_graph(False)
            c.set_true_residual(True)
            _restore(torch, c, snap)
            stc = c.step(kc, H)
            res[name] = (_fields(gspm, c), stc)
            c.set_true_residual(False)
        precision_cmp = {"steps": kc, "from": "state after warm-up (FP32-representable)",
                         "errors_mixed_vs_f64": field_errors(res["mixed"][0], res["f64"][0]),
                         "residuals_last_step": {
                             p: {"recursive_ms": s_["res_ms_last"], "true_ms": s_["true_res_ms_last"],
                                 "recursive_mech": s_["res_mech_last"],
                                 "true_mech": s_["true_res_mech_last"]}
                             for p, (_, s_) in res.items()},
                         "iterations": {p: its(s_, kc) for p, (_, s_) in res.items()}}
        ctx64.close()

    # mechanical-CG initial guesses compared over the same steps from the same state, with the
    # mechanical CG run to 1e-8 (the tolerance of the learned warm-start evaluation)
    x0_cmp = {}
    modes = ["prev", "extrapolate", "zero"] + (["learned"] if weights is not None else [])
    if not args.skip_x0:
        kx = max(1, min(K, 3))
        ctx.set_rtol(rtol_mech=1e-8)
        form = {}
        for mode in modes:
            _restore(torch, ctx, snap)
            ctx.set_x0_mode(x0_code[mode])
            ms_x, st_x, _, prof_x, _ = timed(ctx, kx, ("learned",))
            form[mode] = {"it_mech_per_step": st_x["it_mech"] / kx,
                          "ms_per_step": round(ms_x / kx, 2),
                          "learned_ms_per_step": round(prof_x["learned"][0] / kx, 3)}
        x0_cmp["two_level_pcg"] = form
        ctx.set_rtol(rtol_mech=1e-7)
        ctx.set_x0_mode(x0_code[x0])
    ctx.close()

    small = None
    if not args.skip_graph and ws == 1:
        small = run_small(gspm, torch, barrier)

    batched = None
    if not args.skip_batch:
        batched = run_batch(gspm, torch, args, barrier)

    # the other CG forms in the headline precision, same steps from the same state: the pinned
    # systems of Sec. 2.5 with plain CG (the paper's form) and the singular systems with plain
    # CG; then the paper's form in FP64 (the plain FP64 GPU form the metric names)
    forms, plain = {}, None
    it_full_oracle_form = None
    if not args.skip_plain:
        for name, kw in (("pinned_plain_cg", dict(pinned=True)),
                         ("singular_plain_cg", dict(plain=True))):
            ctxp, _ = make(precision, x0, **kw)
            _restore(torch, ctxp, snap)
            kp2 = max(1, min(K, 3))
            ms_p, st_p, _, _, _ = timed(ctxp, kp2)
            forms[name] = {"steps": kp2, "ms_per_step": round(ms_p / kp2, 2),
                           "steps_per_s": kp2 / (ms_p / 1000.0),
                           "cg_iterations_per_step": its(st_p, kp2)}
            if name == "pinned_plain_cg" and not args.skip_x0:
                ctxp.set_rtol(rtol_mech=1e-8)
                form = {}
                for mode in modes:
                    _restore(torch, ctxp, snap)
                    ctxp.set_x0_mode(x0_code[mode])
                    ms_x, st_x, _, _, _ = timed(ctxp, 1)
                    form[mode] = {"it_mech_per_step": st_x["it_mech"], "ms_per_step": round(ms_x, 2)}
                x0_cmp["pinned_plain_cg"] = form
            ctxp.close()
        if precision != "f64":
            ctx64, _ = make("f64", x0, pinned=True)
            _restore(torch, ctx64, snap)
            k64 = max(1, min(K, 5))
            ms64, st64, _, _, _ = timed(ctx64, k64)
            plain = {"form": "pinned systems (Sec. 2.5), plain CG, FP64 throughout",
                     "value": k64 / (ms64 / 1000.0), "unit": "steps/s", "steps": k64,
                     "ms_per_step": ms64 / k64, "cg_iterations_per_step": its(st64, k64)}
            it_full_oracle_form = {"ms": st64["it_ms"] / k64, "mech": st64["it_mech"] / k64,
                                   "gs": st64["it_gs"] / k64}
            ctx64.close()

    if rank != 0:
        return
    cpu, cpu_all = None, None
    if ws == 1 and not args.skip_cpu:
        sample = _child_result(cpu_oracle_child())
        cpu = cpu_baseline_block(sample, n)
        if it_full_oracle_form:
            t, _, _ = oracle_full_size_model(sample, n, FULL_CELLS, it_full_oracle_form)
            cpu["steps_per_s_with_full_size_iterations"] = 1.0 / t
        if not args.skip_cpu_all:
            cpu_all = cpu_all_cores()
    headline_form = (f"{precision}, consistent singular systems with two-level PCG"
                     if not (args.pinned_cg or args.plain_cg) else precision) + \
                    f", x0 = {x0}" + ("" if x0 == "learned" else
                                      " (no trained warm-start weights in use)")
    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": ws, "steps": K,
        "warmup": args.warmup, "ms_per_step": t_max / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32/f64" if precision == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": cfg["name"], "nodes": n, "tets": info["n_tets"],
                   "magnetic_nodes": info["n_magnetic_nodes"], "precision": precision,
                   "ordering": (args.ordering if args.ordering != "auto" else
                                ("none" if (args.plain_cg or args.pinned_cg) else "aggregate")),
                   "field_A_per_m": list(map(float, H)),
                   "dt_s": cfg["dt"], "alpha": cfg["alpha"], "rtol": 1e-7,
                   "l2": f"inputs > L2: {info['device_bytes'] / 1e9:.2f} GB resident, "
                         "no flush needed",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "mesh_load_s": round(t_load, 2), "mode": headline_mode},
        "headline_form": headline_form,
        "node_updates_per_s": value * info["n_magnetic_nodes"],
        "cg_iterations_per_step": its(st, K),
        "roofline": roofline,
        "assembly_rooflines": {k: v for k, v in rooflines.items() if k != "spmv_mech"},
        "breakdown_ms_per_step": breakdown,
        "other_launch_mode": other_mode,
        "cg_form": "pinned (Sec. 2.5), plain CG" if args.pinned_cg else
                   ("consistent singular system, plain CG" if args.plain_cg else
                    "consistent singular system, two-level preconditioned CG"),
        "n_aggregates": info["n_aggregates"],
        "spmv_schedules": {"mech": info["spmv_schedule_block"], "ms": info["spmv_schedule_scalar"],
                           "gs": info["spmv_schedule_gs"],
                           "ms_per_launch_mech": [round(v, 4) for v in info["spmv_ms_block"]],
                           "ms_per_launch_ms": [round(v, 4) for v in info["spmv_ms_scalar"]],
                           "ms_gs_1_2_3_rhs": [round(v, 4) for v in info["spmv_ms_gs"]]},
        "f64_same_form": f64_form,
        "precision_comparison": precision_cmp,
        "other_cg_forms_same_start": forms,
        "plain_f64": plain,
        "small_mesh_direct_vs_graph": small,
        "batched": batched,
        "x0": x0,
        "x0_comparison_rtol_mech_1e-8": x0_cmp,
        "cpu_baseline": cpu,
        "cpu_all_cores": cpu_all,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "f64"])
    ap.add_argument("--ordering", default="auto", choices=["auto", "none", "rcm", "aggregate"])
    ap.add_argument("--cells", default=None, help="smaller mesh of the same recipe, e.g. 64,64,16")
    ap.add_argument("--direct", action="store_true",
                    help="headline with direct launches instead of graph replay")
    ap.add_argument("--skip-plain", action="store_true")
    ap.add_argument("--skip-graph", action="store_true")
    ap.add_argument("--pinned-cg", action="store_true",
                    help="solve the pinned systems of Sec. 2.5 instead of the singular form")
    ap.add_argument("--coarse-nodes", type=int, default=0,
                    help="nodes per aggregate of the two-level preconditioner (0: default)")
    ap.add_argument("--batch-coarse-nodes", type=int, default=0,
                    help="nodes per aggregate in the batched workload's meshes (0: default)")
    ap.add_argument("--plain-cg", action="store_true",
                    help="no two-level preconditioner for the K^ms / K^mech solves")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-cpu-all", action="store_true")
    ap.add_argument("--skip-x0", action="store_true")
    ap.add_argument("--skip-batch", action="store_true")
    ap.add_argument("--batch-meshes", type=int, default=64)
    ap.add_argument("--batch-steps", type=int, default=500)
    ap.add_argument("--no-clocks", action="store_true", help="no nvidia-smi sampler (profiling)")
    ap.add_argument("--x0", default="auto", choices=["auto", "prev", "zero", "extrapolate", "learned"],
                    help="initial guess of the mechanical CG (auto: learned when trained weights "
                         "exist, else the previous solution)")
    ap.add_argument("--contract", action="store_true",
                    help="run the mixed-precision contract (mixed vs FP64 trajectories) instead")
    ap.add_argument("--contract-cells", default="128,128,32")
    ap.add_argument("--contract-steps", type=int, default=1000)
    ap.add_argument("--cpu-scale", action="store_true",
                    help="time the CPU oracle at a larger size and compare with its model")
    ap.add_argument("--cpu-scale-cells", default="96,96,24")
    ap.add_argument("--cpu-scale-steps", type=int, default=1)
    ap.add_argument("--dt-sweep", action="store_true",
                    help="run the time-step study on the hexahedral cuboid-defect workload instead")
    ap.add_argument("--sweep-cells", default="64,64,16")
    ap.add_argument("--sweep-dt-ps", default="0.25,0.5,0.75,1,1.25,1.5,2,3,5,11")
    ap.add_argument("--sweep-cap", type=int, default=20000)
    ap.add_argument("--sweep-rtol", type=float, default=1e-10)
    ap.add_argument("--sweep-skip-paper-form", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours" and not (args.contract or args.dt_sweep or args.cpu_scale):
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.contract:
        run_contract(args)
    elif args.dt_sweep:
        run_dt_sweep(args)
    elif args.cpu_scale:
        run_cpu_scale(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
