"""Benchmark of the GB300 GSPM step: GSPM steps/s on the 3M-node void + cuboids mesh.

One "step" = one full GSPM time step (volume averages, both RHS assemblies, magnetostatic and
mechanical CG, strain/field recovery, seven GSPM CG solves, projection) through the C ABI.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  N > 1 (torchrun) runs independent replicas of the single-mesh
step, one per GPU (the single-mesh path has no independent units to shard).
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
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GSPM steps/s at 3M nodes, mixed+learned vs plain FP64 on 1 GB300; % HBM peak"
WEIGHTS = os.path.join(ROOT, "paper_2510_09812_gb300", "weights", "warmstart_mpnn.npy")
FALLBACK_HBM = 6800.0


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


def _traffic(kernel, workload):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on this kernel
    source; else None."""
    d = os.path.join(ROOT, "profiles")
    if not os.path.isdir(d):
        return None
    for fn in sorted(os.listdir(d)):
        if not fn.startswith(kernel) or workload not in fn:
            continue
        txt = open(os.path.join(d, fn)).read()
        h = re.search(r"kernels_sha256:\s*([0-9a-f]+)", txt)
        b = re.search(r"dram_bytes_per_launch_full:\s*([0-9.eE+]+)", txt)
        if h and b and h.group(1) == _kernel_src_hash():
            return float(b.group(1))
    return None


def cpu_oracle_sample(wall_budget=25.0, steps=None, warmup=1):
    """Time the CPU oracle (as it stands) on a bounded sample of the workload: a mesh built
    with the same recipe (h, jitter, void + cuboids generator) but 40x40x10 cubes.  Returns
    (steps/s scaled to the full mesh by node count, seconds per sample step, description)."""
    from paper_2510_09812_gb300 import synth
    from oracle.gspm import System
    from oracle.mesh import WrappedMesh
    h = 1024.0 / 228.0
    cells = (40, 40, 10)
    cfg = synth.void_cuboids_box(n_cells=cells, box=tuple(v * h for v in cells))
    full_n = 228 * 228 * 57
    wm = WrappedMesh.from_synth(cfg["mesh"])
    s = System(wm, cfg["material"], cfg["dt"], cfg["alpha"])
    m = np.array(cfg["m0"])
    m[~s.mag] = 0.0
    U, u = np.zeros(wm.n), np.zeros((wm.n, 3))
    for _ in range(warmup):
        m, U, u, _ = s.step(m, U, u, cfg["H"])
    t0 = time.perf_counter()
    k = 0
    while True:
        m, U, u, _ = s.step(m, U, u, cfg["H"])
        k += 1
        el = time.perf_counter() - t0
        if (steps is not None and k >= steps) or (steps is None and (el > wall_budget or k >= 20)):
            break
    per = el / k
    desc = (f"oracle GSPM steps on the same recipe at 40x40x10 cubes ({wm.n} nodes, "
            f"{cfg['mesh'].n_tets} tets), {k} timed after {warmup} warm-up; per-step time "
            f"scaled by node count {wm.n}/{full_n} to the 3M-node mesh")
    return (1.0 / per) * (wm.n / full_n), per, desc, k


def cpu_oracle_sample_1core(steps=None, warmup=1):
    """cpu_oracle_sample in a fresh child process with one BLAS / OpenMP thread, so that the
    sample runs on exactly one core."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.cpu_oracle_sample(steps=%r, warmup=%r)))"
            % (ROOT, steps, warmup))
    out = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, check=True,
                         capture_output=True, text=True).stdout
    rate, per, desc, k = json.loads(out.strip().splitlines()[-1])
    return rate, per, desc, k


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
    n = info["n_unique"]
    snap = {f: torch.empty((n, gspm.FIELD_NCOMP[f]) if gspm.FIELD_NCOMP[f] > 1 else (n,),
                           dtype=torch.float64, device="cuda")
            for f in (gspm.FIELD_M, gspm.FIELD_U, gspm.FIELD_DISP)}
    for f, t in snap.items():
        ctx.get_field(f, t)
    kb = max(1, min(args.steps, 4))

    def timed_batch(graph):
        # the graph is captured by an untimed step; every pass starts from the same state
        ctx.set_graph(graph)
        ctx.batch_step(1, H, stats=False)
        for f, t in snap.items():
            ctx.set_field(f, t)
        l0 = ctx.launch_count()
        barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        st = ctx.batch_step(kb, H)
        ev1.record()
        barrier()
        return ev0.elapsed_time(ev1), ctx.launch_count() - l0, st

    ms_direct, _, st_direct = timed_batch(False)
    ms, launches, st = timed_batch(True)
    same = all(a["it_mech"] == b["it_mech"] for a, b in zip(st, st_direct))
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
                "ms_per_batch_step_direct": ms_direct / kb, "scaling": "weak"}
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
            "graph_replay": True, "ms_per_batch_step_direct": ms_direct / kb,
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


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return
    per_steps = []
    rate, per, desc, k = cpu_oracle_sample_1core(steps=args.steps, warmup=args.warmup)
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": "steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 / rate, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "void_cuboids_1024x1024x256nm_2963088n", "precision": "f64",
                       "solver": "CPU oracle (NumPy/SciPy, single thread)"},
            "cpu_baseline": {"value": rate, "unit": "steps/s", "cores": 1, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": rate, "unit": "steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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

    cfg = _workload(args)
    mesh = cfg["mesh"]
    H = cfg["H"]
    peak, peak_kind = _peaks()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    weights = None
    if os.path.exists(WEIGHTS):
        weights = np.load(WEIGHTS)
    x0_names = {"prev": gspm.X0_PREV, "zero": gspm.X0_ZERO, "extrapolate": gspm.X0_EXTRAPOLATE,
                "learned": gspm.X0_LEARNED}
    # default: the previous step's displacement (the paper's warm start); with the CG projected
    # off the constants the three classical guesses need about the same iterations on this
    # workload (248 / 247 / 254 per step for previous / extrapolated / zero)
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
        ctx.set_x0_mode(x0_names[mode])
        return ctx, time.perf_counter() - t0

    def timed_steps(ctx, k, profile=("spmv_mech",)):
        ctx.profile_enable(profile)
        st_tot = {"it_mech": 0, "it_ms": 0, "it_gs": 0}
        l0 = ctx.launch_count()
        barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local, enabled=not args.no_clocks) as clk:
            ev0.record()
            for _ in range(k):
                st = ctx.step(1, H)
                for key in st_tot:
                    st_tot[key] += st[key]
            ev1.record()
            barrier()
        ms = ev0.elapsed_time(ev1)
        launches = ctx.launch_count() - l0
        prof = {c: ctx.profile_read(c) for c in profile}
        ctx.profile_enable(())
        return ms, st_tot, launches, prof, clk.summary()

    precision = args.precision
    ctx, t_load = make(precision, x0, pinned=args.pinned_cg, plain=args.plain_cg)
    info = ctx.info()
    n = info["n_unique"]
    for _ in range(args.warmup):
        ctx.step(1, H)
    # snapshot of the state after warm-up: every measured pass starts from it, so the timed
    # region, the kernel breakdown and the end-to-end pass do identical work
    snap = {f: torch.empty((n, gspm.FIELD_NCOMP[f]) if gspm.FIELD_NCOMP[f] > 1 else (n,),
                           dtype=torch.float64, device="cuda")
            for f in (gspm.FIELD_M, gspm.FIELD_U, gspm.FIELD_DISP, gspm.FIELD_DISP_PREV)}
    for f, t in snap.items():
        ctx.get_field(f, t)

    def restore():
        for f, t in snap.items():
            ctx.set_field(f, t)
        torch.cuda.synchronize()

    ms, st, launches, prof, clocks = timed_steps(ctx, args.steps)
    from paper_2510_09812_gb300.shard import max_over_ranks
    t_max = max_over_ranks(ms, torch.device("cuda", local))
    value = ws * args.steps / (t_max / 1000.0)

    # roofline of the dominant kernel: 3x3-block SELL SpMV of the mechanical CG
    w = 4 if precision == "mixed" else 8
    bytes_per_iter = (info["sell_entries"] * (9 * w + 4) + ((n + 31) // 32) * 12 + n * 3 * w * 2)
    t_spmv, n_spmv = prof["spmv_mech"]
    achieved = bytes_per_iter * st["it_mech"] / (t_spmv / 1000.0) / 1e9 if t_spmv > 0 else None
    wl = cfg["name"]
    traffic = _traffic("spmv_mech", "void_cuboids_3M") if args.cells is None else None

    # per-class breakdown (separate, untimed pass from the same state)
    classes = ["spmv_mech", "spmv_gs", "spmv_ms", "cg_vec", "cg_init", "rowops", "pointwise"]
    kb = max(1, min(2, args.steps))
    restore()
    bms, bst, _, bprof, _ = timed_steps(ctx, kb, classes)
    breakdown = {c: round(bprof[c][0] / kb, 3) for c in classes}
    breakdown["total_ms_per_step"] = round(bms / kb, 3)

    # end to end through the C ABI with pinned host buffers, from the same state: every step
    # copies m host->device, steps, and copies m device->host (the next step's input)
    restore()
    mh = snap[gspm.FIELD_M].cpu().pin_memory()
    mo = torch.empty_like(mh).pin_memory()
    ke = args.steps
    barrier()
    t0 = time.perf_counter()
    for _ in range(ke):
        ctx.set_field(gspm.FIELD_M, mh)
        ctx.step(1, H, stats=False)
        ctx.get_field(gspm.FIELD_M, mo)
        mh, mo = mo, mh
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": ws * ke / e2e_s, "unit": "steps/s", "h2d_bytes_per_step": n * 3 * 8,
           "d2h_bytes_per_step": n * 3 * 8}

    # mechanical-CG initial guesses compared over the same steps from the same state
    x0_cmp = {}
    if not args.skip_x0:
        modes = ["prev", "extrapolate", "zero"] + (["learned"] if weights is not None else [])
        kx = max(1, min(args.steps, 3))
        for mode in modes:
            restore()
            ctx.set_x0_mode(x0_names[mode])
            ms_x, st_x, _, _, _ = timed_steps(ctx, kx, ())
            x0_cmp[mode] = {"it_mech_per_step": st_x["it_mech"] / kx,
                            "ms_per_step": round(ms_x / kx, 2)}
        ctx.set_x0_mode(x0_names[x0])

    # graph replay of the same steps from the same state (no per-kernel events inside a graph,
    # so the roofline above comes from the direct pass)
    graph = None
    if not args.skip_graph:
        restore()
        ctx.set_graph(True)
        ctx.step(1, H, stats=False)  # capture
        restore()
        ms_g, st_g, l_g, _, _ = timed_steps(ctx, args.steps, ())
        graph = {"value": ws * args.steps / (ms_g / 1000.0), "unit": "steps/s",
                 "ms_per_step": ms_g / args.steps, "gpu_launches": l_g,
                 "same_iterations_as_direct": st_g == st}
        ctx.set_graph(False)
    ctx.close()

    small = None
    if not args.skip_graph and ws == 1:
        small = run_small(gspm, torch, barrier)

    # batched uneven meshes (64 meshes, 2k-200k nodes) in one context
    batched = None
    if not args.skip_batch:
        batched = run_batch(gspm, torch, args, barrier)

    # other CG forms in the headline precision, same steps from the same start: the pinned
    # systems of Sec. 2.5 (plain CG, as the paper) and the singular systems without the
    # two-level preconditioner
    forms = {}
    if not args.skip_plain:
        for name, kw in (("pinned_plain_cg", dict(pinned=True)),
                         ("singular_plain_cg", dict(plain=True))):
            ctxp, _ = make(precision, x0, **kw)
            for _ in range(args.warmup):
                ctxp.step(1, H)
            kp = max(1, min(args.steps, 3))
            ms_p, st_p, _, _, _ = timed_steps(ctxp, kp, ())
            forms[name] = {"steps": kp, "ms_per_step": round(ms_p / kp, 2),
                           "it_mech_per_step": st_p["it_mech"] / kp,
                           "it_ms_per_step": st_p["it_ms"] / kp}
            ctxp.close()

    # plain FP64 GPU form on the same GPU (the comparison the metric names): the paper's
    # formulation (pinned systems, FP64 throughout, previous solution as initial guess)
    plain = None
    if precision != "f64" and not args.skip_plain:
        ctx64, t_load64 = make("f64", pinned=True)
        for _ in range(args.warmup):
            ctx64.step(1, H)
        k64 = max(1, args.steps // 2)
        ms64, st64, l64, prof64, _ = timed_steps(ctx64, k64)
        t64, _ = prof64["spmv_mech"]
        b64 = (info["sell_entries"] * (9 * 8 + 4) + ((n + 31) // 32) * 12 + n * 3 * 8 * 2)
        plain = {"value": k64 / (ms64 / 1000.0), "unit": "steps/s", "steps": k64,
                 "ms_per_step": ms64 / k64, "it_mech_per_step": st64["it_mech"] / k64,
                 "spmv_mech_gbs": b64 * st64["it_mech"] / (t64 / 1000.0) / 1e9 if t64 else None}
        ctx64.close()

    if rank != 0:
        return
    cpu = None
    if ws == 1 and not args.skip_cpu:
        rate, per, desc, k = cpu_oracle_sample_1core()
        cpu = {"value": rate, "unit": "steps/s", "cores": 1, "kind": "oracle", "sample": desc}
    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32/f64" if precision == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": wl, "nodes": n, "tets": info["n_tets"],
                   "magnetic_nodes": info["n_magnetic_nodes"], "precision": precision,
                   "ordering": (args.ordering if args.ordering != "auto" else
                                ("none" if (args.plain_cg or args.pinned_cg) else "aggregate")),
                   "field_A_per_m": list(map(float, H)),
                   "dt_s": cfg["dt"], "alpha": cfg["alpha"], "rtol": 1e-7,
                   "l2": f"inputs > L2: {info['device_bytes'] / 1e9:.2f} GB resident, "
                         "no flush needed",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "mesh_load_s": round(t_load, 2)},
        "node_updates_per_s": value * info["n_magnetic_nodes"],
        "cg_iterations_per_step": {k: v / args.steps for k, v in st.items()},
        "roofline": {"bound": "hbm", "kernel": "spmv_mech (SELL-32 3x3-block SpMV + p.q)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if achieved else None, "traffic": traffic,
                     "peak_kind": peak_kind, "bytes_per_launch": bytes_per_iter,
                     "launches_timed": n_spmv, "iterations_timed": st["it_mech"]},
        "breakdown_ms_per_step": breakdown,
        "cg_form": "pinned (Sec. 2.5), plain CG" if args.pinned_cg else
                   ("consistent singular system, plain CG" if args.plain_cg else
                    "consistent singular system, two-level preconditioned CG"),
        "n_aggregates": info["n_aggregates"],
        "other_cg_forms_same_start": forms,
        "plain_f64": plain,
        "graph_replay": graph,
        "small_mesh_direct_vs_graph": small,
        "batched": batched,
        "x0": x0,
        "x0_comparison": x0_cmp,
        "cpu_baseline": cpu,
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
    ap.add_argument("--skip-x0", action="store_true")
    ap.add_argument("--skip-batch", action="store_true")
    ap.add_argument("--batch-meshes", type=int, default=64)
    ap.add_argument("--no-clocks", action="store_true", help="no nvidia-smi sampler (profiling)")
    ap.add_argument("--x0", default="auto", choices=["auto", "prev", "zero", "extrapolate", "learned"],
                    help="initial guess of the mechanical CG (auto: learned when trained weights "
                         "exist, else the previous solution)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
