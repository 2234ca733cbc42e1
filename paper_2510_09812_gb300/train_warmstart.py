"""Train the learned warm start of the mechanical CG on pairs the plain FP64 solver generates.

  python -m paper_2510_09812_gb300.train_warmstart [--pairs P] [--iters K] [--cells 128,128,32]

Data: GSPM trajectories of the 512x512x128 nm sphere-inclusion workload (0.5M nodes at the
default size) under several applied fields; at every recorded step the pair is
(m^n, u^{n-1}, u^{n-2}) -> u^n, where u^n is the plain FP64 solver's displacement for m^n
(mechanical CG to 1e-10).  All data stays on the GPU.  Training: Adam on single pairs drawn at
random (full-mesh graphs).  Writes the parameters to weights/warmstart_mpnn.npy beside this file
and prints one JSON line with the losses.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "weights", "warmstart_mpnn.npy")


def he_init(seed: int) -> np.ndarray:
    """He-normal weights (zero biases, zero output head) from splitmix64 / Box-Muller."""
    from . import gspm, synth
    flat = np.zeros(gspm.MPNN_PARAMS, dtype=np.float64)
    o = 0
    for k, shp in gspm.MPNN_KEYS:
        size = int(np.prod(shp))
        if k.startswith("W") and k != "W_out":
            fan_in = shp[0]
            flat[o:o + size] = synth.normal(synth.substream(seed, 100 + o), size) * np.sqrt(2.0 / fan_in)
        o += size
    return flat.astype(np.float32)


def generate(ctx, torch, gspm, cfg, pairs, fields, steps_per_field, record_every):
    """Run the plain solver along trajectories and store pairs in the context's dataset."""
    n = ctx.n
    dev = "cuda"
    m_buf = torch.empty((n, 3), dtype=torch.float64, device=dev)
    up = torch.empty_like(m_buf)
    up2 = torch.empty_like(m_buf)
    us = torch.empty_like(m_buf)
    added = 0
    k = 0
    for H in fields:
        for s in range(steps_per_field):
            ctx.get_field(gspm.FIELD_M, m_buf)
            ctx.get_field(gspm.FIELD_DISP, up)
            ctx.get_field(gspm.FIELD_DISP_PREV, up2)
            ctx.step(1, H, stats=False)
            k += 1
            if k % record_every == 0 and added < pairs:
                ctx.get_field(gspm.FIELD_DISP, us)
                ctx.mpnn_dataset_add(m_buf, up, up2, us)
                added += 1
            if added >= pairs:
                return added
    return added


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--pairs", type=int, default=400)
    ap.add_argument("--iters", type=int, default=3000)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--cells", default="128,128,32")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default=WEIGHTS)
    args = ap.parse_args()
    import torch
    from . import build
    build.build()
    from . import gspm, synth
    cells = tuple(int(v) for v in args.cells.split(","))
    box = tuple(4.0 * c for c in cells)
    cfg = synth.sphere_inclusion_box(n_cells=cells, box=box, radius=60.0 * cells[0] / 128.0)
    ctx = gspm.Context(cfg["mesh"], cfg["material"], cfg["dt"], cfg["alpha"], precision="f64",
                       rtol_gs=1e-7, rtol_ms=1e-7, rtol_mech=1e-10)
    ctx.set_field(gspm.FIELD_M, cfg["m0"])
    ctx.mpnn_set_params(he_init(args.seed))
    ctx.mpnn_dataset_reserve(args.pairs)
    mu0 = synth.MU0
    rng_dirs = synth.normal(synth.substream(args.seed, 7), 3 * 16).reshape(16, 3)
    fields = [np.array([-0.1 / mu0, 0, 0]), np.array([0.05 / mu0, 0.05 / mu0, 0])]
    fields += [d / np.linalg.norm(d) * 0.1 / mu0 for d in rng_dirs]
    t0 = time.perf_counter()
    got = generate(ctx, torch, gspm, cfg, args.pairs, fields, steps_per_field=40, record_every=1)
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    l0, _ = ctx.mpnn_train(1, lr=args.lr, seed=args.seed)
    _, l1 = ctx.mpnn_train(args.iters, lr=args.lr, seed=args.seed + 1)
    t_train = time.perf_counter() - t0
    params = ctx.mpnn_get_params()
    os.makedirs(os.path.dirname(args.out), exist_ok=True)
    np.save(args.out, params)
    print(json.dumps({"pairs": got, "nodes": ctx.n, "iters": args.iters, "loss_first": l0,
                      "loss_last": l1, "gen_s": round(t_gen, 1), "train_s": round(t_train, 1),
                      "out": os.path.relpath(args.out, os.path.dirname(HERE))}), flush=True)


if __name__ == "__main__":
    sys.exit(main())
