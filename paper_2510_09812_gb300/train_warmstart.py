"""Train the learned warm start of the mechanical CG on pairs the library's own solver generates.

  python -m paper_2510_09812_gb300.train_warmstart [--pairs P] [--val V] [--iters K]
                                                   [--cells 128,128,32] [--seed S]

Data: GSPM trajectories of the sphere-inclusion workload (512 x 512 x 128 nm, 0.5M nodes at the
default size; the box scales with --cells at h = 4 nm), mixed precision with refined
mechanical solves to 1e-9, initial guess 2 u_prev - u_prev2.  Each trajectory starts from m = e1
or from a seeded random m, under a seeded random applied field (direction uniform on the sphere,
|mu0 H| uniform in [0, 0.2] T); from its third step on every step gives one pair
(m^n, u^{n-1}, u^{n-2}) -> u^n.  The last --val pairs come from trajectories of their own and
are held out.  All data stays on the GPU.  Training: Adam on single pairs drawn at random, the
learning rate 1e-3, then 3e-4, then 1e-4 (a third of the iterations each).

Everything is seeded (the network's initial weights, the fields, the starts, the pair draws),
so a run on the same GPU and library reproduces the weights.  Writes them to
weights/warmstart_mpnn.npy beside this file and prints one JSON line: pairs, training and
held-out losses, and the held-out loss of the zero head (the plain extrapolation), which the
network has to beat to help the CG.
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


def trajectory_spec(seed: int, k: int, n: int):
    """Start and field of trajectory k: m = e1 for even k, a seeded random m for odd k; field
    direction uniform on the sphere, |mu0 H| uniform in [0, 0.2] T."""
    from . import synth
    r = synth.uniform01(synth.substream(seed, 1000 + k), np.arange(3))
    z = 2.0 * r[0] - 1.0
    phi = 2.0 * np.pi * r[1]
    d = np.array([np.sqrt(1 - z * z) * np.cos(phi), np.sqrt(1 - z * z) * np.sin(phi), z])
    H = d * (0.2 * r[2]) / synth.MU0
    m0 = synth.uniform_m(n) if k % 2 == 0 else synth.random_unit_m(n, seed * 7919 + k)
    return m0, H


def generate(ctx, torch, gspm, pairs, seed, k0, steps_per_traj=40, skip=2):
    """Run trajectories k0, k0 + 1, ... and add pairs to the context's dataset; returns
    (pairs added, trajectories used)."""
    n = ctx.n
    m_b = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    up, up2, us = torch.empty_like(m_b), torch.empty_like(m_b), torch.empty_like(m_b)
    added, k = 0, k0
    while added < pairs:
        m0, H = trajectory_spec(seed, k, n)
        ctx.set_field(gspm.FIELD_M, m0)
        ctx.set_field(gspm.FIELD_U, np.zeros(n))
        for f in (gspm.FIELD_DISP, gspm.FIELD_DISP_PREV):
            ctx.set_field(f, np.zeros((n, 3)))
        for s in range(steps_per_traj):
            ctx.get_field(gspm.FIELD_M, m_b)
            ctx.get_field(gspm.FIELD_DISP, up)
            ctx.get_field(gspm.FIELD_DISP_PREV, up2)
            ctx.step(1, H, stats=False)
            if s >= skip and added < pairs:
                ctx.get_field(gspm.FIELD_DISP, us)
                ctx.mpnn_dataset_add(m_b, up, up2, us)
                added += 1
        k += 1
    return added, k - k0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--pairs", type=int, default=5000)
    ap.add_argument("--val", type=int, default=200)
    ap.add_argument("--iters", type=int, default=6000)
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
    cfg = synth.sphere_inclusion_box(n_cells=cells, box=box, radius=60.0 * cells[2] / 32.0)
    ctx = gspm.Context(cfg["mesh"], cfg["material"], cfg["dt"], cfg["alpha"], precision="mixed",
                       rtol_gs=1e-7, rtol_ms=1e-7, rtol_mech=1e-9)
    ctx.set_x0_mode(gspm.X0_EXTRAPOLATE)
    ctx.mpnn_set_params(he_init(args.seed))
    ctx.mpnn_dataset_reserve(args.pairs + args.val)
    t0 = time.perf_counter()
    n_train, n_traj = generate(ctx, torch, gspm, args.pairs, args.seed, 0)
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    third = max(1, args.iters // 3)
    l_first, _ = ctx.mpnn_train(1, lr=1e-3, seed=args.seed + 1)
    losses = []
    for j, lr in enumerate((1e-3, 3e-4, 1e-4)):
        losses.append(ctx.mpnn_train(third, lr=lr, seed=args.seed + 2 + j)[1])
    t_train = time.perf_counter() - t0
    params = ctx.mpnn_get_params()
    # held-out pairs (added after training, so the draws above never saw them)
    n_val, _ = generate(ctx, torch, gspm, args.val, args.seed, n_traj + 1000)

    def mean_loss(first, count):
        return float(np.mean([ctx.mpnn_loss_grad(first + i)[0] for i in range(count)]))

    train_loss = mean_loss(0, min(n_train, 200))
    val_loss = mean_loss(n_train, n_val)
    zero = np.array(params)
    zero[-(64 * 3 + 3):] = 0.0  # output head W_out, b_out = 0: the plain extrapolation
    ctx.mpnn_set_params(zero)
    val_zero = mean_loss(n_train, n_val)
    os.makedirs(os.path.dirname(args.out), exist_ok=True)
    np.save(args.out, params)
    print(json.dumps({"pairs": n_train, "val_pairs": n_val, "trajectories": n_traj,
                      "nodes": ctx.n, "iters": 3 * third, "loss_first_step": l_first,
                      "loss_last_steps": losses, "train_loss": train_loss,
                      "val_loss": val_loss, "val_loss_zero_head": val_zero,
                      "gen_s": round(t_gen, 1), "train_s": round(t_train, 1),
                      "out": os.path.relpath(args.out, os.path.dirname(HERE))}), flush=True)


if __name__ == "__main__":
    sys.exit(main())
