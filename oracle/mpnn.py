"""Oracle for the learned warm start of the mechanical CG: FP64 forward and backward of a small
message-passing network over the tetrahedral mesh, its loss, and one Adam update.

TEST INFRASTRUCTURE ONLY (see the package docstring).  The paper has no learned component; the
network is the library's own design and this file is its reference definition.

Network (hidden width 64, three message-passing layers):
  messages   element message = mean of its 4 vertex features; a node receives the
             volume-weighted mean of the messages of its elements:
             z_i = sum_j A_ij h_j,  A_ij = (sum_{e containing i and j} V_e / k) /
             (sum_{e containing i} V_e), k the vertices per element (on tetrahedra the
             denominator is 4 M_L,i)
  input      h0 = relu(f W_in + b_in)                     f: [n, 16] node features
  layer l    h_l = relu([h_{l-1}, A h_{l-1}] W_l + b_l)   W_l: [128, 64], l = 1..3
  output     y = h_3 W_out + b_out                         y: [n, 3]
Features f_i (16): m_i (3), E0(m_i) in Voigt order / lambda_s (6), u_prev_i / u_s (3),
(u_prev_i - u_prev2_i) / u_s (3), 1.  The warm start is x0 = u_ext + u_s y with the linear
extrapolation u_ext = 2 u_prev - u_prev2 (u_prev = u_prev2 = 0 gives a prediction from m alone).
Loss = mean over nodes and components of (y - t)^2 with t = (u* - u_ext) / u_s.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .material import spontaneous_strain

HIDDEN = 64
NFEAT = 16
LAYERS = 3


def aggregation_matrix(wm):
    """Row-stochastic element-message averaging A (see the module docstring); an element of k
    vertices gives every pair of its vertices the weight V_e / k."""
    t = wm.tets
    k = t.shape[1]
    Be = np.repeat((wm.V / k)[:, None, None], k * k, axis=1).reshape(-1, k, k)
    rows = np.repeat(t[:, :, None], k, axis=2)
    cols = np.repeat(t[:, None, :], k, axis=1)
    B = sp.coo_matrix((Be.ravel(), (rows.ravel(), cols.ravel())), shape=(wm.n, wm.n)).tocsr()
    rs = np.asarray(B.sum(axis=1)).ravel()
    return (sp.diags(1.0 / rs) @ B).tocsr()


def scales(l100, l111, h):
    """(lambda_s, u_s): eigenstrain and displacement scales of the features."""
    ls = max(abs(l100), abs(l111))
    return ls, ls * h


def features(m, mag, u_prev, u_prev2, l100, l111, h):
    ls, us = scales(l100, l111, h)
    E0 = spontaneous_strain(m, l100, l111)
    E0[~mag] = 0.0
    ev = np.stack([E0[:, 0, 0], E0[:, 1, 1], E0[:, 2, 2], E0[:, 1, 2], E0[:, 0, 2], E0[:, 0, 1]],
                  axis=1)
    n = m.shape[0]
    return np.concatenate([m, ev / ls, u_prev / us, (u_prev - u_prev2) / us, np.ones((n, 1))],
                          axis=1)


def init_params(seed=0):
    """He-style initialisation from a seeded generator; output layer starts at zero."""
    rng = np.random.default_rng(seed)
    p = {"W_in": rng.standard_normal((NFEAT, HIDDEN)) * np.sqrt(2.0 / NFEAT),
         "b_in": np.zeros(HIDDEN)}
    for l in range(1, LAYERS + 1):
        p[f"W{l}"] = rng.standard_normal((2 * HIDDEN, HIDDEN)) * np.sqrt(2.0 / (2 * HIDDEN))
        p[f"b{l}"] = np.zeros(HIDDEN)
    p["W_out"] = np.zeros((HIDDEN, 3))
    p["b_out"] = np.zeros(3)
    return p


def forward(p, A, f):
    """Returns (y, cache)."""
    cache = {"f": f}
    a0 = f @ p["W_in"] + p["b_in"]
    h = np.maximum(a0, 0.0)
    cache["a0"] = a0
    cache["h0"] = h
    for l in range(1, LAYERS + 1):
        z = A @ h
        x = np.concatenate([h, z], axis=1)
        a = x @ p[f"W{l}"] + p[f"b{l}"]
        cache[f"x{l}"] = x
        cache[f"a{l}"] = a
        h = np.maximum(a, 0.0)
        cache[f"h{l}"] = h
    y = h @ p["W_out"] + p["b_out"]
    return y, cache


def loss(y, t):
    return float(np.mean((y - t) ** 2))


def backward(p, A, cache, y, t):
    """Gradients of loss(y, t) with respect to every parameter (same keys as p)."""
    g = {}
    dy = 2.0 * (y - t) / y.size
    hL = cache[f"h{LAYERS}"]
    g["W_out"] = hL.T @ dy
    g["b_out"] = dy.sum(axis=0)
    dh = dy @ p["W_out"].T
    for l in range(LAYERS, 0, -1):
        da = dh * (cache[f"a{l}"] > 0)
        g[f"W{l}"] = cache[f"x{l}"].T @ da
        g[f"b{l}"] = da.sum(axis=0)
        dx = da @ p[f"W{l}"].T
        dh = dx[:, :HIDDEN] + A.T @ dx[:, HIDDEN:]
    da0 = dh * (cache["a0"] > 0)
    g["W_in"] = cache["f"].T @ da0
    g["b_in"] = da0.sum(axis=0)
    return g


def adam_step(p, g, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba) of every parameter; state holds t, m, v."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    out = {}
    for k in p:
        m = state.setdefault("m", {}).get(k, np.zeros_like(p[k]))
        v = state.setdefault("v", {}).get(k, np.zeros_like(p[k]))
        m = b1 * m + (1 - b1) * g[k]
        v = b2 * v + (1 - b2) * g[k] ** 2
        state["m"][k], state["v"][k] = m, v
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        out[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
    return out
