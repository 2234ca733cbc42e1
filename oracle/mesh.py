"""Oracle mesh layer: periodic wrap, adjacency, RCM ordering, element geometry.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

from collections import deque

import numpy as np


def default_wrap_tol(coords: np.ndarray, tets: np.ndarray) -> float:
    """1e-6 of the shortest distance between two vertices of an element."""
    X = coords[tets]
    k = tets.shape[1]
    e = []
    for a in range(k):
        for b in range(a + 1, k):
            e.append(np.linalg.norm(X[:, a] - X[:, b], axis=1).min())
    return 1e-6 * float(min(e))


def periodic_wrap(coords, box_lo, box_hi, tol):
    """Sec. 2.5 (Boundary conditions and solvers): a node whose coordinate along an axis lies at
    the domain's maximum extent is wrapped onto the minimum extent; a hash map keyed on the
    wrapped position then gives every set of matching nodes one global index.

    Keys are the wrapped coordinates quantised as floor((x - lo) / tol + 0.5).  Unique indices
    are handed out in stored-node order (first occurrence).  Returns (unique_of_stored, n_unique).
    """
    lo = np.asarray(box_lo, dtype=np.float64)
    hi = np.asarray(box_hi, dtype=np.float64)
    table = {}
    out = np.empty(coords.shape[0], dtype=np.int64)
    for s in range(coords.shape[0]):
        key = []
        for a in range(3):
            x = coords[s, a]
            if abs(x - hi[a]) <= tol:
                x = lo[a]
            key.append(int(np.floor((x - lo[a]) / tol + 0.5)))
        key = tuple(key)
        if key not in table:
            table[key] = len(table)
        out[s] = table[key]
    return out, len(table)


def node_adjacency(tets_u: np.ndarray, n: int):
    """Sorted neighbour lists (self included) of the node graph of the wrapped mesh."""
    nbr = [set() for _ in range(n)]
    for t in tets_u:
        for a in t:
            nbr[a].update(int(b) for b in t)
    return [sorted(s) for s in nbr]


def csr_pattern(tets_u: np.ndarray, n: int):
    """CSR row pointer and ascending column indices of the node graph (self included)."""
    adj = node_adjacency(tets_u, n)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum([len(a) for a in adj])
    cols = np.fromiter((c for a in adj for c in a), dtype=np.int64, count=int(rowptr[-1]))
    return rowptr, cols


def rcm_order(tets_u: np.ndarray, n: int) -> np.ndarray:
    """Reverse Cuthill-McKee order, perm[new] = old.

    Start at the unvisited node of smallest degree (ties: lowest index); breadth-first search
    that enqueues each node's unvisited neighbours sorted by (degree, index); repeat for every
    connected component; reverse the whole sequence.  Degree excludes the node itself.
    """
    adj = node_adjacency(tets_u, n)
    deg = [len(a) - 1 for a in adj]
    visited = [False] * n
    order = []
    by_degree = sorted(range(n), key=lambda v: (deg[v], v))
    for start in by_degree:
        if visited[start]:
            continue
        visited[start] = True
        q = deque([start])
        while q:
            v = q.popleft()
            order.append(v)
            nxt = [w for w in adj[v] if w != v and not visited[w]]
            nxt.sort(key=lambda w: (deg[w], w))
            for w in nxt:
                visited[w] = True
                q.append(w)
    return np.array(order[::-1], dtype=np.int64)


def element_geometry(coords: np.ndarray, tets: np.ndarray):
    """Linear tetrahedron geometry from the stored (unwrapped) vertex coordinates.

    J = [x1 - x0, x2 - x0, x3 - x0] (columns), V = det(J) / 6, grad(phi_1..3) = rows of J^-1,
    grad(phi_0) = -(sum of the others).  Returns (V [Ne], grads [Ne, 4, 3], detJ [Ne]).
    """
    X = coords[tets]
    J = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], axis=2)
    det = np.linalg.det(J)
    Jinv = np.linalg.inv(J)
    grads = np.empty((tets.shape[0], 4, 3))
    grads[:, 1:, :] = Jinv
    grads[:, 0, :] = -Jinv.sum(axis=1)
    return det / 6.0, grads, det


# Linear hexahedron: reference corners s_a in the element's vertex order, 2x2x2 Gauss points
# xi_q = s_q / sqrt(3) with unit weights
HEX_SIGNS = np.array([(-1, -1, -1), (1, -1, -1), (1, 1, -1), (-1, 1, -1), (-1, -1, 1),
                      (1, -1, 1), (1, 1, 1), (-1, 1, 1)], dtype=np.float64)
HEX_GAUSS = HEX_SIGNS / np.sqrt(3.0)


def hex_shape(xi):
    """N_a(xi) = prod_d (1 + s_a,d xi_d) / 2 for points xi [..., 3] -> [..., 8]."""
    xi = np.asarray(xi, dtype=np.float64)
    return np.prod(0.5 * (1.0 + HEX_SIGNS * xi[..., None, :]), axis=-1)


def hex_shape_dxi(xi):
    """dN_a / dxi_d at points xi [..., 3] -> [..., 8, 3]."""
    xi = np.asarray(xi, dtype=np.float64)
    f = 0.5 * (1.0 + HEX_SIGNS * xi[..., None, :])           # [..., 8, 3]
    out = np.empty(f.shape)
    for d in range(3):
        others = [e for e in range(3) if e != d]
        out[..., d] = 0.5 * HEX_SIGNS[:, d] * f[..., others[0]] * f[..., others[1]]
    return out


def hex_geometry(coords: np.ndarray, hexes: np.ndarray):
    """Trilinear hexahedron geometry at the 2x2x2 Gauss points from the stored vertices:
    J_q = sum_a x_a (x) dN_a/dxi (J_ij = dx_i / dxi_j), weights w_eq = det J_q, physical
    gradients grad N_a = J_q^-T dN_a/dxi.  Returns (w [Ne, 8], N [8 q, 8 a], G [Ne, 8 q, 8 a, 3],
    detJ [Ne, 8])."""
    X = coords[hexes]                                           # [Ne, 8, 3]
    dN = hex_shape_dxi(HEX_GAUSS)                              # [8 q, 8 a, 3]
    J = np.einsum("eai,qaj->eqij", X, dN)
    det = np.linalg.det(J)
    Jinv = np.linalg.inv(J)                                    # [Ne, 8, 3, 3] (j, i)
    G = np.einsum("qaj,eqji->eqai", dN, Jinv)
    return det, hex_shape(HEX_GAUSS), G, det


def magnetic_nodes(tets_u: np.ndarray, elem_magnetic: np.ndarray, n: int) -> np.ndarray:
    """A node carries magnetisation iff it belongs to at least one ferromagnetic element."""
    mask = np.zeros(n, dtype=bool)
    mask[tets_u[elem_magnetic.astype(bool)].ravel()] = True
    return mask


class WrappedMesh:
    """A stored mesh after the periodic wrap, with per-element geometry: linear tetrahedra
    (``tets`` [Ne, 4]; V, grads, detJ) or trilinear hexahedra (``tets`` [Ne, 8]; Gauss weights
    gw [Ne, 8], shape values gN [8, 8], gradients gG [Ne, 8, 8, 3], V = sum of the weights)."""

    def __init__(self, coords, tets, elem_magnetic, box_lo, box_hi, tol=None):
        coords = np.asarray(coords, dtype=np.float64)
        tets = np.asarray(tets, dtype=np.int64)
        if tol is None or tol <= 0:
            tol = default_wrap_tol(coords, tets)
        self.tol = tol
        self.nen = tets.shape[1]
        self.unique_of_stored, self.n = periodic_wrap(coords, box_lo, box_hi, tol)
        self.tets = self.unique_of_stored[tets]                  # wrapped connectivity
        self.elem_magnetic = np.asarray(elem_magnetic).astype(bool)
        if self.nen == 8:
            self.gw, self.gN, self.gG, self.detJ = hex_geometry(coords, tets)
            self.V = self.gw.sum(axis=1)
            self.grads = None
            if np.any(self.detJ <= 0):
                raise ValueError("mesh has a hexahedron with det J <= 0 at a Gauss point")
        else:
            self.V, self.grads, self.detJ = element_geometry(coords, tets)
            if np.any(self.detJ <= 0):
                raise ValueError("mesh has a non-positively oriented tetrahedron")
        self.node_magnetic = magnetic_nodes(self.tets, self.elem_magnetic, self.n)
        self.volume = float(self.V.sum())

    @classmethod
    def from_synth(cls, mesh, tol=None):
        return cls(mesh.coords, mesh.tets, mesh.elem_magnetic, mesh.box_lo, mesh.box_hi, tol)
