"""Oracle finite-element operators on the wrapped periodic mesh (Sec. 2.3 - 2.5).

TEST INFRASTRUCTURE ONLY (see the package docstring).

All matrices are assembled element by element and summed into SciPy CSR (COO -> CSR adds the
duplicates).  Linear tetrahedra: with linear shape functions and the one-point (centroid) rule
of Sec. 2.4 every integral below is exact:
  int_e grad(phi_k) . grad(phi_l)    = V grad(phi_k) . grad(phi_l)
  int_e phi_k phi_l                  = V (1 + delta_kl) / 20
  int_e phi_k                        = V / 4
Trilinear hexahedra (the paper's other element, Sec. 3): every integral is the 2x2x2 Gauss sum
sum_q w_q (integrand at xi_q), w_q = det J at the point (exact for the mass and the lumped mass,
and for every integral on parallelepipeds).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def _scatter_scalar(tets, vals, n):
    """Sum element matrices vals [Ne, k, k] into an n x n CSR matrix."""
    k = tets.shape[1]
    rows = np.repeat(tets[:, :, None], k, axis=2)
    cols = np.repeat(tets[:, None, :], k, axis=1)
    return sp.coo_matrix((vals.ravel(), (rows.ravel(), cols.ravel())), shape=(n, n)).tocsr()


def stiffness(wm, elems=None):
    """K_ij = int grad(phi_i) . grad(phi_j) (Eq. LHS, K^ms; and the Laplacian part of K^GS),
    over the selected elements (all of Omega_c by default)."""
    sel = slice(None) if elems is None else elems
    if wm.nen == 8:
        Ke = np.einsum("eq,eqka,eqla->ekl", wm.gw[sel], wm.gG[sel], wm.gG[sel])
        return _scatter_scalar(wm.tets[sel], Ke, wm.n)
    g, V, t = wm.grads[sel], wm.V[sel], wm.tets[sel]
    Ke = V[:, None, None] * np.einsum("eka,ela->ekl", g, g)
    return _scatter_scalar(t, Ke, wm.n)


def mass(wm, elems=None):
    """Consistent mass M_ij = int phi_i phi_j (Eq. RHS_F, F^GS) over the selected elements."""
    sel = slice(None) if elems is None else elems
    if wm.nen == 8:
        Me = np.einsum("eq,qk,ql->ekl", wm.gw[sel], wm.gN, wm.gN)
        return _scatter_scalar(wm.tets[sel], Me, wm.n)
    V, t = wm.V[sel], wm.tets[sel]
    Me = V[:, None, None] * (np.ones((4, 4)) + np.eye(4))[None] / 20.0
    return _scatter_scalar(t, Me, wm.n)


def lumped_mass(wm):
    """Row sums of the consistent mass over Omega_c: M_L,i = sum_{e containing i} int_e phi_i
    (V_e / 4 on a tetrahedron)."""
    ML = np.zeros(wm.n)
    if wm.nen == 8:
        np.add.at(ML, wm.tets.ravel(), np.einsum("eq,qk->ek", wm.gw, wm.gN).ravel())
        return ML
    np.add.at(ML, wm.tets.ravel(), np.repeat(wm.V / 4.0, 4))
    return ML


def f_ms(wm):
    """Eq. RHS_F: (F^ms)_{ij,a} = -int phi_i d_a phi_j, returned as three n x n CSR matrices."""
    out = []
    for a in range(3):
        if wm.nen == 8:
            Fe = -np.einsum("eq,qk,eql->ekl", wm.gw, wm.gN, wm.gG[..., a])
        else:
            Fe = -(wm.V / 4.0)[:, None, None] * np.repeat(wm.grads[:, None, :, a], 4, axis=1)
        out.append(_scatter_scalar(wm.tets, Fe, wm.n))
    return out


def k_mech(wm, C):
    """Eq. LHS: (K^mech)_{(i,a),(j,b)} = int E(phi_j e_b) : C E(phi_i e_a).  With E(phi e_a) the
    symmetric part of e_a (x) grad(phi) and C minor-symmetric this is
    sum_e V_e sum_{c,d} d_c phi_i C_{acbd} d_d phi_j.  DOF (i, a) -> 3 i + a."""
    t = wm.tets
    if wm.nen == 8:
        Ke = np.einsum("eq,eqkc,acbd,eqld->ekalb", wm.gw, wm.gG, C, wm.gG)   # [Ne,8,3,8,3]
    else:
        g, V = wm.grads, wm.V
        Ke = V[:, None, None, None, None] * np.einsum("ekc,acbd,eld->ekalb", g, C, g)
    dof = 3 * t[:, :, None] + np.arange(3)[None, None, :]                         # [Ne,k,3]
    rows = np.broadcast_to(dof[:, :, :, None, None], Ke.shape)
    cols = np.broadcast_to(dof[:, None, None, :, :], Ke.shape)
    n3 = 3 * wm.n
    return sp.coo_matrix((Ke.ravel(), (rows.ravel(), cols.ravel())), shape=(n3, n3)).tocsr()


def f_mech(wm, C):
    """Eq. RHS_F: (F^mech)_{(i,a),(j,rs)} = 1/2 int E(phi_i e_a) : C phi_j (e_r (x) e_s + e_s (x) e_r)
    = sum_e (V_e / 4) sum_q d_q phi_i C_{aqrs}  (C minor-symmetric).
    Shape (3n, 9n); column (j, r, s) -> 9 j + 3 r + s, so that b^mech = F^mech vec(E0) with E0
    stored as full symmetric 3x3 tensors (Eq. RHS_b)."""
    t = wm.tets
    k = t.shape[1]
    # element block [Ne, k (i), 3 (a), k (j), 3 (r), 3 (s)]
    if wm.nen == 8:
        blk = np.einsum("eq,eqic,acrs,qj->eiajrs", wm.gw, wm.gG, C, wm.gN)
    else:
        g, V = wm.grads, wm.V
        blk = np.einsum("eiq,aqrs->eiars", g, C) * (V / 4.0)[:, None, None, None, None]
        blk = np.broadcast_to(blk[:, :, :, None, :, :], (t.shape[0], 4, 3, 4, 3, 3))
    rows = 3 * t[:, :, None, None, None, None] + np.arange(3)[None, None, :, None, None, None]
    cols = (9 * t[:, None, None, :, None, None] + 3 * np.arange(3)[None, None, None, None, :, None]
            + np.arange(3)[None, None, None, None, None, :])
    rows = np.broadcast_to(rows, blk.shape)
    cols = np.broadcast_to(cols, blk.shape)
    return sp.coo_matrix((np.ascontiguousarray(blk).ravel(), (rows.ravel(), cols.ravel())),
                         shape=(3 * wm.n, 9 * wm.n)).tocsr()


def pin(A, dofs):
    """Sec. 2.5: K is PSD with a kernel of constants; pinning d DOFs to zero makes the reduced
    matrix SPD.  Zero the pinned rows and columns and put 1 on their diagonal."""
    keep = np.ones(A.shape[0])
    keep[list(dofs)] = 0.0
    D = sp.diags(keep)
    return (D @ A @ D + sp.diags(1.0 - keep)).tocsr()


def nodal_gradient(F, ML, v):
    """Spatial derivative by the F^ms matrices (Sec. 2.3, derivatives by F^ms).  F_a represents
    -d_a weighted by the test function, so the nodal value divides by the lumped mass:
    (d_a v)_i = -(F_a v)_i / M_L,i.  Returns [n, 3]."""
    return np.stack([-(F[a] @ v) / ML for a in range(3)], axis=1)


def volume_average(wm, g):
    """Sec. 2.4 volume average by element-wise Gauss quadrature (one centroid point, weight 1/6 on
    the reference tetrahedron, |J| = 6 V): gather nodal values per element (g_node [Ne, 4, n]),
    interpolate to the Gauss point with phi_i(r_p) = 1/4, sum g_e |J| w over elements and divide
    by sum |J| w."""
    g = np.asarray(g, dtype=np.float64)
    gn = g[wm.tets]                                  # [Ne, k, ...]
    if wm.nen == 8:
        # hexahedra: the 2x2x2 Gauss points, weights det J_q
        gq = np.einsum("qi,ei...->eq...", wm.gN, gn)
        return np.einsum("eq,eq...->...", wm.gw, gq) / wm.gw.sum()
    phi = np.full(4, 0.25)
    ge = np.einsum("i,ei...->e...", phi, gn)         # value at the Gauss point
    w = wm.detJ * (1.0 / 6.0)
    return np.einsum("e,e...->...", w, ge) / w.sum()
