"""Oracle GSPM time step with magnetostatics and magnetostriction (Sec. 2, App. B).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings where the paper is silent or ambiguous (the CUDA library follows the same ones):
* Fields are nodal (P1).  The nonlinear local field h is evaluated pointwise at the nodes and is
  zero at nodes that carry no magnetisation.
* The derivatives of Sec. 2.3 (H_d = F^ms U, E = -1/2 (F^ms u + ...)) are divided by the lumped
  mass, i.e. nodal gradients are volume-weighted patch averages of the element gradients.
* The reduced potential U = U~ / m_s solves K^ms U = F^ms_{ij,a} m_{j,a} (Eq. weak (a)); the
  local demagnetising field is h~_d = -grad U and the far field is -N_d m_bar (Sec. 2.1).
* Homogeneous strain of a free body: E_bar = <E0(m)> + C^-1 sigma_ext; the total strain is
  E = E_bar + sym grad u, with u from Eq. weak (b).
* Defect elements keep the host stiffness; E0 = 0 and m = 0 at non-magnetic nodes.  The GSPM
  systems (Eq. weak (c)) are assembled over ferromagnetic elements only (natural Neumann
  condition on the defect surface) and solved for the magnetic nodes.
* Node 0 (the first unique node) is pinned in K^ms (1 DOF) and K^mech (3 DOFs) (Sec. 2.5).
* Algorithm B.1 step 2 is the Gauss-Seidel sweep of the cited scheme: the second row uses
  m*_1 and g*_1 (the literal print, with m^n_1 and g^n_1, is available as row2_printed=True).
* h[m*] in step 3 re-evaluates the local terms (anisotropy, Zeeman, magnetoelastic with
  sigma = C (E - E0(m*))) and the far field -N_d m_bar* at m*; h~_d and E are held from step n.
* CG initial guesses: the right-hand-side field f for the GSPM solves, the previous step's
  solution for U and u (zero at the first step).
"""
from __future__ import annotations

import numpy as np

from . import fem
from .material import (Reduced, compliance_apply, contract, h_anisotropy, h_magnetoelastic,
                       spontaneous_strain, tensor_to_voigt, voigt_to_tensor)


def voigt_to_tensor_field(v):
    """[..., 6] Voigt (tensor shear) -> [..., 3, 3]."""
    v = np.asarray(v, dtype=np.float64)
    return np.stack([np.stack([v[..., 0], v[..., 5], v[..., 4]], -1),
                     np.stack([v[..., 5], v[..., 1], v[..., 3]], -1),
                     np.stack([v[..., 4], v[..., 3], v[..., 2]], -1)], -2)
from .mesh import WrappedMesh
from .solvers import cg


class System:
    """Assembled operators for one wrapped mesh, material and time step."""

    def __init__(self, wm: WrappedMesh, material: dict, dt: float, alpha: float,
                 rtol_gs=1e-7, rtol_ms=1e-7, rtol_mech=1e-7, max_iter=20000,
                 row2_printed=False, resolve_at_mstar=False):
        self.wm = wm
        self.red = red = Reduced(material, dt, alpha)
        self.rtol = dict(gs=rtol_gs, ms=rtol_ms, mech=rtol_mech)
        self.max_iter = max_iter
        self.row2_printed = row2_printed
        self.resolve_at_mstar = resolve_at_mstar
        n = wm.n
        # Omega_c operators (Eqs. LHS, RHS_F), node 0 pinned (Sec. 2.5)
        self.K_ms_raw = fem.stiffness(wm)
        self.K_ms = fem.pin(self.K_ms_raw, [0])
        self.F = fem.f_ms(wm)
        self.ML = fem.lumped_mass(wm)
        self.K_mech_raw = fem.k_mech(wm, red.C)
        self.K_mech = fem.pin(self.K_mech_raw, [0, 1, 2])
        self.F_mech = fem.f_mech(wm, red.C)
        # Omega_m operators for Eq. weak (c): (M + eps K) g = M f on the magnetic nodes
        me = wm.elem_magnetic
        self.mag = wm.node_magnetic
        idx = np.flatnonzero(self.mag)
        self.mag_idx = idx
        K_m = fem.stiffness(wm, me)
        M_m = fem.mass(wm, me)
        self.K_m, self.M_m_full = K_m, M_m
        self.M = M_m[idx][:, idx].tocsr()
        self.A_eps = (M_m + red.eps * K_m)[idx][:, idx].tocsr()
        self.A_aeps = (M_m + red.alpha * red.eps * K_m)[idx][:, idx].tocsr()
        self.E_ext = compliance_apply(material["C11"], material["C12"], material["C44"],
                                      red.sigma_ext, red.D)
        self.n = n

    # ---------------------------------------------------------------- pieces of the step
    def volume_average(self, g):
        return fem.volume_average(self.wm, g)

    def rhs_ms(self, m):
        """Eq. RHS_b divided by m_s: b_i = F^ms_{ij,a} m_{j,a}; pinned entry zeroed."""
        b = sum(self.F[a] @ m[:, a] for a in range(3))
        b[0] = 0.0
        return b

    def solve_ms(self, m, U0):
        b = self.rhs_ms(m)
        x0 = np.array(U0, dtype=np.float64, copy=True)
        x0[0] = 0.0
        return cg(self.K_ms, b, x0, self.rtol["ms"], self.max_iter)

    def demag_local(self, U):
        """h~_d = -grad U~ / m_s = (F^ms_a U)_i / M_L,i (Sec. 2.3)."""
        return -fem.nodal_gradient(self.F, self.ML, U)

    def e0_nodal(self, m):
        """Table A.1 at the nodes; rotated crystal (Algorithm D.1 step 1):
        E0_111 = M E0_100(m_100) with m_100 = R^-1 m_111."""
        red = self.red
        if red.rotated:
            m100 = m @ red.R            # rows: R^T m
            E0 = voigt_to_tensor_field(tensor_to_voigt(
                spontaneous_strain(m100, red.l100, red.l111)) @ red.M.T)
        else:
            E0 = spontaneous_strain(m, red.l100, red.l111)
        E0[~self.mag] = 0.0
        return E0

    def rhs_mech(self, E0):
        """Eq. RHS_b: b^mech = F^mech vec(E0); pinned entries zeroed."""
        b = self.F_mech @ E0.reshape(-1)
        b[0:3] = 0.0
        return b

    def solve_mech(self, E0, u0, rtol=None):
        b = self.rhs_mech(E0)
        x0 = np.array(u0, dtype=np.float64, copy=True).reshape(-1)
        x0[0:3] = 0.0
        x, k, rel = cg(self.K_mech, b, x0, self.rtol["mech"] if rtol is None else rtol,
                       self.max_iter)
        return x.reshape(-1, 3), k, rel

    def strain(self, u, E_bar):
        """E = E_bar + sym grad u with nodal gradients from F^ms (Sec. 2.3)."""
        G = np.stack([fem.nodal_gradient(self.F, self.ML, u[:, b]) for b in range(3)], axis=1)
        # G[i, b, a] = d_a u_b ; strain E_ab = (d_a u_b + d_b u_a) / 2
        return E_bar[None] + 0.5 * (G + np.transpose(G, (0, 2, 1)))

    def h_field(self, m, m_bar, hd_local, sigma, H):
        """h(m) = h_anis + H_ext / m_s + h_me + h~_d - N_d m_bar (App. B), zero where there is
        no magnetisation."""
        red = self.red
        if red.rotated:
            # Algorithm D.1 step 4: the crystal terms at m_100 = R^-1 m with the stress in the
            # crystal axes (sigma_100 = M^-1 sigma_111), then h_111 = R h_100
            m100 = m @ red.R
            s100 = voigt_to_tensor_field(np.linalg.solve(red.M, tensor_to_voigt(sigma).T).T)
            h_cr = (h_anisotropy(m100, red.kappa) + h_magnetoelastic(m100, s100, red)) @ red.R.T
        else:
            h_cr = h_anisotropy(m, red.kappa) + h_magnetoelastic(m, sigma, red)
        h = (h_cr + np.asarray(H, float)[None] / red.Ms + hd_local - (red.Nd @ m_bar)[None])
        h[~self.mag] = 0.0
        return h

    def gs_solve(self, A, f, rtol):
        """(M + c eps K) g = M f on the magnetic nodes, x0 = f; zero elsewhere."""
        idx = self.mag_idx
        fi = f[idx]
        x, k, rel = cg(A, self.M @ fi, fi, rtol, self.max_iter)
        g = np.zeros(self.n)
        g[idx] = x
        return g, k, rel

    # ---------------------------------------------------------------- elastic (stand-alone)
    def solve_elastic(self, m, u0, rtol=None):
        """Steps a5-a8: E0, E_bar, mechanical CG, nodal strain and stress."""
        E0 = self.e0_nodal(m)
        E_bar = self.volume_average(E0) + self.E_ext
        u, k, rel = self.solve_mech(E0, u0, rtol)
        E = self.strain(u, E_bar)
        sigma = contract(self.red.C, E - E0)
        return dict(u=u, E=E, E0=E0, E_bar=E_bar, sigma=sigma, iters=k, relres=rel)

    # ---------------------------------------------------------------- one GSPM step
    def step(self, m, U_prev, u_prev, H):
        """One step of Algorithm B.1 with the magnetostatic and mechanical solves.
        Returns (m_new, U, u, info)."""
        red = self.red
        rt = self.rtol["gs"]
        m = np.asarray(m, dtype=np.float64)
        m_bar = self.volume_average(m)                                # Sec. 2.4
        U, it_ms, res_ms = self.solve_ms(m, U_prev)                  # Eq. weak (a)
        hd = self.demag_local(U)
        el = self.solve_elastic(m, u_prev)                            # Eq. weak (b)
        E, u = el["E"], el["u"]
        h = self.h_field(m, m_bar, hd, el["sigma"], H)
        # Step 1 / Step 2 (Gauss-Seidel sweep)
        S = lambda f: self.gs_solve(self.A_eps, f, rt)                # (1 - A* dtau Lap)^-1
        its = []
        m1, m2, m3 = m[:, 0], m[:, 1], m[:, 2]
        if not self.row2_printed:
            g2, k, _ = S(m2 + red.dtau * h[:, 1]); its.append(k)
            g3, k, _ = S(m3 + red.dtau * h[:, 2]); its.append(k)
            ms1 = m1 + (g2 * m3 - g3 * m2)
            gs1, k, _ = S(ms1 + red.dtau * h[:, 0]); its.append(k)
            ms2 = m2 + (g3 * ms1 - gs1 * m3)
        else:
            g1, k, _ = S(m1 + red.dtau * h[:, 0]); its.append(k)
            g2, k, _ = S(m2 + red.dtau * h[:, 1]); its.append(k)
            g3, k, _ = S(m3 + red.dtau * h[:, 2]); its.append(k)
            ms1 = m1 + (g2 * m3 - g3 * m2)
            ms2 = m2 + (g3 * m1 - g1 * m3)
            gs1, k, _ = S(ms1 + red.dtau * h[:, 0]); its.append(k)
        gs2, k, _ = S(ms2 + red.dtau * h[:, 1]); its.append(k)
        ms3 = m3 + (gs1 * ms2 - gs2 * ms1)
        m_star = np.stack([ms1, ms2, ms3], axis=1)
        m_star[~self.mag] = 0.0
        # Step 3: damped solve with h re-evaluated at m*.  Default: local terms and far field at
        # m*, h~_d and E held from step n.  resolve_at_mstar: the magnetostatic and mechanical
        # equilibria are solved again at m* (x0 = the step-n solutions), so h[m*] is the whole
        # effective field of m*; U and u returned are then the solutions at m*.
        mbar_star = self.volume_average(m_star)
        if self.resolve_at_mstar:
            U, _, _ = self.solve_ms(m_star, U)
            hd = self.demag_local(U)
            el_star = self.solve_elastic(m_star, u)
            u, E, sigma_star = el_star["u"], el_star["E"], el_star["sigma"]
        else:
            sigma_star = contract(red.C, E - self.e0_nodal(m_star))
        h_star = self.h_field(m_star, mbar_star, hd, sigma_star, H)
        f = m_star + red.alpha * red.dtau * h_star
        m_ss = np.zeros_like(m)
        for c in range(3):
            m_ss[:, c], k, _ = self.gs_solve(self.A_aeps, f[:, c], rt)
            its.append(k)
        # Step 4: projection onto |m| = 1
        m_new = np.zeros_like(m)
        idx = self.mag_idx
        m_new[idx] = m_ss[idx] / np.linalg.norm(m_ss[idx], axis=1, keepdims=True)
        dm = float(np.mean(np.linalg.norm(m_new[idx] - m[idx], axis=1)))
        info = dict(it_ms=it_ms, res_ms=res_ms, it_mech=el["iters"], res_mech=el["relres"],
                    it_gs=its, m_bar=m_bar, h=h, hd=hd, E=E, sigma=el["sigma"], E0=el["E0"],
                    E_bar=el["E_bar"], m_star=m_star, h_star=h_star, dm=dm)
        return m_new, U, u, info

    # ---------------------------------------------------------------- energy (Eq. 1)
    def energy_density(self, m, U, u, H):
        """Average of Eq. 1's integrand over Omega_c (J/m^3), with the magnetostatic energy
        int_R3 mu0/2 |H_d|^2 taken through the ellipsoid split as
        (mu0 m_s^2 / 2) (m_bar . N_d m_bar + (1/V) int |grad U|^2).
        Exchange and magnetostatic parts are exact for P1 fields; local densities are integrated
        by the lumped mass of their domain."""
        red, wm = self.red, self.wm
        V = wm.volume
        mat = red.mat
        m = np.asarray(m, float)
        e_ex = mat["A"] / red.l_d ** 2 * sum(m[:, c] @ (self.K_m @ m[:, c]) for c in range(3)) / V
        ML_m = np.asarray(self.M_m_full.sum(axis=1)).ravel()
        m2 = (m @ red.R) ** 2 if red.rotated else m ** 2   # cube-axis components
        e_an = mat["K1"] * (ML_m @ (m2[:, 0] * m2[:, 1] + m2[:, 1] * m2[:, 2]
                                    + m2[:, 2] * m2[:, 0])) / V
        el_E0 = self.e0_nodal(m)
        E_bar = self.volume_average(el_E0) + self.E_ext
        E = self.strain(np.asarray(u, float).reshape(-1, 3), E_bar)
        D = E - el_E0
        e_el = 0.5 * (self.ML @ np.einsum("nij,nij->n", D, contract(red.C, D))) / V
        e_st = -np.einsum("ij,ij->", red.sigma_ext, E_bar)
        m_bar = self.volume_average(m)
        e_z = -red.mu0 * red.Ms * float(np.asarray(H, float) @ m_bar)
        e_d = 0.5 * red.scale * (m_bar @ red.Nd @ m_bar + U @ (self.K_ms_raw @ U) / V)
        return dict(total=e_ex + e_an + e_el + e_st + e_z + e_d, exchange=e_ex, anisotropy=e_an,
                    elastic=e_el, stress=e_st, zeeman=e_z, demag=e_d)


def run(system: System, m0, H, steps, U0=None, u0=None):
    """Advance `steps` GSPM steps from m0; returns (m, U, u, infos)."""
    m = np.array(m0, dtype=np.float64, copy=True)
    m[~system.mag] = 0.0
    U = np.zeros(system.n) if U0 is None else np.array(U0, float)
    u = np.zeros((system.n, 3)) if u0 is None else np.array(u0, float)
    infos = []
    for _ in range(steps):
        m, U, u, info = system.step(m, U, u, H)
        infos.append(info)
    return m, U, u, infos
