"""Oracle material laws: reduced constants, cubic stiffness, spontaneous strain, local fields,
ellipsoid demagnetising factors.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Units: lengths of the mesh in l_d = 1 nm, stresses and stiffness in Pa, fields in A/m.  Fields
entering the LLG equation are reduced by m_s (h = H / m_s), energies by mu0 m_s^2 (App. B).
"""
from __future__ import annotations

import numpy as np


class Reduced:
    """Dimensionless constants of App. B: A* = 2A / (mu0 ms^2 l_d^2), tau = gamma ms t."""

    def __init__(self, mat: dict, dt: float, alpha: float):
        self.mat = mat
        self.Ms = mat["Ms"]
        self.mu0 = mat.get("mu0", 1.25663706212e-6)
        self.gamma0 = mat.get("gamma0", 2.2127615e5)
        self.l_d = mat.get("l_d", 1e-9)
        self.scale = self.mu0 * self.Ms ** 2                       # mu0 ms^2, J/m^3
        self.A_star = 2.0 * mat["A"] / (self.scale * self.l_d ** 2)
        self.kappa = 2.0 * mat["K1"] / self.scale                   # anisotropy field coefficient
        self.dtau = self.gamma0 * self.Ms * dt
        self.alpha = alpha
        self.eps = self.A_star * self.dtau                          # (1 - eps Lap), Algorithm B.1
        # App. D: crystal axes rotated against the mesh axes by R (v_mesh = R v_crystal);
        # absent or identity = the mesh axes are the cube axes
        R = np.asarray(mat.get("R", np.eye(3)), dtype=np.float64).reshape(3, 3)
        self.R = R
        self.rotated = not np.array_equal(R, np.eye(3))
        self.M = bond_matrix(R)
        self.D100 = voigt_stiffness(mat["C11"], mat["C12"], mat["C44"])
        # stiffness in the mesh axes: C_111 = M C_100 M^T (Algorithm D.1, first line)
        self.D = self.M @ self.D100 @ self.M.T if self.rotated else self.D100
        self.C = (stiffness_from_voigt(self.D) if self.rotated
                  else cubic_stiffness(mat["C11"], mat["C12"], mat["C44"]))
        self.Nd = np.asarray(mat["Nd"], dtype=np.float64).reshape(3, 3)
        self.sigma_ext = voigt_to_tensor(np.asarray(mat.get("sigma_ext", [0.0] * 6), float))
        self.l100 = mat["lambda100"]
        self.l111 = mat["lambda111"]


def cubic_stiffness(C11, C12, C44) -> np.ndarray:
    """Fourth-order elastic stiffness C_ijkl of a cubic crystal in its cube axes: C_iiii = C11,
    C_iijj = C12 (i != j), C_ijij = C_ijji = C44 (i != j), all other entries zero."""
    C = np.zeros((3, 3, 3, 3))
    for i in range(3):
        for j in range(3):
            if i == j:
                C[i, i, i, i] = C11
            else:
                C[i, i, j, j] = C12
                C[i, j, i, j] = C44
                C[i, j, j, i] = C44
    return C


def rotation_111() -> np.ndarray:
    """App. D: mesh axes along <111>, <-110>, <11-2> of the crystal (rows of R)."""
    return np.array([[1 / np.sqrt(3), 1 / np.sqrt(3), 1 / np.sqrt(3)],
                     [-1 / np.sqrt(2), 1 / np.sqrt(2), 0.0],
                     [-1 / np.sqrt(6), -1 / np.sqrt(6), 2 / np.sqrt(6)]])


# Voigt index pairs in the order (11, 22, 33, 23, 13, 12)
_VP = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]


def bond_matrix(R: np.ndarray) -> np.ndarray:
    """App. D's 6 x 6 matrix M of a rotation R: E_111 = M E_100 for strain vectors with tensor
    shear components (and for stress vectors), C_111 = M C_100 M^T for the Voigt stiffness of
    engineering strain.  Entry (I, J), I = (i, j), J = (k, l): R_ik R_jl for k = l, and
    R_ik R_jl + R_il R_jk for k != l (the symmetric pair counted once)."""
    M = np.zeros((6, 6))
    for I, (i, j) in enumerate(_VP):
        for J, (k, l) in enumerate(_VP):
            M[I, J] = R[i, k] * R[j, l] + (R[i, l] * R[j, k] if k != l else 0.0)
    return M


def voigt_stiffness(C11, C12, C44) -> np.ndarray:
    """Cubic stiffness as the 6 x 6 matrix of sigma_v = D eps_v with engineering shear
    eps_v = (E11, E22, E33, 2E23, 2E13, 2E12)."""
    D = np.zeros((6, 6))
    D[:3, :3] = C12
    np.fill_diagonal(D[:3, :3], C11)
    D[3, 3] = D[4, 4] = D[5, 5] = C44
    return D


def stiffness_from_voigt(D: np.ndarray) -> np.ndarray:
    """C_ijkl = D[v(ij), v(kl)] for the engineering-shear Voigt matrix D (minor symmetric)."""
    v = np.zeros((3, 3), dtype=int)
    for I, (i, j) in enumerate(_VP):
        v[i, j] = v[j, i] = I
    C = np.zeros((3, 3, 3, 3))
    for i in range(3):
        for j in range(3):
            for k in range(3):
                for l in range(3):
                    C[i, j, k, l] = D[v[i, j], v[k, l]]
    return C


def tensor_to_voigt(E: np.ndarray) -> np.ndarray:
    """Symmetric [..., 3, 3] -> [..., 6] in the order (11, 22, 33, 23, 13, 12), tensor shear."""
    return np.stack([E[..., i, j] for i, j in _VP], axis=-1)


def voigt_to_tensor(v) -> np.ndarray:
    """Voigt order (11, 22, 33, 23, 13, 12) -> symmetric 3x3 tensor (tensor shear components)."""
    v = np.asarray(v, dtype=np.float64)
    return np.array([[v[0], v[5], v[4]], [v[5], v[1], v[3]], [v[4], v[3], v[2]]])


def spontaneous_strain(m: np.ndarray, l100: float, l111: float) -> np.ndarray:
    """Table A.1: E0(m) = 3/2 [lambda100 (m_i^2 - 1/3) on the diagonal, lambda111 m_i m_j off it].
    m: [..., 3] -> [..., 3, 3]."""
    outer = m[..., :, None] * m[..., None, :]
    E0 = 1.5 * l111 * outer
    for i in range(3):
        E0[..., i, i] = 1.5 * l100 * (m[..., i] ** 2 - 1.0 / 3.0)
    return E0


def contract(C: np.ndarray, E: np.ndarray) -> np.ndarray:
    """sigma_ij = C_ijkl E_kl for a field of tensors E [..., 3, 3]."""
    return np.einsum("ijkl,...kl->...ij", C, E)


def h_anisotropy(m: np.ndarray, kappa: float) -> np.ndarray:
    """-(1/(mu0 ms^2)) d/dm of K1 (m1^2 m2^2 + m2^2 m3^2 + m3^2 m1^2) (Eq. 1):
    h_1 = -kappa m1 (m2^2 + m3^2), cyclic, with kappa = 2 K1 / (mu0 ms^2)."""
    m2 = m ** 2
    return -kappa * m * (m2.sum(axis=-1, keepdims=True) - m2)


def h_magnetoelastic(m: np.ndarray, sigma: np.ndarray, red: Reduced) -> np.ndarray:
    """-(1/(mu0 ms^2)) d/dm of 1/2 (E - E0(m)) : C (E - E0(m)) = (1/(mu0 ms^2)) (dE0/dm) : sigma,
    sigma = C (E - E0).  With Table A.1's E0 this is
    h_1 = (3 / (mu0 ms^2)) [lambda100 m1 s11 + lambda111 (m2 s12 + m3 s13)], cyclic."""
    out = np.empty_like(m)
    for i in range(3):
        j, k = (i + 1) % 3, (i + 2) % 3
        out[..., i] = (red.l100 * m[..., i] * sigma[..., i, i]
                       + red.l111 * (m[..., j] * sigma[..., i, j] + m[..., k] * sigma[..., i, k]))
    return 3.0 / red.scale * out


# --------------------------------------------------------------------------------------------
# Ellipsoid demagnetising tensor (Sec. 2.1, ellipsoid theorem) via Carlson's R_D
# --------------------------------------------------------------------------------------------

def carlson_rd(x: float, y: float, z: float) -> float:
    """Carlson's symmetric elliptic integral of the second kind,
    R_D(x, y, z) = 3/2 int_0^inf dt / ((t+x)^(1/2) (t+y)^(1/2) (t+z)^(3/2)),
    by the duplication theorem R_D(x,y,z) = R_D(x',y',z') / 4 + 3 / (sqrt(z) (z + lam)) with
    x' = (x + lam) / 4 etc., lam = sqrt(xy) + sqrt(xz) + sqrt(yz), iterated until the arguments
    agree to 1e-10 relative; the remainder R_D(mu, mu, mu) = mu^(-3/2) at the weighted mean
    mu = (x + y + 3z) / 5 carries an error second order in the spread."""
    total, fac = 0.0, 1.0
    for _ in range(200):
        mu = (x + y + 3.0 * z) / 5.0
        spread = max(abs(mu - x), abs(mu - y), abs(mu - z)) / mu
        if spread < 1e-10:
            return total + fac * mu ** -1.5
        sx, sy, sz = np.sqrt(x), np.sqrt(y), np.sqrt(z)
        lam = sx * sy + sx * sz + sy * sz
        total += fac * 3.0 / (sz * (z + lam))
        fac *= 0.25
        x, y, z = (x + lam) / 4.0, (y + lam) / 4.0, (z + lam) / 4.0
    raise RuntimeError("R_D did not converge")


def ellipsoid_demag_factors(a: float, b: float, c: float) -> np.ndarray:
    """Diagonal demagnetising factors of an ellipsoid with semi-axes a, b, c along x, y, z:
    N_x = (abc / 3) R_D(b^2, c^2, a^2), cyclic; trace 1."""
    p = a * b * c / 3.0
    return np.array([p * carlson_rd(b * b, c * c, a * a),
                     p * carlson_rd(c * c, a * a, b * b),
                     p * carlson_rd(a * a, b * b, c * c)])


def compliance_apply(C11: float, C12: float, C44: float, sigma: np.ndarray,
                     D: np.ndarray | None = None) -> np.ndarray:
    """E = C^-1 sigma: solve the Voigt system with engineering shear (sigma_v = D eps_v,
    eps_v = (E11, E22, E33, 2E23, 2E13, 2E12)) and return the tensor E.  D defaults to the cubic
    stiffness in its cube axes."""
    if D is None:
        D = voigt_stiffness(C11, C12, C44)
    s = np.asarray(sigma, dtype=np.float64)
    sv = np.array([s[0, 0], s[1, 1], s[2, 2], s[1, 2], s[0, 2], s[0, 1]])
    ev = np.linalg.solve(D, sv)
    return voigt_to_tensor(np.concatenate([ev[:3], ev[3:] / 2.0]))
