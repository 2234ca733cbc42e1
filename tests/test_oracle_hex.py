"""Pins of the oracle's trilinear hexahedra (the paper's second element type, Sec. 3) against
results that do not come from the oracle's code.

* Element matrices of an axis-aligned box element against tensor products of the 1-D linear
  element matrices (stiffness k = [[1, -1], [-1, 1]] / h, mass m = h [[2, 1], [1, 2]] / 6,
  derivative-times-value c_kl = int N_k N_l' = [[-1, 1], [-1, 1]] / 2), written out here.
* Linear patch tests on an open, jittered patch: K (linear) = 0 and K^mech (linear) = 0 at
  interior nodes, and the nodal gradient of a linear field is exact there.
* Periodic mesh: K 1 = 0, F_a 1 = 0, F_a = -F_a^T, sum M = V, lumped mass = row sums of M; on
  the unjittered lattice every node's lumped mass is h^3.
* Unjittered periodic lattice: Fourier modes are eigenvectors of K and M with the symbols
  k(t) m(t) m(t) + ... built from the 1-D symbols (2 - 2 cos t) / h and h (4 + 2 cos t) / 6, so
  the GSPM solve gives g = lambda_M / (lambda_M + eps lambda_K) f in closed form.
"""
import numpy as np
import pytest

from oracle import fem
from oracle.gspm import System
from oracle.material import Reduced
from oracle.mesh import WrappedMesh
from paper_2510_09812_gb300 import synth


def _kron3(ax, ay, az):
    """Tensor product matrix over the 8 vertices, index ix + 2 iy + 4 iz."""
    return np.kron(az, np.kron(ay, ax))


def _one_element(hx, hy, hz):
    """A single open box element [0,hx] x [0,hy] x [0,hz] (no periodic identification); its
    stored node s = ix + 2 (iy + 2 iz) is the tensor-product index of _kron3."""
    mesh = synth.hex_box((1, 1, 1), (hx, hy, hz))
    wm = WrappedMesh(mesh.coords, mesh.tets, mesh.elem_magnetic, mesh.box_lo,
                     np.array([hx, hy, hz]) + 1e6)
    assert wm.n == 8 and np.array_equal(wm.unique_of_stored, np.arange(8))
    return mesh, wm


def _oned(h):
    k = np.array([[1.0, -1.0], [-1.0, 1.0]]) / h
    m = h * np.array([[2.0, 1.0], [1.0, 2.0]]) / 6.0
    c = 0.5 * np.array([[-1.0, 1.0], [-1.0, 1.0]])   # c_kl = int N_k N_l'
    return k, m, c


def test_box_element_matrices_are_tensor_products():
    hx, hy, hz = 2.0, 3.0, 5.0
    mesh, wm = _one_element(hx, hy, hz)
    (kx, mx, cx), (ky, my, cy), (kz, mz, cz) = _oned(hx), _oned(hy), _oned(hz)
    K = fem.stiffness(wm).toarray()
    M = fem.mass(wm).toarray()
    Kexp = _kron3(kx, my, mz) + _kron3(mx, ky, mz) + _kron3(mx, my, kz)
    Mexp = _kron3(mx, my, mz)
    assert np.allclose(K, Kexp, rtol=0, atol=1e-13 * np.abs(Kexp).max())
    assert np.allclose(M, Mexp, rtol=0, atol=1e-13 * np.abs(Mexp).max())
    F = [f.toarray() for f in fem.f_ms(wm)]
    # F_a = -int phi_k d_a phi_l
    Fexp = [-_kron3(cx, my, mz), -_kron3(mx, cy, mz), -_kron3(mx, my, cz)]
    for a in range(3):
        assert np.allclose(F[a], Fexp[a], rtol=0, atol=1e-13)
    assert np.allclose(fem.lumped_mass(wm), np.full(8, hx * hy * hz / 8), rtol=1e-14)
    # elasticity: D_cd[k, l] = int d_c N_k d_d N_l from the 1-D factors
    one = {0: (kx, cx, mx), 1: (ky, cy, my), 2: (kz, cz, mz)}

    def D(c, d):
        fac = []
        for ax in range(3):
            kk, cc, mm = one[ax]
            if ax == c and ax == d:
                fac.append(kk)
            elif ax == c:
                fac.append(cc.T)          # int N_k' N_l
            elif ax == d:
                fac.append(cc)            # int N_k N_l'
            else:
                fac.append(mm)
        return _kron3(*fac)

    mat = synth.fe_like_material()
    C = Reduced(mat, 1e-12, 0.5).C
    Km = fem.k_mech(wm, C).toarray()
    Kexp = np.zeros((24, 24))
    for a in range(3):
        for b in range(3):
            blk = sum(C[a, c, b, d] * D(c, d) for c in range(3) for d in range(3))
            Kexp[a::3, b::3] = blk
    assert np.allclose(Km, Kexp, rtol=0, atol=1e-12 * np.abs(Kexp).max())


def _open_patch(n_cells=(4, 4, 3), box=(16.0, 16.0, 12.0), jitter=0.2, seed=5):
    mesh = synth.hex_box(n_cells, box, jitter=jitter, seed=seed)
    far = np.asarray(box, float) + 1e6
    wm = WrappedMesh(mesh.coords, mesh.tets, mesh.elem_magnetic, mesh.box_lo, far)
    nx, ny, nz = n_cells
    s = np.arange(mesh.n_stored)
    i, j, k = s % (nx + 1), (s // (nx + 1)) % (ny + 1), s // ((nx + 1) * (ny + 1))
    interior = (i > 0) & (i < nx) & (j > 0) & (j < ny) & (k > 0) & (k < nz)
    return mesh, wm, interior


def test_linear_patch_tests_on_a_jittered_patch():
    mesh, wm, interior = _open_patch()
    x = mesh.coords
    lin = 0.3 + 1.2 * x[:, 0] - 0.7 * x[:, 1] + 2.1 * x[:, 2]
    K = fem.stiffness(wm)
    assert np.abs((K @ lin)[interior]).max() < 1e-11 * np.abs(K).max() * np.abs(lin).max()
    F = fem.f_ms(wm)
    ML = fem.lumped_mass(wm)
    grad = fem.nodal_gradient(F, ML, lin)
    assert np.allclose(grad[interior], [1.2, -0.7, 2.1], rtol=0, atol=1e-12)
    # elasticity: a linear displacement field (strain constant) is in equilibrium inside
    mat = synth.fe_like_material()
    C = Reduced(mat, 1e-12, 0.5).C
    Bm = np.array([[0.1, -0.2, 0.05], [0.3, 0.0, -0.1], [0.02, 0.04, -0.3]])
    u = x @ Bm.T + np.array([1.0, -2.0, 0.5])
    Km = fem.k_mech(wm, C)
    r = (Km @ u.reshape(-1)).reshape(-1, 3)
    assert np.abs(r[interior]).max() < 1e-11 * np.abs(Km).max() * np.abs(u).max()


def test_periodic_hex_operators_invariants():
    mesh = synth.hex_box((6, 5, 4), (24.0, 20.0, 16.0), jitter=0.2, seed=7,
                         defects=[dict(kind="sphere", center=(12.0, 10.0, 8.0), radius=4.5)])
    wm = WrappedMesh.from_synth(mesh)
    one = np.ones(wm.n)
    K = fem.stiffness(wm)
    M = fem.mass(wm)
    assert np.abs(K @ one).max() < 1e-12 * np.abs(K).max()
    assert abs(M.sum() - 24.0 * 20.0 * 16.0) < 1e-10
    assert np.abs((K - K.T)).max() < 1e-14 * np.abs(K).max()
    assert np.allclose(fem.lumped_mass(wm), np.asarray(M.sum(axis=1)).ravel(), rtol=1e-13)
    for Fa in fem.f_ms(wm):
        assert np.abs(Fa @ one).max() < 1e-12 * np.abs(Fa).max()
        assert np.abs(Fa + Fa.T).max() < 1e-12 * np.abs(Fa).max()
    # volume average on the unjittered lattice: every node carries the lumped mass h^3, so the
    # average of any nodal field is its nodal mean
    flat = synth.hex_box((6, 5, 4), (24.0, 20.0, 16.0))
    wf = WrappedMesh.from_synth(flat)
    lat = np.stack([(np.arange(wf.n) % 6) * 4.0, ((np.arange(wf.n) // 6) % 5) * 4.0,
                    (np.arange(wf.n) // 30) * 4.0], axis=1)
    g = np.cos(2 * np.pi * lat[:, 0] / 24.0) + 0.5 + 0.01 * lat[:, 2]
    assert fem.volume_average(wf, g) == pytest.approx(g.mean(), rel=1e-14)
    assert np.allclose(fem.lumped_mass(wf), 64.0, rtol=1e-14)


def test_gspm_solve_fourier_closed_form():
    """Unjittered periodic hex lattice, one Fourier mode f = cos(k . x): (M + eps K) g = M f
    has g = lambda_M / (lambda_M + eps lambda_K) f with the tensor-product symbols."""
    cells, box = (8, 6, 4), (32.0, 24.0, 16.0)
    mesh = synth.hex_box(cells, box)
    wm = WrappedMesh.from_synth(mesh)
    s = System(wm, synth.fe_like_material(), 1e-12, 0.5, rtol_gs=1e-14)
    h = np.array(box) / np.array(cells)
    u = np.arange(wm.n)
    idx = np.stack([u % cells[0], (u // cells[0]) % cells[1], u // (cells[0] * cells[1])], axis=1)
    kvec = (2, 1, 1)
    theta = [2 * np.pi * kvec[a] / cells[a] for a in range(3)]
    phase = sum(theta[a] * idx[:, a] for a in range(3))
    f = np.cos(phase)
    k1 = [(2 - 2 * np.cos(theta[a])) / h[a] for a in range(3)]
    m1 = [h[a] * (4 + 2 * np.cos(theta[a])) / 6 for a in range(3)]
    lamK = k1[0] * m1[1] * m1[2] + m1[0] * k1[1] * m1[2] + m1[0] * m1[1] * k1[2]
    lamM = m1[0] * m1[1] * m1[2]
    eps = s.red.eps
    g, it, rel = s.gs_solve(s.A_eps, f, 1e-14)
    expect = lamM / (lamM + eps * lamK) * f
    assert np.abs(g - expect).max() < 1e-12
    # and the stiffness symbol directly
    assert np.abs(s.K_ms_raw @ f - lamK * f).max() < 1e-12 * lamK
