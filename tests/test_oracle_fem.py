"""Oracle assembly against closed forms: Kuhn-lattice stencils, patch tests, kernels,
antisymmetry, Voigt strain energy, and continuum limits of the magnetostatic and elastic solves."""
import numpy as np
import pytest

from oracle import fem
from oracle.material import cubic_stiffness
from oracle.solvers import cg
from oracle_helpers import lattice_xyz, open_patch, periodic


def _nid(cells, i, j, k):
    nx, ny, nz = cells
    return (i % nx) + nx * ((j % ny) + ny * (k % nz))


def test_unjittered_kuhn_stiffness_is_seven_point_stencil():
    # P1 Laplacian on the Kuhn (Freudenthal) triangulation = h x (7-point finite-difference
    # stencil): 6h on the diagonal, -h to the 6 axis neighbours, 0 to the 8 diagonal neighbours.
    cells, h = (6, 6, 6), 2.0
    mesh, wm = periodic(cells, (12.0, 12.0, 12.0))
    K = fem.stiffness(wm).toarray()
    i0 = _nid(cells, 2, 2, 2)
    expect = np.zeros(wm.n)
    expect[i0] = 6 * h
    for d in [(1, 0, 0), (0, 1, 0), (0, 0, 1)]:
        for s in (1, -1):
            expect[_nid(cells, 2 + s * d[0], 2 + s * d[1], 2 + s * d[2])] = -h
    assert np.allclose(K[i0], expect, rtol=0, atol=1e-13)


def test_unjittered_kuhn_mass_weights():
    # consistent mass: diag = 24 tets x (h^3/6) x 2/20 = 0.4 h^3; off-diagonal = (#tets on the
    # edge) x (h^3/6)/20 with 6 tets on an axis edge, 4 on a (1,1,0)-type face diagonal and 6 on
    # the (1,1,1) body diagonal; row sums h^3.
    cells, h = (6, 6, 6), 2.0
    mesh, wm = periodic(cells, (12.0, 12.0, 12.0))
    M = fem.mass(wm).toarray()
    i0 = _nid(cells, 3, 1, 2)
    expect = np.zeros(wm.n)
    expect[i0] = 48
    for d, w in [((1, 0, 0), 6), ((0, 1, 0), 6), ((0, 0, 1), 6), ((1, 1, 0), 4), ((1, 0, 1), 4),
                 ((0, 1, 1), 4), ((1, 1, 1), 6)]:
        for s in (1, -1):
            expect[_nid(cells, 3 + s * d[0], 1 + s * d[1], 2 + s * d[2])] = w
    assert np.allclose(M[i0] * 120 / h ** 3, expect, rtol=0, atol=1e-12)
    assert np.allclose(M.sum(axis=1), h ** 3, rtol=1e-14)


def test_periodic_kernels_and_antisymmetry():
    mesh, wm = periodic((5, 4, 3), (10.0, 8.0, 6.0), jitter=0.2, seed=4)
    K = fem.stiffness(wm)
    one = np.ones(wm.n)
    assert np.abs(K @ one).max() < 1e-12 * abs(K).max()
    assert abs(K - K.T).max() < 1e-14 * abs(K).max()
    F = fem.f_ms(wm)
    for a in range(3):
        # F_a represents -d_a: it kills constants, and with periodic boundaries
        # int phi_i d_a phi_j + int phi_j d_a phi_i = int d_a (phi_i phi_j) = 0
        assert np.abs(F[a] @ one).max() < 1e-12
        assert abs(F[a] + F[a].T).max() < 1e-12
    assert fem.mass(wm).sum() == pytest.approx(wm.volume, rel=1e-13)
    assert fem.lumped_mass(wm).sum() == pytest.approx(wm.volume, rel=1e-13)
    C = cubic_stiffness(243e9, 138e9, 122e9)
    Km = fem.k_mech(wm, C)
    assert abs(Km - Km.T).max() <= 1e-12 * abs(Km).max()
    for a in range(3):   # rigid translations
        t = np.zeros((wm.n, 3)); t[:, a] = 1.0
        assert np.abs(Km @ t.ravel()).max() < 1e-12 * abs(Km).max()


def test_linear_patch_scalar():
    # open jittered patch: K x (linear field) vanishes at interior rows and the F^ms recovery of
    # its gradient is exact at interior nodes
    mesh, wm, interior = open_patch((5, 5, 4), (10.0, 10.0, 8.0))
    g = np.array([0.3, -1.2, 0.7])
    v = mesh.coords @ g + 2.5
    K = fem.stiffness(wm)
    assert np.abs((K @ v)[interior]).max() < 1e-12
    grad = fem.nodal_gradient(fem.f_ms(wm), fem.lumped_mass(wm), v)
    assert np.allclose(grad[interior], g[None], rtol=0, atol=1e-12)


def _voigt_energy(E, C11, C12, C44):
    # textbook cubic strain energy density in Voigt form
    e = np.array([E[0, 0], E[1, 1], E[2, 2]])
    return 0.5 * (C11 * (e ** 2).sum() + 2 * C12 * (e[0] * e[1] + e[1] * e[2] + e[0] * e[2])
                  + 4 * C44 * (E[1, 2] ** 2 + E[0, 2] ** 2 + E[0, 1] ** 2))


def test_linear_patch_elastic_and_voigt_energy():
    C11, C12, C44 = 243e9, 138e9, 122e9
    mesh, wm, interior = open_patch((4, 4, 4), (8.0, 8.0, 8.0))
    G = np.array([[0.01, -0.02, 0.005], [0.03, -0.01, 0.0], [0.002, 0.004, 0.02]])
    u = mesh.coords @ G.T                                       # u = G x
    Km = fem.k_mech(wm, cubic_stiffness(C11, C12, C44))
    f = (Km @ u.ravel()).reshape(-1, 3)
    scale = abs(Km).max() * np.abs(u).max()
    assert np.abs(f[interior]).max() < 1e-12 * scale
    E = 0.5 * (G + G.T)
    assert 0.5 * u.ravel() @ (Km @ u.ravel()) == pytest.approx(
        wm.volume * _voigt_energy(E, C11, C12, C44), rel=1e-12)


def test_f_mech_kills_uniform_eigenstrain():
    mesh, wm = periodic((4, 4, 3), (8.0, 8.0, 6.0), jitter=0.2, seed=6)
    C = cubic_stiffness(243e9, 138e9, 122e9)
    Fm = fem.f_mech(wm, C)
    E0 = np.tile(np.array([[1.0, 0.2, -0.3], [0.2, -0.5, 0.1], [-0.3, 0.1, 0.4]]), (wm.n, 1, 1))
    b = Fm @ E0.reshape(-1)
    assert np.abs(b).max() < 1e-10 * abs(Fm).max()


def _h_error_magnetostatic(n):
    # continuum: lap U = div m~, m~ = a cos(k.x)  ->  -grad U = -(khat . a) khat cos(k.x)
    L = 16.0
    mesh, wm = periodic((n, n, n), (L, L, L))
    x = lattice_xyz(mesh)
    k = 2 * np.pi * np.array([1.0, 0.0, 1.0]) / L
    a = np.array([0.6, 0.3, -0.2])
    m = a[None] * np.cos(x @ k)[:, None]
    F = fem.f_ms(wm); ML = fem.lumped_mass(wm)
    b = sum(F[c] @ m[:, c] for c in range(3)); b[0] = 0
    U, it, _ = cg(fem.pin(fem.stiffness(wm), [0]), b, np.zeros(wm.n), 1e-13, 10000)
    hd = -fem.nodal_gradient(F, ML, U)
    kh = k / np.linalg.norm(k)
    exact = -(kh @ a) * kh[None] * np.cos(x @ k)[:, None]
    return np.abs(hd - exact).max()


def test_magnetostatic_solve_converges_to_continuum():
    e1, e2 = _h_error_magnetostatic(8), _h_error_magnetostatic(16)
    assert e2 < 0.04
    assert 3.0 < e1 / e2 < 5.0          # second order


def _strain_error_laminate(n):
    # eigenstrain varying along x only; periodic equilibrium gives
    # E~11 = E0~11 + (C12/C11)(E0~22 + E0~33), E~12 = E0~12, E~13 = E0~13, others 0
    C11, C12, C44 = 243e9, 138e9, 122e9
    L = 16.0
    mesh, wm = periodic((n, 4, 4), (L, 8.0, 8.0))
    x = lattice_xyz(mesh)
    c = np.cos(2 * np.pi * x[:, 0] / L)
    A = np.array([[1.0, 0.4, -0.3], [0.4, -0.7, 0.2], [-0.3, 0.2, 0.5]]) * 1e-5
    E0 = A[None] * c[:, None, None]
    C = cubic_stiffness(C11, C12, C44)
    b = fem.f_mech(wm, C) @ E0.reshape(-1); b[:3] = 0
    u, it, _ = cg(fem.pin(fem.k_mech(wm, C), [0, 1, 2]), b, np.zeros(3 * wm.n), 1e-13, 20000)
    u = u.reshape(-1, 3)
    F = fem.f_ms(wm); ML = fem.lumped_mass(wm)
    G = np.stack([fem.nodal_gradient(F, ML, u[:, q]) for q in range(3)], axis=1)
    E = 0.5 * (G + np.transpose(G, (0, 2, 1)))
    ex = np.zeros_like(E)
    ex[:, 0, 0] = (A[0, 0] + C12 / C11 * (A[1, 1] + A[2, 2])) * c
    ex[:, 0, 1] = ex[:, 1, 0] = A[0, 1] * c
    ex[:, 0, 2] = ex[:, 2, 0] = A[0, 2] * c
    return np.abs(E - ex).max() / np.abs(A).max()


def test_elastic_solve_converges_to_laminate_solution():
    e1, e2 = _strain_error_laminate(8), _strain_error_laminate(16)
    assert e2 < 0.05
    assert 3.0 < e1 / e2 < 5.0


def test_volume_average_quadrature():
    mesh, wm = periodic((6, 5, 4), (12.0, 10.0, 8.0), jitter=0.2, seed=8)
    # constants are reproduced exactly; the weights sum to the box volume
    assert np.allclose(fem.volume_average(wm, np.full((wm.n, 3), 0.7)), 0.7, rtol=1e-14)
    # a Fourier mode of the unjittered lattice averages to zero
    mesh0, wm0 = periodic((6, 5, 4), (12.0, 10.0, 8.0))
    x = lattice_xyz(mesh0)
    g = np.cos(2 * np.pi * (x[:, 0] / 12.0 + 2 * x[:, 2] / 8.0))
    assert abs(fem.volume_average(wm0, g)) < 1e-14
    # the P1 interpolant of a linear function has the exact mean over an open patch
    mesh1, wm1, _ = open_patch((4, 4, 4), (8.0, 8.0, 8.0))
    lin = mesh1.coords @ np.array([1.0, -2.0, 0.5]) + 3.0
    cen = (mesh1.coords[mesh1.tets].mean(axis=1) * wm1.V[:, None]).sum(0) / wm1.volume
    assert fem.volume_average(wm1, lin) == pytest.approx(cen @ np.array([1.0, -2.0, 0.5]) + 3.0,
                                                         rel=1e-13)
