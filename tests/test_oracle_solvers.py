"""Oracle CG against dense direct solves and the Kuhn-lattice Fourier closed form."""
import numpy as np
import pytest

from oracle.gspm import System
from oracle.solvers import cg
from oracle_helpers import lattice_xyz, periodic
from paper_2510_09812_gb300 import synth


@pytest.fixture(scope="module")
def c0_system():
    mesh, wm = periodic((8, 8, 4), (32.0, 32.0, 16.0), jitter=0.2, seed=12,
                        defects=[dict(kind="sphere", center=(16.0, 16.0, 8.0), radius=6.0)])
    return System(wm, synth.fe_like_material(), 1e-12, 0.5)


@pytest.mark.parametrize("which", ["K_ms", "K_mech", "A_eps", "A_aeps"])
def test_cg_matches_dense_solve(c0_system, which):
    A = getattr(c0_system, which)
    rng = np.random.default_rng(0)
    b = rng.standard_normal(A.shape[0])
    x, it, rel = cg(A, b, np.zeros_like(b), 1e-13, 10000)
    xd = np.linalg.solve(A.toarray(), b)
    assert rel < 1e-13
    assert np.abs(x - xd).max() <= 1e-9 * np.abs(xd).max()


def test_pinned_operators_are_spd(c0_system):
    for which in ["K_ms", "K_mech", "A_eps", "A_aeps"]:
        np.linalg.cholesky(getattr(c0_system, which).toarray())


def test_cg_zero_rhs_and_converged_start():
    A = np.diag([2.0, 3.0])
    x, it, rel = cg(A, np.zeros(2), np.ones(2), 1e-7, 100)
    assert it == 0 and np.all(x == 0)
    x, it, rel = cg(A, np.array([2.0, 3.0]), np.ones(2), 1e-7, 100)
    assert it == 0 and np.all(x == 1)


def test_gs_solve_fourier_mode_closed_form():
    # unjittered periodic Kuhn lattice, cube edge h: Fourier modes diagonalise M and K with
    # lambda_K = h (6 - 2 sum cos th_a), lambda_M = h^3/120 [48 + 12 sum cos th_a
    #   + 8 (cos(th_x+th_y) + cos(th_x+th_z) + cos(th_y+th_z)) + 12 cos(th_x+th_y+th_z)],
    # so (M + eps K) g = M f gives g = lambda_M / (lambda_M + eps lambda_K) f.
    h = 4.0
    mesh, wm = periodic((8, 8, 4), (32.0, 32.0, 16.0))
    s = System(wm, synth.fe_like_material(), 1e-12, 0.5, rtol_gs=1e-14)
    x = lattice_xyz(mesh)
    kv = 2 * np.pi * np.array([1 / 32.0, 2 / 32.0, 1 / 16.0])
    th = kv * h
    f = np.cos(x @ kv)
    lK = h * (6 - 2 * np.cos(th).sum())
    lM = h ** 3 / 120 * (48 + 12 * np.cos(th).sum()
                         + 8 * (np.cos(th[0] + th[1]) + np.cos(th[0] + th[2]) + np.cos(th[1] + th[2]))
                         + 12 * np.cos(th.sum()))
    for c, A in [(1.0, s.A_eps), (0.5, s.A_aeps)]:
        g, it, rel = s.gs_solve(A, f, 1e-14)
        assert np.allclose(g, lM / (lM + c * s.red.eps * lK) * f, rtol=0, atol=1e-12)
