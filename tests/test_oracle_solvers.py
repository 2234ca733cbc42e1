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


@pytest.mark.parametrize("which", ["ms", "mech"])
def test_pinned_solution_solves_the_unpinned_periodic_system(c0_system, which):
    """Sec. 2.5 pins node 0 so that K becomes SPD.  The CUDA path instead solves the consistent
    singular system K x = b (b with zero sum per component, as every divergence-form right-hand
    side on the periodic mesh has) and subtracts the constant that makes node 0 zero.  Both give
    the pinned system's solution: checked here with a dense direct solve of the pinned system,
    which must satisfy every row of the unpinned one (node 0's included), and with the oracle's
    CG on the singular system after the shift."""
    s = c0_system
    m = synth.random_unit_m(s.n, 21)
    m[~s.mag] = 0.0
    if which == "ms":
        K_raw, K_pin, d = s.K_ms_raw, s.K_ms, 1
        b = sum(s.F[a] @ m[:, a] for a in range(3))
    else:
        K_raw, K_pin, d = s.K_mech_raw, s.K_mech, 3
        b = s.F_mech @ s.e0_nodal(m).reshape(-1)
    # divergence form: zero sum per component up to rounding
    assert np.abs(b.reshape(-1, d).sum(0)).max() < 1e-12 * np.abs(b).sum()
    bp = b.copy()
    bp[:d] = 0.0
    xp = np.linalg.solve(K_pin.toarray(), bp)
    assert np.all(xp[:d] == 0.0)
    assert np.abs(K_raw @ xp - b).max() < 1e-10 * np.abs(b).max()
    bs = (b.reshape(-1, d) - b.reshape(-1, d).mean(0)).reshape(-1)
    xs, it, rel = cg(K_raw, bs, np.zeros_like(bs), 1e-13, 20000)
    xs = (xs.reshape(-1, d) - xs.reshape(-1, d)[0]).reshape(-1)
    assert np.abs(xs - xp).max() < 1e-9 * np.abs(xp).max()
