"""Oracle GSPM step (Algorithm B.1 with magnetostatics and elasticity) against physics:
macrospin reduction, Kittel precession, convergence to the Landau-Lifshitz ODE, |m| = 1,
energy decay, the uniform-state energy, and free-body magnetostriction."""
import numpy as np
import pytest
from scipy.integrate import solve_ivp

from oracle.gspm import System, run
from oracle.material import (compliance_apply, contract, h_magnetoelastic, spontaneous_strain,
                             voigt_to_tensor)
from oracle_helpers import periodic
from paper_2510_09812_gb300 import synth


def _tiny(mat, dt, alpha, **kw):
    mesh, wm = periodic((2, 2, 2), (8.0, 8.0, 8.0), jitter=0.2, seed=21)
    return System(wm, mat, dt, alpha, **kw)


def _ll_rhs(m, h, alpha):
    return -np.cross(m, h) - alpha * np.cross(m, np.cross(m, h))


def _macro_h(m, red, H):
    # uniform state: no exchange, no local demag field, no stress; far field -N_d m
    m2 = m ** 2
    return -red.kappa * m * (m2.sum() - m2) + H / red.Ms - red.Nd @ m


def test_uniform_state_reduces_to_macrospin_recursion():
    # For uniform m every (1 - eps Lap)^-1 is the identity, m_bar = m, grad U = 0, sigma = 0, so
    # the FEM step must equal Algorithm B.1 applied to one spin.
    mat = synth.fe_like_material()
    mat["Nd"] = [0.2, 0, 0, 0, 0.3, 0, 0, 0, 0.5]
    s = _tiny(mat, 2e-12, 0.3)
    red = s.red
    H = np.array([1e4, -3e4, 2e4])
    m0 = np.array([0.3, -0.5, 0.8]); m0 /= np.linalg.norm(m0)
    m = np.tile(m0, (s.n, 1))
    U, u = np.zeros(s.n), np.zeros((s.n, 3))
    v = m0.copy()
    for _ in range(5):
        m, U, u, info = s.step(m, U, u, H)
        g = v + red.dtau * _macro_h(v, red, H)
        hv = _macro_h(v, red, H)
        a1 = v[0] + g[1] * v[2] - g[2] * v[1]
        gs1 = a1 + red.dtau * hv[0]
        a2 = v[1] + g[2] * a1 - gs1 * v[2]
        gs2 = a2 + red.dtau * hv[1]
        a3 = v[2] + gs1 * a2 - gs2 * a1
        ms = np.array([a1, a2, a3])
        # step 3 holds the strain of step n (E = E0(v) for a free uniform body), so the
        # magnetoelastic field at m* comes from sigma* = C (E0(v) - E0(m*))
        sig = contract(red.C, spontaneous_strain(v, red.l100, red.l111)
                       - spontaneous_strain(ms, red.l100, red.l111))
        hme = h_magnetoelastic(ms[None], sig[None], red)[0]
        mss = ms + red.alpha * red.dtau * (_macro_h(ms, red, H) + hme)
        v = mss / np.linalg.norm(mss)
        assert np.abs(m - v[None]).max() < 1e-13
        # right-hand sides vanish up to rounding: no field from U or u
        assert np.abs(info["hd"]).max() < 1e-12
        assert np.abs(info["E"] - info["E_bar"][None]).max() < 1e-15


def test_kittel_precession_frequency():
    # small precession about z of a uniformly magnetised ellipsoid with cubic anisotropy
    # (K1 > 0, easy [001]) and no damping: omega / (gamma0 ms) = sqrt(a b) with
    # a = H/ms + N_x - N_z + 2K1/(mu0 ms^2), b = H/ms + N_y - N_z + 2K1/(mu0 ms^2)   (Kittel)
    mat = synth.fe_like_material()
    mat.update(lambda100=0.0, lambda111=0.0, Nd=[0.2, 0, 0, 0, 0.3, 0, 0, 0, 0.5])
    s = _tiny(mat, 2e-14, 0.0)
    red = s.red
    H = np.array([0.0, 0.0, 0.5 * red.Ms])
    a = 0.5 + 0.2 - 0.5 + red.kappa
    b = 0.5 + 0.3 - 0.5 + red.kappa
    m0 = np.array([0.005, 0.0, 1.0]); m0 /= np.linalg.norm(m0)
    m = np.tile(m0, (s.n, 1))
    U, u = np.zeros(s.n), np.zeros((s.n, 3))
    th = []
    nst = int(round(8.0 / red.dtau))
    for _ in range(nst):
        m, U, u, _ = s.step(m, U, u, H)
        th.append(np.arctan2(m[0, 1] / np.sqrt(a), m[0, 0] / np.sqrt(b)))
    tau = red.dtau * np.arange(1, nst + 1)
    omega = np.polyfit(tau, np.unwrap(th), 1)[0]
    assert omega == pytest.approx(np.sqrt(a * b), rel=2e-4)


def test_damped_gspm_converges_to_landau_lifshitz_ode():
    # large-angle damped motion of a uniform state; reference = LL ODE integrated by RK
    mat = synth.fe_like_material()
    mat.update(lambda100=0.0, lambda111=0.0, Nd=[0.2, 0, 0, 0, 0.3, 0, 0, 0, 0.5])
    H = np.array([2e5, 0.0, 4e5])
    m0 = np.array([0.6, 0.5, 0.3]); m0 /= np.linalg.norm(m0)
    T = 2.0                                       # reduced time tau
    errs = []
    for dt in (2e-14, 1e-14):
        s = _tiny(mat, dt, 0.2)
        red = s.red
        nst = int(round(T / red.dtau))
        m, U, u, _ = run(s, np.tile(m0, (s.n, 1)), H, nst)
        ref = solve_ivp(lambda t, v: _ll_rhs(v, _macro_h(v, red, H), red.alpha), (0, nst * red.dtau),
                        m0, rtol=1e-12, atol=1e-13, method="DOP853").y[:, -1]
        errs.append(np.abs(m[0] - ref).max())
    assert errs[1] < 2e-3
    assert 1.6 < errs[0] / errs[1] < 2.4          # first order in dt


@pytest.fixture(scope="module")
def defect_run():
    mesh, wm = periodic((8, 8, 4), (32.0, 32.0, 16.0), jitter=0.2, seed=5,
                        defects=[dict(kind="sphere", center=(16.0, 16.0, 8.0), radius=6.0)])
    s = System(wm, synth.fe_like_material(), 1e-12, 0.5)
    m0 = synth.random_unit_m(wm.n, 5)
    m0[~s.mag] = 0.0
    ms, Us, us, es = [m0], [np.zeros(wm.n)], [np.zeros((wm.n, 3))], []
    m, U, u = m0, Us[0], us[0]
    for _ in range(8):
        m, U, u, info = s.step(m, U, u, np.zeros(3))
        ms.append(m); Us.append(U); us.append(u)
        es.append(s.energy_density(m, U, u, np.zeros(3))["total"])
    return s, ms, es


def test_unit_length_and_zero_magnetisation_in_defects(defect_run):
    s, ms, _ = defect_run
    assert (~s.mag).sum() > 0
    for m in ms[1:]:
        assert np.abs(np.linalg.norm(m[s.mag], axis=1) - 1).max() < 1e-14
        assert np.all(m[~s.mag] == 0)


def test_energy_decreases_with_damping(defect_run):
    # soft invariant: GSPM with alpha > 0, constant field and no external stress relaxes Eq. 1
    _, _, es = defect_run
    assert np.all(np.diff(es) < 0)


def test_uniform_state_energy_closed_form():
    mat = synth.fe_like_material()
    mat["Nd"] = [0.2, 0, 0, 0, 0.3, 0, 0, 0, 0.5]
    s = _tiny(mat, 1e-12, 0.5)
    m0 = np.array([0.3, -0.5, 0.8]); m0 /= np.linalg.norm(m0)
    H = np.array([1e4, 2e4, -5e3])
    e = s.energy_density(np.tile(m0, (s.n, 1)), np.zeros(s.n), np.zeros((s.n, 3)), H)
    mu0, Ms = mat["mu0"], mat["Ms"]
    m2 = m0 ** 2
    expect = (mat["K1"] * (m2[0] * m2[1] + m2[1] * m2[2] + m2[2] * m2[0])
              + 0.5 * mu0 * Ms ** 2 * m0 @ s.red.Nd @ m0 - mu0 * Ms * H @ m0)
    assert e["total"] == pytest.approx(expect, rel=1e-12)
    assert abs(e["exchange"]) < 1e-6 and abs(e["elastic"]) < 1e-9


@pytest.mark.parametrize("direction,diag,off", [((1, 0, 0), "100", None), ((1, 1, 1), None, "111")])
def test_free_body_magnetostriction(direction, diag, off):
    mat = synth.fe_like_material()
    s = _tiny(mat, 1e-12, 0.5)
    n = np.asarray(direction, float) / np.linalg.norm(direction)
    el = s.solve_elastic(np.tile(n, (s.n, 1)), np.zeros((s.n, 3)))
    l100, l111 = mat["lambda100"], mat["lambda111"]
    assert np.abs(el["u"]).max() < 1e-15                # nm; F^mech kills a uniform E0
    if diag:
        expect = np.diag([l100, -l100 / 2, -l100 / 2])
    else:
        expect = np.full((3, 3), l111 / 2)
        np.fill_diagonal(expect, 0.0)
    assert np.allclose(el["E"], expect[None], rtol=0, atol=1e-18)
    assert np.abs(el["sigma"]).max() < 1e-6            # Pa: stress-free


def test_free_body_under_external_stress():
    mat = synth.fe_like_material()
    mat["sigma_ext"] = [6e6, 0, 0, 0, 0, 0]
    s = _tiny(mat, 1e-12, 0.5)
    el = s.solve_elastic(np.tile([1.0, 0, 0], (s.n, 1)), np.zeros((s.n, 3)))
    E_expect = (np.diag([mat["lambda100"], -mat["lambda100"] / 2, -mat["lambda100"] / 2])
                + compliance_apply(mat["C11"], mat["C12"], mat["C44"], voigt_to_tensor(mat["sigma_ext"])))
    assert np.allclose(el["E"], E_expect[None], rtol=1e-12, atol=1e-20)
    assert np.allclose(el["sigma"], voigt_to_tensor(mat["sigma_ext"])[None], rtol=1e-9, atol=1e-3)


def test_resolve_at_mstar_uniform_state_has_no_magnetoelastic_field():
    """With the equilibria solved again at m*, a uniform free body is strained by exactly
    E0(m*) at m*, so sigma* = 0 and step 3 sees no magnetoelastic field: the FEM step equals
    Algorithm B.1 on one spin whose step-3 field is anisotropy + Zeeman + far field only (the
    held-strain reading adds C (E0(m^n) - E0(m*)) there; see the macrospin test above)."""
    mat = synth.fe_like_material()
    mat["Nd"] = [0.2, 0, 0, 0, 0.3, 0, 0, 0, 0.5]
    s = _tiny(mat, 2e-12, 0.3, resolve_at_mstar=True)
    red = s.red
    H = np.array([1e4, -3e4, 2e4])
    m0 = np.array([0.3, -0.5, 0.8]); m0 /= np.linalg.norm(m0)
    m = np.tile(m0, (s.n, 1))
    U, u = np.zeros(s.n), np.zeros((s.n, 3))
    v = m0.copy()
    for _ in range(5):
        m, U, u, info = s.step(m, U, u, H)
        hv = _macro_h(v, red, H)
        g = v + red.dtau * hv
        a1 = v[0] + g[1] * v[2] - g[2] * v[1]
        gs1 = a1 + red.dtau * hv[0]
        a2 = v[1] + g[2] * a1 - gs1 * v[2]
        gs2 = a2 + red.dtau * hv[1]
        a3 = v[2] + gs1 * a2 - gs2 * a1
        ms = np.array([a1, a2, a3])
        mss = ms + red.alpha * red.dtau * _macro_h(ms, red, H)
        v = mss / np.linalg.norm(mss)
        assert np.abs(m - v[None]).max() < 1e-13
        # the strain returned is the one at m*: E0(m*) throughout the free body
        e0s = spontaneous_strain(info["m_star"][0], red.l100, red.l111)
        assert np.abs(info["E"] - e0s[None]).max() < 1e-15


def test_resolve_at_mstar_matches_held_reading_to_first_order():
    """The two readings of h[m*] differ by O(dt) per step in the step-3 field, so over a fixed
    physical time (2 ps, smooth initial state) their trajectories approach each other linearly
    as dt -> 0."""
    mesh, wm = periodic((6, 6, 3), (24.0, 24.0, 12.0), jitter=0.2, seed=8,
                        defects=[dict(kind="sphere", center=(12.0, 12.0, 6.0), radius=4.0)])
    xs = np.zeros((wm.n, 3))
    xs[wm.unique_of_stored] = mesh.coords
    m0 = np.stack([0.3 * np.sin(2 * np.pi * xs[:, 0] / 24.0),
                   0.2 * np.cos(2 * np.pi * xs[:, 1] / 24.0), np.ones(wm.n)], 1)
    m0 /= np.linalg.norm(m0, axis=1)[:, None]
    diffs = []
    for dt, steps in ((1e-13, 20), (5e-14, 40)):
        out = []
        for resolve in (False, True):
            s = System(wm, synth.fe_like_material(), dt, 0.5, rtol_gs=1e-12, rtol_ms=1e-12,
                       rtol_mech=1e-12, resolve_at_mstar=resolve)
            out.append(run(s, m0, np.array([0.0, 3e4, 0.0]), steps)[0])
        diffs.append(np.abs(out[0] - out[1]).max())
    assert 1.6 < diffs[0] / diffs[1] < 2.4
