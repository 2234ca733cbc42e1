"""The two CG formulations of the K^ms and K^mech solves on the GPU: the pinned systems of
Sec. 2.5 (GSPM_FLAG_PINNED_CG) and the default consistent singular systems (right-hand side
projected off the constants, CG on the unpinned operator, solution shifted to zero at the
pinned node).  Both must give the oracle's pinned solution; the singular form in fewer
iterations.

Tolerances: FP64 solves to rtol 1e-13 agree with the oracle to 1e-10 (the two iterations reach
the same solution by different paths, each within the CG bound); mixed trajectories of the two
forms agree to 1e-4 rad (the mixed-precision bound used throughout) after a few steps at rtol
1e-7.
"""
import numpy as np
import pytest

from oracle.gspm import System
from oracle.mesh import WrappedMesh
from paper_2510_09812_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _relerr(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _angle(a, b):
    na, nb = np.linalg.norm(a, axis=1), np.linalg.norm(b, axis=1)
    ok = (na > 0.5) & (nb > 0.5)
    c = np.clip((a[ok] * b[ok]).sum(1) / (na[ok] * nb[ok]), -1, 1)
    return float(np.arccos(c).max())


@pytest.fixture(scope="module")
def ragged():
    mesh = synth.kuhn_box((10, 9, 5), (40.0, 36.0, 20.0), jitter=0.2, seed=41,
                          defects=[dict(kind="sphere", center=(20.0, 18.0, 10.0), radius=7.0)])
    wm = WrappedMesh.from_synth(mesh)
    return mesh, wm


def _ctx(gspm_lib, mesh, prec, rtol, pinned, **kw):
    return gspm_lib.Context(mesh, synth.fe_like_material(), 1e-12, 0.5, precision=prec,
                            rtol_gs=rtol, rtol_ms=rtol, rtol_mech=rtol, pinned_cg=pinned, **kw)


@pytest.mark.parametrize("pinned", [True, False])
def test_elastic_solve_both_forms_match_oracle(gspm_lib, ragged, pinned):
    mesh, wm = ragged
    s = System(wm, synth.fe_like_material(), 1e-12, 0.5, rtol_mech=1e-13)
    m = synth.random_unit_m(wm.n, 11)
    m[~s.mag] = 0.0
    ref = s.solve_elastic(m, np.zeros((wm.n, 3)))
    ctx = _ctx(gspm_lib, mesh, "f64", 1e-13, pinned)
    u, it, rel, code = ctx.solve_elastic(m, x0_mode=0, rtol=1e-13)
    assert code == gspm_lib.OK and rel < 1e-13
    assert np.all(u[0] == 0.0)
    assert _relerr(u, ref["u"]) < 1e-10
    if pinned:
        assert abs(it - ref["iters"]) <= 2
    else:
        assert it < ref["iters"]


@pytest.mark.parametrize("pinned", [True, False])
def test_given_initial_guess_nonzero_at_pin(gspm_lib, ragged, pinned):
    """x0 with a non-zero pinned entry (and an arbitrary constant) still gives the pinned
    solution."""
    mesh, wm = ragged
    s = System(wm, synth.fe_like_material(), 1e-12, 0.5, rtol_mech=1e-13)
    m = synth.random_unit_m(wm.n, 12)
    m[~s.mag] = 0.0
    ref = s.solve_elastic(m, np.zeros((wm.n, 3)))
    ctx = _ctx(gspm_lib, mesh, "f64", 1e-13, pinned)
    x0 = np.random.default_rng(1).standard_normal((wm.n, 3)) * 1e-3 + 0.5
    u, it, rel, code = ctx.solve_elastic(m, x0_mode=2, x0=x0, rtol=1e-13)
    assert code == gspm_lib.OK
    assert np.all(u[0] == 0.0)
    assert _relerr(u, ref["u"]) < 1e-10


def test_uniform_magnetostriction_gives_no_displacement(gspm_lib):
    """Uniform m without defects: E0 is uniform, so b = F^mech E0 vanishes up to rounding and
    the periodic free body does not deform (u = 0 up to rounding in both forms)."""
    mesh = synth.kuhn_box((6, 6, 3), (24.0, 24.0, 12.0), jitter=0.2, seed=5)
    n = mesh.n_unique
    scale = 2.1e-5 * 24.0  # lambda x box length (nm)
    for pinned in (True, False):
        ctx = _ctx(gspm_lib, mesh, "f64", 1e-10, pinned)
        u, it, rel, code = ctx.solve_elastic(synth.uniform_m(n, (0.6, 0.8, 0.0)), x0_mode=0)
        assert np.abs(u).max() < 1e-8 * scale


def test_singular_form_needs_fewer_iterations(gspm_lib):
    """Mixed precision, 32x32x8 cubes with a spherical inclusion, random m, reversing field:
    same trajectory (to the CG tolerance), at least 25 % fewer K^mech iterations and fewer K^ms
    iterations."""
    cfg = synth.sphere_inclusion_box(n_cells=(32, 32, 8), box=(128.0, 128.0, 32.0), radius=14.0)
    m0 = synth.random_unit_m(cfg["mesh"].n_unique, 13)
    H = [-0.1 / synth.MU0, 0.0, 0.0]
    out = {}
    for pinned in (True, False):
        ctx = gspm_lib.Context(cfg["mesh"], cfg["material"], cfg["dt"], cfg["alpha"],
                               precision="mixed", pinned_cg=pinned)
        ctx.set_field(gspm_lib.FIELD_M, m0)
        st = ctx.step(4, H)
        assert st["noconv"] == 0
        out[pinned] = (st, ctx.get_field(gspm_lib.FIELD_M), ctx.get_field(gspm_lib.FIELD_DISP))
    (sp, mp, up), (ss, ms, us) = out[True], out[False]
    assert ss["it_mech"] < 0.75 * sp["it_mech"]
    assert ss["it_ms"] < sp["it_ms"]
    # two different CG iterations stopped at the same relative residual 1e-7: their U and u
    # differ by the solves' error (up to ~1e-6 of the fields), and four steps from a random m
    # carry that into m at the 1e-5 level; the bound is the mixed-precision one
    assert _angle(ms, mp) < 1e-4
    assert np.all(us[0] == 0.0) and np.all(up[0] == 0.0)
    assert _relerr(us, up) < 1e-3
