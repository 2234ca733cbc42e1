"""GPU parity on trilinear hexahedral meshes (nodes_per_elem 8, 2 x 2 x 2 Gauss quadrature): the
CUDA path through the C ABI against the oracle's hexahedral assembly on the same seeded mesh.

Tolerances as for the tetrahedral meshes: FP64 operators 1e-13 and first-step fields 1e-10
(every CG to 1e-13), mixed-precision operators 2e-6 and a mixed trajectory within 1e-4 radians
of the FP64 one.
"""
import numpy as np
import pytest

from oracle import fem
from oracle.gspm import System, run
from oracle.mesh import WrappedMesh
from paper_2510_09812_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# 10 x 9 x 5 = 450 nodes: 14 SELL slices and a ragged tail of 2 rows; 27-point rows
HEX = dict(cells=(10, 9, 5), box=(40.0, 36.0, 20.0), jitter=0.2, seed=41,
           defects=[dict(kind="sphere", center=(20.0, 18.0, 10.0), radius=7.0),
                    dict(kind="cuboid", center=(1.0, 1.0, 19.0), half_sides=(5.0, 4.0, 3.0))])


def _relerr(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _angle(a, b):
    na, nb = np.linalg.norm(a, axis=1), np.linalg.norm(b, axis=1)
    ok = (na > 0.5) & (nb > 0.5)
    c = np.clip((a[ok] * b[ok]).sum(1) / (na[ok] * nb[ok]), -1, 1)
    return float(np.arccos(c).max())


def _voigt(E):
    return np.stack([E[:, 0, 0], E[:, 1, 1], E[:, 2, 2], E[:, 1, 2], E[:, 0, 2], E[:, 0, 1]], 1)


@pytest.fixture(scope="module")
def hexm():
    mesh = synth.hex_box(HEX["cells"], HEX["box"], jitter=HEX["jitter"], seed=HEX["seed"],
                         defects=HEX["defects"])
    wm = WrappedMesh.from_synth(mesh)
    return mesh, wm, System(wm, synth.fe_like_material(), 1e-12, 0.5)


def _ctx(g, mesh, prec="f64", ordering="none", rtol=1e-13, **kw):
    if ordering == "aggregate":
        kw.setdefault("coarse_nodes", 64)
    return g.Context(mesh, synth.fe_like_material(), kw.pop("dt", 1e-12), kw.pop("alpha", 0.5),
                     precision=prec, ordering=ordering, rtol_gs=rtol, rtol_ms=rtol,
                     rtol_mech=rtol, **kw)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-13), ("mixed", 2e-6)])
@pytest.mark.parametrize("ordering", ["none", "aggregate"])
def test_hex_operators_match_oracle(gspm_lib, hexm, prec, tol, ordering):
    mesh, wm, s = hexm
    g = gspm_lib
    ctx = _ctx(g, mesh, prec, ordering)
    assert ctx.info()["n_tets"] == 450
    rng = np.random.default_rng(17)
    n = wm.n
    x1 = rng.standard_normal(n)
    x3 = rng.standard_normal((n, 3))
    nonmag = (~s.mag).astype(float)
    cases = [(g.OP_K_MS, x1, s.K_ms @ x1),
             (g.OP_A_EPS, x1, (s.M_m_full + s.red.eps * s.K_m) @ x1 + nonmag * x1),
             (g.OP_A_AEPS, x1, (s.M_m_full + s.red.alpha * s.red.eps * s.K_m) @ x1 + nonmag * x1),
             (g.OP_M, x1, s.M_m_full @ x1),
             (g.OP_K_MECH, x3, (s.K_mech @ x3.ravel()).reshape(n, 3)),
             (g.OP_GRAD, x1, -fem.nodal_gradient(s.F, s.ML, x1))]
    b = sum(s.F[a] @ x3[:, a] for a in range(3))
    b[0] = 0.0
    cases.append((g.OP_DIV, x3, b))
    for op, x, ref in cases:
        y = ctx.apply(op, x)
        assert _relerr(y, ref) < tol, (op, _relerr(y, ref))
    f = rng.standard_normal((n, 4))
    assert _relerr(ctx.volume_avg(f), fem.volume_average(wm, f)) < 1e-13


@pytest.mark.parametrize("ordering,pinned", [("none", True), ("none", False),
                                            ("aggregate", False)])
def test_hex_first_step_fields_match_oracle(gspm_lib, hexm, ordering, pinned):
    mesh, wm, _ = hexm
    s = System(wm, synth.fe_like_material(), 1e-12, 0.5, rtol_gs=1e-13, rtol_ms=1e-13,
               rtol_mech=1e-13)
    m0 = synth.random_unit_m(wm.n, 14)
    m0[~s.mag] = 0.0
    H = np.array([-2e4, 3e4, 1e4])
    m1, U, u, info = s.step(m0, np.zeros(wm.n), np.zeros((wm.n, 3)), H)
    ctx = _ctx(gspm_lib, mesh, "f64", ordering, pinned_cg=pinned)
    ctx.set_field(gspm_lib.FIELD_M, m0)
    st = ctx.step(1, H)
    assert st["noconv"] == 0
    if pinned:
        assert abs(st["it_ms_last"] - info["it_ms"]) <= 2
        assert abs(st["it_mech_last"] - info["it_mech"]) <= 2
    assert _relerr(ctx.get_field(gspm_lib.FIELD_U), U) < 1e-10
    assert _relerr(ctx.get_field(gspm_lib.FIELD_DISP), u) < 1e-10
    assert _relerr(ctx.get_field(gspm_lib.FIELD_HD), info["hd"]) < 1e-10
    assert _relerr(ctx.get_field(gspm_lib.FIELD_STRAIN), _voigt(info["E"])) < 1e-10
    assert _relerr(ctx.get_field(gspm_lib.FIELD_H), info["h"]) < 1e-10
    assert _relerr(ctx.get_field(gspm_lib.FIELD_M), m1) < 1e-10
    assert st["dm_last"] == pytest.approx(info["dm"], rel=1e-10)


def test_hex_mixed_trajectory_within_angle(gspm_lib, hexm):
    mesh, wm, s = hexm
    m0 = synth.random_unit_m(wm.n, 15)
    m0[~s.mag] = 0.0
    H = np.array([1e4, 0.0, 5e4])
    out = {}
    for prec, rtol in (("f64", 1e-13), ("mixed", 1e-7)):
        ctx = _ctx(gspm_lib, mesh, prec, rtol=rtol)
        ctx.set_field(gspm_lib.FIELD_M, m0)
        st = ctx.step(40, H)
        assert st["noconv"] == 0
        out[prec] = ctx.get_field(gspm_lib.FIELD_M)
    assert _angle(out["mixed"], out["f64"]) < 1e-4
    assert np.abs(np.linalg.norm(out["mixed"][s.mag], axis=1) - 1).max() < 1e-6


def test_cuboid_defect_relaxation_matches_oracle(gspm_lib):
    """The time-step study's workload (structured hexahedra, a non-magnetic cuboid at the
    centre, needle body N_d = diag(0, 1/2, 1/2), alpha 0.15, m = e1 in 200 A/m) at 16 x 16 x 8
    cells (2048 nodes, 32 defect elements): 60 FP64 steps at dt = 1 ps against the oracle,
    every CG to 1e-13."""
    cfg = synth.cuboid_defect_hex_box(n_cells=(16, 16, 8))
    wm = WrappedMesh.from_synth(cfg["mesh"])
    s = System(wm, cfg["material"], 1e-12, cfg["alpha"], rtol_gs=1e-13, rtol_ms=1e-13,
               rtol_mech=1e-13)
    m_ref, U_ref, u_ref, infos = run(s, cfg["m0"], cfg["H"], 60)
    g = gspm_lib
    ctx = g.Context(cfg["mesh"], cfg["material"], 1e-12, cfg["alpha"], precision="f64",
                    rtol_gs=1e-13, rtol_ms=1e-13, rtol_mech=1e-13)
    ctx.set_field(g.FIELD_M, cfg["m0"])
    st = ctx.step(60, cfg["H"])
    assert st["noconv"] == 0
    assert _relerr(ctx.get_field(g.FIELD_M), m_ref) < 1e-10
    assert _relerr(ctx.get_field(g.FIELD_U), U_ref) < 1e-10
    assert _relerr(ctx.get_field(g.FIELD_DISP), u_ref) < 1e-9
    # <|dm|> of the last step (about 3e-4 here) to the accuracy of m
    assert st["dm_last"] == pytest.approx(infos[-1]["dm"], rel=1e-5)
