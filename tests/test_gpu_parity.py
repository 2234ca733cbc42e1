"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the same seeded inputs.

Tolerances (relative to the largest magnitude of the compared quantity):
* FP64 operators and volume averages: 1e-13 (different summation order only).
* FP64 GSPM trajectory: 1e-10 after 100 steps with every CG solved to 1e-13 (so that no
  iteration-count flip at the threshold can separate the two runs).
* Mixed precision (FP32 matrices and fields, FP64 reductions): operators 2e-6; trajectory within
  1e-4 radians of the FP64 GPU trajectory (largest angle between m vectors).
"""
import numpy as np
import pytest

from oracle import fem
from oracle.gspm import System, run
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


# several SELL slices and a ragged tail: 10 x 9 x 5 = 450 nodes = 14 slices + 2 rows
RAGGED = dict(cells=(10, 9, 5), box=(40.0, 36.0, 20.0), jitter=0.2, seed=31,
              defects=[dict(kind="sphere", center=(20.0, 18.0, 10.0), radius=7.0),
                       dict(kind="cuboid", center=(1.0, 1.0, 19.0), half_sides=(5.0, 4.0, 3.0))])


@pytest.fixture(scope="module")
def ragged():
    mesh = synth.kuhn_box(RAGGED["cells"], RAGGED["box"], jitter=RAGGED["jitter"],
                          seed=RAGGED["seed"], defects=RAGGED["defects"])
    wm = WrappedMesh.from_synth(mesh)
    sysm = System(wm, synth.fe_like_material(), 1e-12, 0.5)
    return mesh, wm, sysm


def _ctx(gspm_lib, mesh, prec="f64", ordering="none", rtol=1e-13, **kw):
    return gspm_lib.Context(mesh, synth.fe_like_material(), kw.pop("dt", 1e-12),
                            kw.pop("alpha", 0.5), precision=prec, ordering=ordering,
                            rtol_gs=rtol, rtol_ms=rtol, rtol_mech=rtol, **kw)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-13), ("mixed", 2e-6)])
@pytest.mark.parametrize("ordering", ["none", "rcm", "aggregate"])
def test_operators_match_oracle(gspm_lib, ragged, prec, tol, ordering):
    mesh, wm, s = ragged
    g = gspm_lib
    # aggregate ordering with several aggregates (the default size would give one here)
    ctx = _ctx(g, mesh, prec, ordering, **({"coarse_nodes": 64} if ordering == "aggregate" else {}))
    rng = np.random.default_rng(7)
    n = wm.n
    x1 = rng.standard_normal(n)
    x3 = rng.standard_normal((n, 3))
    nonmag = (~s.mag).astype(float)
    A_eps = s.M_m_full + s.red.eps * s.K_m
    A_aeps = s.M_m_full + s.red.alpha * s.red.eps * s.K_m
    cases = [(g.OP_K_MS, x1, s.K_ms @ x1),
             (g.OP_A_EPS, x1, A_eps @ x1 + nonmag * x1),
             (g.OP_A_AEPS, x1, A_aeps @ x1 + nonmag * x1),
             (g.OP_M, x1, s.M_m_full @ x1),
             (g.OP_K_MECH, x3, (s.K_mech @ x3.ravel()).reshape(n, 3)),
             (g.OP_GRAD, x1, -fem.nodal_gradient(s.F, s.ML, x1))]
    b = sum(s.F[a] @ x3[:, a] for a in range(3))
    b[0] = 0.0
    cases.append((g.OP_DIV, x3, b))
    for op, x, ref in cases:
        y = ctx.apply(op, x)
        assert _relerr(y, ref) < tol, (op, _relerr(y, ref))
        # device pointers give the same result
        yd = ctx.apply(op, torch.tensor(x, device="cuda"))
        assert np.array_equal(yd.cpu().numpy(), y)


@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_volume_average_matches_oracle(gspm_lib, ragged, prec):
    mesh, wm, s = ragged
    ctx = _ctx(gspm_lib, mesh, prec)
    f = np.random.default_rng(3).standard_normal((wm.n, 6))
    ref = fem.volume_average(wm, f)
    assert _relerr(ctx.volume_avg(f), ref) < 1e-13
    dev = ctx.volume_avg(torch.tensor(f, device="cuda"))
    assert _relerr(dev, ref) < 1e-13
    assert np.allclose(ctx.volume_avg(np.full((wm.n, 1), 0.25)), 0.25, rtol=1e-14)


def test_elastic_solve_matches_oracle(gspm_lib, ragged):
    mesh, wm, s = ragged
    ctx = _ctx(gspm_lib, mesh, "f64")
    m = synth.random_unit_m(wm.n, 9)
    m[~s.mag] = 0.0
    s.rtol["mech"] = 1e-13
    ref = s.solve_elastic(m, np.zeros((wm.n, 3)))
    u, it, rel, code = ctx.solve_elastic(m, x0_mode=0, rtol=1e-13)
    assert rel < 1e-13
    assert _relerr(u, ref["u"]) < 1e-10
    E = ctx.get_field(gspm_lib.FIELD_STRAIN)
    Eref = ref["E"]
    Ev = np.stack([Eref[:, 0, 0], Eref[:, 1, 1], Eref[:, 2, 2], Eref[:, 1, 2], Eref[:, 0, 2],
                   Eref[:, 0, 1]], axis=1)
    assert _relerr(E, Ev) < 1e-10


def _voigt(E):
    return np.stack([E[:, 0, 0], E[:, 1, 1], E[:, 2, 2], E[:, 1, 2], E[:, 0, 2], E[:, 0, 1]], 1)


@pytest.mark.parametrize("ordering,pinned", [("none", True), ("none", False), ("rcm", False),
                                            ("aggregate", False)])
def test_first_step_fields_match_oracle(gspm_lib, ragged, ordering, pinned):
    mesh, wm, s0 = ragged
    s = System(wm, synth.fe_like_material(), 1e-12, 0.5, rtol_gs=1e-13, rtol_ms=1e-13,
               rtol_mech=1e-13)
    m0 = synth.random_unit_m(wm.n, 4)
    m0[~s.mag] = 0.0
    H = np.array([3e4, -1e4, 5e3])
    m1, U, u, info = s.step(m0, np.zeros(wm.n), np.zeros((wm.n, 3)), H)
    ctx = _ctx(gspm_lib, mesh, "f64", ordering, pinned_cg=pinned,
               **({"coarse_nodes": 64} if ordering == "aggregate" else {}))
    ctx.set_field(gspm_lib.FIELD_M, m0)
    st = ctx.step(1, H)
    if pinned:
        # the oracle's own systems: iteration counts may differ by a rounding flip at the
        # stopping threshold
        assert abs(st["it_ms_last"] - info["it_ms"]) <= 2
        assert abs(st["it_mech_last"] - info["it_mech"]) <= 2
        assert np.abs(np.array(st["it_gs_last"][:7]) - info["it_gs"]).max() <= 2
    else:
        # the equivalent consistent singular systems with the two-level preconditioner, and the
        # Jacobi-preconditioned GSPM solves, converge faster to the same solution
        assert st["it_ms_last"] < info["it_ms"] and st["it_mech_last"] < info["it_mech"]
        assert sum(st["it_gs_last"][:7]) < sum(info["it_gs"])
    assert _relerr(ctx.get_field(gspm_lib.FIELD_U), U) < 1e-10
    assert _relerr(ctx.get_field(gspm_lib.FIELD_DISP), u) < 1e-10
    assert _relerr(ctx.get_field(gspm_lib.FIELD_HD), info["hd"]) < 1e-10
    assert _relerr(ctx.get_field(gspm_lib.FIELD_STRAIN), _voigt(info["E"])) < 1e-10
    assert _relerr(ctx.get_field(gspm_lib.FIELD_H), info["h"]) < 1e-10
    assert _relerr(ctx.get_field(gspm_lib.FIELD_M), m1) < 1e-10
    assert st["dm_last"] == pytest.approx(info["dm"], rel=1e-10)
    assert np.allclose(st["m_bar"], info["m_bar"], rtol=0, atol=1e-14)


@pytest.fixture(scope="module")
def fe_box_oracle():
    cfg = synth.fe_box_17x17x5()
    wm = WrappedMesh.from_synth(cfg["mesh"])
    s = System(wm, cfg["material"], cfg["dt"], cfg["alpha"], rtol_gs=1e-13, rtol_ms=1e-13,
               rtol_mech=1e-13)
    m, U, u, infos = run(s, cfg["m0"], cfg["H"], cfg["steps"])
    return cfg, m, U, u, infos


def test_fe_box_100_steps_fp64_matches_oracle(gspm_lib, fe_box_oracle):
    # 64x64x16 nm Fe-like box, 17x17x5 stored nodes, random m, alpha 0.5, dt 1 ps, 100 steps
    cfg, m_ref, U_ref, u_ref, infos = fe_box_oracle
    ctx = _ctx(gspm_lib, cfg["mesh"], "f64", alpha=cfg["alpha"], dt=cfg["dt"])
    ctx.set_field(gspm_lib.FIELD_M, cfg["m0"])
    st = ctx.step(cfg["steps"], cfg["H"])
    assert st["steps"] == 100 and st["noconv"] == 0
    m = ctx.get_field(gspm_lib.FIELD_M)
    assert _relerr(m, m_ref) < 1e-10
    assert np.abs(np.linalg.norm(m, axis=1) - 1).max() < 1e-14
    assert _relerr(ctx.get_field(gspm_lib.FIELD_U), U_ref) < 1e-10
    assert _relerr(ctx.get_field(gspm_lib.FIELD_DISP), u_ref) < 1e-9


def test_fe_box_100_steps_mixed_within_angle(gspm_lib, fe_box_oracle):
    cfg, m_ref, _, _, _ = fe_box_oracle
    ctx = _ctx(gspm_lib, cfg["mesh"], "mixed", rtol=1e-7, alpha=cfg["alpha"], dt=cfg["dt"])
    ctx.set_field(gspm_lib.FIELD_M, cfg["m0"])
    st = ctx.step(cfg["steps"], cfg["H"])
    assert st["noconv"] == 0
    m = ctx.get_field(gspm_lib.FIELD_M)
    assert _angle(m, m_ref) < 1e-4
    assert np.abs(np.linalg.norm(m, axis=1) - 1).max() < 1e-6


def test_printed_row2_variant_matches_oracle(gspm_lib, ragged):
    mesh, wm, _ = ragged
    s = System(wm, synth.fe_like_material(), 1e-12, 0.5, rtol_gs=1e-13, rtol_ms=1e-13,
               rtol_mech=1e-13, row2_printed=True)
    m0 = synth.random_unit_m(wm.n, 8)
    m0[~s.mag] = 0.0
    m_ref, _, _, infos = run(s, m0, np.array([0.0, 2e4, 0.0]), 3)
    for literal in (True, False):
        # literal: the paper's plain CG on the pinned systems, iteration counts as the oracle's
        ctx = _ctx(gspm_lib, mesh, "f64", row2_printed=True, pinned_cg=literal)
        ctx.set_field(gspm_lib.FIELD_M, m0)
        st = ctx.step(3, [0.0, 2e4, 0.0])
        if literal:
            assert np.abs(np.array(st["it_gs_last"]) - infos[-1]["it_gs"]).max() <= 2
        assert _relerr(ctx.get_field(gspm_lib.FIELD_M), m_ref) < 1e-10


def test_device_pointer_state_roundtrip(gspm_lib, ragged):
    mesh, wm, s = ragged
    ctx = _ctx(gspm_lib, mesh, "f64")
    m0 = torch.tensor(synth.random_unit_m(wm.n, 2), device="cuda")
    ctx.set_field(gspm_lib.FIELD_M, m0)
    out = torch.empty_like(m0)
    ctx.get_field(gspm_lib.FIELD_M, out)
    torch.cuda.synchronize()
    ref = m0.cpu().numpy()
    ref[~s.mag] = 0.0
    assert np.array_equal(out.cpu().numpy(), ref)
    assert ctx.launch_count() > 0


@pytest.mark.parametrize("pinned", [True, False])
def test_resolve_at_mstar_variant_matches_oracle(gspm_lib, ragged, pinned):
    """Algorithm B.1 step 3 with the equilibria solved again at m* (the flag's reading of
    h[m*]): state and the fields at m* against the oracle's same variant."""
    mesh, wm, _ = ragged
    s = System(wm, synth.fe_like_material(), 1e-12, 0.5, rtol_gs=1e-13, rtol_ms=1e-13,
               rtol_mech=1e-13, resolve_at_mstar=True)
    m0 = synth.random_unit_m(wm.n, 14)
    m0[~s.mag] = 0.0
    H = np.array([-2e4, 1e4, 3e4])
    m_ref, U_ref, u_ref, infos = run(s, m0, H, 3)
    ctx = _ctx(gspm_lib, mesh, "f64", resolve_at_mstar=True, pinned_cg=pinned)
    ctx.set_field(gspm_lib.FIELD_M, m0)
    st = ctx.step(3, H)
    assert st["noconv"] == 0
    assert _relerr(ctx.get_field(gspm_lib.FIELD_M), m_ref) < 1e-10
    assert _relerr(ctx.get_field(gspm_lib.FIELD_U), U_ref) < 1e-10
    assert _relerr(ctx.get_field(gspm_lib.FIELD_DISP), u_ref) < 1e-10
    assert _relerr(ctx.get_field(gspm_lib.FIELD_HD), infos[-1]["hd"]) < 1e-10
    assert _relerr(ctx.get_field(gspm_lib.FIELD_STRAIN), _voigt(infos[-1]["E"])) < 1e-10
    # the held reading gives a different trajectory
    held = _ctx(gspm_lib, mesh, "f64", pinned_cg=pinned)
    held.set_field(gspm_lib.FIELD_M, m0)
    held.step(3, H)
    assert _relerr(held.get_field(gspm_lib.FIELD_M), m_ref) > 1e-8


def _rotated_material(sigma_ext=None):
    from oracle.material import rotation_111
    mat = synth.fe_like_material()
    mat["R"] = rotation_111().reshape(-1).tolist()
    if sigma_ext is not None:
        mat["sigma_ext"] = sigma_ext
    return mat


@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("mixed", None)])
def test_rotated_111_crystal_matches_oracle(gspm_lib, ragged, prec, tol):
    """App. D: crystal axes <111>, <-110>, <11-2> along the mesh axes, with an external stress;
    three steps against the oracle (FP64: every field to 1e-10; mixed: within 1e-4 rad)."""
    mesh, wm, _ = ragged
    mat = _rotated_material([5e6, -2e6, 0.0, 1e6, 0.0, 3e6])
    s = System(wm, mat, 1e-12, 0.5, rtol_gs=1e-13, rtol_ms=1e-13, rtol_mech=1e-13)
    m0 = synth.random_unit_m(wm.n, 15)
    m0[~s.mag] = 0.0
    H = np.array([1e4, 2e4, -1e4])
    m_ref, U_ref, u_ref, infos = run(s, m0, H, 3)
    rtol = 1e-13 if prec == "f64" else 1e-7
    ctx = gspm_lib.Context(mesh, mat, 1e-12, 0.5, precision=prec, rtol_gs=rtol, rtol_ms=rtol,
                           rtol_mech=rtol)
    ctx.set_field(gspm_lib.FIELD_M, m0)
    st = ctx.step(3, H)
    assert st["noconv"] == 0
    m = ctx.get_field(gspm_lib.FIELD_M)
    if tol is None:
        assert _angle(m, m_ref) < 1e-4
        return
    assert _relerr(m, m_ref) < tol
    assert _relerr(ctx.get_field(gspm_lib.FIELD_DISP), u_ref) < tol
    assert _relerr(ctx.get_field(gspm_lib.FIELD_STRAIN), _voigt(infos[-1]["E"])) < tol
    assert _relerr(ctx.get_field(gspm_lib.FIELD_H), infos[-1]["h"]) < tol
    # the unrotated crystal gives another trajectory
    plain = _ctx(gspm_lib, mesh, "f64")
    plain.set_field(gspm_lib.FIELD_M, m0)
    plain.step(3, H)
    assert _relerr(plain.get_field(gspm_lib.FIELD_M), m_ref) > 1e-8


def test_rotated_elastic_solve_with_external_stress(gspm_lib, ragged):
    mesh, wm, _ = ragged
    mat = _rotated_material([0.0, 4e6, -3e6, 0.0, 2e6, 0.0])
    s = System(wm, mat, 1e-12, 0.5, rtol_mech=1e-13)
    m = synth.random_unit_m(wm.n, 16)
    m[~s.mag] = 0.0
    ref = s.solve_elastic(m, np.zeros((wm.n, 3)))
    ctx = gspm_lib.Context(mesh, mat, 1e-12, 0.5, precision="f64", rtol_mech=1e-13)
    u, it, rel, code = ctx.solve_elastic(m, x0_mode=0, rtol=1e-13)
    assert _relerr(u, ref["u"]) < 1e-10
    assert _relerr(ctx.get_field(gspm_lib.FIELD_STRAIN), _voigt(ref["E"])) < 1e-10
