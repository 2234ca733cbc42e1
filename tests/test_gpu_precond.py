"""Two-level preconditioned CG of the K^ms and K^mech solves and Jacobi-preconditioned GSPM
solves (default) against the unpreconditioned CG (GSPM_FLAG_PLAIN_CG) and the oracle.

The preconditioner changes the iteration, not the system: with the stopping test on the true
recursive residual, FP64 solves to rtol 1e-13 agree with the oracle's pinned solution to 1e-10.
The coarse operators the host builds are checked against P^T K P formed from the oracle's
matrices and the exported aggregates (1e-12 relative: same sums, other order).
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle.gspm import System, run
from oracle.mesh import WrappedMesh
from paper_2510_09812_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _relerr(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.fixture(scope="module")
def medium():
    # 48 x 48 x 12 cubes (27,648 nodes): 54 aggregates of 512 nodes
    mesh = synth.kuhn_box((48, 48, 12), (192.0, 192.0, 48.0), jitter=0.2, seed=61,
                          defects=[dict(kind="sphere", center=(96.0, 96.0, 24.0), radius=20.0)])
    wm = WrappedMesh.from_synth(mesh)
    return mesh, wm


def _ctx(gspm_lib, mesh, prec="f64", rtol=1e-13, **kw):
    return gspm_lib.Context(mesh, synth.fe_like_material(), 1e-12, 0.5, precision=prec,
                            rtol_gs=rtol, rtol_ms=rtol, rtol_mech=rtol, **kw)


def test_coarse_operators_are_galerkin_products(gspm_lib, medium):
    mesh, wm = medium
    ctx = _ctx(gspm_lib, mesh)
    info = ctx.info()
    na = info["n_aggregates"]
    assert na > 16
    agg = ctx.export(gspm_lib.EXPORT_AGGREGATES)
    assert agg.min() == 0 and agg.max() == na - 1 and np.unique(agg).size == na
    s = System(wm, synth.fe_like_material(), 1e-12, 0.5)
    P = sp.csr_matrix((np.ones(wm.n), (np.arange(wm.n), agg)), shape=(wm.n, na))
    Kc = (P.T @ s.K_ms_raw @ P).toarray()
    got = ctx.export(gspm_lib.EXPORT_COARSE_K_MS).reshape(na, na)
    assert _relerr(got, Kc) < 1e-12
    P3 = sp.kron(P, sp.identity(3)).tocsr()
    Kc3 = (P3.T @ s.K_mech_raw @ P3).toarray()
    got3 = ctx.export(gspm_lib.EXPORT_COARSE_K_MECH).reshape(3 * na, 3 * na)
    assert _relerr(got3, Kc3) < 1e-12
    # the constants of each component span its null space
    for a in range(3):
        one = np.zeros(3 * na)
        one[a::3] = 1.0
        assert np.abs(got3 @ one).max() < 1e-12 * np.abs(got3).max()


@pytest.mark.parametrize("ordering", ["aggregate", "none"])
def test_preconditioned_elastic_solve_matches_oracle(gspm_lib, medium, ordering):
    """Aggregate ordering: contiguous aggregates (restriction in row order); none: row lists."""
    mesh, wm = medium
    s = System(wm, synth.fe_like_material(), 1e-12, 0.5, rtol_mech=1e-13)
    m = synth.random_unit_m(wm.n, 62)
    m[~s.mag] = 0.0
    ref = s.solve_elastic(m, np.zeros((wm.n, 3)))
    its = {}
    for plain in (True, False):
        ctx = _ctx(gspm_lib, mesh, plain_cg=plain, ordering=ordering)
        u, it, rel, code = ctx.solve_elastic(m, x0_mode=0, rtol=1e-13)
        assert code == gspm_lib.OK and rel < 1e-13
        assert np.all(u[0] == 0.0)
        assert _relerr(u, ref["u"]) < 1e-10
        its[plain] = it
    assert its[False] < 0.6 * its[True]


def test_preconditioned_steps_match_oracle_and_cut_iterations(gspm_lib, medium):
    mesh, wm = medium
    s = System(wm, synth.fe_like_material(), 1e-12, 0.5, rtol_gs=1e-13, rtol_ms=1e-13,
               rtol_mech=1e-13)
    m0 = synth.random_unit_m(wm.n, 63)
    m0[~s.mag] = 0.0
    H = np.array([2e4, 0.0, -1e4])
    m_ref, U_ref, u_ref, infos = run(s, m0, H, 2)
    st = {}
    for plain in (True, False):
        ctx = _ctx(gspm_lib, mesh, plain_cg=plain)
        ctx.set_field(gspm_lib.FIELD_M, m0)
        st[plain] = ctx.step(2, H)
        assert st[plain]["noconv"] == 0
        assert _relerr(ctx.get_field(gspm_lib.FIELD_M), m_ref) < 1e-10
        assert _relerr(ctx.get_field(gspm_lib.FIELD_U), U_ref) < 1e-10
        assert _relerr(ctx.get_field(gspm_lib.FIELD_DISP), u_ref) < 1e-10
    assert st[False]["it_mech"] < 0.6 * st[True]["it_mech"]
    assert st[False]["it_ms"] < st[True]["it_ms"]
    # Jacobi on the GSPM solves (M + c eps K) g = M f
    assert st[False]["it_gs"] < 0.6 * st[True]["it_gs"]


def test_preconditioned_mixed_graph_and_batch(gspm_lib, medium):
    """Mixed precision: graph replay of the preconditioned loops is bitwise equal to direct
    launches, also in a batch with a second, smaller mesh."""
    mesh, wm = medium
    small = synth.kuhn_box((10, 10, 4), (40.0, 40.0, 16.0), jitter=0.2, seed=64)
    m_all = np.concatenate([synth.random_unit_m(wm.n, 65), synth.random_unit_m(small.n_unique, 66)])
    out = []
    for graph in (False, True):
        ctx = _ctx(gspm_lib, [mesh, small], "mixed", 1e-7, graph=graph, autotune=False)
        ctx.set_field(gspm_lib.FIELD_M, m_all)
        st = ctx.batch_step(3, np.array([[1e4, 0.0, 0.0], [0.0, 2e4, 0.0]]))
        out.append((st, ctx.get_field(gspm_lib.FIELD_M)))
    (sd, md), (sg, mg) = out
    for a, b in zip(sd, sg):
        assert a["it_mech"] == b["it_mech"] and a["it_ms"] == b["it_ms"]
        assert a["noconv"] == 0
    assert np.array_equal(md, mg)


def test_mixed_singular_cg_tracks_f64_iterations(gspm_lib):
    """K rounded to FP32 does not annihilate the constants (K 1 != 0), so the singular-system CG
    runs projected off them (x0 minus its mean, r.r without r's mean, p without z's mean).
    Stepping with x0 = the previous solution, the mixed-precision K^mech and K^ms solves then
    need about as many iterations as the FP64 ones (unprojected, this 16,000-node mesh took up
    to 8x more in some steps)."""
    c = synth.batch_member(63)
    its = {}
    for prec in ("f64", "mixed"):
        ctx = gspm_lib.Context(c["mesh"], c["material"], c["dt"], c["alpha"], precision=prec,
                               rtol_gs=1e-7, rtol_ms=1e-7, rtol_mech=1e-7, coarse_nodes=128)
        ctx.set_field(gspm_lib.FIELD_M, c["m0"])
        sts = [ctx.step(1, c["H"]) for _ in range(6)]
        assert all(s["noconv"] == 0 for s in sts)
        its[prec] = ([s["it_mech"] for s in sts], [s["it_ms"] for s in sts])
        ctx.close()
    (mech64, ms64), (mech32, ms32) = its["f64"], its["mixed"]
    assert max(mech32) <= 1.3 * max(mech64) + 5, (mech32, mech64)
    assert sum(ms32) <= 1.3 * sum(ms64) + 10, (ms32, ms64)
