"""Graph replay of the time step (CUDA graph with conditional WHILE nodes for the CG loops)
against direct launches of the same kernels, and against the oracle.

Graph replay changes only how the kernels are issued: the same kernels run in the same order
on the same data, and the loops stop after the same iteration (the one whose update leaves no
segment active), so the state must match direct launches bit for bit, as must the iteration
statistics (both contexts use the same SpMV schedule).
"""
import numpy as np
import pytest

from oracle.gspm import System, run
from oracle.mesh import WrappedMesh
from paper_2510_09812_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

STAT_KEYS = ("steps", "it_ms", "it_mech", "it_gs", "it_ms_last", "it_mech_last", "noconv",
             "it_gs_last")


def _mesh(cells, box, seed, defects=()):
    mesh = synth.kuhn_box(cells, box, jitter=0.2, seed=seed, defects=list(defects))
    return mesh, WrappedMesh.from_synth(mesh)


@pytest.fixture(scope="module")
def single():
    mesh, wm = _mesh((10, 9, 5), (40.0, 36.0, 20.0), 71,
                     [dict(kind="sphere", center=(20.0, 18.0, 10.0), radius=7.0)])
    m0 = synth.random_unit_m(wm.n, 72)
    m0[~wm.node_magnetic] = 0.0
    return mesh, wm, m0


@pytest.fixture(scope="module")
def batch():
    specs = [((6, 5, 4), (24.0, 20.0, 16.0), 81, []),
             ((9, 8, 5), (36.0, 32.0, 20.0), 82,
              [dict(kind="cuboid", center=(4.0, 30.0, 6.0), half_sides=(5.0, 4.0, 3.0))]),
             ((7, 7, 3), (28.0, 28.0, 12.0), 83, [])]
    out = []
    for k, (c, b, sd, d) in enumerate(specs):
        mesh, wm = _mesh(c, b, sd, d)
        m0 = synth.random_unit_m(wm.n, 90 + k)
        m0[~wm.node_magnetic] = 0.0
        out.append((mesh, wm, m0))
    return out


def _ctx(gspm_lib, mesh, prec="f64", rtol=1e-13, **kw):
    # one fixed SpMV schedule: two contexts may otherwise time different schedules fastest,
    # whose sums differ in order
    return gspm_lib.Context(mesh, synth.fe_like_material(), 1e-12, 0.5, precision=prec,
                            rtol_gs=rtol, rtol_ms=rtol, rtol_mech=rtol, autotune=False, **kw)


def _same_stats(a, b):
    for k in STAT_KEYS:
        assert a[k] == b[k], (k, a[k], b[k])


@pytest.mark.parametrize("prec,printed,resolve,pinned", [
    ("f64", False, False, False), ("mixed", False, False, False), ("f64", True, False, False),
    ("mixed", True, False, True), ("mixed", False, True, False), ("f64", False, True, True)])
def test_graph_replay_is_bitwise_direct(gspm_lib, single, prec, printed, resolve, pinned):
    mesh, wm, m0 = single
    H = [2e4, -1e4, 5e3]
    rtol = 1e-13 if prec == "f64" else 1e-7
    kw = dict(row2_printed=printed, resolve_at_mstar=resolve, pinned_cg=pinned)
    direct = _ctx(gspm_lib, mesh, prec, rtol, **kw)
    graph = _ctx(gspm_lib, mesh, prec, rtol, graph=True, **kw)
    for c in (direct, graph):
        c.set_field(gspm_lib.FIELD_M, m0)
    for _ in range(2):  # the second call replays the graph captured by the first
        sd = direct.step(3, H)
        sg = graph.step(3, H)
        _same_stats(sd, sg)
        assert sd["m_bar"] == sg["m_bar"] and sd["dm_last"] == sg["dm_last"]
    for f in (gspm_lib.FIELD_M, gspm_lib.FIELD_U, gspm_lib.FIELD_DISP, gspm_lib.FIELD_HD,
              gspm_lib.FIELD_STRAIN):
        assert np.array_equal(direct.get_field(f), graph.get_field(f)), f


def test_graph_matches_oracle(gspm_lib, single):
    mesh, wm, m0 = single
    H = np.array([-3e4, 1e4, 0.0])
    g = _ctx(gspm_lib, mesh, graph=True, pinned_cg=True)
    g.set_field(gspm_lib.FIELD_M, m0)
    st = g.step(5, H)
    s = System(wm, synth.fe_like_material(), 1e-12, 0.5, rtol_gs=1e-13, rtol_ms=1e-13,
               rtol_mech=1e-13)
    m_ref, _, _, infos = run(s, m0, H, 5)
    got = g.get_field(gspm_lib.FIELD_M)
    assert np.abs(got - m_ref).max() / np.abs(m_ref).max() < 1e-10
    assert abs(st["it_mech_last"] - infos[-1]["it_mech"]) <= 2
    assert st["steps"] == 5 and st["noconv"] == 0


def test_graph_batch_is_bitwise_direct(gspm_lib, batch):
    meshes = [m for m, _, _ in batch]
    m_all = np.concatenate([m0 for _, _, m0 in batch])
    fields = np.array([[3e4, 0.0, 0.0], [0.0, -2e4, 1e4], [-1e4, 1e4, 5e3]])
    direct = _ctx(gspm_lib, meshes, "mixed", 1e-7)
    graph = _ctx(gspm_lib, meshes, "mixed", 1e-7, graph=True)
    for c in (direct, graph):
        c.set_field(gspm_lib.FIELD_M, m_all)
    sd = direct.batch_step(4, fields)
    sg = graph.batch_step(4, fields)
    for a, b in zip(sd, sg):
        _same_stats(a, b)
    assert np.array_equal(direct.get_field(gspm_lib.FIELD_M), graph.get_field(gspm_lib.FIELD_M))


def test_graph_follows_x0_mode_and_profiling(gspm_lib, single):
    mesh, wm, m0 = single
    H = [1e4, 0.0, 0.0]
    direct = _ctx(gspm_lib, mesh, "mixed", 1e-7)
    graph = _ctx(gspm_lib, mesh, "mixed", 1e-7)
    graph.set_graph(True)
    for c in (direct, graph):
        c.set_field(gspm_lib.FIELD_M, m0)
    for mode in (gspm_lib.X0_PREV, gspm_lib.X0_EXTRAPOLATE, gspm_lib.X0_ZERO):
        for c in (direct, graph):
            c.set_x0_mode(mode)
        _same_stats(direct.step(2, H), graph.step(2, H))
    # kernel-class profiling runs the step directly; the results stay identical
    graph.profile_enable(gspm_lib.KCLASS_NAMES)
    _same_stats(direct.step(1, H), graph.step(1, H))
    assert graph.profile_read("spmv_mech")[1] > 0
    graph.profile_enable(())
    n0 = graph.launch_count()
    _same_stats(direct.step(2, H), graph.step(2, H))
    assert graph.launch_count() > n0
    assert np.array_equal(direct.get_field(gspm_lib.FIELD_M), graph.get_field(gspm_lib.FIELD_M))


def test_graph_loop_stops_at_max_iter(gspm_lib, single):
    """A tolerance no CG can reach: every loop stops at max_iter and the step reports it.  In
    mixed precision a K^ms or K^mech solve is refined (two CG loops, each capped at max_iter)."""
    mesh, wm, m0 = single
    d = _ctx(gspm_lib, mesh, "mixed", 1e-30, max_iter=7)
    g = _ctx(gspm_lib, mesh, "mixed", 1e-30, max_iter=7, graph=True)
    for c in (d, g):
        c.set_field(gspm_lib.FIELD_M, m0)
    sd, sg = d.step(2, [1e4, 0, 0]), g.step(2, [1e4, 0, 0])
    assert sg["status"] == gspm_lib.ENOCONV and sd["status"] == gspm_lib.ENOCONV
    _same_stats(sd, sg)
    assert sg["it_mech_last"] == 14 and sg["it_ms_last"] == 14
    assert np.array_equal(d.get_field(gspm_lib.FIELD_M), g.get_field(gspm_lib.FIELD_M))


@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_autotuner_times_every_schedule_of_the_cg_product(gspm_lib, single, prec):
    """The autotuner times each SpMV schedule as the CG loops run it (the product fused with
    p.Ap) for K^mech, K^ms and the GSPM operators (1 + 2 + 3 right-hand sides), keeps the
    fastest, and a solve with the chosen schedules reaches the fixed-schedule solution."""
    mesh, wm, m0 = single
    g = gspm_lib
    rtol = 1e-13 if prec == "f64" else 1e-7
    ctx = g.Context(mesh, synth.fe_like_material(), 1e-12, 0.5, precision=prec,
                    rtol_gs=rtol, rtol_ms=rtol, rtol_mech=rtol)
    info = ctx.info()
    for times, chosen in (("spmv_ms_block", "spmv_schedule_block"),
                          ("spmv_ms_scalar", "spmv_schedule_scalar"),
                          ("spmv_ms_gs", "spmv_schedule_gs")):
        t = np.asarray(info[times])
        assert t.shape == (4,) and np.all(t > 0.0), (times, t)
        assert info[chosen] == int(np.argmin(t)), (chosen, t)
    fixed = _ctx(g, mesh, prec, rtol=rtol)
    untuned = fixed.info()
    assert untuned["spmv_schedule_block"] == untuned["spmv_schedule_gs"] == 0
    assert np.all(np.asarray(untuned["spmv_ms_gs"]) == 0.0)
    H = np.array([2e4, 0.0, -1e4])
    for c in (ctx, fixed):
        c.set_field(g.FIELD_M, m0)
        c.step(2, H)
    # FP64: the same solution to rounding; mixed: two summation orders stopped at 1e-7
    tol = 1e-10 if prec == "f64" else 1e-4
    a, b = ctx.get_field(g.FIELD_M), fixed.get_field(g.FIELD_M)
    assert np.abs(a - b).max() < tol
