"""State handling on the GPU: checkpoint/resume through the field calls continues bit for bit,
and a non-finite state is reported (GSPM_ENUMERIC) without hanging or faulting, after which the
context is usable again.  Failures are made on the host (poisoned input), never on the device.
"""
import numpy as np
import pytest

from paper_2510_09812_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

STATE = ("FIELD_M", "FIELD_U", "FIELD_DISP", "FIELD_DISP_PREV")


@pytest.fixture(scope="module")
def mesh():
    return synth.kuhn_box((10, 9, 5), (40.0, 36.0, 20.0), jitter=0.2, seed=91,
                          defects=[dict(kind="sphere", center=(20.0, 18.0, 10.0), radius=7.0)])


def _ctx(g, mesh, prec, **kw):
    # fixed SpMV schedule: contexts compared bit for bit must sum in the same order
    return g.Context(mesh, synth.fe_like_material(), 1e-12, 0.5, precision=prec, rtol_gs=1e-9,
                     rtol_ms=1e-9, rtol_mech=1e-9, autotune=False, **kw)


@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_checkpoint_resume_is_bitwise(gspm_lib, mesh, prec):
    g = gspm_lib
    m0 = synth.random_unit_m(mesh.n_unique, 92)
    H = [1e4, -2e4, 5e3]
    whole = _ctx(g, mesh, prec)
    whole.set_x0_mode(g.X0_EXTRAPOLATE)  # uses u_prev too
    whole.set_field(g.FIELD_M, m0)
    whole.step(6, H)
    first = _ctx(g, mesh, prec)
    first.set_x0_mode(g.X0_EXTRAPOLATE)
    first.set_field(g.FIELD_M, m0)
    first.step(3, H)
    saved = {f: first.get_field(getattr(g, f)) for f in STATE}
    first.close()
    resumed = _ctx(g, mesh, prec)
    resumed.set_x0_mode(g.X0_EXTRAPOLATE)
    for f, v in saved.items():
        resumed.set_field(getattr(g, f), v)
    resumed.step(3, H)
    for f in STATE:
        assert np.array_equal(resumed.get_field(getattr(g, f)), whole.get_field(getattr(g, f))), f


@pytest.mark.parametrize("graph", [False, True])
def test_non_finite_state_is_reported_and_recoverable(gspm_lib, mesh, graph):
    g = gspm_lib
    # a NaN right-hand side ends each CG after one iteration (p.q is NaN: the solve stops), so
    # the ordinary iteration cap applies
    ctx = _ctx(g, mesh, "mixed", graph=graph)
    m0 = synth.random_unit_m(mesh.n_unique, 93)
    bad = m0.copy()
    bad[::7] = np.nan  # some of these are magnetic nodes
    ctx.set_field(g.FIELD_M, bad)
    with pytest.raises(g.GSPMError) as e:
        ctx.step(1, [1e4, 0.0, 0.0])
    assert e.value.code == g.ENUMERIC and "not finite" in str(e.value)
    # a valid state makes the context usable again
    ctx.set_field(g.FIELD_M, m0)
    ctx.set_field(g.FIELD_U, np.zeros(mesh.n_unique))
    ctx.set_field(g.FIELD_DISP, np.zeros((mesh.n_unique, 3)))
    ctx.set_field(g.FIELD_DISP_PREV, np.zeros((mesh.n_unique, 3)))
    st = ctx.step(2, [1e4, 0.0, 0.0])
    assert st["noconv"] == 0
    m = ctx.get_field(g.FIELD_M)
    assert np.isfinite(m).all()
