"""GPU parity of the learned warm start (forward on tensor cores, backward, Adam) against the
FP64 oracle in oracle/mpnn.py, through the C ABI.

Tolerances come from the arithmetic: inputs, weights of the four tensor-core layers and all
hidden activations are BF16 (unit roundoff 2^-9); rounding the oracle's FP64 forward at the same
points moves its output by 1.3e-2 of its largest magnitude (8e-3 RMS) on this mesh, so the GPU
forward must agree within 4e-2 (max) and 2e-2 (RMS).  Gradients are compared block by block in
norm within 5e-2; one Adam step from the GPU's own gradient must match the oracle's Adam to FP32
rounding.
"""
import numpy as np
import pytest

from oracle import mpnn
from oracle.gspm import System
from oracle.mesh import WrappedMesh
from paper_2510_09812_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

RAGGED = dict(cells=(10, 9, 5), box=(40.0, 36.0, 20.0))


@pytest.fixture(scope="module")
def setup():
    mesh = synth.kuhn_box(RAGGED["cells"], RAGGED["box"], jitter=0.2, seed=31,
                          defects=[dict(kind="sphere", center=(20.0, 18.0, 10.0), radius=7.0)])
    wm = WrappedMesh.from_synth(mesh)
    A = mpnn.aggregation_matrix(wm)
    h = np.cbrt(wm.volume / wm.n)
    rng = np.random.default_rng(1)
    m = synth.random_unit_m(wm.n, 3)
    m[~wm.node_magnetic] = 0
    up = rng.standard_normal((wm.n, 3)) * 2e-5 * h
    up2 = up + rng.standard_normal((wm.n, 3)) * 2e-6 * h
    p = mpnn.init_params(3)
    p["W_out"] = rng.standard_normal((64, 3)) * 0.1
    p["b_out"] = rng.standard_normal(3) * 0.1
    ustar = up + rng.standard_normal((wm.n, 3)) * 1e-5 * h
    return mesh, wm, A, h, m, up, up2, p, ustar


def _ctx(gspm_lib, mesh, prec="mixed"):
    # one fixed SpMV schedule, so that contexts compared bit for bit sum in the same order
    return gspm_lib.Context(mesh, synth.fe_like_material(), 1e-12, 0.5, precision=prec,
                            autotune=False)


@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_forward_matches_oracle(gspm_lib, setup, prec):
    mesh, wm, A, h, m, up, up2, p, ustar = setup
    ctx = _ctx(gspm_lib, mesh, prec)
    ctx.mpnn_set_params(p)
    f = mpnn.features(m, wm.node_magnetic, up, up2, 2.07e-5, -2.12e-5, h)
    y_ref, _ = mpnn.forward(p, A, f)
    y = ctx.mpnn_predict(m, up, up2, what=0)
    d = y - y_ref
    assert np.abs(d).max() < 4e-2 * np.abs(y_ref).max()
    assert np.sqrt(np.mean(d ** 2)) < 2e-2 * np.sqrt(np.mean(y_ref ** 2))
    # the warm start itself: x0 = 2 u_prev - u_prev2 + u_s y
    ls, us = mpnn.scales(2.07e-5, -2.12e-5, h)
    x0 = ctx.mpnn_predict(torch.tensor(m, device="cuda"), torch.tensor(up, device="cuda"),
                          torch.tensor(up2, device="cuda"), what=1).cpu().numpy()
    assert np.allclose(x0, 2 * up - up2 + us * y, rtol=1e-6, atol=1e-6 * us)


def test_gradients_and_adam_match_oracle(gspm_lib, setup):
    mesh, wm, A, h, m, up, up2, p, ustar = setup
    ctx = _ctx(gspm_lib, mesh, "mixed")
    ctx.mpnn_set_params(p)
    ctx.mpnn_dataset_reserve(2)
    assert ctx.mpnn_dataset_add(m, up, up2, ustar) == 0
    f = mpnn.features(m, wm.node_magnetic, up, up2, 2.07e-5, -2.12e-5, h)
    ls, us = mpnn.scales(2.07e-5, -2.12e-5, h)
    t = (ustar - (2 * up - up2)) / us
    y_ref, cache = mpnn.forward(p, A, f)
    g_ref = mpnn.backward(p, A, cache, y_ref, t)
    loss, g = ctx.mpnn_loss_grad(0)
    assert loss == pytest.approx(mpnn.loss(y_ref, t), rel=3e-2)
    from paper_2510_09812_gb300 import gspm
    gd = gspm.unflatten_params(g)
    for k in g_ref:
        err = np.linalg.norm(gd[k] - g_ref[k]) / max(np.linalg.norm(g_ref[k]), 1e-30)
        assert err < 5e-2, (k, err)
    # one Adam step from the GPU's gradient
    p32 = gspm.unflatten_params(gspm.flatten_params(p))
    expect = mpnn.adam_step(p32, gd, {}, lr=1e-3)
    ctx.mpnn_train(1, lr=1e-3, seed=0)
    got = gspm.unflatten_params(ctx.mpnn_get_params())
    for k in expect:
        assert np.allclose(got[k], expect[k], rtol=1e-5, atol=1e-7), k


def test_training_reduces_loss(gspm_lib, setup):
    mesh, wm, A, h, m, up, up2, p, ustar = setup
    ctx = _ctx(gspm_lib, mesh, "mixed")
    p0 = mpnn.init_params(5)
    ctx.mpnn_set_params(p0)
    rng = np.random.default_rng(4)
    ctx.mpnn_dataset_reserve(4)
    for k in range(4):
        mk = synth.random_unit_m(wm.n, 10 + k)
        mk[~wm.node_magnetic] = 0
        us_k = up + 0.3 * rng.standard_normal((wm.n, 3)) * 1e-5 * h
        ctx.mpnn_dataset_add(mk, up, up2, us_k)
    l_first, _ = ctx.mpnn_train(1, lr=1e-3, seed=1)
    _, l_last = ctx.mpnn_train(300, lr=3e-3, seed=2)
    assert l_last < 0.7 * l_first


def test_learned_x0_with_zero_head_equals_extrapolation(gspm_lib, setup):
    # with W_out = 0, b_out = 0 the learned guess is exactly 2 u_prev - u_prev2: same CG
    mesh, wm, A, h, m, up, up2, p, ustar = setup
    traj = {}
    for mode in ("extrapolate", "learned"):
        ctx = _ctx(gspm_lib, mesh, "f64")
        ctx.mpnn_set_params(mpnn.init_params(7))
        ctx.set_field(gspm_lib.FIELD_M, m)
        g = gspm_lib
        ctx.set_x0_mode(g.X0_EXTRAPOLATE if mode == "extrapolate" else g.X0_LEARNED)
        st = ctx.step(3, [1e4, 0, 0])
        traj[mode] = (ctx.get_field(g.FIELD_M), st["it_mech"])
    assert np.array_equal(traj["extrapolate"][0], traj["learned"][0])
    assert traj["extrapolate"][1] == traj["learned"][1]


def test_solve_elastic_x0_modes_reach_the_same_solution(gspm_lib, setup):
    mesh, wm, A, h, m, up, up2, p, ustar = setup
    g = gspm_lib
    ctx = _ctx(gspm_lib, mesh, "f64")
    ctx.mpnn_set_params(p)
    sols = {}
    for mode in (0, 1, 3, 4):
        ctx.set_field(g.FIELD_DISP, up)
        ctx.set_field(g.FIELD_DISP_PREV, up2)
        u, it, rel, code = ctx.solve_elastic(m, x0_mode=mode, rtol=1e-12)
        assert rel < 1e-12
        sols[mode] = u
    for mode in (1, 3, 4):
        assert np.abs(sols[mode] - sols[0]).max() < 1e-9 * np.abs(sols[0]).max()
