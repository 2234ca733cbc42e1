"""Oracle of the learned warm start: aggregation, gradients by central differences, Adam."""
import numpy as np
import pytest

from oracle import mpnn
from oracle_helpers import periodic
from paper_2510_09812_gb300 import synth


@pytest.fixture(scope="module")
def tiny():
    mesh, wm = periodic((3, 3, 2), (6.0, 6.0, 4.0), jitter=0.2, seed=2,
                        defects=[dict(kind="sphere", center=(3.0, 3.0, 2.0), radius=1.2)])
    A = mpnn.aggregation_matrix(wm)
    rng = np.random.default_rng(1)
    m = synth.random_unit_m(wm.n, 3)
    m[~wm.node_magnetic] = 0
    up = rng.standard_normal((wm.n, 3)) * 2e-5
    up2 = up + rng.standard_normal((wm.n, 3)) * 1e-6
    f = mpnn.features(m, wm.node_magnetic, up, up2, 2.07e-5, -2.12e-5, 2.0)
    p = mpnn.init_params(3)
    p["W_out"] = rng.standard_normal(p["W_out"].shape) * 0.1     # non-zero head for the FD test
    p["b_out"] = rng.standard_normal(3) * 0.1
    t = rng.standard_normal((wm.n, 3))
    return wm, A, f, p, t


def test_aggregation_is_element_message_mean(tiny):
    wm, A, f, p, t = tiny
    assert np.allclose(np.asarray(A.sum(axis=1)).ravel(), 1.0, rtol=1e-14)
    # brute force: node -> element mean -> volume-weighted mean over incident elements
    h = np.random.default_rng(5).standard_normal((wm.n, 4))
    msg = h[wm.tets].mean(axis=1)
    num = np.zeros_like(h)
    den = np.zeros(wm.n)
    for e, tet in enumerate(wm.tets):
        for i in tet:
            num[i] += wm.V[e] * msg[e]
            den[i] += wm.V[e]
    assert np.allclose(A @ h, num / den[:, None], rtol=1e-13, atol=1e-15)


def test_gradients_match_central_differences(tiny):
    wm, A, f, p, t = tiny
    y, cache = mpnn.forward(p, A, f)
    g = mpnn.backward(p, A, cache, y, t)
    rng = np.random.default_rng(9)
    for k in p:
        for _ in range(3):
            idx = tuple(rng.integers(0, s) for s in p[k].shape)
            q = {kk: vv.copy() for kk, vv in p.items()}
            hstep = 1e-6
            q[k][idx] += hstep
            lp = mpnn.loss(mpnn.forward(q, A, f)[0], t)
            q[k][idx] -= 2 * hstep
            lm = mpnn.loss(mpnn.forward(q, A, f)[0], t)
            fd = (lp - lm) / (2 * hstep)
            assert g[k][idx] == pytest.approx(fd, rel=1e-5, abs=1e-9), (k, idx)


def test_adam_first_step_moves_by_lr_times_sign():
    # first Adam step: m_hat = g, v_hat = g^2, so each weight moves by lr * g / (|g| + eps)
    p = {"w": np.array([1.0, -2.0, 0.5])}
    g = {"w": np.array([0.3, -4.0, 1e-3])}
    out = mpnn.adam_step(p, g, {}, lr=0.01, eps=1e-8)
    assert np.allclose(out["w"], p["w"] - 0.01 * g["w"] / (np.abs(g["w"]) + 1e-8), rtol=1e-12)


def test_training_reduces_loss_on_a_fixed_batch(tiny):
    wm, A, f, p, t = tiny
    st = {}
    l0 = mpnn.loss(mpnn.forward(p, A, f)[0], t)
    for _ in range(200):
        y, c = mpnn.forward(p, A, f)
        p = mpnn.adam_step(p, mpnn.backward(p, A, c, y, t), st, lr=3e-3)
    assert mpnn.loss(mpnn.forward(p, A, f)[0], t) < 0.5 * l0
