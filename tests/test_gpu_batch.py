"""Batched stepping (several uneven meshes in one context, one kernel sequence) against the
oracle and against each mesh stepped alone.

Tolerances: FP64 with every CG to 1e-13, as in the single-mesh parity tests: 1e-10 relative to
the oracle; 1e-12 relative to the same mesh in its own context (same arithmetic, different
grouping of the reduction partials).
"""
import numpy as np
import pytest

from oracle import fem
from oracle.gspm import System, run
from oracle.mesh import WrappedMesh
from paper_2510_09812_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SPECS = [
    dict(cells=(6, 5, 4), box=(24.0, 20.0, 16.0), seed=51, defects=[]),
    dict(cells=(10, 9, 5), box=(40.0, 36.0, 20.0), seed=52,
         defects=[dict(kind="sphere", center=(20.0, 18.0, 10.0), radius=7.0)]),
    dict(cells=(8, 8, 3), box=(32.0, 32.0, 12.0), seed=53,
         defects=[dict(kind="cuboid", center=(4.0, 30.0, 6.0), half_sides=(5.0, 4.0, 3.0))]),
]
FIELDS = np.array([[3e4, 0.0, 0.0], [0.0, -2e4, 1e4], [-1e4, 1e4, 5e3]])


def _relerr(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.fixture(scope="module")
def meshes():
    out = []
    for k, sp in enumerate(SPECS):
        mesh = synth.kuhn_box(sp["cells"], sp["box"], jitter=0.2, seed=sp["seed"],
                              defects=sp["defects"])
        wm = WrappedMesh.from_synth(mesh)
        m0 = synth.random_unit_m(wm.n, 60 + k)
        m0[~wm.node_magnetic] = 0.0
        out.append((mesh, wm, m0))
    return out


def _ctx(gspm_lib, mesh, prec="f64", pinned=False):
    return gspm_lib.Context(mesh, synth.fe_like_material(), 1e-12, 0.5, precision=prec,
                            rtol_gs=1e-13, rtol_ms=1e-13, rtol_mech=1e-13, pinned_cg=pinned)


@pytest.mark.parametrize("pinned", [True, False])
def test_batch_matches_oracle_and_single_mesh_runs(gspm_lib, meshes, pinned):
    steps = 3
    batch = _ctx(gspm_lib, [m for m, _, _ in meshes], pinned=pinned)
    assert batch.n_segments == len(meshes)
    m_all = np.concatenate([m0 for _, _, m0 in meshes])
    batch.set_field(gspm_lib.FIELD_M, m_all)
    stats = batch.batch_step(steps, FIELDS)
    got = batch.get_field(gspm_lib.FIELD_M)
    for k, (mesh, wm, m0) in enumerate(meshes):
        off, cnt = batch.segment(k)
        assert cnt == wm.n
        mk = got[off:off + cnt]
        s = System(wm, synth.fe_like_material(), 1e-12, 0.5, rtol_gs=1e-13, rtol_ms=1e-13,
                   rtol_mech=1e-13)
        m_ref, _, _, infos = run(s, m0, FIELDS[k], steps)
        assert _relerr(mk, m_ref) < 1e-10, k
        if pinned:
            assert abs(stats[k]["it_mech_last"] - infos[-1]["it_mech"]) <= 2
        single = _ctx(gspm_lib, mesh, pinned=pinned)
        single.set_field(gspm_lib.FIELD_M, m0)
        single.step(steps, FIELDS[k])
        assert _relerr(mk, single.get_field(gspm_lib.FIELD_M)) < 1e-12, k


def test_batch_volume_averages_per_mesh(gspm_lib, meshes):
    batch = _ctx(gspm_lib, [m for m, _, _ in meshes], "mixed")
    rng = np.random.default_rng(2)
    n = batch.n
    f = rng.standard_normal((n, 4))
    avg = batch.volume_avg(f)
    assert avg.shape == (len(meshes), 4)
    for k, (mesh, wm, m0) in enumerate(meshes):
        off, cnt = batch.segment(k)
        assert _relerr(avg[k], fem.volume_average(wm, f[off:off + cnt])) < 1e-13


def test_batch_mixed_runs_and_reports_per_mesh(gspm_lib, meshes):
    batch = gspm_lib.Context([m for m, _, _ in meshes], synth.fe_like_material(), 5e-12, 0.5,
                             precision="mixed")
    batch.set_field(gspm_lib.FIELD_M, np.concatenate([m0 for _, _, m0 in meshes]))
    stats = batch.batch_step(4, FIELDS)
    assert len(stats) == len(meshes)
    m = batch.get_field(gspm_lib.FIELD_M)
    for k, (mesh, wm, m0) in enumerate(meshes):
        off, cnt = batch.segment(k)
        mk = m[off:off + cnt]
        mag = wm.node_magnetic
        assert np.abs(np.linalg.norm(mk[mag], axis=1) - 1).max() < 1e-6
        assert np.all(mk[~mag] == 0)
        assert stats[k]["steps"] == 4 and stats[k]["noconv"] == 0
