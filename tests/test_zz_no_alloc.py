"""Allocation-free volume average, for callers that cannot call cudaMalloc (code confined to
another framework's memory pool, real-time loops and callbacks that must not take cudaMalloc's
implicit synchronisation).  gspm_volume_avg_noalloc is called through the C ABI with caller-owned
device buffers and compared, on two calls in a row, with the allocating gspm_volume_avg at the
tolerance the other volume-average parity tests use (1e-13 relative), and on the small mesh also
with the CPU oracle's volume average.

This file is collected last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

from oracle import fem
from oracle.mesh import WrappedMesh
from paper_2510_09812_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-13


def _relerr(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("cells,box", [((10, 9, 5), (40.0, 36.0, 20.0)),
                                       # 96 x 96 x 64 periodic cubes = 589,824 unique nodes
                                       # (611,585 stored before the periodic wrap): more rows
                                       # than one pass of the 2048-block scratch covers, so the
                                       # grid-stride path is exercised
                                       ((96, 96, 64), (384.0, 384.0, 256.0))])
def test_noalloc_volume_average_matches_allocating_entry_point(gspm_lib, cells, box):
    g = gspm_lib
    L = np.asarray(box)
    mesh = synth.kuhn_box(cells, L, jitter=0.2, seed=41,
                          defects=[dict(kind="sphere", center=L / 2, radius=0.2 * L[2])])
    ctx = g.Context(mesh, synth.fe_like_material(), 1e-12, 0.5)
    info = ctx.info()
    n = info["n_unique"]
    assert n == cells[0] * cells[1] * cells[2]
    w = torch.tensor(ctx.export(g.EXPORT_LUMPED_MASS) / info["volume"], device="cuda")
    oracle_mesh = WrappedMesh.from_synth(mesh) if n < 10000 else None
    rng = np.random.default_rng(17)
    for ncomp in (1, 3, 6, 9):
        for call in range(2):                                   # two calls in a row
            f = torch.tensor(rng.standard_normal((n, ncomp)), device="cuda")
            ref = ctx.volume_avg(f)
            out = torch.full((ncomp,), float("nan"), dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            before = (torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0])
            g.volume_avg_noalloc(f, w, out)
            torch.cuda.synchronize()
            after = (torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0])
            assert _relerr(out.cpu().numpy(), ref) < TOL, (ncomp, call)
            if oracle_mesh is not None:
                # and with the oracle's Sec. 2.4 quadrature, independently of the library
                want = fem.volume_average(oracle_mesh, f.cpu().numpy())
                assert _relerr(out.cpu().numpy(), want) < TOL, (ncomp, call)
            if call == 1:
                # after the first call (which loads the kernel and looks up the scratch's
                # address) a call leaves the device's allocations as they were
                assert after == before, (before, after)


def test_noalloc_rejects_sizes_beyond_its_scratch(gspm_lib):
    g = gspm_lib
    n = 1000
    w = torch.full((n,), 1.0 / n, dtype=torch.float64, device="cuda")
    f = torch.ones((n, 10), dtype=torch.float64, device="cuda")
    out = torch.zeros(10, dtype=torch.float64, device="cuda")
    with pytest.raises(g.GSPMError) as e:
        g.volume_avg_noalloc(f, w, out)
    assert e.value.code == g.EINVAL and "ncomp" in str(e.value)
