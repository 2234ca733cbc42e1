"""C ABI without a GPU: exported symbols, host-only contexts, and the host mesh layer compared
bit-exactly with the oracle's independent periodic wrap, node graph and RCM order."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle.mesh import WrappedMesh, csr_pattern, rcm_order
from paper_2510_09812_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names += re.findall(r"GSPM_API\s+[\w\s\*]+?\b(gspm_\w+)\s*\(", txt)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(gspm_lib):
    names = _declared_symbols()
    assert "gspm_step" in names and len(names) >= 10
    lib = ctypes.CDLL(gspm_lib._LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


MESHES = [
    dict(cells=(6, 5, 4), box=(24.0, 20.0, 16.0), jitter=0.2, seed=3, defects=[]),
    dict(cells=(8, 8, 4), box=(32.0, 32.0, 16.0), jitter=0.2, seed=4,
         defects=[dict(kind="sphere", center=(16.0, 16.0, 8.0), radius=7.0),
                  dict(kind="cuboid", center=(2.0, 30.0, 1.0), half_sides=(4.0, 3.0, 3.0))]),
    dict(cells=(16, 16, 4), box=(64.0, 64.0, 16.0), jitter=0.0, seed=0, defects=[]),
]


def _bins(mesh, wm, npa):
    """Coordinate bin (x-fastest index) of every unique node for bins of about npa nodes, from
    the wrapped coordinates of each node's first stored copy."""
    first = np.full(wm.n, -1)
    first[wm.unique_of_stored[::-1]] = np.arange(wm.unique_of_stored.size)[::-1]
    xw = mesh.coords[first]
    lo, hi = np.asarray(mesh.box_lo, float), np.asarray(mesh.box_hi, float)
    L = hi - lo
    H = np.cbrt(np.prod(L) * npa / wm.n)
    nb = np.maximum(1, np.floor(L / H + 0.5)).astype(np.int64)
    t = np.clip(np.floor((xw - lo) / L * nb).astype(np.int64), 0, nb - 1)
    return t[:, 0] + nb[0] * (t[:, 1] + nb[1] * t[:, 2])


def _aggregate_order(mesh, wm, npa):
    """Nodes sorted by coordinate bin (ties by index)."""
    return np.argsort(_bins(mesh, wm, npa), kind="stable")


@pytest.mark.parametrize("spec", MESHES)
@pytest.mark.parametrize("ordering", ["none", "rcm", "aggregate"])
def test_host_mesh_matches_oracle_bit_exactly(gspm_lib, spec, ordering):
    mesh = synth.kuhn_box(spec["cells"], spec["box"], jitter=spec["jitter"], seed=spec["seed"],
                          defects=spec["defects"])
    ctx = gspm_lib.Context(mesh, synth.fe_like_material(), 1e-12, 0.5, ordering=ordering,
                           host_only=True, coarse_nodes=24)
    wm = WrappedMesh.from_synth(mesh)
    assert np.array_equal(ctx.export(gspm_lib.EXPORT_UNIQUE_OF_STORED), wm.unique_of_stored)
    rowptr, cols = csr_pattern(wm.tets, wm.n)
    assert np.array_equal(ctx.export(gspm_lib.EXPORT_ROWPTR), rowptr)
    assert np.array_equal(ctx.export(gspm_lib.EXPORT_COLS), cols)
    assert np.array_equal(ctx.export(gspm_lib.EXPORT_NODE_MAGNETIC).astype(bool),
                          wm.node_magnetic)
    perm = ctx.export(gspm_lib.EXPORT_PERM)
    expect = {"rcm": lambda: rcm_order(wm.tets, wm.n), "none": lambda: np.arange(wm.n),
              "aggregate": lambda: _aggregate_order(mesh, wm, 24)}[ordering]()
    assert np.array_equal(perm, expect)
    ML = ctx.export(gspm_lib.EXPORT_LUMPED_MASS)
    from oracle import fem
    assert np.allclose(ML, fem.lumped_mass(wm), rtol=1e-14, atol=0)
    info = ctx.info()
    assert info["n_unique"] == wm.n and info["n_tets"] == mesh.n_tets
    assert info["volume"] == pytest.approx(wm.volume, rel=1e-14)
    assert info["n_magnetic_nodes"] == int(wm.node_magnetic.sum())
    assert info["device_bytes"] == 0


def test_host_only_context_rejects_device_calls(gspm_lib):
    mesh = synth.kuhn_box((3, 3, 3), (3.0, 3.0, 3.0))
    ctx = gspm_lib.Context(mesh, synth.fe_like_material(), 1e-12, 0.5, host_only=True)
    with pytest.raises(gspm_lib.GSPMError) as e:
        ctx.step(1, [0, 0, 0])
    assert e.value.code == gspm_lib.ESTATE


def test_invalid_meshes_are_rejected(gspm_lib):
    mat = synth.fe_like_material()
    mesh = synth.kuhn_box((3, 3, 3), (3.0, 3.0, 3.0))
    bad = synth.kuhn_box((3, 3, 3), (3.0, 3.0, 3.0))
    bad.tets = bad.tets.copy()
    bad.tets[5] = bad.tets[5][[0, 2, 1, 3]]                        # inverted tet
    with pytest.raises(gspm_lib.GSPMError) as e:
        gspm_lib.Context(bad, mat, 1e-12, 0.5, host_only=True)
    assert e.value.code == gspm_lib.EMESH and "det" in str(e.value)
    bad2 = synth.kuhn_box((3, 3, 3), (3.0, 3.0, 3.0))
    bad2.tets = bad2.tets.copy()
    bad2.tets[0, 0] = mesh.n_stored + 7                              # out of range
    with pytest.raises(gspm_lib.GSPMError) as e:
        gspm_lib.Context(bad2, mat, 1e-12, 0.5, host_only=True)
    assert e.value.code == gspm_lib.EMESH
    bad3 = synth.kuhn_box((3, 3, 3), (3.0, 3.0, 3.0))
    bad3.coords = bad3.coords.copy()
    bad3.coords[4, 1] = np.nan
    with pytest.raises(gspm_lib.GSPMError) as e:
        gspm_lib.Context(bad3, mat, 1e-12, 0.5, host_only=True)
    assert e.value.code == gspm_lib.EMESH
    one = synth.kuhn_box((1, 2, 2), (1.0, 2.0, 2.0))                 # wrap collapses tets
    with pytest.raises(gspm_lib.GSPMError) as e:
        gspm_lib.Context(one, mat, 1e-12, 0.5, host_only=True)
    assert e.value.code == gspm_lib.EMESH and "collapses" in str(e.value)
    with pytest.raises(gspm_lib.GSPMError) as e:
        gspm_lib.Context(mesh, mat, -1.0, 0.5, host_only=True)       # dt <= 0
    assert e.value.code == gspm_lib.EINVAL


def test_rotation_must_be_proper(gspm_lib):
    mesh = synth.kuhn_box((3, 3, 3), (3.0, 3.0, 3.0))
    for R in (np.diag([1.0, 1.0, -1.0]), np.diag([1.0, 2.0, 1.0])):   # reflection, not orthogonal
        mat = synth.fe_like_material()
        mat["R"] = R.reshape(-1).tolist()
        with pytest.raises(gspm_lib.GSPMError) as e:
            gspm_lib.Context(mesh, mat, 1e-12, 0.5, host_only=True)
        assert e.value.code == gspm_lib.EINVAL and "rotation" in str(e.value)
    mat = synth.fe_like_material()
    c, s_ = np.cos(0.3), np.sin(0.3)
    mat["R"] = [c, -s_, 0.0, s_, c, 0.0, 0.0, 0.0, 1.0]
    gspm_lib.Context(mesh, mat, 1e-12, 0.5, host_only=True).close()


@pytest.mark.parametrize("ordering", ["aggregate", "none"])
def test_host_coarse_operators_and_inverses(gspm_lib, ordering):
    """Host-only contexts build the two-level preconditioner's coarse space: the aggregates are
    the non-empty coordinate bins in bin order, the coarse operators are the Galerkin products
    P^T K P of the oracle's matrices (same sums, other order), and the kept FP64 inverses invert
    those products plus rho = trace / n_c / n_agg on each component's constants."""
    import scipy.sparse as sp
    from oracle.gspm import System
    spec = MESHES[1]
    mesh = synth.kuhn_box(spec["cells"], spec["box"], jitter=spec["jitter"], seed=spec["seed"],
                          defects=spec["defects"])
    npa = 16
    g = gspm_lib
    ctx = g.Context(mesh, synth.fe_like_material(), 1e-12, 0.5, ordering=ordering,
                    host_only=True, coarse_nodes=npa)
    wm = WrappedMesh.from_synth(mesh)
    na = ctx.info()["n_aggregates"]
    agg = ctx.export(g.EXPORT_AGGREGATES)
    _, expect = np.unique(_bins(mesh, wm, npa), return_inverse=True)
    assert na > 8 and np.array_equal(agg, expect)
    s = System(wm, synth.fe_like_material(), 1e-12, 0.5)
    P = sp.csr_matrix((np.ones(wm.n), (np.arange(wm.n), agg)), shape=(wm.n, na))
    P3 = sp.kron(P, sp.identity(3)).tocsr()
    for Kraw, Pm, comps, ek, ei in ((s.K_ms_raw, P, 1, g.EXPORT_COARSE_K_MS, g.EXPORT_COARSE_INV_MS),
                                    (s.K_mech_raw, P3, 3, g.EXPORT_COARSE_K_MECH,
                                     g.EXPORT_COARSE_INV_MECH)):
        nc = comps * na
        Kc = (Pm.T @ Kraw @ Pm).toarray()
        got = ctx.export(ek).reshape(nc, nc)
        assert np.abs(got - Kc).max() < 1e-12 * np.abs(Kc).max()
        rho = np.trace(Kc) / nc / na
        same = (np.arange(nc)[:, None] % comps) == (np.arange(nc)[None, :] % comps)
        A = Kc + rho * same
        inv = ctx.export(ei).reshape(nc, nc)
        assert np.abs(inv - inv.T).max() < 1e-12 * np.abs(inv).max()
        assert np.abs(A @ inv - np.eye(nc)).max() < 1e-10


def _bf16_np(x):
    """Round to bfloat16 (nearest even of the FP32 value), as float64: written from the format's
    definition (sign, 8 exponent bits, 7 fraction bits), independently of the library."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("precision", ["mixed", "f64"])
def test_stored_coarse_inverses_are_positive_definite(gspm_lib, precision):
    """The device keeps the coarse inverses rounded to its storage type (BF16 under mixed
    precision).  Host-only contexts export the stored values: they are the rounding of the
    symmetric part of the FP64 inverse (no shift needed on a real mesh) and pass a Cholesky
    factorisation, so the preconditioner stays symmetric positive definite."""
    g = gspm_lib
    spec = MESHES[1]
    mesh = synth.kuhn_box(spec["cells"], spec["box"], jitter=spec["jitter"], seed=spec["seed"],
                          defects=spec["defects"])
    ctx = g.Context(mesh, synth.fe_like_material(), 1e-12, 0.5, precision=precision,
                    host_only=True, coarse_nodes=8)
    info = ctx.info()
    na = info["n_aggregates"]
    assert na > 16
    assert info["coarse_shift_ms"] == 0.0 and info["coarse_shift_mech"] == 0.0
    for ei, es, nc in ((g.EXPORT_COARSE_INV_MS, g.EXPORT_COARSE_STORED_MS, na),
                       (g.EXPORT_COARSE_INV_MECH, g.EXPORT_COARSE_STORED_MECH, 3 * na)):
        inv = ctx.export(ei).reshape(nc, nc)
        st = ctx.export(es).reshape(nc, nc)
        sym = 0.5 * (inv + inv.T)
        expect = _bf16_np(sym) if precision == "mixed" else sym
        assert np.array_equal(st, expect)
        np.linalg.cholesky(st)  # raises if not positive definite
        if precision == "mixed":
            assert np.abs(st - sym).max() <= 2.0 ** -8 * np.abs(sym).max()


def test_coarse_round_shifts_an_indefinite_rounding(gspm_lib):
    """A symmetric positive definite matrix whose smallest eigenvalue lies far below the BF16
    rounding of its entries: the rounded matrix is indefinite, so the rule adds the smallest
    accepted diagonal shift 2^k * 2^-8 max A_ii before rounding; the result is positive
    definite.  In FP64 storage the matrix is kept as it is (its symmetric part)."""
    g = gspm_lib
    rng = np.random.default_rng(5)
    n = 96
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.geomspace(1e-7, 1.0, n)
    A = (Q * lam) @ Q.T
    A = 0.5 * (A + A.T)
    assert np.linalg.eigvalsh(_bf16_np(A))[0] < 0.0  # plain rounding is indefinite
    st, shift = g.coarse_round(A, bf16=True)
    base = 2.0 ** -8 * np.abs(np.diag(A)).max()
    k = np.log2(shift / base)
    assert shift > 0.0 and abs(k - round(k)) < 1e-12
    assert np.array_equal(st, _bf16_np(A + shift * np.eye(n)))
    np.linalg.cholesky(st)
    if shift > base:  # the next smaller shift was rejected
        assert np.linalg.eigvalsh(_bf16_np(A + 0.5 * shift * np.eye(n)))[0] <= 0.0
    st64, sh64 = g.coarse_round(A, bf16=False)
    assert sh64 == 0.0 and np.array_equal(st64, A)
    with pytest.raises(g.GSPMError) as e:
        g.coarse_round(-np.eye(4), bf16=True)
    assert e.value.code == g.EMESH


@pytest.mark.parametrize("ordering", ["none", "rcm", "aggregate"])
def test_host_hex_mesh_matches_oracle(gspm_lib, ordering):
    """Linear hexahedra (nodes_per_elem 8): wrap, node graph (27-point stencil on the lattice),
    permutation, lumped mass (2x2x2 Gauss quadrature) and volume against the oracle."""
    mesh = synth.hex_box((6, 5, 4), (24.0, 20.0, 16.0), jitter=0.2, seed=8,
                         defects=[dict(kind="sphere", center=(12.0, 10.0, 8.0), radius=4.5)])
    ctx = gspm_lib.Context(mesh, synth.fe_like_material(), 1e-12, 0.5, ordering=ordering,
                           host_only=True, coarse_nodes=16)
    wm = WrappedMesh.from_synth(mesh)
    assert np.array_equal(ctx.export(gspm_lib.EXPORT_UNIQUE_OF_STORED), wm.unique_of_stored)
    rowptr, cols = csr_pattern(wm.tets, wm.n)
    assert np.array_equal(ctx.export(gspm_lib.EXPORT_ROWPTR), rowptr)
    assert np.array_equal(ctx.export(gspm_lib.EXPORT_COLS), cols)
    assert (rowptr[1:] - rowptr[:-1]).max() == 27
    assert np.array_equal(ctx.export(gspm_lib.EXPORT_NODE_MAGNETIC).astype(bool),
                          wm.node_magnetic)
    from oracle import fem
    assert np.allclose(ctx.export(gspm_lib.EXPORT_LUMPED_MASS), fem.lumped_mass(wm), rtol=1e-13)
    info = ctx.info()
    assert info["volume"] == pytest.approx(24.0 * 20.0 * 16.0, rel=1e-13)
    assert info["n_tets"] == 120


def test_hex_inverted_and_bad_node_count_rejected(gspm_lib):
    mat = synth.fe_like_material()
    bad = synth.hex_box((3, 3, 3), (3.0, 3.0, 3.0))
    bad.tets = bad.tets.copy()
    bad.tets[4] = bad.tets[4][[1, 0, 3, 2, 5, 4, 7, 6]]            # mirrored: det J < 0
    with pytest.raises(gspm_lib.GSPMError) as e:
        gspm_lib.Context(bad, mat, 1e-12, 0.5, host_only=True)
    assert e.value.code == gspm_lib.EMESH and "hexahedron" in str(e.value)
    odd = synth.kuhn_box((3, 3, 3), (3.0, 3.0, 3.0))
    odd.tets = np.concatenate([odd.tets, odd.tets[:, :2]], axis=1)  # 6 nodes per element
    with pytest.raises(gspm_lib.GSPMError) as e:
        gspm_lib.Context(odd, mat, 1e-12, 0.5, host_only=True)
    assert e.value.code == gspm_lib.EINVAL
