"""Oracle mesh layer against closed forms: lattice wrap, volumes, adjacency, RCM."""
import numpy as np
import pytest

from oracle.mesh import WrappedMesh, csr_pattern, rcm_order, node_adjacency
from paper_2510_09812_gb300 import synth
from oracle_helpers import periodic


@pytest.mark.parametrize("cells,box,jit", [((16, 16, 4), (64, 64, 16), 0.0),
                                           ((7, 5, 3), (21.0, 20.0, 9.0), 0.2)])
def test_wrap_matches_lattice_index(cells, box, jit):
    # Sec. 2.5: max-face nodes are the min-face nodes; on the lattice the unique index of stored
    # node (i, j, k) is (i mod nx) + nx ((j mod ny) + ny (k mod nz)).
    mesh, wm = periodic(cells, box, jitter=jit, seed=5)
    nx, ny, nz = cells
    s = np.arange(mesh.n_stored)
    i, j, k = s % (nx + 1), (s // (nx + 1)) % (ny + 1), s // ((nx + 1) * (ny + 1))
    expect = (i % nx) + nx * ((j % ny) + ny * (k % nz))
    assert wm.n == nx * ny * nz
    assert np.array_equal(wm.unique_of_stored, expect)


def test_tet_volumes_fill_the_periodic_box():
    # jitter moves nodes but the periodic cell keeps its volume exactly
    mesh, wm = periodic((6, 5, 4), (24.0, 20.0, 16.0), jitter=0.2, seed=9)
    assert np.all(wm.detJ > 0)
    assert wm.volume == pytest.approx(24 * 20 * 16, rel=1e-13)


def test_periodic_kuhn_adjacency_has_15_entries_per_row():
    # each node of a Kuhn lattice touches 24 tets and 14 neighbours
    mesh, wm = periodic((5, 4, 3), (5.0, 4.0, 3.0), jitter=0.2, seed=1)
    rowptr, cols = csr_pattern(wm.tets, wm.n)
    assert np.all(np.diff(rowptr) == 15)
    counts = np.bincount(wm.tets.ravel(), minlength=wm.n)
    assert np.all(counts == 24)
    A = np.zeros((wm.n, wm.n), bool)
    A[np.repeat(np.arange(wm.n), 15), cols] = True
    assert np.array_equal(A, A.T)
    for r in range(wm.n):
        seg = cols[rowptr[r]:rowptr[r + 1]]
        assert np.all(np.diff(seg) > 0)


def test_rcm_hand_worked_chain():
    # chain of 4 tets over 7 positions, relabelled; worked by hand from the stated tie-breaks:
    # start = min degree (3) with lowest label -> label 2 (position 6); BFS by (degree, label).
    labels = np.array([3, 5, 0, 6, 1, 4, 2])
    tets = np.array([[labels[p], labels[p + 1], labels[p + 2], labels[p + 3]] for p in range(4)])
    assert rcm_order(tets, 7).tolist() == [3, 5, 0, 6, 1, 4, 2]


def test_rcm_is_a_breadth_first_permutation():
    mesh, wm = periodic((6, 6, 3), (6.0, 6.0, 3.0), jitter=0.2, seed=2)
    perm = rcm_order(wm.tets, wm.n)
    assert sorted(perm.tolist()) == list(range(wm.n))
    # reversed order is a BFS: each node (after the first of its component) has a neighbour
    # earlier in the forward order
    fwd = perm[::-1]
    pos = np.empty(wm.n, int)
    pos[fwd] = np.arange(wm.n)
    adj = node_adjacency(wm.tets, wm.n)
    for v in fwd[1:]:
        assert min(pos[w] for w in adj[v]) < pos[v]
