"""Small builders shared by the oracle tests (no method arithmetic)."""
import numpy as np

from oracle.mesh import WrappedMesh
from paper_2510_09812_gb300 import synth


def periodic(n_cells, box, jitter=0.0, seed=0, defects=()):
    mesh = synth.kuhn_box(n_cells, box, jitter=jitter, seed=seed, defects=defects)
    return mesh, WrappedMesh.from_synth(mesh)


def open_patch(n_cells, box, jitter=0.2, seed=3):
    """The same lattice without the periodic identification (box_hi moved out of reach), so the
    outer faces are free boundaries; returns (mesh, wrapped mesh, interior-node mask)."""
    mesh = synth.kuhn_box(n_cells, box, jitter=jitter, seed=seed)
    far = np.asarray(box, float) + 1e6
    wm = WrappedMesh(mesh.coords, mesh.tets, mesh.elem_magnetic, mesh.box_lo, far)
    nx, ny, nz = n_cells
    s = np.arange(mesh.n_stored)
    i, j, k = s % (nx + 1), (s // (nx + 1)) % (ny + 1), s // ((nx + 1) * (ny + 1))
    interior = (i > 0) & (i < nx) & (j > 0) & (j < ny) & (k > 0) & (k < nz)
    assert wm.n == mesh.n_stored and np.array_equal(wm.unique_of_stored, s)
    return mesh, wm, interior


def lattice_xyz(mesh):
    """Unjittered lattice positions of the unique nodes, order u = i + nx (j + ny k)."""
    nx, ny, nz = mesh.n_cells
    u = np.arange(nx * ny * nz)
    h = mesh.box_hi / np.array(mesh.n_cells)
    return np.stack([(u % nx) * h[0], ((u // nx) % ny) * h[1], (u // (nx * ny)) * h[2]], axis=1)
