"""Seeded synthetic inputs for the GSPM micromagnetics step.

This module produces *inputs only*: periodic, jittered Kuhn (Freudenthal) lattices of linear
tetrahedra stored as an unstructured mesh, element defect flags, material constants and initial
magnetisation fields.  It holds none of the method's arithmetic (no periodic wrap, no assembly,
no field evaluation); both the CUDA library and the CPU oracle consume what it returns.

Random numbers come from a counter-based splitmix64 stream (Steele, Lea & Flood 2014): output k
of stream ``s`` is ``mix64(s + (k + 1) * 0x9E3779B97F4A7C15)``.

Stored mesh layout
------------------
* ``coords``  float64 [n_stored, 3] in nm; stored node ``s = i + (nx+1) * (j + (ny+1) * k)`` for
  lattice indices ``0 <= i <= nx`` (likewise j, k).  Nodes on the maximum faces are periodic
  images of the minimum-face nodes: they carry the same in-plane jitter and sit exactly on the
  face (no jitter normal to a periodic face), so matching face nodes differ by one box length.
* ``tets``    int32 [6 * nx * ny * nz, 4]: for each cube (i fastest), six Kuhn tetrahedra, one per
  axis permutation (xyz, xzy, yxz, yzx, zxy, zyx) along the vertex path
  0 -> e_p1 -> e_p1 + e_p2 -> (1,1,1); odd permutations swap the last two vertices so that every
  tetrahedron is positively oriented.  A jitter of at most 0.2 h per axis cannot invert one.
* ``elem_magnetic`` uint8 [n_tets]: 0 when the element centroid lies inside a defect (periodic
  minimum image), else 1.
* ``hex_box`` stores the same lattice as linear hexahedra instead: ``tets`` int32
  [nx * ny * nz, 8], one element per cube with the vertices at the corners (0,0,0) (1,0,0)
  (1,1,0) (0,1,0) (0,0,1) (1,0,1) (1,1,1) (0,1,1) in that order.
* Per unique lattice node ``u = i + nx * (j + ny * k)`` (0 <= i < nx ...) fields such as the initial
  magnetisation are indexed in that order.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(stream: int, counters) -> np.ndarray:
    """Counter-based splitmix64: one 64-bit output per counter of ``stream``."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(stream & 0xFFFFFFFFFFFFFFFF) + (c + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def substream(seed: int, purpose: int) -> int:
    """Independent stream id derived from a seed and a purpose tag."""
    return int(splitmix64(seed, [purpose])[0])


def uniform01(stream: int, counters) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of splitmix64."""
    return (splitmix64(stream, counters) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(stream: int, n: int) -> np.ndarray:
    """n standard normal draws (Box-Muller on pairs of uniforms)."""
    m = (n + 1) // 2
    u1 = uniform01(stream, np.arange(0, 2 * m, 2))
    u2 = uniform01(stream, np.arange(1, 2 * m, 2))
    r = np.sqrt(-2.0 * np.log1p(-u1))
    z = np.concatenate([r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2)])
    return z[:n]


# --------------------------------------------------------------------------------------------
# Materials (SI units).  mu0 in H/m, gamma0 = mu0 * gamma_e in m / (A s), l_d = 1 nm.
# --------------------------------------------------------------------------------------------

MU0 = 1.25663706212e-6
GAMMA0 = 2.2127615e5


def fe_like_material() -> dict:
    """Fe-like cubic magnetostrictive ferromagnet (Ms in A/m, A in J/m, K1 in J/m^3, C in Pa)."""
    return dict(Ms=1.71e6, A=2.1e-11, K1=4.8e4, lambda100=2.07e-5, lambda111=-2.12e-5,
                C11=243e9, C12=138e9, C44=122e9,
                Nd=[1.0 / 3, 0, 0, 0, 1.0 / 3, 0, 0, 0, 1.0 / 3],
                sigma_ext=[0.0] * 6, gamma0=GAMMA0, mu0=MU0, l_d=1e-9)


# --------------------------------------------------------------------------------------------
# Mesh
# --------------------------------------------------------------------------------------------

@dataclass
class Mesh:
    coords: np.ndarray          # float64 [n_stored, 3], nm
    tets: np.ndarray            # int32 [n_elements, 4] tetrahedra or [n_elements, 8] hexahedra
    elem_magnetic: np.ndarray   # uint8 [n_tets]
    box_lo: np.ndarray          # float64 [3]
    box_hi: np.ndarray          # float64 [3]
    n_cells: tuple              # (nx, ny, nz)
    defects: list = field(default_factory=list)

    @property
    def n_stored(self) -> int:
        return self.coords.shape[0]

    @property
    def n_tets(self) -> int:
        return self.tets.shape[0]

    @property
    def nodes_per_elem(self) -> int:
        return self.tets.shape[1]

    @property
    def n_unique(self) -> int:
        nx, ny, nz = self.n_cells
        return nx * ny * nz


# vertex paths of the six Kuhn tetrahedra; odd permutations get their last two vertices swapped
_PERMS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
_ODD = [False, True, True, False, False, True]


def _kuhn_offsets() -> np.ndarray:
    out = np.zeros((6, 4, 3), dtype=np.int64)
    for t, (p0, p1, p2) in enumerate(_PERMS):
        v = np.zeros(3, dtype=np.int64)
        path = [v.copy()]
        for ax in (p0, p1, p2):
            v[ax] += 1
            path.append(v.copy())
        if _ODD[t]:
            path[2], path[3] = path[3], path[2]
        out[t] = np.array(path)
    return out


def _inside_defect(points: np.ndarray, d: dict, box: np.ndarray) -> np.ndarray:
    """Periodic minimum-image point-in-defect test."""
    c = np.asarray(d["center"], dtype=np.float64)
    delta = points - c
    delta -= box * np.round(delta / box)
    kind = d["kind"]
    if kind == "sphere":
        return np.einsum("ij,ij->i", delta, delta) < d["radius"] ** 2
    if kind == "ellipsoid":
        ax = np.asarray(d["semi_axes"], dtype=np.float64)
        return np.einsum("ij,ij->i", delta / ax, delta / ax) < 1.0
    if kind == "cuboid":
        hs = np.asarray(d["half_sides"], dtype=np.float64)
        return np.all(np.abs(delta) < hs, axis=1)
    raise ValueError(f"unknown defect kind {kind!r}")


# corner offsets of the hexahedron of a cube, in the element's vertex order
_HEX = np.array([(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0), (0, 0, 1), (1, 0, 1), (1, 1, 1),
                 (0, 1, 1)], dtype=np.int64)


def hex_box(n_cells, box, jitter: float = 0.0, seed: int = 0, defects=()) -> Mesh:
    """Periodic lattice of ``n_cells`` cubes spanning ``[0, box]`` (nm), one linear hexahedron
    per cube; nodes and jitter exactly as ``kuhn_box``."""
    tm = kuhn_box(n_cells, box, jitter=jitter, seed=seed)
    nx, ny, nz = tm.n_cells
    ck, cj, ci = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cube = np.stack([ci.ravel(), cj.ravel(), ck.ravel()], axis=1)
    vert = cube[:, None, :] + _HEX[None, :, :]
    hexes = (vert[..., 0] + (nx + 1) * (vert[..., 1] + (ny + 1) * vert[..., 2])).astype(np.int32)
    centroid = tm.coords[hexes].mean(axis=1)
    L = tm.box_hi
    mag = np.ones(hexes.shape[0], dtype=bool)
    for d in defects:
        mag &= ~_inside_defect(centroid, d, L)
    return Mesh(coords=tm.coords, tets=hexes, elem_magnetic=mag.astype(np.uint8),
                box_lo=tm.box_lo, box_hi=L, n_cells=tm.n_cells, defects=list(defects))


def kuhn_box(n_cells, box, jitter: float = 0.0, seed: int = 0, defects=()) -> Mesh:
    """Periodic jittered Kuhn lattice of ``n_cells`` cubes spanning ``[0, box]`` (nm)."""
    nx, ny, nz = (int(v) for v in n_cells)
    L = np.asarray(box, dtype=np.float64)
    ncell = np.array([nx, ny, nz])
    # lattice indices of stored nodes
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    idx = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)          # [n_stored, 3]
    base = idx * (L / ncell)
    for a in range(3):                                                   # max faces exactly on L
        base[idx[:, a] == ncell[a], a] = L[a]
    coords = base.copy()
    if jitter > 0.0:
        uidx = idx % ncell                                               # unique lattice node
        u = uidx[:, 0] + nx * (uidx[:, 1] + ny * uidx[:, 2])
        stream = substream(seed, 1)
        h = L / ncell
        for a in range(3):
            r = uniform01(stream, 3 * u + a)
            d = (2.0 * r - 1.0) * jitter * h[a]
            d[uidx[:, a] == 0] = 0.0                                     # stay on periodic faces
            coords[:, a] += d
    # tetrahedra
    off = _kuhn_offsets()
    ck, cj, ci = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cube = np.stack([ci.ravel(), cj.ravel(), ck.ravel()], axis=1)        # [ncubes, 3], i fastest
    vert = cube[:, None, None, :] + off[None, :, :, :]                   # [ncubes, 6, 4, 3]
    sid = vert[..., 0] + (nx + 1) * (vert[..., 1] + (ny + 1) * vert[..., 2])
    tets = sid.reshape(-1, 4).astype(np.int32)
    centroid = coords[tets].mean(axis=1)
    mag = np.ones(tets.shape[0], dtype=bool)
    for d in defects:
        mag &= ~_inside_defect(centroid, d, L)
    return Mesh(coords=coords, tets=tets, elem_magnetic=mag.astype(np.uint8),
                box_lo=np.zeros(3), box_hi=L.copy(), n_cells=(nx, ny, nz), defects=list(defects))


# --------------------------------------------------------------------------------------------
# Initial magnetisation (per unique lattice node, order u = i + nx*(j + ny*k))
# --------------------------------------------------------------------------------------------

def random_unit_m(n: int, seed: int) -> np.ndarray:
    """Per-node direction drawn from the normalised isotropic Gaussian N(0, I3)."""
    z = normal(substream(seed, 2), 3 * n).reshape(n, 3)
    return z / np.linalg.norm(z, axis=1, keepdims=True)


def uniform_m(n: int, direction=(1.0, 0.0, 0.0)) -> np.ndarray:
    d = np.asarray(direction, dtype=np.float64)
    return np.tile(d / np.linalg.norm(d), (n, 1))


# --------------------------------------------------------------------------------------------
# Workloads, named by what they are
# --------------------------------------------------------------------------------------------

def fe_box_17x17x5(seed: int = 0):
    """64x64x16 nm Fe-like box, 16x16x4 cubes (17x17x5 stored nodes), no jitter, no defect,
    seeded random unit m, zero applied field, alpha 0.5, dt 1 ps, 100 steps."""
    mesh = kuhn_box((16, 16, 4), (64.0, 64.0, 16.0), jitter=0.0, seed=seed)
    m0 = random_unit_m(mesh.n_unique, seed)
    return dict(name="fe_box_64x64x16nm_1024n", mesh=mesh, material=fe_like_material(), m0=m0,
                H=np.zeros(3), alpha=0.5, dt=1e-12, steps=100)


def sphere_inclusion_box(n_cells=(128, 128, 32), box=(512.0, 512.0, 128.0), radius=60.0, seed=1):
    """512x512x128 nm box (0.5M nodes at h = 4 nm), jitter 0.2 h, one spherical non-magnetic
    inclusion of radius 60 nm at the centre; m = e1, H = 200 A/m e1, alpha 0.5, dt 5 ps."""
    L = np.asarray(box, dtype=np.float64)
    mesh = kuhn_box(n_cells, L, jitter=0.2, seed=seed,
                    defects=[dict(kind="sphere", center=L / 2, radius=radius)])
    return dict(name=f"sphere_inclusion_{int(L[0])}x{int(L[1])}x{int(L[2])}nm_{mesh.n_unique}n",
                mesh=mesh, material=fe_like_material(), m0=uniform_m(mesh.n_unique),
                H=np.array([200.0, 0.0, 0.0]), alpha=0.5, dt=5e-12, steps=1000)


def cuboid_defect_hex_box(n_cells=(128, 128, 32), h=4.0):
    """Structured (unjittered) periodic lattice of linear hexahedra with edge h nm (128 x 128 x 32
    cells = 524,288 nodes at the default, the size class of the time-step study of Sec. 4) and
    one non-magnetic cuboid at the centre with a quarter of the box's edge on every side; m = e1,
    H = 200 A/m along e1, alpha 0.15.  The enclosing body is a needle along e1 (N_d = diag(0,
    1/2, 1/2)), so the uniform start is stable except for the defect's own stray field and
    relaxes; with N_d = I/3 the far field drives the Fe-like box into moving domains instead.
    The study varies dt; 3 ps is set here."""
    L = h * np.asarray(n_cells, dtype=np.float64)
    mesh = hex_box(n_cells, L, jitter=0.0,
                   defects=[dict(kind="cuboid", center=L / 2, half_sides=L / 8)])
    mat = fe_like_material()
    mat["Nd"] = [0.0, 0, 0, 0, 0.5, 0, 0, 0, 0.5]
    return dict(name=f"cuboid_defect_hex_{int(L[0])}x{int(L[1])}x{int(L[2])}nm_{mesh.n_unique}n",
                mesh=mesh, material=mat, m0=uniform_m(mesh.n_unique),
                H=np.array([200.0, 0.0, 0.0]), alpha=0.15, dt=3e-12, dm_tol=5e-10)


def void_cuboids_box(n_cells=(228, 228, 57), box=(1024.0, 1024.0, 256.0), seed=2):
    """1024x1024x256 nm box (2.96M nodes at h ~ 4.49 nm), jitter 0.2 h, one seeded random
    axis-aligned ellipsoidal void (semi-axes U[40,120] x U[40,120] x U[20,60] nm) and 8 random
    cuboid inclusions (sides U[20,80] nm); m = e1; field sweep -0.2 -> +0.2 T along [100] in 41
    points (H = B / mu0), alpha 0.5, dt 5 ps."""
    L = np.asarray(box, dtype=np.float64)
    s = substream(seed, 3)
    r = uniform01(s, np.arange(64))
    semi = np.array([40 + 80 * r[0], 40 + 80 * r[1], 20 + 40 * r[2]])
    centre = semi + r[3:6] * (L - 2 * semi)
    defects = [dict(kind="ellipsoid", center=centre, semi_axes=semi)]
    for c in range(8):
        q = r[6 + 6 * c: 12 + 6 * c]
        sides = 20 + 60 * q[:3]
        defects.append(dict(kind="cuboid", center=q[3:6] * L, half_sides=sides / 2))
    mesh = kuhn_box(n_cells, L, jitter=0.2, seed=seed, defects=defects)
    sweep_T = np.linspace(-0.2, 0.2, 41)
    return dict(name=f"void_cuboids_{int(L[0])}x{int(L[1])}x{int(L[2])}nm_{mesh.n_unique}n",
                mesh=mesh, material=fe_like_material(), m0=uniform_m(mesh.n_unique),
                H=np.array([sweep_T[0] / MU0, 0.0, 0.0]), H_sweep=sweep_T / MU0,
                alpha=0.5, dt=5e-12, steps_per_point=200)


def batch_member(i: int, base_seed: int = 100):
    """One mesh of the 64-mesh uneven batch: N log-uniform in [2k, 200k] nodes, box of
    4n x 4n x n cubes at h = 4 nm, one random sphere of radius U[0.1, 0.3] * Lz, random applied
    field direction with |mu0 H| in U[0, 0.2] T."""
    seed = base_seed + i
    s = substream(seed, 4)
    r = uniform01(s, np.arange(8))
    n_target = math.exp(math.log(2000) + r[0] * (math.log(200000) - math.log(2000)))
    n = max(2, int(round((n_target / 16.0) ** (1.0 / 3.0))))
    cells = (4 * n, 4 * n, n)
    L = 4.0 * np.asarray(cells, dtype=np.float64)
    radius = (0.1 + 0.2 * r[1]) * L[2]
    centre = r[2:5] * L
    mesh = kuhn_box(cells, L, jitter=0.2, seed=seed,
                    defects=[dict(kind="sphere", center=centre, radius=radius)])
    d = normal(s + 1, 3)
    Bmag = 0.2 * r[5]
    H = d / np.linalg.norm(d) * Bmag / MU0
    return dict(name=f"batch_member_{i}_{mesh.n_unique}n", mesh=mesh, material=fe_like_material(),
                m0=uniform_m(mesh.n_unique), H=H, alpha=0.5, dt=5e-12, steps=500)
