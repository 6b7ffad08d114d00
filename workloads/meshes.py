"""Seeded synthetic hex meshes and problem set-ups (inputs only, no method arithmetic).

Conventions shared with the C interface (they are part of the input format):

* ``hex8`` lists the 8 vertex ids of a hexahedron in the VTK order: with the
  cell mapped to the unit cube, vertex k sits at
  (0,0,0) (1,0,0) (1,1,0) (0,1,0) (0,0,1) (1,0,1) (1,1,1) (0,1,1).
* Local face l of a hex is the quad ``LOCAL_FACES[l]`` (vertex positions in
  ``hex8``), ordered so that the right-hand rule gives the outward normal.
  For an unrotated lattice cell the faces are x-, x+, y-, y+, z-, z+.
* Boundary faces are given as (cell, local face) pairs with a group id; each
  group gets one boundary condition (free stream, zero gradient, symmetry,
  diffuse wall), as in the paper's ``Problem(bc_type_list, bc_data, f_init)``
  (Section 6).
"""
from __future__ import annotations

import dataclasses
import itertools
import math

import numpy as np

BC_FREESTREAM = 0
BC_ZEROGRAD = 1
BC_SYMMETRY = 2
BC_WALL = 3
BC_NAMES = {BC_FREESTREAM: "freestream", BC_ZEROGRAD: "zerograd",
            BC_SYMMETRY: "symmetry", BC_WALL: "wall"}

# Corner position of each VTK hex vertex on the unit cube.
_CORNER = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0],
                    [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]], dtype=np.int64)
LOCAL_FACES = ((0, 4, 7, 3), (1, 2, 6, 5), (0, 1, 5, 4),
               (3, 7, 6, 2), (0, 3, 2, 1), (4, 5, 6, 7))


def _proper_cube_rotations():
    """The 24 signed 3x3 permutation matrices with determinant +1."""
    out = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            m = np.zeros((3, 3), dtype=np.int64)
            for r in range(3):
                m[r, perm[r]] = signs[r]
            if round(np.linalg.det(m)) == 1:
                out.append(m)
    return out


_ROTATIONS = _proper_cube_rotations()
_CORNER_INDEX = {tuple(c): k for k, c in enumerate(_CORNER)}


def _relabel_table(rot):
    """new local vertex k takes the old vertex whose corner is rot(corner_k)."""
    tab = []
    for k in range(8):
        p = 2 * _CORNER[k] - 1                 # corner at +-1
        q = (rot @ p + 1) // 2
        tab.append(_CORNER_INDEX[tuple(int(v) for v in q)])
    return np.array(tab, dtype=np.int64)


_RELABEL = [_relabel_table(r) for r in _ROTATIONS]


@dataclasses.dataclass
class Workload:
    """A complete synthetic problem: mesh, velocity grid, gas, BCs, initial state."""
    name: str
    xyz: np.ndarray            # [n_vert, 3] float64
    hex8: np.ndarray           # [n_cell, 8] int64
    bface: np.ndarray          # [n_bface, 2] int64: (cell, local face)
    bgroup: np.ndarray         # [n_bface] int32
    N: tuple                   # velocity nodes per axis
    lo: tuple                  # velocity box lower corner
    hi: tuple                  # velocity box upper corner
    Pr: float
    omega: float
    Kn: float
    bcs: list                  # [(group, type, params[8])]
    n0: np.ndarray             # [n_cell] initial density
    u0: np.ndarray             # [n_cell, 3] initial velocity
    T0: np.ndarray             # [n_cell] initial temperature
    cell_ijk: np.ndarray       # [n_cell, 3] lattice index of each cell (for analysis)
    steps: int = 100
    cfl: float = 0.5
    rank_cap: int = 8
    tol: float = 1e-5
    h: tuple = (1.0, 1.0, 1.0)

    @property
    def n_cell(self):
        return int(self.hex8.shape[0])

    @property
    def nodes_per_cell(self):
        return int(self.N[0] * self.N[1] * self.N[2])

    def describe(self):
        return {"workload": self.name, "n_cell": self.n_cell,
                "velocity_grid": "x".join(str(int(v)) for v in self.N),
                "vbox": [list(self.lo), list(self.hi)], "Kn": self.Kn,
                "Pr": self.Pr, "omega": self.omega, "cfl": self.cfl}


def lattice_hex_mesh(shape, origin, h, hole=None, jitter=0.0, jitter_seed=None,
                     perm_seed=None, rotate_seed=None, classify=None, keep=None):
    """Hex mesh of a box lattice, optionally with a box-shaped hole.

    shape   (nx, ny, nz) cells;  origin (x0, y0, z0);  h (hx, hy, hz).
    hole    ((i0, i1), (j0, j1), (k0, k1)) half-open cell ranges removed.
    jitter  each coordinate of every vertex not on the outer box or on the hole
            surface is moved by U(-jitter*h, +jitter*h) (seeded).
    perm_seed   shuffles the cell numbering.
    rotate_seed relabels each hex by a random proper rotation of the cube, so
                that local face numbers no longer follow the x/y/z order.
    classify(ijk, axis, sign, on_outer_box) -> group id for each boundary face.
    keep(i, j, k) -> False removes that cell as well (no jitter with it).
    Returns (xyz, hex8, bface, bgroup, cell_ijk).
    """
    nx, ny, nz = shape
    hx, hy, hz = h
    gi, gj, gk = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1),
                             indexing="ij")
    lat = np.stack([gi.ravel(), gj.ravel(), gk.ravel()], axis=1)
    xyz = np.empty((lat.shape[0], 3), dtype=np.float64)
    xyz[:, 0] = origin[0] + lat[:, 0] * hx
    xyz[:, 1] = origin[1] + lat[:, 1] * hy
    xyz[:, 2] = origin[2] + lat[:, 2] * hz

    def vid(i, j, k):
        return (i * (ny + 1) + j) * (nz + 1) + k

    def in_hole(i, j, k):
        if keep is not None and not keep(i, j, k):
            return True
        if hole is None:
            return False
        (i0, i1), (j0, j1), (k0, k1) = hole
        return i0 <= i < i1 and j0 <= j < j1 and k0 <= k < k1

    if jitter > 0.0:
        if keep is not None:
            raise ValueError("jitter with a removal mask is not supported")
        rng = np.random.default_rng(jitter_seed)
        fixed = ((lat[:, 0] == 0) | (lat[:, 0] == nx) | (lat[:, 1] == 0) | (lat[:, 1] == ny)
                 | (lat[:, 2] == 0) | (lat[:, 2] == nz))
        if hole is not None:
            (i0, i1), (j0, j1), (k0, k1) = hole
            fixed |= ((lat[:, 0] >= i0) & (lat[:, 0] <= i1) & (lat[:, 1] >= j0)
                      & (lat[:, 1] <= j1) & (lat[:, 2] >= k0) & (lat[:, 2] <= k1))
        d = rng.uniform(-1.0, 1.0, size=xyz.shape) * jitter * np.array([hx, hy, hz])
        xyz = xyz + np.where(fixed[:, None], 0.0, d)

    cells = [(i, j, k) for i in range(nx) for j in range(ny) for k in range(nz)
             if not in_hole(i, j, k)]
    cell_ijk = np.array(cells, dtype=np.int64).reshape(-1, 3)
    hex8 = np.empty((len(cells), 8), dtype=np.int64)
    for c, (i, j, k) in enumerate(cells):
        for v in range(8):
            dx, dy, dz = _CORNER[v]
            hex8[c, v] = vid(i + dx, j + dy, k + dz)

    # boundary faces in lattice terms: (cell, axis, sign)
    blat = []
    for c, (i, j, k) in enumerate(cells):
        for axis in range(3):
            for sign in (-1, 1):
                nb = [i, j, k]
                nb[axis] += sign
                outer = not (0 <= nb[0] < nx and 0 <= nb[1] < ny and 0 <= nb[2] < nz)
                if outer or in_hole(*nb):
                    g = 0 if classify is None else classify((i, j, k), axis, sign, outer)
                    blat.append((c, axis, sign, g))

    if rotate_seed is not None:
        rng = np.random.default_rng(rotate_seed)
        picks = rng.integers(0, len(_RELABEL), size=hex8.shape[0])
        hex8 = np.stack([hex8[c, _RELABEL[picks[c]]] for c in range(hex8.shape[0])])

    # local face index of each boundary face: match the vertex set
    bface = np.empty((len(blat), 2), dtype=np.int64)
    bgroup = np.empty(len(blat), dtype=np.int32)
    for b, (c, axis, sign, g) in enumerate(blat):
        i, j, k = cells[c]
        canon = LOCAL_FACES[2 * axis + (1 if sign > 0 else 0)]
        want = set()
        for v in canon:
            dx, dy, dz = _CORNER[v]
            want.add(vid(i + dx, j + dy, k + dz))
        for lf in range(6):
            if set(int(hex8[c, v]) for v in LOCAL_FACES[lf]) == want:
                bface[b] = (c, lf)
                break
        else:  # pragma: no cover - the relabelling is a bijection
            raise RuntimeError("face not found")
        bgroup[b] = g

    if perm_seed is not None:
        rng = np.random.default_rng(perm_seed)
        perm = rng.permutation(hex8.shape[0])      # new cell q is old cell perm[q]
        inv = np.empty_like(perm)
        inv[perm] = np.arange(perm.size)
        hex8 = hex8[perm]
        cell_ijk = cell_ijk[perm]
        bface = bface.copy()
        bface[:, 0] = inv[bface[:, 0]]
        order = rng.permutation(bface.shape[0])
        bface = bface[order]
        bgroup = bgroup[order]
    return xyz, hex8, bface, bgroup, cell_ijk


def _params(n=0.0, u=(0.0, 0.0, 0.0), T=0.0, Tw=0.0, uw=(0.0, 0.0, 0.0)):
    """BC parameter block [n, u1, u2, u3, T, 0, 0, 0].

    Free stream: the prescribed Maxwellian's (n, u, T).  Diffuse wall: slot 0 unused
    (the wall density follows from impermeability), slots 1..3 the wall velocity,
    slot 4 the wall temperature."""
    p = np.zeros(8, dtype=np.float64)
    if Tw > 0.0:
        p[1:4] = uw
        p[4] = Tw
    else:
        p[0] = n
        p[1:4] = u
        p[4] = T
    return p


def sod_row(N=12, ncell=16, vmax=5.0, Kn=0.1, steps=100, seed=0):
    """16 cube cells in a row on x in [0,1]; symmetry on the side faces, zero-gradient ends.

    Left half n=1, T=1; right half n=0.5, T=0.8; u=0.  Cell numbering, local vertex
    numbering and boundary-face order are shuffled (seeded) so that the solver sees an
    unstructured mesh.
    """
    h = 1.0 / ncell

    def classify(ijk, axis, sign, outer):
        return 0 if axis == 0 else 1

    xyz, hex8, bface, bgroup, ijk = lattice_hex_mesh(
        (ncell, 1, 1), (0.0, 0.0, 0.0), (h, h, h), perm_seed=seed,
        rotate_seed=None if seed is None else seed + 1, classify=classify)
    left = ijk[:, 0] < ncell // 2
    n0 = np.where(left, 1.0, 0.5)
    T0 = np.where(left, 1.0, 0.8)
    u0 = np.zeros((hex8.shape[0], 3))
    return Workload(
        name=f"sod_row_{ncell}x{N}^3", xyz=xyz, hex8=hex8, bface=bface, bgroup=bgroup,
        N=(N, N, N), lo=(-vmax,) * 3, hi=(vmax,) * 3, Pr=2.0 / 3.0, omega=0.81, Kn=Kn,
        bcs=[(0, BC_ZEROGRAD, np.zeros(8)), (1, BC_SYMMETRY, np.zeros(8))],
        n0=n0, u0=u0, T0=T0, cell_ijk=ijk, steps=steps, h=(h, h, h))


def cavity(nside=16, N=32, vmax=6.0, Kn=0.1, lid=0.2, Tw=1.0, rank_cap=8, tol=1e-5,
           steps=500, seed=None, jitter=0.0):
    """Lid-driven cubic cavity on [0,1]^3 with nside^3 cubes; all walls diffuse at Tw;
    the y=1 wall moves tangentially with velocity (lid, 0, 0).  IC: n=1, T=1, u=0."""
    h = 1.0 / nside

    def classify(ijk, axis, sign, outer):
        return 1 if (axis == 1 and sign > 0) else 0

    xyz, hex8, bface, bgroup, ijk = lattice_hex_mesh(
        (nside,) * 3, (0.0, 0.0, 0.0), (h, h, h), jitter=jitter,
        jitter_seed=None if seed is None else seed + 2, perm_seed=seed,
        rotate_seed=None if seed is None else seed + 1, classify=classify)
    nc = hex8.shape[0]
    return Workload(
        name=f"cavity_{nside}^3x{N}^3", xyz=xyz, hex8=hex8, bface=bface, bgroup=bgroup,
        N=(N, N, N), lo=(-vmax,) * 3, hi=(vmax,) * 3, Pr=2.0 / 3.0, omega=0.81, Kn=Kn,
        bcs=[(0, BC_WALL, _params(Tw=Tw)), (1, BC_WALL, _params(Tw=Tw, uw=(lid, 0.0, 0.0)))],
        n0=np.ones(nc), u0=np.zeros((nc, 3)), T0=np.ones(nc), cell_ijk=ijk, steps=steps,
        rank_cap=rank_cap, tol=tol, h=(h, h, h))


def obstacle(lattice=(64, 40, 40), N=64, vmax=8.0, Kn=0.05, mach_u=3.0 * math.sqrt(5.0 / 6.0),
             jitter=0.1, jitter_seed=1234, perm_seed=1, rank_cap=20, tol=1e-5, steps=100):
    """Free stream (n=1, T=1, u=(mach_u,0,0)) past a unit cube obstacle [-1/2,1/2]^3 in the
    box x in [-3,5], y,z in [-2.5,2.5].  Interior vertices jittered by U(+-jitter*h); the
    outer-box and obstacle vertices stay fixed.  Outer faces: free stream; obstacle:
    diffuse wall at T=1.  The default lattice (64,40,40) gives 101,888 cells; (16,10,10)
    gives 1,592 cells."""
    nx, ny, nz = lattice
    hx, hy, hz = 8.0 / nx, 5.0 / ny, 5.0 / nz
    hole = ((int(round(2.5 / hx)), int(round(3.5 / hx))),
            (int(round(2.0 / hy)), int(round(3.0 / hy))),
            (int(round(2.0 / hz)), int(round(3.0 / hz))))

    def classify(ijk, axis, sign, outer):
        return 0 if outer else 1

    xyz, hex8, bface, bgroup, ijk = lattice_hex_mesh(
        lattice, (-3.0, -2.5, -2.5), (hx, hy, hz), hole=hole, jitter=jitter,
        jitter_seed=jitter_seed, perm_seed=perm_seed, classify=classify)
    nc = hex8.shape[0]
    u0 = np.zeros((nc, 3))
    u0[:, 0] = mach_u
    return Workload(
        name=f"obstacle_{nc}x{N}^3", xyz=xyz, hex8=hex8, bface=bface, bgroup=bgroup,
        N=(N, N, N), lo=(-vmax,) * 3, hi=(vmax,) * 3, Pr=2.0 / 3.0, omega=0.81, Kn=Kn,
        bcs=[(0, BC_FREESTREAM, _params(n=1.0, u=(mach_u, 0.0, 0.0), T=1.0)),
             (1, BC_WALL, _params(Tw=1.0))],
        n0=np.ones(nc), u0=u0, T0=np.ones(nc), cell_ijk=ijk, steps=steps,
        rank_cap=rank_cap, tol=tol, h=(hx, hy, hz))


def specular_box(shape=(2, 2, 2), N=12, vmax=4.4, Kn=0.5, seed=3, jitter=0.0, wall_group=None):
    """Closed box [0,1]^3 with symmetry (specular) planes on every side and a random
    non-uniform initial state (n in [0.5,1.5], |u|<0.3, T in [0.7,1.3]).  If
    ``wall_group`` is an axis index, the two faces normal to it become diffuse walls
    at T=1 instead."""
    h = tuple(1.0 / s for s in shape)

    def classify(ijk, axis, sign, outer):
        return 1 if (wall_group is not None and axis == wall_group) else 0

    xyz, hex8, bface, bgroup, ijk = lattice_hex_mesh(
        shape, (0.0, 0.0, 0.0), h, jitter=jitter, jitter_seed=seed, perm_seed=seed,
        rotate_seed=seed + 1, classify=classify)
    nc = hex8.shape[0]
    rng = np.random.default_rng(seed + 7)
    bcs = [(0, BC_SYMMETRY, np.zeros(8))]
    if wall_group is not None:
        bcs.append((1, BC_WALL, _params(Tw=1.0)))
    return Workload(
        name="specular_box", xyz=xyz, hex8=hex8, bface=bface, bgroup=bgroup,
        N=(N, N, N), lo=(-vmax,) * 3, hi=(vmax,) * 3, Pr=2.0 / 3.0, omega=0.81, Kn=Kn,
        bcs=bcs, n0=rng.uniform(0.5, 1.5, nc), u0=rng.uniform(-0.3, 0.3, (nc, 3)) / math.sqrt(3),
        T0=rng.uniform(0.7, 1.3, nc), cell_ijk=ijk, steps=10, h=h)


def closed_freestream_box(shape=(3, 3, 3), N=12, vmax=5.0, u=(0.3, -0.2, 0.1), Kn=1e12,
                          jitter=0.2, seed=11):
    """Jittered closed box with free-stream faces and the same uniform Maxwellian as the
    initial state (n=1, T=1, velocity u): the exact solution is steady."""
    h = tuple(1.0 / s for s in shape)
    xyz, hex8, bface, bgroup, ijk = lattice_hex_mesh(
        shape, (0.0, 0.0, 0.0), h, jitter=jitter, jitter_seed=seed, perm_seed=seed,
        rotate_seed=seed + 1)
    nc = hex8.shape[0]
    return Workload(
        name="closed_freestream_box", xyz=xyz, hex8=hex8, bface=bface, bgroup=bgroup,
        N=(N, N, N), lo=(-vmax,) * 3, hi=(vmax,) * 3, Pr=2.0 / 3.0, omega=0.81, Kn=Kn,
        bcs=[(0, BC_FREESTREAM, _params(n=1.0, u=u, T=1.0))],
        n0=np.ones(nc), u0=np.tile(np.asarray(u, float), (nc, 1)), T0=np.ones(nc),
        cell_ijk=ijk, steps=5, h=h)


def channel(n_cell_target=2000, N=24, vmax=6.0, Kn=0.1, kind="poiseuille", rank_cap=8,
            tol=1e-5, seed=0):
    """Rectangular duct L:H:W = 4:1:1 made of axis-aligned cubes, about n_cell_target cells.

    kind='poiseuille': end reservoirs (free stream) n=1.0 and n=0.5 at T=1, walls T=1.
    kind='transpiration': walls with T rising linearly 1 -> 2 along x (one BC group per
    x-slab), reservoirs n=1 at T=1 and T=2.
    """
    m = max(1, int(round((n_cell_target / 4.0) ** (1.0 / 3.0))))
    shape = (4 * m, m, m)
    h = (1.0 / m,) * 3
    nxs = shape[0]

    def classify(ijk, axis, sign, outer):
        if axis == 0:
            return 0 if sign < 0 else 1
        return 2 + ijk[0] if kind == "transpiration" else 2

    xyz, hex8, bface, bgroup, ijk = lattice_hex_mesh(
        shape, (0.0, 0.0, 0.0), h, perm_seed=seed, classify=classify)
    nc = hex8.shape[0]
    if kind == "poiseuille":
        bcs = [(0, BC_FREESTREAM, _params(n=1.0, T=1.0)),
               (1, BC_FREESTREAM, _params(n=0.5, T=1.0)),
               (2, BC_WALL, _params(Tw=1.0))]
        n0 = 1.0 - 0.5 * (ijk[:, 0] + 0.5) / nxs
        T0 = np.ones(nc)
    else:
        bcs = [(0, BC_FREESTREAM, _params(n=1.0, T=1.0)),
               (1, BC_FREESTREAM, _params(n=1.0, T=2.0))]
        for s in range(nxs):
            bcs.append((2 + s, BC_WALL, _params(Tw=1.0 + (s + 0.5) / nxs)))
        n0 = np.ones(nc)
        T0 = 1.0 + (ijk[:, 0] + 0.5) / nxs
    return Workload(
        name=f"channel_{kind}_{nc}x{N}^3", xyz=xyz, hex8=hex8, bface=bface, bgroup=bgroup,
        N=(N, N, N), lo=(-vmax,) * 3, hi=(vmax,) * 3, Pr=2.0 / 3.0, omega=0.81, Kn=Kn,
        bcs=bcs, n0=n0, u0=np.zeros((nc, 3)), T0=T0, cell_ijk=ijk, steps=1000,
        rank_cap=rank_cap, tol=tol, h=h)


# Section 7 free stream (argon) in the units of these workloads: speeds in
# sqrt(2 R T_inf), R = 8.314 / 0.039948 J/(kg K), T_inf = 200 K.
_AR_R = 8.314462618 / 0.039948
_C_UNIT = math.sqrt(2.0 * _AR_R * 200.0)          # m/s per speed unit


def cylinder(n_theta=40, n_r=40, N=64, r_out=8.0, dr1=0.05, Kn=0.552, Tw=5.0,
             u_inf=2630.0 / _C_UNIT, vmax=6400.0 / _C_UNIT, rank_cap=16, tol=1e-5,
             seed=None):
    """Hypersonic flow past a circular cylinder, the shape of Section 7's test problem
    (its mesh is not available, so this O-grid stands in for it).

    Half of the flow (y >= 0) around a unit-radius cylinder (lengths in radii), solved
    as 3D with one cell along z: n_theta cells over the half circle (theta = 0 is the
    downstream axis), n_r cells radially with geometric growth from dr1 at the wall to
    the outer radius r_out; 1600 cells at the defaults, as in Section 7.  Groups:
    0 free stream on the outer boundary (n = 1, T = 1, u = (u_inf, 0, 0)), 1 the diffuse
    wall at Tw (Section 7: Tw = 5 T_inf), 2 symmetry on the y = 0 plane and on both z
    planes.  Free stream v0 = 2630 m/s, T0 = 200 K of argon: u_inf = 9.12 (Mach 10),
    the velocity box +-6400 m/s = +-22.2, N = 64 nodes per axis as in Section 7;
    viscosity exponent 0.734; Kn = 0.552 is the printed Kn ~ 0.56 in the collision
    frequency of these units.  Cells are numbered radius-fastest (or shuffled with seed).
    The curved wall's faces leave the coordinate planes, which the full format takes and
    the Tucker format does not (`cylinder_staircase` is its Tucker-ready variant).
    """
    g = _growth(dr1, r_out - 1.0, n_r)
    r = np.concatenate([[1.0], 1.0 + dr1 * np.cumsum(g ** np.arange(n_r))])
    r[-1] = r_out
    th = math.pi * np.arange(n_theta + 1) / n_theta
    hz = math.pi / n_theta
    # vertex (i_theta, j_r, k_z), k fastest; y = 0 exactly on the symmetry line
    xyz = np.empty(((n_theta + 1) * (n_r + 1) * 2, 3))
    vid = lambda i, j, k: (i * (n_r + 1) + j) * 2 + k  # noqa: E731
    for i in range(n_theta + 1):
        c, sn = math.cos(th[i]), math.sin(th[i])
        if i == 0 or i == n_theta:
            sn = 0.0
            c = 1.0 if i == 0 else -1.0
        for j in range(n_r + 1):
            for k in range(2):
                xyz[vid(i, j, k)] = (r[j] * c, r[j] * sn, k * hz)
    # local hex axes (x, y, z) = (radius, theta, z): right-handed, positive volumes
    cells = [(i, j) for i in range(n_theta) for j in range(n_r)]
    hex8 = np.empty((len(cells), 8), dtype=np.int64)
    for q, (i, j) in enumerate(cells):
        for v in range(8):
            dx, dy, dz = _CORNER[v]
            hex8[q, v] = vid(i + dy, j + dx, dz)
    bface, bgroup = [], []
    for q, (i, j) in enumerate(cells):
        if j == 0:
            bface.append((q, 0)); bgroup.append(1)          # wall (local x-)
        if j == n_r - 1:
            bface.append((q, 1)); bgroup.append(0)          # outer free stream (local x+)
        if i == 0:
            bface.append((q, 2)); bgroup.append(2)          # theta = 0 line (local y-)
        if i == n_theta - 1:
            bface.append((q, 3)); bgroup.append(2)          # theta = pi line (local y+)
        bface.append((q, 4)); bgroup.append(2)              # z planes
        bface.append((q, 5)); bgroup.append(2)
    bface = np.array(bface, dtype=np.int64)
    bgroup = np.array(bgroup, dtype=np.int32)
    ijk = np.array([(i, j, 0) for i, j in cells], dtype=np.int64)
    if seed is not None:
        rng = np.random.default_rng(seed)
        perm = rng.permutation(hex8.shape[0])
        inv = np.empty_like(perm)
        inv[perm] = np.arange(perm.size)
        hex8, ijk = hex8[perm], ijk[perm]
        bface[:, 0] = inv[bface[:, 0]]
    nc = hex8.shape[0]
    u0 = np.tile([u_inf, 0.0, 0.0], (nc, 1))
    return Workload(
        name=f"cylinder_{nc}x{N}^3", xyz=xyz, hex8=hex8, bface=bface, bgroup=bgroup,
        N=(N, N, N), lo=(-vmax,) * 3, hi=(vmax,) * 3, Pr=2.0 / 3.0, omega=0.734, Kn=Kn,
        bcs=[(0, BC_FREESTREAM, _params(n=1.0, u=(u_inf, 0.0, 0.0), T=1.0)),
             (1, BC_WALL, _params(Tw=Tw)),
             (2, BC_SYMMETRY, np.zeros(8))],
        n0=np.ones(nc), u0=u0, T0=np.ones(nc), cell_ijk=ijk, steps=4000,
        rank_cap=rank_cap, tol=tol, h=(dr1, hz, hz))


def cylinder_staircase(h=0.25, x_range=(-5.0, 7.0), y_max=8.5, N=64, Kn=0.552, Tw=5.0,
                       u_inf=2630.0 / _C_UNIT, vmax=6400.0 / _C_UNIT, rank_cap=16, tol=1e-5,
                       seed=None):
    """The Mach-10 cylinder of `cylinder` on a Cartesian lattice: square cells of side h
    over x in x_range, y in [0, y_max], one cell along z, with the cells whose centre lies
    inside the unit circle removed, so the wall is a staircase and every face lies on a
    coordinate plane (the Tucker format takes diffuse walls only there).  1607 cells at
    the defaults.  Groups as in `cylinder`: 0 free stream (x ends and y = y_max), 1 the
    wall at Tw, 2 symmetry (y = 0 and both z planes)."""
    nx = int(round((x_range[1] - x_range[0]) / h))
    ny = int(round(y_max / h))

    def keep(i, j, k):
        xc = x_range[0] + (i + 0.5) * h
        yc = (j + 0.5) * h
        return xc * xc + yc * yc >= 1.0

    def classify(ijk, axis, sign, outer):
        if not outer:
            return 1
        if axis == 2 or (axis == 1 and sign < 0):
            return 2
        return 0

    xyz, hex8, bface, bgroup, ijk = lattice_hex_mesh(
        (nx, ny, 1), (x_range[0], 0.0, 0.0), (h, h, h), perm_seed=seed, classify=classify,
        keep=keep)
    nc = hex8.shape[0]
    return Workload(
        name=f"cylinder_staircase_{nc}x{N}^3", xyz=xyz, hex8=hex8, bface=bface, bgroup=bgroup,
        N=(N, N, N), lo=(-vmax,) * 3, hi=(vmax,) * 3, Pr=2.0 / 3.0, omega=0.734, Kn=Kn,
        bcs=[(0, BC_FREESTREAM, _params(n=1.0, u=(u_inf, 0.0, 0.0), T=1.0)),
             (1, BC_WALL, _params(Tw=Tw)),
             (2, BC_SYMMETRY, np.zeros(8))],
        n0=np.ones(nc), u0=np.tile([u_inf, 0.0, 0.0], (nc, 1)), T0=np.ones(nc),
        cell_ijk=ijk, steps=4000, rank_cap=rank_cap, tol=tol, h=(h, h, h))


def _growth(d1, length, n):
    """Ratio q of the geometric series d1 (1 + q + ... + q^(n-1)) = length (bisection)."""
    if abs(d1 * n - length) < 1e-12 * length:
        return 1.0
    lo, hi = (1.0, 10.0) if d1 * n < length else (1e-6, 1.0)
    for _ in range(200):
        q = 0.5 * (lo + hi)
        s = d1 * (q ** n - 1.0) / (q - 1.0)
        if (s < length) == (d1 * n < length):
            lo = q
        else:
            hi = q
    return 0.5 * (lo + hi)


def uniform_random_tucker_ranks(n_cell, lo=4, hi=20, seed=42):
    """Per-cell Tucker ranks drawn uniformly from {lo..hi} in each mode (seeded)."""
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=(n_cell, 3)).astype(np.int32)
