"""The synthetic Mach-10 cylinder (workloads.cylinder), the stand-in for Section 7's test
problem: its geometry against closed forms, its boundary groups, and the compression
properties Section 7 reports, on a small case the oracle finishes in seconds.

* The mesh's volume is that of the polygonal half annulus, n (1/2) sin(pi/n)
  (R^2 - 1) h_z, exactly; every cell is closed.
* Symmetry faces lie on the y = 0 and z planes with exact axis normals; wall normals
  point into the cylinder.
* Section 7: ranks stay minimal (1, a Maxwellian) where the gas is still the free
  stream and grow near the wall; the mean compression ratio grows as eps shrinks
  (the per-mode truncation rule keeps more terms for a smaller eps).
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import tucker as tk


def test_cylinder_geometry_closed_form(oracle_lib):
    n_theta, n_r, r_out = 12, 8, 6.0
    wl = W.cylinder(n_theta=n_theta, n_r=n_r, N=6, r_out=r_out, dr1=0.1)
    o = oracle_lib.FullGridOracle(wl)
    vol, fcell, fgeo = o.geometry()
    hz = math.pi / n_theta
    exact = n_theta * 0.5 * math.sin(math.pi / n_theta) * (r_out ** 2 - 1.0) * hz
    assert abs(vol.sum() - exact) < 1e-13 * exact
    assert np.all(vol > 0)
    # closure: sum of outward area vectors of every cell vanishes
    s = np.zeros((wl.n_cell, 3))
    for j in range(fcell.shape[0]):
        a = fgeo[j, 0] * fgeo[j, 1:]
        s[fcell[j, 0]] += a
        if fcell[j, 1] >= 0:
            s[fcell[j, 1]] -= a
    assert np.max(np.abs(s)) < 1e-14
    # boundary groups: wall and outer rings of n_theta faces, symmetry on the rest
    b = fcell[:, 1] < 0
    groups = fcell[b, 2]
    assert np.sum(groups == 1) == n_theta and np.sum(groups == 0) == n_theta
    assert np.sum(groups == 2) == 2 * n_r + 2 * n_theta * n_r
    e = fgeo[b, 1:]
    sym = e[groups == 2]
    assert np.all(np.isclose(np.max(np.abs(sym), axis=1), 1.0, rtol=0, atol=0))
    # wall normals, outward from the gas, point towards the axis
    centre = np.array([wl.xyz[h].mean(axis=0) for h in wl.hex8])
    wall_cells = fcell[b][groups == 1, 0]
    ew = e[groups == 1]
    assert np.all(np.sum(ew[:, :2] * centre[wall_cells, :2], axis=1) < 0)


def test_cylinder_parameters_are_section7s():
    """Mach 10 argon free stream (v0 = 2630 m/s, T0 = 200 K), box +-6400 m/s, N = 64,
    Tw = 5 T0, viscosity exponent 0.734, 1600 cells."""
    wl = W.cylinder()
    assert wl.n_cell == 1600 and wl.N == (64, 64, 64)
    u = wl.u0[0, 0]
    mach = u / math.sqrt(5.0 / 3.0 / 2.0)      # sound speed sqrt(gamma R T) in these units
    assert abs(mach - 10.0) < 0.02
    assert abs(wl.hi[0] / u - 6400.0 / 2630.0) < 1e-12
    assert wl.omega == 0.734
    tw = [p[4] for g, t, p in wl.bcs if t == W.BC_WALL]
    assert tw == [5.0]


def test_cylinder_shuffled_numbering_is_a_valid_mesh(oracle_lib):
    wl = W.cylinder(n_theta=8, n_r=5, N=6, seed=3)
    o = oracle_lib.FullGridOracle(wl)
    vol, _, _ = o.geometry()
    wl0 = W.cylinder(n_theta=8, n_r=5, N=6)
    vol0, _, _ = oracle_lib.FullGridOracle(wl0).geometry()
    assert abs(vol.sum() - vol0.sum()) < 1e-13 * vol0.sum()


def test_cylinder_ranks_grow_near_the_wall_and_with_accuracy(oracle_lib):
    wl = W.cylinder(n_theta=8, n_r=10, N=16, r_out=6.0, dr1=0.2)
    o = oracle_lib.FullGridOracle(wl)
    o.step(4, o.dt())                # the wall's influence has moved 4 cells at most
    f = o.f()
    j_r = wl.cell_ijk[:, 1]
    C, grown = {}, {}
    for eps in (1e-3, 1e-4, 1e-5):
        r = np.array([tk.ranks(tk.hosvd(f[c], eps)[0]) for c in range(wl.n_cell)])
        C[eps] = np.mean([tk.compression(x, 16) for x in r])
        assert np.all(r[j_r >= 6] == 1)           # untouched free stream: rank 1
        wall = r[j_r == 0].max(axis=1)
        assert wall.max() > 1                      # the wall's gas is no Maxwellian
        grown[eps] = int(np.sum(wall > 1))
    assert C[1e-3] <= C[1e-4] <= C[1e-5] and C[1e-3] < C[1e-5]
    assert grown[1e-3] <= grown[1e-4] <= grown[1e-5] and grown[1e-5] == 8


def test_staircase_cylinder_geometry(oracle_lib):
    """The lattice variant: the rectangle minus the cells whose centre lies in the unit
    half disc, every face on a coordinate plane, the wall facing the removed cells."""
    h = 0.25
    wl = W.cylinder_staircase(h=h, N=6)
    o = oracle_lib.FullGridOracle(wl)
    vol, fcell, fgeo = o.geometry()
    nx, ny = 48, 34
    removed = sum(1 for i in range(nx) for j in range(ny)
                  if (-5.0 + (i + 0.5) * h) ** 2 + ((j + 0.5) * h) ** 2 < 1.0)
    assert wl.n_cell == nx * ny - removed == 1606
    assert abs(vol.sum() - wl.n_cell * h ** 3) < 1e-12
    assert np.all(np.max(np.abs(fgeo[:, 1:]), axis=1) == 1.0)
    b = fcell[:, 1] < 0
    groups = fcell[b, 2]
    assert np.sum(groups == 0) == 2 * ny + nx                 # x ends and the top
    centre = np.array([wl.xyz[q].mean(axis=0) for q in wl.hex8])
    wc = fcell[b][groups == 1, 0]
    ew = fgeo[b][groups == 1, 1:]
    nxt = centre[wc, :2] + h * ew[:, :2]                     # the removed neighbour's centre
    assert np.all(np.sum(nxt ** 2, axis=1) < 1.0)


def _closed_annulus(Tw_outer=1.0, Tw_inner=1.0, N=12, vmax=5.0):
    """The O-grid with the outer circle turned into a diffuse wall too: a closed annulus
    bounded by curved walls and the symmetry planes, gas at rest."""
    wl = W.cylinder(n_theta=8, n_r=4, N=N, r_out=3.0, dr1=0.4, Kn=0.5, u_inf=0.0, vmax=vmax)
    wl.bcs = [(0, W.BC_WALL, np.array([0, 0, 0, 0, Tw_outer, 0, 0, 0], float)),
              (1, W.BC_WALL, np.array([0, 0, 0, 0, Tw_inner, 0, 0, 0], float)),
              (2, W.BC_SYMMETRY, np.zeros(8))]
    return wl


def test_curved_walls_are_impermeable(oracle_lib):
    """Section 2 (wall-bc-f): the wall density from the discrete impermeability sum makes
    the mass flux through every wall face zero, on faces off the coordinate planes as on
    them, so a closed annulus keeps its mass (a hot inner wall drives the gas).  The
    velocity grid is fine enough (spacing 0.4) that the collision term's quadrature defect
    is far below round-off."""
    wl = _closed_annulus(Tw_outer=1.0, Tw_inner=3.0, N=32, vmax=6.2)
    o = oracle_lib.FullGridOracle(wl)
    vol, _, _ = o.geometry()

    def mass():
        return float(np.sum(vol * o.macro()[:, 0]))
    m0 = mass()
    o.step(10, o.dt())
    assert abs(mass() - m0) < 1e-13 * m0
    assert np.max(np.abs(o.macro()[:, 4] - 1.0)) > 1e-3      # the hot wall heated the gas


def test_curved_wall_density_equals_gas_density_at_equilibrium(oracle_lib):
    """Gas at rest at the wall temperature: on a velocity grid symmetric under xi -> -xi
    the outgoing and incoming half-range sums pair up node by node for any normal, so the
    reflected density equals the gas density on curved faces too."""
    wl = _closed_annulus()
    wl.n0 = np.full(wl.n_cell, 0.8)
    o = oracle_lib.FullGridOracle(wl)
    o.step(1, 1e-4)
    nw = o.wall_density()
    _, fcell, fgeo = o.geometry()
    wall = fcell[:, 1] < 0
    wall &= np.isin(fcell[:, 2], (0, 1))
    assert np.sum(np.max(np.abs(fgeo[wall, 1:]), axis=1) < 0.999) > 8   # curved faces
    assert np.max(np.abs(nw[wall] - 0.8)) < 1e-13


def test_compression_study_script_runs(oracle_lib, tmp_path, monkeypatch):
    """The script that wrote tests/golden/cylinder*_compression.json, on a tiny case:
    its output has the fields the stored tables were read from."""
    import importlib.util
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "make_cylinder_compression.py")
    spec = importlib.util.spec_from_file_location("make_cylinder_compression", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    monkeypatch.setattr(mod, "HERE", str(tmp_path))
    monkeypatch.setattr(mod, "STEPS", 10)
    monkeypatch.setattr(mod, "SHAPE", dict(n_theta=6, n_r=5, N=12, dr1=0.3))
    monkeypatch.setattr(mod, "STAIRCASE", dict(h=1.0, N=12))
    for stair in (False, True):
        res = mod.main(staircase=stair)
        name = "cylinder_staircase_compression.json" if stair else "cylinder_compression.json"
        stored = json.load(open(tmp_path / name))
        assert stored["residual_history"][-1][0] == 10
        C = [stored["eps"][k]["mean_compression"] for k in ("0.001", "0.0001", "1e-05")]
        assert C[0] <= C[1] <= C[2]
        key = "rank_map_x_by_y" if stair else "rank_map_theta_by_radius"
        assert all(key in v for v in res["eps"].values())
