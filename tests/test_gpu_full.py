"""Full-grid FP64 CUDA path vs the FP64 CPU oracle, element by element, through the C ABI.

Tolerance (the FP64 path's bar): relative L2 over all (cell, node) <= 1e-12 on f, and the same on
each macroparameter (n, u, T, q; u and q normalised by max(|u|, 1e-3), max(|q|, 1e-6)
where they are ~0).
"""
import os

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def dvm():
    import paper_1912_04582_gb300 as P
    from paper_1912_04582_gb300 import _native
    _native.load()
    return P


def rel_l2(a, b):
    a = np.asarray(a, float).ravel()
    b = np.asarray(b, float).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def macro_err(mg, mo):
    err = {}
    err["n"] = rel_l2(mg[:, 0], mo[:, 0])
    err["T"] = rel_l2(mg[:, 4], mo[:, 4])
    un = max(np.linalg.norm(mo[:, 1:4]), 1e-3 * np.sqrt(mo.shape[0]))
    err["u"] = float(np.linalg.norm(mg[:, 1:4] - mo[:, 1:4]) / un)
    qn = max(np.linalg.norm(mo[:, 5:8]), 1e-6 * np.sqrt(mo.shape[0]))
    err["q"] = float(np.linalg.norm(mg[:, 5:8] - mo[:, 5:8]) / qn)
    return err


def run_pair(dvm, oracle_lib, wl, steps):
    s = dvm.Solver(wl)
    o = oracle_lib.FullGridOracle(wl)
    dt_o = o.dt()
    dt_g = s.dt
    assert abs(dt_g - dt_o) <= 1e-14 * dt_o
    rg = s.step(steps) if steps else 0.0
    ro = o.step(steps, dt_o) if steps else 0.0
    return s, o, rg, ro


def check_pair(s, o, rg, ro, tol=TOL):
    fg, fo = s.f(), o.f()
    assert np.all(np.isfinite(fg))
    e = rel_l2(fg, fo)
    assert e <= tol, f"f rel L2 {e}"
    me = macro_err(s.moments(), o.macro())
    for k, v in me.items():
        assert v <= tol, f"{k}: {v}"
    if ro > 0:
        assert abs(rg - ro) <= 1e-10 * ro
    return e, me


def test_sod_row_100_steps(dvm, oracle_lib):
    """Smallest workload: 16 cells x 12^3, symmetry sides, zero-gradient ends,
    shuffled numbering, 100 steps."""
    wl = W.sod_row()
    check_pair(*run_pair(dvm, oracle_lib, wl, 100))


def test_cavity_walls_and_moving_lid(dvm, oracle_lib):
    wl = W.cavity(nside=4, N=12, seed=3, steps=30)
    check_pair(*run_pair(dvm, oracle_lib, wl, 30))


def test_ragged_nonuniform_grid_and_generic_faces(dvm, oracle_lib):
    """Jittered closed box (non-axis interior faces), free-stream boundary, collisions on,
    a non-cubic velocity grid (N = 10 x 13 x 7, columns not a multiple of the block)."""
    wl = W.closed_freestream_box(shape=(3, 2, 2), N=12, jitter=0.25, Kn=0.3, u=(0.4, -0.3, 0.2))
    wl.N = (10, 13, 7)
    wl.lo = (-5.0, -4.5, -5.5)
    wl.hi = (5.5, 4.5, 5.0)
    rng = np.random.default_rng(0)
    wl.n0 = rng.uniform(0.6, 1.4, wl.n_cell)
    wl.T0 = rng.uniform(0.8, 1.3, wl.n_cell)
    check_pair(*run_pair(dvm, oracle_lib, wl, 12))


def test_specular_box_with_walls(dvm, oracle_lib):
    wl = W.specular_box(shape=(2, 2, 2), N=14, vmax=5.0, wall_group=1)
    check_pair(*run_pair(dvm, oracle_lib, wl, 15))


def test_obstacle_reduced_lattice(dvm, oracle_lib):
    """Mach-3 obstacle geometry (jittered interior, free stream outside, hot-wall cube),
    reduced to the 16x10x10 lattice (1,592 cells) and an 8^3 grid on [-8,8]."""
    wl = W.obstacle(lattice=(16, 10, 10), N=8, steps=4)
    check_pair(*run_pair(dvm, oracle_lib, wl, 4))


def test_geometry_matches_oracle(dvm, oracle_lib):
    wl = W.obstacle(lattice=(8, 5, 5), N=4)
    s = dvm.Solver(wl)
    o = oracle_lib.FullGridOracle(wl)
    vg, fg_cell, fg_geo = dvm.dvm_get_geometry(s.h)
    vo, fo_cell, fo_geo = o.geometry()
    assert np.max(np.abs(vg - vo)) <= 1e-15 * np.max(vo)

    def keyed(fc, fgeo):
        d = {}
        for j in range(fc.shape[0]):
            a, b = int(fc[j, 0]), int(fc[j, 1])
            vec = fgeo[j, 0] * fgeo[j, 1:]
            if b >= 0 and b < a:
                a, b, vec = b, a, -vec
            d.setdefault((a, b), []).append(vec)
        return d
    kg, ko = keyed(fg_cell, fg_geo), keyed(fo_cell, fo_geo)
    assert set(kg) == set(ko)
    for k in ko:
        if k[1] >= 0:
            assert np.max(np.abs(kg[k][0] - ko[k][0])) <= 1e-15


def test_zero_steps_and_single_cell(dvm, oracle_lib):
    wl = W.specular_box(shape=(1, 1, 1), N=6, vmax=4.0)
    s, o, rg, ro = run_pair(dvm, oracle_lib, wl, 0)
    check_pair(s, o, rg, ro)
    s.step(1)
    o.step(1, o.dt())
    check_pair(s, o, 0.0, 0.0)


def test_restart_is_bitwise(dvm, tmp_path):
    wl = W.cavity(nside=3, N=10, seed=1)
    a = dvm.Solver(wl)
    a.step(7)
    p = str(tmp_path / "ck.bin")
    dvm.dvm_save(a.h, p)
    a.step(5)
    b = dvm.Solver(wl, init=False)
    dvm.dvm_load(b.h, p)
    assert dvm.dvm_get_step_count(b.h) == 7
    b.step(5)
    assert np.array_equal(a.f(), b.f())
    assert np.array_equal(a.moments(), b.moments())


def test_errors_are_reported(dvm):
    from paper_1912_04582_gb300 import _native as N
    wl = W.sod_row(N=6)
    wl.lo = (-5.0, -4.0, -5.0)            # symmetry on y needs lo = -hi
    s = dvm.Solver(wl, init=False)
    with pytest.raises(N.DvmError) as ei:
        dvm.dvm_init_maxwellian(s.h, wl.n0, wl.u0, wl.T0)
    assert ei.value.code == N.DVM_ERR_UNSUPPORTED
    wl = W.sod_row(N=6)
    wl.bcs = wl.bcs[:1]                    # group 1 left without a condition
    s = dvm.Solver(wl, init=False)
    with pytest.raises(N.DvmError) as ei:
        dvm.dvm_init_maxwellian(s.h, wl.n0, wl.u0, wl.T0)
    assert ei.value.code == N.DVM_ERR_STATE
    wl = W.sod_row(N=6)
    wl.bface = wl.bface[1:]
    wl.bgroup = wl.bgroup[1:]
    with pytest.raises(N.DvmError) as ei:
        dvm.Solver(wl)
    assert ei.value.code == N.DVM_ERR_INVALID_ARG
    s = dvm.Solver(W.sod_row(N=6), init=False)
    with pytest.raises(N.DvmError) as ei:
        s.step(1)
    assert ei.value.code == N.DVM_ERR_STATE


def test_nonphysical_state_is_reported(dvm):
    from paper_1912_04582_gb300 import _native as N
    wl = W.specular_box(shape=(1, 1, 1), N=6, vmax=4.0)
    s = dvm.Solver(wl, init=False)
    f = -np.ones((1, 6, 6, 6))
    with pytest.raises(N.DvmError) as ei:
        dvm.dvm_init_f(s.h, f)
    assert ei.value.code == N.DVM_ERR_NONPHYSICAL


@pytest.mark.slow
def test_cavity_full_size_three_steps(dvm, oracle_lib):
    """The benchmark workload at full size (16^3 cells x 32^3 nodes, the launch
    configuration the benchmark times): every cell and node after 3 steps."""
    wl = W.cavity()
    check_pair(*run_pair(dvm, oracle_lib, wl, 3))


@pytest.mark.slow
def test_c3_velocity_grid_against_oracle(dvm, oracle_lib):
    """The full-grid FP64 path is the same-run reference of the benchmark's Tucker error
    on the 32^3-cell x 48^3 cavity; here it is checked against the oracle with that
    velocity grid on 16^3 cells (every cell and node after 3 steps)."""
    wl = W.cavity(nside=16, N=48)
    check_pair(*run_pair(dvm, oracle_lib, wl, 3))
