"""Implicit full-grid step (DVM_SCHEME_LUSGS) vs the oracle's sequential LU-SGS step
(Section 3, linear-system and diagonal_term equations), element by element, through
the C ABI.

The GPU runs each sweep one wavefront at a time; the oracle visits the cells one by one
in index order.  Both compute the same values up to FP64 rounding order, so the bar is
the full-grid one: relative L2 <= 1e-12 on f and on every macroparameter."""
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


def _macro_err(mg, mo):
    un = max(np.linalg.norm(mo[:, 1:4]), 1e-3 * np.sqrt(mo.shape[0]))
    qn = max(np.linalg.norm(mo[:, 5:8]), 1e-6 * np.sqrt(mo.shape[0]))
    return {"n": rel_l2(mg[:, 0], mo[:, 0]), "T": rel_l2(mg[:, 4], mo[:, 4]),
            "u": float(np.linalg.norm(mg[:, 1:4] - mo[:, 1:4]) / un),
            "q": float(np.linalg.norm(mg[:, 5:8] - mo[:, 5:8]) / qn)}


def _pair(dvm, oracle_lib, wl, steps, dt_factor, f0=None):
    from paper_1912_04582_gb300 import _native
    o = oracle_lib.FullGridOracle(wl)
    if f0 is not None:
        o.init_f(f0)
    dt = dt_factor * o.dt()
    s = dvm.Solver(wl, dt=dt, scheme=_native.DVM_SCHEME_LUSGS, init=f0 is None)
    if f0 is not None:
        dvm.api.dvm_init_f(s.h, f0)
    assert s.dt == dt
    rg = s.step(steps)
    ro = o.step_lusgs(steps, dt)
    fg, fo = s.f(), o.f()
    assert np.all(np.isfinite(fg))
    e = rel_l2(fg, fo)
    assert e <= TOL, f"f rel L2 {e}"
    for k, v in _macro_err(s.moments(), o.macro()).items():
        assert v <= TOL, f"{k}: {v}"
    assert abs(rg - ro) <= 1e-10 * ro
    s.close()
    return fo


def test_sod_row_shuffled_numbering(dvm, oracle_lib):
    """16 cells, symmetry sides, zero-gradient ends, shuffled cell numbering (so the
    sweep order is not the geometric one), 10 steps at 10 x the explicit CFL step."""
    _pair(dvm, oracle_lib, W.sod_row(N=12, seed=0), 10, 10.0)


def test_cavity_walls_and_moving_lid(dvm, oracle_lib):
    """Lexicographic 4^3 cavity (10 wavefronts per sweep), diffuse walls and the lid."""
    _pair(dvm, oracle_lib, W.cavity(nside=4, N=12, seed=None), 8, 5.0)


def test_cavity_shuffled_ragged_grid(dvm, oracle_lib):
    """Shuffled 5^3 cavity on a non-cubic velocity grid (16 x 10 x 12)."""
    wl = W.cavity(nside=5, N=12, seed=3)
    wl.N = (16, 10, 12)
    _pair(dvm, oracle_lib, wl, 5, 4.0)


def test_jittered_mesh_generic_faces(dvm, oracle_lib):
    """Jittered interior vertices: faces off the coordinate planes take the per-node
    (xi.e)^+- weights; a perturbed free-stream state so that every block acts."""
    wl = W.closed_freestream_box(shape=(4, 3, 3), N=10, jitter=0.25, Kn=0.2, seed=11)
    o = oracle_lib.FullGridOracle(wl)
    f0 = o.f() * np.random.default_rng(2).uniform(0.8, 1.2, o.f().shape)
    _pair(dvm, oracle_lib, wl, 5, 8.0, f0=f0)


def test_specular_box_with_walls(dvm, oracle_lib):
    wl = W.specular_box(shape=(3, 2, 2), N=10, Kn=0.3, wall_group=1)
    _pair(dvm, oracle_lib, wl, 6, 6.0)


def test_cavity_at_the_benchmark_size(dvm, oracle_lib):
    """C2 as the benchmark times it: 16^3 cells x 32^3 nodes (46 wavefronts per sweep,
    256-thread rows), one step at 5 x the explicit step."""
    _pair(dvm, oracle_lib, W.cavity(), 1, 5.0)


def test_lusgs_converges_faster_than_explicit(dvm):
    """Section 3: at 20 x the explicit step the implicit solve gets closer to the
    steady state in the same number of steps (the steady-state residual R^n, read
    as the explicit step's residual on the final state, is smaller)."""
    from paper_1912_04582_gb300 import _native
    wl = W.cavity(nside=6, N=10, Kn=0.5, lid=0.3, seed=None)
    se = dvm.Solver(wl)
    dt = se.dt
    se.step(60)
    si = dvm.Solver(wl, dt=20.0 * dt, scheme=_native.DVM_SCHEME_LUSGS)
    si.step(60)
    fi = si.f()
    probe = dvm.Solver(wl, dt=dt, init=False)          # explicit residual of each state
    dvm.api.dvm_init_f(probe.h, fi)
    r_i = probe.step(1)
    dvm.api.dvm_init_f(probe.h, se.f())
    r_e = probe.step(1)
    assert r_i < 0.5 * r_e, (r_i, r_e)
    m = si.moments()
    assert np.all(m[:, 0] > 0) and np.all(m[:, 4] > 0)
    for s in (se, si, probe):
        s.close()
