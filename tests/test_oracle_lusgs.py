"""Pins of the oracle's implicit LU-SGS step (Section 3: linear-system and
diagonal_term equations) against what the mathematics fixes.

* The blocks the sweeps use are the Jacobian of the explicit right-hand side R^n:
  with collisions off and fixed ghosts R is affine in f, so unit perturbations of one
  cell give the Jacobian exactly; the LU-SGS increment must then satisfy the
  symmetric Gauss-Seidel factorisation (D + L) D^{-1} (D + U) df = R built from that
  differenced Jacobian.
* The diagonal adds the collision frequency of the cell (closed form from n and T).
* On a 1D row ordered along x, every velocity node's system is triangular, so one
  LU-SGS pass is the exact backward-Euler upwind step: compared with numpy's dense
  solve of the textbook implicit upwind matrix.
* dt -> 0 recovers the explicit step; a steady state stays steady at any dt; large
  steps reach a steady state in fewer steps than the explicit scheme.
"""
import math

import numpy as np
import pytest

import workloads as W


def _random_state(o, wl, seed):
    rng = np.random.default_rng(seed)
    f = o.f()
    f = f * rng.uniform(0.5, 1.5, f.shape)
    o.init_f(f)
    return f


def _jacobian_blocks(o, wl, f):
    """Per velocity node k, the nc x nc matrix J_k = dR_i/df_j (exact for affine R)."""
    nc = wl.n_cell
    R0 = o.rhs()
    J = np.empty((nc, nc) + R0.shape[1:])
    for j in range(nc):
        g = f.copy()
        g[j] += 1.0
        o.init_f(g)
        J[:, j] = o.rhs() - R0
    o.init_f(f)
    return R0, J


def test_lusgs_blocks_are_the_jacobian_and_sweeps_factorise(oracle_lib):
    wl = W.closed_freestream_box(shape=(2, 2, 2), N=4, vmax=3.0, Kn=1e300, jitter=0.25, seed=5)
    o = oracle_lib.FullGridOracle(wl)
    f = _random_state(o, wl, 1)
    R, J = _jacobian_blocks(o, wl, f)
    dt = 0.07
    nc = wl.n_cell
    # diagonal_term: D_i = 1/dt + nu_i + sum_l |A_l| |xi.e_l| / (2 |V_i|) = 1/dt - J_ii
    D = o.lusgs_diag(dt)
    Jd = np.stack([J[i, i] for i in range(nc)])
    assert np.max(np.abs(D - (1.0 / dt - Jd))) < 1e-11 * np.max(D)
    o.step_lusgs(1, dt)
    df = o.f() - f
    A = -J.copy()
    for i in range(nc):
        A[i, i] += 1.0 / dt
    # per node: (D + L) D^{-1} (D + U) df = R with L / U the strict lower / upper parts
    Dg = np.stack([A[i, i] for i in range(nc)])
    y = Dg * df
    for i in range(nc):
        for j in range(i + 1, nc):
            y[i] += A[i, j] * df[j]
    z = y / Dg
    lhs = Dg * z
    for i in range(nc):
        for j in range(i):
            lhs[i] += A[i, j] * z[j]
    assert np.max(np.abs(lhs - R)) < 1e-12 * np.max(np.abs(R)), np.max(np.abs(lhs - R))
    # the coupling is real: some lower and upper blocks are non-zero
    low = sum(np.abs(A[i, j]).max() for i in range(nc) for j in range(i))
    up = sum(np.abs(A[i, j]).max() for i in range(nc) for j in range(i + 1, nc))
    assert low > 1.0 and up > 1.0


def test_lusgs_diagonal_adds_the_collision_frequency(oracle_lib):
    kw = dict(shape=(2, 2, 1), N=6, vmax=4.0, seed=3)
    wl = W.specular_box(Kn=0.2, **kw)
    o = oracle_lib.FullGridOracle(wl)
    wl_free = W.specular_box(Kn=1e300, **kw)
    o_free = oracle_lib.FullGridOracle(wl_free)
    dt = 0.05
    a = o.macro()
    nu = math.sqrt(math.pi) / (2.0 * 0.2) * a[:, 0] * a[:, 4] ** (1.0 - wl.omega)
    d = o.lusgs_diag(dt) - o_free.lusgs_diag(dt)
    assert np.max(np.abs(d - nu[:, None, None, None])) < 1e-12 * np.max(nu)


def _implicit_upwind_row(f, xs, h, dt):
    """Backward-Euler first-order upwind along x on an x-ordered row, zero-gradient
    ends and mirror-symmetric sides held at t^n, solved per node with a dense solve."""
    nc = f.shape[0]
    x1 = xs[0][:, None, None]
    gm = np.concatenate([f[:1], f[:-1]])
    gp = np.concatenate([f[1:], f[-1:]])
    R = -(np.maximum(x1, 0) * (f - gm) + np.minimum(x1, 0) * (gp - f)) / h
    diag = 1.0 / dt + (np.abs(xs[0])[:, None, None] + np.abs(xs[1])[None, :, None]
                       + np.abs(xs[2])[None, None, :]) / h
    out = np.empty_like(f)
    for i1, x in enumerate(xs[0]):
        A = np.zeros((nc, nc))
        for i in range(nc):
            if x > 0 and i > 0:
                A[i, i - 1] = -x / h
            if x < 0 and i < nc - 1:
                A[i, i + 1] = x / h
        for i2 in range(len(xs[1])):
            for i3 in range(len(xs[2])):
                Ak = A + np.eye(nc) * diag[i1, i2, i3]
                out[:, i1, i2, i3] = np.linalg.solve(Ak, R[:, i1, i2, i3])
    return f + out


@pytest.mark.parametrize("dt", [2e-3, 0.05, 10.0])
def test_lusgs_row_is_exact_implicit_upwind(oracle_lib, dt):
    wl = W.sod_row(N=8, ncell=12, Kn=1e12, seed=None)
    assert np.array_equal(wl.cell_ijk[:, 0], np.arange(12))
    o = oracle_lib.FullGridOracle(wl)
    f0 = o.f()
    exp = _implicit_upwind_row(f0, o.nodes(), 1.0 / 12, dt)
    o.step_lusgs(1, dt)
    got = o.f()
    assert np.max(np.abs(got - exp)) < 1e-13 * np.max(f0), np.max(np.abs(got - exp))


def test_lusgs_small_dt_is_the_explicit_step(oracle_lib):
    wl = W.cavity(nside=3, N=6, vmax=4.0, Kn=0.3, seed=2)
    errs = []
    for dt in (1e-3, 1e-4):
        o = oracle_lib.FullGridOracle(wl)
        f0 = o.f()
        o.step(2, o.dt())           # leave the initial equilibrium
        f1 = o.f()
        R = o.rhs()
        o.step_lusgs(1, dt)
        errs.append(np.max(np.abs((o.f() - f1) / dt - R)) / np.max(np.abs(R)))
        assert np.max(np.abs(f1 - f0)) > 0
    assert errs[0] < 0.05
    assert errs[1] < errs[0] / 8.0, errs        # first order in dt


def test_lusgs_keeps_a_steady_state_at_any_step(oracle_lib):
    wl = W.closed_freestream_box(shape=(3, 2, 2), N=8, jitter=0.3, Kn=1e12)
    o = oracle_lib.FullGridOracle(wl)
    f0 = o.f()
    o.step_lusgs(3, 1e3)
    assert np.max(np.abs(o.f() - f0)) < 1e-13 * np.max(f0)


def test_lusgs_reaches_steady_state_in_fewer_steps(oracle_lib):
    """Section 3: the implicit scheme is not bound by the explicit stability limit, so
    after the same number of steps the steady-state residual R^n is smaller."""
    wl = W.cavity(nside=4, N=6, vmax=4.0, Kn=0.5, lid=0.3, seed=None)
    oe = oracle_lib.FullGridOracle(wl)
    dt = oe.dt()
    oe.step(40, dt)
    oi = oracle_lib.FullGridOracle(wl)
    oi.step_lusgs(40, 20.0 * dt)
    r_e = np.sqrt(np.mean(oe.rhs() ** 2))
    r_i = np.sqrt(np.mean(oi.rhs() ** 2))
    assert r_i < 0.3 * r_e, (r_i, r_e)
    m = oi.macro()
    assert np.all(m[:, 0] > 0.0) and np.all(m[:, 4] > 0.0)


# ---------------------------------------------------------------------------
# The Tucker format's implicit step (Section 5): division by the rank-1 estimate
# D^est and rounding of every Tucker sum (oracle.tucker.lusgs_step_tucker).

def test_tucker_lusgs_machinery_equals_the_full_grid_step(oracle_lib):
    """With the exact diagonal and no rounding, the Tucker reference's sweeps are the
    full-grid LU-SGS step (two independent codings of the same sweeps)."""
    from oracle import tucker as tk
    wl = W.cavity(nside=3, N=6, vmax=4.0, Kn=0.3, seed=2)
    a = oracle_lib.FullGridOracle(wl)
    b = oracle_lib.FullGridOracle(wl)
    a.step(2, a.dt())
    b.step(2, b.dt())
    dt = 5.0 * a.dt()
    ra = a.step_lusgs(1, dt)
    rb = tk.lusgs_step_tucker(b, dt, 0.0, diag="exact")
    assert np.max(np.abs(a.f() - b.f())) < 1e-14 * np.max(np.abs(a.f()))
    assert abs(ra - rb) < 1e-12 * ra


def test_tucker_lusgs_small_dt_is_the_explicit_step(oracle_lib):
    """D^est = (1/dt) (1 + O(dt)): the rank-1 step is consistent with the explicit one."""
    from oracle import tucker as tk
    wl = W.cavity(nside=3, N=8, vmax=4.0, Kn=0.3, seed=2)
    errs = []
    for dt in (1e-3, 1e-4):
        o = oracle_lib.FullGridOracle(wl)
        o.step(3, o.dt())
        f1, R = o.f(), o.rhs()
        tk.lusgs_step_tucker(o, dt, 0.0)
        errs.append(np.max(np.abs((o.f() - f1) / dt - R)) / np.max(np.abs(R)))
    assert errs[0] < 0.05 and errs[1] < errs[0] / 8.0, errs


def test_tucker_lusgs_rounding_stays_within_eps(oracle_lib):
    """Three roundings per cell (forward sum, backward sum, f + df), each within eps of
    its operand (Section 4, HOSVD bound): the rounded step stays within a few eps of the
    exact one in every cell."""
    from oracle import tucker as tk
    wl = W.cavity(nside=3, N=8, vmax=4.0, Kn=0.3, seed=2)
    out = {}
    for eps in (0.0, 1e-4, 1e-6):
        o = oracle_lib.FullGridOracle(wl)
        o.step(3, o.dt())
        tk.lusgs_step_tucker(o, 5.0 * o.dt(), eps)
        out[eps] = o.f()
    for eps in (1e-4, 1e-6):
        d = np.sqrt(np.sum((out[eps] - out[0.0]) ** 2, axis=(1, 2, 3))
                    / np.sum(out[0.0] ** 2, axis=(1, 2, 3)))
        assert np.all(d <= 3.0 * eps), (eps, d.max())
        assert d.max() > 0.01 * eps           # the rounding really truncates


def test_tucker_lusgs_rank1_diagonal_still_converges_faster(oracle_lib):
    """Section 5: the rank-1 estimate of the diagonal is rough, yet the implicit step
    approaches the steady state faster than the explicit one (here at 20 x its step,
    rounding to eps = 1e-6)."""
    from oracle import tucker as tk
    wl = W.cavity(nside=4, N=6, vmax=4.0, Kn=0.5, lid=0.3, seed=None)
    oe = oracle_lib.FullGridOracle(wl)
    dt = oe.dt()
    oe.step(40, dt)
    oi = oracle_lib.FullGridOracle(wl)
    for _ in range(40):
        tk.lusgs_step_tucker(oi, 20.0 * dt, 1e-6)
    r_e = np.sqrt(np.mean(oe.rhs() ** 2))
    r_i = np.sqrt(np.mean(oi.rhs() ** 2))
    assert r_i < 0.5 * r_e, (r_i, r_e)
