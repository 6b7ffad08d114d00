"""Tucker-format CUDA path through the C ABI vs the FP64 full-grid oracle and the numpy
Tucker reference.

* Compression of given tensors (Section 4 item 1): the rounding error bound
  ||A - B|| <= eps ||A|| per cell, exact recovery of low-rank tensors.
* A Maxwellian initial state is rank 1 (Section 5).
* Time steps (Section 5): with a tight tolerance and a rank cap equal to N the Tucker
  step reproduces the full-grid oracle to round-off of the rounding; at the working
  tolerance the difference is O(eps) per step.
Tucker factors are unique only up to rotations, so expanded tensors and
macroparameters are compared, never raw factors.
"""
import numpy as np
import pytest

import workloads as W
from oracle import tucker as tk

pytestmark = pytest.mark.gpu

FP64 = 0
MIXED = 1


@pytest.fixture(scope="module")
def dvm():
    import paper_1912_04582_gb300 as P
    from paper_1912_04582_gb300 import _native
    _native.load()
    return P


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def macro_err(mg, mo, u_scale=1e-3):
    """Relative L2 errors of n and T; u relative to its own L2 norm or, where the flow is
    slower than u_scale (the problem's characteristic speed), to u_scale per cell; q
    relative to its own norm or, where it is smaller, to the thermal heat-flux scale
    p sqrt(T) = n T^1.5 / 2 per cell (q vanishes in equilibrium, so its own norm is no
    scale for the round-off of a truncated distribution)."""
    err = {"n": rel_l2(mg[:, 0], mo[:, 0]), "T": rel_l2(mg[:, 4], mo[:, 4])}
    un = max(np.linalg.norm(mo[:, 1:4]), u_scale * np.sqrt(mo.shape[0]))
    err["u"] = float(np.linalg.norm(mg[:, 1:4] - mo[:, 1:4]) / un)
    qs = np.linalg.norm(0.5 * mo[:, 0] * mo[:, 4] ** 1.5)
    qn = max(np.linalg.norm(mo[:, 5:8]), qs)
    err["q"] = float(np.linalg.norm(mg[:, 5:8] - mo[:, 5:8]) / qn)
    return err


def tucker_solver(dvm, wl, cap, tol, precision=FP64, init=True):
    return dvm.Solver(wl, format=1, precision=precision, rank_cap=cap, tol=tol, init=init)


def test_maxwellian_initial_state_is_rank_one(dvm, oracle_lib):
    wl = W.cavity(nside=3, N=12, seed=1)
    rng = np.random.default_rng(5)
    wl.n0 = rng.uniform(0.5, 1.5, wl.n_cell)
    wl.u0 = rng.uniform(-0.3, 0.3, (wl.n_cell, 3))
    wl.T0 = rng.uniform(0.7, 1.4, wl.n_cell)
    s = tucker_solver(dvm, wl, 6, 1e-6)
    assert np.all(dvm.dvm_get_ranks(s.h) == 1)
    o = oracle_lib.FullGridOracle(wl)
    assert rel_l2(s.f(), o.f()) < 1e-14
    for k, v in macro_err(s.moments(), o.macro()).items():
        assert v < 1e-12, (k, v)
    fb, _ = dvm.dvm_memory(s.h)
    assert fb == wl.n_cell * (1 + 3 * 12) * 8


@pytest.mark.parametrize("precision,eps,tol_rel", [(FP64, 1e-6, 1e-12), (MIXED, 1e-6, 1e-6)])
def test_compression_recovers_low_rank_tensors(dvm, oracle_lib, precision, eps, tol_rel):
    """Sum of two Maxwellians per cell: Tucker ranks exactly 2 (the mixed path forms its
    Gram matrices from exact FP32 products summed in double-FP32, so tolerances well below
    sqrt(FP32 round-off) are still resolved)."""
    wl = W.specular_box(shape=(2, 2, 1), N=16, vmax=5.0)
    o = oracle_lib.FullGridOracle(wl)
    rng = np.random.default_rng(3)
    f = np.stack([o.maxwellian(rng.uniform(0.5, 1), rng.uniform(-1, 1, 3), rng.uniform(0.6, 1.2))
                  + o.maxwellian(rng.uniform(0.2, 0.5), rng.uniform(-1, 1, 3), rng.uniform(0.6, 1.2))
                  for _ in range(wl.n_cell)])
    s = tucker_solver(dvm, wl, 8, eps, precision=precision, init=False)
    dvm.dvm_init_f(s.h, f)
    r = dvm.dvm_get_ranks(s.h)
    assert np.all(r == 2), r
    assert rel_l2(s.f(), f) < tol_rel


@pytest.mark.parametrize("precision,eps", [(FP64, 1e-2), (FP64, 1e-4), (FP64, 1e-6),
                                           (FP64, 1e-7), (MIXED, 1e-3), (MIXED, 1e-5)])
def test_rounding_respects_error_bound(dvm, oracle_lib, precision, eps):
    """Random decaying-spectrum tensors: ||A - round(A)|| <= eps ||A|| per cell (cap
    inactive), and ranks no larger than the reference HOSVD's (Section 4 items 1, 4)."""
    N = 14
    wl = W.specular_box(shape=(3, 1, 1), N=N, vmax=5.0)
    rng = np.random.default_rng(9)
    f = []
    for _ in range(wl.n_cell):
        G = rng.standard_normal((N, N, N)) * np.exp(-0.7 * np.add.outer(np.add.outer(
            np.arange(N), np.arange(N)), np.arange(N)))
        Q = [np.linalg.qr(rng.standard_normal((N, N)))[0] for _ in range(3)]
        f.append(np.abs(tk.full((G, tuple(Q)))) + 0.0)
    f = np.stack(f)
    s = tucker_solver(dvm, wl, N, eps, precision=precision, init=False)
    dvm.dvm_init_f(s.h, f)
    g = s.f()
    ranks = dvm.dvm_get_ranks(s.h)
    slack = 1e-8 if precision == FP64 else 1e-6   # FP32 storage of the working tensor
    for c in range(wl.n_cell):
        nf = np.linalg.norm(f[c])
        assert np.linalg.norm(g[c] - f[c]) <= eps * nf * (1 + 1e-8) + slack * nf
        ref, _ = tk.hosvd(f[c], eps)
        assert np.all(ranks[c] <= np.array(tk.ranks(ref)) + 2)


def test_step_without_truncation_matches_oracle(dvm, oracle_lib):
    """Cap = N and eps = 0 (no truncation): the Tucker step is the full-grid step
    (assembly + exact re-factorisation), so 20 steps agree with the FP64 oracle to
    round-off."""
    wl = W.sod_row(N=12, seed=2)
    s = tucker_solver(dvm, wl, 12, 0.0)
    o = oracle_lib.FullGridOracle(wl)
    assert abs(s.dt - o.dt()) <= 1e-14 * o.dt()
    s.step(20)
    o.step(20, o.dt())
    assert rel_l2(s.f(), o.f()) < 1e-9
    for k, v in macro_err(s.moments(), o.macro()).items():
        assert v < 1e-9, (k, v)


@pytest.mark.parametrize("precision,bound", [(FP64, 1e-4), (MIXED, 1e-4)])
def test_cavity_walls_lid_working_tolerance(dvm, oracle_lib, precision, bound):
    """Small cavity (diffuse walls, moving lid), eps = 1e-6, cap 12, 40 steps: f, n, T,
    u (relative to the lid speed where the flow is slower) and q within 1e-4 of the FP64
    full-grid oracle.  (eps = 1e-5 leaves ~1.5e-4 in u after 40 steps: the truncation error
    of each step accumulates.)"""
    wl = W.cavity(nside=4, N=16, seed=4)
    s = tucker_solver(dvm, wl, 12, 1e-6, precision=precision)
    o = oracle_lib.FullGridOracle(wl)
    s.step(40)
    o.step(40, o.dt())
    e = rel_l2(s.f(), o.f())
    me = macro_err(s.moments(), o.macro(), u_scale=0.2)
    print(f"cavity 4^3x16^3 eps=1e-6 cap 12 prec={precision}: f {e:.2e} {me} "
          f"ranks max {dvm.dvm_get_ranks(s.h).max()}")
    assert e < bound, e
    for k, v in me.items():
        assert v < bound, (k, v)


def test_non_axis_faces_use_exact_flux(dvm, oracle_lib):
    """Jittered interior faces: the Tucker assembly applies the exact upwind weight, so with
    no truncation it agrees with the full-grid oracle to round-off."""
    wl = W.closed_freestream_box(shape=(3, 2, 2), N=10, jitter=0.25, Kn=0.3,
                                 u=(0.4, -0.3, 0.2))
    rng = np.random.default_rng(1)
    wl.n0 = rng.uniform(0.6, 1.4, wl.n_cell)
    wl.T0 = rng.uniform(0.8, 1.3, wl.n_cell)
    s = tucker_solver(dvm, wl, 10, 0.0)
    o = oracle_lib.FullGridOracle(wl)
    s.step(8)
    o.step(8, o.dt())
    assert rel_l2(s.f(), o.f()) < 1e-9


def test_truncation_error_stays_within_tolerance_per_step(dvm, oracle_lib):
    """eps = 1e-6, cap = N: each rounding adds at most eps relative error, so after k
    steps the difference to the oracle is O(k eps)."""
    wl = W.sod_row(N=12, seed=2)
    s = tucker_solver(dvm, wl, 12, 1e-6)
    o = oracle_lib.FullGridOracle(wl)
    s.step(20)
    o.step(20, o.dt())
    assert rel_l2(s.f(), o.f()) < 20 * 1e-6
    assert np.max(dvm.dvm_get_ranks(s.h)) < 12


def test_tucker_restart_is_bitwise(dvm, tmp_path):
    wl = W.cavity(nside=3, N=12, seed=6)
    a = tucker_solver(dvm, wl, 6, 1e-5)
    a.step(4)
    p = str(tmp_path / "tk.bin")
    dvm.dvm_save(a.h, p)
    a.step(3)
    b = tucker_solver(dvm, wl, 6, 1e-5, init=False)
    dvm.dvm_load(b.h, p)
    b.step(3)
    assert np.array_equal(a.f(), b.f())
    assert np.array_equal(dvm.dvm_get_ranks(a.h), dvm.dvm_get_ranks(b.h))


def test_tucker_memory_is_compressed(dvm):
    wl = W.cavity(nside=4, N=16, seed=4)
    s = tucker_solver(dvm, wl, 8, 1e-5)
    s.step(10)
    fb, _ = dvm.dvm_memory(s.h)
    assert fb <= wl.n_cell * (8 ** 3 + 3 * 16 * 8) * 8
    assert fb < 0.6 * wl.n_cell * 16 ** 3 * 8


def test_graph_replay_equals_single_steps(dvm):
    """Multi-step calls replay a captured CUDA graph of two steps on a private stream;
    the state must equal single-step calls bitwise (and the autotuner's choice of grid
    must not change it)."""
    wl = W.cavity(nside=6, N=12, seed=3)
    a = tucker_solver(dvm, wl, 8, 1e-6, precision=MIXED)
    b = tucker_solver(dvm, wl, 8, 1e-6, precision=MIXED)
    for _ in range(7):
        a.step(1, residual=False)
    b.step(7, residual=False)
    assert np.array_equal(a.f(), b.f())
    grid, tune = dvm.dvm_get_launch_config(a.h)
    assert abs(grid) >= 1 and len(tune) == 5  # negative: the phase-major variant


@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_launch_variants_compute_the_same_values(dvm, precision):
    """The fused persistent kernel and the phase-major variant (assembly, then per mode
    Gram / eigen-solve / projection kernels) run the same per-cell arithmetic in the
    same order (first-mode Gram on the CUDA cores in both), so 12 steps of a cavity with
    walls, a moving lid and an inflow-free interior agree bit for bit; the launch
    configuration reports the variant."""
    from paper_1912_04582_gb300 import _native as NAT
    wl = W.cavity(nside=6, N=16, seed=4)
    out = {}
    for v in (NAT.DVM_VARIANT_FUSED, NAT.DVM_VARIANT_PHASED):
        s = dvm.Solver(wl, format=1, precision=precision, rank_cap=8, tol=1e-6, variant=v,
                       engine=NAT.DVM_ENGINE_CUDA_CORES)
        s.step(12)
        out[v] = (s.f(), s.moments(), dvm.dvm_get_ranks(s.h))
        grid, _ = dvm.dvm_get_launch_config(s.h)
        assert (grid < 0) == (v == NAT.DVM_VARIANT_PHASED)
        s.close()
    a, b = out[NAT.DVM_VARIANT_FUSED], out[NAT.DVM_VARIANT_PHASED]
    assert np.array_equal(a[2], b[2])
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[1], b[1])


def test_launch_variant_is_validated(dvm):
    wl = W.cavity(nside=2, N=8, seed=1)
    with pytest.raises(Exception):
        dvm.Solver(wl, format=1, precision=MIXED, rank_cap=4, tol=1e-5, variant=3)


def test_kernel_timing_covers_the_step(dvm):
    """Per-launch event timing: every kernel launch of a step is counted in its class
    (moments: the macroparameters and the moments kernel) and the class totals add up
    to (at most) the wall time of the steps."""
    import time
    from paper_1912_04582_gb300 import _native as NAT
    wl = W.cavity(nside=6, N=16, seed=4)
    for v, classes in ((NAT.DVM_VARIANT_PHASED,
                        {"tucker_contract": 1, "tucker_asm": 1, "tucker_gram_mode1": 1,
                         "tucker_gram_mode23": 2, "tucker_eig": 3, "tucker_proj": 3,
                         "moments": 2}),
                       (NAT.DVM_VARIANT_FUSED, {"tucker_fused_step": 1, "moments": 2})):
        s = dvm.Solver(wl, format=1, precision=MIXED, rank_cap=8, tol=1e-6, variant=v)
        s.step(2)
        dvm.dvm_set_kernel_timing(s.h, True)
        t0 = time.perf_counter()
        s.step(4, residual=False)
        t = dvm.dvm_get_kernel_timing(s.h)
        wall_ms = 1e3 * (time.perf_counter() - t0)
        dvm.dvm_set_kernel_timing(s.h, False)
        for name, (ms, n) in t.items():
            assert n == 4 * classes.get(name, 0), (name, n)
            assert (ms > 0) == (name in classes)
        assert sum(ms for ms, _ in t.values()) <= wall_ms
        s.close()


@pytest.mark.parametrize("N", [40, 64])
@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_velocity_grids_above_32_nodes(dvm, oracle_lib, N, precision):
    """Velocity grids with more than 32 nodes per axis take the 16 x 16-thread Gram
    tiles and larger eigen blocks: a small cavity, 8 steps at eps = 1e-6, cap 12,
    stays within 1e-4 of the FP64 oracle, in both launch variants, which agree bit for
    bit."""
    from paper_1912_04582_gb300 import _native as NAT
    wl = W.cavity(nside=2, N=N, seed=5)
    o = oracle_lib.FullGridOracle(wl)
    o.step(8, o.dt())
    fo, mo = o.f(), o.macro()
    out = {}
    for v in (NAT.DVM_VARIANT_FUSED, NAT.DVM_VARIANT_PHASED):
        s = dvm.Solver(wl, format=1, precision=precision, rank_cap=12, tol=1e-6, variant=v,
                       engine=NAT.DVM_ENGINE_CUDA_CORES)
        s.step(8)
        out[v] = (s.f(), s.moments(), dvm.dvm_get_ranks(s.h))
        s.close()
    fg, mg, rk = out[NAT.DVM_VARIANT_PHASED]
    assert rel_l2(fg, fo) < 1e-4
    for k, err in macro_err(mg, mo, u_scale=0.2).items():
        assert err < 1e-4, (k, err)
    assert rk.max() <= 12
    assert np.array_equal(out[NAT.DVM_VARIANT_FUSED][0], fg)
    assert np.array_equal(out[NAT.DVM_VARIANT_FUSED][2], rk)


def test_compression_at_64_nodes(dvm):
    """dvm_init_f on tensors of Tucker rank (3, 2, 4) at 64^3 nodes recovers them to the
    tolerance with those ranks (Section 4 item 1)."""
    rng = np.random.default_rng(11)
    wl = W.cavity(nside=2, N=64, seed=2)
    N = 64
    f = np.empty((wl.n_cell, N, N, N))
    for c in range(wl.n_cell):
        G = rng.uniform(0.5, 1.0, (3, 2, 4))  # positive: a physical state
        U = [rng.uniform(0.1, 1.0, (N, r)) for r in (3, 2, 4)]
        f[c] = tk.full((G, tuple(U)))
    s = dvm.Solver(wl, format=1, precision=FP64, rank_cap=8, tol=1e-6, init=False)
    dvm.dvm_init_f(s.h, f)
    g = s.f()
    ranks = dvm.dvm_get_ranks(s.h)
    s.close()
    assert rel_l2(g, f) < 1e-10
    assert np.all(ranks == np.array([3, 2, 4]))


def test_tucker_state_round_trip(dvm):
    """dvm_get_tucker / dvm_init_tucker: a state read from one context and given to a
    fresh one (same time step) reproduces it exactly, and both continue alike (the
    moments are re-taken about each cell's own velocity, so to round-off); ranks out of
    range are rejected."""
    wl = W.cavity(nside=4, N=16, seed=4)
    a = tucker_solver(dvm, wl, 8, 1e-6, precision=MIXED)
    a.step(6)
    ranks, core, fac = dvm.dvm_get_tucker(a.h, 8)
    b = dvm.Solver(wl, format=1, precision=MIXED, rank_cap=8, tol=1e-6,
                   dt=dvm.dvm_get_dt(a.h), init=False)
    dvm.dvm_init_tucker(b.h, ranks, core, fac)
    assert np.array_equal(a.f(), b.f())
    assert np.max(np.abs(a.moments() - b.moments())) < 1e-12
    a.step(3)
    b.step(3)
    assert rel_l2(b.f(), a.f()) < 1e-10
    bad = ranks.copy()
    bad[0, 1] = 9
    with pytest.raises(Exception):
        dvm.dvm_init_tucker(b.h, bad, core, fac)
    a.close()
    b.close()


def test_cavity_at_the_benchmark_size_against_oracle(dvm, oracle_lib):
    """The C2 cavity at full size (16^3 cells x 32^3 nodes) in the mixed-precision
    Tucker path at eps = 1e-6, cap 12, over 20 steps in the launch configuration the
    benchmark times (autotuned variant, graph replay), element by element against the
    FP64 oracle: within 1e-4 on f and on every macroparameter."""
    wl = W.cavity()
    o = oracle_lib.FullGridOracle(wl)
    o.step(20, o.dt())
    s = tucker_solver(dvm, wl, 12, 1e-6, precision=MIXED)
    s.step(20, residual=False)
    assert rel_l2(s.f(), o.f()) < 1e-4
    for k, err in macro_err(s.moments(), o.macro(), u_scale=0.2).items():
        assert err < 1e-4, (k, err)
    s.close()


@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_non_cubic_velocity_grid(dvm, oracle_lib, precision):
    """A 40 x 24 x 20 velocity grid (first mode above 32 nodes, the others below; every
    mode a different size) in both launch variants: within 1e-4 of the oracle after 8
    steps, and the variants agree bit for bit."""
    from paper_1912_04582_gb300 import _native as NAT
    wl = W.cavity(nside=3, N=40, seed=6)
    wl.N = (40, 24, 20)
    wl.lo, wl.hi = (-6.0, -5.5, -5.0), (6.0, 5.5, 5.0)
    o = oracle_lib.FullGridOracle(wl)
    o.step(8, o.dt())
    fo, mo = o.f(), o.macro()
    out = {}
    for v in (NAT.DVM_VARIANT_FUSED, NAT.DVM_VARIANT_PHASED):
        s = dvm.Solver(wl, format=1, precision=precision, rank_cap=12, tol=1e-6, variant=v,
                       engine=NAT.DVM_ENGINE_CUDA_CORES)
        s.step(8)
        out[v] = (s.f(), s.moments(), dvm.dvm_get_ranks(s.h))
        s.close()
    fg, mg, rk = out[NAT.DVM_VARIANT_PHASED]
    assert rel_l2(fg, fo) < 1e-4
    for k, err in macro_err(mg, mo, u_scale=0.2).items():
        assert err < 1e-4, (k, err)
    assert np.array_equal(out[NAT.DVM_VARIANT_FUSED][0], fg)
    assert np.array_equal(out[NAT.DVM_VARIANT_FUSED][2], rk)


def test_chunked_step_equals_single_chunk(dvm):
    """The phase-major step over several chunks of cells (the last one ragged, every
    chunk split over two streams) gives bit for bit the single-chunk result."""
    from paper_1912_04582_gb300 import _native as NAT
    wl = W.cavity(nside=6, N=16, seed=8)
    out = []
    for chunk in (0, 50, 7):
        s = dvm.Solver(wl, format=1, precision=MIXED, rank_cap=8, tol=1e-6,
                       variant=NAT.DVM_VARIANT_PHASED, max_chunk=chunk)
        s.step(6)
        out.append((s.f(), s.moments(), dvm.dvm_get_ranks(s.h)))
        s.close()
    for f, m, r in out[1:]:
        assert np.array_equal(r, out[0][2])
        assert np.array_equal(f, out[0][0])
        assert np.array_equal(m, out[0][1])


@pytest.mark.parametrize("nside,N", [(4, 32), (3, 48)])
def test_auto_engine_matches_cuda_core_engine(dvm, oracle_lib, nside, N):
    """The phase-major mixed path with engine AUTO (first-mode Gram matrices on the tensor
    cores by exact integer split, assembly as one GEMM per cell) and with the CUDA-core
    engine (double-FP32 Gram matrices, term-by-term assembly): both within 1e-4 of the
    oracle after 10 steps and close to each other.  The assemblies differ by FP32
    rounding of the K-term sums and the Gram matrices by rounding far below the
    truncation threshold, so the chosen ranks agree in all but borderline cells, where
    they differ by one; such a cell moves by at most tol = 1e-6 of its norm per step,
    which over 10 steps on a few percent of the cells bounds the gap by a few 1e-6."""
    from paper_1912_04582_gb300 import _native as NAT
    wl = W.cavity(nside=nside, N=N, seed=9)
    o = oracle_lib.FullGridOracle(wl)
    o.step(10, o.dt())
    fo, mo = o.f(), o.macro()
    out = {}
    for eng in (NAT.DVM_ENGINE_AUTO, NAT.DVM_ENGINE_CUDA_CORES):
        s = dvm.Solver(wl, format=1, precision=MIXED, rank_cap=12, tol=1e-6,
                       variant=NAT.DVM_VARIANT_PHASED, engine=eng)
        s.step(10)
        out[eng] = (s.f(), s.moments(), dvm.dvm_get_ranks(s.h))
        s.close()
    for eng, (fg, mg, _) in out.items():
        assert rel_l2(fg, fo) < 1e-4, eng
        for k, err in macro_err(mg, mo, u_scale=0.2).items():
            assert err < 1e-4, (eng, k, err)
    a, b = out[NAT.DVM_ENGINE_AUTO], out[NAT.DVM_ENGINE_CUDA_CORES]
    assert rel_l2(a[0], b[0]) < 5e-6
    assert np.abs(a[2] - b[2]).max() <= 1 and np.mean(a[2] == b[2]) > 0.95


def _engines_agree(dvm, oracle_lib, wl, steps, cap, tol, f0=None, close=1e-5):
    """Run the phase-major mixed step with both engines from the same start (Maxwellian,
    or the tensors f0 compressed at tolerance tol; the oracle then starts from that
    compressed state, so that only the steps are compared): each within 1e-4 of the
    oracle, and within `close` of each other (FP32 rounding of the assembly sums,
    rounding of the Gram matrices)."""
    from paper_1912_04582_gb300 import _native as NAT
    out, start = {}, None
    for eng in (NAT.DVM_ENGINE_AUTO, NAT.DVM_ENGINE_CUDA_CORES):
        s = dvm.Solver(wl, format=1, precision=MIXED, rank_cap=cap, tol=tol,
                       variant=NAT.DVM_VARIANT_PHASED, engine=eng, init=f0 is None)
        if f0 is not None:
            dvm.dvm_init_f(s.h, f0)
            if start is None:
                start = s.f()
            assert np.array_equal(s.f(), start)  # the compression does not depend on it
        s.step(steps)
        out[eng] = (s.f(), s.moments(), dvm.dvm_get_ranks(s.h))
        s.close()
    o = oracle_lib.FullGridOracle(wl)
    if start is not None:
        o.init_f(start)
    o.step(steps, o.dt())
    fo, mo = o.f(), o.macro()
    errs = {eng: dict(f=rel_l2(fg, fo), **macro_err(mg, mo, u_scale=0.1))
            for eng, (fg, mg, _) in out.items()}
    a, b = out[NAT.DVM_ENGINE_AUTO][0], out[NAT.DVM_ENGINE_CUDA_CORES][0]
    gap = rel_l2(a, b)
    for eng, e in errs.items():
        for k, err in e.items():
            assert err < 1e-4, (eng, k, errs, gap)
    assert gap < close, (gap, errs)
    return out


@pytest.mark.parametrize("case", ["sod", "specular", "freestream"])
def test_gemm_form_assembly_face_kinds(dvm, oracle_lib, case):
    """The assembly as one GEMM per cell of its rank-one terms on the face kinds the
    cavity does not have: symmetry faces mirroring the second / third index (the row's
    side faces) and zero-gradient ends (Sod row), symmetry on every side including the
    first index (specular box), free-stream ghosts (closed box)."""
    if case == "sod":
        wl = W.sod_row(N=16, vmax=5.0, Kn=0.3)
    elif case == "specular":
        wl = W.specular_box(shape=(3, 2, 2), N=16, vmax=5.0)
    else:
        wl = W.closed_freestream_box(shape=(3, 2, 2), N=16, jitter=0.0, Kn=0.5)
        rng = np.random.default_rng(2)
        wl.T0 = rng.uniform(0.8, 1.2, wl.n_cell)
    _engines_agree(dvm, oracle_lib, wl, steps=6, cap=8, tol=1e-7)


def test_gemm_form_assembly_many_terms(dvm, oracle_lib):
    """Cells with many rank-one terms: a start of 1..10 Maxwellians per cell and rank cap
    N = 16 (the cap never truncates), so ranks up to 16 and up to 4 + 8 r terms a cell,
    the column factors staged in several chunks of 32 terms."""
    wl = W.cavity(nside=4, N=16, seed=6)
    o = oracle_lib.FullGridOracle(wl)
    rng = np.random.default_rng(8)
    f0 = []
    for c in range(wl.n_cell):
        r = int(rng.integers(1, 11))
        f0.append(sum(o.maxwellian(rng.uniform(0.3, 1.0) / r, rng.uniform(-0.4, 0.4, 3),
                                   rng.uniform(0.7, 1.3)) for _ in range(r)))
    f0 = np.stack(f0)
    out = _engines_agree(dvm, oracle_lib, wl, steps=4, cap=16, tol=1e-6, f0=f0)
    from paper_1912_04582_gb300 import _native as NAT
    assert out[NAT.DVM_ENGINE_AUTO][2][:, 0].max() >= 8


@pytest.mark.parametrize("N", [(12, 10, 9), (20, 14, 11), (40, 24, 20), (64, 16, 12),
                               (20, 60, 36), (24, 64, 40)])
def test_gemm_form_assembly_grid_shapes(dvm, oracle_lib, N):
    """Engine AUTO on velocity grids whose first mode pads to 16, 32, 48 and 64 rows
    (register tiles of 4, 8, 12, 16 rows a thread), with N2 N3 not a multiple of four
    (scalar stores, a ragged last tile of columns) or spanning two tiles; and on both sides
    of the second/third-mode Gram's half-size launch (a 60-node second mode: 120 output
    blocks on 128 threads; a 64-node second mode: 136 blocks, the full-size launch)."""
    wl = W.cavity(nside=3, N=max(N), seed=6)
    wl.N = N
    wl.lo = tuple(-5.0 - 0.02 * n for n in N)
    wl.hi = tuple(5.0 + 0.02 * n for n in N)
    _engines_agree(dvm, oracle_lib, wl, steps=6, cap=min(N) if min(N) < 12 else 12, tol=1e-6)


def test_contexts_of_different_sizes_in_one_process(dvm):
    """The kernels' shared-memory opt-in is one setting per kernel function for the whole
    process: a context with a small velocity grid created after a large one must not
    lower what a later medium one needs (64, then 16, then 40 nodes; mixed precision,
    phase-major)."""
    from paper_1912_04582_gb300 import _native as NAT
    for N in (64, 16, 40, 24, 48):
        wl = W.cavity(nside=2, N=N, seed=1)
        s = dvm.Solver(wl, format=1, precision=MIXED, rank_cap=8, tol=1e-6,
                       variant=NAT.DVM_VARIANT_PHASED)
        assert np.isfinite(s.step(3))
        s.close()
