"""Pins of the numpy Tucker-format reference (Sections 4-5) against exact identities.

The expansions of sums, Hadamard products and convolutions must equal the corresponding
operations on full tensors; the rank-1 Maxwellian, Lemma 1 and the low-rank Shakhov
function must equal their pointwise definitions (the Shakhov one against the C oracle's
full-grid f^S, which is pinned separately); HOSVD must respect its error bound.
"""
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle import tucker as tk

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_tucker(rng, N, r):
    G = rng.standard_normal(r)
    U = tuple(rng.standard_normal((N[a], r[a])) for a in range(3))
    return G, U


def test_sum_hadamard_convolution_identities():
    rng = np.random.default_rng(0)
    N = (5, 6, 7)
    a = _rand_tucker(rng, N, (2, 3, 2))
    b = _rand_tucker(rng, N, (3, 1, 2))
    A, B = tk.full(a), tk.full(b)
    s = tk.add(a, b)
    assert tk.ranks(s) == (5, 4, 4)
    assert np.max(np.abs(tk.full(s) - (A + B))) < 1e-13
    h = tk.hadamard(a, b)
    assert tk.ranks(h) == (6, 3, 4)
    assert np.max(np.abs(tk.full(h) - A * B)) < 1e-12
    w = [rng.standard_normal(n) for n in N]
    brute = sum(A[i, j, k] * w[0][i] * w[1][j] * w[2][k]
                for i in range(N[0]) for j in range(N[1]) for k in range(N[2]))
    assert abs(tk.convolve(a, *w) - brute) < 1e-12 * max(1.0, abs(brute))


def test_hadamard_index_convention_matches_paper():
    """k = (kA - 1) rB + kB (1-based): column k of U^C is U^A(:,kA) * U^B(:,kB)."""
    rng = np.random.default_rng(1)
    a = _rand_tucker(rng, (4, 4, 4), (2, 2, 2))
    b = _rand_tucker(rng, (4, 4, 4), (3, 3, 3))
    G, U = tk.hadamard(a, b)
    for kA in range(1, 3):
        for kB in range(1, 4):
            k = (kA - 1) * 3 + kB
            assert np.allclose(U[0][:, k - 1], a[1][0][:, kA - 1] * b[1][0][:, kB - 1])
    assert G[3 * 1 + 2, 0, 0] == a[0][1, 0, 0] * b[0][2, 0, 0]


def test_lemma1_core_is_the_printed_one():
    rows = [tuple(int(v) for v in ln.split()) for ln in open(os.path.join(GOLDEN, "lemma1_core.txt"))
            if ln.strip() and not ln.startswith("#")]
    rng = np.random.default_rng(2)
    w = [rng.standard_normal(n) for n in (4, 5, 6)]
    G, U = tk.lemma1(*w)
    G_ref = np.zeros((2, 2, 2))
    for k1, k2, k3, v in rows:
        G_ref[k1 - 1, k2 - 1, k3 - 1] = v
    assert np.array_equal(G, G_ref)
    for a in range(3):
        assert np.array_equal(U[a][:, 0], w[a]) and np.all(U[a][:, 1] == 1.0)
    exact = w[0][:, None, None] + w[1][None, :, None] + w[2][None, None, :]
    assert np.max(np.abs(tk.full((G, U)) - exact)) < 1e-15


def test_rank1_maxwellian_matches_pointwise_and_hosvd(oracle_lib):
    wl = W.specular_box(shape=(1, 1, 1), N=20, vmax=6.0)
    o = oracle_lib.FullGridOracle(wl)
    xi = o.nodes()
    n, u, T = 1.3, (0.4, -0.2, 0.7), 0.9
    F = o.maxwellian(n, u, T)
    t = tk.maxwellian_rank1(xi, n, u, T)
    assert np.max(np.abs(tk.full(t) - F)) < 1e-15 * np.max(F) * 10
    _, sig = tk.hosvd(F, 1e-14)
    for s in sig:
        assert s[1] / s[0] < 1e-14


@pytest.mark.parametrize("builder,max_rank", [(tk.shakhov_rank4, 4), (tk.shakhov_rank5, 5)])
def test_low_rank_shakhov_equals_full_grid_shakhov(oracle_lib, builder, max_rank):
    """Proposition 1: f^S is low-rank; both constructions expand to the oracle's
    pointwise f^S (Algorithm 2, line 10) and the numerical ranks are <= 4."""
    wl = W.specular_box(shape=(1, 1, 1), N=24, vmax=7.0)
    o = oracle_lib.FullGridOracle(wl)
    xi = o.nodes()
    a = np.array([1.2, 0.3, -0.5, 0.2, 1.4, 0.21, -0.13, 0.08])
    fs = o.shakhov_from_macro(a)
    t = builder(xi, a, wl.Pr)
    assert max(tk.ranks(t)) == max_rank
    assert np.max(np.abs(tk.full(t) - fs)) < 1e-14 * np.max(np.abs(fs)) * 10
    _, sig = tk.hosvd(fs, 1e-15)
    for s in sig:
        assert s[4] / s[0] < 1e-13                       # numerical ranks <= 4
        assert s[3] / s[0] > 1e-8                        # and the heat flux makes it 4
    bound = [ln.split() for ln in open(os.path.join(GOLDEN, "paper_figures.txt"))
             if ln.startswith("shakhov_rank_bound")][0]
    assert max_rank <= int(bound[1])


def test_hosvd_error_bound_and_truncation_rule():
    rng = np.random.default_rng(3)
    N = 12
    # tensor with decaying multilinear spectrum
    G = rng.standard_normal((N, N, N)) * np.exp(-0.9 * np.add.outer(np.add.outer(
        np.arange(N), np.arange(N)), np.arange(N)))
    Q = [np.linalg.qr(rng.standard_normal((N, N)))[0] for _ in range(3)]
    A = tk.full((G, tuple(Q)))
    nA = np.linalg.norm(A)
    for eps in (1e-2, 1e-4, 1e-6):
        t, sig = tk.hosvd(A, eps)
        assert np.linalg.norm(tk.full(t) - A) <= eps * nA * (1 + 1e-10)
        r = tk.ranks(t)
        # minimality of each mode rank under the per-mode rule
        for a in range(3):
            s2 = sig[a] ** 2
            if r[a] > 1:
                assert np.sum(s2[r[a] - 1:]) > eps * eps / 3 * nA * nA
    t, _ = tk.hosvd(A, 1e-12, cap=3)
    assert tk.ranks(t) == (3, 3, 3)
    z, _ = tk.hosvd(np.zeros((4, 4, 4)), 1e-5)
    assert tk.ranks(z) == (1, 1, 1)


def test_round_reference_recovers_low_rank_sum():
    """A sum of low-rank tensors whose true ranks are small rounds back to those ranks
    without loss (Section 4 item 4)."""
    rng = np.random.default_rng(4)
    a = _rand_tucker(rng, (10, 10, 10), (2, 2, 2))
    s = tk.add(a, tk.scale(a, 0.5))          # ranks 4, true ranks 2
    r = tk.round_reference(s, 1e-12)
    assert tk.ranks(r) == (2, 2, 2)
    assert np.max(np.abs(tk.full(r) - 1.5 * tk.full(a))) < 1e-12


def test_compression_ratio_formula():
    """C = (r1 r2 r3 + N (r1 + r2 + r3)) / N^3 (Section 7)."""
    assert tk.compression((1, 1, 1), 64) == (1 + 64 * 3) / 64 ** 3
    assert tk.compression((64, 64, 64), 64) == 1.0 + 3.0 / 64


def _rand_tucker(rng, N, r):
    G = rng.standard_normal(r)
    U = tuple(rng.standard_normal((N[k], r[k])) for k in range(3))
    return G, U


def test_rank1_division_is_elementwise_division():
    """one_rank_division (Section 5): dividing the factor rows equals dividing the
    expanded tensor element by element, for any ranks."""
    rng = np.random.default_rng(3)
    for N, r in (((7, 5, 6), (3, 2, 4)), ((12, 12, 12), (5, 5, 5)), ((4, 9, 3), (1, 6, 2))):
        t = _rand_tucker(rng, N, r)
        d = [rng.uniform(0.3, 2.0, N[k]) for k in range(3)]
        B = tk.full(tk.divide_rank1(t, d))
        ref = tk.full(t) / (d[0][:, None, None] * d[1][None, :, None] * d[2][None, None, :])
        assert tk.ranks(tk.divide_rank1(t, d)) == r
        assert np.max(np.abs(B - ref)) < 1e-13 * np.max(np.abs(ref))


def test_speed_bound_bounds_every_normal_speed():
    """xin-one-rank-approx: |xi . e| <= |xi| for every unit normal e (Cauchy-Schwarz),
    with equality on the axis planes' normals at nodes on that axis."""
    rng = np.random.default_rng(5)
    xi = [np.linspace(-4, 4, 8), np.linspace(-3, 5, 6), np.linspace(-6, 6, 10)]
    S = tk.speed_bound(xi)
    for _ in range(20):
        e = rng.standard_normal(3)
        e /= np.linalg.norm(e)
        xn = (e[0] * xi[0][:, None, None] + e[1] * xi[1][None, :, None]
              + e[2] * xi[2][None, None, :])
        assert np.all(np.abs(xn) <= S * (1 + 1e-15))
    brute = np.array([[[math.sqrt(a * a + b * b + c * c) for c in xi[2]] for b in xi[1]]
                      for a in xi[0]])
    assert np.max(np.abs(S - brute)) < 1e-14


def test_rank1_diag_estimate_positive_and_exact_for_constants():
    xi = [np.linspace(-5, 5, 12)] * 3
    d = tk.diag_estimate_rank1(xi, 3.0, 0.0)        # b = 0: the constant tensor, rank 1
    D = np.einsum("i,j,k->ijk", *d)
    assert np.max(np.abs(D - 3.0)) < 1e-12
    d = tk.diag_estimate_rank1(xi, 2.0, 1.5)
    assert all(np.all(v > 0) for v in d)
    D = np.einsum("i,j,k->ijk", *d)
    X = 2.0 + 1.5 * tk.speed_bound(xi)
    # best rank-1 approximation: its error is below the one of the constant fit
    # with the mean (another rank-1 tensor), and the residual is orthogonal to D
    err = np.linalg.norm(D - X)
    assert err < np.linalg.norm(X - X.mean())
    assert abs(np.sum((X - D) * D)) < 1e-10 * np.sum(D * D)
