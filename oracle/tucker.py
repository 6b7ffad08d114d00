"""Tucker-format reference operations (arXiv:1912.04582, Sections 4-5), numpy FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Each function restates one
operation of the paper from its mathematics; library primitives used as steps are
``numpy.linalg.svd`` and ``numpy.einsum``.

A Tucker tensor is a tuple ``(G, (U1, U2, U3))`` with core ``G`` of shape
(r1, r2, r3) and factors ``U_a`` of shape (N_a, r_a):
    A(i1,i2,i3) = sum_k G(k1,k2,k3) U1(i1,k1) U2(i2,k2) U3(i3,k3)   (Section 4, Tucker format).
"""
from __future__ import annotations

import math

import numpy as np


def full(t):
    """Expand a Tucker tensor to the full N1 x N2 x N3 array (Section 4)."""
    G, (U1, U2, U3) = t
    return np.einsum("abc,ia,jb,kc->ijk", G, U1, U2, U3, optimize=True)


def ranks(t):
    return tuple(int(s) for s in t[0].shape)


def unfold(A, mode):
    """Mode-a unfolding: rows indexed by i_a, columns by the other two indices."""
    return np.moveaxis(A, mode, 0).reshape(A.shape[mode], -1)


def truncation_rank(sigma, eps, cap, total_sq):
    """Smallest r with sum_{k>r} sigma_k^2 <= (eps^2/3) ||A||_F^2, then r <- min(r, cap),
    r >= 1 (the per-mode rule that makes ||A - B||_F <= eps ||A||_F for HOSVD, Section 4
    item 1)."""
    s2 = np.asarray(sigma, dtype=np.float64) ** 2
    tail = np.concatenate([np.cumsum(s2[::-1])[::-1][1:], [0.0]])  # tail[r-1] = sum_{k>r}
    thr = eps * eps / 3.0 * total_sq
    r = len(s2)
    for cand in range(1, len(s2) + 1):
        if tail[cand - 1] <= thr:
            r = cand
            break
    if cap is not None:
        r = min(r, int(cap))
    return max(1, r)


def hosvd(A, eps, cap=None):
    """Truncated higher-order SVD of a full tensor (Section 4 item 1, after De Lathauwer
    et al.): factors are the leading left singular vectors of each unfolding, the core is
    A x_1 U1^T x_2 U2^T x_3 U3^T.  Returns the Tucker tensor and the singular values."""
    total = float(np.sum(A * A))
    Us, sig = [], []
    for a in range(3):
        Ua, sa, _ = np.linalg.svd(unfold(A, a), full_matrices=False)
        r = truncation_rank(sa, eps, cap, total)
        Us.append(Ua[:, :r])
        sig.append(sa)
    G = np.einsum("ijk,ia,jb,kc->abc", A, Us[0], Us[1], Us[2], optimize=True)
    return (G, tuple(Us)), sig


def round_reference(t, eps, cap=None):
    """Reference rounding of a Tucker tensor: expand to full, then truncated HOSVD.
    (The fast route of Section 4 item 4 — QR of the factors, SVD of the small core — gives
    the same subspaces; this reference takes the definition directly.)"""
    return hosvd(full(t), eps, cap)[0]


def add(a, b):
    """Element-wise sum (Section 4 item 2, element_wise_sum): block-diagonal core,
    concatenated factors; ranks add."""
    Ga, Ua = a
    Gb, Ub = b
    ra, rb = Ga.shape, Gb.shape
    G = np.zeros(tuple(ra[k] + rb[k] for k in range(3)))
    G[:ra[0], :ra[1], :ra[2]] = Ga
    G[ra[0]:, ra[1]:, ra[2]:] = Gb
    U = tuple(np.concatenate([Ua[k], Ub[k]], axis=1) for k in range(3))
    return G, U


def scale(a, s):
    G, U = a
    return G * s, U


def hadamard(a, b):
    """Element-wise product (Section 4 item 3): Kronecker product of the cores and
    row-wise Kronecker products of the factors; with 1-based k = (kA-1) rB + kB."""
    Ga, Ua = a
    Gb, Ub = b
    G = np.kron(Ga, Gb)
    U = tuple(np.einsum("ia,ib->iab", Ua[k], Ub[k]).reshape(Ua[k].shape[0], -1)
              for k in range(3))
    return G, U


def convolve(t, w1, w2, w3):
    """Weighted convolution S = sum_i A(i) w1(i1) w2(i2) w3(i3) in O(n r^3)
    (Section 4 item 5): S_a = U_a^T w_a, then contract the core."""
    G, (U1, U2, U3) = t
    return float(np.einsum("abc,a,b,c->", G, U1.T @ w1, U2.T @ w2, U3.T @ w3))


def maxwellian_rank1(xi, n, u, T):
    """Rank-1 Tucker Maxwellian (Section 5): U_a(i) = n^{1/3} (2 pi R_g T)^{-1/2}
    exp(-(xi_{a,i} - u_a)^2 / (2 R_g T)), with R_g = 1/2."""
    Rg = 0.5
    U = tuple((n ** (1.0 / 3.0) / math.sqrt(2 * math.pi * Rg * T)
               * np.exp(-(xi[a] - u[a]) ** 2 / (2 * Rg * T)))[:, None] for a in range(3))
    return np.ones((1, 1, 1)), U


def lemma1(w1, w2, w3):
    """Lemma 1: w1(i1) + w2(i2) + w3(i3) in Tucker format with ranks 2: core zero except
    G(1,2,2) = G(2,1,2) = G(2,2,1) = 1 (1-based), factors [w_a, 1]."""
    G = np.zeros((2, 2, 2))
    G[0, 1, 1] = G[1, 0, 1] = G[1, 1, 0] = 1.0
    U = tuple(np.stack([w, np.ones_like(w)], axis=1) for w in (w1, w2, w3))
    return G, U


def shakhov_coefficient(n, T, Pr):
    """A in f^S = f^M [1 + A (q.v)(v^2/T - 5/2)] with R_g = 1/2, m = 1:
    (2/5)(1-Pr)/(p R_g T), p = n R_g T  =>  A = (8/5)(1-Pr)/(n T^2)."""
    Rg = 0.5
    p = n * Rg * T
    return 0.4 * (1.0 - Pr) / (p * Rg * T)


def shakhov_rank5(xi, a, Pr):
    """f^S built as in Proposition 1 (fshakhov_structure):
    f^M o (1 + (sum_a c_a v_a) o (b v^2 - 1)), with Lemma 1 for both rank-2 factors,
    Hadamard products and one sum — Tucker ranks 1 + 2*2 = 5."""
    n, u, T, q = a[0], a[1:4], a[4], a[5:8]
    A = shakhov_coefficient(n, T, Pr)
    v = [xi[k] - u[k] for k in range(3)]
    # (sum_a c_a v_a) o (b v^2 - 1) with c_a = A q_a * (5/2),  b = 2/(5T)
    c = [2.5 * A * q[k] for k in range(3)]
    b = 2.0 / (5.0 * T)
    lin = lemma1(c[0] * v[0], c[1] * v[1], c[2] * v[2])
    quad = lemma1(b * v[0] ** 2 - 1.0, b * v[1] ** 2, b * v[2] ** 2)
    one = (np.ones((1, 1, 1)), tuple(np.ones((len(xi[k]), 1)) for k in range(3)))
    bracket = add(one, hadamard(lin, quad))
    return hadamard(maxwellian_rank1(xi, n, u, T), bracket)


def shakhov_rank4(xi, a, Pr):
    """f^S with per-mode basis {1, v, v^2, v^3} x Maxwellian factor: the bracket
    1 + A (q.v)(v^2/T - 5/2) is a cubic polynomial in (v1, v2, v3), so a 4x4x4 core
    with 13 non-zeros represents it exactly (ranks 4 <= 5 of Proposition 1)."""
    n, u, T, q = a[0], a[1:4], a[4], a[5:8]
    A = shakhov_coefficient(n, T, Pr)
    G = np.zeros((4, 4, 4))
    G[0, 0, 0] = 1.0
    e = np.eye(3, dtype=int)
    for al in range(3):
        lin = tuple(e[al])                       # v_al
        G[lin] += -2.5 * A * q[al]
        for be in range(3):                      # v_al * v_be^2 / T
            idx = [int(e[al][k]) + 2 * int(e[be][k]) for k in range(3)]
            G[tuple(idx)] += A * q[al] / T
    _, M = maxwellian_rank1(xi, n, u, T)
    U = tuple(M[k][:, 0:1] * np.stack([(xi[k] - u[k]) ** p for p in range(4)], axis=1)
              for k in range(3))
    return G, U


def speed_bound(xi):
    """The coarse bound |xi_n| <= |xi| = sqrt(xi_1^2 + xi_2^2 + xi_3^2) of every face's
    normal speed (Section 5, xin-one-rank-approx), as a full N1 x N2 x N3 array."""
    return np.sqrt(xi[0][:, None, None] ** 2 + xi[1][None, :, None] ** 2
                   + xi[2][None, None, :] ** 2)


def diag_estimate_rank1(xi, a, b):
    """D_i^est of the implicit scheme (Section 5, diagonal_term with the bound of
    xin-one-rank-approx): the tensor a + b |xi| with a = 1/dt + nu_i and
    b = sum_l |A_l| / (2 |V_i|), approximated with ranks (1, 1, 1) by the truncated
    HOSVD.  The tensor is positive, so its leading singular vectors can be taken
    positive (Perron-Frobenius); returns three positive vectors d_a whose outer
    product is D^est (the core is folded into d_1)."""
    X = a + b * speed_bound(xi)
    (G, U), _ = hosvd(X, eps=0.0, cap=1)
    d = [U[k][:, 0] * np.sign(U[k][0, 0]) for k in range(3)]
    g = float(np.einsum("ijk,i,j,k->", X, d[0], d[1], d[2]))   # projection onto d1 d2 d3
    return d[0] * g, d[1], d[2]


def divide_rank1(t, d):
    """Element-wise division of a Tucker tensor by a rank-1 positive tensor
    d_1 (x) d_2 (x) d_3 (Section 5, one_rank_division): each factor row i of mode a is
    divided by d_a(i); the core and the ranks are unchanged, O(n r) work."""
    G, U = t
    return G, tuple(U[k] / np.asarray(d[k])[:, None] for k in range(3))


def compression(r, N):
    """C = (r1 r2 r3 + N (r1 + r2 + r3)) / N^3 (Section 7)."""
    r1, r2, r3 = r
    return (r1 * r2 * r3 + N * (r1 + r2 + r3)) / float(N) ** 3


def lusgs_step_tucker(o, dt, eps, cap=None, diag="rank1"):
    """One implicit step of Section 5 in the Tucker format's arithmetic, on the state held
    by the full-grid oracle ``o`` (a FullGridOracle), which it advances.

    The linear-system equation [I/dt - dR/df] (f^{n+1} - f^n) = R^n is solved by one
    LU-SGS pass over the cells in index order (the same sweeps as the full-grid oracle),
    with the Tucker format's two departures:
      * the division by the diagonal uses D_i^est, the rank-1 approximation of
        1/dt + nu_i + sum_l |A_l| |xi| / (2 |V_i|) (diagonal_term with the bound of
        xin-one-rank-approx), so it is exact in the Tucker format (one_rank_division);
        diag="exact" divides by the full-grid diagonal instead (a cross-check);
      * every sum of Tucker tensors is rounded to eps (and cap): the forward sweep's
        R_i - sum_{j<i} M_ij g_j, the backward sweep's g_i - D^-1 sum_{j>i} M_ij df_j and
        f^n + df.  eps = 0 keeps every sum exact.
    Tensors are held expanded; a rounding is the truncated HOSVD of the exact sum, which
    is what rounding a Tucker sum computes.  The off-diagonal blocks are the exact
    (xi.e)^- weights.  Returns the residual of the step (the oracle's definition)."""
    f = o.f()
    R = o.rhs()
    vol, fcell, fgeo = o.geometry()
    xi = o.nodes()
    m = o.macro()
    nc = f.shape[0]
    X = [xi[0][:, None, None], xi[1][None, :, None], xi[2][None, None, :]]

    def rnd(A):
        return full(hosvd(A, eps, cap)[0]) if eps > 0 else A

    nbrs = [[] for _ in range(nc)]           # (j, |A_l| / |V_i| * (xi.e_out)^-)
    area = np.zeros(nc)
    for jf in range(fcell.shape[0]):
        a, b = int(fcell[jf, 0]), int(fcell[jf, 1])
        e = fgeo[jf, 1:]
        xn = e[0] * X[0] + e[1] * X[1] + e[2] * X[2]
        area[a] += fgeo[jf, 0]
        if b >= 0:
            area[b] += fgeo[jf, 0]
            nbrs[a].append((b, fgeo[jf, 0] / vol[a] * np.minimum(xn, 0.0)))
            nbrs[b].append((a, fgeo[jf, 0] / vol[b] * np.minimum(-xn, 0.0)))
    if diag == "exact":
        D = o.lusgs_diag(dt)
    else:
        D = np.empty_like(f)
        for i in range(nc):
            nu = o.nu(m[i, 0], m[i, 4])
            d = diag_estimate_rank1(xi, 1.0 / dt + nu, area[i] / (2.0 * vol[i]))
            D[i] = np.einsum("i,j,k->ijk", *d)
    g = np.empty_like(f)
    for i in range(nc):                      # forward sweep
        A = R[i].copy()
        for j, M in nbrs[i]:
            if j < i:
                A -= M * g[j]
        g[i] = rnd(A) / D[i]
    df = np.empty_like(f)
    for i in range(nc - 1, -1, -1):          # backward sweep
        B = np.zeros_like(f[i])
        for j, M in nbrs[i]:
            if j > i:
                B += M * df[j]
        df[i] = rnd(g[i] - B / D[i])
    fn = np.stack([rnd(f[i] + df[i]) for i in range(nc)])
    o.init_f(fn)
    w = o.weight()
    x2 = X[0] ** 2 + X[1] ** 2 + X[2] ** 2

    def U(t):
        return np.array([t.sum(), (X[0] * t).sum(), (X[1] * t).sum(), (X[2] * t).sum(),
                         (x2 * t).sum()]) * w
    num = sum(vol[i] * np.sum((U(fn[i]) - U(f[i])) ** 2) for i in range(nc))
    den = sum(vol[i] * np.sum(U(f[i]) ** 2) for i in range(nc))
    return math.sqrt(num) / (dt * math.sqrt(den))
