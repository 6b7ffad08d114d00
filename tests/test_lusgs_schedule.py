"""Host logic of the implicit LU-SGS step (no GPU): the wavefront schedule of its
sweeps (dvm_lusgs_wavefronts) and the option checks of dvm_create.

The schedule must reproduce the sequential sweep of the linear-system equation
(Section 3): every neighbour that comes before a cell in the sweep lies in an earlier
wavefront, and each wavefront is as early as that allows (its number is the longest
chain of such neighbours), checked against a brute-force recursion."""
import numpy as np
import pytest

import workloads as W


@pytest.fixture(scope="module")
def api():
    from paper_1912_04582_gb300 import build
    build.build()
    from paper_1912_04582_gb300 import api as A
    return A


def _lattice_nb(shape):
    nx, ny, nz = shape
    idx = np.arange(nx * ny * nz).reshape(shape)
    nb = -np.ones((nx * ny * nz, 6), dtype=np.int32)
    for i in range(nx):
        for j in range(ny):
            for k in range(nz):
                c = idx[i, j, k]
                for l, (di, dj, dk) in enumerate([(-1, 0, 0), (1, 0, 0), (0, -1, 0),
                                                  (0, 1, 0), (0, 0, -1), (0, 0, 1)]):
                    a, b, d = i + di, j + dj, k + dk
                    if 0 <= a < nx and 0 <= b < ny and 0 <= d < nz:
                        nb[c, l] = idx[a, b, d]
    return nb


def _random_nb(n, seed):
    """A random symmetric neighbour table with at most 6 neighbours per cell."""
    rng = np.random.default_rng(seed)
    nb = -np.ones((n, 6), dtype=np.int32)
    deg = np.zeros(n, dtype=int)
    for _ in range(3 * n):
        a, b = rng.integers(0, n, 2)
        if a == b or deg[a] == 6 or deg[b] == 6 or b in nb[a]:
            continue
        nb[a, deg[a]] = b
        nb[b, deg[b]] = a
        deg[a] += 1
        deg[b] += 1
    for c in range(n):                     # scatter the -1 slots like boundary faces
        nb[c] = nb[c, rng.permutation(6)]
    return nb


def _brute_waves(nb, forward):
    n = nb.shape[0]
    wave = np.zeros(n, dtype=int)
    seq = range(n) if forward else range(n - 1, -1, -1)
    for i in seq:
        prev = [j for j in nb[i] if j >= 0 and (j < i if forward else j > i)]
        wave[i] = 1 + max(wave[j] for j in prev) if prev else 0
    return wave


def _check_schedule(api, nb, forward):
    order, off = api.dvm_lusgs_wavefronts(nb, forward)
    n = nb.shape[0]
    assert np.array_equal(np.sort(order), np.arange(n))
    assert off[0] == 0 and off[-1] == n and np.all(np.diff(off) > 0)
    wave = np.empty(n, dtype=int)
    for w in range(len(off) - 1):
        cells = order[off[w]:off[w + 1]]
        assert np.all(np.diff(cells) > 0)          # increasing index within a wavefront
        wave[cells] = w
    assert np.array_equal(wave, _brute_waves(nb, forward))
    for i in range(n):                            # earlier neighbours in earlier wavefronts
        for j in nb[i]:
            if j >= 0 and (j < i if forward else j > i):
                assert wave[j] < wave[i]
    return len(off) - 1


@pytest.mark.parametrize("shape", [(4, 3, 2), (6, 1, 1), (5, 5, 5)])
def test_lexicographic_lattice_has_diagonal_wavefronts(api, shape):
    nb = _lattice_nb(shape)
    for forward in (True, False):
        nw = _check_schedule(api, nb, forward)
        assert nw == sum(shape) - 2           # the planes i + j + k = const


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_graphs_match_brute_force(api, seed):
    nb = _random_nb(200, seed)
    for forward in (True, False):
        _check_schedule(api, nb, forward)


def test_shuffled_mesh_numbering(api):
    """A shuffled cell numbering (as in the obstacle and Sod meshes) gives few, wide
    wavefronts; the schedule is still exact."""
    nb = _lattice_nb((6, 6, 6))
    perm = np.random.default_rng(4).permutation(nb.shape[0])
    inv = np.argsort(perm)
    nbp = np.where(nb[perm] >= 0, inv[np.maximum(nb[perm], 0)], -1).astype(np.int32)
    for forward in (True, False):
        nw = _check_schedule(api, nbp, forward)
        assert nw < 16


def test_empty_and_invalid_tables(api):
    order, off = api.dvm_lusgs_wavefronts(np.zeros((0, 6), dtype=np.int32))
    assert order.size == 0 and list(off) == [0]
    bad = -np.ones((3, 6), dtype=np.int32)
    bad[1, 2] = 3
    from paper_1912_04582_gb300 import _native
    with pytest.raises(_native.DvmError) as e:
        api.dvm_lusgs_wavefronts(bad)
    assert e.value.code == _native.DVM_ERR_INVALID_ARG


def test_create_rejects_lusgs_on_tucker_and_unknown_schemes(api):
    from paper_1912_04582_gb300 import _native
    wl = W.sod_row(N=8)
    args = (wl.xyz, wl.hex8, wl.bface, wl.bgroup, wl.N, wl.lo, wl.hi, wl.Pr, wl.omega, wl.Kn)
    with pytest.raises(_native.DvmError) as e:
        api.dvm_create(*args, format=_native.DVM_FORMAT_TUCKER, scheme=_native.DVM_SCHEME_LUSGS)
    assert e.value.code == _native.DVM_ERR_UNSUPPORTED
    with pytest.raises(_native.DvmError) as e:
        api.dvm_create(*args, scheme=7)
    assert e.value.code == _native.DVM_ERR_INVALID_ARG


def test_serving_estimate_counts_the_implicit_buffers(api):
    """Admission by memory: an implicit full-grid request also holds 1/D at every node
    (a third N^3 array per cell) besides the two state copies."""
    from paper_1912_04582_gb300 import _native
    wl = W.cavity(nside=4, N=12)
    e0 = api.dvm_estimate_memory(wl)
    e1 = api.dvm_estimate_memory(wl, scheme=_native.DVM_SCHEME_LUSGS)
    nn = wl.n_cell * int(np.prod(wl.N))
    assert e1 - e0 >= 8 * nn
    assert e0 >= 16 * nn
