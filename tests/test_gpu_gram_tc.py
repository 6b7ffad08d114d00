"""Tensor-core Gram matrices (dvm_gram_tc, the Gram step of the mixed-precision Tucker
rounding, Section 4 item 4) against two references computed here:

* the same integer split done in numpy (row exponent e_a with max |x_a| <= 2^e_a, five
  rounded 7-bit slices of x 2^(6 - e_a), every slice product but (4, 4) formed exactly in
  float64): the kernel must agree to FP64 rounding, which checks the tensor cores'
  exact integer accumulation and every layout, descriptor and tensor-memory mapping;
* the FP64 Gram matrix of the FP32 input itself: the split perturbs each element by at
  most 2^-35 of its row's largest magnitude.

Shapes span one to three MMA groups, ragged column chunks and the largest sums the
split allows (|slice| = 64 everywhere)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _split_gram(X):
    """Gram matrices of the sliced tensor, exactly as the kernel defines them."""
    ncell, n, K = X.shape
    X = X.astype(np.float32)
    out = np.empty((ncell, n, n))
    for c in range(ncell):
        m = np.max(np.abs(X[c]), axis=1)
        _, E = np.frexp(m.astype(np.float64))
        e = np.where(m > 0, E, 0).clip(-100, 100)
        y = X[c] * np.ldexp(np.float32(1.0), 6 - e)[:, None].astype(np.float32)
        S = []
        for _ in range(5):
            s = np.rint(y)
            S.append(s.astype(np.float64))
            y = ((y - s) * np.float32(128.0)).astype(np.float32)
        acc = np.zeros((n, n))
        for k in range(5):
            for l in range(5):
                if k + l <= 7:
                    acc += np.ldexp(S[k] @ S[l].T, -7 * (k + l))
        out[c] = acc * np.ldexp(1.0, (e[:, None] + e[None, :] - 12))
    return out


def _inputs(ncell, n, K, seed):
    rng = np.random.default_rng(seed)
    X = np.empty((ncell, n, K), dtype=np.float32)
    for c in range(ncell):
        j = np.arange(K)
        for a in range(n):
            # Gaussian profiles over many decades, random signs in some rows
            prof = np.exp(-((j - rng.uniform(0, K)) / rng.uniform(2, K)) ** 2)
            row = prof * 10.0 ** rng.uniform(-9, 1)
            if rng.random() < 0.3:
                row = row * rng.choice([-1.0, 1.0], size=K)
            X[c, a] = row
        if n > 2:
            X[c, 1] = 0.0                       # a zero row
    return X


@pytest.mark.parametrize("n,K", [(5, 64), (32, 1024), (40, 968), (48, 2304), (56, 192),
                                 (64, 4096)])
def test_gram_tc_matches_exact_split_and_fp64(n, K):
    import torch
    import paper_1912_04582_gb300 as P
    torch.cuda.set_device(0)
    ncell = 3
    X = _inputs(ncell, n, K, seed=n * 1000 + K)
    xd = torch.from_numpy(X).cuda()
    cd = torch.full((ncell, n, n), float("nan"), dtype=torch.float64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    P.dvm_gram_tc(xd.data_ptr(), ncell, n, K, cd.data_ptr(), st.data_ptr(),
                  torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    C = cd.cpu().numpy()
    ref = _split_gram(X)
    nrm = np.sqrt(np.einsum("caa->ca", np.einsum("caj,cbj->cab", X.astype(np.float64),
                                                 X.astype(np.float64))))
    scale = nrm[:, :, None] * nrm[:, None, :] + 1e-300
    assert np.all(np.isfinite(C))
    assert np.max(np.abs(C - ref) / scale) < 1e-14
    assert np.array_equal(C, np.transpose(C, (0, 2, 1)))      # exactly symmetric
    X64 = X.astype(np.float64)
    full = np.einsum("caj,cbj->cab", X64, X64)
    rowmax = np.max(np.abs(X64), axis=2)
    bound = 2.0 ** -34 * K * rowmax[:, :, None] * rowmax[:, None, :] + 1e-300
    assert np.all(np.abs(C - full) <= bound + 1e-13 * scale)


def test_gram_tc_extreme_slices():
    """x = (63.5/64) 2^e everywhere: the first slice is 64 and the second -64 at every
    element, so with 4096 columns the slice products sum to +-2^24, the largest sums
    the split allows (one cell all positive, one with mixed signs)."""
    import torch
    import paper_1912_04582_gb300 as P
    torch.cuda.set_device(0)
    n, K = 48, 4096
    X = np.full((2, n, K), np.float32(63.5 / 64.0), dtype=np.float32)
    X[1, ::2, ::3] *= -1
    xd = torch.from_numpy(X).cuda()
    cd = torch.zeros((2, n, n), dtype=torch.float64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    P.dvm_gram_tc(xd.data_ptr(), 2, n, K, cd.data_ptr(), st.data_ptr(),
                  torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    C = cd.cpu().numpy()
    ref = _split_gram(X)
    assert np.max(np.abs(C - ref)) <= 1e-15 * np.max(np.abs(ref))


def test_gram_tc_rejects_bad_shapes():
    import torch
    import paper_1912_04582_gb300 as P
    from paper_1912_04582_gb300 import _native as N
    torch.cuda.set_device(0)
    buf = torch.zeros(1024, dtype=torch.float32, device="cuda")
    for n, K in ((65, 64), (8, 12), (8, 8192)):
        with pytest.raises(N.DvmError):
            P.dvm_gram_tc(buf.data_ptr(), 1, n, K, buf.data_ptr(), buf.data_ptr())
