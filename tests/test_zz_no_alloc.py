"""dvm_full_macro_noalloc: moments of device-resident tensors with no device allocation.

This entry point serves callers that cannot allocate device memory where they need the
moments (their memory is owned by their own pool allocator, or a cudaMalloc's implicit
synchronisation would stall work they have queued).  It must give the same
macroparameters as the allocating route — dvm_init_f + dvm_moments on a context — and
as the FP64 oracle on two calls in a row, since every call reuses the same fixed scratch array inside the
library.  The file sorts last so that a stop-at-first-failure run has done all other
tests first; it builds everything it needs, so it also passes alone.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _macro_err(mg, mo):
    err = {"n": np.linalg.norm(mg[:, 0] - mo[:, 0]) / np.linalg.norm(mo[:, 0]),
           "T": np.linalg.norm(mg[:, 4] - mo[:, 4]) / np.linalg.norm(mo[:, 4])}
    un = max(np.linalg.norm(mo[:, 1:4]), 1e-3 * np.sqrt(mo.shape[0]))
    err["u"] = np.linalg.norm(mg[:, 1:4] - mo[:, 1:4]) / un
    qn = max(np.linalg.norm(mo[:, 5:8]), 1e-6 * np.sqrt(mo.shape[0]))
    err["q"] = np.linalg.norm(mg[:, 5:8] - mo[:, 5:8]) / qn
    return err


def _oracle_moments(wl, f):
    import oracle
    o = oracle.FullGridOracle(wl, init=False)
    o.init_f(f)
    return o.macro()


def _reference_moments(P, wl, f):
    s = P.Solver(wl, init=False)
    P.dvm_init_f(s.h, f)
    m = s.moments()
    s.close()
    return m


def test_noalloc_macro_matches_allocating_route_twice():
    import torch
    import paper_1912_04582_gb300 as P

    torch.cuda.set_device(0)
    wl = W.cavity(nside=4, N=12, seed=2)
    run = P.Solver(wl)
    run.step(4)
    f1 = run.f()
    run.step(6)
    f2 = run.f()
    run.close()
    stream = torch.cuda.current_stream()
    for f in (f1, f2):                      # two calls in a row share the scratch array
        ref = _reference_moments(P, wl, f)
        fd = torch.from_numpy(np.ascontiguousarray(f)).cuda()
        out = torch.full((wl.n_cell, 8), float("nan"), dtype=torch.float64, device="cuda")
        P.dvm_full_macro_noalloc(fd.data_ptr(), wl.n_cell, wl.N, wl.lo, wl.hi, out.data_ptr(),
                                 stream.cuda_stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        for k, v in _macro_err(got, ref).items():
            assert v <= TOL, (k, v)
        for k, v in _macro_err(got, _oracle_moments(wl, f)).items():   # and the FP64 oracle's
            assert v <= TOL, ("oracle", k, v)


def test_noalloc_macro_rejects_oversized_batch():
    import torch
    import paper_1912_04582_gb300 as P
    from paper_1912_04582_gb300 import _native as N

    torch.cuda.set_device(0)
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(N.DvmError) as ei:
        P.dvm_full_macro_noalloc(buf.data_ptr(), 16385, (4, 4, 4), (-1, -1, -1), (1, 1, 1),
                                 buf.data_ptr())
    assert ei.value.code == N.DVM_ERR_INVALID_ARG
    assert "16384" in P.dvm_last_error()
