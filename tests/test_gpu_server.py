"""Serving (continuous batching of steady solves) through the C ABI: admission by the
device-memory budget and free slots, interleaved steps on separate streams, retirement at
the residual target, and the same result alone and in a mix."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    import paper_1912_04582_gb300 as P
    torch.cuda.set_device(0)
    return P


def _requests():
    a = W.channel(n_cell_target=256, N=12, Kn=1.0, kind="poiseuille", seed=1)
    b = W.channel(n_cell_target=108, N=12, Kn=0.5, kind="transpiration", seed=2)
    c = W.cavity(nside=3, N=10, Kn=0.5, lid=0.2)
    return [(a, dict(format=0)), (b, dict(format=1, precision=1, rank_cap=8, tol=1e-6)),
            (c, dict(format=1, precision=0, rank_cap=8, tol=1e-6))]


def _solve_alone(P, wl, kw, res_tol, max_steps, check_every):
    srv = P.Server(1 << 34, 1)
    t = srv.submit(wl, res_tol=res_tol, max_steps=max_steps, check_every=check_every, **kw)
    assert srv.run(600.0) == 0
    st = srv.poll(t)
    out = srv.result(t, wl.n_cell)
    srv.close()
    return st, out


def test_mix_equals_alone(P):
    from paper_1912_04582_gb300 import _native as N
    reqs = _requests()
    alone = [_solve_alone(P, wl, kw, 1e-3, 3000, 20) for wl, kw in reqs]
    srv = P.Server(1 << 34, 3)
    tickets = [srv.submit(wl, res_tol=1e-3, max_steps=3000, check_every=20, **kw) for wl, kw in reqs]
    assert srv.run(600.0) == 0
    for (wl, _), t, (st_a, out_a) in zip(reqs, tickets, alone):
        st = srv.poll(t)
        assert st["state"] in (N.DVM_REQ_CONVERGED, N.DVM_REQ_NOT_CONVERGED)
        assert st["state"] == st_a["state"] and st["steps"] == st_a["steps"]
        out = srv.result(t, wl.n_cell)
        assert np.max(np.abs(out - out_a)) <= 1e-12 * np.max(np.abs(out_a))
        assert st["latency_s"] > 0
    srv.close()


def test_admission_respects_budget_and_slots(P):
    from paper_1912_04582_gb300 import _native as N
    wl = W.cavity(nside=4, N=12)
    est = P.dvm_estimate_memory(wl)
    srv = P.Server(int(1.5 * est), 4)
    tickets = [srv.submit(wl, res_tol=1e-12, max_steps=40, check_every=10) for _ in range(3)]
    srv.run(0.0)                       # one pass: admits what fits
    states = [srv.poll(t)["state"] for t in tickets]
    assert states.count(N.DVM_REQ_RUNNING) == 1 and states.count(N.DVM_REQ_QUEUED) == 2
    assert srv.run(600.0) == 0
    for t in tickets:
        st = srv.poll(t)
        assert st["state"] == N.DVM_REQ_NOT_CONVERGED and st["steps"] == 40
    srv.close()
    srv = P.Server(int(0.5 * est), 4)
    with pytest.raises(N.DvmError):
        srv.submit(wl)
    srv.close()


def test_failed_request_does_not_disturb_others(P):
    from paper_1912_04582_gb300 import _native as N
    good = W.cavity(nside=3, N=10, Kn=0.5)
    bad = W.sod_row(N=6)
    bad.lo = (-5.0, -4.0, -5.0)        # symmetry on a non-symmetric grid: unsupported
    srv = P.Server(1 << 34, 2)
    tb = srv.submit(bad, res_tol=1e-3, max_steps=100)
    tg = srv.submit(good, res_tol=1e-3, max_steps=2000, check_every=20)
    assert srv.run(600.0) == 0
    assert srv.poll(tb)["state"] == N.DVM_REQ_FAILED
    assert srv.poll(tg)["state"] in (N.DVM_REQ_CONVERGED, N.DVM_REQ_NOT_CONVERGED)
    srv.close()
