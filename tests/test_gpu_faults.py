"""Error paths through the C ABI, with every failure made on the host: dvm_solve's
NOT_CONVERGED warning, an out-of-memory allocation, the device error flag a timed-out
bulk-copy wait leaves (reported as a failed step and cleared by a new initial state),
forced admission rejection and cancellation in the serving loop.  Nothing here faults,
traps or hangs the GPU: the injected failures are host-side (dvm_fault_inject)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    import paper_1912_04582_gb300 as P
    torch.cuda.set_device(0)
    yield P
    from paper_1912_04582_gb300 import _native as N
    P.dvm_fault_inject(N.DVM_FAULT_NONE)


@pytest.fixture(autouse=True)
def _disarm(P):
    from paper_1912_04582_gb300 import _native as N
    P.dvm_fault_inject(N.DVM_FAULT_NONE)
    yield
    P.dvm_fault_inject(N.DVM_FAULT_NONE)


def test_solve_converges_and_reports_not_converged(P):
    """dvm_solve stops at the residual target (checked every check_every steps) and
    returns the DVM_NOT_CONVERGED warning (1, not an error) when max_steps is hit first;
    the residual it reports is the one dvm_step reports for the same step."""
    from paper_1912_04582_gb300 import _native as N
    wl = W.sod_row(N=8, Kn=0.5)
    s = P.Solver(wl)
    ok, steps, res = P.dvm_solve(s.h, 1e30, 50, check_every=7)   # any residual meets it
    assert ok and steps == 7 and np.isfinite(res)
    ok, steps, res = P.dvm_solve(s.h, 1e-300, 25, check_every=10)
    assert not ok and steps == 25 and res > 0
    rc = N.load().dvm_solve(s.h.ptr, 1e-300, 3, 1, None, None)
    assert rc == N.DVM_NOT_CONVERGED
    assert P.dvm_get_step_count(s.h) == 7 + 25 + 3
    s.close()
    t = P.Solver(wl)                 # the residual of a solve equals that of the steps
    r_step = [t.step(1) for _ in range(4)][-1]
    u = P.Solver(wl)
    _, steps, r_solve = P.dvm_solve(u.h, 1e-300, 4, check_every=4)
    assert steps == 4 and r_solve == r_step
    t.close()
    u.close()


def test_injected_allocation_failure_is_oom(P):
    from paper_1912_04582_gb300 import _native as N
    wl = W.cavity(nside=3, N=8)
    P.dvm_fault_inject(N.DVM_FAULT_ALLOC, 2)     # the third device allocation fails
    with pytest.raises(N.DvmError) as ei:
        P.Solver(wl)
    assert ei.value.code == N.DVM_ERR_OOM
    assert "injected" in P.dvm_last_error()
    s = P.Solver(wl)                              # disarmed after firing
    s.step(2)
    s.close()


@pytest.mark.parametrize("fmt", [0, 1])
def test_timeout_flag_fails_the_step_until_reinitialised(P, fmt):
    """A timed-out bulk-copy wait sets bit 1 of the context's device flag and its blocks
    return without writing; the host must report the step as failed (TIMEOUT) on every
    call that reads the flag, until a new initial state clears it."""
    from paper_1912_04582_gb300 import _native as N
    wl = W.cavity(nside=3, N=8)
    kw = dict(format=1, precision=1, rank_cap=6, tol=1e-6) if fmt else {}
    s = P.Solver(wl, **kw)
    s.step(1)
    P.dvm_fault_inject(N.DVM_FAULT_TIMEOUT, 0)
    for _ in range(2):               # sticky
        with pytest.raises(N.DvmError) as ei:
            s.step(1)
        assert ei.value.code == N.DVM_ERR_TIMEOUT
        assert "state is undefined" in P.dvm_last_error()
    P.dvm_init_maxwellian(s.h, wl.n0, wl.u0, wl.T0)
    assert np.isfinite(s.step(2))
    s.close()


def test_forced_admission_rejection_keeps_requests_queued(P):
    from paper_1912_04582_gb300 import _native as N
    wl = W.cavity(nside=3, N=8, Kn=0.5)
    srv = P.Server(1 << 34, 2)
    t = srv.submit(wl, res_tol=1e-12, max_steps=20, check_every=10)
    P.dvm_fault_inject(N.DVM_FAULT_ADMIT, 1 << 40)   # every admission check sees no room
    assert srv.run(0.2) == 1
    assert srv.poll(t)["state"] == N.DVM_REQ_QUEUED
    P.dvm_fault_inject(N.DVM_FAULT_NONE)
    assert srv.run(600.0) == 0
    assert srv.poll(t)["state"] == N.DVM_REQ_NOT_CONVERGED
    srv.close()


def test_serving_failures_and_cancellation(P):
    """An allocation failure while admitting one request fails that request only; the
    timeout flag fails the request it hits; a queued request is cancelled at once and a
    running one at the end of its chunk, releasing its memory for the rest."""
    from paper_1912_04582_gb300 import _native as N
    wl = W.cavity(nside=3, N=8, Kn=0.5)
    srv = P.Server(1 << 34, 1)
    P.dvm_fault_inject(N.DVM_FAULT_ALLOC, 0)
    ta = srv.submit(wl, res_tol=1e-12, max_steps=20, check_every=10)
    tb = srv.submit(wl, res_tol=1e-12, max_steps=20, check_every=10)
    assert srv.run(600.0) == 0
    assert srv.poll(ta)["state"] == N.DVM_REQ_FAILED and "injected" in srv.error(ta)
    assert srv.poll(tb)["state"] == N.DVM_REQ_NOT_CONVERGED
    P.dvm_fault_inject(N.DVM_FAULT_TIMEOUT, 0)
    tc = srv.submit(wl, res_tol=1e-12, max_steps=20, check_every=10)
    assert srv.run(600.0) == 0
    assert srv.poll(tc)["state"] == N.DVM_REQ_FAILED and "wait limit" in srv.error(tc)
    # cancellation: one running (single slot), one queued behind it
    tr = srv.submit(wl, res_tol=1e-12, max_steps=100000, check_every=5)
    tq = srv.submit(wl, res_tol=1e-12, max_steps=20, check_every=10)
    srv.run(0.0)
    assert srv.poll(tr)["state"] == N.DVM_REQ_RUNNING
    assert srv.poll(tq)["state"] == N.DVM_REQ_QUEUED
    srv.cancel(tq)
    assert srv.poll(tq)["state"] == N.DVM_REQ_CANCELLED
    srv.cancel(tr)
    assert srv.run(600.0) == 0
    st = srv.poll(tr)
    assert st["state"] == N.DVM_REQ_CANCELLED and 0 < st["steps"] < 100000
    assert np.all(np.isfinite(srv.result(tr, wl.n_cell)))
    with pytest.raises(N.DvmError) as ei:
        srv.cancel(tr)
    assert ei.value.code == N.DVM_ERR_STATE
    srv.close()
