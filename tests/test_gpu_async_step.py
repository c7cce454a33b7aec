"""cffyn_rk4_step_async: the RK4 steps of cffyn_rk4_step (Sec. 2.5) enqueued
without the synchronisation at the end.  The results must be bitwise those of
the synchronising call; the status word, read after synchronising, must carry
what the synchronising call reports (non-finite right-hand side, a bounded
wait that gave up); and several calls queued back to back on one stream must
each report their own status."""

import numpy as np
import pytest

from paper_1104_3408_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1104_3408_gb300 import cffyn
    return cffyn


def _shell(cf, precision):
    n_r, N, J, L = 9, 12, 24, 10
    sh = cf.Shell(n_r, N, J, 1.8, 11.0, L, precision=precision)
    u0 = inputs.kerr_schild_state(n_r, N, J, 1.8, 11.0, amp=1e-4, ell=2, seed=3)
    u = torch.from_numpy(u0).cuda()
    sh.init_gauge_from_state(u)
    return sh, u0


def _status(n=1):
    return torch.full((n,), -7, dtype=torch.int32).pin_memory()


@pytest.mark.parametrize("prec", ["MIXED", "FP64"])
def test_async_steps_equal_the_synchronising_call(cf, prec):
    sh, u0 = _shell(cf, getattr(cf, prec))
    dt = sh.default_dt()
    ref = torch.from_numpy(u0).cuda()
    sh.rk4_step(ref, dt, 3)
    got = torch.from_numpy(u0).cuda()
    st = _status()
    sh.rk4_step_async(got, st, dt, 3)
    torch.cuda.synchronize()
    assert int(st[0]) == 0
    cf.check_status(st)
    assert torch.equal(got, ref)
    # queued back to back: one step per call, same result as three at once
    got2 = torch.from_numpy(u0).cuda()
    st3 = _status(3)
    for i in range(3):
        sh.rk4_step_async(got2, st3[i:i + 1], dt, 1)
    torch.cuda.synchronize()
    assert st3.tolist() == [0, 0, 0]
    assert torch.equal(got2, ref)
    sh.destroy()


def test_async_status_reports_nonfinite_and_timeout(cf):
    sh, u0 = _shell(cf, cf.MIXED)
    dt = sh.default_dt()
    bad = torch.from_numpy(u0).cuda()
    bad[25, 3, 2, 1] = float("nan")
    good = torch.from_numpy(u0).cuda()
    ref = torch.from_numpy(u0).cuda()
    sh.rk4_step(ref, dt, 1)
    st = _status(2)
    sh.rk4_step_async(bad, st[0:1], dt, 1)    # the graph is captured again for this buffer
    sh.rk4_step_async(good, st[1:2], dt, 1)   # and again for this one, queued behind
    torch.cuda.synchronize()
    assert cf.load().cffyn_step_status(int(st[0])) == cf.ENONFINITE
    assert int(st[1]) == 0
    assert torch.equal(good, ref)
    with pytest.raises(cf.CffynError) as ei:
        cf.check_status(st)
    assert ei.value.code == cf.ENONFINITE
    # a wait bound of 0: every tensor-core wait gives up, the status says so
    sh.set_wait_limit(0.0)
    t = torch.from_numpy(u0).cuda()
    st1 = _status()
    sh.rk4_step_async(t, st1, dt, 1)
    torch.cuda.synchronize()
    assert cf.load().cffyn_step_status(int(st1[0])) == cf.ETIMEOUT
    sh.set_wait_limit(-1.0)
    again = torch.from_numpy(u0).cuda()
    sh.rk4_step_async(again, st1, dt, 1)
    torch.cuda.synchronize()
    assert int(st1[0]) == 0 and torch.equal(again, ref)
    sh.destroy()


def test_async_argument_errors(cf):
    sh, u0 = _shell(cf, cf.MIXED)
    u = torch.from_numpy(u0).cuda()
    lib = cf.load()
    assert lib.cffyn_rk4_step_async(sh.h, cf._ptr(u, "u"), 0.0, 1, cf._stream(None), None) == cf.EINVAL
    assert lib.cffyn_rk4_step_async(None, cf._ptr(u, "u"), 0.0, 1, cf._stream(None), None) == cf.EINVAL
    st = _status()
    with pytest.raises(cf.CffynError) as ei:
        sh.rk4_step_async(u, st, 0.0, -1)
    assert ei.value.code == cf.EINVAL
    sh.rk4_step_async(u, st, 0.0, 0)          # nothing runs, a zero status word arrives
    torch.cuda.synchronize()
    assert int(st[0]) == 0 and np.array_equal(u.cpu().numpy(), u0)
    sh.set_trace(True)
    with pytest.raises(cf.CffynError) as ei:
        sh.rk4_step_async(u, st, 0.0, 1)
    assert ei.value.code == cf.EINVAL
    sh.set_trace(False)
    with pytest.raises(TypeError):
        sh.rk4_step_async(u, torch.zeros(1, dtype=torch.int64), 0.0, 1)
    sh.destroy()


def test_kept_step_graphs_alternating_and_evicted(cf):
    # the shell keeps the step graphs of its two most recent (u, dt): two
    # buffers stepped in turn replay them, a third evicts one; every state
    # must equal the same number of steps taken on a buffer of its own
    sh, u0 = _shell(cf, cf.MIXED)
    dt = sh.default_dt()
    ref = []
    for k in (1, 2, 3):
        r = torch.from_numpy(u0).cuda()
        sh.rk4_step(r, dt, k)
        ref.append(r)
    bufs = [torch.from_numpy(u0).cuda() for _ in range(3)]
    st = _status(9)
    order = [0, 1, 0, 1, 2, 0, 2, 1, 2]
    for q, b in enumerate(order):
        sh.rk4_step_async(bufs[b], st[q:q + 1], dt, 1)
    torch.cuda.synchronize()
    cf.check_status(st)
    for b in range(3):
        assert torch.equal(bufs[b], ref[order.count(b) - 1])
    sh.destroy()
