"""The CFFYN_ETIMEOUT contract of the tensor-core operator kernels: with a wait
bound of 0 every pipeline wait gives up at once (no GPU fault, no endless
wait: the blocks let the copies and products already issued finish, free
their tensor memory and return), the step reports CFFYN_ETIMEOUT, and with
the default bound restored the same handle steps normally again."""

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


def _shell(cf, n_f=50):
    n_r, N, J, L = 9, 12, 24, 10
    sh = cf.Shell(n_r, N, J, 1.8, 11.0, L, n_fields=n_f, precision=cf.MIXED)
    u = torch.from_numpy(inputs.kerr_schild_state(n_r, N, J, 1.8, 11.0, n_fields=n_f, amp=1e-6,
                                                  ell=2, seed=0)).cuda()
    sh.init_gauge_from_state(u)
    return sh, u


def test_step_reports_timeout_and_recovers(cf):
    sh, u = _shell(cf)
    dt = sh.default_dt()
    ref = u.clone()
    sh.rk4_step(ref, dt, 2)
    sh.set_wait_limit(0.0)
    bad = u.clone()
    with pytest.raises(cf.CffynError) as ei:
        sh.rk4_step(bad, dt, 2)
    assert ei.value.code == cf.ETIMEOUT
    assert "gave up" in str(ei.value)
    sh.set_wait_limit(-1.0)                   # the default bound again
    again = u.clone()
    sh.rk4_step(again, dt, 2)
    torch.cuda.synchronize()
    assert torch.equal(again, ref)
    sh.destroy()


def test_batch_names_the_shell_that_timed_out(cf):
    s0, u0 = _shell(cf)
    s1, u1 = _shell(cf, 54)
    b = cf.Batch([s0, s1])
    r0, r1 = u0.clone(), u1.clone()
    b.rk4_step([r0, r1], None, 1)
    s1.set_wait_limit(0.0)
    with pytest.raises(cf.CffynError) as ei:
        b.rk4_step([u0.clone(), u1.clone()], None, 1)
    assert ei.value.code == cf.ETIMEOUT and "shell 1" in str(ei.value)
    s1.set_wait_limit(-1.0)
    a0, a1 = u0.clone(), u1.clone()
    b.rk4_step([a0, a1], None, 1)
    torch.cuda.synchronize()
    assert torch.equal(a0, r0) and torch.equal(a1, r1)
    b.destroy()
    s0.destroy()
    s1.destroy()


def test_static_derivs_mark_a_timeout_in_the_output_only(cf):
    sh, u = _shell(cf)
    dt = sh.default_dt()
    ref = u.clone()
    sh.rk4_step(ref, dt, 1)
    out = torch.zeros((3, 5) + tuple(u.shape[1:]), dtype=torch.float64, device="cuda")
    sh.derivs_static(u, 5, out)               # set-up call
    sh.set_wait_limit(0.0)
    sh.derivs_static(u, 5, out)
    torch.cuda.synchronize()
    assert torch.isnan(out).all()
    sh.set_wait_limit(-1.0)
    # the shell's own status word was not touched: a step succeeds ...
    v = u.clone()
    sh.rk4_step(v, dt, 1)
    assert torch.equal(v, ref)
    # ... and the next static call is finite again
    sh.derivs_static(u, 5, out)
    torch.cuda.synchronize()
    assert np.isfinite(out.cpu().numpy()).all()
    sh.destroy()


def test_wait_limit_arguments(cf):
    sh, _ = _shell(cf)
    for bad in (float("nan"), 61.0):
        with pytest.raises(cf.CffynError) as ei:
            sh.set_wait_limit(bad)
        assert ei.value.code == cf.EINVAL
    sh.set_wait_limit(2.5)
    sh.set_wait_limit(-1.0)
    sh.destroy()
