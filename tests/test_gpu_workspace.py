"""Caller-attached workspace (cffyn_workspace_size / cffyn_attach_workspace)
through the C-ABI: a shell computing in a PyTorch-owned buffer gives the
same bits as one with the library's own workspace."""

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


@pytest.mark.parametrize("prec", [0, 1])
def test_attached_workspace_is_bitwise_the_library_one(cf, prec):
    n_r, N, J, L = 13, 12, 24, 10
    u0 = torch.from_numpy(inputs.kerr_schild_state(n_r, N, J, 1.8, 11.0, amp=1e-4, ell=2, seed=9)).cuda()
    ref = cf.Shell(n_r, N, J, 1.8, 11.0, L, precision=prec)
    sh = cf.Shell(n_r, N, J, 1.8, 11.0, L, precision=prec, flags=cf.DEFER_WORKSPACE)
    nbytes = sh.workspace_size()
    assert nbytes == ref.workspace_size() > 0
    assert ref.device_bytes() - sh.device_bytes() == nbytes
    u = u0.clone()
    out = torch.empty_like(u)
    with pytest.raises(cf.CffynError) as ei:
        sh.init_gauge_from_state(u)     # needs the workspace (gauge derivatives)
    assert ei.value.code == cf.EINVAL and "workspace" in str(ei.value)
    with pytest.raises(cf.CffynError):
        sh.attach_workspace(torch.empty(nbytes // 8 - 1, dtype=torch.float64, device="cuda"))
    buf = torch.full((nbytes // 8,), float("nan"), dtype=torch.float64, device="cuda")
    sh.attach_workspace(buf)
    assert sh.device_bytes() == ref.device_bytes() - nbytes
    ref.init_gauge_from_state(u)
    sh.init_gauge_from_state(u)
    a, b = torch.empty_like(u), torch.empty_like(u)
    ref.rhs(u, a)
    sh.rhs(u, b)
    assert torch.equal(a, b)
    ref.filter(u, a)
    sh.filter(u, b)
    assert torch.equal(a, b)
    ua, ub = a.clone(), a.clone()
    ref.rk4_step(ua, 0.0, 3)
    sh.rk4_step(ub, 0.0, 3)
    assert torch.equal(ua, ub)
    # back to a library workspace: the step graph is recaptured
    sh.attach_workspace(None)
    assert sh.device_bytes() == ref.device_bytes()
    del buf
    ref.rk4_step(ua, 0.0, 2)
    sh.rk4_step(ub, 0.0, 2)
    assert torch.equal(ua, ub)
    # and a fresh caller buffer between two calls of the same batch
    b1 = cf.Batch([sh])
    b1.rk4_step([ub], None, 1)
    sh.attach_workspace(torch.empty(nbytes // 8, dtype=torch.float64, device="cuda"))
    b1.rk4_step([ub], None, 1)
    ref.rk4_step(ua, 0.0, 2)
    torch.cuda.synchronize()
    assert torch.equal(ua, ub)
    b1.destroy()
    sh.destroy()
    ref.destroy()
