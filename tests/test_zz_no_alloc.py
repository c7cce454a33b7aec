"""cffyn_derivs_static (allocation-free Cartesian derivatives, intermediates in
the library's fixed device array) against cffyn_derivs on the same shell and
inputs, through the C-ABI.  Two calls in a row with inputs of very different
magnitude check that nothing stale survives between calls (the per-field
exponent words of the mixed path must be zeroed by every call).  This file is
collected last on purpose and also passes alone in a fresh process."""

import numpy as np
import pytest

from paper_1104_3408_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-10}   # FP64, MIXED: the tolerances of the derivative parity tests


@pytest.fixture(scope="module")
def cf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1104_3408_gb300 import cffyn
    return cffyn


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def rel(got, ref):
    d = np.abs(got - ref).reshape(-1, ref.shape[-4] * ref.shape[-3] * ref.shape[-2] * ref.shape[-1])
    r = np.abs(ref).reshape(d.shape)
    return (d.max(axis=1) / np.maximum(r.max(axis=1), 1e-300)).max()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n_r,N,J,L,n_f", [(9, 12, 24, 10, 50), (13, 9, 18, 6, 7), (33, 32, 64, 30, 5)])
def test_static_derivs_match_derivs_on_two_calls(cf, prec, n_r, N, J, L, n_f):
    sh = cf.Shell(n_r, N, J, 1.8, 11.0, L, precision=prec)
    P = n_r * N * J
    u1 = inputs.band_limited_fields(n_r, N, J, 1.8, 11.0, seed=11)
    # second input: other fields, 1e-9 of the size (a stale exponent from the
    # first call would cost about 30 bits on the mixed path)
    u2 = 1e-9 * inputs.band_limited_fields(n_r, N, J, 1.8, 11.0, seed=12)
    for u0 in (u1, u2):
        u = dev(u0)
        ref = torch.empty((3,) + u0.shape, dtype=torch.float64, device="cuda")
        sh.derivs(u, ref)
        got = torch.full((3, n_f) + u0.shape[1:], float("nan"), dtype=torch.float64, device="cuda")
        sh.derivs_static(u, n_f, got)
        torch.cuda.synchronize()
        r = ref.cpu().numpy()[:, :n_f]
        g = got.cpu().numpy()
        assert np.isfinite(g).all()
        assert g.shape == (3, n_f, J, N, n_r) and P == J * N * n_r
        e = rel(g, r)
        assert e < TOL[prec], e
    sh.destroy()


@pytest.mark.parametrize("prec,n_ok", [(0, 5), (1, 5)])
def test_static_derivs_reject_requests_above_the_limit(cf, prec, n_ok):
    n_r, N, J, L = 33, 32, 64, 30
    sh = cf.Shell(n_r, N, J, 1.8, 11.0, L, precision=prec)
    u = dev(inputs.band_limited_fields(n_r, N, J, 1.8, 11.0, seed=13))
    out = torch.zeros((3, n_ok + 1, J, N, n_r), dtype=torch.float64, device="cuda")
    sh.derivs_static(u, n_ok, out[:, :n_ok].contiguous())
    with pytest.raises(cf.CffynError) as ei:
        sh.derivs_static(u, n_ok + 1, out)
    assert ei.value.code == cf.EINVAL
    assert "static scratch" in str(ei.value)
    # nothing was launched for the rejected call: out is still zero
    torch.cuda.synchronize()
    assert not out.any()
    with pytest.raises(cf.CffynError):
        sh.derivs_static(u, 0, out)
    sh.destroy()


def test_static_derivs_beside_a_step_of_the_same_shell(cf):
    # the static call reads only the shell's constant operators and keeps its
    # own status word: enqueued on a second stream while an RK4 step of the
    # same shell runs on a first one, both results equal their serial ones
    n_r, N, J, L = 9, 12, 24, 10
    sh = cf.Shell(n_r, N, J, 1.8, 11.0, L)
    a = dev(inputs.kerr_schild_state(n_r, N, J, 1.8, 11.0, amp=1e-6, ell=2, seed=0))
    sh.init_gauge_from_state(a)
    v0 = inputs.band_limited_fields(n_r, N, J, 1.8, 11.0, seed=21)
    v = dev(v0)
    ref = torch.empty((3,) + v0.shape, dtype=torch.float64, device="cuda")
    sh.derivs(v, ref)
    b = a.clone()
    sh.rk4_step(b, 0.0, 3)                    # serial step
    got = torch.full((3, 50) + v0.shape[1:], float("nan"), dtype=torch.float64, device="cuda")
    sh.derivs_static(v, 50, got)              # set-up call before the streams
    torch.cuda.synchronize()
    got.fill_(float("nan"))
    c = a.clone()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    sh.derivs_static(v, 50, got, stream=s2)   # asynchronous: still running ...
    sh.rk4_step(c, 0.0, 3, stream=s1)         # ... while the step runs (and syncs s1)
    torch.cuda.synchronize()
    assert torch.equal(c, b)
    g = got.cpu().numpy()
    assert np.isfinite(g).all()
    assert rel(g, ref.cpu().numpy()) < TOL[1]
    sh.destroy()
