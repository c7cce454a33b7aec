"""Parity of the 54- and 58-field states (App. A.1 with the gauge source H_a
as evolved fields 50..53 and, for 58 fields, G_a = d_t H_a as fields 54..57)
between the CUDA path, through the C-ABI, and the CPU oracle on seeded
inputs.  Tolerances as in the 50-field parity tests: FP64 path 1e-12, mixed
path 1e-10 for the right-hand side and the filter, 1e-8 after RK4 steps."""

import numpy as np
import pytest

import oracle
from oracle import ghg
from paper_1104_3408_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-10}   # FP64, MIXED
SHAPES = [(9, 12, 24, 10), (13, 9, 18, 6), (33, 32, 64, 30)]


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


def rel_rows(got, ref):
    d = np.abs(got - ref).reshape(ref.shape[0], -1).max(axis=1)
    r = np.abs(ref).reshape(ref.shape[0], -1).max(axis=1)
    return (d / np.maximum(r, 1e-300)).max()


def gauge_state(nf, n_r, N, J, amp, seed, h_pert=1e-3, g_amp=1e-2):
    """Perturbed Kerr-Schild data with H_a = -Gamma_a + a smooth perturbation
    (so that d_i H_a and the gauge constraint are not trivial) and, for 58
    fields, a smooth G_a."""
    u50 = inputs.kerr_schild_state(n_r, N, J, 1.8, 11.0, amp=amp, ell=2, seed=seed)
    H = ghg.gauge_source_from_state(u50.reshape(50, -1)).reshape((4,) + u50.shape[1:])
    extra = inputs.band_limited_fields(n_r, N, J, 1.8, 11.0, n_fields=8, seed=seed + 100)
    parts = [u50, H + h_pert * extra[:4]]
    if nf == 58:
        parts.append(g_amp * extra[4:8])
    return np.ascontiguousarray(np.concatenate(parts))


@pytest.mark.parametrize("nf", [54, 58])
@pytest.mark.parametrize("prec", [0, 1])
def test_init_gauge_writes_the_state(cf, nf, prec):
    n_r, N, J, L = 13, 12, 24, 10
    u0 = gauge_state(nf, n_r, N, J, 1e-3, 7)
    want = ghg.gauge_source_from_state(u0[:50].reshape(50, -1)).reshape((4,) + u0.shape[1:])
    sh = cf.Shell(n_r, N, J, 1.8, 11.0, L, n_fields=nf, precision=prec)
    u = dev(u0)
    sh.init_gauge_from_state(u)
    got = u.cpu().numpy()
    sh.destroy()
    assert np.array_equal(got[:50], u0[:50])
    assert rel_rows(got[50:54], want) < 1e-13
    if nf == 58:
        assert not got[54:58].any()


@pytest.mark.parametrize("nf", [54, 58])
@pytest.mark.parametrize("prec", [0, 1])
def test_set_gauge_is_rejected_and_rhs_needs_none(cf, nf, prec):
    n_r, N, J, L = 9, 12, 24, 10
    u0 = gauge_state(nf, n_r, N, J, 1e-4, 1)
    sh = cf.Shell(n_r, N, J, 1.8, 11.0, L, n_fields=nf, precision=prec)
    with pytest.raises(cf.CffynError) as ei:
        sh.set_gauge(dev(u0[50:54]))
    assert ei.value.code == cf.EINVAL
    out = torch.empty_like(dev(u0))
    sh.rhs(dev(u0), out)  # no gauge call needed: H is part of the state
    torch.cuda.synchronize()
    assert np.isfinite(out.cpu().numpy()).all()
    sh.destroy()


@pytest.mark.parametrize("nf", [54, 58])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n_r,N,J,L", SHAPES)
def test_filter_gauge_fields(cf, nf, prec, n_r, N, J, L):
    u0 = inputs.band_limited_fields(n_r, N, J, 1.8, 11.0, n_fields=nf, seed=21)
    ref = oracle.OracleShell(n_r, N, J, 1.8, 11.0, L, n_fields=nf).filter(u0)
    sh = cf.Shell(n_r, N, J, 1.8, 11.0, L, n_fields=nf, precision=prec)
    out = torch.empty_like(dev(u0))
    sh.filter(dev(u0), out)
    got = out.cpu().numpy()
    sh.destroy()
    e = rel_rows(got, ref)
    assert e < TOL[prec], e


@pytest.mark.parametrize("nf", [54, 58])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n_r,N,J,L", SHAPES)
def test_rhs_gauge_fields(cf, nf, prec, n_r, N, J, L):
    u0 = gauge_state(nf, n_r, N, J, 1e-4, 3)
    rs = oracle.OracleShell(n_r, N, J, 1.8, 11.0, L, n_fields=nf)
    ref = rs.rhs(u0)
    scale = np.abs(rs.derivs(u0)).max()
    sh = cf.Shell(n_r, N, J, 1.8, 11.0, L, n_fields=nf, precision=prec)
    out = torch.empty_like(dev(u0))
    sh.rhs(dev(u0), out)
    got = out.cpu().numpy()
    sh.destroy()
    e = np.abs(got[:50] - ref[:50]).max() / scale
    assert e < TOL[prec], e
    # d_t H_a = G_a (58) or 0 (54), d_t G_a = 0: copies, exact on the FP64
    # path; the mixed path keeps the leading 48 significand bits (truncated
    # split into a float pair, |x - hi - lo| <= 2^-47 |x|)
    if prec == 0:
        assert np.array_equal(got[50:], ref[50:])
    else:
        assert (np.abs(got[50:] - ref[50:]) <= 2.0 ** -47 * np.abs(ref[50:])).all()
    if nf == 54:
        assert not got[50:54].any()
    else:
        assert not got[54:58].any()


@pytest.mark.parametrize("nf", [54, 58])
@pytest.mark.parametrize("prec", [0, 1])
def test_rk4_gauge_fields(cf, nf, prec):
    n_r, N, J, L = 9, 12, 24, 10
    u0 = gauge_state(nf, n_r, N, J, 1e-6, 0, h_pert=1e-6, g_amp=1e-4)
    rs = oracle.OracleShell(n_r, N, J, 1.8, 11.0, L, n_fields=nf)
    dt = 0.25 * rs.dx_min()
    uf = rs.filter(u0)
    ref = rs.rk4_step(uf, dt, 10)
    sh = cf.Shell(n_r, N, J, 1.8, 11.0, L, n_fields=nf, precision=prec)
    u = dev(u0)
    v = torch.empty_like(u)
    sh.filter(u, v)
    sh.rk4_step(v, dt, 10)
    got = v.cpu().numpy()
    sh.destroy()
    e = np.abs(got - ref).max() / np.abs(ref).max()
    assert e < (1e-12 if prec == 0 else 1e-8), e
    assert np.abs(ref - uf).max() > 1e-9
    if nf == 58:
        # the gauge source moved by about 10 dt G
        assert np.abs(ref[50:54] - uf[50:54]).max() > 1e-6


@pytest.mark.parametrize("prec", [0, 1])
def test_constraint_norms_read_the_gauge_fields(cf, prec):
    n_r, N, J, L = 13, 12, 24, 10
    u0 = gauge_state(54, n_r, N, J, 1e-3, 5)
    rs = oracle.OracleShell(n_r, N, J, 1.8, 11.0, L, n_fields=54)
    c3, c1 = rs.constraint_norms(u0)
    sh = cf.Shell(n_r, N, J, 1.8, 11.0, L, n_fields=54, precision=prec)
    g3, g1 = sh.constraint_norms(dev(u0))
    sh.destroy()
    assert abs(g3 - c3) < 1e-9 * max(c3, 1e-30) + 1e-14
    # H differs from -Gamma by the perturbation: a gauge-constraint norm of
    # its size, the same on both sides
    assert c1 > 1e-5
    assert abs(g1 - c1) < 1e-12 * c1
