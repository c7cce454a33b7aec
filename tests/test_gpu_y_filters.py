"""The component-wise filters of Sec. 3.5 through the C-ABI against the
oracle: the scalar Y filter and the graded Yg filter (eq. nfofmu), on the
filter alone and inside RK4 steps (both filter placements), for 50- and
58-field states.  Tolerances as for the Yn filter."""

import numpy as np
import pytest

import oracle
from paper_1104_3408_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-10}   # FP64, MIXED
SHAPES = [(9, 12, 24, 10), (13, 9, 18, 6), (33, 32, 64, 30), (9, 12, 24, 9), (9, 12, 24, 0),
          (13, 9, 18, 1), (13, 9, 18, 8)]
KINDS = {"y": 1, "yg": 2}


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


@pytest.mark.parametrize("kind", ["y", "yg"])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n_r,N,J,L", SHAPES)
def test_filter(cf, kind, prec, n_r, N, J, L):
    # (9, 12, 24, 9): L + 3 > N - 1, the graded degrees are capped;
    # L = 0, 1: below every field's spatial degree; (13, 9, 18, 8): L = N - 1
    u0 = inputs.band_limited_fields(n_r, N, J, 1.8, 11.0, seed=31)
    ref = oracle.OracleShell(n_r, N, J, 1.8, 11.0, L, filter_kind=kind).filter(u0)
    sh = cf.Shell(n_r, N, J, 1.8, 11.0, L, precision=prec, filter_kind=KINDS[kind])
    out = torch.empty_like(dev(u0))
    sh.filter(dev(u0), out)
    got = out.cpu().numpy()
    sh.destroy()
    e = rel_rows(got, ref)
    assert e < TOL[prec], e


@pytest.mark.parametrize("kind", ["y", "yg"])
def test_filter_58_fields(cf, kind):
    n_r, N, J, L = 9, 12, 24, 7
    u0 = inputs.band_limited_fields(n_r, N, J, 1.8, 11.0, n_fields=58, seed=32)
    ref = oracle.OracleShell(n_r, N, J, 1.8, 11.0, L, n_fields=58, filter_kind=kind).filter(u0)
    sh = cf.Shell(n_r, N, J, 1.8, 11.0, L, n_fields=58, precision=1, filter_kind=KINDS[kind])
    out = torch.empty_like(dev(u0))
    sh.filter(dev(u0), out)
    got = out.cpu().numpy()
    sh.destroy()
    assert rel_rows(got, ref) < TOL[1]


@pytest.mark.parametrize("kind", ["y", "yg"])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("mode", ["substep", "step"])
def test_rk4_steps(cf, kind, prec, mode):
    n_r, N, J, L = 9, 12, 24, 8
    u0 = inputs.kerr_schild_state(n_r, N, J, 1.8, 11.0, amp=1e-5, ell=2, seed=7)
    rs = oracle.OracleShell(n_r, N, J, 1.8, 11.0, L, filter_mode=mode, filter_kind=kind)
    rs.init_gauge_from_state(u0)
    dt = 0.25 * rs.dx_min()
    start = rs.filter(u0) if mode == "substep" else u0
    ref = rs.rk4_step(start, dt, 5)
    sh = cf.Shell(n_r, N, J, 1.8, 11.0, L, precision=prec, filter_kind=KINDS[kind],
                  filter_mode=cf.FILTER_SUBSTEP if mode == "substep" else cf.FILTER_STEP)
    u = dev(u0)
    sh.init_gauge_from_state(u)
    v = torch.empty_like(u)
    if mode == "substep":
        sh.filter(u, v)
    else:
        v.copy_(u)
    sh.rk4_step(v, dt, 5)
    got = v.cpu().numpy()
    sh.destroy()
    e = np.abs(got - ref).max() / np.abs(ref).max()
    assert e < (1e-12 if prec == 0 else 1e-8), e
    assert np.abs(ref - start).max() > 1e-9
