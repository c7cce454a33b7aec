"""Parity of the CUDA path (through the C-ABI) with the CPU oracle on seeded
inputs.  Tolerances: FP64 path 1e-12 relative (summation order only); mixed
path 1e-10 relative for derivatives, right-hand side and filter, 1e-8 for
fields after RK4 steps.  "Relative" is max|difference| over an output array
divided by max|reference| of that array; for the right-hand side of
near-static Kerr-Schild data (which is truncation error, ~1e-8, far below the
size of the terms that cancel in it) the denominator is max|d_k u|."""

import numpy as np
import pytest

import oracle
from oracle import cff, swsh
from paper_1104_3408_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-10}   # FP64, MIXED


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


def rel(got, ref, axis=None):
    if axis is None:
        return np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300)
    d = np.abs(got - ref).reshape(ref.shape[0], -1).max(axis=1)
    r = np.abs(ref).reshape(ref.shape[0], -1).max(axis=1)
    return (d / np.maximum(r, 1e-300)).max()


SHAPES = [(9, 12, 24, 10), (13, 9, 18, 6), (33, 32, 64, 30)]


@pytest.mark.parametrize("n_r,N,J,L", SHAPES[:2] + [(17, 16, 32, 0), (5, 6, 12, 5)])
def test_operator_matrices_match_oracle(cf, n_r, N, J, L):
    sh = cf.Shell(n_r, N, J, 1.8, 11.0, L, precision=cf.FP64)
    Dr = cff.radial_diff_matrix(n_r, 1.8, 11.0)
    assert rel(sh.get_operator(0), Dr) < 1e-13
    FD = cff.fourier_diff_matrix(2 * N)
    assert np.abs(sh.get_operator(1) - FD[:N]).max() < 1e-13 * np.abs(FD).max()
    assert rel(sh.get_operator(2), cff.fourier_diff_matrix(J)) < 1e-13
    _, t, _ = cff.grid(n_r, N, J, 1.8, 11.0)
    sl = swsh.SpinLegendre(t, N - 1)
    worst = 0.0
    for n in range(-3, 4):
        for m in range(0, L + 1):
            F = swsh.filter_matrix(sl, n, m, N, L)
            G = sh.get_filter_matrix(n, m)
            worst = max(worst, np.abs(F - G).max())
    sh.destroy()
    assert worst < 1e-11


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n_r,N,J,L", SHAPES)
def test_cartesian_derivatives(cf, prec, n_r, N, J, L):
    u0 = inputs.band_limited_fields(n_r, N, J, 1.8, 11.0, seed=1)
    ref = cff.cartesian_derivatives(u0, 1.8, 11.0)
    sh = cf.Shell(n_r, N, J, 1.8, 11.0, L, precision=prec)
    out = torch.empty((3,) + u0.shape, dtype=torch.float64, device="cuda")
    sh.derivs(dev(u0), out)
    got = out.cpu().numpy()
    sh.destroy()
    e = max(rel(got[d], ref[d], axis=0) for d in range(3))
    assert e < TOL[prec], e


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n_r,N,J,L", SHAPES)
def test_filter(cf, prec, n_r, N, J, L):
    u0 = inputs.band_limited_fields(n_r, N, J, 1.8, 11.0, seed=2)
    ref = oracle.OracleShell(n_r, N, J, 1.8, 11.0, L).filter(u0)
    sh = cf.Shell(n_r, N, J, 1.8, 11.0, L, precision=prec)
    out = torch.empty_like(dev(u0))
    sh.filter(dev(u0), out)
    got = out.cpu().numpy()
    sh.destroy()
    e = rel(got, ref, axis=0)
    assert e < TOL[prec], e


@pytest.mark.parametrize("nf", [50, 58])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n_r,N,J", [(13, 9, 18), (9, 12, 24)])
@pytest.mark.parametrize("which", ["0", "1", "2", "N-1"])
def test_filter_edge_degrees(cf, which, n_r, N, J, prec, nf):
    # L < 3: the spin-3 class keeps no mode (l >= |n|, App. B) and the spin-2
    # class keeps none (L < 2) or only l = 2; L = N - 1: only what the
    # grid cannot resolve (the phi Nyquist mode, the projection's null space).
    # Odd and even N; the 58-field state adds the gauge groups' slots.
    L = N - 1 if which == "N-1" else int(which)
    u0 = inputs.band_limited_fields(n_r, N, J, 1.8, 11.0, n_fields=nf, seed=40 + L)
    ref = oracle.OracleShell(n_r, N, J, 1.8, 11.0, L, n_fields=nf).filter(u0)
    sh = cf.Shell(n_r, N, J, 1.8, 11.0, L, n_fields=nf, precision=prec)
    out = torch.empty_like(dev(u0))
    sh.filter(dev(u0), out)
    got = out.cpu().numpy()
    sh.destroy()
    e = rel(got, ref, axis=0)
    assert e < TOL[prec], e


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n_r,N,J,L", SHAPES)
def test_rhs_with_boundary(cf, prec, n_r, N, J, L):
    u0 = inputs.kerr_schild_state(n_r, N, J, 1.8, 11.0, amp=1e-4, ell=4, seed=3)
    ref_sh = oracle.OracleShell(n_r, N, J, 1.8, 11.0, L)
    ref_sh.init_gauge_from_state(u0)
    ref = ref_sh.rhs(u0)
    scale = np.abs(ref_sh.derivs(u0)).max()
    sh = cf.Shell(n_r, N, J, 1.8, 11.0, L, precision=prec)
    u = dev(u0)
    sh.init_gauge_from_state(u)
    out = torch.empty_like(u)
    sh.rhs(u, out)
    got = out.cpu().numpy()
    sh.destroy()
    e = np.abs(got - ref).max() / scale
    assert e < TOL[prec], e


@pytest.mark.parametrize("prec", [0, 1])
def test_rk4_ten_steps_small_shell(cf, prec):
    # 9 x 12 x 24, L = 10, amplitude 1e-6, l <= 2, dt = 0.25 min dx, 10 steps
    n_r, N, J, L = 9, 12, 24, 10
    u0 = inputs.kerr_schild_state(n_r, N, J, 1.8, 11.0, amp=1e-6, ell=2, seed=0)
    rs = oracle.OracleShell(n_r, N, J, 1.8, 11.0, L)
    rs.init_gauge_from_state(u0)
    dt = 0.25 * rs.dx_min()
    uf = rs.filter(u0)
    ref = rs.rk4_step(uf, dt, 10)
    sh = cf.Shell(n_r, N, J, 1.8, 11.0, L, precision=prec)
    assert abs(sh.default_dt() - dt) < 1e-15
    u = dev(u0)
    sh.init_gauge_from_state(u)
    v = torch.empty_like(u)
    sh.filter(u, v)
    sh.rk4_step(v, dt, 10)
    got = v.cpu().numpy()
    sh.destroy()
    e = rel(got, ref)
    assert e < (1e-12 if prec == 0 else 1e-8), e
    # the evolution really moved the state
    assert np.abs(ref - uf).max() > 1e-9


def test_rk4_per_step_filter_mode(cf):
    n_r, N, J, L = 9, 12, 24, 10
    u0 = inputs.kerr_schild_state(n_r, N, J, 1.8, 11.0, amp=1e-5, ell=2, seed=4)
    rs = oracle.OracleShell(n_r, N, J, 1.8, 11.0, L, filter_mode="step")
    rs.init_gauge_from_state(u0)
    dt = 0.25 * rs.dx_min()
    ref = rs.rk4_step(u0, dt, 3)
    sh = cf.Shell(n_r, N, J, 1.8, 11.0, L, precision=cf.MIXED, filter_mode=cf.FILTER_STEP)
    u = dev(u0)
    sh.init_gauge_from_state(u)
    sh.rk4_step(u, dt, 3)
    got = u.cpu().numpy()
    sh.destroy()
    assert rel(got, ref) < 1e-9


@pytest.mark.parametrize("prec", [0, 1])
def test_constraint_norms(cf, prec):
    n_r, N, J, L = 13, 12, 24, 10
    u0 = inputs.kerr_schild_state(n_r, N, J, 1.8, 11.0, amp=1e-3, ell=2, seed=5)
    rs = oracle.OracleShell(n_r, N, J, 1.8, 11.0, L)
    rs.init_gauge_from_state(u0)
    c3, c1 = rs.constraint_norms(u0)
    sh = cf.Shell(n_r, N, J, 1.8, 11.0, L, precision=prec)
    u = dev(u0)
    sh.init_gauge_from_state(u)
    g3, g1 = sh.constraint_norms(u)
    sh.destroy()
    assert abs(g3 - c3) < 1e-9 * max(c3, 1e-30) + 1e-14
    assert g1 < 1e-14 and c1 < 1e-14


def test_nonfinite_state_is_reported(cf):
    n_r, N, J, L = 5, 6, 12, 4
    u0 = inputs.kerr_schild_state(n_r, N, J, 1.8, 11.0, amp=0.0)
    sh = cf.Shell(n_r, N, J, 1.8, 11.0, L)
    u = dev(u0)
    sh.init_gauge_from_state(u)
    u[25, 3, 2, 1] = float("nan")
    with pytest.raises(cf.CffynError) as ei:
        sh.rk4_step(u, 0.0, 1)
    assert ei.value.code == cf.ENONFINITE
    # the handle stays usable
    v = dev(u0)
    sh.rk4_step(v, 0.0, 1)
    assert torch.isfinite(v).all()
    sh.destroy()


def test_trace_and_profile_report_every_kernel_group(cf):
    n_r, N, J, L = 9, 12, 24, 10
    u0 = inputs.kerr_schild_state(n_r, N, J, 1.8, 11.0, amp=1e-6, ell=2, seed=0)
    sh = cf.Shell(n_r, N, J, 1.8, 11.0, L)
    u = dev(u0)
    sh.init_gauge_from_state(u)
    sh.set_trace(True)
    for _ in range(3):
        sh.rk4_step(u, 0.0, 1)
    ms, launches, steps = sh.get_trace()
    assert steps == 3
    assert all(v > 0 for v in ms.values())
    # 4 stages; the mixed path scans the field exponents of each stage's input
    # and of its filter's input (the filter's later operators take bounds)
    assert launches["d_theta_phi"] == 4 and launches["rhs_pp"] == 4
    assert launches["project"] == 4 and launches["d_r"] == 4 and launches["field_exp"] == 8
    # tracing does not change the result: the untraced graph runs the Yn
    # filter's three operator launches as two chains on two streams (twice
    # the launches), the traced one as one chain, with bitwise equal results
    v = dev(u0)
    w = dev(u0)
    sh.set_trace(False)
    sh.rk4_step(v, 0.0, 2)
    plain = sh.get_trace()[1]
    assert plain["project"] == 8 and plain["dft_fwd"] == 8 and plain["dft_inv"] == 8
    assert plain["d_theta_phi"] == 4 and plain["field_exp"] == 8
    sh.set_trace(True)
    sh.rk4_step(w, 0.0, 2)
    assert torch.equal(v, w)
    prof = sh.profile_step(dev(u0))
    assert all(t > 0 and n > 0 for t, n in prof.values())
    assert {k: n for k, (t, n) in prof.items()} == launches
    sh.destroy()


@pytest.mark.parametrize("rows", [48, 96])
def test_operator_row_groups_keep_parity(cf, rows):
    # every family of operator launches on 48- or 96-row groups (the tuner's
    # two candidates): derivatives, filter and right-hand side stay within
    # the mixed path's tolerance against the oracle
    n_r, N, J, L = 17, 32, 64, 30
    u0 = inputs.band_limited_fields(n_r, N, J, 1.8, 11.0, seed=5)
    sh = cf.Shell(n_r, N, J, 1.8, 11.0, L, precision=cf.MIXED)
    for w in range(5):
        sh.set_operator_rows(w, rows)
    assert [sh.get_operator_rows(w) for w in range(5)] == [rows] * 5
    out = torch.empty((3,) + u0.shape, dtype=torch.float64, device="cuda")
    sh.derivs(dev(u0), out)
    ref = cff.cartesian_derivatives(u0, 1.8, 11.0)
    assert max(rel(out[d].cpu().numpy(), ref[d], axis=0) for d in range(3)) < TOL[1]
    f = torch.empty_like(dev(u0))
    sh.filter(dev(u0), f)
    fref = oracle.OracleShell(n_r, N, J, 1.8, 11.0, L).filter(u0)
    assert rel(f.cpu().numpy(), fref, axis=0) < TOL[1]
    ks = inputs.kerr_schild_state(n_r, N, J, 1.8, 11.0, amp=1e-4, ell=4, seed=3)
    rs = oracle.OracleShell(n_r, N, J, 1.8, 11.0, L)
    rs.init_gauge_from_state(ks)
    u = dev(ks)
    sh.init_gauge_from_state(u)
    r = torch.empty_like(u)
    sh.rhs(u, r)
    assert np.abs(r.cpu().numpy() - rs.rhs(ks)).max() / np.abs(rs.derivs(ks)).max() < TOL[1]
    with pytest.raises(cf.CffynError):
        sh.set_operator_rows(5, 48)
    with pytest.raises(cf.CffynError):
        sh.set_operator_rows(0, 64)
    sh.destroy()
