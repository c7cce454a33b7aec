"""The paper's single black hole runs on the shell R10 (Sec. 4.1) on the CUDA
path, through the C-ABI (paper_1104_3408_gb300.r10): initial data with a
numerical Phi, parity of PER_STEP Yn runs at the paper's Courant factor 4
against the oracle, the exponential convergence of the initial truncation
error with N_r (Fig. r10_rconv) and the filter-strength result of
Fig. r10_nf."""

import numpy as np
import pytest

import oracle
from paper_1104_3408_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

R_IN, R_OUT = 1.8, 11.8


@pytest.fixture(scope="module")
def r10():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1104_3408_gb300 import r10
    return r10


def oracle_initial(n_r, N):
    J = 2 * N
    u = inputs.kerr_schild_state(n_r, N, J, R_IN, R_OUT, amp=0.0)
    dg = oracle.OracleShell(n_r, N, J, R_IN, R_OUT, 0).derivs(u[:10])
    u[20:50] = dg.reshape((30,) + u.shape[1:])
    u[10:20] = inputs.kerr_schild_pi_from_phi(dg, n_r, N, J, R_IN, R_OUT)
    return u


def test_initial_data_matches_oracle(r10):
    u = r10.initial_state(13, 9).cpu().numpy()
    ref = oracle_initial(13, 9)
    assert np.abs(u - ref).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("prec", [0, 1])
def test_per_step_run_at_courant_4_matches_oracle(r10, prec):
    # default configuration of the paper's runs: Yn filter after every RK4
    # step, n_f = 4, dt = 4 min dx; odd N_theta = 9 as in the paper
    n_r, N, steps = 13, 9, 12
    cf = r10.cffyn
    u = r10.initial_state(n_r, N)
    sh = r10.make_shell(n_r, N, precision=prec)
    sh.init_gauge_from_state(u)
    dt = sh.default_dt()
    ref = oracle.OracleShell(n_r, N, 2 * N, R_IN, R_OUT, N - 1 - 4, filter_mode="step")
    assert abs(dt - 4.0 * ref.dx_min()) < 1e-14
    u0 = u.cpu().numpy()
    ref.init_gauge_from_state(u0)
    sh.rk4_step(u, dt, steps)
    got = u.cpu().numpy()
    want = ref.rk4_step(u0, dt, steps)
    tol = 1e-12 if prec == cf.FP64 else 1e-10
    assert np.abs(got - want).max() < tol * np.abs(want).max()
    # the monitored quantity: d_t g_tt on the inner sphere
    buf = torch.empty_like(u)
    v = r10.rhs_gtt_inner(sh, u, buf)
    w = np.abs(ref.rhs(want)[0, :, :, 0]).max()
    scale = np.abs(ref.derivs(want)).max()
    assert abs(v - w) < tol * scale
    sh.destroy()


@pytest.mark.parametrize("prec", [0, 1])
def test_initial_truncation_error_converges_with_n_r(r10, prec):
    # Fig. r10_rconv: the analytic data's error decays exponentially with N_r
    # at N_theta = 9, N_phi = 18
    got, want = [], []
    for n_r in (13, 19, 25, 31, 37):
        u = r10.initial_state(n_r, 9)
        sh = r10.make_shell(n_r, 9, precision=prec)
        sh.init_gauge_from_state(u)
        buf = torch.empty_like(u)
        sh.rhs(u, buf)
        got.append(float(buf.abs().max()))
        sh.destroy()
        u0 = oracle_initial(n_r, 9)
        ref = oracle.OracleShell(n_r, 9, 18, R_IN, R_OUT, 4)
        ref.init_gauge_from_state(u0)
        want.append(np.abs(ref.rhs(u0)).max())
        scale = np.abs(ref.derivs(u0)).max()
        # near the inner sphere the right-hand side sums derivative terms
        # weighted by metric factors up to 1 + 2M/r_in = 2.1, so FP64
        # summation order alone moves it by a few 1e-12 of max |d_k u|
        tol = 4e-12 if prec == 0 else 1e-10
        assert abs(got[-1] - want[-1]) < tol * scale, (n_r, got[-1], want[-1])
    assert all(a > 30.0 * b for a, b in zip(got, got[1:])), got


def test_filter_strength_decides_stability_as_in_fig_r10_nf(r10):
    # n_f = 0, 1, 2 fail within t = 110; n_f = 3, 4 do not
    runs = {nf: r10.run_one(13, 9, 110.0, n_f=nf) for nf in range(5)}
    for nf in (0, 1, 2):
        assert runs[nf]["failed_at"] is not None and runs[nf]["failed_at"] <= 110.0, runs[nf]
    for nf in (3, 4):
        assert runs[nf]["failed_at"] is None, runs[nf]
        assert runs[nf]["rhs_gtt_max"] < 1e-3


def test_courant_limit_brackets_tab_dtfac(r10):
    # Tab. dtfac gives lambda_max = 6.1 on 25 x 9 x 18 (its Delta t_stab
    # 0.2651 and Delta t_unst 0.2666 over min dx = 0.0428): 6.0 runs, 6.5 fails
    ok = r10.run_one(25, 9, 500.0, courant=6.0, sample_steps=10)
    bad = r10.run_one(25, 9, 500.0, courant=6.5, sample_steps=10)
    assert ok["failed_at"] is None and ok["rhs_gtt_final"] < 1e-9
    assert bad["failed_at"] is not None and bad["failed_at"] < 500.0


def test_scalar_y_filter_fails_where_yn_settles_as_in_fig_r10_f0(r10):
    # Fig. r10_f0: with the scalar Y filter (n_f = 4) the run fails within a
    # few thousand; with the Yn filter it settles at round-off level
    cf = r10.cffyn
    y = r10.run_one(25, 9, 4000.0, filter_kind=cf.FILTER_Y, sample_steps=50)
    yn = r10.run_one(25, 9, 4000.0, filter_kind=cf.FILTER_YN, sample_steps=50)
    assert y["failed_at"] is not None and y["failed_at"] < 4000.0
    assert yn["failed_at"] is None and yn["rhs_gtt_late_max"] < 1e-10
