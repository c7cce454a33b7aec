"""Pins of the oracle's 54- and 58-field states (App. A.1): the gauge source
H_a as evolved fields 50..53 and, for 58 fields, G_a = d_t H_a as fields
54..57 with d_t H_a = G_a, d_t G_a = 0 (the reading of the unspecified
extended-gauge equation that reproduces the static gauge).  CPU only."""

import numpy as np
import pytest

import oracle
from oracle import ghg
from paper_1104_3408_gb300 import inputs

N_R, N_T, N_P, L = 9, 8, 16, 6


def _state50(seed=0):
    return inputs.kerr_schild_state(N_R, N_T, N_P, 1.8, 11.0, amp=1e-4, ell=2, seed=seed)


def _gauge(u50):
    return ghg.gauge_source_from_state(u50.reshape(50, -1)).reshape((4,) + u50.shape[1:])


def test_54_field_rhs_equals_the_static_gauge_rhs():
    u50 = _state50()
    H = _gauge(u50)
    s50 = oracle.OracleShell(N_R, N_T, N_P, 1.8, 11.0, L)
    s50.set_gauge(H)
    ref = s50.rhs(u50)
    s54 = oracle.OracleShell(N_R, N_T, N_P, 1.8, 11.0, L, n_fields=54)
    got = s54.rhs(np.concatenate([u50, H]))
    scale = np.abs(s50.derivs(u50)).max()
    assert np.abs(got[:50] - ref).max() <= 1e-13 * scale
    assert not got[50:54].any()


def test_58_field_gauge_velocity_enters_as_d_t_h():
    # d_t H_a = G_a, d_t G_a = 0, and in eq. Pidot the term
    # -alpha (nabla_a H_b + nabla_b H_a) with d_0 H_b = G_b adds
    # -alpha (delta_a0 G_b + delta_b0 G_a) to d_t Pi_ab
    u50 = _state50(1)
    H = _gauge(u50)
    G = inputs.band_limited_fields(N_R, N_T, N_P, 1.8, 11.0, seed=3)[:4] * 1e-2
    s58 = oracle.OracleShell(N_R, N_T, N_P, 1.8, 11.0, L, n_fields=58)
    r0 = s58.rhs(np.concatenate([u50, H, np.zeros_like(H)]))
    r1 = s58.rhs(np.concatenate([u50, H, G]))
    assert np.array_equal(r1[50:54], G)
    assert not r1[54:58].any()
    g, _, _ = ghg.split_state(u50.reshape(50, -1))
    alpha = ghg.three_plus_one(g)[0].reshape(u50.shape[1:])
    interior = (slice(None), slice(None), slice(0, N_R - 1))  # the outer sphere has the BC
    for a in range(4):
        for b in range(a, 4):
            s = oracle.ynfilter.sym_index(a, b)
            want = np.zeros_like(alpha)
            if a == 0:
                want = want - alpha * G[b]
            if b == 0:
                want = want - alpha * G[a]
            d = (r1[10 + s] - r0[10 + s])[interior]
            assert np.abs(d - want[interior]).max() <= 1e-12 * (1 + np.abs(want).max())
    # d_t g is untouched everywhere; d_t Phi in the interior (on the outer
    # sphere the boundary condition mixes the Pi and Phi right-hand sides)
    for f in range(0, 10):
        assert np.abs(r1[f] - r0[f]).max() <= 1e-13 * (1 + np.abs(r0[f]).max())
    for f in range(20, 50):
        assert np.abs(r1[f] - r0[f])[interior].max() <= 1e-13 * (1 + np.abs(r0[f]).max())


@pytest.mark.parametrize("nf", [54, 58])
def test_gauge_groups_keep_constant_vectors_and_filter_idempotently(nf):
    u = np.zeros((nf, N_P, N_T, N_R))
    u[:50] = _state50(2)
    c = np.array([0.3, -1.2, 0.7, 2.0])
    for a in range(4):
        u[50 + a] = c[a]
        if nf == 58:
            u[54 + a] = -0.5 * c[a]
    s = oracle.OracleShell(N_R, N_T, N_P, 1.8, 11.0, L, n_fields=nf)
    f = s.filter(u)
    assert np.abs(f[50:nf] - u[50:nf]).max() < 1e-12
    v = u.copy()
    v[50:nf] += inputs.band_limited_fields(N_R, N_T, N_P, 1.8, 11.0, seed=5)[:nf - 50]
    f1 = s.filter(v)
    assert np.abs(s.filter(f1)[50:nf] - f1[50:nf]).max() < 1e-12


def test_58_field_rk4_moves_h_linearly_in_time():
    # constant G survives the filter, so every stage slope of H is G and
    # RK4 gives H(t) = H(0) + t G exactly
    u50 = _state50(3)
    H = _gauge(u50)
    G = np.broadcast_to(np.array([1e-3, -2e-3, 0.5e-3, 1.5e-3])[:, None, None, None], H.shape)
    u = np.concatenate([u50, H, G])
    s = oracle.OracleShell(N_R, N_T, N_P, 1.8, 11.0, L, n_fields=58)
    dt = 0.25 * s.dx_min()
    out = s.rk4_step(u, dt, 3)
    assert np.abs(out[50:54] - (H + 3 * dt * G)).max() < 1e-14
    assert np.abs(out[54:58] - G).max() == 0.0
