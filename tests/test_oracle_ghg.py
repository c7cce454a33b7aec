"""Pins of the oracle's GHG right-hand side, boundary condition, gauge and RK4
(paper App. A, Secs. 2.5, 4.1).  CPU only."""

import os

import numpy as np
import pytest

import oracle
from oracle import ghg
from paper_1104_3408_gb300 import inputs


def test_kerr_schild_closed_form_3plus1():
    u = inputs.kerr_schild_state(7, 6, 12, 1.8, 11.0, amp=0.0)
    r, t, p = oracle.cff.grid(7, 6, 12, 1.8, 11.0)
    uf = u.reshape(50, -1)
    g, _, _ = ghg.split_state(uf)
    alpha, beta_up, gamma_inv, _, _, _ = ghg.three_plus_one(g)
    R = (r[None, None, :] * np.ones((12, 6, 1))).ravel()
    T = (t[None, :, None] * np.ones((12, 1, 7))).ravel()
    P = (p[:, None, None] * np.ones((1, 6, 7))).ravel()
    l = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)])
    f = 2.0 / R
    assert np.max(np.abs(alpha - (1 + f) ** -0.5)) < 1e-14
    assert np.max(np.abs(beta_up - l * f / (1 + f))) < 1e-14
    ref = np.eye(3)[:, :, None] - (f / (1 + f))[None, None] * l[:, None] * l[None, :]
    assert np.max(np.abs(gamma_inv - ref)) < 1e-14


def test_characteristic_speeds_of_app_a3(golden_dir):
    rows = [l.split() for l in open(os.path.join(golden_dir, "appA3_char_speeds.txt"))
            if l.strip() and not l.startswith("#")]
    for rr, speed, tol in rows:
        rr, speed, tol = float(rr), float(speed), float(tol)
        u = inputs.kerr_schild_state(3, 2, 4, rr, rr + 1.0, amp=0.0)[:, :, :, 0].reshape(50, -1)
        g, _, _ = ghg.split_state(u)
        alpha, beta_up, gamma_inv, _, _, _ = ghg.three_plus_one(g)
        _, t, p = oracle.cff.grid(3, 2, 4, rr, rr + 1.0)
        T = (t[None, :] * np.ones((4, 1))).ravel()
        P = (p[:, None] * np.ones((1, 2))).ravel()
        l = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)])
        s = l / np.sqrt(np.einsum("ijP,iP,jP->P", gamma_inv, l, l))
        b = np.einsum("iP,iP->P", s, beta_up)
        assert np.max(np.abs((-alpha - b) - speed)) <= tol


def test_principal_part_matches_printed_characteristic_matrix():
    # App. A.2: s_k A^k = [[0,0,0],[b,-b,alpha s^i],[-alpha s_i, alpha s_i, -b]]
    # acting on (g, Pi, Phi_i); the rhs is -A^k d_k u + S, linear in d_k u.
    rng = np.random.default_rng(4)
    P = 7
    u = inputs.kerr_schild_state(3, 2, 4, 2.5, 6.0, amp=0.0).reshape(50, -1)[:, :P].copy()
    u += 0.05 * rng.standard_normal(u.shape) * (np.arange(50) >= 10)[:, None]
    H = rng.standard_normal((4, P))
    dH = rng.standard_normal((3, 4, P))
    g, _, _ = ghg.split_state(u)
    alpha, beta_up, gamma_inv, _, _, _ = ghg.three_plus_one(g)
    s_lo = rng.standard_normal((3, P))
    s_lo /= np.sqrt(np.einsum("ijP,iP,jP->P", gamma_inv, s_lo, s_lo))
    s_up = np.einsum("ijP,jP->iP", gamma_inv, s_lo)
    b = np.einsum("iP,iP->P", s_lo, beta_up)
    v = rng.standard_normal((50, P))
    du = s_lo[:, None, :] * v[None]                      # d_k u = s_k v
    lin = (ghg.rhs_pointwise(u, du, H, dH) - ghg.rhs_pointwise(u, 0 * du, H, dH))
    vg, vPi = v[0:10], v[10:20]
    vPhi = np.stack([v[20 + 10 * i:30 + 10 * i] for i in range(3)])
    exp_g = 0 * vg
    exp_Pi = -(b * vg - b * vPi + alpha * np.einsum("iP,isP->sP", s_up, vPhi))
    exp_Phi = -(-alpha * s_lo[:, None] * vg[None] + alpha * s_lo[:, None] * vPi[None]
                - b * vPhi)
    assert np.max(np.abs(lin[0:10] - exp_g)) < 1e-13
    assert np.max(np.abs(lin[10:20] - exp_Pi)) < 1e-12
    for i in range(3):
        assert np.max(np.abs(lin[20 + 10 * i:30 + 10 * i] - exp_Phi[i])) < 1e-12


def test_outer_bc_freezes_incoming_and_keeps_outgoing():
    rng = np.random.default_rng(7)
    n_r, N, J = 4, 6, 12
    u = inputs.kerr_schild_state(n_r, N, J, 1.8, 11.0, amp=1e-3, seed=1)
    sh = oracle.OracleShell(n_r, N, J, 1.8, 11.0, 4)
    rhs = rng.standard_normal(u.shape)
    B1 = ghg.apply_outer_bc(rhs, u, sh.theta, sh.phi)
    B2 = ghg.apply_outer_bc(B1, u, sh.theta, sh.phi)
    assert np.max(np.abs(B2 - B1)) < 1e-13                         # projection
    assert np.array_equal(B1[:, :, :, :-1], rhs[:, :, :, :-1])    # interior untouched
    uo = u[:, :, :, -1].reshape(50, -1)
    g, _, _ = ghg.split_state(uo)
    gi = ghg.inv_batched(g[1:, 1:])
    T = (sh.theta[None, :] * np.ones((J, 1))).ravel()
    P = (sh.phi[:, None] * np.ones((1, N))).ravel()
    l = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)])
    s = l / np.sqrt(np.einsum("ijP,iP,jP->P", gi, l, l))
    su = np.einsum("ijP,jP->iP", gi, s)

    def chars(x):
        x = x[:, :, :, -1].reshape(50, -1)
        dg, dPi = x[0:10], x[10:20]
        dPhi = np.stack([x[20 + 10 * i:30 + 10 * i] for i in range(3)])
        sP = np.einsum("iP,isP->sP", su, dPhi)
        tang = dPhi - s[:, None] * sP[None]
        return dg, -dg + dPi + sP, -dg + dPi - sP, tang

    g0, up0, _, _ = chars(rhs)
    g1, up1, um1, tg1 = chars(B1)
    assert np.max(np.abs(g1 - g0)) < 1e-14 and np.max(np.abs(up1 - up0)) < 1e-12
    assert np.max(np.abs(um1)) < 1e-12 and np.max(np.abs(tg1)) < 1e-12


def test_gauge_init_zeroes_gauge_constraint():
    u = inputs.kerr_schild_state(7, 8, 16, 1.8, 11.0, amp=1e-4, seed=2)
    sh = oracle.OracleShell(7, 8, 16, 1.8, 11.0, 6)
    sh.init_gauge_from_state(u)
    _, ca = sh.constraint_norms(u)
    assert ca < 1e-15


def test_exact_kerr_schild_rhs_converges_spectrally():
    # Sec. 4.1 / Fig. r10_rconv: R10 shell, 9 x 18 angular grid, n_r = 13..37;
    # exponential convergence towards the round-off floor
    errs = []
    for n_r in (13, 19, 25, 31, 37):
        u = inputs.kerr_schild_state(n_r, 9, 18, 1.8, 11.8, amp=0.0)
        sh = oracle.OracleShell(n_r, 9, 18, 1.8, 11.8, 7)
        sh.init_gauge_from_state(u)
        errs.append(np.max(np.abs(sh.rhs(u))))
    for a, b in zip(errs, errs[1:]):
        assert b < a / 20.0
    assert errs[-1] < 1e-9


def test_rk4_amplification_polynomial(monkeypatch):
    sh = oracle.OracleShell(3, 2, 4, 1.0, 2.0, 1)
    lam = -0.7 + 0.3j
    monkeypatch.setattr(sh, "stage", lambda u: lam * u)
    u0 = np.ones((1, 4, 2, 3), dtype=complex)
    dt = 0.37
    z = lam * dt
    # run the RK4 combination with complex state directly
    k1 = sh.stage(u0); k2 = sh.stage(u0 + 0.5 * dt * k1)
    k3 = sh.stage(u0 + 0.5 * dt * k2); k4 = sh.stage(u0 + dt * k3)
    ref = u0 + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    assert np.max(np.abs(ref - (1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24))) < 1e-15
    # and the oracle's own step on a real decay
    monkeypatch.setattr(sh, "stage", lambda u: -0.7 * u)
    got = sh.rk4_step(np.ones((1, 4, 2, 3)), dt)
    zr = -0.7 * dt
    assert np.max(np.abs(got - (1 + zr + zr ** 2 / 2 + zr ** 3 / 6 + zr ** 4 / 24))) < 1e-15
