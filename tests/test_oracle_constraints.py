"""Pins of the oracle's constraint quantities and of the constraint-damping
terms of its GHG right-hand side (paper App. A.1).  CPU only.

* Gamma_a of exact Kerr-Schild data against its closed form: with det g = -1,
  Gamma^c = -box x^c = -d_a g^ac, which for g^ab = eta^ab - f l^a l^b gives
  Gamma_a = (2M / r^2) l_a, l_a = (1, x_i / r).
* The constraint norms on data with a known, non-zero violation: C_iab = -c
  on one of the 30 stored components, C_a = h (RMS over points and
  components, unweighted).
* The gamma_2 terms of eqs. Phidot and Pidot are multiples of the constraint
  C_iab = d_i g_ab - Phi_iab (the paper introduces gamma_2 as its
  coefficient): with C_iab = 0 the right-hand side does not depend on
  gamma_2.  The size of the d_i g_ab parts is fixed by the printed
  characteristic matrix of App. A.2 (tests/test_oracle_ghg.py).
* Spatially constant perturbations of flat space: every term but the damping
  terms is quadratic in the perturbation, so at linear order
  C_iab(t) = C_iab(0) exp(-gamma_2 t) and, for the gauge constraint with
  H_a = 0, C_t(t) = C_t(0) exp(-2 gamma_0 t), C_i(t) = C_i(0) exp(-gamma_0 t)
  (Gamma_t = (Pi_tt + Pi_xx + Pi_yy + Pi_zz) / 2 and Gamma_i = Pi_ti at
  g = eta, Phi = 0; the gamma_0 term adds -gamma_0 C_t to Pi_tt and to each
  Pi_ii and -gamma_0 C_i to Pi_ti).
"""

import numpy as np

import oracle
from oracle import ghg
from paper_1104_3408_gb300 import inputs

R_IN, R_OUT = 1.8, 11.0


def _exact_du(u):
    """d_i of every field with the closed-form d_i g_ab (the generator's Phi
    fields of unperturbed or perturbed Kerr-Schild data) and zero elsewhere."""
    du = np.zeros((3,) + u.shape)
    for i in range(3):
        du[i, 0:10] = u[20 + 10 * i:30 + 10 * i]
    return du


def _kerr_schild_gamma(n_r, N, J, mass=1.0):
    r, t, p = oracle.cff.grid(n_r, N, J, R_IN, R_OUT)
    R = (r[None, None, :] * np.ones((J, N, 1))).ravel()
    T = (t[None, :, None] * np.ones((J, 1, n_r))).ravel()
    P = (p[:, None, None] * np.ones((1, N, n_r))).ravel()
    l = np.stack([np.ones_like(R), np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)])
    return 2.0 * mass / R ** 2 * l


def test_christoffel_contraction_of_kerr_schild_closed_form():
    n_r, N, J = 5, 6, 12
    u = inputs.kerr_schild_state(n_r, N, J, R_IN, R_OUT, amp=0.0).reshape(50, -1)
    g, Pi, Phi = ghg.split_state(u)
    alpha, beta_up, _, _, _, ginv = ghg.three_plus_one(g)
    _, gam_c = ghg.christoffel(g, Pi, Phi, alpha, beta_up, ginv)
    ref = _kerr_schild_gamma(n_r, N, J)
    assert np.max(np.abs(gam_c - ref)) < 1e-14 * np.max(np.abs(ref)) * 50
    # and the gauge source of the state is its negative (eq. gauge)
    H = ghg.gauge_source_from_state(u)
    assert np.max(np.abs(H + ref)) < 1e-13


def test_constraint_norm_of_a_known_phi_violation():
    n_r, N, J = 5, 6, 12
    u = inputs.kerr_schild_state(n_r, N, J, R_IN, R_OUT, amp=1e-3, seed=3).reshape(50, -1)
    du = _exact_du(u)
    H = ghg.gauge_source_from_state(u)
    c3, ca = ghg.constraint_norms(u, du, H)
    assert c3 < 1e-15 and ca < 1e-15
    c = 3.0e-4
    for comp in (20, 31, 45):     # Phi_x tt, Phi_y tx, Phi_z xz: one of 30 components
        v = u.copy()
        v[comp] += c
        c3, _ = ghg.constraint_norms(v, du, H)
        assert abs(c3 - c / np.sqrt(30.0)) < 1e-12 * c
    # a violation varying over the points: RMS = sqrt(mean(c(p)^2) / 30)
    v = u.copy()
    cp = c * np.cos(np.arange(u.shape[1]) * 0.37)
    v[37] -= cp
    c3, _ = ghg.constraint_norms(v, du, H)
    assert abs(c3 - np.sqrt(np.mean(cp ** 2) / 30.0)) < 1e-12 * c


def test_constraint_norm_of_a_known_gauge_violation():
    n_r, N, J = 5, 6, 12
    u = inputs.kerr_schild_state(n_r, N, J, R_IN, R_OUT, amp=0.0).reshape(50, -1)
    du = _exact_du(u)
    P = u.shape[1]
    h = np.zeros((4, P))
    h[0] = 2.0e-5
    _, ca = ghg.constraint_norms(u, du, -_kerr_schild_gamma(n_r, N, J) + h)
    assert abs(ca - 2.0e-5 / 2.0) < 1e-10 * 2.0e-5
    h = 1e-5 * np.stack([np.sin(np.arange(P) * (0.1 + 0.2 * a)) for a in range(4)])
    _, ca = ghg.constraint_norms(u, du, -_kerr_schild_gamma(n_r, N, J) + h)
    assert abs(ca - np.sqrt(np.mean(h ** 2))) < 1e-9 * 1e-5


def test_gamma2_terms_vanish_with_the_constraint():
    rng = np.random.default_rng(11)
    n_r, N, J = 4, 4, 8
    u = inputs.kerr_schild_state(n_r, N, J, R_IN, R_OUT, amp=5e-3, ell=2, seed=5).reshape(50, -1)
    P = u.shape[1]
    u[10:20] += 0.05 * rng.standard_normal((10, P))          # Pi off the static solution
    du = 0.1 * rng.standard_normal((3, 50, P))
    for i in range(3):
        du[i, 0:10] = u[20 + 10 * i:30 + 10 * i]            # C_iab = 0
    H = rng.standard_normal((4, P))
    dH = rng.standard_normal((3, 4, P))
    r1 = ghg.rhs_pointwise(u, du, H, dH)
    scale = np.max(np.abs(r1))
    for g2 in (0.0, 2.5):
        r2 = ghg.rhs_pointwise(u, du, H, dH, gamma2=g2)
        assert np.max(np.abs(r2 - r1)) < 1e-14 * scale
    # negative control: with C_iab != 0 the gamma2 terms are there
    du[0, 4] += 1e-2
    assert np.max(np.abs(ghg.rhs_pointwise(u, du, H, dH, gamma2=0.0)
                         - ghg.rhs_pointwise(u, du, H, dH))) > 1e-4


def _flat_state(rng, eps_pi, eps_phi, P=3):
    u = np.zeros((50, P))
    u[0] = -1.0          # g_tt
    u[4] = u[7] = u[9] = 1.0   # g_xx, g_yy, g_zz
    u[10:20] = eps_pi * rng.standard_normal((10, P))
    u[20:50] = eps_phi * rng.standard_normal((30, P))
    return u


def _integrate(u, t_end, n, gamma0=1.0, gamma2=1.0):
    """Classical RK4 of the spatially constant system du/dt = S(u) (no
    derivatives, H_a = 0)."""
    P = u.shape[1]
    zero_du, H, dH = np.zeros((3, 50, P)), np.zeros((4, P)), np.zeros((3, 4, P))

    def f(v):
        return ghg.rhs_pointwise(v, zero_du, H, dH, gamma0=gamma0, gamma2=gamma2)

    dt = t_end / n
    for _ in range(n):
        k1 = f(u)
        k2 = f(u + 0.5 * dt * k1)
        k3 = f(u + 0.5 * dt * k2)
        k4 = f(u + dt * k3)
        u = u + dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    return u


def _gauge_constraint(u):
    g, Pi, Phi = ghg.split_state(u)
    alpha, beta_up, _, _, _, ginv = ghg.three_plus_one(g)
    return ghg.christoffel(g, Pi, Phi, alpha, beta_up, ginv)[1]   # H = 0: C_a = Gamma_a


def test_gauge_constraint_damping_rates_on_flat_space():
    rng = np.random.default_rng(2)
    eps, T = 1e-7, 1.2
    for gamma0 in (1.0, 0.5):
        u0 = _flat_state(rng, eps, 0.0)
        c0 = _gauge_constraint(u0)
        c1 = _gauge_constraint(_integrate(u0, T, 240, gamma0=gamma0))
        rate = np.array([2.0, 1.0, 1.0, 1.0]) * gamma0
        ref = c0 * np.exp(-rate * T)[:, None]
        assert np.max(np.abs(c1 - ref)) < 1e-5 * np.max(np.abs(c0))


def test_derivative_constraint_damping_rate_on_flat_space():
    rng = np.random.default_rng(3)
    eps, T = 1e-7, 1.2
    for gamma2 in (1.0, 0.5):
        u0 = _flat_state(rng, 0.0, eps)
        c0 = -u0[20:50]                       # C_iab = d_i g_ab - Phi_iab, d_i g = 0
        u1 = _integrate(u0, T, 240, gamma2=gamma2)
        c1 = -u1[20:50]
        # (Pi picks up O(eps) terms through the gauge constraint, which Phi
        # enters linearly, but Pi enters d_t Phi only quadratically)
        assert np.max(np.abs(c1 - c0 * np.exp(-gamma2 * T))) < 1e-5 * np.max(np.abs(c0))
