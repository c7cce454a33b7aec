"""Pins of the oracle's grid and derivative operators (paper Sec. 2) against
closed forms and brute force.  CPU only."""

import numpy as np
import numpy.polynomial.chebyshev as C
import pytest

from oracle import cff


def test_grid_closed_form():
    r, t, p = cff.grid(9, 12, 24, 1.8, 11.0)
    assert r[0] == pytest.approx(1.8, abs=1e-15) and r[-1] == pytest.approx(11.0, abs=1e-14)
    assert np.all(np.diff(r) > 0)
    assert t[0] == pytest.approx(np.pi / 24) and t[-1] == pytest.approx(np.pi - np.pi / 24)
    assert p[12] == pytest.approx(np.pi)


def test_cheb_matrix_explicit_corner_and_row_sums():
    # textbook explicit corner value (descending nodes give +(2N^2+1)/6; the
    # paper's nodes x_i = -cos(pi i/(n-1)) ascend, so the sign flips)
    for n in (5, 9, 17, 33):
        D = cff.cheb_diff_matrix(n)
        N = n - 1
        assert D[0, 0] == pytest.approx(-(2 * N * N + 1) / 6.0, rel=1e-12)
        assert D[-1, -1] == pytest.approx((2 * N * N + 1) / 6.0, rel=1e-12)
        assert np.max(np.abs(D.sum(axis=1))) < 1e-12 * np.max(np.abs(D))


@pytest.mark.parametrize("n_r", [9, 17, 33])
def test_radial_matrix_exact_on_chebyshev_polynomials(n_r):
    r_in, r_out = 1.8, 11.0
    Dr = cff.radial_diff_matrix(n_r, r_in, r_out)
    r, _, _ = cff.grid(n_r, 2, 4, r_in, r_out)
    x = (2 * r - r_in - r_out) / (r_out - r_in)
    for q in range(n_r):
        c = np.zeros(q + 1)
        c[q] = 1.0
        f = C.chebval(x, c)
        df = C.chebval(x, C.chebder(c)) * 2.0 / (r_out - r_in)
        scale = max(1.0, np.max(np.abs(df)))
        assert np.max(np.abs(Dr @ f - df)) < 2e-12 * scale * n_r


@pytest.mark.parametrize("n", [8, 24, 96])
def test_fourier_matrix_exact_on_modes(n):
    D = cff.fourier_diff_matrix(n)
    x = 2 * np.pi * np.arange(n) / n
    for m in range(n // 2):
        assert np.max(np.abs(D @ np.sin(m * x) - m * np.cos(m * x))) < 1e-12 * n
        assert np.max(np.abs(D @ np.cos(m * x) + m * np.sin(m * x))) < 1e-12 * n
    assert np.max(np.abs(D @ np.cos(n // 2 * x))) < 1e-12 * n       # Nyquist annihilated
    assert np.max(np.abs(D @ np.ones(n))) < 1e-13 * n


def test_theta_derivative_equals_kronecker_brute_force():
    rng = np.random.default_rng(1)
    n_r, N, J = 3, 4, 8
    u = rng.standard_normal((2, J, N, n_r))
    ext = cff.double_cover(u)                               # [mu, j, 2N, k]
    D3 = cff.kron_theta_matrix(n_r, N, J)
    for mu in range(2):
        flat = ext[mu].reshape(-1)                          # p = k + n1 (i + n2 j)
        ref = (D3 @ flat).reshape(J, 2 * N, n_r)[:, :N, :]
        assert np.max(np.abs(cff.d_theta(u)[mu] - ref)) < 1e-13


@pytest.mark.parametrize("N", [6, 12, 13])
def test_theta_derivative_exact_on_parity_consistent_modes(N):
    J = 2 * N
    n_r = 2
    _, t, p = cff.grid(n_r, N, J, 1.0, 2.0)
    T = t[None, :, None] * np.ones((J, 1, n_r))
    P = p[:, None, None] * np.ones((1, N, n_r))
    for q in range(N):
        for m in range(0, 4):
            if m % 2 == 0:
                f, df = np.cos(q * T) * np.cos(m * P), -q * np.sin(q * T) * np.cos(m * P)
            else:
                f, df = np.sin(q * T) * np.cos(m * P), q * np.cos(q * T) * np.cos(m * P)
            got = cff.d_theta(f[None])[0]
            assert np.max(np.abs(got - df)) < 1e-11 * max(1, q)


def test_phi_derivative_exact():
    N, J = 6, 12
    _, t, p = cff.grid(2, N, J, 1.0, 2.0)
    P = p[:, None, None] * np.ones((1, N, 2))
    for m in range(J // 2):
        f = np.sin(m * P)
        assert np.max(np.abs(cff.d_phi(f[None])[0] - m * np.cos(m * P))) < 1e-12


def test_chain_rule_exact_on_cartesian_polynomials():
    n_r, N, J = 9, 10, 20
    r, t, p = cff.grid(n_r, N, J, 1.8, 11.0)
    R = r[None, None, :]
    T = t[None, :, None]
    P = p[:, None, None]
    x = R * np.sin(T) * np.cos(P)
    y = R * np.sin(T) * np.sin(P)
    z = R * np.cos(T) * np.ones_like(P)
    f = x * x * y + 3 * z - x * y * z + 0.5 * z * z
    grad = [2 * x * y - y * z, x * x - x * z, 3 - x * y + z]
    d = cff.cartesian_derivatives(f[None], 1.8, 11.0)[:, 0]
    for i in range(3):
        assert np.max(np.abs(d[i] - grad[i])) < 1e-10 * np.max(np.abs(grad[i])) * 10
