"""CFF collocation grid and pseudospectral derivatives (paper Sec. 2).

Test infrastructure only (see ``oracle/__init__``).

Layout of every field array: ``u[mu, j, i, k]`` with ``mu`` the field, ``j`` the
phi index, ``i`` the theta index (single cover) and ``k`` the radial index, so
that the flat index is ``k + n_r*(i + N_theta*(j + N_phi*mu))`` -- the paper's
linear 4-d index of Sec. 2.4 with the single theta cover stored (Sec. 2.1).

Parity pins (tests/test_oracle_cff.py): D_r exact on Chebyshev polynomials of
degree <= n_r-1; FD exact on trigonometric modes below Nyquist; the double
cover theta derivative equals the Kronecker 3-d matrix of eq. D3d on tiny
grids and is exact on parity-consistent modes; the chain rule is exact on
Cartesian polynomials.
"""

import numpy as np


def grid(n_r, n_theta, n_phi, r_in, r_out):
    """Collocation points, Sec. 2.1 eqs. rk, thetai, phij.

    r_k increases with k (Chebyshev extrema plus end points), theta_i staggers
    the poles by half a spacing, phi_j is uniform.
    """
    k = np.arange(n_r)
    r = 0.5 * (r_out + r_in) - 0.5 * (r_out - r_in) * np.cos(np.pi * k / (n_r - 1))
    i = np.arange(n_theta)
    theta = np.pi * (i + 0.5) / n_theta
    j = np.arange(n_phi)
    phi = 2.0 * np.pi * j / n_phi
    return r, theta, phi


def dx_min(r, theta, phi):
    """Smallest grid distance of Sec. 4.1 (text before the Courant factor):
    min(r_1 - r_0, 2 r_0 sin(theta_0) sin(dphi/2))."""
    dphi = phi[1] - phi[0]
    return min(r[1] - r[0], 2.0 * r[0] * np.sin(theta[0]) * np.sin(0.5 * dphi))


def fourier_diff_matrix(n):
    """Fourier differentiation matrix for an even number of equally spaced
    periodic points, Sec. 2.3: FD_ij = (-1)^(i+j) / (2 tan((x_i - x_j)/2)),
    FD_ii = 0, with x_i = 2 pi i / n (any constant offset cancels)."""
    assert n % 2 == 0
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = (-1.0) ** (i + j) / (2.0 * np.tan(np.pi * (i - j) / n))
    return D


def cheb_diff_matrix(n):
    """Chebyshev differentiation matrix on x_i = -cos(pi i/(n-1)), eq. CDhat:
    CD_ij = (c_i/c_j) (-1)^(i+j) / (x_i - x_j), diagonal = minus the row sum."""
    x = -np.cos(np.pi * np.arange(n) / (n - 1))
    c = np.ones(n)
    c[0] = c[-1] = 2.0
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = (c[i] / c[j]) * (-1.0) ** (i + j) / (x[i] - x[j])
        D[i, i] = -np.sum(D[i, :])
    return D


def radial_diff_matrix(n_r, r_in, r_out):
    """Rescaled Chebyshev matrix for [r_in, r_out], Sec. 2.3:
    hat CD = 2 CD / (r_max - r_min)."""
    return 2.0 * cheb_diff_matrix(n_r) / (r_out - r_in)


def d_r(u, Dr):
    """Radial derivative, eq. D1: (d_1 u) = D_1 u with r the leading index."""
    return np.einsum("kl,...l->...k", Dr, u)


def double_cover(u):
    """Extend theta lines to the double cover, Sec. 2.1: the point theta_{N+q}
    at phi_j carries u(theta_{N-1-q}, phi_j + pi), from
    f(theta, phi) = f(2 pi - theta, pi + phi).  Cartesian components are
    scalars on the sphere, so no sign changes.  Returns [mu, j, 2N, k]."""
    n_phi = u.shape[1]
    shifted = np.roll(u, -(n_phi // 2), axis=1)      # shifted[:, j] = u[:, j + N_phi/2]
    return np.concatenate([u, shifted[:, :, ::-1, :]], axis=2)


def d_theta(u):
    """Theta derivative, eq. D2, via the explicit double cover: apply the full
    2N x 2N Fourier matrix to the extended theta line and keep the single
    cover (Sec. 2.1)."""
    N = u.shape[2]
    ext = double_cover(u)
    D2 = fourier_diff_matrix(2 * N)
    return np.einsum("iq,mjqk->mjik", D2, ext)[:, :, :N, :]


def d_phi(u):
    """Phi derivative, eq. D3: D_3 (N_phi x N_phi) along the phi index."""
    D3 = fourier_diff_matrix(u.shape[1])
    return np.einsum("jl,mlik->mjik", D3, u)


def spherical_derivatives(u, r_in, r_out):
    """(d_r u, d_theta u, d_phi u) for all fields."""
    Dr = radial_diff_matrix(u.shape[3], r_in, r_out)
    return d_r(u, Dr), d_theta(u), d_phi(u)


def cartesian_gradient(dr, dth, dph, r, theta, phi):
    """Chain rule of eq. dvdx with the analytic Jacobian d(r,theta,phi)/d(x,y,z):
    d_x = sin t cos p d_r + cos t cos p / r d_t - sin p /(r sin t) d_p
    d_y = sin t sin p d_r + cos t sin p / r d_t + cos p /(r sin t) d_p
    d_z = cos t d_r - sin t / r d_t
    Returns an array [3, ...] (x, y, z)."""
    st = np.sin(theta)[None, None, :, None]
    ct = np.cos(theta)[None, None, :, None]
    sp = np.sin(phi)[None, :, None, None]
    cp = np.cos(phi)[None, :, None, None]
    rr = r[None, None, None, :]
    dx = st * cp * dr + ct * cp / rr * dth - sp / (rr * st) * dph
    dy = st * sp * dr + ct * sp / rr * dth + cp / (rr * st) * dph
    dz = ct * dr - st / rr * dth
    return np.stack([dx, dy, dz])


def cartesian_derivatives(u, r_in, r_out):
    """All three Cartesian derivatives of every field: [3, mu, j, i, k]."""
    n_r, N, n_phi = u.shape[3], u.shape[2], u.shape[1]
    r, theta, phi = grid(n_r, N, n_phi, r_in, r_out)
    dr, dth, dph = spherical_derivatives(u, r_in, r_out)
    return cartesian_gradient(dr, dth, dph, r, theta, phi)


def kron_theta_matrix(n_r, n_theta, n_phi):
    """Brute-force 3-d theta derivative of eq. D3d on the double-covered grid
    (n1 = N_r, n2 = 2 N_theta, n3 = N_phi) for the flat index
    p = k + n1 (i + n2 j): I_3 (x) D_2 (x) I_1.  For tiny-grid tests only."""
    return np.kron(np.eye(n_phi), np.kron(fourier_diff_matrix(2 * n_theta), np.eye(n_r)))
