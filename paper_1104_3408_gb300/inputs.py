"""Seeded synthetic inputs shaped like the paper's single black hole runs.

This module is the only code shared by the CUDA path's tests/benchmarks and
the CPU oracle.  It holds none of the method's arithmetic (no differentiation
matrices, no transforms, no filter, no GHG right-hand side): it only samples
closed-form functions at the collocation points.

Recipes
-------
``kerr_schild_state``
    Schwarzschild in Kerr-Schild form, paper App. A.3 eq. KSmetric:
    g_ab = eta_ab + f l_a l_b, f = 2M/r, l_a = (1, x_i/r), plus a seeded
    perturbation dg_ab = A exp(-((r-r_c)/w)^2) Q_ab(x), r_c = (r_in+r_out)/2,
    w = (r_out-r_in)/8, Q_ab a polynomial of total degree <= ell in x/r_c
    (so only spherical-harmonic degrees l <= ell on every sphere), with
    coefficients N(0,1)/sqrt(#monomials) drawn from PCG64(seed), symmetric
    in ab.  Phi_iab = d_i g_ab in closed form (product rule); Pi_ab from its
    definition (eq. defPiPhi) with d_t g_ab = 0: Pi_ab = beta^k Phi_kab / alpha.
    For 54/58 fields the extra gauge fields are left zero (a gauge
    initialisation fills H_a).
``band_limited_fields``
    Random smooth fields for the operator micro-benchmark: per field a sum of
    six von-Mises bumps exp(kappa (n.e - 1)) on the sphere (kappa ~ U[1, 6],
    random centre e) times a Chebyshev series in r with N(0,1) coefficients
    scaled by 10^(-q/4).  Cartesian components of such fields carry every
    spin weight; their angular spectra decay exponentially.
``kerr_schild_pi_from_phi``
    Pi_ab of unperturbed Kerr-Schild data from a given Phi_iab (the paper's
    R10 runs take Phi as the numerical derivative of g_ab), with the
    closed-form lapse and shift of App. A.3.
``shell_batch``
    The uneven-shell batch: n_theta from {16, 24, 32, 48}, n_phi = 2 n_theta,
    n_r from {17, 25, 33}, amplitude log-uniform in [1e-6, 1e-3].
"""

import itertools

import numpy as np

SYM_PAIRS = [(0, 0), (0, 1), (0, 2), (0, 3), (1, 1), (1, 2), (1, 3), (2, 2), (2, 3), (3, 3)]


def collocation_points(n_r, n_theta, n_phi, r_in, r_out):
    """Sampling points of the shell grid (paper Sec. 2.1, eqs. rk, thetai,
    phij): Chebyshev extrema in r (increasing), pole-staggered theta,
    uniform phi."""
    k = np.arange(n_r)
    r = 0.5 * (r_out + r_in) - 0.5 * (r_out - r_in) * np.cos(np.pi * k / (n_r - 1))
    theta = np.pi * (np.arange(n_theta) + 0.5) / n_theta
    phi = 2.0 * np.pi * np.arange(n_phi) / n_phi
    return r, theta, phi


def _cartesian(n_r, n_theta, n_phi, r_in, r_out):
    r, theta, phi = collocation_points(n_r, n_theta, n_phi, r_in, r_out)
    R = r[None, None, :]
    T = theta[None, :, None]
    P = phi[:, None, None]
    x = R * np.sin(T) * np.cos(P)
    y = R * np.sin(T) * np.sin(P)
    z = R * np.cos(T) * np.ones_like(P)
    R = R * np.ones_like(x)
    return np.stack([x, y, z]), R


def kerr_schild_state(n_r, n_theta, n_phi, r_in=1.8, r_out=11.0, n_fields=50,
                      amp=0.0, ell=2, seed=0, mass=1.0, center=None, width=None):
    """Perturbed Kerr-Schild GHG state u[n_fields, n_phi, n_theta, n_r].
    center / width (default: the shell's mid radius and an eighth of its
    thickness) place the Gaussian of the perturbation, so that shells that
    share a sphere can sample one perturbation."""
    X, R = _cartesian(n_r, n_theta, n_phi, r_in, r_out)
    shp = R.shape
    f = 2.0 * mass / R
    lvec = np.concatenate([np.ones((1,) + shp), X / R[None]])          # l_a
    eta = np.diag([-1.0, 1.0, 1.0, 1.0])
    g = np.empty((4, 4) + shp)
    dg = np.zeros((3, 4, 4) + shp)                                       # d_i g_ab
    df = -2.0 * mass * X / R[None] ** 3                                  # d_i f
    dl = np.zeros((3, 4) + shp)                                          # d_i l_a
    for i in range(3):
        for j in range(3):
            dl[i, j + 1] = ((1.0 if i == j else 0.0) - X[i] * X[j] / R ** 2) / R
    for a in range(4):
        for b in range(4):
            g[a, b] = eta[a, b] + f * lvec[a] * lvec[b]
            for i in range(3):
                dg[i, a, b] = (df[i] * lvec[a] * lvec[b] + f * dl[i, a] * lvec[b]
                               + f * lvec[a] * dl[i, b])
    if amp != 0.0:
        rng = np.random.default_rng(seed)
        rc = 0.5 * (r_in + r_out) if center is None else float(center)
        w = (r_out - r_in) / 8.0 if width is None else float(width)
        G = np.exp(-((R - rc) / w) ** 2)
        dG = -2.0 * (R - rc) / w ** 2 * G
        monos = [a for a in itertools.product(range(ell + 1), repeat=3) if sum(a) <= ell]
        xs = X / rc
        for (a, b) in SYM_PAIRS:
            c = rng.standard_normal(len(monos)) / np.sqrt(len(monos))
            Q = np.zeros(shp)
            dQ = np.zeros((3,) + shp)
            for coef, al in zip(c, monos):
                Q += coef * xs[0] ** al[0] * xs[1] ** al[1] * xs[2] ** al[2]
                for i in range(3):
                    if al[i] == 0:
                        continue
                    e = list(al)
                    e[i] -= 1
                    dQ[i] += coef * al[i] / rc * xs[0] ** e[0] * xs[1] ** e[1] * xs[2] ** e[2]
            dgab = amp * G * Q
            g[a, b] += dgab
            if a != b:
                g[b, a] += dgab
            for i in range(3):
                d = amp * (dG * X[i] / R * Q + G * dQ[i])
                dg[i, a, b] += d
                if a != b:
                    dg[i, b, a] += d
    # Pi_ab = beta^k Phi_kab / alpha (eq. defPiPhi with d_t g = 0)
    gam = np.moveaxis(g[1:, 1:], (0, 1), (-2, -1))
    gam_inv = np.moveaxis(np.linalg.inv(gam), (-2, -1), (0, 1))
    beta_lo = g[0, 1:]
    beta_up = np.einsum("ij...,j...->i...", gam_inv, beta_lo)
    alpha = np.sqrt(np.einsum("i...,i...->...", beta_lo, beta_up) - g[0, 0])
    Pi = np.einsum("k...,kab...->ab...", beta_up, dg) / alpha[None, None]
    u = np.zeros((n_fields,) + shp)
    for s, (a, b) in enumerate(SYM_PAIRS):
        u[s] = g[a, b]
        u[10 + s] = Pi[a, b]
        for i in range(3):
            u[20 + 10 * i + s] = dg[i, a, b]
    return np.ascontiguousarray(u)


def kerr_schild_pi_from_phi(Phi, n_r, n_theta, n_phi, r_in=1.8, r_out=11.0, mass=1.0):
    """Pi_ab = beta^k Phi_kab / alpha for unperturbed Kerr-Schild data
    (eq. defPiPhi with d_t g_ab = 0), with the closed-form lapse
    alpha = (1 + f)^(-1/2) and shift beta^k = f/(1 + f) x^k/r of App. A.3.

    Phi: [3, 10, n_phi, n_theta, n_r] in the symmetric-pair order of
    SYM_PAIRS, any approximation of d_k g_ab (the paper's runs take the
    numerical derivative of eq. KSmetric).  Returns Pi[10, n_phi, n_theta, n_r].
    """
    X, R = _cartesian(n_r, n_theta, n_phi, r_in, r_out)
    f = 2.0 * mass / R
    alpha = 1.0 / np.sqrt(1.0 + f)
    beta = X / R[None] * (f / (1.0 + f))[None]
    return np.ascontiguousarray(np.einsum("k...,kf...->f...", beta, np.asarray(Phi)) / alpha[None])


def band_limited_fields(n_r, n_theta, n_phi, r_in=1.8, r_out=11.0, n_fields=50, seed=0,
                        bumps=6):
    """Random smooth fields u[n_fields, n_phi, n_theta, n_r] (see module doc)."""
    rng = np.random.default_rng(seed)
    X, R = _cartesian(n_r, n_theta, n_phi, r_in, r_out)
    nhat = X / R[None]
    xr = (2.0 * R - r_in - r_out) / (r_out - r_in)
    cheb = [np.ones_like(xr), xr]
    for q in range(2, n_r):
        cheb.append(2.0 * xr * cheb[-1] - cheb[-2])
    u = np.zeros((n_fields,) + R.shape)
    for mu in range(n_fields):
        for _ in range(bumps):
            e = rng.standard_normal(3)
            e /= np.linalg.norm(e)
            kappa = rng.uniform(1.0, 6.0)
            ang = np.exp(kappa * (np.einsum("i,i...->...", e, nhat) - 1.0))
            coef = rng.standard_normal(n_r) * 10.0 ** (-np.arange(n_r) / 4.0)
            rad = sum(c * t for c, t in zip(coef, cheb))
            u[mu] += rng.standard_normal() * ang * rad
    return np.ascontiguousarray(u)


def shell_batch(n_shells=256, seed=0):
    """Descriptors of the uneven-shell batch: list of dicts."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(n_shells):
        nt = int(rng.choice([16, 24, 32, 48]))
        nr = int(rng.choice([17, 25, 33]))
        amp = float(10.0 ** rng.uniform(-6.0, -3.0))
        out.append(dict(n_r=nr, n_theta=nt, n_phi=2 * nt, r_in=1.8, r_out=11.0,
                        L=nt - 2, amp=amp, ell=4, seed=seed * 100003 + s))
    return out


# Named workloads (sizes only; the recipes above generate the data).
WORKLOADS = {
    "ks_9x12x24": dict(n_r=9, n_theta=12, n_phi=24, r_in=1.8, r_out=11.0, L=10,
                       n_fields=50, amp=1e-6, ell=2, seed=0, lam=0.25, steps=10),
    "ops_33x32x64": dict(n_r=33, n_theta=32, n_phi=64, r_in=1.8, r_out=11.0, L=30,
                         n_fields=50, seed=0),
    "ks_33x48x96": dict(n_r=33, n_theta=48, n_phi=96, r_in=1.8, r_out=11.0, L=46,
                        n_fields=50, amp=1e-4, ell=4, seed=0, lam=0.25, steps=1000),
    "ks_65x96x192_58f": dict(n_r=65, n_theta=96, n_phi=192, r_in=1.8, r_out=41.0, L=94,
                             n_fields=58, amp=1e-4, ell=4, seed=0, lam=0.25, steps=200),
    # the uneven-shell batch: shell_batch(n_shells, seed) draws the shells
    "batch_256": dict(n_shells=256, n_fields=50, seed=0, lam=0.25, steps=100),
}
