"""Spin-weighted spherical harmonics and projection filter matrices
(paper Secs. 3.2, 3.3, 3.5 and App. B).

Test infrastructure only (see ``oracle/__init__``).

Y^n_lm(theta, phi) = P^n_lm(theta) e^{i m phi} (App. B notation P^n_{l,m}; the
body writes P^n_{ml}, the same function).

* P^0_lm: normalised associated Legendre functions with the Condon-Shortley
  phase (App. B prints P^0_{1,1} < 0), built here by the textbook three-term
  recursion in l from P^m_m; negative m from P^0_{l,-m} = (-1)^m P^0_{lm}.
* n > 0: eq. Yninc with the coefficients of eq. Yncoeffs, applied recursively
  down to n = 0 (Sec. 3.3, last paragraphs).
* n < 0: eq. Ynnegative in the form P^n_lm = (-1)^(n+m) P^{-n}_{l,-m}.
* zero whenever l < max(|m|, |n|).

Synthesis matrix for spin n and azimuthal number m (any sign):
(P^n_m)_ik = P^n_{l m}(theta_i) with columns l = |m| .. N-1 (Sec. 3.3,
L = N-1 of Sec. 3.2); identically zero columns (l < |n|) are dropped before
the pseudo-inverse (reading of Sec. 3.2: they carry no coefficient).

Pseudo-inverse by SVD, A^+ = V S^+ U^T (eq. forwardL and the paragraph after
it), singular values below max(rows, cols) * eps * s_max treated as zero.

Filter matrix, eq. FasPfQ: F^n_m = P^n_m f (P^n_m)^+ with f = diag(1 for
l <= L_keep, 0 above).  ``L_keep`` is the retained maximum degree
(n_f = N - 1 - L_keep in the paper's terms, Sec. 3.5).

Parity pins (tests/test_oracle_swsh.py): every entry of the App. B table at
the grid angles; the App. B inner products by Gauss-Legendre quadrature; the
App. B expansion of m_x; an independent Wigner-d factorial sum for l <= 8;
orthonormality; the Penrose identities; F idempotent, reproducing Y^n_lm for
l <= L and annihilating l > L.
"""

import numpy as np


def assoc_legendre(lmax, m, theta):
    """P^0_{l m}(theta) for l = 0..lmax, m >= 0, normalised so that the Y_lm
    are orthonormal on the sphere (Sec. 3.2), Condon-Shortley phase included.
    Rows l < m are zero.  Returns [lmax+1, len(theta)]."""
    theta = np.asarray(theta, dtype=np.float64)
    x = np.cos(theta)
    s = np.sin(theta)
    out = np.zeros((lmax + 1, theta.size))
    if m > lmax:
        return out
    fac = 1.0
    for k in range(1, m + 1):
        fac *= (2.0 * k - 1.0) / (2.0 * k)
    pmm = (-1.0) ** m * np.sqrt((2.0 * m + 1.0) / (4.0 * np.pi) * fac) * s ** m
    out[m] = pmm
    if m + 1 <= lmax:
        out[m + 1] = x * np.sqrt(2.0 * m + 3.0) * pmm
    for l in range(m + 2, lmax + 1):
        a = np.sqrt((4.0 * l * l - 1.0) / (l * l - m * m))
        b = np.sqrt(((l - 1.0) ** 2 - m * m) / (4.0 * (l - 1.0) ** 2 - 1.0))
        out[l] = a * (x * out[l - 1] - b * out[l - 2])
    return out


class SpinLegendre:
    """Evaluates P^n_{l m}(theta_i) on a fixed set of angles, memoised."""

    def __init__(self, theta, lmax):
        self.theta = np.asarray(theta, dtype=np.float64)
        self.lmax = lmax
        self.cos = np.cos(self.theta)
        self.sin = np.sin(self.theta)
        self._p0 = {}
        self._memo = {}

    def _spin0(self, l, m):
        am = abs(m)
        if am not in self._p0:
            self._p0[am] = assoc_legendre(self.lmax, am, self.theta)
        v = self._p0[am][l]
        return v if m >= 0 else (-1.0) ** am * v

    def __call__(self, n, l, m):
        """P^n_{l m}(theta_i) as an array over i."""
        if l < max(abs(m), abs(n)) or l > self.lmax:
            return np.zeros_like(self.theta)
        key = (n, l, m)
        if key in self._memo:
            return self._memo[key]
        if n == 0:
            v = self._spin0(l, m)
        elif n < 0:
            # eq. Ynnegative: P^n_lm = (-1)^(n+m) P^{-n}_{l,-m}
            v = (-1.0) ** (n + m) * self(-n, l, -m)
        else:
            # eq. Yninc with eq. Yncoeffs
            alpha = np.sqrt((l - n + 1.0) / (l + n))
            beta = (1.0 / l) * np.sqrt((2.0 * l + 1.0) / (2.0 * l - 1.0)
                                       * (l + n - 1.0) * (l * l - m * m) / (l + n))
            v = (alpha * (m / l - self.cos) / self.sin * self(n - 1, l, m)
                 + beta / self.sin * self(n - 1, l - 1, m))
        self._memo[key] = v
        return v


def synthesis_matrix(sl, n, m, N):
    """(P^n_m)_ik = P^n_{l m}(theta_i), columns l = max(|m|, |n|) .. N-1
    (zero columns l < |n| dropped).  Returns (P [N x c], list of l)."""
    ls = [l for l in range(abs(m), N) if l >= abs(n)]
    if not ls:
        return np.zeros((N, 0)), ls
    P = np.stack([sl(n, l, m) for l in ls], axis=1)
    return P, ls


def synthesis_condition(sl, n, m, N):
    """2-norm condition number sigma_max / sigma_min of P^n_m (the synthesis
    matrix of eq. forwardL without its zero columns); inf if rank deficient,
    0 for an empty matrix."""
    P, _ = synthesis_matrix(sl, n, m, N)
    if P.shape[1] == 0:
        return 0.0
    S = np.linalg.svd(P, compute_uv=False)
    return float(S[0] / S[-1]) if S[-1] > 0 else float("inf")


def pinv_svd(A):
    """Moore-Penrose pseudo-inverse by the SVD A = U S V^T: A^+ = V S^+ U^T."""
    if A.shape[1] == 0:
        return np.zeros((0, A.shape[0]))
    U, S, Vt = np.linalg.svd(A, full_matrices=False)
    tol = max(A.shape) * np.finfo(np.float64).eps * S[0]
    Sinv = np.where(S > tol, 1.0 / np.where(S > tol, S, 1.0), 0.0)
    return (Vt.T * Sinv[None, :]) @ U.T


def filter_matrix(sl, n, m, N, L_keep):
    """F^n_m = P^n_m f (P^n_m)^+ (eq. FasPfQ), N x N."""
    P, ls = synthesis_matrix(sl, n, m, N)
    if P.shape[1] == 0:
        return np.zeros((N, N))
    keep = np.array([1.0 if l <= L_keep else 0.0 for l in ls])
    return (P * keep[None, :]) @ pinv_svd(P)


def filter_matrices(theta, L_keep, spins=range(-3, 4)):
    """All F^n_m for the given spins and every m in [-(N-1), N-1].
    Returns dict {(n, m): N x N array}."""
    N = len(theta)
    sl = SpinLegendre(theta, N - 1)
    out = {}
    for n in spins:
        for m in range(-(N - 1), N):
            out[(n, m)] = filter_matrix(sl, n, m, N, L_keep)
    return out
