"""Yn tensor filter (paper Secs. 3.4 and 3.5).

Test infrastructure only (see ``oracle/__init__``).

Triad (eq. tetrad, spatial part): r = (sin t cos p, sin t sin p, cos t),
theta = (cos t cos p, cos t sin p, -sin t), phi = (-sin p, cos p, 0),
m = (theta + i phi)/sqrt(2), mbar = conj(m).

Decomposition (eq. tensorexpansion): a Cartesian rank-k tensor T is contracted
on every index with one of (r, m, mbar); the dual basis reconstructs it,
T = sum_tau T~_tau d_tau1 ... d_tauk with d(r) = r, d(m) = mbar, d(mbar) = m
(m . mbar = 1, m . m = 0).

Spin convention (reading, fixed by App. B where x.m expands in Y^{+1}):
a component with p legs contracted with m and q legs contracted with mbar has
spin n = p - q in the P^n family generated by eq. Yninc.

Filter of one complex spin-n function (Sec. 3.3 last paragraph, Sec. 3.5):
real phi analysis of eq. Fanalysis on real and imaginary parts, complex modes
c_{+m} = (a_m - i b_m)/2, c_{-m} = (a_m + i b_m)/2, c_0 = a_0; projection
c'_m = F^n_m c_m along theta for every m in [-(N-1), N-1] (F^n_m built for the
signed m, so no symmetry of eq. ccFn is assumed here); back to a', b' and real
synthesis.  The full 3^k tuple set is filtered, each tuple on its own; the
reconstructed tensor is real up to round-off (its imaginary part is returned
for the invariant test).

Parity pins (tests/test_oracle_filter.py): triad round trip; constant
Cartesian tensors of rank k preserved for L >= k; exact Kerr-Schild data
preserved; projection idempotent; negative control with the scalar filter.
"""

import itertools

import numpy as np

from . import dft as _dft
from . import swsh as _swsh

SYM_PAIRS = [(0, 0), (0, 1), (0, 2), (0, 3), (1, 1), (1, 2), (1, 3), (2, 2), (2, 3), (3, 3)]


def sym_index(a, b):
    if a > b:
        a, b = b, a
    return SYM_PAIRS.index((a, b))


def triad(theta, phi):
    """Spatial triad vectors on the (phi_j, theta_i) grid: r[3,J,N], m[3,J,N]."""
    t = theta[None, :]
    p = phi[:, None]
    st, ct, sp, cp = np.sin(t), np.cos(t), np.sin(p), np.cos(p)
    one = np.ones_like(st * cp)
    r = np.stack([st * cp, st * sp, ct * one])
    th = np.stack([ct * cp, ct * sp, -st * one])
    ph = np.stack([-sp * one, cp * one, 0.0 * one])
    m = (th + 1j * ph) / np.sqrt(2.0)
    return r, m


class SpinFilter:
    """Holds F^n_m for n in [-3, 3], m in [-(N-1), N-1] and the DFT matrices."""

    def __init__(self, theta, phi, L_keep):
        self.theta, self.phi = theta, phi
        self.N, self.J = len(theta), len(phi)
        self.L_keep = L_keep
        self.F = _swsh.filter_matrices(theta, L_keep)
        self.A, self.B, self.At, self.Bt = _dft.real_dft_matrices(self.J)
        self.r, self.m = triad(theta, phi)

    def filter_function(self, f, n):
        """Filter complex functions f[c, J, N, K] of spin n."""
        M = self.J // 2
        f = np.asarray(f, dtype=complex)
        a = np.einsum("mj,cjik->cmik", self.At, f)          # a_m, m = 0..M-1
        b = np.einsum("mj,cjik->cmik", self.Bt, f)          # b_m, m = 1..M-1
        a2 = np.zeros_like(a)
        b2 = np.zeros_like(b)
        c0 = np.einsum("ip,cpk->cik", self.F[(n, 0)], a[:, 0])
        a2[:, 0] = c0
        for mm in range(1, M):
            cp = 0.5 * (a[:, mm] - 1j * b[:, mm - 1])
            cm = 0.5 * (a[:, mm] + 1j * b[:, mm - 1])
            cp2 = np.einsum("ip,cpk->cik", self.F[(n, mm)], cp)
            cm2 = np.einsum("ip,cpk->cik", self.F[(n, -mm)], cm)
            a2[:, mm] = cp2 + cm2
            b2[:, mm - 1] = 1j * (cp2 - cm2)
        return (np.einsum("jm,cmik->cjik", self.A, a2)
                + np.einsum("jm,cmik->cjik", self.B, b2))

    def filter_tensor(self, T, rank):
        """Yn filter of a real Cartesian rank-k tensor T[3,...,3, J, N, K].
        Returns (real part, imaginary part) of the reconstruction."""
        if rank == 0:
            out = self.filter_function(T[None].astype(complex), 0)[0]
            return out.real, out.imag
        shp = (self.J, self.N, 1)
        vec = {"r": self.r, "m": self.m, "mb": np.conj(self.m)}
        dual = {"r": self.r, "m": np.conj(self.m), "mb": self.m}
        spin = {"r": 0, "m": 1, "mb": -1}
        out = np.zeros(T.shape, dtype=complex)
        for tau in itertools.product(("r", "m", "mb"), repeat=rank):
            comp = T.astype(complex)
            for leg in tau:                       # contract the leading index each time
                c = vec[leg].reshape((3,) + (1,) * (comp.ndim - 4) + shp)
                comp = np.sum(comp * c, axis=0)
            n = sum(spin[leg] for leg in tau)
            comp_f = self.filter_function(comp[None], n)[0]
            basis = np.ones(shp, dtype=complex)
            for leg in tau:                       # outer product of the dual vectors
                basis = basis[None] * dual[leg].reshape((3,) + (1,) * (basis.ndim - 3) + shp)
            # the newest leg is the leading index; transpose to leg order
            basis = np.transpose(basis, list(range(rank))[::-1] + [rank, rank + 1, rank + 2])
            out += basis * comp_f[(None,) * rank]
        return out.real, out.imag


def filter_state(u, sf, n_fields=50, return_imag=False):
    """Yn filter of the whole GHG state (Sec. 3.5, filter procedure): each
    tensor group is decomposed, filtered by spin and recombined.

    Groups: g_tt, Pi_tt (rank 0); g_ti, Pi_ti, Phi_itt (rank 1);
    g_ij, Pi_ij, Phi_itj (rank 2); Phi_ijk (rank 3); for 54/58 fields also
    H_t (rank 0), H_i (rank 1) and likewise dH_t/dt, dH_i/dt."""
    out = np.array(u, copy=True)
    imag_max = 0.0

    def run(T, rank):
        nonlocal imag_max
        re, im = sf.filter_tensor(T, rank)
        imag_max = max(imag_max, float(np.max(np.abs(im))) if im.size else 0.0)
        return re

    for base in (0, 10):  # g_ab and Pi_ab
        T4 = np.empty((4, 4) + u.shape[1:])
        for a in range(4):
            for b in range(4):
                T4[a, b] = u[base + sym_index(a, b)]
        out[base + sym_index(0, 0)] = run(T4[0, 0], 0)
        v = run(T4[0, 1:], 1)
        for i in range(3):
            out[base + sym_index(0, i + 1)] = v[i]
        t = run(T4[1:, 1:], 2)
        for i in range(3):
            for j in range(i, 3):
                out[base + sym_index(i + 1, j + 1)] = t[i, j]
    P = np.empty((3, 4, 4) + u.shape[1:])
    for i in range(3):
        for a in range(4):
            for b in range(4):
                P[i, a, b] = u[20 + 10 * i + sym_index(a, b)]
    v = run(P[:, 0, 0], 1)
    for i in range(3):
        out[20 + 10 * i + sym_index(0, 0)] = v[i]
    t2 = run(P[:, 0, 1:], 2)
    for i in range(3):
        for j in range(3):
            out[20 + 10 * i + sym_index(0, j + 1)] = t2[i, j]
    t3 = run(P[:, 1:, 1:], 3)
    for i in range(3):
        for j in range(3):
            for k in range(j, 3):
                out[20 + 10 * i + sym_index(j + 1, k + 1)] = t3[i, j, k]
    for base in range(50, n_fields, 4):  # H_a, then dH_a/dt
        out[base] = run(u[base], 0)
        v = run(u[base + 1:base + 4], 1)
        out[base + 1:base + 4] = v
    if return_imag:
        return out, imag_max
    return out


def spatial_degree(mu):
    """d(u^mu) of Sec. 3.5: the number of spatial indices of field mu in the
    field order of this project (g_ab 0..9, Pi_ab 10..19, Phi_iab 20..49 with
    i the derivative leg, H_a 50..53, dH_a/dt 54..57; pairs in the order
    tt, tx, ty, tz, xx, xy, xz, yy, yz, zz)."""
    if mu >= 50:
        return 0 if (mu - 50) % 4 == 0 else 1
    s = mu % 10
    pair = SYM_PAIRS[s]
    d = sum(1 for x in pair if x > 0)
    return d + (1 if mu >= 20 else 0)


def filter_state_scalar(u, sfs, n_fields=50, graded=False):
    """The component-wise filters of Sec. 3.5: every field u^mu filtered as a
    scalar (spin 0) function.  Y filter (graded=False): retained degree L for
    every field.  Yg filter (graded=True, eq. nfofmu): n_f(mu) = n_f - d(u^mu)
    top modes zeroed, i.e. retained degree L + d(u^mu) (at most N - 1).
    sfs maps a retained degree to a SpinFilter; sfs[None] is the one of L."""
    out = np.array(u, copy=True)
    base = sfs[None].L_keep
    N = sfs[None].N
    for mu in range(n_fields):
        Lk = min(base + spatial_degree(mu), N - 1) if graded else base
        sf = sfs[Lk] if Lk != base else sfs[None]
        out[mu] = sf.filter_function(u[mu][None].astype(complex), 0)[0].real
    return out
