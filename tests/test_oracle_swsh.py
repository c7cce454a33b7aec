"""Pins of the oracle's spin-weighted harmonics, pseudo-inverse, filter matrices
and real DFT (paper Secs. 3.1-3.3, 3.5, App. B).  CPU only."""

import math
import os

import numpy as np
import pytest

from oracle import dft, swsh


def _read(path):
    rows = []
    with open(path) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split(None, 3) if "appB_spin" in path else line.split())
    return rows


def test_app_b_table(golden_dir):
    rows = _read(os.path.join(golden_dir, "appB_spin_legendre.txt"))
    assert len(rows) == 27
    t = np.pi * (np.arange(17) + 0.5) / 17
    sl = swsh.SpinLegendre(t, 4)
    env = {"pi": math.pi, "sqrt": np.sqrt, "sin": np.sin, "cos": np.cos}
    for n, l, m, expr in rows:
        env["t"] = t
        ref = eval(expr, {}, env) * np.ones_like(t)
        got = sl(int(n), int(l), int(m))
        assert np.max(np.abs(got - ref)) < 1e-14, (n, l, m)


def test_negative_spin_rule_of_app_b():
    t = np.pi * (np.arange(11) + 0.5) / 11
    sl = swsh.SpinLegendre(t, 6)
    for l in range(0, 6):
        for m in range(-l, l + 1):
            assert np.max(np.abs(sl(-1, l, m) + (-1.0) ** m * sl(1, l, -m))) < 1e-14


def _wigner_d(j, mp, m, beta):
    """Explicit factorial sum for d^j_{m'm}(beta) (standard convention)."""
    tot = np.zeros_like(beta)
    f = math.factorial
    pref = math.sqrt(f(j + mp) * f(j - mp) * f(j + m) * f(j - m))
    for s in range(0, 2 * j + 1):
        a, b, c, d = j + m - s, s, mp - m + s, j - mp - s
        if min(a, b, c, d) < 0:
            continue
        tot += ((-1.0) ** (mp - m + s) * pref / (f(a) * f(b) * f(c) * f(d))
                * np.cos(beta / 2) ** (2 * j + m - mp - 2 * s) * np.sin(beta / 2) ** (mp - m + 2 * s))
    return tot


def test_recursion_matches_wigner_d_brute_force():
    # P^n_lm = (-1)^n sqrt((2l+1)/4pi) d^l_{m,-n}  (Sec. 3.3).  The recursion
    # of eq. Yninc divides by sin(theta) |n| times, so next to the poles its
    # round-off grows like eps / sin^|n|(theta_0): tolerance 1e-11.
    t = np.pi * (np.arange(23) + 0.5) / 23
    sl = swsh.SpinLegendre(t, 8)
    for n in range(-3, 4):
        for l in range(0, 9):
            for m in range(-l, l + 1):
                if l < abs(n):
                    assert np.all(sl(n, l, m) == 0)
                    continue
                ref = (-1.0) ** n * math.sqrt((2 * l + 1) / (4 * math.pi)) * _wigner_d(l, m, -n, t)
                assert np.max(np.abs(sl(n, l, m) - ref)) < 1e-11, (n, l, m)


def _gl_theta(nq=200):
    x, w = np.polynomial.legendre.leggauss(nq)
    th = 0.5 * np.pi * (x + 1.0)
    return th, 0.5 * np.pi * w


def test_app_b_inner_products(golden_dir):
    rows = _read(os.path.join(golden_dir, "appB_inner_products.txt"))
    th, w = _gl_theta()
    sl = swsh.SpinLegendre(th, 4)
    for n1, l1, m1, n2, l2, m2, expr in rows:
        n1, l1, m1, n2, l2, m2 = map(int, (n1, l1, m1, n2, l2, m2))
        assert m1 == m2
        val = 2 * np.pi * np.sum(w * np.sin(th) * sl(n1, l1, m1) * sl(n2, l2, m2))
        ref = eval(expr, {}, {"pi": math.pi, "sqrt": math.sqrt})
        assert val == pytest.approx(ref, abs=1e-13)


def test_orthonormality_by_quadrature():
    th, w = _gl_theta()
    sl = swsh.SpinLegendre(th, 12)
    for n in (-3, -1, 0, 2, 3):
        for m in (-4, 0, 5):
            ls = [l for l in range(max(abs(n), abs(m)), 13)]
            G = np.array([[2 * np.pi * np.sum(w * np.sin(th) * sl(n, a, m) * sl(n, b, m))
                           for b in ls] for a in ls])
            assert np.max(np.abs(G - np.eye(len(ls)))) < 1e-12


def test_mx_expansion_of_app_b():
    # m_x = (cos t cos p - i sin p)/sqrt 2 = sqrt(2 pi/3) (Y^1_{1,1} - Y^1_{1,-1})
    rng = np.random.default_rng(0)
    t = rng.uniform(0.05, 3.1, 40)
    p = rng.uniform(0, 2 * np.pi, 40)
    sl = swsh.SpinLegendre(t, 2)
    lhs = (np.cos(t) * np.cos(p) - 1j * np.sin(p)) / np.sqrt(2)
    rhs = np.sqrt(2 * np.pi / 3) * (sl(1, 1, 1) * np.exp(1j * p) - sl(1, 1, -1) * np.exp(-1j * p))
    assert np.max(np.abs(lhs - rhs)) < 1e-15


def test_pseudo_inverse_penrose_identities():
    N = 16
    t = np.pi * (np.arange(N) + 0.5) / N
    sl = swsh.SpinLegendre(t, N - 1)
    for n in (-3, 0, 2):
        for m in (0, 3, 9, -7):
            A, _ = swsh.synthesis_matrix(sl, n, m, N)
            Ap = swsh.pinv_svd(A)
            s = np.max(np.abs(A))
            assert np.max(np.abs(A @ Ap @ A - A)) < 1e-12 * s
            assert np.max(np.abs(Ap @ A @ Ap - Ap)) < 1e-12 * np.max(np.abs(Ap))
            assert np.max(np.abs((A @ Ap).T - A @ Ap)) < 1e-12
            assert np.max(np.abs(Ap @ A - np.eye(A.shape[1]))) < 1e-11   # full column rank


@pytest.mark.parametrize("N", [9, 12, 48, 96])
def test_synthesis_matrices_have_full_column_rank_and_small_condition(N):
    # eq. forwardL solves with P^n_m after its zero columns (l < |n|) are
    # dropped; on the pole-staggered grids of the benchmark shells every such
    # matrix has full column rank, with condition numbers below 2 sqrt(N)
    # (2.9 at N = 9, 9.1 at N = 96, largest for n = m = 0)
    t = np.pi * (np.arange(N) + 0.5) / N
    sl = swsh.SpinLegendre(t, N - 1)
    worst = 0.0
    for n in range(-3, 4):
        for m in range(-(N - 1), N):
            c = swsh.synthesis_condition(sl, n, m, N)
            A, _ = swsh.synthesis_matrix(sl, n, m, N)
            if A.shape[1]:
                ev = np.linalg.eigvalsh(A.T @ A)
                assert abs(c - math.sqrt(ev[-1] / ev[0])) < 1e-6 * c
            worst = max(worst, c)
    assert 1.0 < worst < 2.0 * math.sqrt(N)


def test_filter_matrix_projection_properties():
    N = 14
    L = 9
    t = np.pi * (np.arange(N) + 0.5) / N
    sl = swsh.SpinLegendre(t, N - 1)
    for n in range(-3, 4):
        for m in (-6, -1, 0, 1, 4, 9, 12):
            F = swsh.filter_matrix(sl, n, m, N, L)
            assert np.max(np.abs(F @ F - F)) < 1e-11
            for l in range(max(abs(n), abs(m)), N):
                y = sl(n, l, m)
                err = np.max(np.abs(F @ y - (y if l <= L else 0 * y)))
                assert err < 1e-11 * np.max(np.abs(y)), (n, m, l)
            # conjugation symmetry used by a real tensor: F^n_{-m} = F^{-n}_m
            G = swsh.filter_matrix(sl, -n, -m, N, L)
            assert np.max(np.abs(F - G)) < 1e-11


def test_real_dft_matrices():
    for J in (8, 24, 96):
        A, B, At, Bt = dft.real_dft_matrices(J)
        M = J // 2
        assert np.max(np.abs(At @ A - np.eye(M))) < 1e-13
        assert np.max(np.abs(Bt @ B - np.eye(M - 1))) < 1e-13
        assert np.max(np.abs(At @ B)) < 1e-13 and np.max(np.abs(Bt @ A)) < 1e-13
        phi = 2 * np.pi * np.arange(J) / J
        f = 0.3 + 2.0 * np.cos(3 * phi) - 1.5 * np.sin((M - 1) * phi)
        a, b = At @ f, Bt @ f
        assert a[0] == pytest.approx(0.3) and a[3] == pytest.approx(2.0)
        assert b[M - 2] == pytest.approx(-1.5)
        assert np.max(np.abs(A @ a + B @ b - f)) < 1e-13
