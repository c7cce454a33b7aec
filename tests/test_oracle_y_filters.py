"""Pins of the oracle's component-wise filters of Sec. 3.5: the scalar
Y filter (every field filtered as a spin-0 function at the retained degree
L) and the graded Yg filter of eq. nfofmu (n_f(mu) = n_f - d(u^mu), so a
field with d spatial indices keeps l <= L + d).  CPU only."""

import numpy as np
import pytest

import oracle
from oracle import ynfilter
from paper_1104_3408_gb300 import inputs

N_R, N_T, N_P = 5, 10, 20


def _nhat():
    _, theta, phi = oracle.cff.grid(N_R, N_T, N_P, 1.8, 11.0)
    t = theta[None, :, None]
    p = phi[:, None, None]
    one = np.ones((N_P, N_T, N_R))
    return [np.sin(t) * np.cos(p) * one, np.sin(t) * np.sin(p) * one, np.cos(t) * one]


def test_spatial_degrees_follow_the_paper():
    # d(g_tt) = 0, d(g_tx) = 1, d(g_xx) = 2 (Sec. 3.5); Phi_ijk has 3
    d = [ynfilter.spatial_degree(mu) for mu in range(58)]
    assert d[0] == 0 and d[1] == 1 and d[4] == 2
    assert d[10] == 0 and d[11] == 1 and d[14] == 2        # Pi_ab like g_ab
    assert d[20] == 1 and d[21] == 2 and d[24] == 3        # Phi_x tt, tx, xx
    assert [d.count(k) for k in range(4)] == [2 + 2, 9 + 6, 21, 18]
    assert d[50:58] == [0, 1, 1, 1, 0, 1, 1, 1]


def _shell(L, kind, nf=50):
    return oracle.OracleShell(N_R, N_T, N_P, 1.8, 11.0, L, n_fields=nf, filter_kind=kind)


def test_y_filter_is_the_yn_filter_on_scalar_components():
    u = inputs.band_limited_fields(N_R, N_T, N_P, 1.8, 11.0, seed=4)
    y = _shell(6, "y").filter(u)
    yn = _shell(6, "yn").filter(u)
    for mu in (0, 10):                      # g_tt, Pi_tt: rank 0 in the tensor filter
        assert np.array_equal(y[mu], yn[mu])
    assert np.abs(y[1] - yn[1]).max() > 1e-6   # a vector component: the filters differ


def _monomials(d, k):
    """A polynomial of degree exactly d in the unit normal (l <= d on each
    sphere), different for each k, times a radial factor."""
    n = _nhat()
    r = oracle.cff.grid(N_R, N_T, N_P, 1.8, 11.0)[0][None, None, :]
    f = (1.0 + 0.1 * k) / r * np.ones_like(n[0])
    for j in range(d):
        f = f * n[(k + j) % 3]
    return f


def test_graded_filter_keeps_l_up_to_L_plus_degree():
    # the paper's example: the projection onto spherically symmetric data
    # (retained degree 0) must keep l = 1 in vector components, l <= 3 in
    # Phi_ijk ...
    u = np.stack([_monomials(ynfilter.spatial_degree(mu), mu) for mu in range(50)])
    yg = _shell(0, "yg").filter(u)
    assert np.abs(yg - u).max() < 1e-12 * np.abs(u).max()
    # ... which the plain Y filter does not: it removes every l >= 1 part
    y = _shell(0, "y").filter(u)
    for mu in range(50):
        if ynfilter.spatial_degree(mu) == 0:
            assert np.abs(y[mu] - u[mu]).max() < 1e-12
        else:
            assert np.abs(y[mu] - u[mu]).max() > 1e-3


def test_graded_filter_removes_degree_L_plus_d_plus_one():
    # one degree more than a field keeps is removed from that field
    u = np.stack([_monomials(ynfilter.spatial_degree(mu) + 2, mu) for mu in range(50)])
    yg = _shell(1, "yg").filter(u)
    for mu in range(50):
        d = ynfilter.spatial_degree(mu)
        # degree d + 2 = L + d + 1: its top spherical-harmonic part is removed,
        # the lower parts (same parity) are kept
        assert np.abs(yg[mu] - u[mu]).max() > 1e-3 * np.abs(u[mu]).max()
        assert np.abs(_shell(2, "yg").filter(u)[mu] - u[mu]).max() < 1e-12 * np.abs(u[mu]).max()


@pytest.mark.parametrize("kind", ["y", "yg"])
@pytest.mark.parametrize("nf", [50, 58])
def test_component_filters_are_idempotent(kind, nf):
    u = inputs.band_limited_fields(N_R, N_T, N_P, 1.8, 11.0, n_fields=nf, seed=6)
    s = _shell(4, kind, nf)
    f1 = s.filter(u)
    assert np.abs(s.filter(f1) - f1).max() < 1e-12 * np.abs(f1).max()
    assert np.abs(f1 - u).max() > 1e-6
