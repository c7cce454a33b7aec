"""Pins of the oracle's Yn tensor filter (paper Secs. 3.4, 3.5, App. B).
CPU only."""

import itertools

import numpy as np
import pytest

import oracle
from oracle import cff, ynfilter
from paper_1104_3408_gb300 import inputs


@pytest.fixture(scope="module")
def sf_small():
    _, t, p = cff.grid(3, 8, 16, 1.8, 11.0)
    return ynfilter.SpinFilter(t, p, 3)


def test_triad_round_trip_and_orthonormality(sf_small):
    r, m = sf_small.r, sf_small.m
    mb = np.conj(m)
    dot = lambda a, b: np.sum(a * b, axis=0)
    assert np.max(np.abs(dot(r, r) - 1)) < 1e-15
    assert np.max(np.abs(dot(m, mb) - 1)) < 1e-15
    assert np.max(np.abs(dot(m, m))) < 1e-15 and np.max(np.abs(dot(r, m))) < 1e-15
    rng = np.random.default_rng(0)
    v = rng.standard_normal((3,) + r.shape[1:])
    rec = dot(v, r) * r + dot(v, m) * mb + dot(v, mb) * m
    assert np.max(np.abs(rec - v)) < 1e-14


def _constant_tensor(rank, shape, rng):
    T = rng.standard_normal((3,) * rank)
    return T.reshape(T.shape + (1, 1, 1)) * np.ones(shape)


@pytest.mark.parametrize("rank", [0, 1, 2, 3])
def test_constant_cartesian_tensor_preserved_for_L_ge_rank(rank):
    # a constant Cartesian rank-k tensor has triad components of spin |n| <= k
    # and degree l = k only (App. B's m_x is the rank-1 example)
    _, t, p = cff.grid(2, 8, 16, 1.8, 11.0)
    sf = ynfilter.SpinFilter(t, p, rank)
    rng = np.random.default_rng(rank)
    T = _constant_tensor(rank, (16, 8, 2), rng)
    re, im = sf.filter_tensor(T, rank)
    assert np.max(np.abs(re - T)) < 1e-12
    assert np.max(np.abs(im)) < 1e-12
    if rank >= 1:   # one degree less removes it
        sf2 = ynfilter.SpinFilter(t, p, rank - 1)
        re2, _ = sf2.filter_tensor(T, rank)
        assert np.max(np.abs(re2 - T)) > 1e-3


def test_flipped_spin_convention_is_caught(monkeypatch):
    # planted mistake: opposite spin sign (the body text of Sec. 3.4 read
    # literally); a constant vector is then not preserved at L = 1
    _, t, p = cff.grid(2, 8, 16, 1.8, 11.0)
    sf = ynfilter.SpinFilter(t, p, 1)
    orig = sf.filter_function
    monkeypatch.setattr(sf, "filter_function", lambda f, n: orig(f, -n))
    T = _constant_tensor(1, (16, 8, 2), np.random.default_rng(5))
    re, _ = sf.filter_tensor(T, 1)
    assert np.max(np.abs(re - T)) > 1e-3


@pytest.mark.parametrize("L", [0, 2, 10])
def test_exact_kerr_schild_preserved(L):
    u = inputs.kerr_schild_state(5, 12, 24, 1.8, 11.0, amp=0.0)
    sh = oracle.OracleShell(5, 12, 24, 1.8, 11.0, L)
    uf, im = ynfilter.filter_state(u, sh.sf, return_imag=True)
    assert np.max(np.abs(uf - u)) < 5e-13 * np.max(np.abs(u))
    assert im < 1e-13


def test_scalar_filter_negative_control():
    # spin-0 filtering of every Cartesian component with L = 2 changes the
    # rank-3 components Phi_ijk of exact Kerr-Schild data (they carry l = 3)
    u = inputs.kerr_schild_state(5, 12, 24, 1.8, 11.0, amp=0.0)
    sh = oracle.OracleShell(5, 12, 24, 1.8, 11.0, 2)
    scal = sh.sf.filter_function(u[20:50].astype(complex), 0).real
    assert np.max(np.abs(scal - u[20:50])) > 1e-4


def test_filter_idempotent_and_symmetric_on_random_state():
    u = inputs.band_limited_fields(4, 8, 16, 1.8, 11.0, seed=3)
    sh = oracle.OracleShell(4, 8, 16, 1.8, 11.0, 5)
    f1, im = ynfilter.filter_state(u, sh.sf, return_imag=True)
    f2 = sh.filter(f1)
    assert np.max(np.abs(f2 - f1)) < 1e-12 * np.max(np.abs(f1))
    assert im < 1e-12 * np.max(np.abs(u))
    assert np.max(np.abs(f1 - u)) > 1e-3      # random data really filtered


def test_full_tuple_expansion_matches_independent_rank2_formula(sf_small):
    # rank-2 reconstruction written out by hand for the (r, m, mbar) basis
    rng = np.random.default_rng(2)
    T = rng.standard_normal((3, 3) + (16, 8, 2))
    re, im = sf_small.filter_tensor(T, 2)
    vec = {"r": sf_small.r, "m": sf_small.m, "mb": np.conj(sf_small.m)}
    dual = {"r": sf_small.r, "m": np.conj(sf_small.m), "mb": sf_small.m}
    spin = {"r": 0, "m": 1, "mb": -1}
    ref = np.zeros(T.shape, complex)
    for a, b in itertools.product(vec, vec):
        comp = np.einsum("ij...,i...,j...->...", T, vec[a][..., None], vec[b][..., None])
        fc = sf_small.filter_function(comp[None], spin[a] + spin[b])[0]
        ref += np.einsum("i...,j...->ij...", dual[a][..., None], dual[b][..., None]) * fc
    assert np.max(np.abs(re - ref.real)) < 1e-13
