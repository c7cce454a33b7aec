"""Pins of the oracle's nested shells (oracle/nested.py): the characteristic
coupling on a common sphere against the left eigenvectors printed in App. A.2
(eq. characteristics), its reduction to the freeze-incoming condition and to
the identity, exact Kerr-Schild data, and a perturbation crossing the common
sphere against one shell that contains the same sphere.  CPU only."""

import numpy as np
import pytest

from oracle import ghg, nested
from oracle.evolve import OracleShell
from paper_1104_3408_gb300 import inputs

R0, R1, R2 = 1.8, 6.4, 11.0


def _sphere(n_r=5, N=6, J=12, seed=0):
    rng = np.random.default_rng(seed)
    u = inputs.kerr_schild_state(n_r, N, J, R0, R1, amp=1e-3, ell=2, seed=seed)[..., -1]
    sh = OracleShell(n_r, N, J, R0, R1, 4)
    a = rng.standard_normal(u.shape)
    b = rng.standard_normal(u.shape)
    return u, a, b, sh.theta, sh.phi


def _normal(u, theta, phi):
    st, ct = np.sin(theta)[None, :], np.cos(theta)[None, :]
    sp, cp = np.sin(phi)[:, None], np.cos(phi)[:, None]
    l = np.stack([(st * cp).ravel(), (st * sp).ravel(), (ct * np.ones_like(sp)).ravel()])
    g, _, _ = ghg.split_state(u.reshape(50, -1))
    gi = ghg.inv_batched(g[1:, 1:])
    s_lo = l / np.sqrt(np.einsum("ijP,iP,jP->P", gi, l, l))[None]
    return s_lo, np.einsum("ijP,jP->iP", gi, s_lo)


def _printed_fields(x, s_lo, s_up):
    """The five characteristic fields of every symmetric component with the
    left eigenvector matrix as printed in App. A.2 (rows: speed 0, alpha - b,
    -alpha - b, -b, -b; valid where s_1 != 0)."""
    x = x.reshape(50, -1)
    out = []
    for c in range(10):
        v = np.stack([x[c], x[10 + c], x[20 + c], x[30 + c], x[40 + c]])   # g, Pi, Phi_1..3
        E = np.zeros((5, 5) + v.shape[1:])
        E[0, 0] = 1.0
        E[1, 0], E[1, 1], E[1, 2], E[1, 3], E[1, 4] = -1.0, 1.0, s_up[0], s_up[1], s_up[2]
        E[2, 0], E[2, 1], E[2, 2], E[2, 3], E[2, 4] = -1.0, 1.0, -s_up[0], -s_up[1], -s_up[2]
        E[3, 2], E[3, 4] = -s_lo[2], s_lo[0]
        E[4, 2], E[4, 3] = -s_lo[1], s_lo[0]
        out.append(np.einsum("abP,bP->aP", E, v))
    return np.stack(out)        # [component, field, point]


def test_interface_takes_each_characteristic_field_from_its_upwind_shell():
    u, a, b, theta, phi = _sphere()
    c = nested.interface_rhs(a, b, u, theta, phi)
    s_lo, s_up = _normal(u, theta, phi)
    ok = np.abs(s_lo[0]) > 0.1                # the printed form assumes s_1 != 0
    assert ok.sum() > ok.size // 2
    fa, fb, fc = (_printed_fields(x, s_lo, s_up)[..., ok] for x in (a, b, c))
    assert np.max(np.abs(fc[:, 0:2] - fa[:, 0:2])) < 1e-12     # speeds 0, alpha - b: inner shell
    assert np.max(np.abs(fc[:, 2:5] - fb[:, 2:5])) < 1e-12     # -alpha - b, -b, -b: outer shell


def test_interface_reduces_to_identity_and_to_freeze_incoming():
    u, a, _, theta, phi = _sphere(seed=1)
    assert np.max(np.abs(nested.interface_rhs(a, a, u, theta, phi) - a)) < 1e-12
    # with nothing coming in from outside it is App. A.2's boundary operator
    zero = np.zeros_like(a)
    frozen = ghg.apply_outer_bc(a[..., None], u[..., None], theta, phi)[..., 0]
    assert np.max(np.abs(nested.interface_rhs(a, zero, u, theta, phi) - frozen)) < 1e-12


def test_exact_kerr_schild_on_nested_shells_converges():
    errs = []
    for n_r in (9, 13, 17):
        ns = nested.NestedOracle([n_r, n_r], 6, [R0, R1, R2], 5)
        us = [inputs.kerr_schild_state(n_r, 6, 12, sh.r_in, sh.r_out, amp=0.0) for sh in ns.shells]
        ns.init_gauge_from_state(us)
        rh = ns.rhs(us)
        # the common sphere carries one right-hand side
        assert np.array_equal(rh[0][..., -1], rh[1][..., 0])
        errs.append(max(np.abs(r).max() for r in rh))
    assert errs[1] < errs[0] / 10 and errs[2] < errs[1] / 10


@pytest.mark.slow
def test_perturbation_crossing_the_common_sphere_matches_one_shell():
    # one shell over [R0, R2] with an odd n_r has R1 = (R0 + R2) / 2 as its
    # middle point; two nested shells of m points each share that sphere.
    N, L, lam, T = 6, 4, 1.0, 1.5
    kw = dict(amp=1e-4, ell=2, seed=3, center=5.6, width=0.7)
    diffs = []
    for m in (9, 13):
        one = OracleShell(2 * m - 1, N, 2 * N, R0, R2, L)
        u1 = inputs.kerr_schild_state(2 * m - 1, N, 2 * N, R0, R2, **kw)
        one.init_gauge_from_state(u1)
        two = nested.NestedOracle([m, m], N, [R0, R1, R2], L)
        u2 = [inputs.kerr_schild_state(m, N, 2 * N, sh.r_in, sh.r_out, **kw) for sh in two.shells]
        two.init_gauge_from_state(u2)
        dt = lam * min(one.dx_min(), two.dx_min())
        n = int(round(T / dt))
        u1 = one.rk4_step(one.filter(u1), dt, n)
        u2 = two.rk4_step(two.filter(u2), dt, n)
        mid = u1[..., m - 1]
        moved = np.abs(u1[..., m - 1] - inputs.kerr_schild_state(2 * m - 1, N, 2 * N, R0, R2, **kw)[..., m - 1])
        assert moved.max() > 1e-6          # the pulse has moved through the sphere
        diffs.append(max(np.abs(u2[0][..., -1] - mid).max(), np.abs(u2[1][..., 0] - mid).max()))
        # both shells carry the same values on the common sphere (up to the
        # last-bit difference of the radius the two grids compute for it)
        assert np.abs(u2[0][..., -1] - u2[1][..., 0]).max() < 1e-13
    assert diffs[1] < diffs[0] / 4, diffs
