"""First-order generalized harmonic (GHG) system (paper App. A).

Test infrastructure only (see ``oracle/__init__``).

State vector u^mu = {g_ab, Pi_ab, Phi_iab} (50 fields), optionally + H_a (54)
and + dH_a/dt (58).  Field order (a convention of this project; the paper
fixes none): symmetric pairs (tt, tx, ty, tz, xx, xy, xz, yy, yz, zz) for g_ab
(fields 0..9), Pi_ab (10..19), Phi_xab (20..29), Phi_yab (30..39), Phi_zab
(40..49), then H_t..H_z (50..53), then dH_t/dt..dH_z/dt (54..57).

Dependent quantities (eqs. normal, abgfromgab, Gamma): gamma_ij = g_ij,
beta_j = g_tj, beta^i = gamma^ij beta_j, alpha = sqrt(beta_i beta^i - g_tt),
n^a = (1/alpha, -beta^i/alpha), n_a = (-alpha, 0, 0, 0), g^ab the inverse
4-metric, d_i g_ab = Phi_iab, d_t g_ab = -alpha Pi_ab + beta^i Phi_iab,
Gamma_cab = 1/2 (d_a g_bc + d_b g_ac - d_c g_ab), Gamma_c = g^ab Gamma_cab,
nabla_a H_b = d_a H_b - g^cd Gamma_cab H_d.

Evolution equations eqs. gdot, Phidot, Pidot with gamma_0 = gamma_2 = 1,
gamma_1 = -1, gamma_3 = gamma_1 gamma_2 (already substituted in the paper's
printed form).  d_t H_a = 0 (eq. gauge) for 50 and 54 fields; for 58 fields
d_t H_a = G_a and d_t G_a = 0 (reading: the paper leaves the second-order gauge
evolution unspecified; this keeps the static gauge of eq. gauge).

Outer boundary (App. A.2, freeze-incoming, the B = E^{-1} Z E formulas at the
end of A.2) at the largest radius only; s_i = l_i / sqrt(gamma^ij l_i l_j),
l_i = x_i / r, s^k = gamma^kl s_l with the current metric.

Parity pins (tests/test_oracle_ghg.py, tests/test_oracle_constraints.py):
closed-form Kerr-Schild 3+1 quantities (App. A.3); the characteristic speeds
printed in App. A.3; the linear part of the rhs in d_k u against the printed
characteristic matrix of App. A.2 (this fixes every derivative term,
including the gamma_2 d_i g_ab terms); the BC is a projection that keeps the
outgoing characteristic field; exact Kerr-Schild data give a right-hand side
at truncation level converging with n_r (Sec. 4.1); Gamma_a of exact
Kerr-Schild data equals its closed form (2M/r^2) l_a; the constraint norms of
data with a known violation (one of the 30 C_iab components, or C_a = h)
equal the RMS over points and components; the gamma_2 terms drop out when
C_iab = 0; and on spatially constant perturbations of flat space the
constraints decay at the rates the damping terms give at linear order
(C_iab at gamma_2, C_t at 2 gamma_0, C_i at gamma_0).  The R10 runs of
Sec. 4.1 (tests/test_oracle_r10.py) also need both damping terms to settle.
"""

import numpy as np

from .ynfilter import SYM_PAIRS, sym_index


def unpack_sym(block):
    """[10, ...] symmetric-pair fields -> [4, 4, ...]."""
    out = np.empty((4, 4) + block.shape[1:], dtype=block.dtype)
    for s, (a, b) in enumerate(SYM_PAIRS):
        out[a, b] = block[s]
        out[b, a] = block[s]
    return out


def pack_sym(T):
    """[4, 4, ...] -> [10, ...]."""
    return np.stack([T[a, b] for (a, b) in SYM_PAIRS])


def split_state(u):
    """u[mu, P] -> g[4,4,P], Pi[4,4,P], Phi[3,4,4,P]."""
    g = unpack_sym(u[0:10])
    Pi = unpack_sym(u[10:20])
    Phi = np.stack([unpack_sym(u[20 + 10 * i:30 + 10 * i]) for i in range(3)])
    return g, Pi, Phi


def inv_batched(M):
    """Inverse of [n, n, P] matrices, pointwise."""
    return np.moveaxis(np.linalg.inv(np.moveaxis(M, -1, 0)), 0, -1)


def three_plus_one(g):
    """3+1 quantities of eqs. normal and abgfromgab."""
    gamma_inv = inv_batched(g[1:, 1:])
    beta_lo = g[0, 1:]
    beta_up = np.einsum("ijP,jP->iP", gamma_inv, beta_lo)
    alpha = np.sqrt(np.einsum("iP,iP->P", beta_lo, beta_up) - g[0, 0])
    n_up = np.concatenate([(1.0 / alpha)[None], -beta_up / alpha[None]])
    n_lo = np.zeros_like(n_up)
    n_lo[0] = -alpha
    ginv = inv_batched(g)
    return alpha, beta_up, gamma_inv, n_up, n_lo, ginv


def christoffel(g, Pi, Phi, alpha, beta_up, ginv):
    """Gamma_cab and Gamma_c from undifferentiated variables (eq. Gamma and
    the expressions for d_c g_ab after it)."""
    dg4 = np.empty((4, 4, 4) + g.shape[2:])
    dg4[0] = -alpha[None, None] * Pi + np.einsum("iP,iabP->abP", beta_up, Phi)
    dg4[1:] = Phi
    Gam = 0.5 * (np.einsum("abcP->cabP", dg4) + np.einsum("bacP->cabP", dg4) - dg4)
    Gam_c = np.einsum("abP,cabP->cP", ginv, Gam)
    return Gam, Gam_c


def gauge_source_from_state(u):
    """H_a = -Gamma_a (eq. gauge), pointwise.  u[mu, ...] -> H[4, ...]."""
    shp = u.shape[1:]
    uf = u.reshape(u.shape[0], -1)
    g, Pi, Phi = split_state(uf)
    alpha, beta_up, _, _, _, ginv = three_plus_one(g)
    _, Gam_c = christoffel(g, Pi, Phi, alpha, beta_up, ginv)
    return (-Gam_c).reshape((4,) + shp)


def rhs_pointwise(u, du, H, dH, n_fields=50, gamma0=1.0, gamma2=1.0):
    """Right-hand side of eqs. gdot, Phidot, Pidot for every point.

    u[mu, P], du[3, mu, P] (numerical Cartesian derivatives of every field),
    H[4, P] and dH[3, 4, P] (d_i H_a).  Returns rhs[mu, P].

    gamma0 and gamma2 are the constraint-damping factors of App. A.1, which
    the printed equations take as 1 (with gamma1 = -1, gamma3 = gamma1
    gamma2): gamma2 multiplies alpha (d_i g_ab - Phi_iab) in eq. Phidot and
    -beta^k (d_k g_ab - Phi_kab) in eq. Pidot, gamma0 the gauge-constraint
    term of eq. Pidot.  Other values exist only for tests of the damping."""
    g, Pi, Phi = split_state(u)
    dg = np.stack([unpack_sym(du[i, 0:10]) for i in range(3)])            # d_i g_ab
    dPi = np.stack([unpack_sym(du[i, 10:20]) for i in range(3)])          # d_i Pi_ab
    dPhi = np.stack([np.stack([unpack_sym(du[k, 20 + 10 * i:30 + 10 * i])
                               for i in range(3)]) for k in range(3)])    # d_k Phi_iab
    alpha, beta_up, gamma_inv, n_up, n_lo, ginv = three_plus_one(g)
    Gam, Gam_c = christoffel(g, Pi, Phi, alpha, beta_up, ginv)
    P = u.shape[1]

    dH4 = np.zeros((4, 4, P))
    if n_fields == 58:
        dH4[0] = u[54:58]
    dH4[1:] = dH
    DH = dH4 - np.einsum("cdP,cabP,dP->abP", ginv, Gam, H, optimize=True)
    C = H + Gam_c

    al = alpha[None, None]
    dt_g = -al * Pi + np.einsum("iP,iabP->abP", beta_up, Phi)

    nnPhi = np.einsum("cP,dP,icdP->iP", n_up, n_up, Phi, optimize=True)
    dt_Phi = (np.einsum("kP,kiabP->iabP", beta_up, dPhi)
              - alpha[None, None, None] * dPi
              + gamma2 * alpha[None, None, None] * dg
              + 0.5 * alpha[None, None, None] * nnPhi[:, None, None] * Pi[None]
              + alpha[None, None, None] * np.einsum("jkP,cP,ijcP,kabP->iabP", gamma_inv, n_up,
                                                    Phi[:, 1:], Phi, optimize=True)
              - gamma2 * alpha[None, None, None] * Phi)

    Q1 = np.einsum("cdP,ijP,iacP,jbdP->abP", ginv, gamma_inv, Phi, Phi, optimize=True)
    Q2 = np.einsum("cdP,acP,bdP->abP", ginv, Pi, Pi, optimize=True)
    Q3 = np.einsum("cdP,efP,aceP,bdfP->abP", ginv, ginv, Gam, Gam, optimize=True)
    nnPi = np.einsum("cP,dP,cdP->P", n_up, n_up, Pi)
    nC = np.einsum("cP,cP->P", n_up, C)
    dt_Pi = (np.einsum("kP,kabP->abP", beta_up, dPi)
             - al * np.einsum("ikP,kiabP->abP", gamma_inv, dPhi)
             - gamma2 * np.einsum("kP,kabP->abP", beta_up, dg)
             + 2.0 * al * (Q1 - Q2 - Q3)
             - al * (DH + np.einsum("abP->baP", DH))
             - 0.5 * al * nnPi[None, None] * Pi
             - al * np.einsum("cP,ciP,ijP,jabP->abP", n_up, Pi[:, 1:], gamma_inv, Phi, optimize=True)
             + gamma0 * al * (np.einsum("bP,aP->abP", n_lo, C) + np.einsum("aP,bP->abP", n_lo, C)
                              - g * nC[None, None])
             + gamma2 * np.einsum("iP,iabP->abP", beta_up, Phi))

    out = np.zeros_like(u)
    out[0:10] = pack_sym(dt_g)
    out[10:20] = pack_sym(dt_Pi)
    for i in range(3):
        out[20 + 10 * i:30 + 10 * i] = pack_sym(dt_Phi[i])
    if n_fields == 58:
        out[50:54] = u[54:58]
    return out


def apply_outer_bc(rhs, u, theta, phi):
    """Freeze-incoming condition B(d_t u) of App. A.2 on the outermost sphere
    (largest k).  rhs, u: [mu, J, N, K]; modified copy returned."""
    out = np.array(rhs, copy=True)
    uo = u[:, :, :, -1].reshape(u.shape[0], -1)
    ro = out[:, :, :, -1].reshape(u.shape[0], -1)
    st, ct = np.sin(theta)[None, :], np.cos(theta)[None, :]
    sp, cp = np.sin(phi)[:, None], np.cos(phi)[:, None]
    l = np.stack([(st * cp).ravel(), (st * sp).ravel(), (ct * np.ones_like(sp)).ravel()])
    g, _, _ = split_state(uo)
    gamma_inv = inv_batched(g[1:, 1:])
    s_lo = l / np.sqrt(np.einsum("ijP,iP,jP->P", gamma_inv, l, l))[None]
    s_up = np.einsum("klP,lP->kP", gamma_inv, s_lo)
    dtg = ro[0:10]
    dtPi = ro[10:20]
    dtPhi = np.stack([ro[20 + 10 * i:30 + 10 * i] for i in range(3)])
    sdPhi = np.einsum("kP,ksP->sP", s_up, dtPhi)
    newPi = 0.5 * (dtg + dtPi + sdPhi)
    newPhi = 0.5 * s_lo[:, None, :] * (-dtg + dtPi + sdPhi)[None]
    ro[10:20] = newPi
    for i in range(3):
        ro[20 + 10 * i:30 + 10 * i] = newPhi[i]
    out[:, :, :, -1] = ro.reshape(out[:, :, :, -1].shape)
    return out


def constraint_norms(u, du, H):
    """RMS of C_iab = d_i g_ab - Phi_iab (30 components) and of
    C_a = H_a + Gamma_a (4 components) over all points (App. A.1)."""
    uf = u.reshape(u.shape[0], -1)
    duf = du.reshape(3, du.shape[1], -1)
    Hf = H.reshape(4, -1)
    g, Pi, Phi = split_state(uf)
    c3 = np.stack([duf[i, 0:10] - uf[20 + 10 * i:30 + 10 * i] for i in range(3)])
    alpha, beta_up, _, _, _, ginv = three_plus_one(g)
    _, Gam_c = christoffel(g, Pi, Phi, alpha, beta_up, ginv)
    ca = Hf + Gam_c
    return float(np.sqrt(np.mean(c3 ** 2))), float(np.sqrt(np.mean(ca ** 2)))


__all__ = ["unpack_sym", "pack_sym", "split_state", "three_plus_one", "christoffel",
           "gauge_source_from_state", "rhs_pointwise", "apply_outer_bc", "constraint_norms",
           "sym_index"]
