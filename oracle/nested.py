"""Nested spherical shells coupled at their common spheres: the domain
decomposition the paper names as the way to resolve local features and as
its next step (Secs. 1 and 5), with the characteristic analysis of App. A.2.

Test infrastructure only (see ``oracle/__init__``).

Shells s = 0 .. S-1 cover [R_s, R_{s+1}], R_0 < R_1 < ... < R_S, with the
same angular grid (n_theta, n_phi = 2 n_theta) and retained degree L and
their own n_r.  The Chebyshev-Gauss-Lobatto grid of every shell contains its
end radii, so the outer sphere of shell s and the inner sphere of shell s+1
are the same points.  Every shell computes derivatives and the right-hand
side of eq. dotu on its own; the outermost shell applies the freeze-incoming
condition of App. A.2 on its outer sphere; on each common sphere the two
right-hand sides are combined through the characteristic fields of eq.
characteristics with the normal s_i of the common sphere (outward, from the
inner shell's metric there):

    w0 = g                        speed 0
    w+ = -g + Pi + s^k Phi_k      speed  alpha - b
    w- = -g + Pi - s^k Phi_k      speed -alpha - b
    wT_i = Phi_i - s_i s^k Phi_k  speed -b           (b = s_k beta^k)

The fields that App. A.2's outer boundary condition freezes (w-, wT:
incoming from outside, since alpha - b > 0 > -b outside the horizon) take
the outer shell's right-hand side, where they leave that shell; w0 and w+
take the inner shell's.  Transforming back (the inverse of the eigenvector
matrix),

    d_t g = w0,  d_t Pi = (w+ + w-)/2 + w0,  d_t Phi_i = s_i (w+ - w-)/2 + wT_i,

and both shells get this right-hand side on the common sphere (the gauge
fields of 54/58-field states have no derivative terms and take the inner
shell's).  This is the reading of the paper's future-work remark used here;
with the outer shell's values replaced by zeros it is the freeze-incoming
condition itself.  Filter and RK4 as on one shell (Sec. 2.5), with one dt
for all shells.
"""

import numpy as np

from . import ghg
from .evolve import OracleShell


def interface_rhs(a, b, u, theta, phi):
    """Combined right-hand side on a common sphere.

    a: the inner shell's right-hand side on its outer sphere, b: the outer
    shell's on its inner sphere, u: the inner shell's state there; all
    [mu, J, N].  Returns the combined right-hand side [mu, J, N]."""
    mu = a.shape[0]
    af = a.reshape(mu, -1)
    bf = b.reshape(mu, -1)
    st, ct = np.sin(theta)[None, :], np.cos(theta)[None, :]
    sp, cp = np.sin(phi)[:, None], np.cos(phi)[:, None]
    l = np.stack([(st * cp).ravel(), (st * sp).ravel(), (ct * np.ones_like(sp)).ravel()])
    g, _, _ = ghg.split_state(u.reshape(mu, -1)[:50])
    gamma_inv = ghg.inv_batched(g[1:, 1:])
    s_lo = l / np.sqrt(np.einsum("ijP,iP,jP->P", gamma_inv, l, l))[None]
    s_up = np.einsum("klP,lP->kP", gamma_inv, s_lo)

    def fields(x):
        dg = x[0:10]
        dPi = x[10:20]
        dPhi = np.stack([x[20 + 10 * i:30 + 10 * i] for i in range(3)])
        sPhi = np.einsum("kP,ksP->sP", s_up, dPhi)
        return dg, -dg + dPi + sPhi, -dg + dPi - sPhi, dPhi - s_lo[:, None, :] * sPhi[None]

    w0, wp, _, _ = fields(af)
    _, _, wm, wT = fields(bf)
    out = np.array(af, copy=True)
    out[0:10] = w0
    out[10:20] = 0.5 * (wp + wm) + w0
    for i in range(3):
        out[20 + 10 * i:30 + 10 * i] = s_lo[i][None] * 0.5 * (wp - wm) + wT[i]
    return out.reshape(a.shape)


class NestedOracle:
    """Shells over radii[0] < radii[1] < ... with n_rs[s] radial points each."""

    def __init__(self, n_rs, n_theta, radii, L, n_fields=50, filter_mode="substep", filter_kind="yn"):
        assert len(radii) == len(n_rs) + 1 and all(a < b for a, b in zip(radii, radii[1:]))
        self.shells = [OracleShell(n_r, n_theta, 2 * n_theta, radii[s], radii[s + 1], L,
                                   n_fields=n_fields, filter_mode=filter_mode, filter_kind=filter_kind)
                       for s, n_r in enumerate(n_rs)]
        self.filter_mode = filter_mode

    def init_gauge_from_state(self, us):
        for sh, u in zip(self.shells, us):
            sh.init_gauge_from_state(u)

    def dx_min(self):
        return min(sh.dx_min() for sh in self.shells)

    def rhs(self, us):
        """Right-hand sides of every shell with the outer boundary condition on
        the outermost sphere and the characteristic coupling on the common
        spheres; no filter."""
        S = len(self.shells)
        out = [sh.rhs(u, outer_bc=(s == S - 1)) for s, (sh, u) in enumerate(zip(self.shells, us))]
        for s in range(S - 1):
            sh = self.shells[s]
            c = interface_rhs(out[s][..., -1], out[s + 1][..., 0], us[s][..., -1], sh.theta, sh.phi)
            out[s][..., -1] = c
            out[s + 1][..., 0] = c
        return out

    def filter(self, us):
        return [sh.filter(u) for sh, u in zip(self.shells, us)]

    def stage(self, us):
        k = self.rhs(us)
        if self.filter_mode == "substep":
            k = self.filter(k)
        return k

    def rk4_step(self, us, dt=None, n_steps=1):
        if dt is None or dt <= 0:
            dt = 0.25 * self.dx_min()
        us = [np.array(u, dtype=np.float64, copy=True) for u in us]
        for _ in range(n_steps):
            k1 = self.stage(us)
            k2 = self.stage([u + 0.5 * dt * k for u, k in zip(us, k1)])
            k3 = self.stage([u + 0.5 * dt * k for u, k in zip(us, k2)])
            k4 = self.stage([u + dt * k for u, k in zip(us, k3)])
            us = [u + (dt / 6.0) * (a + 2.0 * b + 2.0 * c + d)
                  for u, a, b, c, d in zip(us, k1, k2, k3, k4)]
            if self.filter_mode == "step":
                us = self.filter(us)
        return us
