"""Method of lines with classical RK4 (paper Sec. 2.5) on one shell.

Test infrastructure only (see ``oracle/__init__``).

One RK4 step: four evaluations of S - A^k d_k u (eq. dotu), boundary
conditions in every substep (Sec. 2.5).  Filter placement:

* ``"step"`` (the paper, Sec. 2.5): u_{n+1} = F(RK4 step of B(rhs)).
* ``"substep"`` (reading used for the benchmark workloads, which ask for the
  filter in every substep): k_s = F(B(rhs(U_s))), U_2 = u_n + dt/2 k_1,
  U_3 = u_n + dt/2 k_2, U_4 = u_n + dt k_3,
  u_{n+1} = u_n + dt/6 (k_1 + 2 k_2 + 2 k_3 + k_4).  F is linear and
  idempotent, so a state that starts in range(F) stays there; the caller
  filters the initial data once.

dt defaults to lambda * min dx (Sec. 4.1, Courant factor).
"""

import numpy as np

from . import cff, ghg, ynfilter


class OracleShell:
    """All precomputed matrices of one shell plus the static gauge source."""

    def __init__(self, n_r, n_theta, n_phi, r_in, r_out, L, n_fields=50,
                 filter_mode="substep", filter_kind="yn"):
        assert n_phi == 2 * n_theta
        assert n_fields in (50, 54, 58)
        assert filter_kind in ("yn", "y", "yg")
        self.filter_kind = filter_kind
        self._sf_at = {}
        self.n_r, self.N, self.J = n_r, n_theta, n_phi
        self.r_in, self.r_out, self.L = r_in, r_out, L
        self.n_fields = n_fields
        self.filter_mode = filter_mode
        self.r, self.theta, self.phi = cff.grid(n_r, n_theta, n_phi, r_in, r_out)
        self._sf = None
        self.H = None
        self.dH = None
        # constraint-damping factors of App. A.1 (the paper's values; tests of
        # the damping change them)
        self.gamma0 = 1.0
        self.gamma2 = 1.0

    @property
    def sf(self):
        if self._sf is None:
            self._sf = ynfilter.SpinFilter(self.theta, self.phi, self.L)
        return self._sf

    def dx_min(self):
        return cff.dx_min(self.r, self.theta, self.phi)

    # -- derivatives -------------------------------------------------------
    def spherical_derivs(self, u):
        return cff.spherical_derivatives(u, self.r_in, self.r_out)

    def derivs(self, u):
        """Cartesian derivatives of every field: [3, mu, J, N, K]."""
        dr, dth, dph = self.spherical_derivs(u)
        return cff.cartesian_gradient(dr, dth, dph, self.r, self.theta, self.phi)

    # -- gauge ---------------------------------------------------------------
    def set_gauge(self, H):
        """Static gauge source H_a[4, J, N, K]; d_i H_a by the spectral
        Cartesian derivative (App. A.1, last paragraph)."""
        self.H = np.array(H, dtype=np.float64)
        self.dH = cff.cartesian_derivatives(self.H, self.r_in, self.r_out)

    def init_gauge_from_state(self, u):
        """H_a = -Gamma_a(u) (eq. gauge)."""
        self.set_gauge(ghg.gauge_source_from_state(u[:50]))

    def _gauge(self, u, du):
        if self.n_fields == 50:
            return self.H, self.dH
        return u[50:54], du[:, 50:54]

    # -- operators -----------------------------------------------------------
    def rhs(self, u, outer_bc=True):
        """Derivatives + GHG right-hand side + outer BC (unless outer_bc is
        False: the inner shells of a nested set), no filter."""
        du = self.derivs(u)
        H, dH = self._gauge(u, du)
        mu = u.shape[0]
        shp = u.shape[1:]
        out = ghg.rhs_pointwise(u.reshape(mu, -1), du.reshape(3, mu, -1),
                                H.reshape(4, -1), dH.reshape(3, 4, -1), self.n_fields,
                                self.gamma0, self.gamma2)
        out = out.reshape(u.shape)
        del shp
        if not outer_bc:
            return out
        return ghg.apply_outer_bc(out, u, self.theta, self.phi)

    def sf_at(self, L_keep):
        """SpinFilter of another retained degree (the graded filter's)."""
        if L_keep == self.L:
            return self.sf
        if L_keep not in self._sf_at:
            self._sf_at[L_keep] = ynfilter.SpinFilter(self.theta, self.phi, L_keep)
        return self._sf_at[L_keep]

    def filter(self, u):
        """Yn tensor filter (Sec. 3.5), or the component-wise Y / Yg filters."""
        if self.filter_kind == "yn":
            return ynfilter.filter_state(u, self.sf, self.n_fields)
        sfs = {None: self.sf}
        if self.filter_kind == "yg":
            for d in range(1, 4):
                Lk = min(self.L + d, self.N - 1)
                sfs[Lk] = self.sf_at(Lk)
        return ynfilter.filter_state_scalar(u, sfs, self.n_fields, graded=self.filter_kind == "yg")

    def stage(self, u):
        k = self.rhs(u)
        if self.filter_mode == "substep":
            k = self.filter(k)
        return k

    def rk4_step(self, u, dt=None, n_steps=1):
        if dt is None or dt <= 0:
            dt = 0.25 * self.dx_min()
        u = np.array(u, dtype=np.float64, copy=True)
        for _ in range(n_steps):
            k1 = self.stage(u)
            k2 = self.stage(u + 0.5 * dt * k1)
            k3 = self.stage(u + 0.5 * dt * k2)
            k4 = self.stage(u + dt * k3)
            u = u + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
            if self.filter_mode == "step":
                u = self.filter(u)
        return u

    def constraint_norms(self, u):
        du = self.derivs(u)
        H = self.H if self.n_fields == 50 else u[50:54]
        return ghg.constraint_norms(u[:50], du[:, :50], H)
