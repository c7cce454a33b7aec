"""The paper's single black hole runs on the shell R10 (Sec. 4.1), on the GPU.

R10 is the shell r in [1.8, 11.8] around a Schwarzschild black hole of mass 1
in Kerr-Schild form (App. A.3).  Initial data as in the paper: g_ab from
eq. KSmetric, Phi_iab its numerical (spectral, FP64) Cartesian derivative,
Pi_ab from eq. defPiPhi with d_t g_ab = 0; the gauge source is frozen at
H_a = -Gamma_a(t = 0) (eq. gauge).  Default configuration of the paper's runs:
Yn filter with n_f = 4 (the library's L = N_theta - 1 - n_f) applied after
every full RK4 step, dt = lambda min dx with lambda = 4.

Monitored quantity (the paper's): max |d_t g_tt| over the innermost sphere,
i.e. the right-hand side of g_tt at r = r_in.

Studies, each printing one JSON line per run (``python -m
paper_1104_3408_gb300.r10 <study> [options]``):

``rconv``    Fig. r10_rconv: N_r = 13..37 at N_theta = 9, N_phi = 18; the
             truncation error of the analytic data converges exponentially
             with N_r and the runs settle to a stationary state.
``nf``       Fig. r10_nf: n_f = 0..4 on one grid; n_f <= 2 fail within
             t = 110, n_f >= 3 do not.
``filters``  Figs. r10_f0 / r10_f1: the scalar Y and graded Yg filters
             against the Yn filter on long runs.
``dtfac``    Tab. dtfac: a ladder of Courant factors on each of the table's
             grids; the largest stable and the smallest unstable one.
``nested``   R10 split into two nested shells [1.8, 6.8] and [6.8, 11.8]
             (n_r each, coupled on the common sphere through the
             characteristic fields of App. A.2) beside one shell of the same
             radial points (2 n_r - 1); same filter, Courant factor and
             monitored quantity.

Every step runs in the CUDA library (cffyn_rk4_step, cffyn_rhs); torch only
holds the arrays and reduces the monitored maximum.
"""

import argparse
import json
import math
import sys
import time

from . import cffyn, inputs

R_IN, R_OUT = 1.8, 11.8
N_F, COURANT = 4, 4.0
BLOWUP = 1e-2          # |d_t g_tt| above this on the inner sphere counts as a failed run

# grids of Tab. dtfac with the paper's largest stable Courant factor
DTFAC_GRIDS = [((13, 9), 4.4), ((19, 9), 5.9), ((19, 15), 5.9), ((25, 9), 6.1),
               ((25, 15), 6.0), ((31, 9), 6.3), ((31, 15), 6.3)]


def make_shell(n_r, n_theta, n_f=N_F, courant=COURANT, precision=cffyn.MIXED,
               filter_kind=cffyn.FILTER_YN, filter_mode=cffyn.FILTER_STEP):
    """An R10 shell; L = n_theta - 1 - n_f (the paper's n_f top modes removed)."""
    return cffyn.Shell(n_r, n_theta, 2 * n_theta, R_IN, R_OUT, n_theta - 1 - n_f,
                       precision=precision, filter_mode=filter_mode, courant=courant,
                       filter_kind=filter_kind)


def initial_state(n_r, n_theta, device="cuda", r_in=R_IN, r_out=R_OUT):
    """Kerr-Schild data with Phi_iab the numerical Cartesian derivative of
    g_ab (taken by an FP64 shell of the library) and Pi_ab = beta^k Phi_kab /
    alpha; returns the 50-field state as a float64 CUDA tensor."""
    import torch
    n_phi = 2 * n_theta
    u = inputs.kerr_schild_state(n_r, n_theta, n_phi, r_in, r_out, amp=0.0)
    sh = cffyn.Shell(n_r, n_theta, n_phi, r_in, r_out, 0, precision=cffyn.FP64)
    try:
        ud = torch.from_numpy(u).to(device)
        d = torch.empty((3,) + tuple(ud.shape), dtype=torch.float64, device=device)
        sh.derivs(ud, d)
        phi = d[:, :10].cpu().numpy()
    finally:
        sh.destroy()
    u[20:50] = phi.reshape((30,) + u.shape[1:])
    u[10:20] = inputs.kerr_schild_pi_from_phi(phi, n_r, n_theta, n_phi, r_in, r_out)
    return torch.from_numpy(u).to(device)


def rhs_gtt_inner(sh, u, buf):
    """max |d_t g_tt| over the innermost sphere (k = 0 is r = r_in)."""
    sh.rhs(u, buf)
    return float(buf[0, :, :, 0].abs().max())


def evolve(sh, u, t_end, sample_steps=20, blowup=BLOWUP, dt=None):
    """Advance u in place to t_end (or until it fails), sampling the
    monitored quantity every sample_steps steps.  A run fails when a stage
    right-hand side turns non-finite (CFFYN_ENONFINITE) or the monitored
    value exceeds blowup."""
    import torch
    dt = sh.default_dt() if dt is None else dt
    n = max(1, int(round(t_end / dt)))
    buf = torch.empty_like(u)
    series = [(0.0, rhs_gtt_inner(sh, u, buf))]
    s, failed_at = 0, None
    t0 = time.perf_counter()
    while s < n:
        k = min(sample_steps, n - s)
        try:
            sh.rk4_step(u, dt, k)
        except cffyn.CffynError as e:
            if e.code != cffyn.ENONFINITE:
                raise
            failed_at = (s + k) * dt
            break
        s += k
        v = rhs_gtt_inner(sh, u, buf)
        series.append((s * dt, v))
        if not math.isfinite(v) or v > blowup:
            failed_at = s * dt
            break
    torch.cuda.synchronize()
    return dict(dt=dt, steps=s, t=s * dt, failed_at=failed_at, series=series,
                seconds=time.perf_counter() - t0)


def _summary(run, keep=60):
    ser = run["series"]
    vals = [v for _, v in ser if math.isfinite(v)]
    late = [v for t, v in ser if t >= 0.8 * run["t"] and math.isfinite(v)]
    stride = max(1, len(ser) // keep)
    return dict(dt=run["dt"], steps=run["steps"], t=run["t"], failed_at=run["failed_at"],
                rhs_gtt_first=ser[1][1] if len(ser) > 1 else None,
                rhs_gtt_max=max(vals) if vals else None,
                rhs_gtt_final=ser[-1][1], rhs_gtt_late_max=max(late) if late else None,
                seconds=run["seconds"],
                series_log10=[(round(t, 2), round(math.log10(v), 3) if v > 0 and math.isfinite(v) else None)
                              for t, v in ser[::stride]])


def run_one(n_r, n_theta, t_end, n_f=N_F, courant=COURANT, precision=cffyn.MIXED,
            filter_kind=cffyn.FILTER_YN, sample_steps=20, device="cuda"):
    """One R10 run: initial data, gauge, evolution; returns its summary."""
    u = initial_state(n_r, n_theta, device)
    sh = make_shell(n_r, n_theta, n_f, courant, precision, filter_kind)
    try:
        sh.init_gauge_from_state(u)
        import torch
        buf = torch.empty_like(u)
        sh.rhs(u, buf)
        trunc0 = float(buf.abs().max())
        run = evolve(sh, u, t_end, sample_steps)
    finally:
        sh.destroy()
    out = _summary(run)
    out.update(grid=f"{n_r}x{n_theta}x{2 * n_theta}", n_f=n_f, courant=courant,
               precision="fp64" if precision == cffyn.FP64 else "mixed",
               filter={cffyn.FILTER_YN: "yn", cffyn.FILTER_Y: "y", cffyn.FILTER_YG: "yg"}[filter_kind],
               rhs_all_t0=trunc0)
    return out


def _precisions(name):
    return {"mixed": [cffyn.MIXED], "fp64": [cffyn.FP64], "both": [cffyn.MIXED, cffyn.FP64]}[name]


def study_rconv(a, emit):
    for prec in _precisions(a.precision):
        for n_r in a.n_r or [13, 19, 25, 31, 37]:
            emit("rconv", run_one(n_r, a.n_theta or 9, a.t_end or 1000.0, precision=prec))


def study_nf(a, emit):
    for prec in _precisions(a.precision):
        for nf in range(5):
            emit("nf", run_one((a.n_r or [13])[0], a.n_theta or 9, a.t_end or 110.0, n_f=nf,
                               precision=prec))


def study_filters(a, emit):
    kinds = {"yn": cffyn.FILTER_YN, "y": cffyn.FILTER_Y, "yg": cffyn.FILTER_YG}
    for prec in _precisions(a.precision):
        for name in a.kinds.split(","):
            emit("filters", run_one((a.n_r or [25])[0], a.n_theta or 9, a.t_end or 8000.0,
                                    precision=prec, filter_kind=kinds[name], sample_steps=50))


def study_dtfac(a, emit):
    ladder = [float(x) for x in a.ladder.split(",")]
    for (n_r, n_theta), lam_paper in DTFAC_GRIDS:
        if a.n_r and n_r not in a.n_r:
            continue
        if a.n_theta and n_theta != a.n_theta:
            continue
        for prec in _precisions(a.precision):
            stable, unstable, runs = None, None, []
            for lam in ladder:
                r = run_one(n_r, n_theta, a.t_end or 500.0, courant=lam, precision=prec,
                            sample_steps=10)
                runs.append(dict(courant=lam, failed_at=r["failed_at"], t=r["t"],
                                 rhs_gtt_final=r["rhs_gtt_final"], seconds=r["seconds"]))
                if r["failed_at"] is None:
                    stable = lam
                else:
                    unstable = lam
                    break                      # larger factors fail sooner
            emit("dtfac", dict(grid=f"{n_r}x{n_theta}x{2 * n_theta}",
                               precision="fp64" if prec == cffyn.FP64 else "mixed",
                               t_end=a.t_end or 500.0, largest_stable=stable,
                               smallest_unstable=unstable, paper_lambda_max=lam_paper, runs=runs))


def run_nested(n_r, n_theta, t_end, r_mid=6.8, n_f=N_F, courant=COURANT, precision=cffyn.MIXED,
               sample_steps=20, device="cuda", dt=None):
    """R10 as two nested shells [R_IN, r_mid], [r_mid, R_OUT] of n_r points
    each (cffyn_nest_*), per-step Yn filter; the monitored quantity is taken
    on the inner shell's inner sphere.  dt: the nest's default (the Courant
    factor times its smallest spacing) if None."""
    import torch
    radii = [R_IN, r_mid, R_OUT]
    us = [initial_state(n_r, n_theta, device, radii[i], radii[i + 1]) for i in range(2)]
    shells = [cffyn.Shell(n_r, n_theta, 2 * n_theta, radii[i], radii[i + 1], n_theta - 1 - n_f,
                          precision=precision, filter_mode=cffyn.FILTER_STEP, courant=courant)
              for i in range(2)]
    nest = cffyn.Nest(shells)
    try:
        for sh, u in zip(shells, us):
            sh.init_gauge_from_state(u)
        bufs = [torch.empty_like(u) for u in us]

        def monitored():
            nest.rhs(us, bufs)
            return float(bufs[0][0, :, :, 0].abs().max())

        nest.rhs(us, bufs)
        trunc0 = max(float(b.abs().max()) for b in bufs)
        dt = nest.default_dt() if dt is None else dt
        n = max(1, int(round(t_end / dt)))
        series = [(0.0, monitored())]
        s, failed_at = 0, None
        t0 = time.perf_counter()
        while s < n:
            k = min(sample_steps, n - s)
            try:
                nest.rk4_step(us, dt, k)
            except cffyn.CffynError as e:
                if e.code != cffyn.ENONFINITE:
                    raise
                failed_at = (s + k) * dt
                break
            s += k
            v = monitored()
            series.append((s * dt, v))
            if not math.isfinite(v) or v > BLOWUP:
                failed_at = s * dt
                break
        torch.cuda.synchronize()
        run = dict(dt=dt, steps=s, t=s * dt, failed_at=failed_at, series=series,
                   seconds=time.perf_counter() - t0)
        common = float((us[0][..., -1] - us[1][..., 0]).abs().max())
    finally:
        nest.destroy()
        for sh in shells:
            sh.destroy()
    out = _summary(run)
    out.update(grid=f"2 x {n_r}x{n_theta}x{2 * n_theta}", radii=radii, n_f=n_f, courant=courant,
               precision="fp64" if precision == cffyn.FP64 else "mixed", rhs_all_t0=trunc0,
               common_sphere_diff=common)
    return out


def study_nested(a, emit):
    for prec in _precisions(a.precision):
        for n_r in a.n_r or [13]:
            t_end = a.t_end or 1000.0
            # the single shell of the same radial resolution, then the nest at
            # its own default dt and at the single shell's dt (the nest's
            # radial spacing is twice the single shell's, so its default dt
            # is twice as large against the same angular grid)
            single = run_one(2 * n_r - 1, a.n_theta or 9, t_end, precision=prec)
            emit("nested_single_reference", single)
            emit("nested", run_nested(n_r, a.n_theta or 9, t_end, precision=prec))
            emit("nested_at_single_dt", run_nested(n_r, a.n_theta or 9, t_end, precision=prec, dt=single["dt"]))
            # the Courant factor on the nest's own smallest spacing: which the
            # interface coupling keeps stable
            base = run_nested(n_r, a.n_theta or 9, 1.0, precision=prec)["dt"] / COURANT
            for lam in (2.0, 2.5, 3.0, 3.5):
                r = run_nested(n_r, a.n_theta or 9, min(t_end, 500.0), precision=prec, dt=lam * base)
                r["courant"] = lam
                emit("nested_courant", r)


STUDIES = {"rconv": study_rconv, "nf": study_nf, "filters": study_filters, "dtfac": study_dtfac,
           "nested": study_nested}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("studies", nargs="+", choices=sorted(STUDIES))
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64", "both"])
    ap.add_argument("--n-r", type=int, nargs="*", dest="n_r", default=None)
    ap.add_argument("--n-theta", type=int, default=None)
    ap.add_argument("--t-end", type=float, default=None)
    ap.add_argument("--kinds", default="yn,y,yg", help="filters study: comma list of yn,y,yg")
    ap.add_argument("--ladder", default="4.0,4.5,5.0,5.5,6.0,6.5,7.0",
                    help="dtfac study: Courant factors, increasing")
    ap.add_argument("--out", default=None, help="also append the JSON lines to this file")
    a = ap.parse_args(argv)
    fh = open(a.out, "a") if a.out else None

    def emit(study, rec):
        line = json.dumps(dict(study=study, **rec))
        print(line, flush=True)
        if fh:
            fh.write(line + "\n")
            fh.flush()

    cffyn.load()
    for name in a.studies:
        STUDIES[name](a, emit)
    if fh:
        fh.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
