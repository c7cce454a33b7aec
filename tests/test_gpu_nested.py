"""Nested shells through the C-ABI (cffyn_nest_*) against the oracle's nested
shells (oracle/nested.py): right-hand sides with the characteristic coupling
on the common spheres, RK4 steps, three shells of different n_r, and the
argument checks.  Tolerances as for one shell."""

import numpy as np
import pytest

from oracle import nested
from paper_1104_3408_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-10}   # FP64, MIXED
KW = dict(amp=1e-4, ell=2, seed=3, center=5.6, width=0.7)


@pytest.fixture(scope="module")
def cf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1104_3408_gb300 import cffyn
    return cffyn


def _states(n_rs, N, radii, nf=50):
    us = [inputs.kerr_schild_state(n_r, N, 2 * N, radii[s], radii[s + 1], n_fields=nf, **KW)
          for s, n_r in enumerate(n_rs)]
    if nf > 50:
        from oracle import ghg
        for u in us:
            u[50:54] = ghg.gauge_source_from_state(u[:50].reshape(50, -1)).reshape((4,) + u.shape[1:])
    return us


def _gpu_nest(cf, n_rs, N, radii, L, prec, nf=50):
    shells = [cf.Shell(n_r, N, 2 * N, radii[s], radii[s + 1], L, n_fields=nf, precision=prec)
              for s, n_r in enumerate(n_rs)]
    return shells, cf.Nest(shells)


@pytest.mark.parametrize("nf", [50, 54])
@pytest.mark.parametrize("prec", [0, 1])
def test_nest_rhs_matches_oracle(cf, prec, nf):
    n_rs, N, L, radii = [9, 13], 12, 10, [1.8, 6.4, 11.0]
    us = _states(n_rs, N, radii, nf)
    ref_n = nested.NestedOracle(n_rs, N, radii, L, n_fields=nf)
    if nf == 50:
        ref_n.init_gauge_from_state(us)
    ref = ref_n.rhs(us)
    scale = max(np.abs(sh.derivs(u)).max() for sh, u in zip(ref_n.shells, us))
    shells, nest = _gpu_nest(cf, n_rs, N, radii, L, prec, nf)
    du = [torch.from_numpy(u).cuda() for u in us]
    if nf == 50:
        for sh, u in zip(shells, du):
            sh.init_gauge_from_state(u)
    outs = [torch.empty_like(u) for u in du]
    nest.rhs(du, outs)
    got = [o.cpu().numpy() for o in outs]
    for g, r in zip(got, ref):
        e = np.abs(g - r).max() / scale
        assert e < TOL[prec], e
    # one right-hand side on the common sphere
    assert np.abs(got[0][..., -1] - got[1][..., 0]).max() < 1e-14 * scale
    nest.destroy()
    for sh in shells:
        sh.destroy()


@pytest.mark.parametrize("prec", [0, 1])
def test_nest_rk4_steps_match_oracle(cf, prec):
    n_rs, N, L, radii = [9, 9], 12, 10, [1.8, 6.4, 11.0]
    us = _states(n_rs, N, radii)
    ref_n = nested.NestedOracle(n_rs, N, radii, L)
    ref_n.init_gauge_from_state(us)
    start = ref_n.filter(us)
    dt = ref_n.dx_min()
    ref = ref_n.rk4_step(start, dt, 5)
    shells, nest = _gpu_nest(cf, n_rs, N, radii, L, prec)
    du = [torch.from_numpy(u).cuda() for u in us]
    vs = []
    for sh, u in zip(shells, du):
        sh.init_gauge_from_state(u)
        v = torch.empty_like(u)
        sh.filter(u, v)
        vs.append(v)
    assert abs(nest.default_dt() - 0.25 * dt) < 1e-15
    nest.rk4_step(vs, dt, 5)
    got = [v.cpu().numpy() for v in vs]
    for g, r, s0 in zip(got, ref, start):
        e = np.abs(g - r).max() / np.abs(r).max()
        assert e < (1e-12 if prec == 0 else 1e-8), e
        assert np.abs(r - s0).max() > 1e-7       # the fields moved
    # the common sphere: one right-hand side, but each shell's filter (the
    # mixed path's fixed point is relative to the whole shell's field)
    assert np.abs(got[0][..., -1] - got[1][..., 0]).max() < (1e-13 if prec == 0 else 1e-10)
    nest.destroy()
    for sh in shells:
        sh.destroy()


def test_three_shells_mixed_vs_fp64(cf):
    n_rs, N, L, radii = [13, 9, 17], 12, 10, [1.8, 4.0, 6.4, 11.0]
    us = _states(n_rs, N, radii)
    res = []
    for prec in (1, 0):
        shells, nest = _gpu_nest(cf, n_rs, N, radii, L, prec)
        vs = []
        for sh, u0 in zip(shells, us):
            u = torch.from_numpy(u0).cuda()
            sh.init_gauge_from_state(u)
            v = torch.empty_like(u)
            sh.filter(u, v)
            vs.append(v)
        nest.rk4_step(vs, 0.0, 50)
        res.append([v.cpu().numpy() for v in vs])
        nest.destroy()
        for sh in shells:
            sh.destroy()
    for a, b in zip(*res):
        assert np.isfinite(a).all()
        assert np.abs(a - b).max() / np.abs(b).max() < 1e-8
    for s in range(2):
        assert np.abs(res[1][s][..., -1] - res[1][s + 1][..., 0]).max() < 1e-13        # FP64
        assert np.abs(res[0][s][..., -1] - res[0][s + 1][..., 0]).max() < 1e-10        # mixed


def test_nest_arguments(cf):
    a = cf.Shell(9, 12, 24, 1.8, 6.4, 10)
    b = cf.Shell(9, 12, 24, 6.5, 11.0, 10)          # a gap
    c = cf.Shell(9, 8, 16, 6.4, 11.0, 6)            # another angular grid
    for bad in ([a, b], [a, c], [a, a]):
        with pytest.raises(cf.CffynError) as ei:
            cf.Nest(bad)
        assert ei.value.code == cf.EINVAL
    for s in (a, b, c):
        s.destroy()


@pytest.mark.parametrize("mode,kind", [("step", "yn"), ("substep", "yg")])
def test_nest_filter_placements_and_kinds_match_oracle(cf, mode, kind):
    n_rs, N, L, radii = [9, 7], 12, 8, [1.8, 5.0, 11.0]
    us = _states(n_rs, N, radii)
    ref_n = nested.NestedOracle(n_rs, N, radii, L, filter_mode=mode, filter_kind=kind)
    ref_n.init_gauge_from_state(us)
    start = ref_n.filter(us) if mode == "substep" else us
    dt = ref_n.dx_min()
    ref = ref_n.rk4_step(start, dt, 4)
    fm = cf.FILTER_STEP if mode == "step" else cf.FILTER_SUBSTEP
    fk = {"yn": cf.FILTER_YN, "yg": cf.FILTER_YG}[kind]
    shells = [cf.Shell(n_r, N, 2 * N, radii[s], radii[s + 1], L, precision=cf.MIXED, filter_mode=fm,
                       filter_kind=fk) for s, n_r in enumerate(n_rs)]
    nest = cf.Nest(shells)
    vs = []
    for sh, u0 in zip(shells, us):
        u = torch.from_numpy(u0).cuda()
        sh.init_gauge_from_state(u)
        if mode == "substep":
            v = torch.empty_like(u)
            sh.filter(u, v)
            u = v
        vs.append(u)
    nest.rk4_step(vs, dt, 4)
    for g, r in zip([v.cpu().numpy() for v in vs], ref):
        assert np.abs(g - r).max() / np.abs(r).max() < 1e-8
    nest.destroy()
    for sh in shells:
        sh.destroy()
