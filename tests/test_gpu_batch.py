"""The uneven-shell batch (cffyn_create_batch / cffyn_batch_rk4_step) through
the C-ABI: every shell of a batch step runs the same kernels as a lone
cffyn_rk4_step, so the results must be bit-identical to stepping the shells
one by one; small batches are also compared with the CPU oracle."""

import numpy as np
import pytest

import oracle
from paper_1104_3408_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1104_3408_gb300 import cffyn
    return cffyn


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def make(cf, d, prec, nf=50):
    sh = cf.Shell(d["n_r"], d["n_theta"], d["n_phi"], d["r_in"], d["r_out"], d["L"], n_fields=nf,
                  precision=prec)
    u0 = inputs.kerr_schild_state(d["n_r"], d["n_theta"], d["n_phi"], d["r_in"], d["r_out"],
                                  n_fields=nf, amp=d["amp"], ell=d["ell"], seed=d["seed"])
    u = dev(u0)
    sh.init_gauge_from_state(u)
    v = torch.empty_like(u)
    sh.filter(u, v)
    return sh, v


def test_batch_is_bitwise_the_lone_step(cf):
    descs = inputs.shell_batch(6, seed=1)
    precs = [cf.MIXED, cf.FP64, cf.MIXED, cf.MIXED, cf.FP64, cf.MIXED]
    nfs = [50, 50, 54, 50, 58, 50]
    shells, us = [], []
    for d, p, nf in zip(descs, precs, nfs):
        sh, v = make(cf, d, p, nf)
        shells.append(sh)
        us.append(v)
    alone = [u.clone() for u in us]
    dts = [0.5 * sh.default_dt() for sh in shells]
    b = cf.Batch(shells)
    b.rk4_step(us, dts, n_steps=3)
    for sh, u, dt in zip(shells, alone, dts):
        sh.rk4_step(u, dt, 3)
    torch.cuda.synchronize()
    for i, (x, y) in enumerate(zip(us, alone)):
        assert torch.equal(x, y), i
        assert torch.isfinite(x).all()
    # a second call replays the captured graph; default dt (None) recaptures
    b.rk4_step(us, dts, n_steps=2)
    b.rk4_step(us, None, n_steps=1)
    for sh, u, dt in zip(shells, alone, dts):
        sh.rk4_step(u, dt, 2)
        sh.rk4_step(u, 0.0, 1)
    torch.cuda.synchronize()
    for i, (x, y) in enumerate(zip(us, alone)):
        assert torch.equal(x, y), i
    b.destroy()
    for sh in shells:
        sh.destroy()


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_matches_the_oracle(cf, prec):
    descs = [dict(n_r=9, n_theta=12, n_phi=24, r_in=1.8, r_out=11.0, L=10, amp=1e-6, ell=2, seed=0),
             dict(n_r=13, n_theta=9, n_phi=18, r_in=1.8, r_out=11.0, L=6, amp=1e-5, ell=2, seed=1),
             dict(n_r=9, n_theta=8, n_phi=16, r_in=1.8, r_out=11.0, L=6, amp=1e-4, ell=2, seed=2)]
    shells, us, refs = [], [], []
    for d in descs:
        sh, v = make(cf, d, prec)
        shells.append(sh)
        us.append(v)
        rs = oracle.OracleShell(d["n_r"], d["n_theta"], d["n_phi"], d["r_in"], d["r_out"], d["L"])
        u0 = inputs.kerr_schild_state(d["n_r"], d["n_theta"], d["n_phi"], d["r_in"], d["r_out"],
                                      amp=d["amp"], ell=d["ell"], seed=d["seed"])
        rs.init_gauge_from_state(u0)
        refs.append(rs.rk4_step(rs.filter(u0), 0.25 * rs.dx_min(), 4))
    b = cf.Batch(shells)
    b.rk4_step(us, None, n_steps=4)
    for u, ref in zip(us, refs):
        got = u.cpu().numpy()
        e = np.abs(got - ref).max() / np.abs(ref).max()
        assert e < (1e-12 if prec == 0 else 1e-8), e
    b.destroy()
    for sh in shells:
        sh.destroy()


def test_batch_names_the_shell_with_a_nonfinite_state(cf):
    descs = inputs.shell_batch(3, seed=2)
    shells, us = [], []
    for d in descs:
        sh, v = make(cf, d, cf.MIXED)
        shells.append(sh)
        us.append(v)
    us[1][12, 3, 2, 1] = float("nan")
    b = cf.Batch(shells)
    with pytest.raises(cf.CffynError) as ei:
        b.rk4_step(us, None, n_steps=1)
    assert ei.value.code == cf.ENONFINITE
    assert "shell 1" in str(ei.value)
    # the batch and the context stay usable
    us[1].copy_(make(cf, descs[1], cf.MIXED)[1])
    b.rk4_step(us, None, n_steps=1)
    b.destroy()
    for sh in shells:
        sh.destroy()


def test_batch_argument_errors(cf):
    d = inputs.shell_batch(2, seed=3)
    sh0, u0 = make(cf, d[0], cf.MIXED)
    sh1 = cf.Shell(d[1]["n_r"], d[1]["n_theta"], d[1]["n_phi"], 1.8, 11.0, d[1]["L"])
    u1 = dev(inputs.kerr_schild_state(d[1]["n_r"], d[1]["n_theta"], d[1]["n_phi"], 1.8, 11.0))
    with pytest.raises(cf.CffynError) as ei:
        cf.Batch([sh0, sh0])
    assert ei.value.code == cf.EINVAL
    b = cf.Batch([sh0, sh1])
    before = u0.clone()
    with pytest.raises(cf.CffynError) as ei:   # shell 1 has no gauge yet
        b.rk4_step([u0, u1], None, 1)
    assert ei.value.code == cf.EINVAL and "shell 1" in str(ei.value)
    torch.cuda.synchronize()
    assert torch.equal(u0, before)   # nothing was enqueued
    sh1.init_gauge_from_state(u1)
    b.rk4_step([u0, u1], None, 1)
    b.destroy()
    sh0.destroy()
    sh1.destroy()


@pytest.mark.parametrize("prec,nf", [(1, 50), (0, 50), (1, 58)])
def test_stacked_classes_are_bitwise_the_lone_step(cf, prec, nf):
    # three shells of one shape, two of another and one alone: three classes,
    # each stepped by one stacked handle; results equal lone steps bit for bit
    shapes = [(9, 12, 24, 10), (13, 8, 16, 6), (9, 12, 24, 10), (9, 12, 24, 10), (13, 8, 16, 6), (5, 6, 12, 4)]
    shells, us = [], []
    for k, (n_r, N, J, L) in enumerate(shapes):
        sh = cf.Shell(n_r, N, J, 1.8, 11.0, L, n_fields=nf, precision=prec)
        u = torch.from_numpy(inputs.kerr_schild_state(n_r, N, J, 1.8, 11.0, n_fields=nf, amp=1e-4 * (k + 1),
                                                      ell=2, seed=k)).cuda()
        sh.init_gauge_from_state(u)
        v = torch.empty_like(u)
        sh.filter(u, v)
        shells.append(sh)
        us.append(v)
    alone = [u.clone() for u in us]
    b = cf.Batch(shells)
    assert b.units() == 3
    b.rk4_step(us, None, 3)
    for sh, u in zip(shells, alone):
        sh.rk4_step(u, 0.0, 3)
    torch.cuda.synchronize()
    for i, (x, y) in enumerate(zip(us, alone)):
        assert torch.isfinite(x).all()
        assert torch.equal(x, y), i
    # one class needs one step size
    dts = [sh.default_dt() for sh in shells]
    dts[2] *= 0.5
    with pytest.raises(cf.CffynError) as ei:
        b.rk4_step(us, dts, 1)
    assert ei.value.code == cf.EINVAL
    b.destroy()
    for sh in shells:
        sh.destroy()
