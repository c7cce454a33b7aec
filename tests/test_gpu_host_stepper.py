"""cffyn.HostStepper: RK4 steps of independent states held in pinned host
memory, with the host <-> device copies overlapped with the steps.  Each
result must be exactly what cffyn_rk4_step gives for that state on the
device (the same kernels and arithmetic; only the copies are scheduled
around them), and the last problem's result must not be left in flight."""

import numpy as np
import pytest

from paper_1104_3408_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cffyn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1104_3408_gb300 import cffyn
    return cffyn


def _states(n_r, N, J, n):
    return [inputs.kerr_schild_state(n_r, N, J, 1.8, 11.0, amp=10.0 ** (-3 - i), ell=2, seed=i) for i in range(n)]


@pytest.mark.parametrize("precision", ["MIXED", "FP64"])
def test_host_stepper_matches_device_steps(cffyn, precision):
    n_r, N, J, L = 9, 12, 24, 10
    sh = cffyn.Shell(n_r, N, J, 1.8, 11.0, L, precision=getattr(cffyn, precision))
    states = _states(n_r, N, J, 4)
    dev = torch.from_numpy(states[0]).cuda()
    sh.init_gauge_from_state(dev)
    dt = sh.default_dt()
    # reference: each state stepped on the device with the plain call
    want = []
    for s in states:
        v = torch.from_numpy(s).cuda()
        sh.rk4_step(v, dt, 2)
        want.append(v.cpu().numpy())
    hs = cffyn.HostStepper(sh, dev)
    hins = [torch.from_numpy(s).pin_memory() for s in states]
    houts = [torch.full_like(h, float("nan")).pin_memory() for h in hins]
    hs.run(hins, houts, dt, 2)
    torch.cuda.current_stream().synchronize()
    for got, ref in zip(houts, want):
        assert np.array_equal(got.numpy(), ref)
    # a second run through the same stepper (buffers and events reused)
    houts2 = [torch.full_like(h, float("nan")).pin_memory() for h in hins[::-1]]
    hs.run(hins[::-1], houts2, dt, 2)
    torch.cuda.current_stream().synchronize()
    for got, ref in zip(houts2, want[::-1]):
        assert np.array_equal(got.numpy(), ref)
    sh.destroy()


def test_host_stepper_rejects_bad_arguments(cffyn):
    sh = cffyn.Shell(9, 12, 24, 1.8, 11.0, 10)
    dev = torch.from_numpy(_states(9, 12, 24, 1)[0]).cuda()
    with pytest.raises(TypeError):
        cffyn.HostStepper(sh, dev.cpu())
    hs = cffyn.HostStepper(sh, dev)
    good = dev.cpu()
    with pytest.raises(TypeError):
        hs.run([good[:10]], [good.clone()], 0.0)
    with pytest.raises(TypeError):
        hs.run([dev], [good.clone()], 0.0)
    with pytest.raises(ValueError):
        hs.run([good], [], 0.0)
    assert hs.run([], [], 0.0) == []
    sh.destroy()


def test_host_stepper_over_a_batch(cffyn):
    # three shells, two of one shape (a stacked class) and one of another;
    # each problem is the list of the three members' states
    shapes = [(9, 12, 24, 10), (9, 12, 24, 10), (5, 6, 12, 4)]
    shells = [cffyn.Shell(n_r, N, J, 1.8, 11.0, L) for n_r, N, J, L in shapes]
    problems = []
    for q in range(3):
        problems.append([inputs.kerr_schild_state(n_r, N, J, 1.8, 11.0, amp=10.0 ** (-3 - q), ell=2,
                                                  seed=10 * q + i)
                         for i, (n_r, N, J, L) in enumerate(shapes)])
    devs = [torch.from_numpy(s).cuda() for s in problems[0]]
    for sh, d in zip(shells, devs):
        sh.init_gauge_from_state(d)
    b = cffyn.Batch(shells)
    want = []
    for prob in problems:
        vs = [torch.from_numpy(s).cuda() for s in prob]
        b.rk4_step(vs, None, 2)
        want.append([v.cpu().numpy() for v in vs])
    hs = cffyn.HostStepper(b, devs)
    hins = [[torch.from_numpy(s).pin_memory() for s in prob] for prob in problems]
    houts = [[torch.full_like(h, float("nan")).pin_memory() for h in prob] for prob in hins]
    hs.run(hins, houts, None, 2)
    for got, ref in zip(houts, want):
        for g, r in zip(got, ref):
            assert np.array_equal(g.numpy(), r)
    with pytest.raises(ValueError):
        hs.run([hins[0][:2]], [houts[0][:2]])
    b.destroy()
    for sh in shells:
        sh.destroy()
