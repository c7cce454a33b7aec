"""The FFT derivative path (cffyn_derivs_fft, the alternative of Sec. 5 /
Fig. mmfft) through the C-ABI: Cartesian derivatives against the oracle's
matrix derivatives (eqs. D1-D3 and dvdx) and against the FP64 matrix path,
FP64 tolerance 1e-12 relative on small and odd grids; on the benchmarked
33 x 48 x 96 shell and the 65 x 96 x 192 shell with 58 fields (whose theta
gather needs more than 48 KB of shared memory) the bound carries the chain
rule's polar factor (see the test)."""

import numpy as np
import pytest

import oracle
from paper_1104_3408_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def cf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1104_3408_gb300 import cffyn
    return cffyn


def rel(got, ref):
    return np.abs(got - ref).max() / np.abs(ref).max()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n_r,N,J", [(9, 12, 24), (13, 9, 18), (5, 6, 12), (33, 32, 64), (3, 2, 4)])
def test_fft_derivatives_match_oracle(cf, prec, n_r, N, J):
    u0 = inputs.band_limited_fields(n_r, N, J, 1.8, 11.0, seed=7)
    sh = cf.Shell(n_r, N, J, 1.8, 11.0, max(N - 2, 0), precision=prec)
    u = torch.from_numpy(u0).cuda()
    out = torch.empty((3,) + tuple(u.shape), dtype=torch.float64, device="cuda")
    sh.derivs_fft(u, out)
    first = out.cpu().numpy()
    ref = oracle.OracleShell(n_r, N, J, 1.8, 11.0, 0).derivs(u0)
    for d in range(3):
        assert rel(first[d], ref[d]) < TOL, (d, rel(first[d], ref[d]))
    # the second call reuses the plans and gives the same bits
    out.zero_()
    sh.derivs_fft(u, out)
    assert np.array_equal(out.cpu().numpy(), first)
    sh.destroy()


@pytest.mark.parametrize("n_r,N,J,nv,r_out", [(33, 48, 96, 50, 11.0), (65, 96, 192, 58, 41.0)],
                         ids=["33x48x96", "65x96x192_58f"])
def test_fft_derivatives_match_fp64_matrices_full_size(cf, n_r, N, J, nv, r_out):
    # Near the poles the chain rule (eq. dvdx) multiplies the phi derivative by
    # up to 1 / (r_in sin theta_0): 17 on 33 x 48 x 96, 34 on 65 x 96 x 192.
    # Two FP64 spectral derivatives of these fields differ by a few 1e-12 of
    # their scale (rounding only), so the Cartesian bound carries that factor.
    tol = 4e-12 / (1.8 * np.sin(np.pi / (2 * N)))
    u0 = inputs.kerr_schild_state(n_r, N, J, 1.8, r_out, n_fields=nv, amp=1e-4, ell=4, seed=0)
    sh = cf.Shell(n_r, N, J, 1.8, r_out, N - 2, n_fields=nv, precision=cf.FP64)
    u = torch.from_numpy(u0).cuda()
    a = torch.empty((3,) + tuple(u.shape), dtype=torch.float64, device="cuda")
    b = torch.empty_like(a)
    sh.derivs(u, a)
    sh.derivs_fft(u, b)
    for d in range(3):
        scale = float(a[d].abs().max())
        assert float((a[d] - b[d]).abs().max()) < tol * scale
    # and the oracle on a few fields
    ref = oracle.OracleShell(n_r, N, J, 1.8, r_out, 0, n_fields=50).derivs(u0[:3])
    got = b[:, :3].cpu().numpy()
    assert rel(got, ref) < tol
    sh.destroy()


def test_fft_derivatives_argument_errors(cf):
    sh = cf.Shell(9, 12, 24, 1.8, 11.0, 10)
    u = torch.zeros((50, 24, 12, 9), dtype=torch.float64, device="cuda")
    lib = cf.load()
    assert lib.cffyn_derivs_fft(None, None, None, None) == cf.EINVAL
    rc = lib.cffyn_derivs_fft(sh.h, cf.ctypes.c_void_p(u.data_ptr() + 8),
                              cf.ctypes.c_void_p(u.data_ptr()), None)
    assert rc == cf.EINVAL
    sh.destroy()
