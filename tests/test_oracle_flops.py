"""The operation counter of the oracle (oracle/flops.py) and the right-hand
side count per point that the benchmark's whole-step roofline uses.  CPU only."""

import numpy as np

import bench
from oracle import flops


def test_counter_on_known_expressions():
    a = np.ones((3, 3, 10)).view(flops._C)
    x = np.ones((3, 10)).view(flops._C)
    flops._STATE.ops = 0
    y = np.einsum("ijP,jP->iP", a, x)          # 90 products and their sums
    assert 2 * 90 - 30 <= flops._STATE.ops <= 2 * 90 + 1
    flops._STATE.ops = 0
    z = y * y + x                               # two ufunc calls of 30 elements
    assert flops._STATE.ops == 60 and isinstance(z, flops._C)
    flops._STATE.ops = 0
    np.linalg.inv(np.eye(4)[None].repeat(5, 0).view(flops._C))
    assert flops._STATE.ops == 5 * 2 * 64


def test_rhs_count_used_by_the_bench():
    n = flops.rhs_ops_per_point(P=16)
    assert abs(n - bench.RHS_OPS_PER_POINT) < 2.0
    # the paper quotes about 1e4 per point (Sec. 4.2): same order
    assert 3e3 < n < 2e4
