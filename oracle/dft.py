"""Real discrete Fourier transform as matrices (paper Sec. 3.1).

Test infrastructure only (see ``oracle/__init__``).

J = 2M sampling points phi_j = 2 pi j / J.  Synthesis f = A a + B b with
A_jm = cos(2 pi j m / J) (m = 0..M-1) and B_jm = sin(2 pi j m / J)
(m = 1..M-1); analysis a = A~ f, b = B~ f with A~_0j = 1/J,
A~_mj = (2/J) A_jm, B~_mj = (2/J) B_jm.  The Nyquist mode m = M is dropped.

Reading: eq. Fsynthesis prints B_jm with a cosine; eqs. Fsynthesis0 and
Fanalysis0 fix it as the sine.

Parity pins (tests/test_oracle_swsh.py): analysis after synthesis is the
identity on the (J-1) retained real modes; analysis of single cos/sin modes
gives unit coefficients.
"""

import numpy as np


def real_dft_matrices(J):
    """Returns (A [J x M], B [J x (M-1)], At [M x J], Bt [(M-1) x J])."""
    assert J % 2 == 0
    M = J // 2
    j = np.arange(J)[:, None]
    A = np.cos(2.0 * np.pi * j * np.arange(M)[None, :] / J)
    B = np.sin(2.0 * np.pi * j * np.arange(1, M)[None, :] / J)
    At = (2.0 / J) * A.T
    At[0, :] = 1.0 / J
    Bt = (2.0 / J) * B.T
    return A, B, At, Bt
