"""FP64 operation count of the oracle's pointwise GHG right-hand side.

Test infrastructure only (see ``oracle/__init__``): it runs
``ghg.rhs_pointwise`` (eqs. gdot, Phidot, Pidot with the 3+1 quantities of
eqs. normal, abgfromgab and the Christoffel symbols of eq. Gamma) on arrays of
a counting ndarray subclass and adds up

* one operation per output element of every arithmetic ufunc call (add,
  subtract, multiply, divide, sqrt, ...; negation and copies are free),
* numpy's own count for every einsum on the path it takes
  (``np.einsum_path(..., optimize=True)``: multiplications and additions of
  the contraction),
* 2 n^3 per n x n matrix inverse (LU factorisation and the inverse from it).

The count per point is the algorithmic work of the right-hand side that the
whole-step roofline divides by an ALU peak (the paper quotes about 10^4
floating point operations per point, Sec. 4.2).
"""

import re

import numpy as np

from . import ghg

_COUNTED = {np.add, np.subtract, np.multiply, np.divide, np.true_divide, np.sqrt, np.reciprocal,
            np.power, np.square}


class _Counter:
    def __init__(self):
        self.ops = 0


_STATE = _Counter()


def _unwrap(x):
    if isinstance(x, _C):
        return x.view(np.ndarray)
    if isinstance(x, (list, tuple)):
        return type(x)(_unwrap(v) for v in x)
    if isinstance(x, dict):
        return {k: _unwrap(v) for k, v in x.items()}
    return x


def _wrap(x):
    if isinstance(x, np.ndarray) and not isinstance(x, _C):
        return x.view(_C)
    if isinstance(x, tuple):
        return tuple(_wrap(v) for v in x)
    return x


class _C(np.ndarray):
    def __array_ufunc__(self, ufunc, method, *inputs, **kw):
        out = getattr(ufunc, method)(*_unwrap(inputs), **_unwrap(kw))
        if method == "__call__" and ufunc in _COUNTED:
            _STATE.ops += int(np.size(out))
        return _wrap(out)

    def __array_function__(self, func, types, args, kwargs):
        a, k = _unwrap(args), _unwrap(kwargs)
        if func is np.einsum:
            ops = [x for x in a[1:]]
            info = np.einsum_path(a[0], *ops, optimize=True)[1]
            _STATE.ops += int(float(re.search(r"Optimized FLOP count:\s*([0-9.eE+]+)", info).group(1)))
        elif func is np.linalg.inv:
            n = a[0].shape[-1]
            _STATE.ops += 2 * n ** 3 * int(np.prod(a[0].shape[:-2]))
        return _wrap(func(*a, **k))


class _NumpyCounting:
    """numpy as ``ghg`` sees it while counting: arrays it creates from shapes
    alone (empty, zeros, ones) are counting arrays too, so that values stored
    into them keep being counted."""

    def __getattr__(self, name):
        return getattr(np, name)

    @staticmethod
    def empty(*a, **k):
        return np.empty(*a, **k).view(_C)

    @staticmethod
    def zeros(*a, **k):
        return np.zeros(*a, **k).view(_C)

    @staticmethod
    def ones(*a, **k):
        return np.ones(*a, **k).view(_C)


def rhs_ops_per_point(n_fields=50, P=64, seed=0):
    """Operations of one right-hand side evaluation per point (eqs. gdot,
    Phidot, Pidot) on P points of a perturbed Kerr-Schild-like state."""
    rng = np.random.default_rng(seed)
    u = np.zeros((n_fields, P))
    u[0] = -1.0 + 0.1 * rng.random(P)
    u[4] = u[7] = u[9] = 1.0
    u += 0.01 * rng.standard_normal(u.shape)
    du = 0.01 * rng.standard_normal((3, n_fields, P))
    H = 0.01 * rng.standard_normal((4, P))
    dH = 0.01 * rng.standard_normal((3, 4, P))
    _STATE.ops = 0
    saved = ghg.np
    ghg.np = _NumpyCounting()
    try:
        out = ghg.rhs_pointwise(u.view(_C), du.view(_C), H.view(_C), dH.view(_C), n_fields)
    finally:
        ghg.np = saved
    if not isinstance(out, _C):
        raise RuntimeError("the right-hand side left the counting arrays")
    return _STATE.ops / P
