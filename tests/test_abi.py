"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/cffyn.h declares; argument checks run on the host.  No GPU needed
(no compute call is made)."""

import ctypes
import os
import re

import pytest

from paper_1104_3408_gb300 import _build, cffyn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return cffyn.load()


def _declared():
    with open(os.path.join(ROOT, "include", "cffyn.h")) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"CFFYN_API\s+[\w\s\*]+?\b(cffyn_\w+)\s*\(", text)))


def test_header_declares_the_binding_names():
    names = _declared()
    assert names == sorted(cffyn.EXPORTED)


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_version_and_error_strings(lib):
    assert b"sm_103a" in lib.cffyn_version()
    assert isinstance(lib.cffyn_last_error(), bytes)


@pytest.mark.parametrize("bad", [
    dict(n_r=2), dict(n_theta=1, n_phi=2), dict(n_phi=30), dict(r_in=0.0), dict(r_out=1.0),
    dict(L=12), dict(L=-1), dict(precision=7), dict(filter_mode=3), dict(n_fields=49),
    dict(n_theta=97, n_phi=194),
])
def test_create_rejects_bad_arguments_on_host(lib, bad):
    kw = dict(n_r=9, n_theta=12, n_phi=24, r_in=1.8, r_out=11.0, L=10, n_fields=50,
              precision=cffyn.MIXED, filter_mode=cffyn.FILTER_SUBSTEP, courant=0.25)
    kw.update(bad)
    desc = cffyn.ShellDesc(kw["n_r"], kw["n_theta"], kw["n_phi"], kw["r_in"], kw["r_out"],
                           kw["L"], kw["n_fields"], kw["precision"], kw["filter_mode"],
                           kw["courant"])
    h = ctypes.c_void_p(1)
    rc = lib.cffyn_create_shell_ex(ctypes.byref(desc), ctypes.byref(h))
    assert rc == cffyn.EINVAL
    assert h.value is None
    assert len(lib.cffyn_last_error()) > 0


def test_null_handles_are_rejected(lib):
    assert lib.cffyn_destroy(None) == cffyn.OK
    assert lib.cffyn_rhs(None, None, None, None) == cffyn.EINVAL
    assert lib.cffyn_filter(None, None, None, None) == cffyn.EINVAL
    assert lib.cffyn_rk4_step(None, None, 0.1, 1, None) == cffyn.EINVAL
    assert lib.cffyn_rk4_step_async(None, None, 0.1, 1, None, None) == cffyn.EINVAL
    assert lib.cffyn_create_shell_ex(None, None) == cffyn.EINVAL
    assert lib.cffyn_derivs_fft(None, None, None, None) == cffyn.EINVAL
    assert b"NULL" in lib.cffyn_last_error()
    assert lib.cffyn_set_wait_limit(None, 1.0) == cffyn.EINVAL
    assert b"NULL" in lib.cffyn_last_error()
    assert lib.cffyn_create_nest(2, None, None) == cffyn.EINVAL
    assert lib.cffyn_nest_rhs(None, None, None, None) == cffyn.EINVAL
    assert lib.cffyn_nest_rk4_step(None, None, 0.1, 1, None) == cffyn.EINVAL
    assert lib.cffyn_destroy_nest(None) == cffyn.OK


def test_static_scratch_limit_and_null_shell(lib):
    with open(os.path.join(ROOT, "include", "cffyn.h")) as fh:
        m = re.search(r"#define CFFYN_STATIC_SCRATCH_BYTES \((\d+)u \* (\d+)u \* (\d+)u\)", fh.read())
    assert m and int(m[1]) * int(m[2]) * int(m[3]) == cffyn.STATIC_SCRATCH_BYTES
    assert lib.cffyn_derivs_static(None, None, 1, None, None) == cffyn.EINVAL
    assert b"NULL" in lib.cffyn_last_error()


def test_profile_phase_names_match_the_header():
    with open(os.path.join(ROOT, "include", "cffyn.h")) as fh:
        n = int(re.search(r"#define CFFYN_PROFILE_PHASES (\d+)", fh.read())[1])
    assert len(cffyn.PROFILE_PHASES) == n == len(set(cffyn.PROFILE_PHASES))


def test_batch_arguments_are_checked_on_host(lib):
    out = ctypes.c_void_p(1)
    assert lib.cffyn_create_batch(0, None, ctypes.byref(out)) == cffyn.EINVAL
    assert out.value is None
    assert lib.cffyn_create_batch(1, None, None) == cffyn.EINVAL
    assert lib.cffyn_batch_rk4_step(None, None, None, 1, None) == cffyn.EINVAL
    assert b"batch" in lib.cffyn_last_error()
    assert lib.cffyn_destroy_batch(None) == cffyn.OK


@pytest.mark.parametrize("field,value,code", [
    ("flags", 2, cffyn.EINVAL), ("filter_kind", 7, cffyn.EINVAL), ("filter_kind", -1, cffyn.EINVAL),
])
def test_create_checks_filter_kind_and_flags_on_host(lib, field, value, code):
    desc = cffyn.ShellDesc(9, 12, 24, 1.8, 11.0, 10, 50, cffyn.MIXED, cffyn.FILTER_SUBSTEP, 0.25)
    setattr(desc, field, value)
    h = ctypes.c_void_p(1)
    assert lib.cffyn_create_shell_ex(ctypes.byref(desc), ctypes.byref(h)) == code
    assert h.value is None


def test_workspace_calls_reject_null_shell(lib):
    assert lib.cffyn_workspace_size(None) == 0
    assert lib.cffyn_attach_workspace(None, None, 0) == cffyn.EINVAL


def test_step_status_words(lib):
    # the status word of cffyn_rk4_step_async: bit 0 a non-finite stage
    # right-hand side, bit 1 a bounded tensor-core wait that gave up (the
    # timeout wins when both are set); host-side decoding only
    assert lib.cffyn_step_status(0) == cffyn.OK
    assert lib.cffyn_step_status(1) == cffyn.ENONFINITE
    assert b"non-finite" in lib.cffyn_last_error()
    assert lib.cffyn_step_status(2) == cffyn.ETIMEOUT
    assert b"gave up" in lib.cffyn_last_error()
    assert lib.cffyn_step_status(3) == cffyn.ETIMEOUT
    cffyn.check_status(0)
    with pytest.raises(cffyn.CffynError) as ei:
        cffyn.check_status(1)
    assert ei.value.code == cffyn.ENONFINITE
