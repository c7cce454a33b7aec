"""Thin ctypes binding of libcffyn.so (include/cffyn.h).

Argument marshalling only: every step of the method runs in the CUDA
library.  Device memory and streams come from PyTorch: arrays are contiguous
float64 CUDA tensors in the layout u[mu, n_phi, n_theta, n_r]; the stream is
torch's current stream unless one is passed.  If the library is missing the
calls raise -- there is no CPU fallback.
"""

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libcffyn.so")

OK, EINVAL, ENOMEM, ECUDA, ENONFINITE, ETIMEOUT, ENOTIMPL = 0, -1, -2, -3, -4, -5, -6
FP64, MIXED = 0, 1
FILTER_SUBSTEP, FILTER_STEP = 0, 1
FILTER_YN, FILTER_Y, FILTER_YG = 0, 1, 2
DEFER_WORKSPACE = 1
STATIC_SCRATCH_BYTES = 8 * 1024 * 1024   # CFFYN_STATIC_SCRATCH_BYTES

EXPORTED = [
    "cffyn_create_shell", "cffyn_create_shell_ex", "cffyn_destroy", "cffyn_device_bytes",
    "cffyn_default_dt", "cffyn_set_gauge", "cffyn_init_gauge_from_state", "cffyn_derivs",
    "cffyn_rhs", "cffyn_filter", "cffyn_rk4_step", "cffyn_rk4_step_async", "cffyn_step_status",
    "cffyn_constraint_norms",
    "cffyn_get_filter_matrix", "cffyn_get_operator", "cffyn_last_error", "cffyn_version",
    "cffyn_profile_step", "cffyn_set_trace", "cffyn_get_trace", "cffyn_derivs_static",
    "cffyn_set_wait_limit", "cffyn_set_operator_rows", "cffyn_get_operator_rows",
    "cffyn_create_batch", "cffyn_batch_rk4_step", "cffyn_destroy_batch", "cffyn_batch_units",
    "cffyn_create_nest", "cffyn_nest_rhs", "cffyn_nest_rk4_step", "cffyn_nest_default_dt",
    "cffyn_destroy_nest",
    "cffyn_workspace_size", "cffyn_attach_workspace", "cffyn_derivs_fft",
]
PROFILE_PHASES = ["d_r", "d_theta_phi", "rhs_gamma", "rhs_quad", "rhs_pp", "decompose",
                  "dft_fwd", "project", "dft_inv", "reconstruct", "field_exp"]


class ShellDesc(ctypes.Structure):
    _fields_ = [
        ("n_r", ctypes.c_int), ("n_theta", ctypes.c_int), ("n_phi", ctypes.c_int),
        ("r_in", ctypes.c_double), ("r_out", ctypes.c_double), ("L", ctypes.c_int),
        ("n_fields", ctypes.c_int), ("precision", ctypes.c_int), ("filter_mode", ctypes.c_int),
        ("courant", ctypes.c_double), ("filter_kind", ctypes.c_int), ("flags", ctypes.c_int),
    ]


class CffynError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"cffyn error {code}: {msg}")
        self.code = code


_lib = None


def load(path=LIB_PATH):
    """Load libcffyn.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} not found: build it with __graft_entry__.build() "
                           "(paper_1104_3408_gb300._build.build())")
    lib = ctypes.CDLL(path)
    vp, dp, i, d = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "cffyn_create_shell": ([i, i, i, d, d, i, ctypes.POINTER(vp)], i),
        "cffyn_create_shell_ex": ([ctypes.POINTER(ShellDesc), ctypes.POINTER(vp)], i),
        "cffyn_destroy": ([vp], i),
        "cffyn_device_bytes": ([vp], ctypes.c_size_t),
        "cffyn_workspace_size": ([vp], ctypes.c_size_t),
        "cffyn_attach_workspace": ([vp, vp, ctypes.c_size_t], i),
        "cffyn_default_dt": ([vp], d),
        "cffyn_set_gauge": ([vp, dp, vp], i),
        "cffyn_init_gauge_from_state": ([vp, dp, vp], i),
        "cffyn_derivs": ([vp, dp, dp, vp], i),
        "cffyn_derivs_static": ([vp, dp, i, dp, vp], i),
        "cffyn_set_wait_limit": ([vp, d], i),
        "cffyn_set_operator_rows": ([vp, i, i], i),
        "cffyn_get_operator_rows": ([vp, i], i),
        "cffyn_derivs_fft": ([vp, dp, dp, vp], i),
        "cffyn_rhs": ([vp, dp, dp, vp], i),
        "cffyn_filter": ([vp, dp, dp, vp], i),
        "cffyn_rk4_step": ([vp, dp, d, i, vp], i),
        "cffyn_rk4_step_async": ([vp, dp, d, i, vp, vp], i),
        "cffyn_step_status": ([i], i),
        "cffyn_constraint_norms": ([vp, dp, ctypes.POINTER(ctypes.c_double), vp], i),
        "cffyn_get_filter_matrix": ([vp, i, i, ctypes.POINTER(ctypes.c_double)], i),
        "cffyn_get_operator": ([vp, i, ctypes.POINTER(ctypes.c_double)], i),
        "cffyn_profile_step": ([vp, dp, d, ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_int), vp], i),
        "cffyn_set_trace": ([vp, i], i),
        "cffyn_get_trace": ([vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int),
                             ctypes.POINTER(ctypes.c_longlong)], i),
        "cffyn_create_batch": ([i, ctypes.POINTER(vp), ctypes.POINTER(vp)], i),
        "cffyn_batch_rk4_step": ([vp, ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_double), i, vp], i),
        "cffyn_destroy_batch": ([vp], i),
        "cffyn_batch_units": ([vp], i),
        "cffyn_create_nest": ([i, ctypes.POINTER(vp), ctypes.POINTER(vp)], i),
        "cffyn_nest_rhs": ([vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp], i),
        "cffyn_nest_rk4_step": ([vp, ctypes.POINTER(vp), d, i, vp], i),
        "cffyn_nest_default_dt": ([vp], d),
        "cffyn_destroy_nest": ([vp], i),
        "cffyn_last_error": ([], ctypes.c_char_p),
        "cffyn_version": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(rc):
    if rc != OK:
        raise CffynError(rc, load().cffyn_last_error().decode())
    return rc


def check_status(status):
    """Raise CffynError if a step status word (see Shell.rk4_step_async) is
    not CFFYN_OK; status: an int32 CPU tensor or an int."""
    words = status.tolist() if hasattr(status, "tolist") else [status]
    for w in (words if isinstance(words, list) else [words]):
        _check(load().cffyn_step_status(int(w)))


def _ptr(t, what):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
        raise TypeError(f"{what} must be a float64 CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Shell:
    """One spherical shell (a cffyn_shell handle)."""

    def __init__(self, n_r, n_theta, n_phi, r_in, r_out, L, n_fields=50, precision=MIXED,
                 filter_mode=FILTER_SUBSTEP, courant=0.25, filter_kind=FILTER_YN, flags=0):
        lib = load()
        desc = ShellDesc(n_r, n_theta, n_phi, r_in, r_out, L, n_fields, precision, filter_mode,
                         courant, filter_kind, flags)
        self._workspace = None
        h = ctypes.c_void_p()
        _check(lib.cffyn_create_shell_ex(ctypes.byref(desc), ctypes.byref(h)))
        self.h = h
        self.n_r, self.n_theta, self.n_phi = n_r, n_theta, n_phi
        self.r_in, self.r_out, self.L = r_in, r_out, L
        self.n_fields, self.precision, self.filter_mode = n_fields, precision, filter_mode

    @property
    def shape(self):
        return (self.n_fields, self.n_phi, self.n_theta, self.n_r)

    def destroy(self):
        if self.h:
            load().cffyn_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def device_bytes(self):
        return load().cffyn_device_bytes(self.h)

    def workspace_size(self):
        return load().cffyn_workspace_size(self.h)

    def attach_workspace(self, buf):
        """Use `buf` (a contiguous CUDA tensor of at least workspace_size()
        bytes, 256-byte aligned) as the shell's workspace; None returns to a
        library-allocated one.  The Shell keeps a reference to buf."""
        if buf is None:
            _check(load().cffyn_attach_workspace(self.h, None, 0))
        else:
            import torch
            if not isinstance(buf, torch.Tensor) or not buf.is_cuda or not buf.is_contiguous():
                raise TypeError("workspace must be a contiguous CUDA tensor")
            _check(load().cffyn_attach_workspace(self.h, ctypes.c_void_p(buf.data_ptr()),
                                                 buf.numel() * buf.element_size()))
        self._workspace = buf

    def default_dt(self):
        return load().cffyn_default_dt(self.h)

    def set_gauge(self, H, stream=None):
        _check(load().cffyn_set_gauge(self.h, _ptr(H, "H"), _stream(stream)))

    def init_gauge_from_state(self, u, stream=None):
        _check(load().cffyn_init_gauge_from_state(self.h, _ptr(u, "u"), _stream(stream)))

    def derivs(self, u, out, stream=None):
        _check(load().cffyn_derivs(self.h, _ptr(u, "u"), _ptr(out, "dxyz"), _stream(stream)))
        return out

    def derivs_fft(self, u, out, stream=None):
        """Cartesian derivatives like derivs(), by FFTs (cuFFT, FP64); the
        first call makes the plans and allocates their scratch."""
        _check(load().cffyn_derivs_fft(self.h, _ptr(u, "u"), _ptr(out, "dxyz"), _stream(stream)))
        return out

    def derivs_static(self, u, n_f, out, stream=None):
        """Cartesian derivatives of the first n_f fields of u into out
        ([3][n_f][P]) with no allocation: intermediates in the library's
        fixed STATIC_SCRATCH_BYTES device array (see cffyn_derivs_static)."""
        _check(load().cffyn_derivs_static(self.h, _ptr(u, "u"), int(n_f), _ptr(out, "dxyz"),
                                          _stream(stream)))
        return out

    def rhs(self, u, out, stream=None):
        _check(load().cffyn_rhs(self.h, _ptr(u, "u"), _ptr(out, "dudt"), _stream(stream)))
        return out

    def filter(self, u, out, stream=None):
        _check(load().cffyn_filter(self.h, _ptr(u, "u"), _ptr(out, "out"), _stream(stream)))
        return out

    def rk4_step(self, u, dt=0.0, n_steps=1, stream=None):
        _check(load().cffyn_rk4_step(self.h, _ptr(u, "u"), float(dt), int(n_steps), _stream(stream)))
        return u

    def rk4_step_async(self, u, status, dt=0.0, n_steps=1, stream=None):
        """Enqueue n_steps RK4 steps on the stream and return; the steps'
        status word lands in status (an int32 CPU tensor, pinned for the copy
        to stay asynchronous) in stream order: check_status(status) after
        synchronising."""
        import torch
        if status.is_cuda or status.dtype != torch.int32 or status.numel() < 1:
            raise TypeError("status must be an int32 CPU tensor")
        _check(load().cffyn_rk4_step_async(self.h, _ptr(u, "u"), float(dt), int(n_steps), _stream(stream),
                                           ctypes.c_void_p(status.data_ptr())))
        return u

    def profile_step(self, u, dt=0.0, stream=None):
        """Per-phase device ms and launch counts of one eager RK4 step."""
        n = len(PROFILE_PHASES)
        ms = (ctypes.c_double * n)()
        la = (ctypes.c_int * n)()
        _check(load().cffyn_profile_step(self.h, _ptr(u, "u"), float(dt), ms, la, _stream(stream)))
        return {k: (float(ms[i]), int(la[i])) for i, k in enumerate(PROFILE_PHASES)}

    def set_operator_rows(self, family, rows):
        """Row-group size (0, 48, 96) of an operator family (0 d_r, 1 d_theta +
        d_phi, 2 phi analysis, 3 projections, 4 phi synthesis)."""
        _check(load().cffyn_set_operator_rows(self.h, int(family), int(rows)))

    def get_operator_rows(self, family):
        return int(load().cffyn_get_operator_rows(self.h, int(family)))

    def set_wait_limit(self, seconds):
        """Bound (s) of the tensor-core kernels' waits; < 0 restores 1 s, 0
        gives up at once (cffyn_set_wait_limit)."""
        _check(load().cffyn_set_wait_limit(self.h, float(seconds)))

    def set_trace(self, on=True):
        _check(load().cffyn_set_trace(self.h, 1 if on else 0))

    def get_trace(self):
        """({group: total ms}, {group: launches per step}, traced steps)."""
        n = len(PROFILE_PHASES)
        ms = (ctypes.c_double * n)()
        la = (ctypes.c_int * n)()
        st = ctypes.c_longlong()
        _check(load().cffyn_get_trace(self.h, ms, la, ctypes.byref(st)))
        return ({k: float(ms[i]) for i, k in enumerate(PROFILE_PHASES)},
                {k: int(la[i]) for i, k in enumerate(PROFILE_PHASES)}, int(st.value))

    def constraint_norms(self, u, stream=None):
        out = (ctypes.c_double * 2)()
        _check(load().cffyn_constraint_norms(self.h, _ptr(u, "u"), out, _stream(stream)))
        return float(out[0]), float(out[1])

    def get_filter_matrix(self, n, m):
        import numpy as np
        a = np.zeros((self.n_theta, self.n_theta))
        _check(load().cffyn_get_filter_matrix(self.h, n, m,
                                              a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return a

    def get_operator(self, which):
        import numpy as np
        shapes = {0: (self.n_r, self.n_r), 1: (self.n_theta, 2 * self.n_theta),
                  2: (self.n_phi, self.n_phi)}
        a = np.zeros(shapes[which])
        _check(load().cffyn_get_operator(self.h, which,
                                         a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return a


class HostStepper:
    """RK4 steps of independent states held in pinned host memory, with the
    host <-> device copies overlapped with the steps.

    stepper is a Shell (one state per problem; like: a device tensor of the
    state's shape) or a Batch (one state per member shell; like: the list of
    the members' device states).  run(host_ins, host_outs, dt) steps every
    problem host_ins[i] once (n_steps RK4 steps) and writes the result into
    host_outs[i]; for a Batch each problem is a list of the members' host
    states and dt the members' dts (None: each shell's default).  While
    problem i steps on the given stream, problem i + 1 is copied in on a copy
    stream and the result of problem i - 1 is copied out on another, so a
    sequence of problems costs about the steps alone plus one copy in and one
    out.

    A Shell alternates two device state buffers (the shell keeps a step
    graph for each) and enqueues its steps with cffyn_rk4_step_async, so the
    host queues every problem's work without waiting and the copies go
    straight to and from the buffer being stepped.  A Batch steps one fixed
    set of member buffers (its graphs are captured for one set), with two
    staging sets between them and the copies, each moved with one
    device-to-device copy per problem; its step call synchronises and the
    neighbouring problems' copies run beside it.  run() synchronises once at
    the end and raises CffynError if any problem's steps reported an error.
    Marshalling only: every step is the library's.  Host states are float64
    CPU tensors of the device states' shapes, pinned for the copies to
    overlap."""

    def __init__(self, stepper, like):
        import torch
        self.sh = stepper
        self.batch = isinstance(stepper, Batch)
        likes = list(like) if self.batch else [like]
        if self.batch and len(likes) != len(stepper.shells):
            raise ValueError(f"{len(stepper.shells)} member states expected")
        for t in likes:
            if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
                raise TypeError("like must be float64 CUDA tensors of the states' shapes")
        self.shapes = [t.shape for t in likes]
        new = lambda: [torch.empty_like(t, memory_format=torch.contiguous_format) for t in likes]  # noqa: E731
        if self.batch:
            self.state, self.stage_in, self.stage_out = new(), new(), new()
        else:
            self.bufs = [new(), new()]
        dev = likes[0].device
        self.h2d = torch.cuda.Stream(device=dev)
        self.d2h = torch.cuda.Stream(device=dev)
        ev = lambda: [torch.cuda.Event(), torch.cuda.Event()]  # noqa: E731
        self.ev_in, self.ev_done, self.ev_free = ev(), ev(), ev()

    def _members(self, h):
        hs = list(h) if self.batch else [h]
        if len(hs) != len(self.shapes):
            raise ValueError(f"{len(self.shapes)} host states per problem expected")
        return hs

    @staticmethod
    def _copy(dst, src):
        for d, s_ in zip(dst, src):
            d.copy_(s_, non_blocking=True)

    def run(self, host_ins, host_outs, dt=None, n_steps=1, stream=None):
        import torch
        n = len(host_ins)
        if len(host_outs) != n:
            raise ValueError("one output per input expected")
        ins = [self._members(h) for h in host_ins]
        outs = [self._members(h) for h in host_outs]
        for prob in ins + outs:
            for t, shape in zip(prob, self.shapes):
                if t.is_cuda or t.dtype != torch.float64 or t.shape != shape:
                    raise TypeError("host states must be float64 CPU tensors of the states' shapes")
        if n == 0:
            return host_outs
        st = stream if stream is not None else torch.cuda.current_stream()
        self.h2d.wait_stream(st)
        self.d2h.wait_stream(st)
        status = torch.zeros(n, dtype=torch.int32).pin_memory()
        if self.batch:
            self._run_staged(ins, outs, dt, n_steps, st)
        else:
            self._run_alternating(ins, outs, 0.0 if dt is None else dt, n_steps, st, status)
        st.wait_stream(self.h2d)
        st.wait_stream(self.d2h)
        st.synchronize()
        check_status(status)
        return host_outs

    def _run_alternating(self, ins, outs, dt, n_steps, st, status):
        import torch
        for i in range(len(ins)):
            b = i % 2
            buf = self.bufs[b]
            # copy in once the copy out of problem i - 2 has read this buffer
            with torch.cuda.stream(self.h2d):
                self.h2d.wait_event(self.ev_free[b])
                self._copy(buf, ins[i])
                self.ev_in[b].record(self.h2d)
            st.wait_event(self.ev_in[b])
            self.sh.rk4_step_async(buf[0], status[i:i + 1], dt, n_steps, st)
            self.ev_done[b].record(st)
            with torch.cuda.stream(self.d2h):
                self.d2h.wait_event(self.ev_done[b])
                self._copy(outs[i], buf)
                self.ev_free[b].record(self.d2h)

    def _run_staged(self, ins, outs, dts, n_steps, st):
        import torch
        # ev_in[0]: stage_in holds the next problem; ev_done[0]: stage_in has
        # been moved into the state; ev_in[1]: stage_out holds the last
        # result; ev_free[1]: stage_out has been copied out
        with torch.cuda.stream(self.h2d):
            self._copy(self.stage_in, ins[0])
            self.ev_in[0].record(self.h2d)
        for i in range(len(ins)):
            st.wait_event(self.ev_in[0])
            with torch.cuda.stream(st):
                self._copy(self.state, self.stage_in)
            self.ev_done[0].record(st)
            if i + 1 < len(ins):
                # the next problem's copy in runs beside this step
                with torch.cuda.stream(self.h2d):
                    self.h2d.wait_event(self.ev_done[0])
                    self._copy(self.stage_in, ins[i + 1])
                    self.ev_in[0].record(self.h2d)
            self.sh.rk4_step(self.state, dts, n_steps, st)
            st.wait_event(self.ev_free[1])
            with torch.cuda.stream(st):
                self._copy(self.stage_out, self.state)
            self.ev_in[1].record(st)
            # this result's copy out runs beside the next step
            with torch.cuda.stream(self.d2h):
                self.d2h.wait_event(self.ev_in[1])
                self._copy(outs[i], self.stage_out)
                self.ev_free[1].record(self.d2h)


class Batch:
    """Independent shells advanced together (a cffyn_batch handle).  The
    batch borrows the Shell objects and keeps references to them."""

    def __init__(self, shells):
        self.shells = list(shells)
        arr = (ctypes.c_void_p * len(self.shells))(*[s.h.value for s in self.shells])
        h = ctypes.c_void_p()
        _check(load().cffyn_create_batch(len(self.shells), arr, ctypes.byref(h)))
        self.h = h

    def rk4_step(self, us, dts=None, n_steps=1, stream=None):
        n = len(self.shells)
        if len(us) != n:
            raise ValueError(f"{n} states expected")
        ptrs = (ctypes.c_void_p * n)(*[_ptr(u, "u[i]").value for u in us])
        dt_arr = None if dts is None else (ctypes.c_double * n)(*[float(d) for d in dts])
        _check(load().cffyn_batch_rk4_step(self.h, ptrs, dt_arr, int(n_steps), _stream(stream)))
        return us

    def units(self):
        """Independent branches of the step graph: the batch's shape classes."""
        return int(load().cffyn_batch_units(self.h))

    def destroy(self):
        if self.h:
            load().cffyn_destroy_batch(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class Nest:
    """Nested shells over consecutive radial intervals, coupled on their
    common spheres (a cffyn_nest handle); borrows the Shell objects."""

    def __init__(self, shells):
        self.shells = list(shells)
        arr = (ctypes.c_void_p * len(self.shells))(*[s.h.value for s in self.shells])
        h = ctypes.c_void_p()
        _check(load().cffyn_create_nest(len(self.shells), arr, ctypes.byref(h)))
        self.h = h

    def _ptrs(self, ts, what):
        n = len(self.shells)
        if len(ts) != n:
            raise ValueError(f"{n} arrays expected for {what}")
        return (ctypes.c_void_p * n)(*[_ptr(t, what).value for t in ts])

    def default_dt(self):
        return float(load().cffyn_nest_default_dt(self.h))

    def rhs(self, us, outs, stream=None):
        _check(load().cffyn_nest_rhs(self.h, self._ptrs(us, "u[i]"), self._ptrs(outs, "dudt[i]"),
                                     _stream(stream)))
        return outs

    def rk4_step(self, us, dt=0.0, n_steps=1, stream=None):
        _check(load().cffyn_nest_rk4_step(self.h, self._ptrs(us, "u[i]"), float(dt), int(n_steps),
                                          _stream(stream)))
        return us

    def destroy(self):
        if self.h:
            load().cffyn_destroy_nest(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


# C-ABI names, one to one (module-level functions taking a Shell)
def create_shell(n_r, n_theta, n_phi, r_in, r_out, L, **kw):
    return Shell(n_r, n_theta, n_phi, r_in, r_out, L, **kw)


def rhs(sh, u, out, stream=None):
    return sh.rhs(u, out, stream)


def filter(sh, u, out, stream=None):  # noqa: A001 - the C-ABI name
    return sh.filter(u, out, stream)


def rk4_step(sh, u, dt=0.0, n_steps=1, stream=None):
    return sh.rk4_step(u, dt, n_steps, stream)


def derivs(sh, u, out, stream=None):
    return sh.derivs(u, out, stream)


def derivs_fft(sh, u, out, stream=None):
    return sh.derivs_fft(u, out, stream)


def create_batch(shells):
    return Batch(shells)


def batch_rk4_step(b, us, dts=None, n_steps=1, stream=None):
    return b.rk4_step(us, dts, n_steps, stream)


def destroy_batch(b):
    b.destroy()


def destroy(sh):
    sh.destroy()


def version():
    return load().cffyn_version().decode()
