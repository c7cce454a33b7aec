/*
 * cffyn.h -- C-ABI of the GB300 (sm_103a) implementation of the Chebyshev /
 * double-Fourier pseudospectral method with the spin-weighted (Yn) tensor
 * filter on one spherical shell (Bruegmann, arXiv:1104.3408).
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 * Field arrays.  FP64, contiguous, device memory owned by the caller, at least
 * 16-byte aligned (256 recommended), laid out as the paper's linear 4-d index
 * (Sec. 2.4) with the single theta cover stored (Sec. 2.1):
 *     u[((mu * n_phi + j) * n_theta + i) * n_r + k]
 * k: radius (Chebyshev extrema, increasing r, eq. rk), i: theta (pole
 * staggered, eq. thetai), j: phi (eq. phij), mu: field.  The library never
 * frees or retains caller pointers.
 *
 * Fields (n_fields = 50, 54 or 58; App. A.1 eqs. gdot, Phidot, Pidot): the
 * symmetric pairs (tt,tx,ty,tz,xx,xy,xz,yy,yz,zz) of g_ab (fields 0..9),
 * Pi_ab (10..19), Phi_xab (20..29), Phi_yab (30..39), Phi_zab (40..49); then
 * H_a (50..53) and dH_a/dt (54..57) where present.  With 54 fields the
 * gauge source is evolved with d_t H_a = 0; with 58 fields d_t H_a = G_a
 * (fields 54..57) and d_t G_a = 0, and G_a enters eq. Pidot as the time
 * derivative of H_b in nabla_(a H_b).  The gauge fields are filtered like
 * the others (H_t a scalar, H_i a vector) and keep their right-hand sides on
 * the outermost sphere.
 *
 * Streams.  `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream).  Calls enqueue work and return; results are ready when the stream
 * is.  Exceptions: cffyn_create_*, cffyn_destroy and cffyn_constraint_norms
 * synchronise, cffyn_get_* copy to host synchronously.
 *
 * Errors.  Every call returns an int status (0 = CFFYN_OK, negative =
 * error) and never aborts, traps or throws.  cffyn_last_error() returns a
 * thread-local message for the last failing call on the calling thread.
 * CFFYN_ENONFINITE is reported by cffyn_rk4_step when its fused finiteness
 * check saw a NaN/Inf in a stage right-hand side (the state is then
 * meaningless but the context stays usable).
 *
 * Threading.  A shell handle is not thread-safe: serialise calls on one
 * handle.  Distinct handles are independent.
 */
#ifndef CFFYN_H
#define CFFYN_H

#include <stddef.h>

#if defined(__GNUC__)
#define CFFYN_API __attribute__((visibility("default")))
#else
#define CFFYN_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define CFFYN_OK 0
#define CFFYN_EINVAL (-1)    /* bad argument (sizes, null pointer, mode) */
#define CFFYN_ENOMEM (-2)    /* device allocation failed */
#define CFFYN_ECUDA (-3)     /* a CUDA runtime call failed */
#define CFFYN_ENONFINITE (-4)/* non-finite value seen by the step's check */
#define CFFYN_ETIMEOUT (-5)  /* a bounded device wait gave up */
#define CFFYN_ENOTIMPL (-6)  /* option not implemented */

/* Arithmetic of the operator applications and of the pointwise RHS. */
#define CFFYN_FP64 0   /* FP64 CUDA-core arithmetic throughout */
#define CFFYN_MIXED 1  /* split-precision BF16 tensor-core products with exact
                          FP32 partial sums, recombined in 64-bit integers;
                          double-float (FP32 pair) pointwise arithmetic; FP64
                          state accumulation */

/* Where the Yn filter is applied (Sec. 2.5). */
#define CFFYN_FILTER_SUBSTEP 0 /* every stage right-hand side after the BC */
#define CFFYN_FILTER_STEP 1    /* the state after each full RK4 step (paper) */

/* Which filter (Sec. 3.5).  Yn: the tensor filter (triad decomposition,
 * projection of every spin-weight component with F^n_m).  Y: every field
 * projected as a scalar with F^0_m at the retained degree L.  Yg: the graded
 * Y filter of eq. nfofmu, n_f(mu) = n_f - d(u^mu): a field with d spatial
 * indices (g_tt 0, g_ti 1, g_ij 2, Phi_ijk 3, H_t 0, H_i 1) keeps
 * l <= min(L + d, n_theta - 1). */
#define CFFYN_FILTER_YN 0
#define CFFYN_FILTER_Y 1
#define CFFYN_FILTER_YG 2

/* cffyn_shell_desc.flags */
#define CFFYN_DEFER_WORKSPACE 1 /* allocate no workspace at creation: attach one
                                   with cffyn_attach_workspace before the first
                                   call that computes (CFFYN_EINVAL before) */

typedef struct cffyn_shell cffyn_shell;

typedef struct cffyn_shell_desc {
  int n_r;          /* radial points, >= 3 (eq. rk) */
  int n_theta;      /* theta points N, >= 2 (eq. thetai) */
  int n_phi;        /* phi points, must equal 2 * n_theta (Sec. 2.1) */
  double r_in;      /* inner radius, > 0 */
  double r_out;     /* outer radius, > r_in */
  int L;            /* retained spherical-harmonic degree, 0 <= L <= n_theta-1;
                       the filter keeps l <= L (n_f = n_theta-1-L, Sec. 3.5) */
  int n_fields;     /* 50, 54 or 58 (App. A.1) */
  int precision;    /* CFFYN_FP64 or CFFYN_MIXED */
  int filter_mode;  /* CFFYN_FILTER_SUBSTEP or CFFYN_FILTER_STEP */
  double courant;   /* lambda of dt = lambda * min dx (Sec. 4.1); <= 0 -> 0.25 */
  int filter_kind;  /* CFFYN_FILTER_YN (0), CFFYN_FILTER_Y or CFFYN_FILTER_YG */
  int flags;        /* 0 or CFFYN_DEFER_WORKSPACE */
} cffyn_shell_desc;

/* Builds a shell: collocation grid (Sec. 2.1), differentiation matrices
 * (Sec. 2.3), real DFT matrices (Sec. 3.1), spin-weighted synthesis matrices by
 * the recursion of eqs. Yninc/Yncoeffs/Ynnegative and the filter matrices
 * F^n_m = P^n_m f (P^n_m)^+ of eq. FasPfQ for n in [-3,3], m in [0,L], all in
 * FP64 on the current CUDA device, plus the library's workspace.
 * Defaults of cffyn_create_shell: 50 fields, CFFYN_MIXED, CFFYN_FILTER_SUBSTEP,
 * courant 0.25.  Synchronous.  Returns CFFYN_EINVAL for sizes outside the
 * ranges above (or n_theta > 96, n_r > 96), for an unknown filter kind or
 * flags, CFFYN_ENOMEM / CFFYN_ECUDA on device failures; *out is NULL on
 * error.  cffyn_create_shell takes filter_kind CFFYN_FILTER_YN and flags 0. */
CFFYN_API int cffyn_create_shell(int n_r, int n_theta, int n_phi, double r_in, double r_out, int L,
                       cffyn_shell** out);
CFFYN_API int cffyn_create_shell_ex(const cffyn_shell_desc* desc, cffyn_shell** out);

/* Frees the handle and its device memory (synchronises the device first).
 * NULL is allowed. */
CFFYN_API int cffyn_destroy(cffyn_shell* sh);

/* Workspace: the scratch arrays of one call (stage state, RK4 accumulator,
 * spherical derivatives / DFT coefficients, right-hand side and its source
 * terms, and on the mixed path the pair copy of the step's initial state);
 * nothing in it survives from one call to the next.  cffyn_workspace_size is
 * its size in bytes (8 or 7 arrays of n_fields x points doubles, each rounded
 * up to 256 bytes).  By default the library allocates it at creation. */
CFFYN_API size_t cffyn_workspace_size(const cffyn_shell* sh);

/* Makes `ptr` (device memory of the shell's device, 256-byte aligned, at
 * least cffyn_workspace_size bytes, caller-owned: the caller keeps it alive
 * and unused by other work until the shell is destroyed or another workspace
 * is attached) the shell's workspace, and frees the workspace the library
 * allocated, if any.  ptr == NULL gives the shell a library-allocated
 * workspace again.  Synchronises the device first (no call of this shell may
 * be in flight); drops the captured step graphs (the next cffyn_rk4_step
 * recaptures; so does a batch holding the shell).  Not during a stream
 * capture.  CFFYN_EINVAL for a misaligned or short buffer. */
CFFYN_API int cffyn_attach_workspace(cffyn_shell* sh, void* ptr, size_t bytes);

/* Bytes of device memory the handle owns (matrices, gauge, and the workspace
 * while it is library-allocated). */
CFFYN_API size_t cffyn_device_bytes(const cffyn_shell* sh);

/* dt = courant * min(r_1 - r_0, 2 r_0 sin(theta_0) sin(dphi/2)) (Sec. 4.1). */
CFFYN_API double cffyn_default_dt(const cffyn_shell* sh);

/* Static gauge source H_a (eq. gauge), H[4][n_phi][n_theta][n_r] device FP64.
 * The library stores H and its Cartesian derivatives d_i H_a computed with the
 * shell's spectral operators.  n_fields == 50 only; CFFYN_EINVAL for 54/58
 * fields, whose gauge source is fields 50..53 of the state. */
CFFYN_API int cffyn_set_gauge(cffyn_shell* sh, const double* H, void* stream);

/* H_a = -Gamma_a(u) (eq. gauge and eq. Gamma from undifferentiated fields),
 * pointwise.  n_fields == 50: stored as the static gauge (like
 * cffyn_set_gauge).  n_fields 54/58: written into fields 50..53 of u (u is
 * then read-write) and dH/dt (54..57) set to zero. */
CFFYN_API int cffyn_init_gauge_from_state(cffyn_shell* sh, double* u, void* stream);

/* Cartesian derivatives of every field (Secs. 2.3-2.4, chain rule eq. dvdx):
 * dxyz[d][mu][n_phi][n_theta][n_r], d = x, y, z (3 * n_fields arrays).
 * The theta derivative uses the double cover of Sec. 2.1. */
CFFYN_API int cffyn_derivs(cffyn_shell* sh, const double* u, double* dxyz, void* stream);

/* Right-hand side d_t u = S - A^k d_k u of eqs. gdot, Phidot, Pidot with the
 * freeze-incoming outer boundary condition of App. A.2 applied on the
 * outermost sphere; no filter.  Requires the gauge for 50 fields. */
CFFYN_API int cffyn_rhs(cffyn_shell* sh, const double* u, double* dudt, void* stream);

/* The shell's filter (Secs. 3.4-3.5).  Yn: per tensor group, triad
 * decomposition (eq. tensorexpansion), phi DFT (eq. forwardF), projection with
 * F^n_m per spin n and azimuthal m (eq. FasPfQ), inverse DFT, recombination.
 * Y / Yg: phi DFT, projection with F^0_m at each field's retained degree,
 * inverse DFT.  out may alias u. */
CFFYN_API int cffyn_filter(cffyn_shell* sh, const double* u, double* out, void* stream);

/* n_steps classical RK4 steps of the method of lines (Sec. 2.5) in place on u
 * with the shell's filter mode; dt <= 0 selects cffyn_default_dt.  In
 * CFFYN_FILTER_SUBSTEP mode every stage right-hand side is filtered after the
 * boundary condition; the caller filters the initial data once.  The first
 * call for a given (u, dt) captures one step in a CUDA graph (so it must not
 * itself be made during a stream capture); the shell keeps the graphs of the
 * two most recently used (u, dt) pairs (and trace settings), so later calls
 * with either replay it, e.g. a caller alternating two state buffers.  The call
 * synchronises `stream` at its end to read the fused finiteness flag and
 * returns CFFYN_ENONFINITE if a stage right-hand side was not finite, or
 * CFFYN_ETIMEOUT if a bounded wait of a tensor-core operator kernel gave up
 * (the results are then invalid; the context stays usable). */
CFFYN_API int cffyn_rk4_step(cffyn_shell* sh, double* u, double dt, int n_steps, void* stream);

/* cffyn_rk4_step (Sec. 2.5, the same steps and results) without the
 * synchronisation at its end: the call enqueues the steps on `stream` and
 * returns, so that the host can queue the next work (copies, the next
 * problem's steps) while these run.  After the last step the steps' status
 * word is copied on `stream` to *status, host memory the caller owns (pinned
 * memory keeps the copy asynchronous); once the stream has passed that
 * point, cffyn_step_status(*status) is what cffyn_rk4_step would have
 * returned (CFFYN_OK, CFFYN_ENONFINITE or CFFYN_ETIMEOUT).  n_steps == 0
 * runs nothing and writes a zero status word.  Errors found before anything
 * is enqueued are returned at once: CFFYN_EINVAL for the arguments
 * cffyn_rk4_step rejects, a NULL status or tracing switched on (the trace
 * needs the synchronising call); CFFYN_ECUDA if the graph capture or a
 * launch fails.  Like cffyn_rk4_step, the first call for a given (u, dt)
 * captures the step graph and must not be made during a stream capture.
 * Calls on one shell share its workspace: order them on one stream. */
CFFYN_API int cffyn_rk4_step_async(cffyn_shell* sh, double* u, double dt, int n_steps, void* stream,
                                   int* status);

/* The status code of a step status word written by cffyn_rk4_step_async:
 * CFFYN_OK, CFFYN_ENONFINITE or CFFYN_ETIMEOUT (cffyn_last_error() then
 * names the cause). */
CFFYN_API int cffyn_step_status(int status_word);

/* Batch of independent shells advanced together (the uneven-shell batch;
 * the shells need not share sizes, field counts, precision or filter mode).
 * Shells of one shape (n_r, n_theta, n_phi, r_in, r_out, L, n_fields,
 * precision, filter mode and kind, Courant factor and wait bound) are
 * stacked: the batch keeps one internal handle per such class whose every
 * kernel covers all the class's shells in one launch (the operators see
 * n_fields x shells fields, the pointwise kernels n_fields fields of
 * shells x points), with its own workspace and stacked state; a class of one
 * shell is stepped as itself.  The batch borrows the handles: they must stay
 * alive, on the device that is current at cffyn_create_batch, until
 * cffyn_destroy_batch, and must not be used by other calls while a batch
 * call runs.  A shell may appear in one batch position only (duplicates are
 * CFFYN_EINVAL).  The batch owns its stacked handles and states, streams,
 * events, graphs and a pinned flag array.  n >= 1. */
typedef struct cffyn_batch cffyn_batch;
CFFYN_API int cffyn_create_batch(int n, cffyn_shell* const* shells, cffyn_batch** out);

/* Number of independent branches of the batch's step graph: its shape
 * classes (0 for NULL). */
CFFYN_API int cffyn_batch_units(const cffyn_batch* b);

/* n_steps RK4 steps (as cffyn_rk4_step, Sec. 2.5) of every shell of the
 * batch: u is a host array of n device state pointers (u[i] in the layout of
 * shells[i]); dt a host array of n step sizes (NULL, or an entry <= 0,
 * selects that shell's cffyn_default_dt); shells of one class must get one
 * step size (CFFYN_EINVAL otherwise).  Every call copies the states (and,
 * for 50 fields, the gauge sources) of stacked shells into their class,
 * advances all classes, and copies the states back; one step of the whole
 * batch is one CUDA graph launch in which each class is an independent
 * branch; the graphs are captured on the first call and replayed while u and
 * dt stay the same.  Results are bit-identical to stepping each shell
 * alone.  Every 50-field shell needs its gauge (CFFYN_EINVAL before anything
 * is enqueued otherwise).  Synchronises `stream` at the end and returns
 * CFFYN_ETIMEOUT / CFFYN_ENONFINITE as cffyn_rk4_step does, naming the
 * first shell of the class that reported it; a stacked class takes its first
 * shell's wait bound. */
CFFYN_API int cffyn_batch_rk4_step(cffyn_batch* b, double* const* u, const double* dt, int n_steps,
                                   void* stream);

/* Releases the batch (not its shells).  NULL is allowed. */
CFFYN_API int cffyn_destroy_batch(cffyn_batch* b);

/* Nested shells: n shells over consecutive radial intervals, shell i over
 * [r_in_i, r_out_i] with r_out_i == r_in_{i+1} (to 1e-12 relative), sharing
 * n_theta, L, n_fields, precision, filter mode and filter kind (n_r and the
 * Courant factor may differ).  The domain decomposition the paper names as
 * its next step (Secs. 1 and 5); the coupling is this library's reading of
 * the characteristic analysis of App. A.2 (eq. characteristics): on every
 * common sphere (the outer sphere of shell i is the inner sphere of shell
 * i + 1) the right-hand sides are split into the characteristic fields
 * w0 = g, w+ = -g + Pi + s^k Phi_k, w- = -g + Pi - s^k Phi_k and
 * wT_i = Phi_i - s_i s^k Phi_k with the unit normal s_i of the sphere (the
 * inner shell's metric); w- and wT, which App. A.2's outer condition freezes,
 * come from the outer shell, w0 and w+ from the inner one, and both shells
 * get the recombined right-hand side there (gauge fields: the inner
 * shell's).  Only the outermost shell's outer sphere has the freeze-incoming
 * condition.  The nest borrows the handles like a batch: they stay alive and
 * unused by other calls while a nest call runs.  Synchronous.  CFFYN_EINVAL
 * for mismatched or non-adjacent shells, duplicates, NULL. */
typedef struct cffyn_nest cffyn_nest;
CFFYN_API int cffyn_create_nest(int n, cffyn_shell* const* shells, cffyn_nest** out);

/* Right-hand sides of every shell of the nest (host array of n device
 * pointers each way, FP64, each shell's layout) with the coupling above; no
 * filter.  Every 50-field shell needs its gauge. */
CFFYN_API int cffyn_nest_rhs(cffyn_nest* ns, const double* const* u, double* const* dudt, void* stream);

/* n_steps RK4 steps (Sec. 2.5) of all shells with one dt (dt <= 0: the
 * smallest cffyn_default_dt of the shells), every stage coupling the
 * right-hand sides on the common spheres before the shells' filters and
 * stage updates; one CUDA graph per step, captured on the first call and
 * replayed while u and dt stay the same.  Synchronises `stream`; returns
 * CFFYN_ETIMEOUT / CFFYN_ENONFINITE as cffyn_rk4_step does, naming the
 * shell.  The caller filters each shell's initial data once. */
CFFYN_API int cffyn_nest_rk4_step(cffyn_nest* ns, double* const* u, double dt, int n_steps, void* stream);

/* The smallest default dt of the nest's shells.  The coupling on the
 * common spheres lowers the largest stable Courant factor below a lone
 * shell's (measured on two 13x9x18 shells over [1.8, 6.8, 11.8] with the Yn
 * filter per step: stable at 3.0 times the smallest spacing, unstable at
 * 3.5, where one 13x9x18 shell is stable up to 6.0); callers that raise the
 * shells' Courant factor set dt explicitly. */
CFFYN_API double cffyn_nest_default_dt(const cffyn_nest* ns);

/* Releases the nest (not its shells).  NULL is allowed. */
CFFYN_API int cffyn_destroy_nest(cffyn_nest* ns);

/* RMS over all points of C_iab = d_i g_ab - Phi_iab (30 components, numerical
 * derivative) and of C_a = H_a + Gamma_a (4 components) (App. A.1), reduced
 * in FP64 on the device; out[0] = C_iab RMS, out[1] = C_a RMS (host memory).
 * Synchronous. */
CFFYN_API int cffyn_constraint_norms(cffyn_shell* sh, const double* u, double out[2], void* stream);

/* Copies the shell's FP64 filter matrix F^n_m (n in [-3,3], m in [0,L];
 * N x N row-major, N = n_theta) to host memory.  Synchronous.  For checks of
 * the on-device construction. */
CFFYN_API int cffyn_get_filter_matrix(const cffyn_shell* sh, int n, int m, double* host_out);

/* Copies one FP64 operator to host: which = 0: D_r (n_r x n_r),
 * 1: theta derivative of the double cover restricted to the single cover
 * (N x 2N: columns 0..N-1 act on theta_0..theta_{N-1} at phi_j, column N+q on
 * theta_{N-1-q} at phi_j + pi), 2: D_phi (n_phi x n_phi).  Row-major. */
CFFYN_API int cffyn_get_operator(const cffyn_shell* sh, int which, double* host_out);

/* Phase timing of one RK4 step (for benchmarks and tracing): runs one step
 * on u eagerly (no graph, same kernels as cffyn_rk4_step) with CUDA events
 * around every kernel group on `stream`, synchronising after each group, and
 * returns per group the device time in milliseconds summed over the step
 * (ms_out) and the number of kernel launches (launches_out).  Groups, in
 * order: d_r, d_theta and d_phi (one launch per stage on the CFFYN_MIXED
 * path), right-hand-side sources with Christoffel symbols,
 * quadratic sources, principal parts + BC, spin decomposition, phi analysis,
 * projection, phi synthesis, reconstruction + RK4 update, and the per-field
 * exponent scans of the CFFYN_MIXED path in front of each operator group
 * (no launches on the FP64 path).  u is advanced by one step.  Both output
 * arrays hold CFFYN_PROFILE_PHASES entries (host memory). */
#define CFFYN_PROFILE_PHASES 11
CFFYN_API int cffyn_profile_step(cffyn_shell* sh, double* u, double dt, double* ms_out,
                                 int* launches_out, void* stream);

/* Row-group size of one family of tensor-core operator launches of the
 * CFFYN_MIXED path: family 0 d_r, 1 d_theta with d_phi, 2 phi analysis,
 * 3 projections, 4 phi synthesis; rows 48 (two blocks per SM, more row
 * groups when the operator has more rows) or 96 (one block per SM), 0 for
 * the rule (48 up to 48 operator rows, else 96).  Shapes measured by the
 * library's tuner get their fastest choice at creation.  Rebuilds the
 * family's split operators (synchronises the device; not during a stream
 * capture) and drops the captured step graphs.  The results of the two
 * choices agree to the mixed path's rounding (the digit sums of the tensor
 * cores are exact, their FP32 tail is not).  CFFYN_EINVAL for another family
 * or size; a no-op on the FP64 path apart from recording the choice.
 * cffyn_get_operator_rows returns the size in use (0 for bad arguments). */
CFFYN_API int cffyn_set_operator_rows(cffyn_shell* sh, int family, int rows);
CFFYN_API int cffyn_get_operator_rows(const cffyn_shell* sh, int family);

/* Bound of every wait inside the tensor-core operator kernels of the
 * CFFYN_MIXED path (mbarrier waits for operand copies, for the producers'
 * operand slices and for the tensor-core products), in seconds; the default
 * is 1.  A wait that runs out makes that kernel stop, mark the shell's status
 * word and return; cffyn_rk4_step / cffyn_batch_rk4_step then report
 * CFFYN_ETIMEOUT (cffyn_derivs_static writes NaN), the results are invalid
 * and the context stays usable.  seconds < 0 restores the default; 0 makes
 * every such wait give up at once without polling, the way to exercise the
 * CFFYN_ETIMEOUT path.  The waits that let copies and products already in
 * flight finish before a kernel block exits keep the 1 s bound whatever the
 * setting.  Drops the shell's captured step graphs (the next step
 * recaptures; so does a batch holding the shell).  CFFYN_EINVAL for more
 * than 60 s or NaN. */
CFFYN_API int cffyn_set_wait_limit(cffyn_shell* sh, double seconds);

/* Live tracing of cffyn_rk4_step: with tracing on, the captured step graph
 * records a CUDA event after every kernel group (same groups as
 * cffyn_profile_step) and each cffyn_rk4_step call adds the group durations
 * of its last replay (times n_steps) to per-group totals.  Switching tracing
 * on or off resets the totals; the next step replays the traced or untraced
 * graph of its (u, dt) if the shell still keeps it, else captures it. */
CFFYN_API int cffyn_set_trace(cffyn_shell* sh, int on);
/* Per-group totals in ms, kernel launches per step per group, and the number
 * of traced steps.  Host memory, CFFYN_PROFILE_PHASES entries each. */
CFFYN_API int cffyn_get_trace(const cffyn_shell* sh, double* ms_out, int* launches_out,
                              long long* steps);

/* Allocation-free Cartesian derivatives.  A library facility with no
 * counterpart in the paper: a variant of cffyn_derivs.
 * Computes what cffyn_derivs computes, for the first n_f fields of u only:
 *     dxyz[d][mu][n_phi][n_theta][n_r], d = x, y, z, mu < n_f (3 * n_f arrays).
 * Every intermediate (the spherical derivatives and, on the CFFYN_MIXED
 * path, the per-field exponents and the call's status word) lives in one
 * fixed array of CFFYN_STATIC_SCRATCH_BYTES of the library's own device
 * memory, which exists on each device once the library's device code is
 * loaded there.  The call allocates nothing (no cudaMalloc, no library
 * allocator) and neither reads nor writes the shell's workspace or its
 * status word: it reads only the shell's constant grid and operators.
 *
 * Who it is for: callers that cannot get device memory at the point of the
 * call, or must not cause an allocation there: code running with the
 * device's memory fully reserved by another allocator (a new allocation would
 * fail), code that must not take the device-wide synchronisation of
 * cudaMalloc / cudaFree in its loop, and code that differentiates a few
 * auxiliary or diagnostic fields without disturbing work of the same shell
 * enqueued on other streams (cffyn_derivs / cffyn_rhs / cffyn_filter write the
 * shell's workspace; this call does not).
 *
 * Size limit: with P = n_r * n_theta * n_phi the call needs
 * round256(24 * n_f * P) bytes, plus 256 on the CFFYN_MIXED path (round256
 * rounds up to a multiple of 256).  More than CFFYN_STATIC_SCRATCH_BYTES
 * (8 MiB) returns CFFYN_EINVAL, with the bytes needed in cffyn_last_error(),
 * and launches nothing.  Examples: 9 x 12 x 24, all 50 fields; 33 x 32 x 64,
 * 5 fields.
 *
 * Zeroing: the 64 words after the derivatives on the mixed path (per-field
 * exponents, maxima accumulated with atomics, and the status word) must
 * start at zero on every call; the call zeroes them itself on `stream`
 * (cudaMemsetAsync, no allocation).  The caller clears nothing; every other
 * byte is written before it is read.
 *
 * Timeouts: the call is asynchronous and returns before the device work
 * ends.  If a bounded wait of the tensor-core kernel gives up (CFFYN_ETIMEOUT
 * elsewhere), every value of dxyz is written as a quiet NaN, so the caller
 * sees the failure in the output itself.
 *
 * Races: there is one array per device, shared by every call on that device
 * for every shell.  Calls whose device work can overlap (other streams,
 * other threads, other shells on the same device) race on it and give wrong
 * results: order them (one stream, or events).  The array is free for the
 * next call once `stream` has passed the end of this one.
 *
 * Set-up: the first call on each device looks up the array's address with
 * cudaGetSymbolAddress (the shell's device current), which may load the
 * library's device code there; make that first call before any stream
 * capture begins on the calling thread.  Later calls only reuse the address.
 *
 * Errors: CFFYN_EINVAL for a NULL shell, NULL or unaligned u / dxyz, n_f
 * outside [1, n_fields], the size limit, or a current device other than the
 * shell's; CFFYN_ECUDA if the address lookup or a launch fails.  Asynchronous
 * like cffyn_derivs. */
#define CFFYN_STATIC_SCRATCH_BYTES (8u * 1024u * 1024u)
CFFYN_API int cffyn_derivs_static(const cffyn_shell* sh, const double* u, int n_f, double* dxyz,
                                  void* stream);

/* Cartesian derivatives of every field, like cffyn_derivs (same output
 * layout and meaning), computed with fast Fourier transforms instead of the
 * differentiation matrices: the alternative the paper weighs against the
 * matrix method in Sec. 5 (Fig. mmfft).  FP64 on either precision path:
 * Chebyshev coefficients by a real FFT of the even extension in r (DCT-I),
 * the derivative's coefficients by the recurrence
 * c_k b_k = b_{k+2} + 2 (k + 1) a_{k+1}, and an inverse FFT; the theta
 * derivative over the double cover of Sec. 2.1 (2 n_theta points per line)
 * and the phi derivative by FFTs with the Nyquist mode set to zero, as the
 * matrices of eq. FD do.  Results agree with cffyn_derivs on an FP64 shell to
 * rounding.  Uses cuFFT (library code) for the transforms and the shell's
 * workspace for the spherical derivatives (like cffyn_derivs).
 *
 * The first call on a shell creates six cuFFT plans and allocates FFT scratch
 * (cudaMalloc, about 4 x n_fields x P doubles, plus cuFFT's own work area):
 * make it before any stream capture.  cffyn_destroy frees them.
 * Errors: CFFYN_EINVAL for a NULL shell or NULL / unaligned arrays, no
 * workspace, or a current device other than the shell's; CFFYN_ENOMEM or
 * CFFYN_ECUDA if a plan, the scratch or a launch fails.  Asynchronous after
 * the first call. */
CFFYN_API int cffyn_derivs_fft(cffyn_shell* sh, const double* u, double* dxyz, void* stream);

/* Message of the last failing call on this thread (never NULL). */
CFFYN_API const char* cffyn_last_error(void);

/* Library version string. */
CFFYN_API const char* cffyn_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CFFYN_H */
