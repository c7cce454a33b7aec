// Internal definitions of the cffyn library: the shell handle, the operator
// descriptors shared by the FP64 and the split-precision kernels, and error
// plumbing.  Not part of the public ABI (see include/cffyn.h).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/cffyn.h"

namespace cffyn {

constexpr int kMaxN = 96;      // n_theta limit (N_phi <= 192)
constexpr int kMaxNr = 96;     // n_r limit
constexpr int kNumSpinFns = 50;

// Number of split-precision digits per operand (8-bit balanced digits of a
// 47-bit fixed-point value) and the highest digit-sum kept (pairs i + j <= D).
constexpr int kSlices = 6;

// Thread-local error message.
void set_error(const char* fmt, ...);
// Kernel launches issued by this thread (for the launch counts reported by
// the profiling entry point).
void count_launch();
#define CF_CUDA(call)                                                              \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      ::cffyn::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call,                \
                         cudaGetErrorString(e_));                                  \
      return CFFYN_ECUDA;                                                          \
    }                                                                              \
  } while (0)

// --------------------------------------------------------------------------
// Split-precision operator for the tcgen05 core: W cut into row groups of
// `rows` = 48 (P <= 48) or 96 rows and k-steps of 16 columns; per (group,
// k-step) sixteen BF16 digit slices of rows x 16 in the K-major no-swizzle
// core-matrix order (core matrix = 8 rows x 8 columns, 128 contiguous bytes;
// the two core matrices of an 8-row group adjacent, groups 256 bytes apart).
// Slices 0..4 are digits 0..4 of W; slices 5..10 are digits 0..5 scaled by
// 2^-8 and slices 11..15 digits 1..5 scaled by 2^-16 (they carry the
// digit-sum-5 and digit-sum-6 products into the digit-sum-4 accumulator).
constexpr int kTcWSlices = 16;
// families of operator launches whose row-group size can be chosen
// (cffyn_set_operator_rows): d_r, d_theta + d_phi, phi analysis,
// projections, phi synthesis
constexpr int kOpFamilies = 5;
struct TcOp {
  unsigned short* w = nullptr;  // [batch][group][kstep][slice][rows x 16]
  int* rowexp = nullptr;        // [batch][groups * rows]
  int P = 0, K = 0, rows = 0, ngroups = 0, ksteps = 0, nbatch = 1;
  size_t w_stride = 0, rowexp_stride = 0;  // per batch (elements)
};

struct cffyn_shell_impl;
struct FftPath;  // fft.cu: plans and scratch of cffyn_derivs_fft

}  // namespace cffyn

struct cffyn_shell {
  cffyn_shell_desc d;
  int n_r, N, J, L, nv, R;      // R = 2 Lrows + 1 Fourier rows kept
  int Lrows;                    // azimuthal modes kept by the phi DFT: L, or L + 3 (at most N - 1) for Yg
  size_t P;                     // points per field of one shell
  int ns = 1;                   // shells stacked in this handle (the uneven-shell batch stacks
                                // shells of one shape: fields [mu][s][P], so that the operators
                                // see nv * ns fields of P points and the pointwise kernels nv
                                // fields of ns * P points)
  double dt_default;
  size_t bytes = 0;
  int device = 0;

  // grid (device)
  double *r = nullptr, *sth = nullptr, *cth = nullptr, *sph = nullptr, *cph = nullptr;
  double* triad = nullptr;  // [n_phi][n_theta][9] real triad rows, internal storage

  // FP64 operators (device, row-major)
  double* Dr = nullptr;     // n_r x n_r
  double* Dth2 = nullptr;   // 2N x 2N (paired planes j, j + J/2)
  double* Dph = nullptr;    // J x J
  double* Fan = nullptr;    // R x J   analysis rows a_0..a_L, b_1..b_L
  double* Fsy = nullptr;    // J x R   synthesis
  double* Fraw = nullptr;   // [7][L+1] N x N : F^n_m, n = -3..3
  double* Fproj0 = nullptr; // [L+1] N x N : F^0_m
  double* FprojC = nullptr; // [3][L+1] N x 2N : [F_s | F_d] for spin 1..3
  double* F0g = nullptr;    // graded filter: [4][Lrows+1] N x N : F^0_m at retained degree L + d

  // split-precision operators (tcgen05 core); tF0 and tFC are batched over
  // m = 0..L, tFC per spin 1..3
  cffyn::TcOp tDr, tDth2, tDph, tFan, tFsy, tF0, tFC[3], tF0g[4];
  // row-group size of each operator family (0: the rule, 48 up to 48 rows,
  // else 96), set at creation from the tuned table or by
  // cffyn_set_operator_rows
  int op_rows[cffyn::kOpFamilies] = {0, 0, 0, 0, 0};

  // spin slots of the filter (one real slot per Cartesian field): nR0 real
  // functions filtered with F^0_m (spin 0, including the real and imaginary
  // parts of the two complex spin-0 components), then nC[s - 1] complex
  // functions of spin s as (re, im) slot pairs; `slots` holds the slot
  // indices of each list.  Each gauge group of a 54/58-field state adds two
  // real slots (H_t, H_r) and one spin-1 pair.
  int ng = 0;                    // gauge groups: (nv - 50) / 4
  int nR0 = 16, nC[3] = {11, 5, 1};
  // component-wise filters: fields by spatial degree d (Yg: 4 lists; Y: one
  // list of every field) in yslots, ny[d] entries each
  int* yslots = nullptr;
  int ny[4] = {0, 0, 0, 0};
  // exponent gains of the filter's operators: ceil(log2) of the largest row
  // sum of |entries| of the phi analysis and of the projection matrices, so
  // that |coefficients| < 2^(E_input + gain_dft) and |projected| <
  // 2^(E_input + gain_dft + gain_proj) bound the next operators' inputs
  int gain_dft = 1, gain_proj = 0;

  // gauge
  double* H = nullptr;    // [4][P]
  double* dH = nullptr;   // [3][4][P] d_i H_a, + [4][P] d_t H_a for 58 fields
  bool gauge_set = false;

  // bound of every pipeline wait of the tensor-core operator kernel (ns;
  // 0: give up at once), cffyn_set_wait_limit
  unsigned long long tc_wait_ns = 1000000000ull;

  // workspace: one block (ws, ws_bytes) carved into the arrays below; owned
  // by the library (ws_owned) or attached by the caller; ws_gen counts the
  // changes that make captured graphs stale (attachments, wait limits)
  void* ws = nullptr;
  size_t ws_bytes = 0;
  bool ws_owned = false;
  unsigned ws_gen = 0;
  double* U = nullptr;     // stage state [nv][P]
  double* Uf = nullptr;    // mixed path: the step's initial state in internal storage [nv][P]
  double* kacc = nullptr;  // RK4 accumulator [nv][P]
  double* D = nullptr;     // spherical derivatives [3][nv][P] (also DFT coefficients)
  double* S = nullptr;     // rhs / spin functions [nv][P]
  double* Rsrc = nullptr;  // right-hand-side source terms [nv][P]
  int* exps = nullptr;     // per-field exponents of the next operator input (64 entries)
  double* red = nullptr;   // device reduction words (2 doubles)
  cffyn::FftPath* fft = nullptr;  // FFT derivative path, made by its first call
  int* flag = nullptr;     // device non-finite flag
  int* flag_host = nullptr;  // pinned host copy of the flag
  int* slots = nullptr;    // device slot lists: R0 (nR0) | C1 (nC[0]) | C2 (nC[1]) | C3 (nC[2])
  cudaStream_t cap_stream = nullptr;  // private stream for graph capture
  // second stream of a stage: the algebraic right-hand-side kernels run on
  // it beside the derivative launches (fork / join events)
  cudaStream_t aux_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;

  // tracing: event nodes at every phase boundary of the captured step
  int trace = 0;
  static constexpr int kPhases = 11;
  static constexpr int kMaxMarks = 64;

  // graphs of one RK4 step for the two most recently used (u, dt, trace):
  // a caller alternating two state buffers replays both without capturing
  // again.  Each keeps what its capture recorded about its kernel groups.
  struct StepGraph {
    cudaGraphExec_t exec = nullptr;
    double* u = nullptr;
    double dt = 0.0;
    int trace = 0;
    int n_marks = 0;
    int mark_phase[kMaxMarks] = {};
    int launches[kPhases] = {};
  };
  static constexpr int kStepGraphs = 2;
  StepGraph graphs[kStepGraphs];
  int graph_victim = 0;  // the entry the next capture replaces
  cudaEvent_t marks[kMaxMarks] = {};
  int mark_phase[kMaxMarks] = {};   // phase that ends at mark i (-1: start)
  int n_marks = 0;
  int launches_per_step[kPhases] = {};
  double trace_ms[kPhases] = {};
  long long trace_steps = 0;
};

namespace cffyn {
// fft.cu: frees the FFT derivative path's plans and scratch (no-op without)
void fft_release(cffyn_shell*);
// fields the operators see (nv per stacked shell) and points of every array
inline int nv_ops(const cffyn_shell* sh) { return sh->nv * sh->ns; }
inline size_t P_all(const cffyn_shell* sh) { return sh->P * (size_t)sh->ns; }
}  // namespace cffyn
