// C-ABI entry points of include/cffyn.h: argument checks, workspace, and the
// orchestration of one right-hand side / filter / RK4 step (paper Sec. 2.5)
// out of the operator kernels (ops.cu) and the pointwise kernels
// (pointwise.cu).  One RK4 step is captured once into a CUDA graph and
// replayed.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "common.cuh"
#include "tile_table.h"

namespace cffyn {

static thread_local char g_err[512] = "no error";
static thread_local long long g_launches = 0;

void count_launch() { ++g_launches; }

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

// ops.cu
int set_op_smem_limits();
int op_deriv_r(const cffyn_shell*, const double*, double*, int, bool, cudaStream_t);
int op_deriv_theta(const cffyn_shell*, const double*, double*, int, bool, cudaStream_t);
int op_deriv_phi(const cffyn_shell*, const double*, double*, int, bool, cudaStream_t);
int op_deriv_theta_phi(const cffyn_shell*, const double*, double*, double*, int, bool, cudaStream_t);
int op_dft_fwd(const cffyn_shell*, const double*, double*, int, cudaStream_t, int, int f0 = 0);
int op_dft_inv(const cffyn_shell*, const double*, double*, int, cudaStream_t, int, int, int f0 = 0);
int op_project_scalar(const cffyn_shell*, const double*, double*, cudaStream_t, int);
int op_project(const cffyn_shell*, const double*, double*, const int*, int, const int* const[3],
               const int[3], cudaStream_t, int);
int op_prepare(const cffyn_shell*, const double*, bool, int, long long, int, cudaStream_t);
// setup.cu
int build_operators(cffyn_shell*);
int build_tc_family(cffyn_shell*, int);
void free_tc(TcOp&);
// pointwise.cu
int pw_rhs(const cffyn_shell*, const double*, const double*, double*, cudaStream_t);
int pw_rhs_part(const cffyn_shell*, const double*, const double*, double*, int, bool, bool, cudaStream_t);
int pw_decompose(const cffyn_shell*, const double*, double*, bool, cudaStream_t);
int pw_reconstruct(const cffyn_shell*, const double*, double*, int, double*, double*, double*, double*,
                   double, int*, cudaStream_t);
int pw_cart(const cffyn_shell*, const double*, double*, int, bool, cudaStream_t);
int pw_triad_table(const cffyn_shell*);
int pw_gauge(const cffyn_shell*, const double*, double*, cudaStream_t);
int pw_gauge_into_state(const cffyn_shell*, double*, cudaStream_t);
int pw_to_internal(const cffyn_shell*, const double*, double*, long long, cudaStream_t);
int pw_constraints(const cffyn_shell*, const double*, const double*, const double*, bool, double*, cudaStream_t);

}  // namespace cffyn

using namespace cffyn;

static_assert(cffyn_shell::kPhases == CFFYN_PROFILE_PHASES, "phase count of the trace and the ABI");

namespace {

// Destroy the kept step graphs (their parameters changed: workspace, wait
// bound, operator row groups); a replay still in flight completes first.
void drop_step_graphs(cffyn_shell* sh) {
  for (int e = 0; e < cffyn_shell::kStepGraphs; ++e) {
    if (sh->graphs[e].exec) cudaGraphExecDestroy(sh->graphs[e].exec);
    sh->graphs[e] = cffyn_shell::StepGraph{};
  }
  sh->graph_victim = 0;
}

const int* slots_r0(const cffyn_shell* sh) { return sh->slots; }
const int* slots_c(const cffyn_shell* sh, int s) {
  int o = sh->nR0;
  for (int q = 0; q < s; ++q) o += sh->nC[q];
  return sh->slots + o;
}

int check_ptr(const void* p, const char* what) {
  if (!p) {
    set_error("%s is NULL", what);
    return CFFYN_EINVAL;
  }
  if (((uintptr_t)p) & 15) {
    set_error("%s is not 16-byte aligned", what);
    return CFFYN_EINVAL;
  }
  return CFFYN_OK;
}

// Workspace layout: U, kacc, D (three arrays), S, Rsrc and on the mixed path
// Uf, each nv x P doubles rounded up to 256 bytes, in this order.
size_t ws_array_bytes(const cffyn_shell* sh) {
  return ((size_t)sh->nv * P_all(sh) * sizeof(double) + 255) / 256 * 256;
}
size_t ws_total_bytes(const cffyn_shell* sh) {
  return ws_array_bytes(sh) * (sh->d.precision == CFFYN_MIXED ? 8 : 7);
}
void carve_workspace(cffyn_shell* sh, void* base) {
  const size_t one = ws_array_bytes(sh);
  char* p = static_cast<char*>(base);
  auto take = [&](int n) {
    double* q = base ? reinterpret_cast<double*>(p) : nullptr;
    p += n * one;
    return q;
  };
  sh->U = take(1);
  sh->kacc = take(1);
  sh->D = take(3);
  sh->S = take(1);
  sh->Rsrc = take(1);
  sh->Uf = sh->d.precision == CFFYN_MIXED ? take(1) : nullptr;
  sh->ws = base;
}
int check_ws(const cffyn_shell* sh) {
  if (!sh->ws) {
    set_error("no workspace attached (cffyn_attach_workspace)");
    return CFFYN_EINVAL;
  }
  return CFFYN_OK;
}

// spherical derivatives of nf fields into D (internal storage); in_pairs: u is
// a pair-stored internal buffer of the mixed path (else FP64)
int derivs_spherical(cffyn_shell* sh, const double* u, double* D, int nf, bool in_pairs, cudaStream_t st) {
  const size_t P = sh->P;
  int rc;
  if ((rc = op_prepare(sh, u, in_pairs, nf, (long long)P, 0, st))) return rc;
  if ((rc = op_deriv_r(sh, u, D, nf, in_pairs, st))) return rc;
  if ((rc = op_deriv_theta(sh, u, D + (size_t)nf * P, nf, in_pairs, st))) return rc;
  if ((rc = op_deriv_phi(sh, u, D + (size_t)2 * nf * P, nf, in_pairs, st))) return rc;
  return CFFYN_OK;
}

// Filter of the functions in `spin` (nv x P), in place, scratch D (2 nv P):
// Yn: the spin slots of the triad decomposition, projected per spin class;
// Y / Yg: the Cartesian fields themselves, each with F^0_m (Sec. 3.5).
bool yn_filter(const cffyn_shell* sh) { return sh->d.filter_kind == CFFYN_FILTER_YN; }

// One exponent scan of the filter's input; the coefficients and the projected
// coefficients take bounds from it (exponent + the operators' gains) instead
// of scans of their own.
int filter_spin_slots(cffyn_shell* sh, double* spin, cudaStream_t st) {
  const size_t nvP = (size_t)sh->nv * sh->P;
  int rc;
  double* C = sh->D;
  double* C2 = sh->D + nvP;
  const int pairing = yn_filter(sh) ? 1 : 0;
  const int e1 = sh->gain_dft, e2 = sh->gain_dft + sh->gain_proj;
  if ((rc = op_prepare(sh, spin, true, sh->nv, (long long)sh->P, pairing, st))) return rc;
  if ((rc = op_dft_fwd(sh, spin, C, sh->nv, st, pairing))) return rc;
  const int* cl[3] = {slots_c(sh, 0), slots_c(sh, 1), slots_c(sh, 2)};
  if ((rc = yn_filter(sh) ? op_project(sh, C, C2, slots_r0(sh), sh->nR0, cl, sh->nC, st, e1)
                          : op_project_scalar(sh, C, C2, st, e1)))
    return rc;
  if ((rc = op_dft_inv(sh, C2, spin, sh->nv, st, pairing, e2))) return rc;
  return CFFYN_OK;
}

void free_shell(cffyn_shell* sh) {
  if (!sh) return;
  cudaDeviceSynchronize();
  double** ptrs[] = {&sh->r,   &sh->sth, &sh->cth,  &sh->sph,  &sh->cph,    &sh->Dr,     &sh->Dth2,
                     &sh->Dph, &sh->Fan, &sh->Fsy,  &sh->Fraw, &sh->Fproj0, &sh->FprojC, &sh->F0g, &sh->H,
                     &sh->dH,  &sh->red, &sh->triad};
  for (double** p : ptrs)
    if (*p) cudaFree(*p);
  if (sh->ws_owned && sh->ws) cudaFree(sh->ws);
  TcOp* to[] = {&sh->tDr, &sh->tDth2, &sh->tDph, &sh->tFan, &sh->tFsy, &sh->tF0,
                &sh->tFC[0], &sh->tFC[1], &sh->tFC[2], &sh->tF0g[0], &sh->tF0g[1], &sh->tF0g[2], &sh->tF0g[3]};
  for (TcOp* t : to) free_tc(*t);
  if (sh->slots) cudaFree(sh->slots);
  if (sh->yslots) cudaFree(sh->yslots);
  if (sh->exps) cudaFree(sh->exps);
  if (sh->cap_stream) cudaStreamDestroy(sh->cap_stream);
  if (sh->aux_stream) cudaStreamDestroy(sh->aux_stream);
  if (sh->ev_fork) cudaEventDestroy(sh->ev_fork);
  if (sh->ev_join) cudaEventDestroy(sh->ev_join);
  if (sh->flag_host) cudaFreeHost(sh->flag_host);
  if (sh->flag) cudaFree(sh->flag);
  drop_step_graphs(sh);
  for (int i = 0; i < cffyn_shell::kMaxMarks; ++i)
    if (sh->marks[i]) cudaEventDestroy(sh->marks[i]);
  fft_release(sh);
  delete sh;
}

}  // namespace

extern "C" {

const char* cffyn_last_error(void) { return g_err; }
const char* cffyn_version(void) { return "cffyn 0.1 (sm_103a)"; }

static int create_shell(const cffyn_shell_desc* desc, int ns, cffyn_shell** out);

int cffyn_create_shell_ex(const cffyn_shell_desc* desc, cffyn_shell** out) { return create_shell(desc, 1, out); }

}  // extern "C"

extern "C++" {
namespace cffyn {
// A handle of ns shells of one shape stacked as fields [mu][s][P] (the
// uneven-shell batch's units; stepped with the single-shell step sequence).
int create_stacked_shell(const cffyn_shell_desc* desc, int ns, cffyn_shell** out) {
  return create_shell(desc, ns, out);
}
}  // namespace cffyn
}  // extern "C++"

extern "C" {

static int create_shell(const cffyn_shell_desc* desc, int ns, cffyn_shell** out) {
  if (!out) {
    set_error("out is NULL");
    return CFFYN_EINVAL;
  }
  *out = nullptr;
  if (!desc) {
    set_error("desc is NULL");
    return CFFYN_EINVAL;
  }
  const cffyn_shell_desc& d = *desc;
  if (d.n_r < 3 || d.n_r > kMaxNr || d.n_theta < 2 || d.n_theta > kMaxN ||
      d.n_phi != 2 * d.n_theta || !(d.r_in > 0) || !(d.r_out > d.r_in) || d.L < 0 ||
      d.L > d.n_theta - 1) {
    set_error("invalid shell sizes (n_r %d, n_theta %d, n_phi %d, r %g..%g, L %d)", d.n_r, d.n_theta,
              d.n_phi, d.r_in, d.r_out, d.L);
    return CFFYN_EINVAL;
  }
  if (d.n_fields != 50 && d.n_fields != 54 && d.n_fields != 58) {
    set_error("n_fields must be 50, 54 or 58");
    return CFFYN_EINVAL;
  }
  if (d.precision != CFFYN_FP64 && d.precision != CFFYN_MIXED) {
    set_error("precision must be CFFYN_FP64 or CFFYN_MIXED");
    return CFFYN_EINVAL;
  }
  if (d.filter_mode != CFFYN_FILTER_SUBSTEP && d.filter_mode != CFFYN_FILTER_STEP) {
    set_error("filter_mode must be CFFYN_FILTER_SUBSTEP or CFFYN_FILTER_STEP");
    return CFFYN_EINVAL;
  }
  if (d.flags & ~CFFYN_DEFER_WORKSPACE) {
    set_error("unknown flags 0x%x", d.flags);
    return CFFYN_EINVAL;
  }
  if (d.filter_kind != CFFYN_FILTER_YN && d.filter_kind != CFFYN_FILTER_Y && d.filter_kind != CFFYN_FILTER_YG) {
    set_error("unknown filter kind %d", d.filter_kind);
    return CFFYN_EINVAL;
  }
  cffyn_shell* sh = new (std::nothrow) cffyn_shell();
  if (!sh) {
    set_error("host allocation failed");
    return CFFYN_ENOMEM;
  }
  sh->d = d;
  sh->ns = ns < 1 ? 1 : ns;
  sh->n_r = d.n_r;
  sh->N = d.n_theta;
  sh->J = d.n_phi;
  sh->L = d.L;
  sh->Lrows = d.filter_kind == CFFYN_FILTER_YG ? std::min(d.L + 3, d.n_theta - 1) : d.L;
  sh->R = 2 * sh->Lrows + 1;
  sh->nv = d.n_fields;
  sh->ng = (d.n_fields - 50) / 4;
  sh->nR0 = 16 + 2 * sh->ng;
  sh->nC[0] = 11 + sh->ng;
  sh->P = (size_t)d.n_r * d.n_theta * d.n_phi;
  cudaGetDevice(&sh->device);
  {
    const double pi = 3.14159265358979323846;
    double r0 = 0.5 * (d.r_out + d.r_in) - 0.5 * (d.r_out - d.r_in);
    double r1 = 0.5 * (d.r_out + d.r_in) - 0.5 * (d.r_out - d.r_in) * cos(pi / (d.n_r - 1));
    double th0 = pi * 0.5 / d.n_theta;
    double dphi = 2.0 * pi / d.n_phi;
    double dx = r1 - r0;
    double ch = 2.0 * r0 * sin(th0) * sin(0.5 * dphi);
    if (ch < dx) dx = ch;
    sh->dt_default = (d.courant > 0 ? d.courant : 0.25) * dx;
  }
  int rc;
  auto fail = [&](int code) {
    free_shell(sh);
    return code;
  };
  if (set_op_smem_limits() != CFFYN_OK) return fail(CFFYN_ECUDA);
  for (const TileEntry* t = kTileTable; t->n_r; ++t)
    if (t->n_r == d.n_r && t->n_theta == d.n_theta && t->L == d.L && t->n_fields == d.n_fields &&
        t->filter_kind == d.filter_kind)
      for (int w = 0; w < kOpFamilies; ++w) sh->op_rows[w] = t->rows[w];
  if ((rc = build_operators(sh))) return fail(rc);
  const size_t nvP = (size_t)sh->nv * sh->P;
  auto alloc = [&](double** p, size_t n) -> int {
    if (cudaMalloc(p, n * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      set_error("device allocation of %zu bytes failed", n * sizeof(double));
      return CFFYN_ENOMEM;
    }
    sh->bytes += n * sizeof(double);
    return CFFYN_OK;
  };
  if ((rc = alloc(&sh->H, 4 * P_all(sh))) || (rc = alloc(&sh->dH, (sh->nv == 58 ? 16 : 12) * P_all(sh))) ||
      (rc = alloc(&sh->red, 2)) || (rc = alloc(&sh->triad, (size_t)9 * sh->N * sh->J)))
    return fail(rc);
  (void)nvP;
  if ((rc = pw_triad_table(sh))) return fail(rc);
  if (d.precision == CFFYN_MIXED && cudaMalloc(&sh->exps, std::max(64, nv_ops(sh)) * sizeof(int)) != cudaSuccess)
    return fail(CFFYN_ENOMEM);
  sh->ws_bytes = ws_total_bytes(sh);
  if (!(d.flags & CFFYN_DEFER_WORKSPACE)) {
    void* w = nullptr;
    if (cudaMalloc(&w, sh->ws_bytes) != cudaSuccess) {
      cudaGetLastError();
      set_error("device allocation of %zu bytes (workspace) failed", sh->ws_bytes);
      return fail(CFFYN_ENOMEM);
    }
    sh->ws_owned = true;
    sh->bytes += sh->ws_bytes;
    carve_workspace(sh, w);
  }
  {
    // R0: the 16 real slots of the 50 GHG fields, then H_t and H_r of every
    // gauge group; C1: the 11 spin-1 pairs, then each gauge group's angular
    // pair; C2 and C3 as for 50 fields
    int host[64];
    int n = 0;
    for (int i = 0; i < 16; ++i) host[n++] = i;
    for (int q = 0; q < sh->ng; ++q) {
      host[n++] = 50 + 4 * q;
      host[n++] = 51 + 4 * q;
    }
    for (int q = 0; q < 11; ++q) host[n++] = 16 + 2 * q;
    for (int q = 0; q < sh->ng; ++q) host[n++] = 52 + 4 * q;
    for (int q = 0; q < 5; ++q) host[n++] = 38 + 2 * q;
    host[n++] = 48;
    if (cudaMalloc(&sh->slots, n * sizeof(int)) != cudaSuccess) return fail(CFFYN_ENOMEM);
    if (cudaMemcpy(sh->slots, host, n * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(CFFYN_ECUDA);
  }
  if (d.filter_kind != CFFYN_FILTER_YN) {
    // component-wise filters: the fields, by spatial degree d(u^mu) for Yg
    // (Sec. 3.5: pairs tt, ti, ij of g_ab and Pi_ab have 0, 1, 2 spatial
    // indices, Phi_iab one more, H_t 0 and H_i 1), all in one list for Y
    auto degree = [](int mu) {
      if (mu >= 50) return (mu - 50) % 4 == 0 ? 0 : 1;
      const int s = mu % 10;
      return (s == 0 ? 0 : (s < 4 ? 1 : 2)) + (mu >= 20 ? 1 : 0);
    };
    const bool graded = d.filter_kind == CFFYN_FILTER_YG;
    int host[64];
    int n = 0;
    for (int dd = 0; dd < 4; ++dd) {
      const int n0 = n;
      for (int mu = 0; mu < sh->nv; ++mu)
        if (graded ? degree(mu) == dd : dd == 0) host[n++] = mu;
      sh->ny[dd] = n - n0;
    }
    if (cudaMalloc(&sh->yslots, n * sizeof(int)) != cudaSuccess) return fail(CFFYN_ENOMEM);
    if (cudaMemcpy(sh->yslots, host, n * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(CFFYN_ECUDA);
  }
  if (cudaMalloc(&sh->flag, 64) != cudaSuccess) return fail(CFFYN_ENOMEM);
  if (cudaMemset(sh->flag, 0, 64) != cudaSuccess) return fail(CFFYN_ECUDA);
  if (cudaStreamCreateWithFlags(&sh->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
    return fail(CFFYN_ECUDA);
  if (cudaStreamCreateWithFlags(&sh->aux_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&sh->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&sh->ev_join, cudaEventDisableTiming) != cudaSuccess)
    return fail(CFFYN_ECUDA);
  if (cudaMallocHost(&sh->flag_host, sizeof(int)) != cudaSuccess) return fail(CFFYN_ENOMEM);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    set_error("shell construction failed: %s", cudaGetErrorString(cudaGetLastError()));
    return fail(CFFYN_ECUDA);
  }
  *out = sh;
  return CFFYN_OK;
}

int cffyn_create_shell(int n_r, int n_theta, int n_phi, double r_in, double r_out, int L,
                       cffyn_shell** out) {
  cffyn_shell_desc d;
  d.n_r = n_r;
  d.n_theta = n_theta;
  d.n_phi = n_phi;
  d.r_in = r_in;
  d.r_out = r_out;
  d.L = L;
  d.n_fields = 50;
  d.precision = CFFYN_MIXED;
  d.filter_mode = CFFYN_FILTER_SUBSTEP;
  d.courant = 0.25;
  d.filter_kind = CFFYN_FILTER_YN;
  d.flags = 0;
  return cffyn_create_shell_ex(&d, out);
}

int cffyn_destroy(cffyn_shell* sh) {
  free_shell(sh);
  return CFFYN_OK;
}

size_t cffyn_device_bytes(const cffyn_shell* sh) { return sh ? sh->bytes : 0; }

size_t cffyn_workspace_size(const cffyn_shell* sh) { return sh ? sh->ws_bytes : 0; }

int cffyn_attach_workspace(cffyn_shell* sh, void* ptr, size_t bytes) {
  if (!sh) { set_error("shell is NULL"); return CFFYN_EINVAL; }
  if (ptr && (((uintptr_t)ptr) & 255)) {
    set_error("workspace is not 256-byte aligned");
    return CFFYN_EINVAL;
  }
  if (ptr && bytes < sh->ws_bytes) {
    set_error("workspace of %zu bytes, %zu needed", bytes, sh->ws_bytes);
    return CFFYN_EINVAL;
  }
  if (!ptr && sh->ws_owned) return CFFYN_OK;
  CF_CUDA(cudaDeviceSynchronize());
  void* fresh = nullptr;
  if (!ptr) {
    if (cudaMalloc(&fresh, sh->ws_bytes) != cudaSuccess) {
      cudaGetLastError();
      set_error("device allocation of %zu bytes (workspace) failed", sh->ws_bytes);
      return CFFYN_ENOMEM;
    }
  }
  if (sh->ws_owned) {
    cudaFree(sh->ws);
    sh->bytes -= sh->ws_bytes;
  }
  sh->ws_owned = !ptr;
  if (!ptr) sh->bytes += sh->ws_bytes;
  carve_workspace(sh, ptr ? ptr : fresh);
  drop_step_graphs(sh);
  ++sh->ws_gen;
  return CFFYN_OK;
}

double cffyn_default_dt(const cffyn_shell* sh) { return sh ? sh->dt_default : 0.0; }

static int gauge_derivs(cffyn_shell* sh, cudaStream_t st) {
  // d_i H_a with the shell's operators: spherical derivatives into D, chain rule into dH
  int rc;
  if ((rc = check_ws(sh))) return rc;
  const bool pairs = sh->d.precision == CFFYN_MIXED;
  if ((rc = derivs_spherical(sh, sh->H, sh->D, 4, pairs, st))) return rc;
  if ((rc = pw_cart(sh, sh->D, sh->dH, 4, true, st))) return rc;
  sh->gauge_set = true;
  return CFFYN_OK;
}

int cffyn_set_gauge(cffyn_shell* sh, const double* H, void* stream) {
  if (!sh) { set_error("shell is NULL"); return CFFYN_EINVAL; }
  if (sh->nv != 50) {
    set_error("n_fields %d: the gauge source is fields 50..53 of the state", sh->nv);
    return CFFYN_EINVAL;
  }
  int rc;
  if ((rc = check_ptr(H, "H"))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if ((rc = pw_to_internal(sh, H, sh->H, 4 * (long long)sh->P, st))) return rc;
  return gauge_derivs(sh, st);
}

int cffyn_init_gauge_from_state(cffyn_shell* sh, double* u, void* stream) {
  if (!sh) { set_error("shell is NULL"); return CFFYN_EINVAL; }
  int rc;
  if ((rc = check_ptr(u, "u"))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if (sh->nv != 50) return pw_gauge_into_state(sh, u, st);
  if ((rc = pw_gauge(sh, u, sh->H, st))) return rc;
  return gauge_derivs(sh, st);
}

int cffyn_derivs(cffyn_shell* sh, const double* u, double* dxyz, void* stream) {
  if (!sh) { set_error("shell is NULL"); return CFFYN_EINVAL; }
  int rc;
  if ((rc = check_ptr(u, "u")) || (rc = check_ptr(dxyz, "dxyz"))) return rc;
  if ((rc = check_ws(sh))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if ((rc = derivs_spherical(sh, u, sh->D, sh->nv, false, st))) return rc;
  return pw_cart(sh, sh->D, dxyz, sh->nv, false, st);
}

int cffyn_rhs(cffyn_shell* sh, const double* u, double* dudt, void* stream) {
  if (!sh) { set_error("shell is NULL"); return CFFYN_EINVAL; }
  int rc;
  if ((rc = check_ptr(u, "u")) || (rc = check_ptr(dudt, "dudt"))) return rc;
  if ((rc = check_ws(sh))) return rc;
  if (sh->nv == 50 && !sh->gauge_set) {
    set_error("gauge source not set (cffyn_set_gauge / cffyn_init_gauge_from_state)");
    return CFFYN_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if ((rc = derivs_spherical(sh, u, sh->D, sh->nv, false, st))) return rc;
  return pw_rhs(sh, u, sh->D, dudt, st);
}

int cffyn_filter(cffyn_shell* sh, const double* u, double* out, void* stream) {
  if (!sh) { set_error("shell is NULL"); return CFFYN_EINVAL; }
  int rc;
  if ((rc = check_ptr(u, "u")) || (rc = check_ptr(out, "out"))) return rc;
  if ((rc = check_ws(sh))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if (yn_filter(sh)) {
    if ((rc = pw_decompose(sh, u, sh->S, false, st))) return rc;
    if ((rc = filter_spin_slots(sh, sh->S, st))) return rc;
    return pw_reconstruct(sh, sh->S, out, 0, nullptr, nullptr, nullptr, nullptr, 0.0, sh->flag, st);
  }
  if ((rc = pw_to_internal(sh, u, sh->S, (long long)sh->nv * sh->P, st))) return rc;
  if ((rc = filter_spin_slots(sh, sh->S, st))) return rc;
  return pw_reconstruct(sh, sh->S, out, 9, nullptr, nullptr, nullptr, nullptr, 0.0, sh->flag, st);
}

// The kernel groups of one RK4 step (Sec. 2.5) in order.  run(phase, fn)
// enqueues fn() as part of `phase` (the groups of cffyn_profile_step; phase
// 10 is the per-field exponent scan of the mixed path in front of each
// operator group); tracing and profiling hooks live in run.  A step is, for
// every stage s = 0..3, stage_front (derivatives and right-hand side of the
// stage state into sh->S) then stage_back (filter of the right-hand side and
// the stage update), then step_tail (the filter of the new state in
// per-step mode).  Nested shells run the fronts of all their shells, couple
// the right-hand sides on the common spheres, then run the backs.
extern "C++" {

// the state that stage s reads: on the mixed path the pair copy Uf of the
// step's initial state in stage 0 (cffyn_rk4_step fills it from u before the
// first step and the last stage keeps it current) and the pair-stored stage
// state U after it; on the FP64 path u, then U
static const double* stage_state_of(const cffyn_shell* sh, const double* u, int s) {
  const bool mixed = sh->d.precision == CFFYN_MIXED;
  return s == 0 ? (mixed ? sh->Uf : u) : sh->U;
}

// The two halves of the Yn filter's spin slots that conc runs as two chains
// (phi analysis, projection, phi synthesis) on two streams: slots 0 .. 23 (the
// 16 real spin-0 slots and the first 4 spin-1 pairs) and the rest (the other
// spin-1 pairs, spin 2, spin 3 and the gauge slots).  Each half is a whole
// set of projection classes, so the chains share no buffer; each fills the
// partly empty last wave of the other's launches (3.228 -> 3.135 ms per step
// on the 33 x 48 x 96 shell).
constexpr int kSplitR0 = 16, kSplitC1 = 4, kSplitSlots = kSplitR0 + 2 * kSplitC1;

// filter of the functions in `spin` (in place through D and D + nvP): the
// spin slots for Yn, the Cartesian fields for Y / Yg; one exponent scan per
// filter (the coefficients and the projected ones take bounds: the scan's
// exponents + the operators' gains).  conc: the Yn filter of the mixed path
// as two chains on the shell's two streams (see kSplitSlots).
template <class Run>
static int filter_in_step(cffyn_shell* sh, double* spin, cudaStream_t st, Run&& run, bool conc) {
  const size_t nvP = (size_t)sh->nv * P_all(sh);
  const int nf = nv_ops(sh);
  const bool yn = yn_filter(sh);
  const int pairing = yn ? 1 : 0;
  const int e1 = sh->gain_dft, e2 = sh->gain_dft + sh->gain_proj;
  const int* cl[3] = {slots_c(sh, 0), slots_c(sh, 1), slots_c(sh, 2)};
  int r;
  if ((r = run(10, [&] { return op_prepare(sh, spin, true, nf, (long long)sh->P, pairing, st); })))
    return r;
  if (conc && yn && sh->d.precision == CFFYN_MIXED && sh->aux_stream && sh->nR0 >= kSplitR0 &&
      sh->nC[0] >= kSplitC1) {
    cudaStream_t sa = sh->aux_stream;
    const int fa = kSplitSlots * sh->ns;  // arrays of the first half (stacked: [slot][shell])
    const int* ca[3] = {cl[0], nullptr, nullptr};
    const int na[3] = {kSplitC1, 0, 0};
    const int* cb[3] = {cl[0] + kSplitC1, cl[1], cl[2]};
    const int nb[3] = {sh->nC[0] - kSplitC1, sh->nC[1], sh->nC[2]};
    CF_CUDA(cudaEventRecord(sh->ev_fork, st));
    CF_CUDA(cudaStreamWaitEvent(sa, sh->ev_fork, 0));
    if ((r = run(6, [&] {
           int q = op_dft_fwd(sh, spin, sh->D, fa, st, pairing, 0);
           return q ? q : op_dft_fwd(sh, spin, sh->D, nf - fa, sa, pairing, fa);
         })))
      return r;
    if ((r = run(7, [&] {
           int q = op_project(sh, sh->D, sh->D + nvP, slots_r0(sh), kSplitR0, ca, na, st, e1);
           return q ? q
                    : op_project(sh, sh->D, sh->D + nvP, slots_r0(sh) + kSplitR0, sh->nR0 - kSplitR0, cb, nb,
                                 sa, e1);
         })))
      return r;
    if ((r = run(8, [&] {
           int q = op_dft_inv(sh, sh->D + nvP, spin, fa, st, pairing, e2, 0);
           return q ? q : op_dft_inv(sh, sh->D + nvP, spin, nf - fa, sa, pairing, e2, fa);
         })))
      return r;
    CF_CUDA(cudaEventRecord(sh->ev_join, sa));
    CF_CUDA(cudaStreamWaitEvent(st, sh->ev_join, 0));
    return CFFYN_OK;
  }
  if ((r = run(6, [&] { return op_dft_fwd(sh, spin, sh->D, nf, st, pairing); }))) return r;
  if ((r = run(7, [&] {
         return yn ? op_project(sh, sh->D, sh->D + nvP, slots_r0(sh), sh->nR0, cl, sh->nC, st, e1)
                   : op_project_scalar(sh, sh->D, sh->D + nvP, st, e1);
       })))
    return r;
  return run(8, [&] { return op_dft_inv(sh, sh->D + nvP, spin, nf, st, pairing, e2); });
}

// conc: the algebraic right-hand-side kernels (k_rhs_gamma, k_rhs_quad: they
// read the stage state only) run on the shell's second stream beside the
// d_theta + d_phi launch, which they share no buffer with, and join before
// the principal parts; forked after d_r (forked at the start of the stage,
// they held up the exponent scan and d_r: 3.233 vs 3.248 ms per step); not
// for the evolved gauge of 54/58 fields (k_gauge_rhs reads the derivatives)
// nor under per-group timing.
template <class Run>
static int stage_front(cffyn_shell* sh, double* u, int s, cudaStream_t st, Run&& run, bool conc) {
  const size_t nvP = (size_t)sh->nv * P_all(sh);
  const long long P = (long long)sh->P;
  const int nf = nv_ops(sh);
  const bool xp = sh->d.precision == CFFYN_MIXED;
  const double* X = stage_state_of(sh, u, s);
  int rc;
  const bool fork = conc && sh->ng == 0 && sh->aux_stream;
  cudaStream_t sa = fork ? sh->aux_stream : st;
  if ((rc = run(10, [&] { return op_prepare(sh, X, xp, nf, P, 0, st); }))) return rc;
  if ((rc = run(0, [&] { return op_deriv_r(sh, X, sh->D, nf, xp, st); }))) return rc;
  if (fork) {
    CF_CUDA(cudaEventRecord(sh->ev_fork, st));
    CF_CUDA(cudaStreamWaitEvent(sa, sh->ev_fork, 0));
    if ((rc = run(2, [&] { return pw_rhs_part(sh, X, sh->D, sh->S, 1, xp, true, sa); }))) return rc;
    if ((rc = run(3, [&] { return pw_rhs_part(sh, X, sh->D, sh->S, 2, xp, true, sa); }))) return rc;
    CF_CUDA(cudaEventRecord(sh->ev_join, sa));
  }
  if ((rc = run(1, [&] { return op_deriv_theta_phi(sh, X, sh->D + nvP, sh->D + 2 * nvP, nf, xp, st); })))
    return rc;
  if (fork) {
    CF_CUDA(cudaStreamWaitEvent(st, sh->ev_join, 0));
  } else {
    if ((rc = run(2, [&] { return pw_rhs_part(sh, X, sh->D, sh->S, 1, xp, true, st); }))) return rc;
    if ((rc = run(3, [&] { return pw_rhs_part(sh, X, sh->D, sh->S, 2, xp, true, st); }))) return rc;
  }
  return run(4, [&] { return pw_rhs_part(sh, X, sh->D, sh->S, 3, xp, true, st); });
}

template <class Run>
static int stage_back(cffyn_shell* sh, double* u, double dt, int s, cudaStream_t st, Run&& run, bool conc) {
  const size_t nvP = (size_t)sh->nv * P_all(sh);
  const bool per_sub = sh->d.filter_mode == CFFYN_FILTER_SUBSTEP;
  int rc;
  if (per_sub && yn_filter(sh)) {
    double* spin = sh->D + 2 * nvP;  // derivatives are dead after the rhs
    if ((rc = run(5, [&] { return pw_decompose(sh, sh->S, spin, true, st); }))) return rc;
    if ((rc = filter_in_step(sh, spin, st, run, conc))) return rc;
    return run(9, [&] {
      return pw_reconstruct(sh, spin, nullptr, 1 + s, u, sh->U, sh->kacc, sh->Uf, dt, sh->flag, st);
    });
  }
  // unfiltered stage rhs (per-step placement), or the component-wise filter
  // applied to the Cartesian rhs in place
  if (per_sub && (rc = filter_in_step(sh, sh->S, st, run, conc))) return rc;
  return run(9, [&] {
    return pw_reconstruct(sh, sh->S, nullptr, 5 + s, u, sh->U, sh->kacc, sh->Uf, dt, sh->flag, st);
  });
}

template <class Run>
static int step_tail(cffyn_shell* sh, double* u, cudaStream_t st, Run&& run, bool conc) {
  if (sh->d.filter_mode == CFFYN_FILTER_SUBSTEP) return CFFYN_OK;
  const size_t nvP = (size_t)sh->nv * P_all(sh);
  const bool mixed = sh->d.precision == CFFYN_MIXED;
  const bool yn = yn_filter(sh);
  int rc;
  if (yn) {
    if ((rc = run(5, [&] { return pw_decompose(sh, mixed ? sh->Uf : u, sh->S, mixed, st); }))) return rc;
  } else {
    // the Cartesian state itself (pairs on the mixed path)
    if ((rc = run(5, [&] {
           CF_CUDA(cudaMemcpyAsync(sh->S, mixed ? sh->Uf : u, nvP * sizeof(double), cudaMemcpyDeviceToDevice, st));
           return CFFYN_OK;
         })))
      return rc;
  }
  if ((rc = filter_in_step(sh, sh->S, st, run, conc))) return rc;
  return run(9, [&] {
    return pw_reconstruct(sh, sh->S, u, yn ? 0 : 9, nullptr, nullptr, nullptr, sh->Uf, 0.0, sh->flag, st);
  });
}

template <class Run>
static int step_sequence(cffyn_shell* sh, double* u, double dt, cudaStream_t st, Run&& run, bool conc) {
  int rc;
  for (int s = 0; s < 4; ++s) {
    if ((rc = stage_front(sh, u, s, st, run, conc))) return rc;
    if ((rc = stage_back(sh, u, dt, s, st, run, conc))) return rc;
  }
  return step_tail(sh, u, st, run, conc);
}
}  // extern "C++"

// One RK4 step on u (enqueued on st); see cffyn_rk4_step.  With tracing on,
// an event is recorded after every kernel group; mark_phase says which group
// ended at each mark, launches_per_step counts kernel launches per group.
static int enqueue_step(cffyn_shell* sh, double* u, double dt, cudaStream_t st) {
  const bool tr = sh->trace != 0;
  int nm = 0;
  for (int k = 0; k < cffyn_shell::kPhases; ++k) sh->launches_per_step[k] = 0;
  auto mark = [&](int phase) -> int {
    if (!tr) return CFFYN_OK;
    if (nm >= cffyn_shell::kMaxMarks || !sh->marks[nm]) return CFFYN_OK;
    sh->mark_phase[nm] = phase;
    // inside a capture a plain record only joins streams; External makes it an
    // event-record node of the graph
    CF_CUDA(cudaEventRecordWithFlags(sh->marks[nm], st, cudaEventRecordExternal));
    ++nm;
    return CFFYN_OK;
  };
  auto run = [&](int phase, auto&& fn) -> int {
    long long l0 = g_launches;
    int r = fn();
    if (r) return r;
    sh->launches_per_step[phase] += (int)(g_launches - l0);
    return mark(phase);
  };
  int rc;
  if ((rc = mark(-1))) return rc;
  // traced: one stream, so that the marks bound the kernel groups
  if ((rc = step_sequence(sh, u, dt, st, run, !tr))) return rc;
  sh->n_marks = nm;
  return CFFYN_OK;
}

extern "C++" {
namespace cffyn {

// One RK4 step enqueued on st without trace marks (a branch of a batch graph).
int enqueue_step_branch(cffyn_shell* sh, double* u, double dt, cudaStream_t st) {
  auto run = [](int, auto&& fn) -> int { return fn(); };
  return step_sequence(sh, u, dt, st, run, true);
}

// The pieces of a step for nested shells (no trace marks): stage s's
// derivatives and right-hand side into sh->S, its filter and update, and
// the per-step filter after the last stage.
int enqueue_stage_front(cffyn_shell* sh, double* u, int s, cudaStream_t st) {
  auto run = [](int, auto&& fn) -> int { return fn(); };
  return stage_front(sh, u, s, st, run, true);
}
int enqueue_stage_back(cffyn_shell* sh, double* u, double dt, int s, cudaStream_t st) {
  auto run = [](int, auto&& fn) -> int { return fn(); };
  return stage_back(sh, u, dt, s, st, run, true);
}
int enqueue_step_tail(cffyn_shell* sh, double* u, cudaStream_t st) {
  auto run = [](int, auto&& fn) -> int { return fn(); };
  return step_tail(sh, u, st, run, true);
}
const double* stage_state(const cffyn_shell* sh, const double* u, int s) { return stage_state_of(sh, u, s); }

// Derivatives and right-hand side (with the outer boundary condition) of an
// FP64 state u into the FP64 array dudt, as cffyn_rhs does.
int enqueue_rhs(cffyn_shell* sh, const double* u, double* dudt, cudaStream_t st) {
  int rc;
  if ((rc = derivs_spherical(sh, u, sh->D, sh->nv, false, st))) return rc;
  return pw_rhs(sh, u, sh->D, dudt, st);
}

// Work in front of the first step of a call: clear the finiteness flag and,
// on the mixed path, copy u into the pair-stored initial state Uf (the last
// stage of every step keeps Uf current afterwards).
int enqueue_step_prologue(cffyn_shell* sh, double* u, cudaStream_t st) {
  CF_CUDA(cudaMemsetAsync(sh->flag, 0, sizeof(int), st));
  if (sh->Uf) return pw_to_internal(sh, u, sh->Uf, (long long)sh->nv * (long long)P_all(sh), st);
  return CFFYN_OK;
}

// Status of a step call from the flag word its kernels set.
int step_flag_status(int flag) {
  if (flag & 2) {
    set_error("a bounded tensor-core wait gave up (operator results are invalid)");
    return CFFYN_ETIMEOUT;
  }
  if (flag) {
    set_error("non-finite value in a stage right-hand side");
    return CFFYN_ENONFINITE;
  }
  return CFFYN_OK;
}

int check_step_ready(const cffyn_shell* sh) {
  int rc;
  if ((rc = check_ws(sh))) return rc;
  if (sh->nv == 50 && !sh->gauge_set) {
    set_error("gauge source not set (cffyn_set_gauge / cffyn_init_gauge_from_state)");
    return CFFYN_EINVAL;
  }
  return CFFYN_OK;
}

int check_state_ptr(const void* p, const char* what) { return check_ptr(p, what); }

}  // namespace cffyn
}  // extern "C++"

// The captured step graph for (u, dt) and the shell's trace setting: one of
// the two kept (the shell's mark table and launch counts then describe it),
// else captured and instantiated in place of the less recently used one.
static int step_graph(cffyn_shell* sh, double* u, double dt, cudaGraphExec_t* out) {
  for (int e = 0; e < cffyn_shell::kStepGraphs; ++e) {
    cffyn_shell::StepGraph& g = sh->graphs[e];
    if (g.exec && g.u == u && g.dt == dt && g.trace == sh->trace) {
      sh->n_marks = g.n_marks;
      for (int i = 0; i < cffyn_shell::kMaxMarks; ++i) sh->mark_phase[i] = g.mark_phase[i];
      for (int k = 0; k < cffyn_shell::kPhases; ++k) sh->launches_per_step[k] = g.launches[k];
      sh->graph_victim = (e + 1) % cffyn_shell::kStepGraphs;
      *out = g.exec;
      return CFFYN_OK;
    }
  }
  cffyn_shell::StepGraph& g = sh->graphs[sh->graph_victim];
  if (g.exec) {
    cudaGraphExecDestroy(g.exec);  // a replay still in flight completes first
    g.exec = nullptr;
  }
  cudaGraph_t cg;
  CF_CUDA(cudaStreamBeginCapture(sh->cap_stream, cudaStreamCaptureModeThreadLocal));
  int erc = enqueue_step(sh, u, dt, sh->cap_stream);
  cudaError_t ce = cudaStreamEndCapture(sh->cap_stream, &cg);
  if (erc) return erc;
  if (ce != cudaSuccess) {
    set_error("graph capture failed: %s", cudaGetErrorString(ce));
    return CFFYN_ECUDA;
  }
  ce = cudaGraphInstantiate(&g.exec, cg, 0);
  cudaGraphDestroy(cg);
  if (ce != cudaSuccess) {
    g.exec = nullptr;
    set_error("graph instantiation failed: %s", cudaGetErrorString(ce));
    return CFFYN_ECUDA;
  }
  g.u = u;
  g.dt = dt;
  g.trace = sh->trace;
  g.n_marks = sh->n_marks;
  for (int i = 0; i < cffyn_shell::kMaxMarks; ++i) g.mark_phase[i] = sh->mark_phase[i];
  for (int k = 0; k < cffyn_shell::kPhases; ++k) g.launches[k] = sh->launches_per_step[k];
  sh->graph_victim = (sh->graph_victim + 1) % cffyn_shell::kStepGraphs;
  *out = g.exec;
  return CFFYN_OK;
}

// Argument checks shared by the synchronous and asynchronous step calls.
static int check_step_call(cffyn_shell* sh, double* u, int n_steps) {
  if (!sh) { set_error("shell is NULL"); return CFFYN_EINVAL; }
  int rc;
  if ((rc = check_ptr(u, "u"))) return rc;
  if (n_steps < 0) { set_error("n_steps < 0"); return CFFYN_EINVAL; }
  return check_step_ready(sh);
}

int cffyn_rk4_step_async(cffyn_shell* sh, double* u, double dt, int n_steps, void* stream, int* status) {
  int rc;
  if ((rc = check_step_call(sh, u, n_steps))) return rc;
  if (!status) { set_error("status is NULL"); return CFFYN_EINVAL; }
  if (sh->trace) { set_error("tracing is on: use cffyn_rk4_step"); return CFFYN_EINVAL; }
  cudaStream_t st = (cudaStream_t)stream;
  if (n_steps == 0) {
    // nothing runs; the status word still arrives in stream order
    CF_CUDA(cudaMemsetAsync(sh->flag, 0, sizeof(int), st));
  } else {
    if (!(dt > 0)) dt = sh->dt_default;
    cudaGraphExec_t ge = nullptr;
    if ((rc = step_graph(sh, u, dt, &ge))) return rc;
    if ((rc = enqueue_step_prologue(sh, u, st))) return rc;
    for (int i = 0; i < n_steps; ++i) CF_CUDA(cudaGraphLaunch(ge, st));
  }
  CF_CUDA(cudaMemcpyAsync(status, sh->flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  return CFFYN_OK;
}

int cffyn_step_status(int status_word) { return step_flag_status(status_word); }

int cffyn_rk4_step(cffyn_shell* sh, double* u, double dt, int n_steps, void* stream) {
  int rc;
  if ((rc = check_step_call(sh, u, n_steps))) return rc;
  if (n_steps == 0) return CFFYN_OK;
  if (!(dt > 0)) dt = sh->dt_default;
  cudaStream_t st = (cudaStream_t)stream;
  cudaGraphExec_t ge = nullptr;
  if ((rc = step_graph(sh, u, dt, &ge))) return rc;
  if ((rc = enqueue_step_prologue(sh, u, st))) return rc;
  for (int i = 0; i < n_steps; ++i) CF_CUDA(cudaGraphLaunch(ge, st));
  CF_CUDA(cudaMemcpyAsync(sh->flag_host, sh->flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  CF_CUDA(cudaStreamSynchronize(st));
  if (sh->trace && sh->n_marks > 1) {
    // the marks hold the last replay; count it n_steps times
    for (int i = 1; i < sh->n_marks; ++i) {
      float ms = 0.f;
      cudaError_t e = cudaEventElapsedTime(&ms, sh->marks[i - 1], sh->marks[i]);
      if (e != cudaSuccess) {
        cudaGetLastError();  // do not leave the failure for the next launch check
        set_error("trace: %s", cudaGetErrorString(e));
        return CFFYN_ECUDA;
      }
      if (sh->mark_phase[i] >= 0) sh->trace_ms[sh->mark_phase[i]] += (double)ms * n_steps;
    }
    sh->trace_steps += n_steps;
  }
  return step_flag_status(*sh->flag_host);
}

int cffyn_set_operator_rows(cffyn_shell* sh, int family, int rows) {
  if (!sh) { set_error("shell is NULL"); return CFFYN_EINVAL; }
  if (family < 0 || family >= kOpFamilies || (rows != 0 && rows != 48 && rows != 96)) {
    set_error("operator family %d outside 0..%d or rows %d not 0, 48 or 96", family, kOpFamilies - 1, rows);
    return CFFYN_EINVAL;
  }
  if (sh->op_rows[family] == rows) return CFFYN_OK;
  if (sh->d.precision != CFFYN_MIXED) {
    sh->op_rows[family] = rows;
    return CFFYN_OK;
  }
  CF_CUDA(cudaDeviceSynchronize());
  const int old = sh->op_rows[family];
  sh->op_rows[family] = rows;
  int rc;
  if ((rc = build_tc_family(sh, family))) {
    sh->op_rows[family] = old;
    build_tc_family(sh, family);
    return rc;
  }
  drop_step_graphs(sh);
  ++sh->ws_gen;
  return CFFYN_OK;
}

int cffyn_get_operator_rows(const cffyn_shell* sh, int family) {
  if (!sh || family < 0 || family >= kOpFamilies) return 0;
  const cffyn::TcOp* t[kOpFamilies] = {&sh->tDr, &sh->tDth2, &sh->tFan, &sh->tF0, &sh->tFsy};
  return sh->d.precision == CFFYN_MIXED ? t[family]->rows : sh->op_rows[family];
}

int cffyn_set_wait_limit(cffyn_shell* sh, double seconds) {
  if (!sh) { set_error("shell is NULL"); return CFFYN_EINVAL; }
  if (!(seconds == seconds) || seconds > 60.0) {
    set_error("wait limit %g s outside [0, 60]", seconds);
    return CFFYN_EINVAL;
  }
  const unsigned long long ns = seconds < 0 ? 1000000000ull : (unsigned long long)(seconds * 1e9);
  if (ns == sh->tc_wait_ns) return CFFYN_OK;
  sh->tc_wait_ns = ns;
  // the bound is a parameter of the captured kernels
  drop_step_graphs(sh);
  ++sh->ws_gen;
  return CFFYN_OK;
}

int cffyn_set_trace(cffyn_shell* sh, int on) {
  if (!sh) { set_error("shell is NULL"); return CFFYN_EINVAL; }
  sh->trace = on ? 1 : 0;
  if (sh->trace)  // events are created here, never during a stream capture
    for (int i = 0; i < cffyn_shell::kMaxMarks; ++i)
      if (!sh->marks[i]) CF_CUDA(cudaEventCreate(&sh->marks[i]));
  for (int k = 0; k < cffyn_shell::kPhases; ++k) sh->trace_ms[k] = 0.0;
  sh->trace_steps = 0;
  return CFFYN_OK;
}

int cffyn_get_trace(const cffyn_shell* sh, double* ms_out, int* launches_out, long long* steps) {
  if (!sh || !ms_out || !launches_out || !steps) { set_error("NULL argument"); return CFFYN_EINVAL; }
  for (int k = 0; k < cffyn_shell::kPhases; ++k) {
    ms_out[k] = sh->trace_ms[k];
    launches_out[k] = sh->launches_per_step[k];
  }
  *steps = sh->trace_steps;
  return CFFYN_OK;
}

int cffyn_constraint_norms(cffyn_shell* sh, const double* u, double out[2], void* stream) {
  if (!sh) { set_error("shell is NULL"); return CFFYN_EINVAL; }
  int rc;
  if ((rc = check_ptr(u, "u"))) return rc;
  if (!out) { set_error("out is NULL"); return CFFYN_EINVAL; }
  if ((rc = check_ws(sh))) return rc;
  if (sh->nv == 50 && !sh->gauge_set) {
    set_error("gauge source not set");
    return CFFYN_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  // derivatives of g_ab only (fields 0..9)
  if ((rc = derivs_spherical(sh, u, sh->D, 10, false, st))) return rc;
  double* dcart = sh->S;  // [3][10][P], FP64
  if ((rc = pw_cart(sh, sh->D, dcart, 10, false, st))) return rc;
  double* red = sh->red;
  CF_CUDA(cudaMemsetAsync(red, 0, 2 * sizeof(double), st));
  // the gauge source: the stored one (50 fields) or fields 50..53 of u
  const bool h_int = sh->nv == 50;
  if ((rc = pw_constraints(sh, u, dcart, h_int ? sh->H : u + (size_t)50 * sh->P, h_int, red, st))) return rc;
  double h[2];
  CF_CUDA(cudaMemcpyAsync(h, red, sizeof(h), cudaMemcpyDeviceToHost, st));
  CF_CUDA(cudaStreamSynchronize(st));
  out[0] = sqrt(h[0] / (30.0 * sh->P));
  out[1] = sqrt(h[1] / (4.0 * sh->P));
  return CFFYN_OK;
}

int cffyn_get_filter_matrix(const cffyn_shell* sh, int n, int m, double* host_out) {
  if (!sh || !host_out) { set_error("NULL argument"); return CFFYN_EINVAL; }
  if (n < -3 || n > 3 || m < 0 || m > sh->L) {
    set_error("n must be in [-3,3] and m in [0,L]");
    return CFFYN_EINVAL;
  }
  const size_t per = (size_t)sh->N * sh->N;
  CF_CUDA(cudaMemcpy(host_out, sh->Fraw + ((size_t)(n + 3) * (sh->L + 1) + m) * per, per * sizeof(double),
                     cudaMemcpyDeviceToHost));
  return CFFYN_OK;
}

int cffyn_get_operator(const cffyn_shell* sh, int which, double* host_out) {
  if (!sh || !host_out) { set_error("NULL argument"); return CFFYN_EINVAL; }
  if (which == 0) {
    CF_CUDA(cudaMemcpy(host_out, sh->Dr, (size_t)sh->n_r * sh->n_r * sizeof(double), cudaMemcpyDeviceToHost));
  } else if (which == 1) {
    // top N rows of the 2N x 2N pair operator
    CF_CUDA(cudaMemcpy(host_out, sh->Dth2, (size_t)sh->N * 2 * sh->N * sizeof(double), cudaMemcpyDeviceToHost));
  } else if (which == 2) {
    CF_CUDA(cudaMemcpy(host_out, sh->Dph, (size_t)sh->J * sh->J * sizeof(double), cudaMemcpyDeviceToHost));
  } else {
    set_error("which must be 0, 1 or 2");
    return CFFYN_EINVAL;
  }
  return CFFYN_OK;
}

int cffyn_profile_step(cffyn_shell* sh, double* u, double dt, double* ms_out, int* launches_out,
                       void* stream) {
  if (!sh) { set_error("shell is NULL"); return CFFYN_EINVAL; }
  int rc;
  if ((rc = check_ptr(u, "u"))) return rc;
  if (!ms_out || !launches_out) { set_error("outputs are NULL"); return CFFYN_EINVAL; }
  if ((rc = check_ws(sh))) return rc;
  if (sh->nv == 50 && !sh->gauge_set) { set_error("gauge source not set"); return CFFYN_EINVAL; }
  if (!(dt > 0)) dt = sh->dt_default;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t ev[2];
  CF_CUDA(cudaEventCreate(&ev[0]));
  CF_CUDA(cudaEventCreate(&ev[1]));
  for (int k = 0; k < CFFYN_PROFILE_PHASES; ++k) {
    ms_out[k] = 0.0;
    launches_out[k] = 0;
  }
  auto phase = [&](int k, auto&& fn) -> int {
    long long l0 = g_launches;
    cudaEventRecord(ev[0], st);
    int r = fn();
    cudaEventRecord(ev[1], st);
    if (r) return r;
    if (cudaEventSynchronize(ev[1]) != cudaSuccess) {
      set_error("profiling: %s", cudaGetErrorString(cudaGetLastError()));
      return CFFYN_ECUDA;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev[0], ev[1]);
    ms_out[k] += ms;
    launches_out[k] += (int)(g_launches - l0);
    return CFFYN_OK;
  };
  if ((rc = enqueue_step_prologue(sh, u, st))) return rc;
  rc = step_sequence(sh, u, dt, st, phase, false);
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  return rc;
}

}  // extern "C"
