// Nested spherical shells (the domain decomposition the paper names as the
// way to resolve local features and as its next step, Secs. 1 and 5):
// shells s = 0 .. n-1 over [R_s, R_{s+1}] with a common angular grid, each
// advanced by the single-shell kernels, coupled on every common sphere (the
// outer sphere of shell s is the inner sphere of shell s + 1: both
// Chebyshev-Gauss-Lobatto grids contain their end radii) through the
// characteristic fields of App. A.2 (eq. characteristics), with the normal
// s_i of the common sphere from the inner shell's metric:
//
//   w0 = g (speed 0), w+ = -g + Pi + s^k Phi_k (alpha - b),
//   w- = -g + Pi - s^k Phi_k (-alpha - b), wT_i = Phi_i - s_i s^k Phi_k (-b).
//
// The fields that App. A.2's outer condition freezes (w-, wT: they enter the
// inner shell from outside) take the outer shell's right-hand side, w0 and
// w+ the inner shell's; back-transformed,
//   d_t g = w0, d_t Pi = (w+ + w-)/2 + w0, d_t Phi_i = s_i (w+ - w-)/2 + wT_i,
// written into both shells' right-hand sides on the common sphere (gauge
// fields of 54/58-field states: the inner shell's).  The inner shells'
// freeze-incoming condition on their outer sphere keeps w0 and w+, so the
// coupling may follow it.  One RK4 step of the nest runs, for every stage,
// the derivatives and right-hand sides of all shells, the couplings, then
// the filters and stage updates of all shells; it is captured in one CUDA
// graph.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <new>
#include <vector>

#include "pw_common.cuh"

namespace cffyn {
int enqueue_stage_front(cffyn_shell*, double*, int, cudaStream_t);
int enqueue_stage_back(cffyn_shell*, double*, double, int, cudaStream_t);
int enqueue_step_tail(cffyn_shell*, double*, cudaStream_t);
int enqueue_step_prologue(cffyn_shell*, double*, cudaStream_t);
int enqueue_rhs(cffyn_shell*, const double*, double*, cudaStream_t);
const double* stage_state(const cffyn_shell*, const double*, int);
int step_flag_status(int);
int check_step_ready(const cffyn_shell*);
int check_state_ptr(const void*, const char*);

// One thread per point of the common sphere (j, i).  XA: the inner shell's
// state (storage FX), SA / SB: the right-hand sides of the inner and outer
// shells (storage FR), updated in place on the common sphere.
template <class T, bool FX, bool FR>
__global__ void __launch_bounds__(128) k_interface(const double* __restrict__ XA, double* __restrict__ SA,
                                                   double* __restrict__ SB, Geo ga, int nrB, long long PB) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= ga.N * ga.J) return;
  const int i = q % ga.N, jj = q / ga.N;
  const long long PA = ga.P;
  const long long pa = (long long)q * ga.n_r + (ga.n_r - 1);
  const long long pb = (long long)q * nrB;
  T g[10];
#pragma unroll
  for (int c = 0; c < 10; ++c) g[c] = Store<T, FX>::ld(XA, (long long)c * PA + pa);
  Metric<T> M;
  metric_from(g, M);
  const T st = S<T>::c(ga.sth[i]), ct = S<T>::c(ga.cth[i]);
  const T sp = S<T>::c(ga.sph[jj]), cp = S<T>::c(ga.cph[jj]);
  const T l[3] = {st * cp, st * sp, ct};
  Acc<T> qa;
#pragma unroll
  for (int x = 0; x < 3; ++x)
#pragma unroll
    for (int y = 0; y < 3; ++y) qa.fma_(M.gi[x][y] * l[x], l[y]);
  const T iq = S<T>::c(1.0) / sqrt_s(qa.get());
  T sl[3], su[3];
#pragma unroll
  for (int x = 0; x < 3; ++x) sl[x] = l[x] * iq;
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    Acc<T> acc;
#pragma unroll
    for (int y = 0; y < 3; ++y) acc.fma_(M.gi[x][y], sl[y]);
    su[x] = acc.get();
  }
  const T half = S<T>::c(0.5);
#pragma unroll 1
  for (int c = 0; c < 10; ++c) {
    auto lda = [&](int f) { return Store<T, FR>::ld(SA, (long long)f * PA + pa); };
    auto ldb = [&](int f) { return Store<T, FR>::ld(SB, (long long)f * PB + pb); };
    const T ag = lda(c), aPi = lda(10 + c), bg = ldb(c), bPi = ldb(10 + c);
    T aPh[3], bPh[3];
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      aPh[x] = lda(20 + 10 * x + c);
      bPh[x] = ldb(20 + 10 * x + c);
    }
    Acc<T> sa, sb;
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      sa.fma_(su[x], aPh[x]);
      sb.fma_(su[x], bPh[x]);
    }
    const T sPa = sa.get(), sPb = sb.get();
    const T w0 = ag;
    const T wp = (aPi - ag) + sPa;
    const T wm = (bPi - bg) - sPb;
    const T rPi = half * (wp + wm) + w0;
    const T d = half * (wp - wm);
    T rPh[3];
#pragma unroll
    for (int x = 0; x < 3; ++x) rPh[x] = sl[x] * d + (bPh[x] - sl[x] * sPb);
    const int fs[5] = {c, 10 + c, 20 + c, 30 + c, 40 + c};
    const T vs[5] = {w0, rPi, rPh[0], rPh[1], rPh[2]};
#pragma unroll
    for (int e = 0; e < 5; ++e) {
      Store<T, FR>::st(SA, (long long)fs[e] * PA + pa, vs[e]);
      Store<T, FR>::st(SB, (long long)fs[e] * PB + pb, vs[e]);
    }
  }
  for (int f = 50; f < ga.nv; ++f)
    Store<T, FR>::st(SB, (long long)f * PB + pb, Store<T, FR>::ld(SA, (long long)f * PA + pa));
}

// Coupling on the common sphere of shells a (inner) and b (outer): XA the
// inner shell's state, SA / SB the right-hand sides.  x_pairs / r_pairs: the
// state / the right-hand sides are pair-stored internal buffers of the mixed
// path (else FP64 arrays).
static int couple(const cffyn_shell* a, const cffyn_shell* b, const double* XA, double* SA, double* SB,
                  bool x_pairs, bool r_pairs, cudaStream_t st) {
  Geo g = geo_of(a);
  const unsigned nb = blocks_for((long long)a->N * a->J, 128);
  const long long PB = (long long)b->P;
  if (a->d.precision == CFFYN_FP64)
    k_interface<double, false, false><<<nb, 128, 0, st>>>(XA, SA, SB, g, b->n_r, PB);
  else if (x_pairs && r_pairs)
    k_interface<ff, true, true><<<nb, 128, 0, st>>>(XA, SA, SB, g, b->n_r, PB);
  else if (!x_pairs && !r_pairs)
    k_interface<ff, false, false><<<nb, 128, 0, st>>>(XA, SA, SB, g, b->n_r, PB);
  else {
    set_error("internal: coupling storage (state %d, rhs %d) not instantiated", (int)x_pairs, (int)r_pairs);
    return CFFYN_EINVAL;
  }
  count_launch();
  CF_CUDA(cudaGetLastError());
  return CFFYN_OK;
}

}  // namespace cffyn

using namespace cffyn;

struct cffyn_nest {
  int n = 0;
  int device = 0;
  std::vector<cffyn_shell*> sh;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t graph = nullptr;
  std::vector<double*> gu;
  double gdt = 0.0;
  std::vector<unsigned> ggen;
  int* flags_host = nullptr;  // pinned, one word per shell
  double dt_default = 0.0;
};

namespace {

void free_nest(cffyn_nest* ns) {
  if (!ns) return;
  cudaDeviceSynchronize();
  if (ns->graph) cudaGraphExecDestroy(ns->graph);
  if (ns->cap) cudaStreamDestroy(ns->cap);
  if (ns->flags_host) cudaFreeHost(ns->flags_host);
  delete ns;
}

// One RK4 step of every shell of the nest on st.
int enqueue_nest_step(cffyn_nest* ns, double* const* u, double dt, cudaStream_t st) {
  int rc;
  const bool mixed = ns->sh[0]->d.precision == CFFYN_MIXED;
  for (int s = 0; s < 4; ++s) {
    for (int i = 0; i < ns->n; ++i)
      if ((rc = enqueue_stage_front(ns->sh[i], u[i], s, st))) return rc;
    for (int i = 0; i + 1 < ns->n; ++i) {
      cffyn_shell* a = ns->sh[i];
      if ((rc = couple(a, ns->sh[i + 1], stage_state(a, u[i], s), a->S, ns->sh[i + 1]->S, mixed, mixed, st)))
        return rc;
    }
    for (int i = 0; i < ns->n; ++i)
      if ((rc = enqueue_stage_back(ns->sh[i], u[i], dt, s, st))) return rc;
  }
  for (int i = 0; i < ns->n; ++i)
    if ((rc = enqueue_step_tail(ns->sh[i], u[i], st))) return rc;
  return CFFYN_OK;
}

int check_states(const cffyn_nest* ns, const double* const* u, const char* what) {
  if (!u) {
    set_error("%s is NULL", what);
    return CFFYN_EINVAL;
  }
  for (int i = 0; i < ns->n; ++i) {
    int rc;
    if ((rc = check_state_ptr(u[i], what))) return rc;
  }
  return CFFYN_OK;
}

}  // namespace

extern "C" {

int cffyn_create_nest(int n, cffyn_shell* const* shells, cffyn_nest** out) {
  if (!out) {
    set_error("out is NULL");
    return CFFYN_EINVAL;
  }
  *out = nullptr;
  if (n < 1 || !shells) {
    set_error("a nest needs n >= 1 shells (n = %d)", n);
    return CFFYN_EINVAL;
  }
  int dev = 0;
  CF_CUDA(cudaGetDevice(&dev));
  for (int i = 0; i < n; ++i) {
    const cffyn_shell* s = shells[i];
    if (!s) {
      set_error("shell %d is NULL", i);
      return CFFYN_EINVAL;
    }
    if (s->device != dev) {
      set_error("shell %d lives on device %d, the current device is %d", i, s->device, dev);
      return CFFYN_EINVAL;
    }
    const cffyn_shell* f = shells[0];
    if (s->N != f->N || s->L != f->L || s->nv != f->nv || s->d.precision != f->d.precision ||
        s->d.filter_mode != f->d.filter_mode || s->d.filter_kind != f->d.filter_kind) {
      set_error("shell %d differs from shell 0 in n_theta, L, n_fields, precision or filter", i);
      return CFFYN_EINVAL;
    }
    for (int j = 0; j < i; ++j)
      if (shells[j] == s) {
        set_error("a shell appears twice in the nest");
        return CFFYN_EINVAL;
      }
    if (i > 0) {
      const double a = shells[i - 1]->d.r_out, b = s->d.r_in;
      if (!(std::fabs(a - b) <= 1e-12 * std::fabs(b))) {
        set_error("shell %d starts at r = %.17g but shell %d ends at r = %.17g", i, b, i - 1, a);
        return CFFYN_EINVAL;
      }
    }
  }
  cffyn_nest* ns = new (std::nothrow) cffyn_nest();
  if (!ns) {
    set_error("host allocation failed");
    return CFFYN_ENOMEM;
  }
  ns->n = n;
  ns->device = dev;
  ns->sh.assign(shells, shells + n);
  ns->dt_default = shells[0]->dt_default;
  for (int i = 1; i < n; ++i) ns->dt_default = std::min(ns->dt_default, shells[i]->dt_default);
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&ns->cap, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaMallocHost(&ns->flags_host, (size_t)n * sizeof(int))) != cudaSuccess) {
    cudaGetLastError();
    set_error("nest creation: %s", cudaGetErrorString(e));
    free_nest(ns);
    return e == cudaErrorMemoryAllocation ? CFFYN_ENOMEM : CFFYN_ECUDA;
  }
  *out = ns;
  return CFFYN_OK;
}

double cffyn_nest_default_dt(const cffyn_nest* ns) { return ns ? ns->dt_default : 0.0; }

int cffyn_nest_rhs(cffyn_nest* ns, const double* const* u, double* const* dudt, void* stream) {
  if (!ns) {
    set_error("nest is NULL");
    return CFFYN_EINVAL;
  }
  int rc;
  if ((rc = check_states(ns, u, "u")) || (rc = check_states(ns, dudt, "dudt"))) return rc;
  for (int i = 0; i < ns->n; ++i)
    if ((rc = check_step_ready(ns->sh[i]))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  for (int i = 0; i < ns->n; ++i)
    if ((rc = enqueue_rhs(ns->sh[i], u[i], dudt[i], st))) return rc;
  for (int i = 0; i + 1 < ns->n; ++i)
    if ((rc = couple(ns->sh[i], ns->sh[i + 1], u[i], dudt[i], dudt[i + 1], false, false, st))) return rc;
  return CFFYN_OK;
}

int cffyn_nest_rk4_step(cffyn_nest* ns, double* const* u, double dt, int n_steps, void* stream) {
  if (!ns) {
    set_error("nest is NULL");
    return CFFYN_EINVAL;
  }
  if (n_steps < 0) {
    set_error("n_steps < 0");
    return CFFYN_EINVAL;
  }
  int rc;
  if ((rc = check_states(ns, u, "u"))) return rc;
  for (int i = 0; i < ns->n; ++i)
    if ((rc = check_step_ready(ns->sh[i]))) {
      char msg[512];
      snprintf(msg, sizeof(msg), "%s", cffyn_last_error());
      set_error("shell %d: %s", i, msg);
      return rc;
    }
  if (n_steps == 0) return CFFYN_OK;
  if (!(dt > 0)) dt = ns->dt_default;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<unsigned> gens(ns->n);
  for (int i = 0; i < ns->n; ++i) gens[i] = ns->sh[i]->ws_gen;
  const bool same = ns->graph && std::equal(ns->gu.begin(), ns->gu.end(), u) && ns->gdt == dt && ns->ggen == gens;
  if (!same) {
    if (ns->graph) {
      cudaGraphExecDestroy(ns->graph);
      ns->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    CF_CUDA(cudaStreamBeginCapture(ns->cap, cudaStreamCaptureModeThreadLocal));
    const int erc = enqueue_nest_step(ns, u, dt, ns->cap);
    const cudaError_t ce = cudaStreamEndCapture(ns->cap, &g);
    if (erc || ce != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      if (erc) return erc;
      set_error("nest graph capture failed: %s", cudaGetErrorString(ce));
      return CFFYN_ECUDA;
    }
    const cudaError_t ie = cudaGraphInstantiate(&ns->graph, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
      ns->graph = nullptr;
      cudaGetLastError();
      set_error("nest graph instantiation failed: %s", cudaGetErrorString(ie));
      return CFFYN_ECUDA;
    }
    ns->gu.assign(u, u + ns->n);
    ns->gdt = dt;
    ns->ggen = gens;
  }
  for (int i = 0; i < ns->n; ++i)
    if ((rc = enqueue_step_prologue(ns->sh[i], u[i], st))) return rc;
  for (int k = 0; k < n_steps; ++k) CF_CUDA(cudaGraphLaunch(ns->graph, st));
  for (int i = 0; i < ns->n; ++i)
    CF_CUDA(cudaMemcpyAsync(ns->flags_host + i, ns->sh[i]->flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  CF_CUDA(cudaStreamSynchronize(st));
  for (int i = 0; i < ns->n; ++i)
    if (ns->flags_host[i]) {
      rc = step_flag_status(ns->flags_host[i]);
      char msg[512];
      snprintf(msg, sizeof(msg), "%s", cffyn_last_error());
      set_error("shell %d: %s", i, msg);
      return rc;
    }
  return CFFYN_OK;
}

int cffyn_destroy_nest(cffyn_nest* ns) {
  free_nest(ns);
  return CFFYN_OK;
}

}  // extern "C"
