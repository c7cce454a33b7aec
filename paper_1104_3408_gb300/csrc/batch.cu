// Batched independent shells (the uneven-shell batch).  Shells of one shape
// (grid, radii, L, field count, precision, filter and Courant factor) have
// identical operators; the batch stacks each such class into one internal
// handle whose fields are [mu][s][P] (s: the class's shells), so that every
// kernel of a step runs once per class over all its shells: the operators
// see nv * ns fields of P points, the pointwise kernels nv fields of ns * P
// points.  A class of one shell is stepped as itself.  One CUDA graph holds
// one RK4 step (Sec. 2.5) of every class as an independent branch (forked
// from and joined into one origin stream during capture), so that a batch
// step is a single graph launch and the classes run side by side.  Two more
// graphs run once per call: the gathers of the shells' states and gauges
// into their classes with the step prologue (flag reset, pair copy of the
// initial state), and the scatters back with the read-back of every class's
// flag into one pinned array.  The arithmetic of every point and every
// operator column is that of a lone step: batch results are bit-identical
// to stepping the shells one by one.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"

namespace cffyn {
int enqueue_step_branch(cffyn_shell*, double*, double, cudaStream_t);
int enqueue_step_prologue(cffyn_shell*, double*, cudaStream_t);
int step_flag_status(int);
int check_step_ready(const cffyn_shell*);
int check_state_ptr(const void*, const char*);
int create_stacked_shell(const cffyn_shell_desc*, int, cffyn_shell**);
}  // namespace cffyn

using namespace cffyn;

namespace {

// One branch of the batch graph: a shell of the caller (stack == nullptr) or a
// stack of same-shape shells with its own FP64 state U = [mu][s][P].
struct Unit {
  std::vector<int> members;   // batch positions, in order
  cffyn_shell* stack = nullptr;
  double* U = nullptr;
  cffyn_shell* handle(const std::vector<cffyn_shell*>& sh) const { return stack ? stack : sh[members[0]]; }
};

bool same_shape(const cffyn_shell* a, const cffyn_shell* b) {
  const cffyn_shell_desc &x = a->d, &y = b->d;
  return x.n_r == y.n_r && x.n_theta == y.n_theta && x.n_phi == y.n_phi && x.r_in == y.r_in &&
         x.r_out == y.r_out && x.L == y.L && x.n_fields == y.n_fields && x.precision == y.precision &&
         x.filter_mode == y.filter_mode && x.filter_kind == y.filter_kind && x.courant == y.courant &&
         a->tc_wait_ns == b->tc_wait_ns && std::equal(a->op_rows, a->op_rows + kOpFamilies, b->op_rows);
}

}  // namespace

struct cffyn_batch {
  int n = 0;
  int device = 0;
  int stacking = 1;
  std::vector<cffyn_shell*> sh;
  std::vector<Unit> units;
  std::vector<cudaStream_t> br;  // capture stream of each unit
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  cudaStream_t origin = nullptr;
  cudaGraphExec_t pre = nullptr, step = nullptr, post = nullptr;
  std::vector<double*> gu;  // state pointers, step sizes and generations
  std::vector<double> gdt;  // the graphs were captured with
  std::vector<unsigned> ggen;
  int* flags_host = nullptr;  // pinned, one word per unit
};

namespace {

void free_graphs(cffyn_batch* b) {
  cudaGraphExec_t* gs[] = {&b->pre, &b->step, &b->post};
  for (cudaGraphExec_t* g : gs)
    if (*g) {
      cudaGraphExecDestroy(*g);
      *g = nullptr;
    }
}

void free_units(cffyn_batch* b) {
  for (Unit& u : b->units) {
    if (u.U) cudaFree(u.U);
    if (u.stack) cffyn_destroy(u.stack);
    u.U = nullptr;
    u.stack = nullptr;
  }
}

void free_batch(cffyn_batch* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  free_graphs(b);
  free_units(b);
  for (cudaStream_t s : b->br)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->join)
    if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->origin) cudaStreamDestroy(b->origin);
  if (b->flags_host) cudaFreeHost(b->flags_host);
  delete b;
}

// Captures per_unit(i, stream) for every unit as parallel branches of one
// graph and instantiates it into *out.
template <class F>
int capture_branches(cffyn_batch* b, cudaGraphExec_t* out, F&& per_unit) {
  CF_CUDA(cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal));
  int rc = CFFYN_OK;
  cudaError_t e = cudaEventRecord(b->fork, b->origin);
  const int nu = (int)b->units.size();
  for (int i = 0; i < nu && e == cudaSuccess && rc == CFFYN_OK; ++i) {
    e = cudaStreamWaitEvent(b->br[i], b->fork, 0);
    if (e != cudaSuccess) break;
    rc = per_unit(i, b->br[i]);
    if (rc) break;
    e = cudaEventRecord(b->join[i], b->br[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->origin, b->join[i], 0);
  }
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(b->origin, &g);
  if (rc != CFFYN_OK || e != cudaSuccess || ce != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    if (rc) return rc;
    set_error("batch graph capture failed: %s", cudaGetErrorString(e != cudaSuccess ? e : ce));
    return CFFYN_ECUDA;
  }
  const cudaError_t ie = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) {
    *out = nullptr;
    cudaGetLastError();
    set_error("batch graph instantiation failed: %s", cudaGetErrorString(ie));
    return CFFYN_ECUDA;
  }
  return CFFYN_OK;
}

// Groups the shells into units (classes of one shape, in order of first
// appearance), making a stacked handle and state for every class of two or
// more shells when stacking is on.
int make_units(cffyn_batch* b) {
  std::vector<int> cls(b->n, -1);
  std::vector<std::vector<int>> groups;
  for (int i = 0; i < b->n; ++i) {
    for (size_t g = 0; g < groups.size() && cls[i] < 0; ++g)
      if (b->stacking && same_shape(b->sh[groups[g][0]], b->sh[i])) {
        groups[g].push_back(i);
        cls[i] = (int)g;
      }
    if (cls[i] < 0) {
      cls[i] = (int)groups.size();
      groups.push_back({i});
    }
  }
  for (auto& g : groups) {
    Unit u;
    u.members = g;
    if (g.size() > 1) {
      const cffyn_shell* f = b->sh[g[0]];
      cffyn_shell_desc d = f->d;
      d.flags = 0;
      int rc = create_stacked_shell(&d, (int)g.size(), &u.stack);
      if (rc) {
        b->units.push_back(u);
        return rc;
      }
      u.stack->tc_wait_ns = f->tc_wait_ns;
      for (int w = 0; w < kOpFamilies; ++w)
        if (u.stack->op_rows[w] != f->op_rows[w] && (rc = cffyn_set_operator_rows(u.stack, w, f->op_rows[w]))) {
          b->units.push_back(u);
          return rc;
        }
      u.stack->gauge_set = true;  // gathered from the members before every call
      if (cudaMalloc(&u.U, (size_t)d.n_fields * P_all(u.stack) * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        b->units.push_back(u);
        set_error("device allocation of a stacked state failed");
        return CFFYN_ENOMEM;
      }
    }
    b->units.push_back(u);
  }
  return CFFYN_OK;
}

// Copies rows arrays of P values between a member's [rows][P] array and its
// slot s in a stack's [rows][ns][P] array (to_stack: member -> stack).
int stack_copy(double* stack, double* member, size_t P, int ns, int s, int rows, bool to_stack,
               cudaStream_t st) {
  const size_t w = P * sizeof(double), sp = (size_t)ns * w;
  double* sdst = stack + (size_t)s * P;
  if (to_stack)
    CF_CUDA(cudaMemcpy2DAsync(sdst, sp, member, w, w, rows, cudaMemcpyDeviceToDevice, st));
  else
    CF_CUDA(cudaMemcpy2DAsync(member, w, sdst, sp, w, rows, cudaMemcpyDeviceToDevice, st));
  return CFFYN_OK;
}

}  // namespace

extern "C" {

int cffyn_create_batch(int n, cffyn_shell* const* shells, cffyn_batch** out) {
  if (!out) {
    set_error("out is NULL");
    return CFFYN_EINVAL;
  }
  *out = nullptr;
  if (n < 1 || !shells) {
    set_error("a batch needs n >= 1 shells (n = %d)", n);
    return CFFYN_EINVAL;
  }
  int dev = 0;
  CF_CUDA(cudaGetDevice(&dev));
  std::vector<cffyn_shell*> v(shells, shells + n);
  for (int i = 0; i < n; ++i) {
    if (!v[i]) {
      set_error("shell %d is NULL", i);
      return CFFYN_EINVAL;
    }
    if (v[i]->device != dev) {
      set_error("shell %d lives on device %d, the current device is %d", i, v[i]->device, dev);
      return CFFYN_EINVAL;
    }
  }
  {
    std::vector<cffyn_shell*> s = v;
    std::sort(s.begin(), s.end());
    if (std::adjacent_find(s.begin(), s.end()) != s.end()) {
      set_error("a shell appears twice in the batch");
      return CFFYN_EINVAL;
    }
  }
  cffyn_batch* b = new (std::nothrow) cffyn_batch();
  if (!b) {
    set_error("host allocation failed");
    return CFFYN_ENOMEM;
  }
  b->n = n;
  b->device = dev;
  b->sh = v;
  int rc;
  if ((rc = make_units(b))) {
    free_batch(b);
    return rc;
  }
  const int nu = (int)b->units.size();
  b->br.assign(nu, nullptr);
  b->join.assign(nu, nullptr);
  auto fail = [&](const char* what, cudaError_t e) {
    cudaGetLastError();
    set_error("batch creation: %s: %s", what, cudaGetErrorString(e));
    free_batch(b);
    return e == cudaErrorMemoryAllocation ? CFFYN_ENOMEM : CFFYN_ECUDA;
  };
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking)) != cudaSuccess) return fail("stream", e);
  if ((e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming)) != cudaSuccess) return fail("event", e);
  for (int i = 0; i < nu; ++i) {
    if ((e = cudaStreamCreateWithFlags(&b->br[i], cudaStreamNonBlocking)) != cudaSuccess) return fail("stream", e);
    if ((e = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming)) != cudaSuccess) return fail("event", e);
  }
  if ((e = cudaMallocHost(&b->flags_host, (size_t)nu * sizeof(int))) != cudaSuccess) return fail("pinned flags", e);
  *out = b;
  return CFFYN_OK;
}

int cffyn_batch_units(const cffyn_batch* b) { return b ? (int)b->units.size() : 0; }

int cffyn_batch_rk4_step(cffyn_batch* b, double* const* u, const double* dt, int n_steps, void* stream) {
  if (!b) {
    set_error("batch is NULL");
    return CFFYN_EINVAL;
  }
  if (!u) {
    set_error("u is NULL");
    return CFFYN_EINVAL;
  }
  if (n_steps < 0) {
    set_error("n_steps < 0");
    return CFFYN_EINVAL;
  }
  int rc;
  std::vector<double> dts(b->n);
  for (int i = 0; i < b->n; ++i) {
    if ((rc = check_state_ptr(u[i], "u[i]"))) return rc;
    if ((rc = check_step_ready(b->sh[i]))) {
      char msg[512];
      snprintf(msg, sizeof(msg), "%s", cffyn_last_error());
      set_error("shell %d: %s", i, msg);
      return rc;
    }
    dts[i] = (dt && dt[i] > 0) ? dt[i] : b->sh[i]->dt_default;
  }
  // a stack advances its shells with one dt
  for (const Unit& un : b->units)
    for (int m : un.members)
      if (dts[m] != dts[un.members[0]]) {
        set_error("shells %d and %d have the same shape but step sizes %.17g and %.17g", un.members[0], m,
                  dts[un.members[0]], dts[m]);
        return CFFYN_EINVAL;
      }
  if (n_steps == 0) return CFFYN_OK;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<unsigned> gens(b->n);
  for (int i = 0; i < b->n; ++i) gens[i] = b->sh[i]->ws_gen;
  const bool same = b->step && std::equal(b->gu.begin(), b->gu.end(), u) && b->gdt == dts && b->ggen == gens;
  if (!same) {
    free_graphs(b);
    // the stacks' kernels take the members' wait bound
    for (Unit& un : b->units)
      if (un.stack && un.stack->tc_wait_ns != b->sh[un.members[0]]->tc_wait_ns) {
        un.stack->tc_wait_ns = b->sh[un.members[0]]->tc_wait_ns;
        ++un.stack->ws_gen;
      }
    if ((rc = capture_branches(b, &b->pre, [&](int i, cudaStream_t s) {
           const Unit& un = b->units[i];
           if (!un.stack) return enqueue_step_prologue(b->sh[un.members[0]], u[un.members[0]], s);
           cffyn_shell* k = un.stack;
           const int ns = k->ns;
           for (int q = 0; q < ns; ++q) {
             cffyn_shell* m = b->sh[un.members[q]];
             int r;
             if ((r = stack_copy(un.U, u[un.members[q]], k->P, ns, q, k->nv, true, s))) return r;
             if (k->nv == 50) {
               if ((r = stack_copy(k->H, m->H, k->P, ns, q, 4, true, s))) return r;
               if ((r = stack_copy(k->dH, m->dH, k->P, ns, q, 12, true, s))) return r;
             }
           }
           return enqueue_step_prologue(k, un.U, s);
         })))
      return rc;
    if ((rc = capture_branches(b, &b->step, [&](int i, cudaStream_t s) {
           const Unit& un = b->units[i];
           const int m0 = un.members[0];
           return enqueue_step_branch(un.handle(b->sh), un.stack ? un.U : u[m0], dts[m0], s);
         }))) {
      free_graphs(b);
      return rc;
    }
    if ((rc = capture_branches(b, &b->post, [&](int i, cudaStream_t s) {
           const Unit& un = b->units[i];
           cffyn_shell* k = un.handle(b->sh);
           if (un.stack)
             for (int q = 0; q < k->ns; ++q) {
               int r;
               if ((r = stack_copy(un.U, u[un.members[q]], k->P, k->ns, q, k->nv, false, s))) return r;
             }
           CF_CUDA(cudaMemcpyAsync(b->flags_host + i, k->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
           return CFFYN_OK;
         }))) {
      free_graphs(b);
      return rc;
    }
    b->gu.assign(u, u + b->n);
    b->gdt = dts;
    b->ggen = gens;
  }
  CF_CUDA(cudaGraphLaunch(b->pre, st));
  for (int k = 0; k < n_steps; ++k) CF_CUDA(cudaGraphLaunch(b->step, st));
  CF_CUDA(cudaGraphLaunch(b->post, st));
  CF_CUDA(cudaStreamSynchronize(st));
  for (size_t i = 0; i < b->units.size(); ++i)
    if (b->flags_host[i]) {
      rc = step_flag_status(b->flags_host[i]);
      char msg[512];
      snprintf(msg, sizeof(msg), "%s", cffyn_last_error());
      set_error("shell %d: %s", b->units[i].members[0], msg);
      return rc;
    }
  return CFFYN_OK;
}

int cffyn_destroy_batch(cffyn_batch* b) {
  free_batch(b);
  return CFFYN_OK;
}

}  // extern "C"
