// Batched independent shells (the uneven-shell batch): one CUDA graph holds
// one RK4 step (Sec. 2.5) of every shell of the batch as an independent
// branch, forked from and joined into one origin stream during capture, so
// that a batch step is a single graph launch and the kernels of small shells
// run side by side.  Two further graphs run once per call: the step prologue
// of every shell (flag reset, pair copy of the initial state) and the
// read-back of every shell's flag into one pinned array.
#include <algorithm>
#include <cstdio>
#include <new>
#include <vector>

#include "common.cuh"

namespace cffyn {
int enqueue_step_branch(cffyn_shell*, double*, double, cudaStream_t);
int enqueue_step_prologue(cffyn_shell*, double*, cudaStream_t);
int step_flag_status(int);
int check_step_ready(const cffyn_shell*);
int check_state_ptr(const void*, const char*);
}  // namespace cffyn

using namespace cffyn;

struct cffyn_batch {
  int n = 0;
  int device = 0;
  std::vector<cffyn_shell*> sh;
  std::vector<cudaStream_t> br;  // capture stream of each branch
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  cudaStream_t origin = nullptr;
  cudaGraphExec_t pre = nullptr, step = nullptr, post = nullptr;
  std::vector<double*> gu;  // state pointers, step sizes and workspace generations
  std::vector<double> gdt;  // the graphs were captured with
  std::vector<unsigned> ggen;
  int* flags_host = nullptr;  // pinned, one word per shell
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

void free_batch(cffyn_batch* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  free_graphs(b);
  for (cudaStream_t s : b->br)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->join)
    if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->origin) cudaStreamDestroy(b->origin);
  if (b->flags_host) cudaFreeHost(b->flags_host);
  delete b;
}

// Captures per_shell(i, stream) for every shell as parallel branches of one
// graph and instantiates it into *out.
template <class F>
int capture_branches(cffyn_batch* b, cudaGraphExec_t* out, F&& per_shell) {
  CF_CUDA(cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal));
  int rc = CFFYN_OK;
  cudaError_t e = cudaEventRecord(b->fork, b->origin);
  for (int i = 0; i < b->n && e == cudaSuccess && rc == CFFYN_OK; ++i) {
    e = cudaStreamWaitEvent(b->br[i], b->fork, 0);
    if (e != cudaSuccess) break;
    rc = per_shell(i, b->br[i]);
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
  b->br.assign(n, nullptr);
  b->join.assign(n, nullptr);
  auto fail = [&](const char* what, cudaError_t e) {
    cudaGetLastError();
    set_error("batch creation: %s: %s", what, cudaGetErrorString(e));
    free_batch(b);
    return e == cudaErrorMemoryAllocation ? CFFYN_ENOMEM : CFFYN_ECUDA;
  };
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking)) != cudaSuccess) return fail("stream", e);
  if ((e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming)) != cudaSuccess) return fail("event", e);
  for (int i = 0; i < n; ++i) {
    if ((e = cudaStreamCreateWithFlags(&b->br[i], cudaStreamNonBlocking)) != cudaSuccess) return fail("stream", e);
    if ((e = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming)) != cudaSuccess) return fail("event", e);
  }
  if ((e = cudaMallocHost(&b->flags_host, (size_t)n * sizeof(int))) != cudaSuccess) return fail("pinned flags", e);
  *out = b;
  return CFFYN_OK;
}

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
  if (n_steps == 0) return CFFYN_OK;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<unsigned> gens(b->n);
  for (int i = 0; i < b->n; ++i) gens[i] = b->sh[i]->ws_gen;
  const bool same = b->step && std::equal(b->gu.begin(), b->gu.end(), u) && b->gdt == dts && b->ggen == gens;
  if (!same) {
    free_graphs(b);
    if ((rc = capture_branches(b, &b->pre, [&](int i, cudaStream_t s) {
           return enqueue_step_prologue(b->sh[i], u[i], s);
         })))
      return rc;
    if ((rc = capture_branches(b, &b->step, [&](int i, cudaStream_t s) {
           return enqueue_step_branch(b->sh[i], u[i], dts[i], s);
         }))) {
      free_graphs(b);
      return rc;
    }
    if ((rc = capture_branches(b, &b->post, [&](int i, cudaStream_t s) {
           CF_CUDA(cudaMemcpyAsync(b->flags_host + i, b->sh[i]->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
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
  for (int i = 0; i < b->n; ++i)
    if (b->flags_host[i]) {
      rc = step_flag_status(b->flags_host[i]);
      char msg[512];
      snprintf(msg, sizeof(msg), "%s", cffyn_last_error());
      set_error("shell %d: %s", i, msg);
      return rc;
    }
  return CFFYN_OK;
}

int cffyn_destroy_batch(cffyn_batch* b) {
  free_batch(b);
  return CFFYN_OK;
}

}  // extern "C"
