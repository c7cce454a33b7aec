// cffyn_derivs_static: a variant of cffyn_derivs (the Cartesian derivatives)
// for the first n_f fields, with every intermediate in one fixed array of the
// library's own device memory instead of the shell's workspace or a new
// allocation.  The paper has no counterpart; this is a library facility for
// callers that cannot allocate at the point of the call (see
// include/cffyn.h).
#include <mutex>

#include "common.cuh"

namespace cffyn {
// ops.cu
int op_derivs_at(const cffyn_shell*, const double*, double*, int, int*, int*, cudaStream_t);
// pointwise.cu
int pw_cart_status(const cffyn_shell*, const double*, double*, int, bool, const int*, cudaStream_t);
}  // namespace cffyn

using namespace cffyn;

namespace {

// One array per device, reserved when the module's device code is loaded
// there.  Layout of one call: spherical derivatives [3][n_f][P] (8 bytes per
// value on both paths), then on the mixed path one 256-byte block of 64
// words, 256-byte aligned: words 0..n_f-1 the per-field exponents (n_f <= 58),
// word 63 the call's own status word (a timed-out wait of the tensor-core
// kernel sets it; the chain-rule kernel then writes NaN).  All 64 words are
// zeroed at the start of every call.
__device__ __align__(256) unsigned char g_static_scratch[CFFYN_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
void* g_addr[kMaxDevices] = {};

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

// Device address of the array on the current device `dev`, looked up once per
// device (cudaGetSymbolAddress, with `dev` current).
int scratch_address(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("cffyn_derivs_static: device %d outside the supported 0..%d", dev, kMaxDevices - 1);
    return CFFYN_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_addr_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
      set_error("cffyn_derivs_static: cudaGetSymbolAddress on device %d: %s", dev,
                cudaGetErrorString(e));
      return CFFYN_ECUDA;
    }
    g_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_addr[dev]);
  return CFFYN_OK;
}

}  // namespace

extern "C" int cffyn_derivs_static(const cffyn_shell* sh, const double* u, int n_f, double* dxyz,
                                   void* stream) {
  if (!sh) {
    set_error("cffyn_derivs_static: shell is NULL");
    return CFFYN_EINVAL;
  }
  if (!u || !dxyz || (((uintptr_t)u | (uintptr_t)dxyz) & 15)) {
    set_error("cffyn_derivs_static: u and dxyz must be non-NULL and 16-byte aligned");
    return CFFYN_EINVAL;
  }
  if (n_f < 1 || n_f > sh->nv) {
    set_error("cffyn_derivs_static: n_f = %d outside [1, %d]", n_f, sh->nv);
    return CFFYN_EINVAL;
  }
  const bool mixed = sh->d.precision == CFFYN_MIXED;
  const size_t vals = (size_t)n_f * sh->P;
  const size_t d_bytes = round256(3 * vals * sizeof(double));
  const size_t need = d_bytes + (mixed ? 256 : 0);
  if (need > (size_t)CFFYN_STATIC_SCRATCH_BYTES) {
    set_error("cffyn_derivs_static: %d fields of %zu points need %zu bytes of static scratch; "
              "the limit is %zu bytes",
              n_f, sh->P, need, (size_t)CFFYN_STATIC_SCRATCH_BYTES);
    return CFFYN_EINVAL;
  }
  int dev = -1;
  CF_CUDA(cudaGetDevice(&dev));
  if (dev != sh->device) {
    set_error("cffyn_derivs_static: the shell lives on device %d but device %d is current",
              sh->device, dev);
    return CFFYN_EINVAL;
  }
  unsigned char* base = nullptr;
  int rc;
  if ((rc = scratch_address(dev, &base))) return rc;
  double* D = reinterpret_cast<double*>(base);
  int* exps = mixed ? reinterpret_cast<int*>(base + d_bytes) : nullptr;
  int* status = mixed ? exps + 63 : nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  if ((rc = op_derivs_at(sh, u, D, n_f, exps, status, st))) return rc;
  return pw_cart_status(sh, D, dxyz, n_f, false, status, st);
}
