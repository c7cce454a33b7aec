// Spectral derivatives by fast Fourier transforms: the alternative to the
// matrix method that Sec. 5 weighs against it (Fig. mmfft), here for the
// three derivatives of Secs. 2.3-2.4 on the shell's grid, in FP64 with cuFFT.
// The results equal those of the differentiation matrices (eqs. D1-D3) up to
// rounding:
//
//   r      Chebyshev extrema x_k = -cos(pi k / (n_r - 1)) (eq. rk).  The
//          samples, read as values at xi_k = cos(pi k / (n_r - 1)) = -x_k,
//          are extended evenly to 2 (n_r - 1) points; a real FFT gives the
//          Chebyshev coefficients a_m (the DCT-I), the derivative's
//          coefficients follow from c_k b_k = b_{k+2} + 2 (k + 1) a_{k+1}
//          (b_{n_r-1} = b_{n_r} = 0, c_0 = 2, else 1), an inverse FFT of the
//          even extension of b evaluates d/dxi at the extrema, and
//          d/dr = -(2 / (r_out - r_in)) d/dxi.
//   theta  the double cover of Sec. 2.1: for phi_j, j < n_phi / 2, the line
//          of 2 n_theta values u(theta_0..theta_{N-1}, phi_j) followed by
//          u(theta_{N-1}..theta_0, phi_j + pi) is 2 pi periodic in the
//          extended angle; its FFT derivative (mode l times i l, the Nyquist
//          mode to zero as in eq. FD for an even number of points) gives
//          d_theta at phi_j in its first half and minus d_theta at
//          phi_j + pi, in reverse order, in its second half (the extended
//          angle runs against theta there).
//   phi    per (theta, r) line of n_phi values: mode m times i m, Nyquist to
//          zero (eq. D3 with eq. FD).
//
// The chain rule (eq. dvdx) is the FP64 Cartesian kernel of the matrix path.
// Data movement around the transforms is done by the kernels below: the even
// extension in r, a shared-memory gather / scatter of the double-cover lines
// in theta, and tiled transposes that make phi the contiguous index.
#include <cufft.h>

#include <algorithm>
#include <new>

#include "common.cuh"

namespace cffyn {
// pointwise.cu
int pw_cart_fp64(const cffyn_shell*, const double*, double*, int, cudaStream_t);

// Plans (forward real-to-complex and inverse complex-to-real per direction)
// and the two scratch arrays, made by the first cffyn_derivs_fft call.
struct FftPath {
  cufftHandle plan[6] = {0, 0, 0, 0, 0, 0};  // r fwd, r inv, theta fwd, theta inv, phi fwd, phi inv
  bool made[6] = {false, false, false, false, false, false};
  double* re = nullptr;   // real lines (extended in r and theta, transposed in phi)
  double2* cx = nullptr;  // their half spectra
  size_t re_n = 0, cx_n = 0;
};

void fft_release(cffyn_shell* sh) {
  if (!sh || !sh->fft) return;
  FftPath* f = sh->fft;
  for (int q = 0; q < 6; ++q)
    if (f->made[q]) cufftDestroy(f->plan[q]);
  if (f->re) cudaFree(f->re);
  if (f->cx) cudaFree(f->cx);
  delete f;
  sh->fft = nullptr;
}

}  // namespace cffyn

using namespace cffyn;

namespace {

constexpr int kTile = 32;
constexpr size_t kThetaSmem = 2 * sizeof(double) * kMaxN * kMaxNr;

// r: even extension of every column of n values (k contiguous) to M = 2 (n - 1)
__global__ void k_fft_r_extend(const double* __restrict__ u, double* __restrict__ ext, long long ncol, int n) {
  const int M = 2 * (n - 1);
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= ncol * M) return;
  const long long col = t / M;
  const int p = (int)(t - col * M);
  ext[t] = u[col * n + (p < n ? p : M - p)];
}

// r: half spectra V_m (m < n, real for even input) of 32 columns per block ->
// Chebyshev coefficients a_m, derivative coefficients b_k by the downward
// recurrence, and the half spectrum of b's even extension (W_0 = b_0,
// W_m = b_m / 2, W_{n-1} = b_{n-1} = 0) times `scale` (= -2 / (r_out - r_in)).
// a_{k+1} is read just before slot k + 1 is overwritten with W_{k+1}.
__global__ void __launch_bounds__(kTile) k_fft_r_spec(double2* __restrict__ X, long long ncol, int n, double scale) {
  __shared__ double s[kTile][kMaxNr + 1];
  const long long col0 = (long long)blockIdx.x * kTile;
  const int nc = (int)min((long long)kTile, ncol - col0);
  for (int idx = threadIdx.x; idx < nc * n; idx += blockDim.x) {
    const int c = idx / n;
    s[c][idx - c * n] = X[col0 * n + idx].x;
  }
  __syncthreads();
  if (threadIdx.x < nc) {
    double* a = s[threadIdx.x];
    const double inv = 1.0 / (double)(n - 1);
    double b2 = 0.0, b1 = 0.0;  // b_{k+2}, b_{k+1}
    for (int k = n - 2; k >= 0; --k) {
      const double am = a[k + 1] * (k + 1 == n - 1 ? 0.5 * inv : inv);
      double bk = b2 + 2.0 * (double)(k + 1) * am;
      if (k == 0) bk *= 0.5;
      a[k + 1] = (k + 1 <= n - 2) ? 0.5 * b1 * scale : 0.0;
      b2 = b1;
      b1 = bk;
    }
    a[0] = b1 * scale;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < nc * n; idx += blockDim.x) {
    const int c = idx / n;
    X[col0 * n + idx] = make_double2(s[c][idx - c * n], 0.0);
  }
}

// r: first n values of every extended column -> D (same layout as u)
__global__ void k_fft_r_out(const double* __restrict__ ext, double* __restrict__ D, long long ncol, int n) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= ncol * n) return;
  const long long col = t / n;
  D[t] = ext[col * 2 * (n - 1) + (t - col * n)];
}

// theta: one block per (field, j < J/2): slabs j and j + J/2 (N x n_r each)
// through shared memory into n_r lines of 2N values:
// line[p] = u[j][p][k] for p < N, u[j + J/2][2N - 1 - p][k] for p >= N.
__global__ void k_fft_t_gather(const double* __restrict__ u, double* __restrict__ ext, int n_r, int N, int J) {
  extern __shared__ double sm[];
  const int half = J / 2;
  const int mu = blockIdx.x / half, j = blockIdx.x - mu * half;
  const int slab = N * n_r;
  const double* a = u + ((long long)mu * J + j) * slab;
  const double* b = u + ((long long)mu * J + j + half) * slab;
  for (int idx = threadIdx.x; idx < slab; idx += blockDim.x) {
    sm[idx] = a[idx];
    sm[slab + idx] = b[idx];
  }
  __syncthreads();
  const int L = 2 * N;
  double* out = ext + (long long)blockIdx.x * n_r * L;
  for (int idx = threadIdx.x; idx < n_r * L; idx += blockDim.x) {
    const int k = idx / L, p = idx - k * L;
    out[idx] = p < N ? sm[p * n_r + k] : sm[slab + (L - 1 - p) * n_r + k];
  }
}

// theta: the inverse of the gather for the derivative lines d:
// D[j][i][k] = d[k][i], D[j + J/2][i][k] = -d[k][2N - 1 - i].
__global__ void k_fft_t_scatter(const double* __restrict__ ext, double* __restrict__ D, int n_r, int N, int J) {
  extern __shared__ double sm[];
  const int half = J / 2;
  const int mu = blockIdx.x / half, j = blockIdx.x - mu * half;
  const int L = 2 * N;
  const double* in = ext + (long long)blockIdx.x * n_r * L;
  for (int idx = threadIdx.x; idx < n_r * L; idx += blockDim.x) sm[idx] = in[idx];
  __syncthreads();
  const int slab = N * n_r;
  double* a = D + ((long long)mu * J + j) * slab;
  double* b = D + ((long long)mu * J + j + half) * slab;
  for (int idx = threadIdx.x; idx < slab; idx += blockDim.x) {
    const int i = idx / n_r, k = idx - i * n_r;
    a[idx] = sm[k * L + i];
    b[idx] = -sm[k * L + (L - 1 - i)];
  }
}

// theta, phi: half spectrum of every line (H + 1 modes, H = Nyquist) times
// i l s; the Nyquist mode to zero
__global__ void k_fft_mul_ik(double2* __restrict__ X, long long nlines, int H, double s) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= nlines * (H + 1)) return;
  const int l = (int)(t % (H + 1));
  const double f = l == H ? 0.0 : (double)l * s;
  const double2 v = X[t];
  X[t] = make_double2(-v.y * f, v.x * f);
}

// phi: per batch b, in[b][rows][cols] -> out[b][cols][rows] through 32 x 32
// shared-memory tiles (both sides coalesced); block (32, 8)
__global__ void k_fft_transpose(const double* __restrict__ in, double* __restrict__ out, int rows, int cols) {
  __shared__ double tile[kTile][kTile + 1];
  const long long off = (long long)blockIdx.z * rows * cols;
  const int c0 = blockIdx.x * kTile, r0 = blockIdx.y * kTile;
  for (int y = threadIdx.y; y < kTile; y += blockDim.y) {
    const int r = r0 + y, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[y][threadIdx.x] = in[off + (long long)r * cols + c];
  }
  __syncthreads();
  for (int y = threadIdx.y; y < kTile; y += blockDim.y) {
    const int c = c0 + y, r = r0 + threadIdx.x;
    if (r < rows && c < cols) out[off + (long long)c * rows + r] = tile[threadIdx.x][y];
  }
}

unsigned blocks(long long n, int t) { return (unsigned)((n + t - 1) / t); }

int fft_check(cufftResult r, const char* what) {
  if (r == CUFFT_SUCCESS) return CFFYN_OK;
  set_error("cuFFT %s failed (cufftResult %d)", what, (int)r);
  return r == CUFFT_ALLOC_FAILED ? CFFYN_ENOMEM : CFFYN_ECUDA;
}

// Plans and scratch for all n_fields fields of the shell (first call).
int fft_prepare(cffyn_shell* sh) {
  if (sh->fft) return CFFYN_OK;
  FftPath* f = new (std::nothrow) FftPath();
  if (!f) {
    set_error("host allocation failed");
    return CFFYN_ENOMEM;
  }
  sh->fft = f;
  const long long nv = sh->nv, n_r = sh->n_r, N = sh->N, J = sh->J;
  const long long lines[3] = {nv * J * N, nv * (J / 2) * n_r, nv * N * n_r};
  const int len[3] = {(int)(2 * (n_r - 1)), (int)(2 * N), (int)J};
  size_t re_n = 0, cx_n = 0;
  for (int d = 0; d < 3; ++d) {
    re_n = std::max(re_n, (size_t)(lines[d] * len[d]));
    cx_n = std::max(cx_n, (size_t)(lines[d] * (len[d] / 2 + 1)));
  }
  int rc;
  for (int d = 0; d < 3; ++d) {
    int n = len[d];
    if ((rc = fft_check(cufftPlanMany(&f->plan[2 * d], 1, &n, nullptr, 1, n, nullptr, 1, n / 2 + 1, CUFFT_D2Z,
                                      (int)lines[d]),
                        "plan (D2Z)"))) {
      fft_release(sh);
      return rc;
    }
    f->made[2 * d] = true;
    if ((rc = fft_check(cufftPlanMany(&f->plan[2 * d + 1], 1, &n, nullptr, 1, n / 2 + 1, nullptr, 1, n, CUFFT_Z2D,
                                      (int)lines[d]),
                        "plan (Z2D)"))) {
      fft_release(sh);
      return rc;
    }
    f->made[2 * d + 1] = true;
  }
  if (cudaMalloc(&f->re, re_n * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&f->cx, cx_n * sizeof(double2)) != cudaSuccess) {
    cudaGetLastError();
    set_error("device allocation of %zu bytes (FFT scratch) failed", re_n * sizeof(double) + cx_n * sizeof(double2));
    fft_release(sh);
    return CFFYN_ENOMEM;
  }
  f->re_n = re_n;
  f->cx_n = cx_n;
  const size_t smem = (size_t)2 * sizeof(double) * N * n_r;
  if (smem > 48 * 1024) {
    CF_CUDA(cudaFuncSetAttribute(k_fft_t_gather, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kThetaSmem));
    CF_CUDA(cudaFuncSetAttribute(k_fft_t_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kThetaSmem));
  }
  return CFFYN_OK;
}

}  // namespace

extern "C" int cffyn_derivs_fft(cffyn_shell* sh, const double* u, double* dxyz, void* stream) {
  if (!sh) {
    set_error("shell is NULL");
    return CFFYN_EINVAL;
  }
  if (!u || !dxyz || (((uintptr_t)u | (uintptr_t)dxyz) & 15)) {
    set_error("u and dxyz must be non-NULL and 16-byte aligned");
    return CFFYN_EINVAL;
  }
  if (!sh->ws) {
    set_error("no workspace attached (cffyn_attach_workspace)");
    return CFFYN_EINVAL;
  }
  int dev = -1;
  CF_CUDA(cudaGetDevice(&dev));
  if (dev != sh->device) {
    set_error("the shell lives on device %d but device %d is current", sh->device, dev);
    return CFFYN_EINVAL;
  }
  int rc;
  if ((rc = fft_prepare(sh))) return rc;
  FftPath* f = sh->fft;
  cudaStream_t st = (cudaStream_t)stream;
  for (int q = 0; q < 6; ++q)
    if ((rc = fft_check(cufftSetStream(f->plan[q], st), "set stream"))) return rc;
  const int nv = sh->nv, n_r = sh->n_r, N = sh->N, J = sh->J;
  const long long P = (long long)sh->P;
  double* D = sh->D;  // spherical derivatives [3][nv][P], FP64 in this call
  double* re = f->re;
  double2* cx = f->cx;

  // r
  const long long ncol = (long long)nv * J * N;
  const int M = 2 * (n_r - 1);
  k_fft_r_extend<<<blocks(ncol * M, 256), 256, 0, st>>>(u, re, ncol, n_r);
  count_launch();
  if ((rc = fft_check(cufftExecD2Z(f->plan[0], re, cx), "r forward"))) return rc;
  k_fft_r_spec<<<blocks(ncol, kTile), kTile, 0, st>>>(cx, ncol, n_r, -2.0 / (sh->d.r_out - sh->d.r_in));
  count_launch();
  if ((rc = fft_check(cufftExecZ2D(f->plan[1], cx, re), "r inverse"))) return rc;
  k_fft_r_out<<<blocks(ncol * n_r, 256), 256, 0, st>>>(re, D, ncol, n_r);
  count_launch();
  CF_CUDA(cudaGetLastError());

  // theta over the double cover
  const unsigned tb = (unsigned)(nv * (J / 2));
  const size_t smem = (size_t)2 * sizeof(double) * N * n_r;
  k_fft_t_gather<<<tb, 256, smem, st>>>(u, re, n_r, N, J);
  count_launch();
  if ((rc = fft_check(cufftExecD2Z(f->plan[2], re, cx), "theta forward"))) return rc;
  const long long tl = (long long)tb * n_r;
  k_fft_mul_ik<<<blocks(tl * (N + 1), 256), 256, 0, st>>>(cx, tl, N, 1.0 / (2.0 * N));
  count_launch();
  if ((rc = fft_check(cufftExecZ2D(f->plan[3], cx, re), "theta inverse"))) return rc;
  k_fft_t_scatter<<<tb, 256, smem, st>>>(re, D + (long long)nv * P, n_r, N, J);
  count_launch();
  CF_CUDA(cudaGetLastError());

  // phi: [mu][j][c] -> [mu][c][j], c = (i, k)
  const int C = N * n_r;
  const dim3 tblk(kTile, 8);
  k_fft_transpose<<<dim3(blocks(C, kTile), blocks(J, kTile), nv), tblk, 0, st>>>(u, re, J, C);
  count_launch();
  if ((rc = fft_check(cufftExecD2Z(f->plan[4], re, cx), "phi forward"))) return rc;
  const long long pl = (long long)nv * C;
  k_fft_mul_ik<<<blocks(pl * (J / 2 + 1), 256), 256, 0, st>>>(cx, pl, J / 2, 1.0 / (double)J);
  count_launch();
  if ((rc = fft_check(cufftExecZ2D(f->plan[5], cx, re), "phi inverse"))) return rc;
  k_fft_transpose<<<dim3(blocks(J, kTile), blocks(C, kTile), nv), tblk, 0, st>>>(re, D + 2LL * nv * P, C, J);
  count_launch();
  CF_CUDA(cudaGetLastError());

  return pw_cart_fp64(sh, D, dxyz, nv, st);
}
