// On-device FP64 construction of every operator of a shell (create time, not
// on the timed path):
//   grid                      paper Sec. 2.1, eqs. rk, thetai, phij
//   D_r                       Sec. 2.3, eq. CDhat (diagonal = minus row sum), rescaled
//   theta pair operator       Sec. 2.1 double cover + Sec. 2.3 Fourier matrix
//   D_phi                     Sec. 2.3 Fourier matrix
//   real DFT rows / columns   Sec. 3.1, eqs. Fsynthesis, Fanalysis (sine reading of B)
//   P^n_lm(theta_i)           Sec. 3.3: normalised associated Legendre recursion for
//                             n = 0, eqs. Yninc/Yncoeffs for n = 1..3, eq. Ynnegative
//                             for n < 0
//   F^n_m = P f P^+           eq. FasPfQ; P^+ from a Householder QR (P = QR,
//                             P^+ = R^-1 Q^T; P has full column rank once the zero
//                             columns l < |n| are dropped)
//   split-precision digits    8-bit balanced digits of each operator row in the
//                             mma.m16n8k16 A-fragment order.
#include <cmath>
#include <cstdio>
#include <cstring>

#include "common.cuh"

namespace cffyn {

__global__ void k_grid(double* r, double* sth, double* cth, double* sph, double* cph, int n_r,
                       int N, int J, double r_in, double r_out) {
  const double pi = 3.14159265358979323846;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n_r) r[t] = 0.5 * (r_out + r_in) - 0.5 * (r_out - r_in) * cos(pi * t / (n_r - 1));
  if (t < N) {
    double th = pi * (t + 0.5) / N;
    sth[t] = sin(th);
    cth[t] = cos(th);
  }
  if (t < J) {
    double ph = 2.0 * pi * t / J;
    sph[t] = sin(ph);
    cph[t] = cos(ph);
  }
}

// One thread per row of the Chebyshev matrix.
__global__ void k_cheb(double* D, int n, double scale) {
  const double pi = 3.14159265358979323846;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double xi = -cos(pi * i / (n - 1));
  double ci = (i == 0 || i == n - 1) ? 2.0 : 1.0;
  double sum = 0.0;
  for (int j = 0; j < n; ++j) {
    if (j == i) continue;
    double xj = -cos(pi * j / (n - 1));
    double cj = (j == 0 || j == n - 1) ? 2.0 : 1.0;
    double v = (ci / cj) * (((i + j) & 1) ? -1.0 : 1.0) / (xi - xj);
    D[i * n + j] = scale * v;
    sum += v;
  }
  D[i * n + i] = -scale * sum;
}

__device__ double fourier_entry(int i, int j, int n) {
  const double pi = 3.14159265358979323846;
  if (i == j) return 0.0;
  return (((i + j) & 1) ? -1.0 : 1.0) / (2.0 * tan(pi * (double)(i - j) / n));
}

// D_phi (n x n) and the theta pair operator (2N x 2N):
//   rows p <  N: FD_2N[p][q]
//   rows p >= N: FD_2N[p-N][2N-1-q]
// acting on X = [u(theta_0..theta_{N-1}, phi_j) ; u(theta_{N-1}..theta_0, phi_j + pi)].
__global__ void k_fourier_ops(double* Dph, int J, double* Dth2, int N) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < J * J) Dph[t] = fourier_entry(t / J, t % J, J);
  int M = 2 * N;
  if (t < M * M) {
    int p = t / M, q = t % M;
    Dth2[t] = (p < N) ? fourier_entry(p, q, M) : fourier_entry(p - N, M - 1 - q, M);
  }
}

// Analysis rows (R x J): a_0, a_1..a_L, b_1..b_L; synthesis (J x R).
__global__ void k_dft(double* Fan, double* Fsy, int J, int L) {
  const double pi = 3.14159265358979323846;
  int R = 2 * L + 1;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= R * J) return;
  int row = t / J, j = t % J;
  double an, sy;
  if (row == 0) {
    an = 1.0 / J;
    sy = 1.0;
  } else if (row <= L) {
    double c = cos(2.0 * pi * (double)((long long)j * row % J) / J);
    an = 2.0 / J * c;
    sy = c;
  } else {
    int m = row - L;
    double s = sin(2.0 * pi * (double)((long long)j * m % J) / J);
    an = 2.0 / J * s;
    sy = s;
  }
  Fan[row * J + j] = an;
  Fsy[j * R + row] = sy;
}

// P^n_{l,m}(theta_i) for n in [-3, 3], m in [0, Mmax], l in [0, N-1].
// Output layout Pn[(n+3)][m][i][l].  One thread per (i, m); the recursions run
// through global memory (create time only).
__global__ void k_spin_legendre(double* Pn, double* tmp, int N, int Mmax) {
  const double pi = 3.14159265358979323846;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int nm = Mmax + 1;
  if (t >= N * nm) return;
  int i = t % N, m = t / N;
  double th = pi * (i + 0.5) / N;
  double x = cos(th), s = sin(th);
  // tmp[(sgn)][n][l] scratch for +m (sgn 0) and -m (sgn 1), n = 0..3
  double* W = tmp + (size_t)t * 2 * 4 * N;
  auto w = [&](int sg, int n, int l) -> double& { return W[(sg * 4 + n) * N + l]; };
  for (int sg = 0; sg < 2; ++sg)
    for (int n = 0; n < 4; ++n)
      for (int l = 0; l < N; ++l) w(sg, n, l) = 0.0;
  // n = 0, m >= 0: normalised associated Legendre with Condon-Shortley phase
  if (m <= N - 1) {
    double prod = 1.0;
    for (int k = 1; k <= m; ++k) prod *= (2.0 * k - 1.0) / (2.0 * k);
    double pmm = ((m & 1) ? -1.0 : 1.0) * sqrt((2.0 * m + 1.0) / (4.0 * pi) * prod) * pow(s, (double)m);
    w(0, 0, m) = pmm;
    if (m + 1 <= N - 1) w(0, 0, m + 1) = x * sqrt(2.0 * m + 3.0) * pmm;
    for (int l = m + 2; l <= N - 1; ++l) {
      double a = sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
      double b = sqrt(((l - 1.0) * (l - 1.0) - (double)m * m) / (4.0 * (l - 1.0) * (l - 1.0) - 1.0));
      w(0, 0, l) = a * (x * w(0, 0, l - 1) - b * w(0, 0, l - 2));
    }
    // -m at n = 0: P^0_{l,-m} = (-1)^m P^0_{l,m}
    for (int l = 0; l < N; ++l) w(1, 0, l) = ((m & 1) ? -1.0 : 1.0) * w(0, 0, l);
  }
  // n = 1..3 by eq. Yninc for both signs of m
  for (int sg = 0; sg < 2; ++sg) {
    double mm = sg ? -(double)m : (double)m;
    for (int n = 1; n <= 3; ++n) {
      for (int l = 0; l < N; ++l) {
        if (l < (m > n ? m : n)) {
          w(sg, n, l) = 0.0;
          continue;
        }
        double al = sqrt((l - n + 1.0) / (double)(l + n));
        double be = (1.0 / l) * sqrt((2.0 * l + 1.0) / (2.0 * l - 1.0) * (l + n - 1.0) *
                                     ((double)l * l - mm * mm) / (double)(l + n));
        double prev_l1 = (l >= 1) ? w(sg, n - 1, l - 1) : 0.0;
        w(sg, n, l) = al * (mm / l - x) / s * w(sg, n - 1, l) + be / s * prev_l1;
      }
    }
  }
  // scatter: n >= 0 from +m; n < 0: P^{-n}_{l,m} = (-1)^(n+m) P^{n}_{l,-m}
  for (int n = -3; n <= 3; ++n) {
    double* out = Pn + (((size_t)(n + 3) * nm + m) * N + i) * N;
    for (int l = 0; l < N; ++l) {
      double v;
      if (n >= 0) {
        v = w(0, n, l);
      } else {
        int an = -n;
        v = (((an + m) & 1) ? -1.0 : 1.0) * w(1, an, l);
      }
      out[l] = v;
    }
  }
}

// F^n_m for one (n, m) per block: Householder QR of P (N x c, c = N - lmin),
// X = R^-1 Q^T with rows l > L zeroed, F = P X.  Scratch per block in global
// memory: A (N x c, column-major), Q (N x c), X (c x N).
__global__ void k_filter_qr(const double* Pn, double* Fraw, double* scratch, int N, int Mmax,
                            int L) {
  int m = blockIdx.x, nidx = blockIdx.y, n = nidx - 3;
  int tid = threadIdx.x, nt = blockDim.x;
  int nm = Mmax + 1;
  int an = n < 0 ? -n : n;
  int lmin = m > an ? m : an;
  int c = N - lmin;
  double* F = Fraw + ((size_t)nidx * nm + m) * N * N;
  const double* Pm = Pn + ((size_t)nidx * nm + m) * N * N;  // [i][l]
  double* A = scratch + ((size_t)nidx * nm + m) * 4 * N * N;  // 4 slabs per block
  double* Q = A + N * N;
  double* tau = Q + N * N;
  double* X = tau + N * N;
  __shared__ double red[256];
  __shared__ double sh_beta, sh_alpha;
  if (c <= 0) {
    for (int t = tid; t < N * N; t += nt) F[t] = 0.0;
    return;
  }
  for (int t = tid; t < N * c; t += nt) {
    int i = t % N, j = t / N;
    A[j * N + i] = Pm[i * N + (lmin + j)];
  }
  __syncthreads();
  // Householder vectors are stored in A below the diagonal with v_j = 1
  // implicit, R on and above the diagonal, tau separately.
  for (int j = 0; j < c; ++j) {
    double part = 0.0;
    for (int i = j + tid; i < N; i += nt) part += A[j * N + i] * A[j * N + i];
    red[tid] = part;
    __syncthreads();
    for (int w = nt / 2; w > 0; w >>= 1) {
      if (tid < w) red[tid] += red[tid + w];
      __syncthreads();
    }
    if (tid == 0) {
      double nrm = sqrt(red[0]);
      double a0 = A[j * N + j];
      double alpha = a0 >= 0 ? -nrm : nrm;  // R_jj
      double v0 = a0 - alpha;
      double tj = 0.0;
      if (nrm > 0.0 && v0 != 0.0) tj = -v0 / alpha;  // tau = (alpha - a0)/alpha ... = -v0/alpha
      sh_alpha = alpha;
      sh_beta = (v0 != 0.0) ? 1.0 / v0 : 0.0;
      tau[j] = tj;
    }
    __syncthreads();
    // scale v (rows below j) by 1/v0
    for (int i = j + 1 + tid; i < N; i += nt) A[j * N + i] *= sh_beta;
    __syncthreads();
    double tj = tau[j];
    // apply H = I - tau v v^T to columns k > j
    for (int k = j + 1; k < c; ++k) {
      double p2 = 0.0;
      for (int i = j + tid; i < N; i += nt) {
        double vi = (i == j) ? 1.0 : A[j * N + i];
        p2 += vi * A[k * N + i];
      }
      red[tid] = p2;
      __syncthreads();
      for (int w = nt / 2; w > 0; w >>= 1) {
        if (tid < w) red[tid] += red[tid + w];
        __syncthreads();
      }
      double dot = red[0];
      __syncthreads();
      for (int i = j + tid; i < N; i += nt) {
        double vi = (i == j) ? 1.0 : A[j * N + i];
        A[k * N + i] -= tj * vi * dot;
      }
      __syncthreads();
    }
    if (tid == 0) A[j * N + j] = sh_alpha;
    __syncthreads();
  }
  // Q = H_0 H_1 ... H_{c-1} applied to the first c columns of I
  for (int t = tid; t < N * c; t += nt) {
    int i = t % N, k = t / N;
    Q[k * N + i] = (i == k) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int j = c - 1; j >= 0; --j) {
    double tj = tau[j];
    for (int k = 0; k < c; ++k) {
      double p2 = 0.0;
      for (int i = j + tid; i < N; i += nt) {
        double vi = (i == j) ? 1.0 : A[j * N + i];
        p2 += vi * Q[k * N + i];
      }
      red[tid] = p2;
      __syncthreads();
      for (int w = nt / 2; w > 0; w >>= 1) {
        if (tid < w) red[tid] += red[tid + w];
        __syncthreads();
      }
      double dot = red[0];
      __syncthreads();
      for (int i = j + tid; i < N; i += nt) {
        double vi = (i == j) ? 1.0 : A[j * N + i];
        Q[k * N + i] -= tj * vi * dot;
      }
      __syncthreads();
    }
  }
  // X = R^-1 Q^T (c x N), one column of Q^T per thread; then zero rows l > L
  __syncthreads();
  for (int col = tid; col < N; col += nt) {
    for (int rr = c - 1; rr >= 0; --rr) {
      double v = Q[rr * N + col];
      for (int k = rr + 1; k < c; ++k) v -= A[k * N + rr] * X[k * N + col];
      X[rr * N + col] = v / A[rr * N + rr];
    }
  }
  __syncthreads();
  for (int t = tid; t < N * N; t += nt) {
    int i = t / N, k = t % N;
    double v = 0.0;
    for (int j = 0; j < c; ++j) {
      int l = lmin + j;
      if (l > L) continue;
      v += Pm[i * N + l] * X[j * N + k];
    }
    F[i * N + k] = v;
  }
}

// Fproj0[m] = F^0_m; FprojC[s-1][m] = [ (F^s_m + F^-s_m)/2 | (F^s_m - F^-s_m)/2 ]
__global__ void k_proj_ops(const double* Fraw, double* F0, double* FC, int N, int Mmax, int L) {
  int nm = Mmax + 1;
  size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  size_t per = (size_t)N * N;
  if (t >= (size_t)(L + 1) * per) return;
  int m = (int)(t / per);
  size_t e = t % per;
  int i = (int)(e / N), k = (int)(e % N);
  F0[m * per + e] = Fraw[((size_t)3 * nm + m) * per + e];
  for (int s = 1; s <= 3; ++s) {
    double fp = Fraw[((size_t)(3 + s) * nm + m) * per + e];
    double fm = Fraw[((size_t)(3 - s) * nm + m) * per + e];
    double* out = FC + (((size_t)(s - 1) * (L + 1) + m) * N + i) * (2 * N);
    out[k] = 0.5 * (fp + fm);
    out[N + k] = 0.5 * (fp - fm);
  }
}

// ---------------------------------------------------------------------------
// Split-precision digits of an FP64 operator (row-major P x K, leading dim
// ld).  Row exponent E: |A[p][k]| < 2^E for all k.  Z = rint(A 2^(47-E)),
// |Z| <= 2^47, balanced base-256 digits d_0..d_5 (d_0 most significant,
// d_1..d_5 in [-128, 127]).  A ~= 2^(E-47) sum_i d_i 256^(5-i).
__global__ void k_slice_rows(const double* A, int P, int K, int ld, int* rowexp) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= ((P + 15) / 16) * 16) return;
  int E = -2000;
  if (p < P) {
    for (int k = 0; k < K; ++k) {
      double v = A[(size_t)p * ld + k];
      if (v != 0.0) {
        int e;
        frexp(v, &e);
        E = e > E ? e : E;
      }
    }
  }
  rowexp[p] = (E == -2000) ? 0 : E;
}

// Largest row sum of |entries| over nmat row-major matrices of rows x cols
// (contiguous), as the bit pattern of a non-negative double in *out.
__global__ void k_max_row_sum(const double* A, int rows, int cols, long long nmat, unsigned long long* out) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= nmat * rows) return;
  const double* a = A + t * cols;
  double s = 0.0;
  for (int k = 0; k < cols; ++k) s += fabs(a[k]);
  atomicMax(out, (unsigned long long)__double_as_longlong(s));
}

// One thread per BF16 value of the tcgen05 operator layout (see TcOp).
__global__ void k_tc_pack(const double* A, int P, int K, int ld, const int* rowexp, unsigned short* w,
                          int rows, int ksteps, size_t total) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= total) return;
  const int blk = (int)(t % (rows * 16));
  size_t r = t / (rows * 16);
  const int q = (int)(r % kTcWSlices);
  r /= kTcWSlices;
  const int ks = (int)(r % ksteps);
  const int grp = (int)(r / ksteps);
  const int core = blk >> 6, rg = core >> 1, kh = core & 1, rr = (blk >> 3) & 7, kk = blk & 7;
  const int row = grp * rows + rg * 8 + rr, col = ks * 16 + kh * 8 + kk;
  if (row >= P || col >= K) {
    w[t] = 0;
    return;
  }
  const double v = A[(size_t)row * ld + col];
  long long Z = (long long)rint(ldexp(v, 47 - rowexp[row]));
  int d[kSlices];
  for (int i = kSlices - 1; i >= 1; --i) {
    long long lo = ((Z % 256) + 256) % 256;
    if (lo >= 128) lo -= 256;
    d[i] = (int)lo;
    Z = (Z - lo) / 256;
  }
  d[0] = (int)Z;
  // slice q: digit q (q < 5), digit q - 5 times 2^-8 (q < 11), digit q - 10
  // times 2^-16; all exact in BF16 (|d| <= 128)
  float f = (float)(q < 5 ? d[q] : (q < 11 ? d[q - 5] : d[q - 10]));
  if (q >= 11)
    f *= 1.52587890625e-05f;  // 2^-16
  else if (q >= 5)
    f *= 0.00390625f;         // 2^-8
  w[t] = (unsigned short)(__float_as_uint(f) >> 16);
}

int build_tc(TcOp& s, const double* A, int P, int K, int ld, size_t& bytes, int nbatch = 1,
             size_t a_stride = 0, int rows = 0) {
  s.P = P;
  s.K = K;
  s.rows = rows == 48 || rows == 96 ? rows : (P <= 48 ? 48 : 96);
  s.ngroups = (P + s.rows - 1) / s.rows;
  s.ksteps = (K + 15) / 16;
  s.nbatch = nbatch;
  s.w_stride = (size_t)s.ngroups * s.ksteps * kTcWSlices * s.rows * 16;
  s.rowexp_stride = (size_t)s.ngroups * s.rows;
  CF_CUDA(cudaMalloc(&s.w, s.w_stride * nbatch * sizeof(unsigned short)));
  CF_CUDA(cudaMalloc(&s.rowexp, s.rowexp_stride * nbatch * sizeof(int)));
  CF_CUDA(cudaMemset(s.rowexp, 0, s.rowexp_stride * nbatch * sizeof(int)));
  bytes += s.w_stride * nbatch * sizeof(unsigned short) + s.rowexp_stride * nbatch * sizeof(int);
  for (int b = 0; b < nbatch; ++b) {
    const double* Ab = A + (size_t)b * a_stride;
    int* re = s.rowexp + (size_t)b * s.rowexp_stride;
    k_slice_rows<<<(unsigned)((s.rowexp_stride + 127) / 128), 128>>>(Ab, P, K, ld, re);
    k_tc_pack<<<(unsigned)((s.w_stride + 255) / 256), 256>>>(Ab, P, K, ld, re, s.w + (size_t)b * s.w_stride,
                                                             s.rows, s.ksteps, s.w_stride);
  }
  CF_CUDA(cudaGetLastError());
  return CFFYN_OK;
}

void free_tc(TcOp& s) {
  if (s.w) cudaFree(s.w);
  if (s.rowexp) cudaFree(s.rowexp);
  s.w = nullptr;
  s.rowexp = nullptr;
}

// The split-precision operators of one family of launches (the families of
// cffyn_set_operator_rows): 0 d_r, 1 d_theta with d_phi, 2 phi analysis,
// 3 projections (every spin class and the graded sets), 4 phi synthesis; with
// the shell's row-group choice (0: 48 up to 48 rows, else 96).  Frees the
// family's previous operators.
int build_tc_family(cffyn_shell* sh, int which) {
  const int n_r = sh->n_r, N = sh->N, J = sh->J, R = sh->R, Lrows = sh->Lrows;
  const int nm = sh->L + 1;
  const int rows = sh->op_rows[which];
  size_t& B = sh->bytes;
  int rc = CFFYN_OK;
  auto rebuild = [&](TcOp& t, const double* A, int P, int K, int ld, int nb, size_t st) {
    if (t.w) B -= t.w_stride * t.nbatch * sizeof(unsigned short) + t.rowexp_stride * t.nbatch * sizeof(int);
    free_tc(t);
    return build_tc(t, A, P, K, ld, B, nb, st, rows);
  };
  switch (which) {
    case 0:
      rc = rebuild(sh->tDr, sh->Dr, n_r, n_r, n_r, 1, 0);
      break;
    case 1:
      if (!(rc = rebuild(sh->tDth2, sh->Dth2, 2 * N, 2 * N, 2 * N, 1, 0)))
        rc = rebuild(sh->tDph, sh->Dph, J, J, J, 1, 0);
      break;
    case 2:
      rc = rebuild(sh->tFan, sh->Fan, R, J, J, 1, 0);
      break;
    case 3:
      rc = rebuild(sh->tF0, sh->Fproj0, N, N, N, nm, (size_t)N * N);
      for (int s = 0; s < 3 && !rc; ++s)
        rc = rebuild(sh->tFC[s], sh->FprojC + (size_t)s * nm * N * 2 * N, N, 2 * N, 2 * N, nm,
                     (size_t)N * 2 * N);
      if (sh->F0g)
        for (int d = 0; d < 4 && !rc; ++d)
          rc = rebuild(sh->tF0g[d], sh->F0g + (size_t)d * (Lrows + 1) * N * N, N, N, N, Lrows + 1,
                       (size_t)N * N);
      break;
    case 4:
      rc = rebuild(sh->tFsy, sh->Fsy, J, R, R, 1, 0);
      break;
    default:
      set_error("operator family %d outside 0..%d", which, kOpFamilies - 1);
      return CFFYN_EINVAL;
  }
  if (rc) return rc;
  CF_CUDA(cudaDeviceSynchronize());
  return CFFYN_OK;
}

// Builds every operator of the shell.  Called from cffyn_create_shell_ex.
int build_operators(cffyn_shell* sh) {
  const int n_r = sh->n_r, N = sh->N, J = sh->J, L = sh->L, R = sh->R, Lrows = sh->Lrows;
  size_t& B = sh->bytes;
  auto alloc = [&](double** p, size_t n) -> int {
    CF_CUDA(cudaMalloc(p, n * sizeof(double)));
    B += n * sizeof(double);
    return CFFYN_OK;
  };
  int rc;
  if ((rc = alloc(&sh->r, n_r)) || (rc = alloc(&sh->sth, N)) || (rc = alloc(&sh->cth, N)) ||
      (rc = alloc(&sh->sph, J)) || (rc = alloc(&sh->cph, J)))
    return rc;
  int mx = n_r > J ? n_r : J;
  k_grid<<<(mx + 127) / 128, 128>>>(sh->r, sh->sth, sh->cth, sh->sph, sh->cph, n_r, N, J,
                                   sh->d.r_in, sh->d.r_out);
  if ((rc = alloc(&sh->Dr, (size_t)n_r * n_r))) return rc;
  k_cheb<<<(n_r + 63) / 64, 64>>>(sh->Dr, n_r, 2.0 / (sh->d.r_out - sh->d.r_in));
  if ((rc = alloc(&sh->Dph, (size_t)J * J)) || (rc = alloc(&sh->Dth2, (size_t)4 * N * N))) return rc;
  k_fourier_ops<<<(J * J + 255) / 256, 256>>>(sh->Dph, J, sh->Dth2, N);
  if ((rc = alloc(&sh->Fan, (size_t)R * J)) || (rc = alloc(&sh->Fsy, (size_t)J * R))) return rc;
  k_dft<<<(R * J + 255) / 256, 256>>>(sh->Fan, sh->Fsy, J, Lrows);
  CF_CUDA(cudaGetLastError());

  // spin-weighted Legendre and filter matrices for m = 0..L
  const int Mmax = L;
  const int nm = Mmax + 1;
  double *Pn = nullptr, *tmp = nullptr, *scratch = nullptr;
  CF_CUDA(cudaMalloc(&Pn, (size_t)7 * nm * N * N * sizeof(double)));
  CF_CUDA(cudaMalloc(&tmp, (size_t)N * nm * 8 * N * sizeof(double)));
  CF_CUDA(cudaMalloc(&scratch, (size_t)7 * nm * 4 * N * N * sizeof(double)));
  k_spin_legendre<<<(N * nm + 63) / 64, 64>>>(Pn, tmp, N, Mmax);
  if ((rc = alloc(&sh->Fraw, (size_t)7 * nm * N * N))) return rc;
  k_filter_qr<<<dim3(nm, 7), 128>>>(Pn, sh->Fraw, scratch, N, Mmax, L);
  if ((rc = alloc(&sh->Fproj0, (size_t)nm * N * N)) || (rc = alloc(&sh->FprojC, (size_t)3 * nm * N * 2 * N)))
    return rc;
  k_proj_ops<<<(unsigned)(((size_t)nm * N * N + 255) / 256), 256>>>(sh->Fraw, sh->Fproj0,
                                                                    sh->FprojC, N, Mmax, L);
  CF_CUDA(cudaGetLastError());
  CF_CUDA(cudaDeviceSynchronize());
  cudaFree(Pn);
  cudaFree(tmp);
  cudaFree(scratch);

  // graded filter (eq. nfofmu): F^0_m at the retained degrees L + d,
  // d = 0..3 (at most N - 1), for m = 0..Lrows
  if (sh->d.filter_kind == CFFYN_FILTER_YG) {
    const int nmg = Lrows + 1;
    double *Pg = nullptr, *tg = nullptr, *sg = nullptr, *Fg = nullptr;
    CF_CUDA(cudaMalloc(&Pg, (size_t)7 * nmg * N * N * sizeof(double)));
    CF_CUDA(cudaMalloc(&tg, (size_t)N * nmg * 8 * N * sizeof(double)));
    CF_CUDA(cudaMalloc(&sg, (size_t)7 * nmg * 4 * N * N * sizeof(double)));
    CF_CUDA(cudaMalloc(&Fg, (size_t)7 * nmg * N * N * sizeof(double)));
    if ((rc = alloc(&sh->F0g, (size_t)4 * nmg * N * N))) return rc;
    k_spin_legendre<<<(N * nmg + 63) / 64, 64>>>(Pg, tg, N, Lrows);
    for (int d = 0; d < 4; ++d) {
      const int cut = L + d < N - 1 ? L + d : N - 1;
      k_filter_qr<<<dim3(nmg, 7), 128>>>(Pg, Fg, sg, N, Lrows, cut);
      // the n = 0 matrices
      CF_CUDA(cudaMemcpyAsync(sh->F0g + (size_t)d * nmg * N * N, Fg + (size_t)3 * nmg * N * N,
                              (size_t)nmg * N * N * sizeof(double), cudaMemcpyDeviceToDevice));
    }
    CF_CUDA(cudaGetLastError());
    CF_CUDA(cudaDeviceSynchronize());
    cudaFree(Pg);
    cudaFree(tg);
    cudaFree(sg);
    cudaFree(Fg);
  }

  // exponent gains of the filter operators (see cffyn_shell::gain_dft)
  {
    unsigned long long* g = nullptr;
    CF_CUDA(cudaMalloc(&g, 2 * sizeof(unsigned long long)));
    CF_CUDA(cudaMemset(g, 0, 2 * sizeof(unsigned long long)));
    auto rows = [&](const double* A, int r, int c, long long n, unsigned long long* o) {
      const long long t = n * r;
      k_max_row_sum<<<(unsigned)((t + 127) / 128), 128>>>(A, r, c, n, o);
    };
    rows(sh->Fan, R, J, 1, g);
    rows(sh->Fproj0, N, N, nm, g + 1);
    rows(sh->FprojC, N, 2 * N, 3LL * nm, g + 1);
    if (sh->F0g) rows(sh->F0g, N, N, 4LL * (Lrows + 1), g + 1);
    unsigned long long h[2];
    CF_CUDA(cudaMemcpy(h, g, sizeof(h), cudaMemcpyDeviceToHost));
    cudaFree(g);
    double mx[2];
    memcpy(mx, h, sizeof(h));
    int e[2];
    for (int i = 0; i < 2; ++i) {
      frexp(mx[i], &e[i]);  // mx < 2^e
      if (!(mx[i] > 0.0)) e[i] = 0;
      if (e[i] < 0) e[i] = 0;
    }
    sh->gain_dft = e[0];
    sh->gain_proj = e[1];
  }

  // split-precision digits of every operator (used by the mixed path)
  if (sh->d.precision == CFFYN_MIXED)
    for (int w = 0; w < kOpFamilies; ++w)
      if ((rc = build_tc_family(sh, w))) return rc;
  return CFFYN_OK;
}

}  // namespace cffyn
