// Helpers shared by the pointwise kernels (pointwise.cu, rhs.cu): grid
// geometry, the chain-rule Jacobian of eq. dvdx, the 3+1 quantities of eqs.
// normal / abgfromgab and the Christoffel symbols of eq. Gamma.
#pragma once
#include "common.cuh"
#include "scalar.cuh"

namespace cffyn {

struct Geo {
  int n_r, N, J, nv;
  long long P;
  const double *r, *sth, *cth, *sph, *cph;
  const double* triad;  // [J][N][9] rows of the real triad (internal storage)
};

// symmetric pair index of (a, b), a, b in 0..3 (tt,tx,ty,tz,xx,xy,xz,yy,yz,zz)
// (flat, so that it folds to a constant inside unrolled loops and every
// tensor array stays in registers)
__host__ __device__ __forceinline__ constexpr int SI(int a, int b) {
  const int lo = a < b ? a : b, hi = a < b ? b : a;
  return lo == 0 ? hi : (lo == 1 ? 3 + hi : (lo == 2 ? 5 + hi : 9));
}

template <class T>
struct Jac {
  // d/dx^k = J[k][0] d_r + J[k][1] d_theta + J[k][2] d_phi
  T j[3][3];
  T st, ct, sp, cp;
};

template <class T>
__device__ __forceinline__ Jac<T> jacobian(const Geo& g, int k, int i, int jj) {
  Jac<T> J;
  const T st = S<T>::c(g.sth[i]), ct = S<T>::c(g.cth[i]);
  const T sp = S<T>::c(g.sph[jj]), cp = S<T>::c(g.cph[jj]);
  const T one = S<T>::c(1.0);
  const T ir = one / S<T>::c(g.r[k]);
  const T irs = ir / st;
  J.j[0][0] = st * cp; J.j[0][1] = ct * cp * ir; J.j[0][2] = -(sp * irs);
  J.j[1][0] = st * sp; J.j[1][1] = ct * sp * ir; J.j[1][2] = cp * irs;
  J.j[2][0] = ct;      J.j[2][1] = -(st * ir);   J.j[2][2] = S<T>::c(0.0);
  J.st = st; J.ct = ct; J.sp = sp; J.cp = cp;
  return J;
}

// Cartesian derivative d_k of field mu at point p from the three spherical
// derivative arrays D[3][nv][P].
template <class T>
__device__ __forceinline__ void cart3(const Jac<T>& J, const double* __restrict__ D, long long P,
                                      int nv, int mu, long long p, T out[3]) {
  const T dr = S<T>::load(D + (long long)mu * P + p);
  const T dt = S<T>::load(D + ((long long)nv + mu) * P + p);
  const T dp = S<T>::load(D + ((long long)2 * nv + mu) * P + p);
#pragma unroll
  for (int k = 0; k < 3; ++k) out[k] = J.j[k][0] * dr + J.j[k][1] * dt + J.j[k][2] * dp;
}

// 3+1 quantities and Christoffel symbols from the undifferentiated fields.
template <class T>
struct Metric {
  T gi4[10];          // g^ab (symmetric pairs)
  T gi[3][3];         // gamma^ij
  T bu[3];            // beta^i
  T alpha, ialpha;
  T nu[4];            // n^a
};

template <class T>
__device__ __forceinline__ void metric_from(const T g[10], Metric<T>& M) {
  const T gxx = g[4], gxy = g[5], gxz = g[6], gyy = g[7], gyz = g[8], gzz = g[9];
  const T cxx = gyy * gzz - gyz * gyz, cxy = gxz * gyz - gxy * gzz, cxz = gxy * gyz - gxz * gyy;
  const T cyy = gxx * gzz - gxz * gxz, cyz = gxy * gxz - gxx * gyz, czz = gxx * gyy - gxy * gxy;
  const T idet = S<T>::c(1.0) / (gxx * cxx + gxy * cxy + gxz * cxz);
  M.gi[0][0] = cxx * idet; M.gi[0][1] = M.gi[1][0] = cxy * idet; M.gi[0][2] = M.gi[2][0] = cxz * idet;
  M.gi[1][1] = cyy * idet; M.gi[1][2] = M.gi[2][1] = cyz * idet; M.gi[2][2] = czz * idet;
  const T b[3] = {g[1], g[2], g[3]};
#pragma unroll
  for (int i = 0; i < 3; ++i) M.bu[i] = M.gi[i][0] * b[0] + M.gi[i][1] * b[1] + M.gi[i][2] * b[2];
  const T a2 = b[0] * M.bu[0] + b[1] * M.bu[1] + b[2] * M.bu[2] - g[0];
  M.alpha = sqrt_s(a2);
  M.ialpha = S<T>::c(1.0) / M.alpha;
  const T ia2 = M.ialpha * M.ialpha;
  M.nu[0] = M.ialpha;
#pragma unroll
  for (int i = 0; i < 3; ++i) M.nu[i + 1] = -(M.bu[i] * M.ialpha);
  M.gi4[0] = -ia2;
#pragma unroll
  for (int i = 0; i < 3; ++i) M.gi4[SI(0, i + 1)] = M.bu[i] * ia2;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) M.gi4[SI(i + 1, j + 1)] = M.gi[i][j] - M.bu[i] * M.bu[j] * ia2;
}

// dg4[c][s] = d_c g_ab; Gam[c][s] = Gamma_cab; Gc[c] = Gamma_c
template <class T>
__device__ __forceinline__ void christoffel(const Metric<T>& M, const T Pi[10], const T Ph[3][10],
                                            T dg4[4][10], T Gam[4][10], T Gc[4]) {
#pragma unroll
  for (int s = 0; s < 10; ++s) {
    dg4[0][s] = M.bu[0] * Ph[0][s] + M.bu[1] * Ph[1][s] + M.bu[2] * Ph[2][s] - M.alpha * Pi[s];
#pragma unroll
    for (int i = 0; i < 3; ++i) dg4[i + 1][s] = Ph[i][s];
  }
  const T half = S<T>::c(0.5);
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = a; b < 4; ++b)
        Gam[c][SI(a, b)] = half * (dg4[a][SI(b, c)] + dg4[b][SI(a, c)] - dg4[c][SI(a, b)]);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    T acc = S<T>::c(0.0);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc = acc + M.gi4[SI(a, b)] * Gam[c][SI(a, b)];
    Gc[c] = acc;
  }
}


inline Geo geo_of(const cffyn_shell* sh) {
  Geo g;
  g.n_r = sh->n_r;
  g.N = sh->N;
  g.J = sh->J;
  g.nv = sh->nv;
  g.P = (long long)P_all(sh);
  g.r = sh->r;
  g.sth = sh->sth;
  g.cth = sh->cth;
  g.sph = sh->sph;
  g.cph = sh->cph;
  g.triad = sh->triad;
  return g;
}

inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace cffyn
