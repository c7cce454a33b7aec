// GHG right-hand side (paper App. A.1, eqs. gdot, Phidot, Pidot; gamma_0 =
// gamma_2 = 1, gamma_1 = -1) with the freeze-incoming boundary condition of
// App. A.2, as three pointwise kernels so that none of them spills registers
// (the state of one point alone is 50 values; in the double-float path that
// is 100 registers):
//
//   k_rhs_gamma  3+1 quantities (eqs. normal, abgfromgab), d_t g_ab (eq. gdot,
//                written as the first ten outputs), Christoffel symbols from
//                undifferentiated fields (eq. Gamma), Gamma_c, the gauge
//                constraint C_a = H_a + Gamma_a, nabla_(a H_b), and the
//                Gamma-Gamma term of eq. Pidot -> partial source of d_t Pi.
//   k_rhs_quad   the Phi-Phi and Pi-Pi terms of eq. Pidot, the remaining
//                algebraic terms of eqs. Pidot and Phidot -> sources.
//   k_rhs_pp     principal parts -A^k d_k u from the spherical derivatives,
//                with the chain rule (eq. dvdx) contracted into the shift and
//                inverse metric once per point, plus the boundary condition
//                on the outermost sphere.
//   k_gauge_rhs  54/58-field states only, ahead of k_rhs_gamma: H_a and its
//                derivatives from the state, and the gauge fields' own
//                right-hand sides.
//
// Source buffer src[50][P]: [0,10) source of d_t Pi_ab, [10,40) source of
// d_t Phi_iab (10 + 10 i + s), 40 alpha, [41,44) beta^i, [44,50) gamma^ij
// (xx, xy, xz, yy, yz, zz).
#include "pw_common.cuh"

namespace cffyn {

template <class T, bool F>
__device__ __forceinline__ T ldA(const double* a, long long P, long long p, int f) {
  return Store<T, F>::ld(a, (long long)f * P + p);
}
template <class T, bool F>
__device__ __forceinline__ void stA(double* a, long long P, long long p, int f, T v) {
  Store<T, F>::st(a, (long long)f * P + p, v);
}
// internal buffers are pair-stored in the double-float path
template <class T> constexpr bool kInt = false;
template <> constexpr bool kInt<ff> = true;

// Per-thread working tensors that rolled loops index at run time live in
// shared memory as [slot][thread] (consecutive threads, consecutive words: no
// bank conflicts); the outer contraction loops stay rolled so that the code
// of a kernel fits the instruction caches, the inner ones unrolled so that
// independent accumulations overlap.
template <class T, int NB>
struct Slots {
  T* s;
  __device__ __forceinline__ T& operator()(int v) const { return s[v * NB + (int)threadIdx.x]; }
};

constexpr int kRhsBlock = 128;
constexpr int kGamSlots = 54;   // Gamma_cab (c*10 + s) | S_Pi 40..49 | C_a 50..53
constexpr int kQuadSlots = 50;  // Pi 0..9 | Phi_iab 10 + 10 i + s | Q 40..49

// Four blocks per SM: 128 registers, 54 KB of slots (g_ab is read again from
// u where the gauge terms need it instead of holding ten more slots).
template <class T, bool FU, bool FO>
__global__ void __launch_bounds__(kRhsBlock, 4) k_rhs_gamma(const double* __restrict__ u,
                                                         const double* __restrict__ H,
                                                         const double* __restrict__ dH,
                                                         double* __restrict__ src, double* __restrict__ out,
                                                         Geo geo, int dtH) {
  __shared__ T sm[kGamSlots * kRhsBlock];
  const Slots<T, kRhsBlock> V{sm};
  const long long P = geo.P;
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= P) return;
  const T zero = S<T>::c(0.0), half = S<T>::c(0.5);

  Metric<T> M;
  {
    T g[10];
#pragma unroll
    for (int s = 0; s < 10; ++s) {
      g[s] = ldA<T, FU>(u, P, p, s);
    }
    metric_from(g, M);
  }
  stA<T, kInt<T>>(src, P, p, 40, M.alpha);
#pragma unroll
  for (int x = 0; x < 3; ++x) stA<T, kInt<T>>(src, P, p, 41 + x, M.bu[x]);
  stA<T, kInt<T>>(src, P, p, 44, M.gi[0][0]);
  stA<T, kInt<T>>(src, P, p, 45, M.gi[0][1]);
  stA<T, kInt<T>>(src, P, p, 46, M.gi[0][2]);
  stA<T, kInt<T>>(src, P, p, 47, M.gi[1][1]);
  stA<T, kInt<T>>(src, P, p, 48, M.gi[1][2]);
  stA<T, kInt<T>>(src, P, p, 49, M.gi[2][2]);

  // d_t g_ab (eq. gdot) and the Christoffel symbols Gamma_cab
  {
    T dtg[10], Ph[3][10];
#pragma unroll
    for (int s = 0; s < 10; ++s) {
#pragma unroll
      for (int x = 0; x < 3; ++x) Ph[x][s] = ldA<T, FU>(u, P, p, 20 + 10 * x + s);
      Acc<T> a;
#pragma unroll
      for (int x = 0; x < 3; ++x) a.fma_(M.bu[x], Ph[x][s]);
      a.fma_(-M.alpha, ldA<T, FU>(u, P, p, 10 + s));
      dtg[s] = a.get();
      stA<T, FO>(out, P, p, s, dtg[s]);
    }
    auto dg4 = [&](int c, int s) -> T { return c == 0 ? dtg[s] : Ph[c - 1][s]; };
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = a; b < 4; ++b)
          V(c * 10 + SI(a, b)) = half * (dg4(a, SI(b, c)) + dg4(b, SI(a, c)) - dg4(c, SI(a, b)));
  }
  // Gamma_c = g^ab Gamma_cab (symmetric pairs counted twice off the diagonal);
  // gauge constraint C_c = H_c + Gamma_c, H^c, n^c C_c
  T Hup[4], nC;
  {
    T Hd[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) Hd[a] = ldA<T, kInt<T>>(H, P, p, a);
    Acc<T> an;
#pragma unroll 1
    for (int c = 0; c < 4; ++c) {
      Acc<T> acc;
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = a; b < 4; ++b) {
          const T w = (a == b) ? M.gi4[SI(a, b)] : M.gi4[SI(a, b)] + M.gi4[SI(a, b)];
          acc.fma_(w, V(c * 10 + SI(a, b)));
        }
      const T hc = c == 0 ? Hd[0] : (c == 1 ? Hd[1] : (c == 2 ? Hd[2] : Hd[3]));
      acc.add(hc);
      V(50 + c) = acc.get();
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      Acc<T> acc;
#pragma unroll
      for (int d = 0; d < 4; ++d) acc.fma_(M.gi4[SI(c, d)], Hd[d]);
      Hup[c] = acc.get();
      an.fma_(M.nu[c], V(50 + c));
    }
    nC = an.get();
  }
  // S_Pi = -2 alpha nabla_(a H_b) + alpha (n_b C_a + n_a C_b - g_ab n^c C_c)
  {
    const T twoal = M.alpha + M.alpha;
    const T aa = M.alpha * (-M.alpha);  // alpha n_0, n_a = (-alpha, 0, 0, 0)
    const T anC = M.alpha * nC;
#pragma unroll 1
    for (int s = 0; s < 10; ++s) {
      const int a = s < 4 ? 0 : (s < 7 ? 1 : (s < 9 ? 2 : 3));
      const int b = s - (a == 0 ? 0 : (a == 1 ? 3 : (a == 2 ? 5 : 6)));
      // d_a H_b: rows (x, b) = 4 x + b of dH for a = x + 1; d_t H_b is row
      // 12 + b when the gauge source is evolved with its time derivative
      // (58 fields), else zero
      const T dHab = a == 0 ? (dtH ? ldA<T, kInt<T>>(dH, P, p, 12 + b) : zero)
                            : ldA<T, kInt<T>>(dH, P, p, (a - 1) * 4 + b);
      const T dHba = b == 0 ? (dtH ? ldA<T, kInt<T>>(dH, P, p, 12 + a) : zero)
                            : ldA<T, kInt<T>>(dH, P, p, (b - 1) * 4 + a);
      Acc<T> acc;
      acc.fma_(half, dHab + dHba);
#pragma unroll
      for (int c = 0; c < 4; ++c) acc.fma_(-V(c * 10 + s), Hup[c]);
      const T DH = acc.get();
      Acc<T> v;
      v.fma_(-twoal, DH);
      v.fma_(-(anC), ldA<T, FU>(u, P, p, s));
      if (a == 0) v.fma_(aa, V(50 + b));
      if (b == 0) v.fma_(aa, V(50 + a));
      V(40 + s) = v.get();
    }
  }
  // -2 alpha g^cd g^ef Gamma_ace Gamma_bdf
  {
    const T m2al = -(M.alpha + M.alpha);
#pragma unroll 1
    for (int b = 0; b < 4; ++b) {
      T Gce[10];  // Gamma_b^{ce}, symmetric, off-diagonal weight 2
      {
        T Gcf[4][4];  // Gamma_b^c_f = g^cd Gamma_bdf
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int f = 0; f < 4; ++f) {
            Acc<T> acc;
#pragma unroll
            for (int d = 0; d < 4; ++d) acc.fma_(M.gi4[SI(c, d)], V(b * 10 + SI(d, f)));
            Gcf[c][f] = acc.get();
          }
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int e = c; e < 4; ++e) {
            Acc<T> acc;
#pragma unroll
            for (int f = 0; f < 4; ++f) acc.fma_(M.gi4[SI(e, f)], Gcf[c][f]);
            Gce[SI(c, e)] = (c == e) ? acc.get() : acc.get() + acc.get();
          }
      }
#pragma unroll 1
      for (int a = 0; a <= b; ++a) {
        Acc<T> qa;
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int e = c; e < 4; ++e) qa.fma_(V(a * 10 + SI(c, e)), Gce[SI(c, e)]);
        Acc<T> acc;
        acc.add(V(40 + SI(a, b)));
        acc.fma_(m2al, qa.get());
        V(40 + SI(a, b)) = acc.get();
      }
    }
  }
#pragma unroll
  for (int s = 0; s < 10; ++s) stA<T, kInt<T>>(src, P, p, s, V(40 + s));
}

// The Phi-Phi and Pi-Pi terms of eq. Pidot and the remaining algebraic terms
// of eqs. Pidot and Phidot; alpha, beta^i, gamma^ij come from k_rhs_gamma.
template <class T, bool FU>
__global__ void __launch_bounds__(kRhsBlock) k_rhs_quad(const double* __restrict__ u, double* __restrict__ src,
                                                        Geo geo) {
  __shared__ T sm[kQuadSlots * kRhsBlock];
  const Slots<T, kRhsBlock> V{sm};
  const long long P = geo.P;
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= P) return;
  const T half = S<T>::c(0.5);
  // 3+1 quantities (eqs. normal, abgfromgab) as k_rhs_gamma derived them
  const T alpha = ldA<T, kInt<T>>(src, P, p, 40);
  T bu[3], gi[3][3];
#pragma unroll
  for (int x = 0; x < 3; ++x) bu[x] = ldA<T, kInt<T>>(src, P, p, 41 + x);
  gi[0][0] = ldA<T, kInt<T>>(src, P, p, 44);
  gi[0][1] = gi[1][0] = ldA<T, kInt<T>>(src, P, p, 45);
  gi[0][2] = gi[2][0] = ldA<T, kInt<T>>(src, P, p, 46);
  gi[1][1] = ldA<T, kInt<T>>(src, P, p, 47);
  gi[1][2] = gi[2][1] = ldA<T, kInt<T>>(src, P, p, 48);
  gi[2][2] = ldA<T, kInt<T>>(src, P, p, 49);
  const T ialpha = S<T>::c(1.0) / alpha;
  const T ia2 = ialpha * ialpha;
  T nu[4], gi4[10];
  nu[0] = ialpha;
#pragma unroll
  for (int i = 0; i < 3; ++i) nu[i + 1] = -(bu[i] * ialpha);
  gi4[0] = -ia2;
#pragma unroll
  for (int i = 0; i < 3; ++i) gi4[SI(0, i + 1)] = bu[i] * ia2;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) gi4[SI(i + 1, j + 1)] = gi[i][j] - bu[i] * bu[j] * ia2;

#pragma unroll
  for (int s = 0; s < 10; ++s) {
    V(s) = ldA<T, FU>(u, P, p, 10 + s);
#pragma unroll
    for (int x = 0; x < 3; ++x) V(10 + 10 * x + s) = ldA<T, FU>(u, P, p, 20 + 10 * x + s);
  }
  const T twoal = alpha + alpha;
  // Q = Q1 - Q2 into slots 40..49; Q2_ab = Pi_ac g^cd Pi_db
#pragma unroll 1
  for (int b = 0; b < 4; ++b) {
    T Piu[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      Acc<T> acc;
#pragma unroll
      for (int d = 0; d < 4; ++d) acc.fma_(gi4[SI(c, d)], V(SI(b, d)));
      Piu[c] = acc.get();
    }
#pragma unroll 1
    for (int a = 0; a <= b; ++a) {
      Acc<T> acc;
#pragma unroll
      for (int c = 0; c < 4; ++c) acc.fma_(-V(SI(a, c)), Piu[c]);
      V(40 + SI(a, b)) = acc.get();
    }
  }
  // Q1_ab = gamma^ij g^cd Phi_iac Phi_jbd
#pragma unroll 1
  for (int b = 0; b < 4; ++b) {
    T W[3][4];
    {
      T Y[3][4];
#pragma unroll
      for (int x = 0; x < 3; ++x)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          Acc<T> acc;
#pragma unroll
          for (int d = 0; d < 4; ++d) acc.fma_(gi4[SI(c, d)], V(10 + 10 * x + SI(b, d)));
          Y[x][c] = acc.get();
        }
#pragma unroll
      for (int x = 0; x < 3; ++x)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          Acc<T> acc;
#pragma unroll
          for (int y = 0; y < 3; ++y) acc.fma_(gi[x][y], Y[y][c]);
          W[x][c] = acc.get();
        }
    }
#pragma unroll 1
    for (int a = 0; a <= b; ++a) {
      Acc<T> acc;
      acc.add(V(40 + SI(a, b)));
#pragma unroll
      for (int x = 0; x < 3; ++x)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc.fma_(V(10 + 10 * x + SI(a, c)), W[x][c]);
      V(40 + SI(a, b)) = acc.get();
    }
  }
  // remaining algebraic terms of eq. Pidot
  T nnPi;
  {
    Acc<T> acc;
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int d = 0; d < 4; ++d) acc.fma_(nu[c] * nu[d], V(SI(c, d)));
    nnPi = acc.get();
  }
  T cPh[3];  // beta^j - alpha n^c Pi_ci gamma^ij
  {
    T nPi[3];
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      Acc<T> acc;
#pragma unroll
      for (int c = 0; c < 4; ++c) acc.fma_(nu[c], V(SI(c, x + 1)));
      nPi[x] = acc.get();
    }
#pragma unroll
    for (int y = 0; y < 3; ++y) {
      Acc<T> acc;
#pragma unroll
      for (int x = 0; x < 3; ++x) acc.fma_(nPi[x], gi[x][y]);
      cPh[y] = bu[y] - alpha * acc.get();
    }
  }
  const T hal = half * alpha;
  const T cPi = -(hal * nnPi);
#pragma unroll 1
  for (int s = 0; s < 10; ++s) {
    Acc<T> acc;
    acc.add(ldA<T, kInt<T>>(src, P, p, s));
    acc.fma_(twoal, V(40 + s));
    acc.fma_(cPi, V(s));
#pragma unroll
    for (int x = 0; x < 3; ++x) acc.fma_(cPh[x], V(10 + 10 * x + s));
    stA<T, kInt<T>>(src, P, p, s, acc.get());
  }
  // algebraic terms of eq. Phidot
#pragma unroll 1
  for (int x = 0; x < 3; ++x) {
    T nnPhi;
    {
      Acc<T> acc;
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int d = 0; d < 4; ++d) acc.fma_(nu[c] * nu[d], V(10 + 10 * x + SI(c, d)));
      nnPhi = acc.get();
    }
    T Mk[3];  // alpha gamma^jk n^c Phi_x,j,c
    {
      T nP[3];
#pragma unroll
      for (int y = 0; y < 3; ++y) {
        Acc<T> acc;
#pragma unroll
        for (int c = 0; c < 4; ++c) acc.fma_(nu[c], V(10 + 10 * x + SI(y + 1, c)));
        nP[y] = acc.get();
      }
#pragma unroll
      for (int z = 0; z < 3; ++z) {
        Acc<T> acc;
#pragma unroll
        for (int y = 0; y < 3; ++y) acc.fma_(nP[y], gi[y][z]);
        Mk[z] = alpha * acc.get();
      }
    }
    const T hnn = hal * nnPhi;
#pragma unroll 1
    for (int s = 0; s < 10; ++s) {
      Acc<T> acc;
      acc.fma_(hnn, V(s));
#pragma unroll
      for (int z = 0; z < 3; ++z) acc.fma_(Mk[z], V(10 + 10 * z + s));
      acc.fma_(-alpha, V(10 + 10 * x + s));
      stA<T, kInt<T>>(src, P, p, 10 + 10 * x + s, acc.get());
    }
  }
}

template <class T, bool FO>
__global__ void __launch_bounds__(128) k_rhs_pp(const double* __restrict__ D, const double* __restrict__ src,
                                                double* __restrict__ out, Geo geo) {
  const long long P = geo.P;
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= P) return;
  const int k = (int)(p % geo.n_r);
  const int i = (int)((p / geo.n_r) % geo.N);
  const int jj = (int)((p / ((long long)geo.n_r * geo.N)) % geo.J);
  const int nv = geo.nv;
  const T half = S<T>::c(0.5);
  const Jac<T> J = jacobian<T>(geo, k, i, jj);
  const T alpha = ldA<T, kInt<T>>(src, P, p, 40);
  T bu[3], gi[3][3];
#pragma unroll
  for (int x = 0; x < 3; ++x) bu[x] = ldA<T, kInt<T>>(src, P, p, 41 + x);
  gi[0][0] = ldA<T, kInt<T>>(src, P, p, 44);
  gi[0][1] = gi[1][0] = ldA<T, kInt<T>>(src, P, p, 45);
  gi[0][2] = gi[2][0] = ldA<T, kInt<T>>(src, P, p, 46);
  gi[1][1] = ldA<T, kInt<T>>(src, P, p, 47);
  gi[1][2] = gi[2][1] = ldA<T, kInt<T>>(src, P, p, 48);
  gi[2][2] = ldA<T, kInt<T>>(src, P, p, 49);
  // beta^k d_k = sum_m b_m D_m; alpha gamma^ik d_k = sum_m G_im D_m; J_xm for d_x
  T b[3], G[3][3];
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    Acc<T> acc;
#pragma unroll
    for (int x = 0; x < 3; ++x) acc.fma_(bu[x], J.j[x][m]);
    b[m] = acc.get();
  }
#pragma unroll
  for (int x = 0; x < 3; ++x)
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      Acc<T> acc;
#pragma unroll
      for (int y = 0; y < 3; ++y) acc.fma_(gi[x][y], J.j[y][m]);
      G[x][m] = alpha * acc.get();
    }
  T aJ[3][3];
#pragma unroll
  for (int x = 0; x < 3; ++x)
#pragma unroll
    for (int m = 0; m < 3; ++m) aJ[x][m] = alpha * J.j[x][m];
  const bool outer = (k == geo.n_r - 1);
  T sl[3], su[3];
  if (outer) {
    const T l[3] = {J.st * J.cp, J.st * J.sp, J.ct};
    Acc<T> q;
#pragma unroll
    for (int x = 0; x < 3; ++x)
#pragma unroll
      for (int y = 0; y < 3; ++y) q.fma_(gi[x][y] * l[x], l[y]);
    const T iq = S<T>::c(1.0) / sqrt_s(q.get());
#pragma unroll
    for (int x = 0; x < 3; ++x) sl[x] = l[x] * iq;
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      Acc<T> acc;
#pragma unroll
      for (int y = 0; y < 3; ++y) acc.fma_(gi[x][y], sl[y]);
      su[x] = acc.get();
    }
  }
#pragma unroll 1
  for (int s = 0; s < 10; ++s) {
    T Dd[3], DPh[3][3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const long long base = (long long)m * nv * P + p;
      const T dg = Store<T, kInt<T>>::ld(D, base + (long long)s * P);
      const T dpi = Store<T, kInt<T>>::ld(D, base + (long long)(10 + s) * P);
      Dd[m] = dg - dpi;
#pragma unroll
      for (int x = 0; x < 3; ++x) DPh[x][m] = Store<T, kInt<T>>::ld(D, base + (long long)(20 + 10 * x + s) * P);
    }
    Acc<T> aPi;
    aPi.add(ldA<T, kInt<T>>(src, P, p, s));
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      aPi.fma_(-b[m], Dd[m]);
#pragma unroll
      for (int x = 0; x < 3; ++x) aPi.fma_(-G[x][m], DPh[x][m]);
    }
    T rPi = aPi.get();
    T rPh[3];
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      Acc<T> a;
      a.add(ldA<T, kInt<T>>(src, P, p, 10 + 10 * x + s));
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        a.fma_(b[m], DPh[x][m]);
        a.fma_(aJ[x][m], Dd[m]);
      }
      rPh[x] = a.get();
    }
    if (outer) {
      const T rg = ldA<T, FO>(out, P, p, s);
      Acc<T> sd;
#pragma unroll
      for (int x = 0; x < 3; ++x) sd.fma_(su[x], rPh[x]);
      const T wplus = rPi + sd.get();
      const T w2 = half * (wplus - rg);
      rPi = half * (rg + wplus);
#pragma unroll
      for (int x = 0; x < 3; ++x) rPh[x] = sl[x] * w2;
    }
    stA<T, FO>(out, P, p, 10 + s, rPi);
#pragma unroll
    for (int x = 0; x < 3; ++x) stA<T, FO>(out, P, p, 20 + 10 * x + s, rPh[x]);
  }
}

// Gauge fields of 54/58-field states (App. A.1; eq. gauge with H_a a field
// of the state): H_a from fields 50..53 into the gauge buffer, d_i H_a from
// their spherical derivatives by the chain rule (eq. dvdx), and for 58
// fields d_t H_a = G_a (fields 54..57) as rows 12..15 of dH.  The gauge
// fields' right-hand sides: d_t H_a = G_a for 58 fields (0 for 54) and
// d_t G_a = 0; the outer boundary condition leaves them alone.
template <class T, bool FU, bool FO>
__global__ void __launch_bounds__(128) k_gauge_rhs(const double* __restrict__ u, const double* __restrict__ D,
                                                   double* __restrict__ H, double* __restrict__ dH,
                                                   double* __restrict__ out, Geo geo) {
  const long long P = geo.P;
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= P) return;
  const int k = (int)(p % geo.n_r);
  const int i = (int)((p / geo.n_r) % geo.N);
  const int jj = (int)((p / ((long long)geo.n_r * geo.N)) % geo.J);
  const int nv = geo.nv;
  const Jac<T> J = jacobian<T>(geo, k, i, jj);
  const T zero = S<T>::c(0.0);
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    stA<T, kInt<T>>(H, P, p, b, ldA<T, FU>(u, P, p, 50 + b));
    T ds[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) ds[m] = Store<T, kInt<T>>::ld(D, ((long long)m * nv + 50 + b) * P + p);
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      Acc<T> a;
#pragma unroll
      for (int m = 0; m < 3; ++m) a.fma_(J.j[x][m], ds[m]);
      stA<T, kInt<T>>(dH, P, p, 4 * x + b, a.get());
    }
    if (nv == 58) {
      const T Gb = ldA<T, FU>(u, P, p, 54 + b);
      stA<T, kInt<T>>(dH, P, p, 12 + b, Gb);
      stA<T, FO>(out, P, p, 50 + b, Gb);
      stA<T, FO>(out, P, p, 54 + b, zero);
    } else {
      stA<T, FO>(out, P, p, 50 + b, zero);
    }
  }
}

// stage = 0: all three kernels; 1: sources with Christoffels; 2: quadratic
// sources; 3: principal parts + boundary.  u_pairs: the state is a pair-stored
// internal buffer (the stage states of the mixed path); out_pairs: the output
// is the internal rhs buffer (else an FP64 caller array); on the mixed path
// both are pairs (a step) or neither (cffyn_rhs).
int pw_rhs_part(const cffyn_shell* sh, const double* u, const double* D, double* out, int stage,
                bool u_pairs, bool out_pairs, cudaStream_t st) {
  Geo g = geo_of(sh);
  const unsigned nb = blocks_for(g.P, 128), nbr = blocks_for(g.P, kRhsBlock);
  const bool mixed = sh->d.precision == CFFYN_MIXED;
  if (mixed && u_pairs != out_pairs) {
    set_error("internal: right-hand side storage (state %d, output %d) not instantiated", (int)u_pairs,
              (int)out_pairs);
    return CFFYN_EINVAL;
  }
  if (stage == 0 || stage == 1) {
    const int dtH = sh->nv == 58;
    if (sh->ng > 0) {
      if (!mixed)
        k_gauge_rhs<double, false, false><<<nb, 128, 0, st>>>(u, D, sh->H, sh->dH, out, g);
      else if (u_pairs)
        k_gauge_rhs<ff, true, true><<<nb, 128, 0, st>>>(u, D, sh->H, sh->dH, out, g);
      else
        k_gauge_rhs<ff, false, false><<<nb, 128, 0, st>>>(u, D, sh->H, sh->dH, out, g);
      count_launch();
    }
    if (!mixed)
      k_rhs_gamma<double, false, false><<<nbr, kRhsBlock, 0, st>>>(u, sh->H, sh->dH, sh->Rsrc, out, g, dtH);
    else if (u_pairs)
      k_rhs_gamma<ff, true, true><<<nbr, kRhsBlock, 0, st>>>(u, sh->H, sh->dH, sh->Rsrc, out, g, dtH);
    else
      k_rhs_gamma<ff, false, false><<<nbr, kRhsBlock, 0, st>>>(u, sh->H, sh->dH, sh->Rsrc, out, g, dtH);
    count_launch();
  }
  if (stage == 0 || stage == 2) {
    if (!mixed)
      k_rhs_quad<double, false><<<nbr, kRhsBlock, 0, st>>>(u, sh->Rsrc, g);
    else if (u_pairs)
      k_rhs_quad<ff, true><<<nbr, kRhsBlock, 0, st>>>(u, sh->Rsrc, g);
    else
      k_rhs_quad<ff, false><<<nbr, kRhsBlock, 0, st>>>(u, sh->Rsrc, g);
    count_launch();
  }
  if (stage == 0 || stage == 3) {
    if (!mixed)
      k_rhs_pp<double, false><<<nb, 128, 0, st>>>(D, sh->Rsrc, out, g);
    else if (out_pairs)
      k_rhs_pp<ff, true><<<nb, 128, 0, st>>>(D, sh->Rsrc, out, g);
    else
      k_rhs_pp<ff, false><<<nb, 128, 0, st>>>(D, sh->Rsrc, out, g);
    count_launch();
  }
  CF_CUDA(cudaGetLastError());
  return CFFYN_OK;
}

int pw_rhs(const cffyn_shell* sh, const double* u, const double* D, double* out, cudaStream_t st) {
  return pw_rhs_part(sh, u, D, out, 0, false, false, st);
}

}  // namespace cffyn
