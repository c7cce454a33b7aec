// Pointwise kernels of the hot path, templated on the arithmetic type
// (double for the FP64 path, ff = FP32 pair for the mixed path):
//
//   k_rhs          Cartesian derivatives by the chain rule (eq. dvdx), the
//                  first-order GHG right-hand side (App. A.1 eqs. gdot, Phidot,
//                  Pidot, dependent quantities from eqs. normal, abgfromgab,
//                  Gamma) and the freeze-incoming boundary condition on the
//                  outermost sphere (App. A.2, B = E^-1 Z E).
//   k_decompose    Cartesian tensor groups -> spin-weighted components
//                  (Sec. 3.4, eq. tensorexpansion) written as real multiples of
//                  the triad components: every tensor is first rotated to the
//                  real orthonormal triad (r, theta, phi) of eq. tetrad, then
//                  combined with constant coefficients into the m / mbar
//                  contractions (m = (theta + i phi)/sqrt 2).  A component with
//                  p legs on m and q legs on mbar has spin p - q.
//   k_reconstruct  the inverse map, fused with the RK4 stage update (Sec. 2.5)
//                  or writing the filtered tensor.
//   k_cart         spherical -> Cartesian derivatives (chain rule only).
//   k_gauge        H_a = -Gamma_a (eq. gauge).
//   k_constraints  sums of squares of C_iab = d_i g_ab - Phi_iab and
//                  C_a = H_a + Gamma_a (App. A.1).
#include <cstdio>
#include <type_traits>

#include "pw_common.cuh"

namespace cffyn {

// ---------------------------------------------------------------------------
// Spin decomposition in the real triad.  Rm rows: r, theta, phi.

template <class T>
struct Triad {
  T R[3][3];
};

// rows e_r, e_theta, e_phi in Cartesian components at (theta_i, phi_jj),
// formed in T arithmetic (set-up of the triad table)
template <class T>
__device__ __forceinline__ Triad<T> triad_eval(const Geo& g, int i, int jj) {
  Triad<T> t;
  const T st = S<T>::c(g.sth[i]), ct = S<T>::c(g.cth[i]);
  const T sp = S<T>::c(g.sph[jj]), cp = S<T>::c(g.cph[jj]);
  t.R[0][0] = st * cp; t.R[0][1] = st * sp; t.R[0][2] = ct;
  t.R[1][0] = ct * cp; t.R[1][1] = ct * sp; t.R[1][2] = -st;
  t.R[2][0] = -sp;     t.R[2][1] = cp;      t.R[2][2] = S<T>::c(0.0);
  return t;
}

template <class T>
__global__ void k_triad_table(Geo g, double* tab) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.N * g.J) return;
  const int i = e % g.N, jj = e / g.N;
  const Triad<T> t = triad_eval<T>(g, i, jj);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) Store<T, !std::is_same<T, double>::value>::st(tab, (long long)e * 9 + 3 * a + b, t.R[a][b]);
}

template <class T>
__device__ __forceinline__ Triad<T> triad_at(const Geo& g, int i, int jj) {
  Triad<T> t;
  const long long o = ((long long)jj * g.N + i) * 9;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) t.R[a][b] = Store<T, !std::is_same<T, double>::value>::ld(g.triad, o + 3 * a + b);
  return t;
}

template <class T>
__device__ __forceinline__ void rot_vec(const Triad<T>& t, const T v[3], T o[3]) {
#pragma unroll
  for (int A = 0; A < 3; ++A) o[A] = t.R[A][0] * v[0] + t.R[A][1] * v[1] + t.R[A][2] * v[2];
}
template <class T>
__device__ __forceinline__ void unrot_vec(const Triad<T>& t, const T o[3], T v[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) v[a] = t.R[0][a] * o[0] + t.R[1][a] * o[1] + t.R[2][a] * o[2];
}
// general 3x3: O_AB = R_Aa R_Bb T_ab
template <class T>
__device__ __forceinline__ void rot_mat(const Triad<T>& t, const T Tm[3][3], T O[3][3]) {
  T X[3][3];
#pragma unroll
  for (int A = 0; A < 3; ++A)
#pragma unroll
    for (int b = 0; b < 3; ++b) X[A][b] = t.R[A][0] * Tm[0][b] + t.R[A][1] * Tm[1][b] + t.R[A][2] * Tm[2][b];
#pragma unroll
  for (int A = 0; A < 3; ++A)
#pragma unroll
    for (int B = 0; B < 3; ++B) O[A][B] = X[A][0] * t.R[B][0] + X[A][1] * t.R[B][1] + X[A][2] * t.R[B][2];
}
template <class T>
__device__ __forceinline__ void unrot_mat(const Triad<T>& t, const T O[3][3], T Tm[3][3]) {
  T X[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int B = 0; B < 3; ++B) X[a][B] = t.R[0][a] * O[0][B] + t.R[1][a] * O[1][B] + t.R[2][a] * O[2][B];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) Tm[a][b] = X[a][0] * t.R[0][b] + X[a][1] * t.R[1][b] + X[a][2] * t.R[2][b];
}

// symmetric 3x3 (only b <= c of Tm read, only B <= C of O written):
// O_BC = R_Bb R_Cc T_bc
template <class T>
__device__ __forceinline__ void rot_sym(const Triad<T>& t, const T Tm[3][3], T O[3][3]) {
  auto sym = [&](int i, int j) -> T { return i <= j ? Tm[i][j] : Tm[j][i]; };
  T X[3][3];  // X[B][c] = R_Bb T_bc
#pragma unroll
  for (int B = 0; B < 3; ++B)
#pragma unroll
    for (int c = 0; c < 3; ++c) X[B][c] = t.R[B][0] * sym(0, c) + t.R[B][1] * sym(1, c) + t.R[B][2] * sym(2, c);
#pragma unroll
  for (int B = 0; B < 3; ++B)
#pragma unroll
    for (int C = B; C < 3; ++C) O[B][C] = X[B][0] * t.R[C][0] + X[B][1] * t.R[C][1] + X[B][2] * t.R[C][2];
}
// inverse of rot_sym: T_bc = R_Bb R_Cc O_BC (B <= C read, b <= c written)
template <class T>
__device__ __forceinline__ void unrot_sym(const Triad<T>& t, const T O[3][3], T Tm[3][3]) {
  auto sym = [&](int i, int j) -> T { return i <= j ? O[i][j] : O[j][i]; };
  T X[3][3];  // X[b][C] = R_Bb O_BC
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int C = 0; C < 3; ++C) X[b][C] = t.R[0][b] * sym(0, C) + t.R[1][b] * sym(1, C) + t.R[2][b] * sym(2, C);
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int c = b; c < 3; ++c) Tm[b][c] = X[b][0] * t.R[0][c] + X[b][1] * t.R[1][c] + X[b][2] * t.R[2][c];
}
// R_Ab with A known only at run time, and R_Ab with b known only at run time
// (selects, so that the triad stays in registers)
template <class T>
__device__ __forceinline__ T triad_row_el(const Triad<T>& t, int A, int b) {
  return A == 0 ? t.R[0][b] : (A == 1 ? t.R[1][b] : t.R[2][b]);
}
template <class T>
__device__ __forceinline__ T triad_col_el(const Triad<T>& t, int A, int b) {
  return b == 0 ? t.R[A][0] : (b == 1 ? t.R[A][1] : t.R[A][2]);
}

// Per-thread scratch in shared memory, [slot][thread] for blocks of 128
// threads (consecutive threads, consecutive words): the rank-3 group keeps
// its intermediates there so that its loops over the legs stay rolled (fully
// unrolled, its double-float rotations overflow the instruction caches).
template <class T>
struct Scratch {
  T* s;
  __device__ __forceinline__ T& operator()(int v) const { return s[v * 128 + (int)threadIdx.x]; }
};
constexpr int kDecSlots = 26;  // Trot_a (3 x 6) | (P_rm, P_mm) of legs 1, 2 (2 x 4)
constexpr int kRecSlots = 18;  // Trot_A (3 x 6), each overwritten by its X_A

// Slot assignment: 16 real spin-0 slots, then (re, im) pairs of spin 1 from
// slot 16, of spin 2 from slot 38 and of spin 3 at slot 48; the numbers
// below are the slots written by k_decompose and read back by k_reconstruct.
#define SLOT_R0(n) (n)
#define SLOT_C1(q) (16 + 2 * (q))
#define SLOT_C2(q) (38 + 2 * (q))
#define SLOT_C3 48

template <class T, bool F = false>
__device__ __forceinline__ T ld(const double* a, long long P, long long p, int f) {
  return Store<T, F>::ld(a, (long long)f * P + p);
}
template <bool F = false, class T>
__device__ __forceinline__ void st(double* a, long long P, long long p, int f, T v) {
  Store<T, F>::st(a, (long long)f * P + p, v);
}
// internal buffers are pair-stored in the double-float path
template <class T> constexpr bool kIn = false;
template <> constexpr bool kIn<ff> = true;

// Tensor groups handled by one thread each (blockIdx.y), so that a thread
// holds at most the 18 components of Phi_ijk:
//   0: g_tt, Pi_tt   1: g_ti   2: Pi_ti   3: Phi_itt   4: g_ij   5: Pi_ij
//   6: Phi_itj       7: Phi_ijk
// and for 54/58-field states the gauge groups 8: H_a (fields 50..53) and
// 9: d_t H_a (54..57), each a scalar and a vector; group 8 + g writes the
// slots 50 + 4g: H_t and the radial component (spin 0), then the spin-1
// pair of the angular components.
constexpr int kGroups = 8;
constexpr int kMaxNv = 58;

template <class T, bool FI>
__device__ __forceinline__ void decompose_group(int grp, Scratch<T> sc, const double* __restrict__ in,
                                                double* __restrict__ out, long long P, long long p,
                                                const Triad<T>& t) {
  const T two = S<T>::c(2.0);
  switch (grp) {
    case 0:
      st<kIn<T>>(out, P, p, SLOT_R0(0), ld<T, FI>(in, P, p, SI(0, 0)));
      st<kIn<T>>(out, P, p, SLOT_R0(1), ld<T, FI>(in, P, p, 10 + SI(0, 0)));
      break;
    case 1:
    case 2:
    case 3: {
      const int gph = grp - 1;
      const int b0 = gph == 0 ? 1 : (gph == 1 ? 11 : 20);
      const int st_ = gph == 2 ? 10 : 1;
      T v[3], o[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) v[a] = ld<T, FI>(in, P, p, b0 + st_ * a);
      rot_vec(t, v, o);
      st<kIn<T>>(out, P, p, SLOT_R0(2 + gph), o[0]);
      st<kIn<T>>(out, P, p, SLOT_C1(gph), o[1]);
      st<kIn<T>>(out, P, p, SLOT_C1(gph) + 1, o[2]);
      break;
    }
    case 4:
    case 5: {
      const int gph = grp - 4;
      const int b0 = gph * 10;
      T Tm[3][3], O[3][3];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) Tm[a][b] = ld<T, FI>(in, P, p, b0 + SI(a + 1, b + 1));
      rot_mat(t, Tm, O);
      st<kIn<T>>(out, P, p, SLOT_R0(5 + 2 * gph), O[0][0]);
      st<kIn<T>>(out, P, p, SLOT_R0(6 + 2 * gph), O[1][1] + O[2][2]);
      st<kIn<T>>(out, P, p, SLOT_C1(3 + gph), O[0][1]);
      st<kIn<T>>(out, P, p, SLOT_C1(3 + gph) + 1, O[0][2]);
      st<kIn<T>>(out, P, p, SLOT_C2(gph), O[1][1] - O[2][2]);
      st<kIn<T>>(out, P, p, SLOT_C2(gph) + 1, two * O[1][2]);
      break;
    }
    case 6: {
      T Tm[3][3], O[3][3];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) Tm[a][b] = ld<T, FI>(in, P, p, 20 + 10 * a + SI(0, b + 1));
      rot_mat(t, Tm, O);
      st<kIn<T>>(out, P, p, SLOT_R0(9), O[0][0]);
      st<kIn<T>>(out, P, p, SLOT_C1(5), O[0][1]);
      st<kIn<T>>(out, P, p, SLOT_C1(5) + 1, O[0][2]);
      st<kIn<T>>(out, P, p, SLOT_C1(6), O[1][0]);
      st<kIn<T>>(out, P, p, SLOT_C1(6) + 1, O[2][0]);
      st<kIn<T>>(out, P, p, SLOT_C2(2), O[1][1] - O[2][2]);
      st<kIn<T>>(out, P, p, SLOT_C2(2) + 1, O[1][2] + O[2][1]);
      st<kIn<T>>(out, P, p, SLOT_R0(12), O[1][1] + O[2][2]);
      st<kIn<T>>(out, P, p, SLOT_R0(13), O[2][1] - O[1][2]);
      break;
    }
    case 8:
    case 9: {
      const int fb = 50 + 4 * (grp - 8);
      st<kIn<T>>(out, P, p, fb, ld<T, FI>(in, P, p, fb));
      T v[3], o[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) v[a] = ld<T, FI>(in, P, p, fb + 1 + a);
      rot_vec(t, v, o);
      st<kIn<T>>(out, P, p, fb + 1, o[0]);
      st<kIn<T>>(out, P, p, fb + 2, o[1]);
      st<kIn<T>>(out, P, p, fb + 3, o[2]);
      break;
    }
    default: {
      // T_ijk (leg i: fields 20 + 10 i; jk symmetric): the pair jk into the
      // triad for each i, then the leg i; slots 6 a + q hold Trot_a, q the
      // index of (rr, r1, r2, 11, 12, 22)
#pragma unroll 1
      for (int a = 0; a < 3; ++a) {
        T Tm[3][3], O[3][3];
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
          for (int c = b; c < 3; ++c) Tm[b][c] = ld<T, FI>(in, P, p, 20 + 10 * a + SI(b + 1, c + 1));
        rot_sym(t, Tm, O);
#pragma unroll
        for (int B = 0; B < 3; ++B)
#pragma unroll
          for (int C = B; C < 3; ++C) sc(6 * a + SI(B + 1, C + 1) - 4) = O[B][C];
      }
#pragma unroll 1
      for (int A = 0; A < 3; ++A) {
        const T r0 = triad_row_el(t, A, 0), r1 = triad_row_el(t, A, 1), r2 = triad_row_el(t, A, 2);
        T O[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) O[q] = r0 * sc(q) + r1 * sc(6 + q) + r2 * sc(12 + q);
        const T pr = O[0], pmb = O[3] + O[5], prm0 = O[1], prm1 = O[2], pmm0 = O[3] - O[5], pmm1 = two * O[4];
        if (A == 0) {
          st<kIn<T>>(out, P, p, SLOT_R0(10), pr);
          st<kIn<T>>(out, P, p, SLOT_R0(11), pmb);
          st<kIn<T>>(out, P, p, SLOT_C1(7), prm0);
          st<kIn<T>>(out, P, p, SLOT_C1(7) + 1, prm1);
          st<kIn<T>>(out, P, p, SLOT_C2(3), pmm0);
          st<kIn<T>>(out, P, p, SLOT_C2(3) + 1, pmm1);
        } else {
          st<kIn<T>>(out, P, p, SLOT_C1(8) + A - 1, pr);
          st<kIn<T>>(out, P, p, SLOT_C1(9) + A - 1, pmb);
          sc(18 + 4 * (A - 1)) = prm0;
          sc(19 + 4 * (A - 1)) = prm1;
          sc(20 + 4 * (A - 1)) = pmm0;
          sc(21 + 4 * (A - 1)) = pmm1;
        }
      }
      const T prm10 = sc(18), prm11 = sc(19), pmm10 = sc(20), pmm11 = sc(21);
      const T prm20 = sc(22), prm21 = sc(23), pmm20 = sc(24), pmm21 = sc(25);
      // (mbar; mm) = P_mm^theta - i P_mm^phi
      st<kIn<T>>(out, P, p, SLOT_C1(10), pmm10 + pmm21);
      st<kIn<T>>(out, P, p, SLOT_C1(10) + 1, pmm11 - pmm20);
      // (m; rm) = P_rm^theta + i P_rm^phi
      st<kIn<T>>(out, P, p, SLOT_C2(4), prm10 - prm21);
      st<kIn<T>>(out, P, p, SLOT_C2(4) + 1, prm11 + prm20);
      // (m; r mbar) = conj(P_rm^theta) + i conj(P_rm^phi)   (spin 0)
      st<kIn<T>>(out, P, p, SLOT_R0(14), prm10 + prm21);
      st<kIn<T>>(out, P, p, SLOT_R0(15), prm20 - prm11);
      // (m; mm) = P_mm^theta + i P_mm^phi
      st<kIn<T>>(out, P, p, SLOT_C3, pmm10 - pmm21);
      st<kIn<T>>(out, P, p, SLOT_C3 + 1, pmm11 + pmm20);
    }
  }
}

// Inverse of decompose_group: the group's spin slots -> its Cartesian
// components, each handed to emit(field, value).
template <class T, class Emit>
__device__ __forceinline__ void reconstruct_group(int grp, Scratch<T> sc, const double* __restrict__ sp, long long P,
                                                  long long p, const Triad<T>& t, Emit&& emit) {
  const T half = S<T>::c(0.5);
  switch (grp) {
    case 0:
      emit(SI(0, 0), ld<T, kIn<T>>(sp, P, p, SLOT_R0(0)));
      emit(10 + SI(0, 0), ld<T, kIn<T>>(sp, P, p, SLOT_R0(1)));
      break;
    case 1:
    case 2:
    case 3: {
      const int gph = grp - 1;
      const int b0 = gph == 0 ? 1 : (gph == 1 ? 11 : 20);
      const int st_ = gph == 2 ? 10 : 1;
      T o[3] = {ld<T, kIn<T>>(sp, P, p, SLOT_R0(2 + gph)), ld<T, kIn<T>>(sp, P, p, SLOT_C1(gph)),
                ld<T, kIn<T>>(sp, P, p, SLOT_C1(gph) + 1)};
      T v[3];
      unrot_vec(t, o, v);
#pragma unroll
      for (int a = 0; a < 3; ++a) emit(b0 + st_ * a, v[a]);
      break;
    }
    case 4:
    case 5: {
      const int gph = grp - 4;
      const int b0 = gph * 10;
      const T rr = ld<T, kIn<T>>(sp, P, p, SLOT_R0(5 + 2 * gph));
      const T mmb = ld<T, kIn<T>>(sp, P, p, SLOT_R0(6 + 2 * gph));
      const T rmr = ld<T, kIn<T>>(sp, P, p, SLOT_C1(3 + gph)), rmi = ld<T, kIn<T>>(sp, P, p, SLOT_C1(3 + gph) + 1);
      const T mmr = ld<T, kIn<T>>(sp, P, p, SLOT_C2(gph)), mmi = ld<T, kIn<T>>(sp, P, p, SLOT_C2(gph) + 1);
      T O[3][3], Tm[3][3];
      O[0][0] = rr;
      O[0][1] = O[1][0] = rmr;
      O[0][2] = O[2][0] = rmi;
      O[1][1] = half * (mmb + mmr);
      O[2][2] = half * (mmb - mmr);
      O[1][2] = O[2][1] = half * mmi;
      unrot_mat(t, O, Tm);
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = a; b < 3; ++b) emit(b0 + SI(a + 1, b + 1), Tm[a][b]);
      break;
    }
    case 6: {
      const T s9 = ld<T, kIn<T>>(sp, P, p, SLOT_R0(9));
      const T s12 = ld<T, kIn<T>>(sp, P, p, SLOT_R0(12)), s13 = ld<T, kIn<T>>(sp, P, p, SLOT_R0(13));
      const T s42 = ld<T, kIn<T>>(sp, P, p, SLOT_C2(2)), s43 = ld<T, kIn<T>>(sp, P, p, SLOT_C2(2) + 1);
      T O[3][3], Tm[3][3];
      O[0][0] = s9;
      O[0][1] = ld<T, kIn<T>>(sp, P, p, SLOT_C1(5));
      O[0][2] = ld<T, kIn<T>>(sp, P, p, SLOT_C1(5) + 1);
      O[1][0] = ld<T, kIn<T>>(sp, P, p, SLOT_C1(6));
      O[2][0] = ld<T, kIn<T>>(sp, P, p, SLOT_C1(6) + 1);
      O[1][1] = half * (s42 + s12);
      O[2][2] = half * (s12 - s42);
      O[1][2] = half * (s43 - s13);
      O[2][1] = half * (s43 + s13);
      unrot_mat(t, O, Tm);
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) emit(20 + 10 * a + SI(0, b + 1), Tm[a][b]);
      break;
    }
    case 8:
    case 9: {
      const int fb = 50 + 4 * (grp - 8);
      emit(fb, ld<T, kIn<T>>(sp, P, p, fb));
      T o[3] = {ld<T, kIn<T>>(sp, P, p, fb + 1), ld<T, kIn<T>>(sp, P, p, fb + 2),
                ld<T, kIn<T>>(sp, P, p, fb + 3)};
      T v[3];
      unrot_vec(t, o, v);
#pragma unroll
      for (int a = 0; a < 3; ++a) emit(fb + 1 + a, v[a]);
      break;
    }
    default: {
      T Pr[3], Pmb[3], Prm[3][2], Pmm[3][2];
      Pr[0] = ld<T, kIn<T>>(sp, P, p, SLOT_R0(10));
      Pmb[0] = ld<T, kIn<T>>(sp, P, p, SLOT_R0(11));
      Prm[0][0] = ld<T, kIn<T>>(sp, P, p, SLOT_C1(7));
      Prm[0][1] = ld<T, kIn<T>>(sp, P, p, SLOT_C1(7) + 1);
      Pmm[0][0] = ld<T, kIn<T>>(sp, P, p, SLOT_C2(3));
      Pmm[0][1] = ld<T, kIn<T>>(sp, P, p, SLOT_C2(3) + 1);
      Pr[1] = ld<T, kIn<T>>(sp, P, p, SLOT_C1(8));
      Pr[2] = ld<T, kIn<T>>(sp, P, p, SLOT_C1(8) + 1);
      Pmb[1] = ld<T, kIn<T>>(sp, P, p, SLOT_C1(9));
      Pmb[2] = ld<T, kIn<T>>(sp, P, p, SLOT_C1(9) + 1);
      {
        // X = (m; rm) = P^th + i P^ph, Y = (m; r mbar) = conj(P^th) + i conj(P^ph)
        const T xr = ld<T, kIn<T>>(sp, P, p, SLOT_C2(4)), xi = ld<T, kIn<T>>(sp, P, p, SLOT_C2(4) + 1);
        const T yr = ld<T, kIn<T>>(sp, P, p, SLOT_R0(14)), yi = ld<T, kIn<T>>(sp, P, p, SLOT_R0(15));
        Prm[1][0] = half * (xr + yr);
        Prm[1][1] = half * (xi - yi);
        Prm[2][0] = half * (xi + yi);
        Prm[2][1] = half * (yr - xr);
      }
      {
        // X = (m; mm) = P^th + i P^ph, Z = (mbar; mm) = P^th - i P^ph
        const T xr = ld<T, kIn<T>>(sp, P, p, SLOT_C3), xi = ld<T, kIn<T>>(sp, P, p, SLOT_C3 + 1);
        const T zr = ld<T, kIn<T>>(sp, P, p, SLOT_C1(10)), zi = ld<T, kIn<T>>(sp, P, p, SLOT_C1(10) + 1);
        Pmm[1][0] = half * (xr + zr);
        Pmm[1][1] = half * (xi + zi);
        Pmm[2][0] = half * (xi - zi);
        Pmm[2][1] = half * (zr - xr);
      }
      // slots 6 A + q: the pair part Trot_A of triad leg A (q: rr, r1, r2,
      // 11, 12, 22), then in its place X_A, the pair back in Cartesian
#pragma unroll
      for (int A = 0; A < 3; ++A) {
        sc(6 * A + 0) = Pr[A];
        sc(6 * A + 1) = Prm[A][0];
        sc(6 * A + 2) = Prm[A][1];
        sc(6 * A + 3) = half * (Pmb[A] + Pmm[A][0]);
        sc(6 * A + 4) = half * Pmm[A][1];
        sc(6 * A + 5) = half * (Pmb[A] - Pmm[A][0]);
      }
#pragma unroll 1
      for (int A = 0; A < 3; ++A) {
        T Trot[3][3], X[3][3];
#pragma unroll
        for (int B = 0; B < 3; ++B)
#pragma unroll
          for (int C = B; C < 3; ++C) Trot[B][C] = sc(6 * A + SI(B + 1, C + 1) - 4);
        unrot_sym(t, Trot, X);
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
          for (int c = b; c < 3; ++c) sc(6 * A + SI(b + 1, c + 1) - 4) = X[b][c];
      }
#pragma unroll 1
      for (int a = 0; a < 3; ++a) {
        const T r0 = triad_col_el(t, 0, a), r1 = triad_col_el(t, 1, a), r2 = triad_col_el(t, 2, a);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          const int f = 20 + 10 * a + 4 + q;  // SI(b + 1, c + 1) = 4 + q
          emit(f, r0 * sc(q) + r1 * sc(6 + q) + r2 * sc(12 + q));
        }
      }
    }
  }
}

// Tensor group of blockIdx.y, the groups with the most components first
// (7: 18, 6: 9, 4 and 5: 6, the gauge groups: 4, 1..3: 3, 0: 2), so that the
// light ones fill the last wave of a launch; ng gauge groups.
__device__ __forceinline__ int group_of(int y, int ng) {
  if (y < 4) return y == 0 ? 7 : (y == 1 ? 6 : (y == 2 ? 4 : 5));
  y -= 4;
  if (y < ng) return 8 + y;
  y -= ng;
  return y < 3 ? 1 + y : 0;
}

template <class T, bool FI>
__global__ void __launch_bounds__(128) k_decompose(const double* __restrict__ in, double* __restrict__ out,
                                                   Geo geo) {
  __shared__ T sm[kDecSlots * 128];
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= geo.P) return;
  const int i = (int)((p / geo.n_r) % geo.N);
  const int jj = (int)((p / ((long long)geo.n_r * geo.N)) % geo.J);
  const Triad<T> t = triad_at<T>(geo, i, jj);
  decompose_group<T, FI>(group_of((int)blockIdx.y, (geo.nv - 50) / 4), Scratch<T>{sm}, in, out, geo.P, p, t);
}

// Output fields of each tensor group (see kGroups).
__host__ __device__ constexpr bool in_group(int G, int f) {
  return G == 0 ? (f == 0 || f == 10)
       : G == 1 ? (f >= 1 && f <= 3)
       : G == 2 ? (f >= 11 && f <= 13)
       : G == 3 ? (f == 20 || f == 30 || f == 40)
       : G == 4 ? (f >= 4 && f <= 9)
       : G == 5 ? (f >= 14 && f <= 19)
       : G == 6 ? (f >= 20 && f < 50 && (f % 10) >= 1 && (f % 10) <= 3)
       : G == 7 ? (f >= 20 && f < 50 && (f % 10) >= 4)
       : G == 8 ? (f >= 50 && f < 54)
                : (f >= 54 && f < 58);
}

// mode: 0 = write filtered tensor to `dst`; 9 = the same from Cartesian
//       values in sp (component-wise filters);
//       1..4 = RK4 stage s (1-based) with filtered rhs k_s = reconstruct(sp);
//       5..8 = RK4 stage without filter: k_s read as Cartesian from sp.
// Stage updates: k_1: acc = k, U = u + dt/2 k; k_2: acc += 2k, U = u + dt/2 k;
// k_3: acc += 2k, U = u + dt k; k_4: u = u + dt/6 (acc + k) (classical RK4).
// The state sums are FP64 additions; the increments are formed in T.  On the
// mixed path uf holds the step's initial state as pairs: stages 1-3 read it
// as the base of U, the last stage (and mode 0) write the new state into it.
// One
// instance per tensor group G: the group's Cartesian k_s is formed into
// registers first, then the state words of all its fields are loaded at once
// and updated.
template <class T, bool FD, int G, int KIND>
__device__ __forceinline__ void reconstruct_update(Scratch<T> sc, const double* __restrict__ sp,
                                                   double* __restrict__ dst, const Geo& geo, int mode,
                                                   double* __restrict__ u, double* __restrict__ U,
                                                   double* __restrict__ kacc, double* __restrict__ uf, double dt,
                                                   long long p, bool& bad) {
  const long long P = geo.P;
  using SI_ = Store<T, kIn<T>>;
  constexpr bool kPair = kIn<T>;  // mixed path: the step's initial state also as pairs in uf
  const int stage = KIND == 0 ? 0 : (mode - 1) % 4;  // 0..3 for modes 1..8; KIND 2 is stage 3
  const T cU = S<T>::c(stage == 2 ? dt : 0.5 * dt);
  const T sixth = S<T>::c(dt / 6.0);
  // the update of field f with its right-hand side k, as each k is formed
  auto update = [&](int f, T k) {
    const long long o = (long long)f * P + p;
    if (KIND == 0) {
      Store<T, FD>::st(dst, o, k);
      if (kPair && uf) SI_::st(uf, o, k);
    } else if (KIND == 1) {
      bad |= !finite_s(k);
      // stage state: FP64 sum on the FP64 path, double-float on the mixed path
      const T base = kPair ? SI_::ld(uf, o) : S<T>::c(u[o]);
      SI_::st(kacc, o, stage == 0 ? k : SI_::ld(kacc, o) + (k + k));
      SI_::st(U, o, base + cU * k);
    } else {
      bad |= !finite_s(k);
      const double un = u[o] + S<T>::to_double(sixth * (SI_::ld(kacc, o) + k));
      u[o] = un;
      if (kPair && uf) SI_::st(uf, o, S<T>::c(un));
    }
  };
  if (mode <= 4) {
    const int i = (int)((p / geo.n_r) % geo.N);
    const int jj = (int)((p / ((long long)geo.n_r * geo.N)) % geo.J);
    const Triad<T> t = triad_at<T>(geo, i, jj);
    reconstruct_group<T>(G, sc, sp, P, p, t, update);
  } else {
#pragma unroll
    for (int f = 0; f < kMaxNv; ++f)
      if (in_group(G, f)) update(f, ld<T, kIn<T>>(sp, P, p, f));
  }
}

// Latency-bound (a few dependent loads and stores per field): nine blocks
// per SM, i.e. at most 56 registers and 18 KB of slots per block (with 80
// registers and 36 slots, six blocks: 0.423 ms per step on the 33 x 48 x 96
// shell; eight blocks, 64 registers: 0.340; nine: 0.335, same results).
template <class T, bool FD, int KIND>
__global__ void __launch_bounds__(128, 9) k_reconstruct(const double* __restrict__ sp, double* __restrict__ dst,
                                                     Geo geo, int mode, double* __restrict__ u,
                                                     double* __restrict__ U, double* __restrict__ kacc,
                                                     double* __restrict__ uf, double dt,
                                                     int* __restrict__ flag) {
  __shared__ T sm[kRecSlots * 128];
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= geo.P) return;
  bool bad = false;
  const Scratch<T> sc{sm};
#define CFFYN_RECON(G) reconstruct_update<T, FD, G, KIND>(sc, sp, dst, geo, mode, u, U, kacc, uf, dt, p, bad)
  switch (group_of((int)blockIdx.y, (geo.nv - 50) / 4)) {
    case 0: CFFYN_RECON(0); break;
    case 1: CFFYN_RECON(1); break;
    case 2: CFFYN_RECON(2); break;
    case 3: CFFYN_RECON(3); break;
    case 4: CFFYN_RECON(4); break;
    case 5: CFFYN_RECON(5); break;
    case 6: CFFYN_RECON(6); break;
    case 7: CFFYN_RECON(7); break;
    case 8: CFFYN_RECON(8); break;
    default: CFFYN_RECON(9); break;
  }
#undef CFFYN_RECON
  if (bad) atomicOr(flag, 1);
}

// Spherical -> Cartesian derivatives: D[3][nf][P] -> out[3][nf][P] (FP64
// arithmetic; D and out in the given storages).  Setup and API paths only.
// One thread per point: the Jacobian (FP64 divisions) is formed once and
// applied to every field, whose values are coalesced across the threads.
// status (may be NULL): a status word of the operator launches that produced
// D; if it is non-zero (a timed-out wait) every output value is a NaN.
template <bool FI, bool FO>
__global__ void k_cart(const double* __restrict__ D, double* __restrict__ out, int nf, Geo geo,
                       const int* __restrict__ status) {
  const long long P = geo.P;
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= P) return;
  if (status && *status) {
    const double qnan = __longlong_as_double(0x7ff8000000000000ll);
    for (int e = 0; e < 3 * nf; ++e) Store<double, FO>::st(out, (long long)e * P + p, qnan);
    return;
  }
  const int k = (int)(p % geo.n_r);
  const int i = (int)((p / geo.n_r) % geo.N);
  const int jj = (int)((p / ((long long)geo.n_r * geo.N)) % geo.J);
  const Jac<double> J = jacobian<double>(geo, k, i, jj);
#pragma unroll 2
  for (int mu = 0; mu < nf; ++mu) {
    const double dr = Store<double, FI>::ld(D, (long long)mu * P + p);
    const double dt = Store<double, FI>::ld(D, ((long long)nf + mu) * P + p);
    const double dp = Store<double, FI>::ld(D, ((long long)2 * nf + mu) * P + p);
#pragma unroll
    for (int x = 0; x < 3; ++x)
      Store<double, FO>::st(out, ((long long)x * nf + mu) * P + p,
                            J.j[x][0] * dr + J.j[x][1] * dt + J.j[x][2] * dp);
  }
}

// H_a = -Gamma_a(u), pointwise (FP64); H in storage FO
template <bool FO>
__global__ void k_gauge(const double* __restrict__ u, double* __restrict__ H, Geo geo) {
  const long long P = geo.P;
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= P) return;
  double g[10], Pi[10], Ph[3][10];
#pragma unroll
  for (int s = 0; s < 10; ++s) {
    g[s] = u[(long long)s * P + p];
    Pi[s] = u[(long long)(10 + s) * P + p];
#pragma unroll
    for (int a = 0; a < 3; ++a) Ph[a][s] = u[(long long)(20 + 10 * a + s) * P + p];
  }
  Metric<double> M;
  metric_from(g, M);
  double dg4[4][10], Gam[4][10], Gc[4];
  christoffel(M, Pi, Ph, dg4, Gam, Gc);
#pragma unroll
  for (int a = 0; a < 4; ++a) Store<double, FO>::st(H, (long long)a * P + p, -Gc[a]);
}

// FP64 array -> storage FO (copies of caller arrays into internal buffers)
template <bool FO>
__global__ void k_to_store(const double* __restrict__ in, double* __restrict__ out, long long n) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t < n) Store<double, FO>::st(out, t, in[t]);
}

// sum over points of C_iab^2 (30 components) and C_a^2 (4) -> red[0], red[1]
template <bool FH>
__global__ void k_constraints(const double* __restrict__ u, const double* __restrict__ dcart /*[3][10][P]*/,
                              const double* __restrict__ H, Geo geo, double* red) {
  const long long P = geo.P;
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double s3 = 0.0, s1 = 0.0;
  if (p < P) {
    double g[10], Pi[10], Ph[3][10];
#pragma unroll
    for (int s = 0; s < 10; ++s) {
      g[s] = u[(long long)s * P + p];
      Pi[s] = u[(long long)(10 + s) * P + p];
#pragma unroll
      for (int a = 0; a < 3; ++a) Ph[a][s] = u[(long long)(20 + 10 * a + s) * P + p];
    }
#pragma unroll
    for (int x = 0; x < 3; ++x)
#pragma unroll
      for (int s = 0; s < 10; ++s) {
        double c = dcart[((long long)x * 10 + s) * P + p] - Ph[x][s];
        s3 += c * c;
      }
    Metric<double> M;
    metric_from(g, M);
    double dg4[4][10], Gam[4][10], Gc[4];
    christoffel(M, Pi, Ph, dg4, Gam, Gc);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      double c = Store<double, FH>::ld(H, (long long)a * P + p) + Gc[a];
      s1 += c * c;
    }
  }
  __shared__ double r3[128], r1[128];
  r3[threadIdx.x] = s3;
  r1[threadIdx.x] = s1;
  __syncthreads();
  for (int w = 64; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      r3[threadIdx.x] += r3[threadIdx.x + w];
      r1[threadIdx.x] += r1[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    atomicAdd(red, r3[0]);
    atomicAdd(red + 1, r1[0]);
  }
}

// ---------------------------------------------------------------------------
// Host launchers

// in_pairs: the input is a pair-stored internal buffer (else an FP64 array)
int pw_decompose(const cffyn_shell* sh, const double* in, double* out, bool in_pairs, cudaStream_t st) {
  Geo g = geo_of(sh);
  const dim3 grid(blocks_for(g.P, 128), kGroups + sh->ng);
  if (sh->d.precision != CFFYN_MIXED)
    k_decompose<double, false><<<grid, 128, 0, st>>>(in, out, g);
  else if (in_pairs)
    k_decompose<ff, true><<<grid, 128, 0, st>>>(in, out, g);
  else
    k_decompose<ff, false><<<grid, 128, 0, st>>>(in, out, g);
  count_launch();
  CF_CUDA(cudaGetLastError());
  return CFFYN_OK;
}

// dst (mode 0) is an FP64 array; uf (mixed path): the step's initial state as
// pairs, read by stages 1-3 and written by the last stage and by mode 0
int pw_reconstruct(const cffyn_shell* sh, const double* sp, double* dst, int mode, double* u, double* U,
                   double* kacc, double* uf, double dt, int* flag, cudaStream_t st) {
  Geo g = geo_of(sh);
  const dim3 grid(blocks_for(g.P, 128), kGroups + sh->ng);
  // kernel instance by stage kind: 0 filtered result, 1 stages 1-3, 2 last stage
  const int kind = (mode == 0 || mode == 9) ? 0 : ((mode - 1) % 4 == 3 ? 2 : 1);
  if (sh->d.precision == CFFYN_MIXED) {
    if (kind == 0)
      k_reconstruct<ff, false, 0><<<grid, 128, 0, st>>>(sp, dst, g, mode, u, U, kacc, uf, dt, flag);
    else if (kind == 1)
      k_reconstruct<ff, false, 1><<<grid, 128, 0, st>>>(sp, dst, g, mode, u, U, kacc, uf, dt, flag);
    else
      k_reconstruct<ff, false, 2><<<grid, 128, 0, st>>>(sp, dst, g, mode, u, U, kacc, uf, dt, flag);
  } else {
    if (kind == 0)
      k_reconstruct<double, false, 0><<<grid, 128, 0, st>>>(sp, dst, g, mode, u, U, kacc, nullptr, dt, flag);
    else if (kind == 1)
      k_reconstruct<double, false, 1><<<grid, 128, 0, st>>>(sp, dst, g, mode, u, U, kacc, nullptr, dt, flag);
    else
      k_reconstruct<double, false, 2><<<grid, 128, 0, st>>>(sp, dst, g, mode, u, U, kacc, nullptr, dt, flag);
  }
  count_launch();
  CF_CUDA(cudaGetLastError());
  return CFFYN_OK;
}

// D: internal storage; out_pairs: out is an internal buffer; status: see k_cart
int pw_cart_status(const cffyn_shell* sh, const double* D, double* out, int nf, bool out_pairs,
                   const int* status, cudaStream_t st) {
  Geo g = geo_of(sh);
  const bool in_pairs = sh->d.precision == CFFYN_MIXED;
  const unsigned nb = blocks_for(g.P, 256);
  if (in_pairs && out_pairs)
    k_cart<true, true><<<nb, 256, 0, st>>>(D, out, nf, g, status);
  else if (in_pairs)
    k_cart<true, false><<<nb, 256, 0, st>>>(D, out, nf, g, status);
  else
    k_cart<false, false><<<nb, 256, 0, st>>>(D, out, nf, g, status);
  count_launch();
  CF_CUDA(cudaGetLastError());
  return CFFYN_OK;
}

int pw_cart(const cffyn_shell* sh, const double* D, double* out, int nf, bool out_pairs, cudaStream_t st) {
  return pw_cart_status(sh, D, out, nf, out_pairs, nullptr, st);
}

// FP64 spherical derivatives D (not internal storage) -> FP64 Cartesian out,
// on either path (the FFT derivative path writes FP64 into the workspace)
int pw_cart_fp64(const cffyn_shell* sh, const double* D, double* out, int nf, cudaStream_t st) {
  Geo g = geo_of(sh);
  k_cart<false, false><<<blocks_for(g.P, 256), 256, 0, st>>>(D, out, nf, g, nullptr);
  count_launch();
  CF_CUDA(cudaGetLastError());
  return CFFYN_OK;
}

// Table of the real triad rows at every (theta_i, phi_j) (set-up).
int pw_triad_table(const cffyn_shell* sh) {
  Geo g = geo_of(sh);
  const unsigned nb = blocks_for((long long)g.N * g.J, 128);
  if (sh->d.precision == CFFYN_MIXED)
    k_triad_table<ff><<<nb, 128>>>(g, sh->triad);
  else
    k_triad_table<double><<<nb, 128>>>(g, sh->triad);
  CF_CUDA(cudaGetLastError());
  return CFFYN_OK;
}

// H (internal storage) = -Gamma(u)
int pw_gauge(const cffyn_shell* sh, const double* u, double* H, cudaStream_t st) {
  Geo g = geo_of(sh);
  if (sh->d.precision == CFFYN_MIXED)
    k_gauge<true><<<blocks_for(g.P, 128), 128, 0, st>>>(u, H, g);
  else
    k_gauge<false><<<blocks_for(g.P, 128), 128, 0, st>>>(u, H, g);
  count_launch();
  CF_CUDA(cudaGetLastError());
  return CFFYN_OK;
}

// 54/58-field states: H_a = -Gamma_a(u) into fields 50..53 of u (FP64) and
// d_t H_a (54..57) set to zero
int pw_gauge_into_state(const cffyn_shell* sh, double* u, cudaStream_t st) {
  Geo g = geo_of(sh);
  k_gauge<false><<<blocks_for(g.P, 128), 128, 0, st>>>(u, u + (size_t)50 * g.P, g);
  count_launch();
  CF_CUDA(cudaGetLastError());
  if (sh->nv == 58) CF_CUDA(cudaMemsetAsync(u + (size_t)54 * g.P, 0, (size_t)4 * g.P * sizeof(double), st));
  return CFFYN_OK;
}

// FP64 caller array -> internal storage
int pw_to_internal(const cffyn_shell* sh, const double* in, double* out, long long n, cudaStream_t st) {
  if (sh->d.precision == CFFYN_MIXED)
    k_to_store<true><<<blocks_for(n, 256), 256, 0, st>>>(in, out, n);
  else
    k_to_store<false><<<blocks_for(n, 256), 256, 0, st>>>(in, out, n);
  count_launch();
  CF_CUDA(cudaGetLastError());
  return CFFYN_OK;
}

// h_internal: H is the library's gauge buffer (internal storage), else FP64
// (fields 50..53 of a 54/58-field state)
int pw_constraints(const cffyn_shell* sh, const double* u, const double* dcart, const double* H, bool h_internal,
                   double* red, cudaStream_t st) {
  Geo g = geo_of(sh);
  if (sh->d.precision == CFFYN_MIXED && h_internal)
    k_constraints<true><<<blocks_for(g.P, 128), 128, 0, st>>>(u, dcart, H, g, red);
  else
    k_constraints<false><<<blocks_for(g.P, 128), 128, 0, st>>>(u, dcart, H, g, red);
  count_launch();
  CF_CUDA(cudaGetLastError());
  return CFFYN_OK;
}

}  // namespace cffyn
