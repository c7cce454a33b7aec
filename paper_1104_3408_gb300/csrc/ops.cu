// Dense operator applications of the hot path: every derivative (paper Sec.
// 2.4, eqs. D1, D2, D3, with the theta double cover of Sec. 2.1) and every
// matrix of the Yn filter (Sec. 3.5: phi DFT of eq. forwardF, projection of
// eq. FasPfQ, inverse DFT of eq. backwardF) is a product
//     Out[:, c] = W (P x K) * In[:, c]
// of a small operator W with many columns c.  Each column has its own gather
// of K input rows (two segments, the second optionally reversed and signed:
// the theta double cover and the complex spin projection) and its own scatter
// of P output rows (two segments).  No transposes are materialised.
//
// Two arithmetic cores share the tiling and the gathers:
//   FP64   plain double FMA on CUDA cores (the reference path);
//   MIXED  split-precision products on the tensor cores: W and each input
//          column are written as 47-bit fixed-point integers relative to a
//          per-row / per-column power of two and cut into six balanced 8-bit
//          digits held exactly in BF16; digit products i + j = d are summed by
//          mma.sync m16n8k16 in FP32, where they are exact integers (at most
//          6 * 96 * 2^14 < 2^24), and folded into a 64-bit integer with weight
//          256^(5-d); pairs with i + j > 5 are dropped (relative truncation
//          about 6 * 2^-48 of |W| |x| K).  The result is rebuilt as an FP64
//          number with integer operations only (this part's FP64 and
//          conversion pipes are narrow).
#include <algorithm>
#include <cstdio>

#include "common.cuh"
#include "scalar.cuh"

namespace cffyn {

// ---------------------------------------------------------------------------
// Column descriptors

struct ColDesc {
  long long in0, in1, out0, out1;  // base offsets of the two row segments
  int sgn1;                        // second input segment: 0 as is, 1 negated, 2 zero
  int valid;
  int fld;                         // field (or function) whose exponent the column uses
};

struct OpGeom {
  int K, K0, P, P0;     // rows of W's columns (K), split of the input gather (K0),
                        // rows of W (P), split of the output scatter (P0)
  int in_rs, out_rs;    // row strides of input / output
  int rev1;             // second input segment reversed (row k -> K-1-k+K0... see load)
  long long ncols;
};

// All operators used by the shell, as one tagged descriptor.
enum OpKind : int { OP_R = 0, OP_ROWS = 1, OP_THETA = 2, OP_PROJ0 = 3, OP_PROJC = 4 };

struct OpArgs {
  OpKind kind;
  OpGeom g;
  const double* in;
  double* out;
  // OP_ROWS
  int Q;
  long long in_bs, out_bs;
  // OP_THETA / projections
  int n_r, N, J, R, L;
  int m;                 // projection: azimuthal number (set per block from blockIdx)
  const int* slots;      // projection: list of slots (R0: functions; C: re-slots of pairs)
  int nslots;
  int batched_m;         // projection launched for all m = 0..L at once
  long long w_stride;    // FP64 operator stride between consecutive m
};

__device__ __forceinline__ ColDesc make_col(const OpArgs& a, long long c) {
  ColDesc d;
  d.valid = c < a.g.ncols;
  d.sgn1 = 0;
  if (!d.valid) c = 0;
  switch (a.kind) {
    case OP_R: {
      d.fld = (int)(c / ((long long)a.J * a.N));
      d.in0 = c * a.n_r;
      d.out0 = d.in0;
      d.in1 = d.out1 = 0;
      break;
    }
    case OP_ROWS: {
      long long b = c / a.Q, q = c - b * a.Q;
      d.fld = (int)b;
      d.in0 = b * a.in_bs + q;
      d.out0 = b * a.out_bs + q;
      d.in1 = d.out1 = 0;
      break;
    }
    case OP_THETA: {
      long long pb = c / a.n_r;
      int kr = (int)(c - pb * a.n_r);
      int half = a.J / 2;
      long long mu = pb / half;
      int jp = (int)(pb - mu * half);
      d.fld = (int)mu;
      d.in0 = ((mu * a.J + jp) * a.N) * a.n_r + kr;
      d.in1 = ((mu * a.J + jp + half) * a.N) * a.n_r + kr;
      d.out0 = d.in0;
      d.out1 = d.in1;
      break;
    }
    case OP_PROJ0: {
      // columns: (slot index, part, kr); parts: a (row m) and b (row L+m, m >= 1)
      int nparts = a.m == 0 ? 1 : 2;
      long long per = (long long)nparts * a.n_r;
      if (c >= per * a.nslots) { d.valid = 0; c = 0; }
      long long fi = c / per;
      int rem = (int)(c - fi * per);
      int part = rem / a.n_r, kr = rem - part * a.n_r;
      int f = a.slots[fi < a.nslots ? fi : 0];
      d.fld = f;
      int row = part == 0 ? a.m : a.L + a.m;
      d.in0 = (((long long)f * a.R + row) * a.N) * a.n_r + kr;
      d.out0 = d.in0;
      d.in1 = d.out1 = 0;
      break;
    }
    case OP_PROJC: {
      // columns: (pair, output part, kr); parts aR, aI, bR, bI (m >= 1) or aR, aI
      int nparts = a.m == 0 ? 2 : 4;
      long long per = (long long)nparts * a.n_r;
      if (c >= per * a.nslots) { d.valid = 0; c = 0; }
      long long pi = c / per;
      int rem = (int)(c - pi * per);
      int part = rem / a.n_r, kr = rem - part * a.n_r;
      int fre = a.slots[pi < a.nslots ? pi : 0], fim = fre + 1;
      d.fld = fre;
      int ra = a.m, rb = a.L + a.m;
      auto base = [&](int f, int row) {
        return (((long long)f * a.R + row) * a.N) * a.n_r + kr;
      };
      long long aR = base(fre, ra), aI = base(fim, ra);
      long long bR = a.m ? base(fre, rb) : aR, bI = a.m ? base(fim, rb) : aI;
      // at m = 0 the F_d half of the operator is zero: gather nothing there
      switch (part) {
        case 0: d.in0 = aR; d.in1 = bI; d.sgn1 = a.m ? 0 : 2; d.out0 = aR; break;
        case 1: d.in0 = aI; d.in1 = bR; d.sgn1 = a.m ? 1 : 2; d.out0 = aI; break;
        case 2: d.in0 = bR; d.in1 = aI; d.sgn1 = a.m ? 1 : 2; d.out0 = bR; break;
        default: d.in0 = bI; d.in1 = aR; d.sgn1 = a.m ? 0 : 2; d.out0 = bI; break;
      }
      d.out1 = 0;
      break;
    }
  }
  return d;
}

__device__ __forceinline__ double load_elem(const OpArgs& a, const ColDesc& d, int k) {
  if (!d.valid || k >= a.g.K) return 0.0;
  if (k < a.g.K0) return __ldg(a.in + d.in0 + (long long)k * a.g.in_rs);
  if (d.sgn1 == 2) return 0.0;
  int kk = a.g.rev1 ? (a.g.K - 1 - k) : (k - a.g.K0);
  const double v = __ldg(a.in + d.in1 + (long long)kk * a.g.in_rs);
  // sign flip on the bit pattern (no FP64 instruction)
  return __longlong_as_double(__double_as_longlong(v) ^ ((long long)d.sgn1 << 63));
}

// Raw 64-bit element of a column for the split-precision core: an FP64 word
// (FI = false) or a (hi, lo) float pair (FI = true), sign applied on the bits.
template <bool FI>
__device__ __forceinline__ long long load_raw(const OpArgs& a, const ColDesc& d, int k) {
  if (!d.valid || k >= a.g.K) return 0;
  const long long* in = reinterpret_cast<const long long*>(a.in);
  if (k < a.g.K0) return __ldg(in + d.in0 + (long long)k * a.g.in_rs);
  if (d.sgn1 == 2) return 0;
  int kk = a.g.rev1 ? (a.g.K - 1 - k) : (k - a.g.K0);
  const long long w = __ldg(in + d.in1 + (long long)kk * a.g.in_rs);
  const long long m = FI ? (long long)0x8000000080000000ull : (long long)0x8000000000000000ull;
  return d.sgn1 ? (w ^ m) : w;
}

__device__ __forceinline__ void store_elem(const OpArgs& a, const ColDesc& d, int p, double v) {
  if (!d.valid || p >= a.g.P) return;
  if (p < a.g.P0)
    a.out[d.out0 + (long long)p * a.g.out_rs] = v;
  else
    a.out[d.out1 + (long long)(p - a.g.P0) * a.g.out_rs] = v;
}

// ---------------------------------------------------------------------------
// FP64 core: CTA tile = PT rows x QT columns, whole K staged in shared memory.

constexpr int F64_QT = 32;
constexpr int F64_PT = 64;

__global__ void __launch_bounds__(256) k_op_fp64(OpArgs a, const double* __restrict__ W) {
  extern __shared__ double sm64[];
  if (a.batched_m) {
    a.m = blockIdx.z;
    W += (size_t)a.m * a.w_stride;
  }
  const int K = a.g.K, P = a.g.P;
  const int p0 = blockIdx.y * F64_PT;
  const int PT = min(F64_PT, P - p0);
  double* Ws = sm64;                 // PT x K
  double* Xs = sm64 + F64_PT * K;    // K x QT
  __shared__ ColDesc cols[F64_QT];
  const long long c0 = (long long)blockIdx.x * F64_QT;
  const int tid = threadIdx.x;
  if (tid < F64_QT) cols[tid] = make_col(a, c0 + tid);
  for (int e = tid; e < PT * K; e += 256) Ws[e] = W[(size_t)(p0 + e / K) * K + (e % K)];
  __syncthreads();
  const bool kfast = a.kind == OP_R;
  for (int e = tid; e < K * F64_QT; e += 256) {
    int k, c;
    if (kfast) { k = e % K; c = e / K; } else { c = e % F64_QT; k = e / F64_QT; }
    Xs[k * F64_QT + c] = load_elem(a, cols[c], k);
  }
  __syncthreads();
  const int tq = tid % F64_QT, tp = tid / F64_QT;  // 8 row groups
  double acc[F64_PT / 8];
#pragma unroll
  for (int r = 0; r < F64_PT / 8; ++r) acc[r] = 0.0;
  for (int k = 0; k < K; ++k) {
    double x = Xs[k * F64_QT + tq];
#pragma unroll
    for (int r = 0; r < F64_PT / 8; ++r) {
      int row = tp + 8 * r;
      if (row < PT) acc[r] = fma(Ws[row * K + k], x, acc[r]);
    }
  }
  if (kfast) {
    // transpose through shared memory so that stores run along p
    __syncthreads();
    double* Os = Xs;  // reuse: PT x QT
#pragma unroll
    for (int r = 0; r < F64_PT / 8; ++r) {
      int row = tp + 8 * r;
      if (row < PT) Os[row * F64_QT + tq] = acc[r];
    }
    __syncthreads();
    for (int e = tid; e < PT * F64_QT; e += 256) {
      int p = e % PT, c = e / PT;
      store_elem(a, cols[c], p0 + p, Os[p * F64_QT + c]);
    }
  } else {
#pragma unroll
    for (int r = 0; r < F64_PT / 8; ++r) {
      int row = tp + 8 * r;
      if (row < PT) store_elem(a, cols[tq], p0 + row, acc[r]);
    }
  }
}

// ---------------------------------------------------------------------------
// Split-precision core.

constexpr int OZ_QT = 32;        // columns per CTA (4 n-tiles of 8)
constexpr int OZ_NT = OZ_QT / 8;
constexpr int OZ_MAXK = 192;
constexpr int OZ_KCHUNK = 6;     // k-steps (of 16) per exact partial sum

__device__ __forceinline__ int exp_field(double x) {
  return (int)((__double_as_longlong(x) >> 52) & 0x7ff);
}

// frexp exponent + 1022 of a raw element (0 for zero): FP64 word, or the
// leading float of a pair (|hi + lo| < 2^frexp(hi) for a normalised pair)
template <bool FI>
__device__ __forceinline__ int raw_exp(long long w) {
  if (FI) {
    const int e = (int)(((unsigned int)w >> 23) & 0xff);
    return e ? e - 126 + 1022 : 0;
  }
  return (int)((w >> 52) & 0x7ff);
}

// round(x 2^(47-E)) for one float, integer operations only
__device__ __forceinline__ long long fixed47f(unsigned int u, int E) {
  const int e = (int)((u >> 23) & 0xff);
  if (e == 0) return 0;
  const long long M = (long long)((u & 0x7fffff) | 0x800000);
  const int sh = e - 103 - E;  // <= 23 because |x| < 2^E
  long long Z;
  if (sh >= 0) Z = M << sh;
  else if (sh > -26) Z = (M + (1ll << (-sh - 1))) >> (-sh);
  else Z = 0;
  return (u >> 31) ? -Z : Z;
}

// 47-bit fixed point Z = round(x 2^(47-E)) of x relative to 2^E (|x| < 2^E),
// integer operations only.
__device__ __forceinline__ long long fixed47(double x, int E) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff);
  long long Z = 0;
  if (e != 0) {
    const unsigned long long M = (b & 0x000fffffffffffffull) | 0x0010000000000000ull;
    const int sh = 1028 + E - e;  // >= 6 because |x| < 2^E
    if (sh < 54) Z = (long long)((M + (1ull << (sh - 1))) >> sh);
    if (b >> 63) Z = -Z;
  }
  return Z;
}

template <bool FI>
__device__ __forceinline__ long long raw_fixed47(long long w, int E) {
  if (FI) return fixed47f((unsigned int)w, E) + fixed47f((unsigned int)((unsigned long long)w >> 32), E);
  return fixed47(__longlong_as_double(w), E);
}

// Balanced base-256 digits of Z (|Z| <= 2^47): with Zb = Z + sum_{k<5} 128*256^k
// byte k of Zb is e_k + 128 for the five low digits and Zb >> 40 is the top
// digit.  Returned as BF16 bit patterns, slice 0 = most significant.
__device__ __forceinline__ void digits_bf16(long long Z, unsigned int out[kSlices]) {
  const long long Zb = Z + 0x8080808080ll;
  const unsigned int lo = (unsigned int)Zb;
  const int hi = (int)(Zb >> 32);
  // bf16(b - 128) for a byte b: exact small integer through the 1.5*2^23 trick
  auto bf = [](int b) -> unsigned int {
    return __float_as_uint(__int_as_float(0x4B400000 + b) - 12583040.0f) >> 16;
  };
  out[5] = bf((int)(lo & 255u));
  out[4] = bf((int)((lo >> 8) & 255u));
  out[3] = bf((int)((lo >> 16) & 255u));
  out[2] = bf((int)(lo >> 24));
  out[1] = bf(hi & 255);
  const int top = hi >> 8;  // arithmetic shift: the signed top digit
  out[0] = __float_as_uint(__int_as_float(0x4B400000 + top) - 12582912.0f) >> 16;
}

// FP32 value holding an exact integer |v| < 2^24 -> int, integer ops only.
__device__ __forceinline__ int f32_int_exact(float v) {
  const unsigned int u = __float_as_uint(v);
  const int e = (int)((u >> 23) & 0xff);
  const int m = (int)((u & 0x7fffff) | 0x800000);
  const int sh = 150 - e;
  int r = (sh < 32 && e != 0) ? (m >> sh) : 0;
  return (u >> 31) ? -r : r;
}

// T * 2^sc as a double (round to nearest), integer ops only.
__device__ __forceinline__ double i64_scaled_to_double(long long T, int sc) {
  if (T == 0) return 0.0;
  const unsigned long long s = T < 0 ? 0x8000000000000000ull : 0ull;
  unsigned long long v = T < 0 ? (unsigned long long)(-T) : (unsigned long long)T;
  const int nb = 64 - __clzll((long long)v);
  int ex = nb - 1 + sc;
  unsigned long long m;
  if (nb > 53) {
    const int sh = nb - 53;
    m = (v + (1ull << (sh - 1))) >> sh;
    if (m >> 53) {
      m >>= 1;
      ex += 1;
    }
  } else {
    m = v << (53 - nb);
  }
  if (ex + 1023 <= 0) return 0.0;
  const unsigned long long bits = s | ((unsigned long long)(ex + 1023) << 52) | (m & 0x000fffffffffffffull);
  return __longlong_as_double((long long)bits);
}

// Four 8x8 BF16 tiles from shared memory; lane l addresses row (l % 8) of tile
// (l / 8) and receives, per tile, the pair at row lane/4, columns 2*(lane%4).
__device__ __forceinline__ void ldmatrix_x4(unsigned int& r0, unsigned int& r1, unsigned int& r2,
                                            unsigned int& r3, const void* p) {
  const unsigned int a = (unsigned int)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(a));
}

// T * 2^sc as a (hi, lo) float pair packed in 64 bits: hi exact leading 24
// bits, lo the next 24 (truncated).
__device__ __forceinline__ long long i64_scaled_to_pair(long long T, int sc) {
  if (T == 0) return 0;
  const bool neg = T < 0;
  const unsigned long long v = neg ? (unsigned long long)(-T) : (unsigned long long)T;
  const int nb = 64 - __clzll((long long)v);
  float hi, lo = 0.0f;
  if (nb <= 24) {
    hi = u64_scaled_to_float(v, sc, neg);
  } else {
    const int sh = nb - 24;
    const unsigned long long hm = v >> sh;
    hi = u64_scaled_to_float(hm, sc + sh, neg);
    lo = u64_scaled_to_float(v - (hm << sh), sc, neg);
  }
  return (long long)(((unsigned long long)__float_as_uint(lo) << 32) | __float_as_uint(hi));
}

__device__ __forceinline__ void mma_bf16(float c[4], const uint4& a, unsigned int b0, unsigned int b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
}

// ---------------------------------------------------------------------------
// Slicing pass: per-field exponents and 16-byte digit records.
//
// exps[f] = max over the field of (frexp exponent + 1022), 0 for an all-zero
// field.  With pairing, slots f >= kPairedFrom form (re, im) pairs (f, f^1)
// that share one exponent (the projection of a complex function gathers
// both).  A record holds the six balanced digits (slice 0 first) of the
// 47-bit fixed point round(x 2^(47-E)), E = exps - 1022, as BF16 halves.

constexpr int kPairedFrom = 16;

template <bool FI>
__global__ void k_field_exp(const long long* __restrict__ in, long long len, int* __restrict__ exps) {
  const int f = blockIdx.y;
  const long long* x = in + (long long)f * len;
  int m = 0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len;
       e += (long long)gridDim.x * blockDim.x)
    m = max(m, raw_exp<FI>(__ldg(x + e)));
  m = (int)__reduce_max_sync(0xffffffffu, (unsigned)m);
  if ((threadIdx.x & 31) == 0 && m) atomicMax(exps + f, m);
}

template <bool FI>
__global__ void k_slice(const long long* __restrict__ in, long long len, long long n,
                        const int* __restrict__ exps, int pairing, uint4* __restrict__ rec) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int f = (int)(e / len);
  int ex = exps[f];
  if (pairing && f >= kPairedFrom) ex = max(ex, exps[f ^ 1]);
  unsigned int d[kSlices];
  digits_bf16(raw_fixed47<FI>(__ldg(in + e), ex - 1022), d);
  rec[e] = make_uint4(d[0] | (d[1] << 16), d[2] | (d[3] << 16), d[4] | (d[5] << 16), 0u);
}

// Digit record of one column element (zero record outside K or for the empty
// second segment; negation flips the sign bit of every BF16 digit).
__device__ __forceinline__ uint4 load_rec(const OpArgs& a, const uint4* __restrict__ rec, const ColDesc& d,
                                          int k) {
  if (!d.valid || k >= a.g.K) return make_uint4(0u, 0u, 0u, 0u);
  if (k < a.g.K0) return __ldg(rec + d.in0 + (long long)k * a.g.in_rs);
  if (d.sgn1 == 2) return make_uint4(0u, 0u, 0u, 0u);
  const int kk = a.g.rev1 ? (a.g.K - 1 - k) : (k - a.g.K0);
  uint4 r = __ldg(rec + d.in1 + (long long)kk * a.g.in_rs);
  if (d.sgn1) {
    r.x ^= 0x80008000u;
    r.y ^= 0x80008000u;
    r.z ^= 0x80008000u;
  }
  return r;
}

// CTA: one warp per m-tile of W (mtiles warps), OZ_QT columns.  The input is
// given as digit records (see k_slice); the prologue only copies them into
// the slice-major shared-memory tile.
template <bool FO>
__global__ void __launch_bounds__(384) k_op_rec(OpArgs a, SlicedOp W, const uint4* __restrict__ rec,
                                              const int* __restrict__ exps, int pairing) {
  extern __shared__ unsigned short smoz[];
  if (a.batched_m) {
    a.m = blockIdx.y;
    W.frag += (size_t)a.m * W.frag_stride;
    W.rowexp += (size_t)a.m * W.rowexp_stride;
  }
  const int K = a.g.K;
  const int ksteps = W.ksteps;
  const int KP = ksteps * 16 + 8;                    // row pitch (halfwords), odd multiple of 8
  unsigned short* Bs = smoz;                         // [kSlices][OZ_QT][KP]
  __shared__ ColDesc cols[OZ_QT];
  __shared__ int colE[OZ_QT];
  const long long c0 = (long long)blockIdx.x * OZ_QT;
  const int tid = threadIdx.x, nthr = blockDim.x;
  if (tid < OZ_QT) cols[tid] = make_col(a, c0 + tid);
  __syncthreads();
  const bool kfast = a.kind == OP_R;
  const int Kp = ksteps * 16;
  const int KH = Kp / 2;                 // k pairs per column
  const int KPW = KP / 2;                // row pitch in 32-bit words
  unsigned int* Bw = reinterpret_cast<unsigned int*>(Bs);
  const int nitems = KH * OZ_QT;
  if (tid < OZ_QT) {
    const int f = cols[tid].fld;
    int e = exps[f];
    if (pairing && f >= kPairedFrom) e = max(e, exps[f ^ 1]);
    colE[tid] = e - 1022;
  }
  // copy the digit records of the tile: two k values of one column per item
  for (int e = tid; e < nitems; e += nthr) {
    int kp, c;
    if (kfast) { kp = e % KH; c = e / KH; } else { c = e % OZ_QT; kp = e / OZ_QT; }
    const uint4 r0 = load_rec(a, rec, cols[c], 2 * kp);
    const uint4 r1 = load_rec(a, rec, cols[c], 2 * kp + 1);
    unsigned int* dst = Bw + (size_t)c * KPW + kp;
    const size_t sstride = (size_t)OZ_QT * KPW;
    dst[0] = __byte_perm(r0.x, r1.x, 0x5410);
    dst[sstride] = __byte_perm(r0.x, r1.x, 0x7632);
    dst[2 * sstride] = __byte_perm(r0.y, r1.y, 0x5410);
    dst[3 * sstride] = __byte_perm(r0.y, r1.y, 0x7632);
    dst[4 * sstride] = __byte_perm(r0.z, r1.z, 0x5410);
    dst[5 * sstride] = __byte_perm(r0.z, r1.z, 0x7632);
  }
  __syncthreads();

  const int warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, tg = lane & 3;
  const int mt = warp;
  if (mt >= W.mtiles) return;
  long long T[OZ_NT][4];
#pragma unroll
  for (int n = 0; n < OZ_NT; ++n)
#pragma unroll
    for (int q = 0; q < 4; ++q) T[n][q] = 0;

  // k-step outer: the six operator digit fragments A_i(ks) are loaded once per
  // k-step, each data slice B_j(ks) once per k-step, and every pair (i, j)
  // accumulates into the digit-sum accumulator d = i + j (exact FP32 integers
  // per K chunk, folded into T with weight 256^(5-d)).
  const unsigned short* Bl = Bs + (size_t)(((lane >> 4) * 8) + (lane & 7)) * KP + ((lane >> 3) & 1) * 8;
  const uint4* Am = W.frag + ((size_t)mt * ksteps) * 32 + lane;
  const size_t aslice = (size_t)W.mtiles * ksteps * 32;
  for (int kc = 0; kc < ksteps; kc += OZ_KCHUNK) {
    const int kend = min(ksteps, kc + OZ_KCHUNK);
    float acc[kSlices][OZ_NT][4];
#pragma unroll
    for (int d = 0; d < kSlices; ++d)
#pragma unroll
      for (int n = 0; n < OZ_NT; ++n)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[d][n][q] = 0.0f;
    for (int ks = kc; ks < kend; ++ks) {
      uint4 af[kSlices];
#pragma unroll
      for (int i = 0; i < kSlices; ++i) af[i] = __ldg(Am + i * aslice + (size_t)ks * 32);
#pragma unroll
      for (int j = 0; j < kSlices; ++j) {
        const unsigned short* Bj = Bl + (size_t)j * OZ_QT * KP + ks * 16;
#pragma unroll
        for (int n = 0; n < OZ_NT; n += 2) {
          unsigned int b00, b01, b10, b11;
          ldmatrix_x4(b00, b01, b10, b11, Bj + (size_t)n * 8 * KP);
#pragma unroll
          for (int i = 0; i < kSlices - j; ++i) {
            mma_bf16(acc[i + j][n], af[i], b00, b01);
            mma_bf16(acc[i + j][n + 1], af[i], b10, b11);
          }
        }
      }
    }
#pragma unroll
    for (int d = 0; d < kSlices; ++d)
#pragma unroll
      for (int n = 0; n < OZ_NT; ++n)
#pragma unroll
        for (int q = 0; q < 4; ++q)
          T[n][q] += ((long long)__float2int_rz(acc[d][n][q])) << (8 * (kSlices - 1 - d));
  }
  // epilogue: rows mt*16 + g (+8), columns n*8 + 2tg (+1)
  const int rowA = mt * 16 + g, rowB = rowA + 8;
  const int eA = W.rowexp[rowA], eB = W.rowexp[rowB];
#pragma unroll
  for (int n = 0; n < OZ_NT; ++n) {
    const int cA = n * 8 + 2 * tg, cB = cA + 1;
    const int sA = colE[cA], sB = colE[cB];
    auto put = [&](const ColDesc& d, int row, long long t, int sc) {
      const long long w = FO ? i64_scaled_to_pair(t, sc)
                             : __double_as_longlong(i64_scaled_to_double(t, sc));
      store_elem(a, d, row, __longlong_as_double(w));
    };
    put(cols[cA], rowA, T[n][0], eA + sA - 54);
    put(cols[cB], rowA, T[n][1], eA + sB - 54);
    put(cols[cA], rowB, T[n][2], eB + sA - 54);
    put(cols[cB], rowB, T[n][3], eB + sB - 54);
  }
}

// ---------------------------------------------------------------------------
// Host side

// Mixed path: the operator input must have been sliced by op_prepare into
// sh->rec / sh->exps (pairing as given there); outputs are pair-stored.
static int launch(const cffyn_shell* sh, const OpArgs& a, const double* W64, const SlicedOp* Ws,
                  dim3 extra, cudaStream_t st, int pairing = 0) {
  if (a.g.ncols <= 0) return CFFYN_OK;
  if (sh->d.precision == CFFYN_FP64 || Ws == nullptr) {
    unsigned gx = (unsigned)((a.g.ncols + F64_QT - 1) / F64_QT);
    unsigned gy = (unsigned)((a.g.P + F64_PT - 1) / F64_PT);
    size_t smem = (size_t)(F64_PT * a.g.K + a.g.K * F64_QT) * sizeof(double);
    k_op_fp64<<<dim3(gx, gy, extra.y), 256, smem, st>>>(a, W64);
    count_launch();
  } else {
    unsigned gx = (unsigned)((a.g.ncols + OZ_QT - 1) / OZ_QT);
    int KP = Ws->ksteps * 16 + 8;
    size_t smem = (size_t)kSlices * OZ_QT * KP * sizeof(unsigned short);
    int threads = Ws->mtiles * 32;  // one warp per m-tile
    k_op_rec<true><<<dim3(gx, extra.y), threads, smem, st>>>(a, *Ws, reinterpret_cast<const uint4*>(sh->rec),
                                                           sh->exps, pairing);
    count_launch();
  }
  CF_CUDA(cudaGetLastError());
  return CFFYN_OK;
}

int set_op_smem_limits() {
  CF_CUDA(cudaFuncSetAttribute(k_op_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  CF_CUDA(cudaFuncSetAttribute(k_op_rec<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  return CFFYN_OK;
}

// Slicing pass of the mixed path (no-op on the FP64 path): per-field
// exponents of nf fields of len values each, then one digit record per value
// into sh->rec.  in_pairs: the input is pair-stored.
int op_prepare(const cffyn_shell* sh, const double* in, bool in_pairs, int nf, long long len, int pairing,
               cudaStream_t st) {
  if (sh->d.precision != CFFYN_MIXED) return CFFYN_OK;
  CF_CUDA(cudaMemsetAsync(sh->exps, 0, sizeof(int) * 64, st));
  const long long* x = reinterpret_cast<const long long*>(in);
  const int bx = (int)std::min<long long>((len + 255) / 256, 64);
  if (in_pairs)
    k_field_exp<true><<<dim3(bx, nf), 256, 0, st>>>(x, len, sh->exps);
  else
    k_field_exp<false><<<dim3(bx, nf), 256, 0, st>>>(x, len, sh->exps);
  count_launch();
  const long long n = (long long)nf * len;
  const unsigned nb = (unsigned)((n + 255) / 256);
  uint4* rec = reinterpret_cast<uint4*>(sh->rec);
  if (in_pairs)
    k_slice<true><<<nb, 256, 0, st>>>(x, len, n, sh->exps, pairing, rec);
  else
    k_slice<false><<<nb, 256, 0, st>>>(x, len, n, sh->exps, pairing, rec);
  count_launch();
  CF_CUDA(cudaGetLastError());
  return CFFYN_OK;
}

static OpArgs base_args(const cffyn_shell* sh) {
  OpArgs a;
  memset(&a, 0, sizeof(a));
  a.n_r = sh->n_r;
  a.N = sh->N;
  a.J = sh->J;
  a.R = sh->R;
  a.L = sh->L;
  return a;
}

// d_r of nfields fields: in/out [nfields][P]
int op_deriv_r(const cffyn_shell* sh, const double* in, double* out, int nfields, bool in_pairs,
                 cudaStream_t st) {
  OpArgs a = base_args(sh);
  a.kind = OP_R;
  a.in = in;
  a.out = out;
  a.g.K = a.g.K0 = a.g.P = a.g.P0 = sh->n_r;
  a.g.in_rs = a.g.out_rs = 1;
  a.g.ncols = (long long)nfields * sh->J * sh->N;
  (void)in_pairs;
  return launch(sh, a, sh->Dr, &sh->sDr, dim3(1, 1), st, 0);
}

int op_deriv_theta(const cffyn_shell* sh, const double* in, double* out, int nfields, bool in_pairs,
                   cudaStream_t st) {
  OpArgs a = base_args(sh);
  a.kind = OP_THETA;
  a.in = in;
  a.out = out;
  a.g.K = a.g.P = 2 * sh->N;
  a.g.K0 = a.g.P0 = sh->N;
  a.g.rev1 = 1;
  a.g.in_rs = a.g.out_rs = sh->n_r;
  a.g.ncols = (long long)nfields * (sh->J / 2) * sh->n_r;
  (void)in_pairs;
  return launch(sh, a, sh->Dth2, &sh->sDth2, dim3(1, 1), st, 0);
}

static int op_rows(const cffyn_shell* sh, const double* in, double* out, int nb, int K, int P,
                   long long in_bs, long long out_bs, const double* W, const SlicedOp* Ws,
                   cudaStream_t st, int pairing) {
  OpArgs a = base_args(sh);
  a.kind = OP_ROWS;
  a.in = in;
  a.out = out;
  a.Q = sh->N * sh->n_r;
  a.in_bs = in_bs;
  a.out_bs = out_bs;
  a.g.K = a.g.K0 = K;
  a.g.P = a.g.P0 = P;
  a.g.in_rs = a.g.out_rs = a.Q;
  a.g.ncols = (long long)nb * a.Q;
  return launch(sh, a, W, Ws, dim3(1, 1), st, pairing);
}

int op_deriv_phi(const cffyn_shell* sh, const double* in, double* out, int nfields, bool in_pairs,
                 cudaStream_t st) {
  long long bs = (long long)sh->P;
  (void)in_pairs;
  return op_rows(sh, in, out, nfields, sh->J, sh->J, bs, bs, sh->Dph, &sh->sDph, st, 0);
}

// phi analysis: S[f][j][i][k] -> C[f][row][i][k]
int op_dft_fwd(const cffyn_shell* sh, const double* in, double* out, int nf, cudaStream_t st) {
  long long Q = (long long)sh->N * sh->n_r;
  return op_rows(sh, in, out, nf, sh->J, sh->R, (long long)sh->J * Q, (long long)sh->R * Q, sh->Fan,
                 &sh->sFan, st, 1);
}

int op_dft_inv(const cffyn_shell* sh, const double* in, double* out, int nf, cudaStream_t st) {
  long long Q = (long long)sh->N * sh->n_r;
  return op_rows(sh, in, out, nf, sh->R, sh->J, (long long)sh->R * Q, (long long)sh->J * Q, sh->Fsy,
                 &sh->sFsy, st, 1);
}

// Projection of all spin classes, coefficients C -> C2 (same layout); one
// launch per class covering every m = 0..L.
int op_project(const cffyn_shell* sh, const double* C, double* C2, const int* slots_r0, int n_r0,
               const int* const slots_c[3], const int n_c[3], cudaStream_t st) {
  const int N = sh->N;
  const int nm = sh->L + 1;
  if (n_r0 > 0) {
    OpArgs a = base_args(sh);
    a.in = C;
    a.out = C2;
    a.kind = OP_PROJ0;
    a.slots = slots_r0;
    a.nslots = n_r0;
    a.batched_m = 1;
    a.w_stride = (long long)N * N;
    a.g.K = a.g.K0 = a.g.P = a.g.P0 = N;
    a.g.in_rs = a.g.out_rs = sh->n_r;
    a.g.ncols = (long long)n_r0 * 2 * sh->n_r;
    int rc = launch(sh, a, sh->Fproj0, &sh->sF0, dim3(1, nm), st, 1);
    if (rc) return rc;
  }
  for (int s = 0; s < 3; ++s) {
    if (n_c[s] <= 0) continue;
    OpArgs b = base_args(sh);
    b.in = C;
    b.out = C2;
    b.kind = OP_PROJC;
    b.slots = slots_c[s];
    b.nslots = n_c[s];
    b.batched_m = 1;
    b.w_stride = (long long)N * 2 * N;
    b.g.K = 2 * N;
    b.g.K0 = N;
    b.g.P = b.g.P0 = N;
    b.g.in_rs = b.g.out_rs = sh->n_r;
    b.g.ncols = (long long)n_c[s] * 4 * sh->n_r;
    int rc = launch(sh, b, sh->FprojC + (size_t)s * nm * N * 2 * N, &sh->sFC[s], dim3(1, nm), st, 1);
    if (rc) return rc;
  }
  return CFFYN_OK;
}

// Spherical derivatives of nf fields (FP64 input) into D = [3][nf][P], with the
// mixed path's digit records (16 bytes per value, nf * P of them) and field
// exponents (64 ints) at the given device addresses instead of the shell's
// workspace.  exps is zeroed here on st: its words are atomicMax targets.  The
// FP64 path uses neither.  Same kernels and arithmetic as op_prepare followed
// by op_deriv_r / op_deriv_theta / op_deriv_phi.
int op_derivs_at(const cffyn_shell* sh, const double* u, double* D, int nf, uint4* rec, int* exps,
                 cudaStream_t st) {
  const long long P = (long long)sh->P;
  if (sh->d.precision != CFFYN_MIXED) {
    int rc;
    if ((rc = op_deriv_r(sh, u, D, nf, false, st))) return rc;
    if ((rc = op_deriv_theta(sh, u, D + nf * P, nf, false, st))) return rc;
    return op_deriv_phi(sh, u, D + 2 * nf * P, nf, false, st);
  }
  CF_CUDA(cudaMemsetAsync(exps, 0, sizeof(int) * 64, st));
  const long long* x = reinterpret_cast<const long long*>(u);
  const int bx = (int)std::min<long long>((P + 255) / 256, 64);
  k_field_exp<false><<<dim3(bx, nf), 256, 0, st>>>(x, P, exps);
  count_launch();
  const long long n = (long long)nf * P;
  k_slice<false><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, P, n, exps, 0, rec);
  count_launch();
  CF_CUDA(cudaGetLastError());

  OpArgs a[3] = {base_args(sh), base_args(sh), base_args(sh)};
  const SlicedOp* W[3] = {&sh->sDr, &sh->sDth2, &sh->sDph};
  a[0].kind = OP_R;                                    // as op_deriv_r
  a[0].g.K = a[0].g.K0 = a[0].g.P = a[0].g.P0 = sh->n_r;
  a[0].g.in_rs = a[0].g.out_rs = 1;
  a[0].g.ncols = (long long)nf * sh->J * sh->N;
  a[1].kind = OP_THETA;                                // as op_deriv_theta
  a[1].g.K = a[1].g.P = 2 * sh->N;
  a[1].g.K0 = a[1].g.P0 = sh->N;
  a[1].g.rev1 = 1;
  a[1].g.in_rs = a[1].g.out_rs = sh->n_r;
  a[1].g.ncols = (long long)nf * (sh->J / 2) * sh->n_r;
  a[2].kind = OP_ROWS;                                 // as op_deriv_phi
  a[2].Q = sh->N * sh->n_r;
  a[2].in_bs = a[2].out_bs = P;
  a[2].g.K = a[2].g.K0 = a[2].g.P = a[2].g.P0 = sh->J;
  a[2].g.in_rs = a[2].g.out_rs = a[2].Q;
  a[2].g.ncols = (long long)nf * a[2].Q;
  for (int i = 0; i < 3; ++i) {
    a[i].in = u;
    a[i].out = D + i * nf * P;
    if (a[i].g.ncols <= 0) continue;
    const unsigned gx = (unsigned)((a[i].g.ncols + OZ_QT - 1) / OZ_QT);
    const int KP = W[i]->ksteps * 16 + 8;
    const size_t smem = (size_t)kSlices * OZ_QT * KP * sizeof(unsigned short);
    k_op_rec<true><<<dim3(gx, 1), W[i]->mtiles * 32, smem, st>>>(a[i], *W[i], rec, exps, 0);
    count_launch();
    CF_CUDA(cudaGetLastError());
  }
  return CFFYN_OK;
}

}  // namespace cffyn
