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
// Two arithmetic cores share the column descriptors and the gathers:
//   FP64   plain double FMA on CUDA cores (k_op_fp64, the reference path);
//   MIXED  split-precision products on the fifth-generation tensor cores
//          (k_op_tc): W and each input column are written as 47-bit
//          fixed-point integers relative to a per-row / per-field power of two
//          and cut into six balanced 8-bit digits held exactly in BF16; digit
//          products are summed by tcgen05.mma in FP32 accumulators in tensor
//          memory (see the k_op_tc comment for the exactness argument); pairs
//          with i + j > 5 are dropped (relative truncation about 6 * 2^-48 of
//          |W| |x| K).
#include <algorithm>
#include <cstdio>

#include "common.cuh"
#include "scalar.cuh"
#include "tc.cuh"

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
  int ns;                // stacked shells: function f of shell s is array f * ns + s
  int fld0;              // OP_ROWS: array index of the launch's first array (its exponent word, pairing)
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
      d.fld = a.fld0 + (int)b;
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
      // columns: (slot index, stacked shell, part, kr); parts: a (row m) and
      // b (row L+m, m >= 1)
      int nparts = a.m == 0 ? 1 : 2;
      long long per = (long long)nparts * a.n_r;
      if (c >= per * a.nslots * a.ns) { d.valid = 0; c = 0; }
      long long fi = c / per;
      int rem = (int)(c - fi * per);
      int part = rem / a.n_r, kr = rem - part * a.n_r;
      const long long fs = fi / a.ns;
      int f = a.slots[fs < a.nslots ? fs : 0] * a.ns + (int)(fi - fs * a.ns);
      d.fld = f;
      int row = part == 0 ? a.m : a.L + a.m;
      d.in0 = (((long long)f * a.R + row) * a.N) * a.n_r + kr;
      d.out0 = d.in0;
      d.in1 = d.out1 = 0;
      break;
    }
    case OP_PROJC: {
      // columns: (pair, stacked shell, output part, kr); parts aR, aI, bR, bI
      // (m >= 1) or aR, aI
      int nparts = a.m == 0 ? 2 : 4;
      long long per = (long long)nparts * a.n_r;
      if (c >= per * a.nslots * a.ns) { d.valid = 0; c = 0; }
      long long pi = c / per;
      int rem = (int)(c - pi * per);
      int part = rem / a.n_r, kr = rem - part * a.n_r;
      const long long ps = pi / a.ns;
      int fre = a.slots[ps < a.nslots ? ps : 0] * a.ns + (int)(pi - ps * a.ns), fim = fre + a.ns;
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

// ---------------------------------------------------------------------------
// Per-field exponents of the mixed path's operator inputs.
//
// exps[f] = max over the field of (frexp exponent + 1022), 0 for an all-zero
// field.  With pairing, slots f >= kPairedFrom form (re, im) pairs (f, f^1)
// that share one exponent (the projection of a complex function gathers
// both).  Column values are cut into 47-bit fixed point round(x 2^(47-E)),
// E = exps - 1022, inside the operator kernel.

constexpr int kPairedFrom = 16;

// The exponent word of a field is read off the largest magnitude bit pattern
// (monotone in the exponent): the leading float of a pair, or the high word of
// an FP64 value, sign cleared.  Each thread covers eight values (16-byte loads
// when the field length is even), each CTA 2048, one atomic per CTA.
constexpr int kExpThreads = 256, kExpPerThread = 8;

template <bool FI>
__device__ __forceinline__ unsigned int mag_key(long long w) {
  return FI ? ((unsigned int)w & 0x7fffffffu) : ((unsigned int)((unsigned long long)w >> 32) & 0x7fffffffu);
}

template <bool FI>
__global__ void __launch_bounds__(kExpThreads) k_field_exp(const long long* __restrict__ in, long long len,
                                                           int* __restrict__ exps) {
  __shared__ unsigned int wm[kExpThreads / 32];
  const int f = blockIdx.y;
  const long long* x = in + (long long)f * len;
  const long long b0 = (long long)blockIdx.x * kExpThreads * kExpPerThread;
  unsigned int m = 0;
  if ((len & 1) == 0) {
    const longlong2* x2 = reinterpret_cast<const longlong2*>(x);
#pragma unroll
    for (int i = 0; i < kExpPerThread / 2; ++i) {
      const long long q = b0 / 2 + (long long)i * kExpThreads + threadIdx.x;  // pair index
      if (2 * q < len) {
        const longlong2 v = __ldg(x2 + q);
        m = max(m, max(mag_key<FI>(v.x), mag_key<FI>(v.y)));
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < kExpPerThread; ++i) {
      const long long e = b0 + (long long)i * kExpThreads + threadIdx.x;
      if (e < len) m = max(m, mag_key<FI>(__ldg(x + e)));
    }
  }
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kExpThreads / 32; ++w) m = max(m, wm[w]);
    const int e = FI ? (int)(m >> 23) : (int)(m >> 20);
    const int word = FI ? (e ? e - 126 + 1022 : 0) : e;
    if (word) atomicMax(exps + f, word);
  }
}

// ---------------------------------------------------------------------------
// Split-precision core on the fifth-generation tensor cores (tcgen05).
//
// CTA: 128 data columns (the MMA's M: one TMEM lane each) x one row group of
// W (N = 48 or 96 rows), all of K in k-steps of 16 through a ring of
// shared-memory stages.  Warp-specialised:
//   producer warps (256 or 512 threads; one column and KQ = 8 or 4
//     consecutive k of every k-step each): write the six BF16 digit slices of
//     their values (47-bit fixed point relative to the field's exponent; the
//     next k-step's input words loaded right after the arrive) into the
//     stage, then arrive on its `xfull` barrier; after the last k-step they
//     run the epilogue;
//   one MMA warp: bulk-copies (TMA) the operator's sixteen slices of each
//     k-step (see TcOp) a stage ahead and, once a stage is full, issues the
//     digit-pair MMAs into five FP32 accumulators in TMEM and commits them to
//     the stage's `empty` barrier:
//   acc_d = sum_{i+j=d} W_i X_j                            d = 0..3
//   acc_4 = sum_{i+j=4} W_i X_j + 2^-8 sum_{i+j=5} W_i X_j + 2^-16 sum_{i+j=6} W_i X_j
// The digit-sum <= 4 pairs of one input slice X_j go out as one MMA of up to
// 256 rows over adjacent operator slices into adjacent accumulators (fewer
// MMAs per k-step, each input slice read from shared memory fewer times).
// A block's time goes mostly to the producers' loads and slicing, to its
// set-up and to the epilogue; the tensor core is busy about a third of it.
// The digit-sum-6 pairs are issued for the derivatives only (TcBatch::sum6);
// the filter's DFTs and projections stop at digit sum 5 (21 pairs) and copy
// eleven operator slices per k-step.
// acc_0..acc_3 are exact integers (below 4 * 192 * 2^14 < 2^24).  acc_4 is
// not exact; its rounding is below 2^-24 of a term of weight 256^-4 relative
// to the leading one, about 2^-56 of the result's scale, at the level of the
// dropped pairs i + j > 6 (about 4 * 2^-56).  With the digit-sum-6 pairs the
// result is as accurate as the 47-bit fixed point of its inputs; without
// them the dropped digit-sum-6 products (weight 2^-48) were the largest
// error.  The epilogue sums (acc_0 + acc_1 2^-8 + ... + acc_4 2^-32)
// 2^(E_row + E_col - 14) as a float pair (fold_pair).

constexpr int kTcCols = 128;
constexpr int kTcXSlice = kTcCols * 16 * 2;                 // bytes of one data slice per k-step
constexpr int kTcXBytes = kSlices * kTcXSlice;               // 24576
constexpr unsigned long long kTcWaitNs = 1000000000ull;      // bound of the drain waits: 1 s

// A wait of the pipeline with the shell's bound; a bound of 0 gives up at
// once without polling (the way callers exercise the timeout path).
__device__ __forceinline__ bool pipe_wait(uint64_t* b, unsigned parity, unsigned long long limit_ns) {
  return limit_ns ? tc::bar_wait(b, parity, limit_ns) : false;
}

// Up to four operator applications with the same row-group size in one
// launch (the projections of the spin classes); blockIdx.y = class * nm + m.
constexpr int kMaxBatch = 4;
struct TcBatch {
  OpArgs a[kMaxBatch];
  TcOp W[kMaxBatch];
  long long tiles[kMaxBatch];  // column tiles of each class
  int nclass, nm;
  int eoff;  // added to every column exponent: a bound from an earlier scan times the operator gain
  int sum6;  // issue the digit-sum-6 pairs (derivatives); the filter's operators stop at digit sum 5
  unsigned long long wait_ns;  // bound of every pipeline wait (the shell's setting; 0: give up at once)
};

template <int ROWS>
struct TcCfg {
  static constexpr int kProd = ROWS == 48 ? 256 : 512;                 // producer threads
  static constexpr int kThreads = kProd + 32;                          // + the MMA warp
  static constexpr int kKQ = 16 * kTcCols / kProd;                     // k per producer per k-step
  static constexpr int kWSlice = ROWS * 16 * 2;                        // bytes of one operator slice
  static constexpr int kWBytes = kTcWSlices * kWSlice;                 // 24576 | 49152
  static constexpr int kStage = kTcXBytes + kWBytes;                   // 49152 | 73728
  static constexpr int kStages = ROWS == 48 ? 2 : 3;                   // 2 CTAs / 1 CTA per SM
  static constexpr int kSmem = kStages * kStage;                       // 98304 | 221184
  static constexpr uint32_t kTmemCols = ROWS == 48 ? 256 : 512;        // 5 accumulators x ROWS
  static_assert(kSmem <= 227 * 1024, "dynamic shared memory per CTA");
  static_assert(kStage % 1024 == 0, "stage alignment of the descriptors and bulk copies");
};

// Raw 64-bit words of N consecutive k of one column (zero outside K or in an
// empty second segment; the sign of a negated segment applied on the bits).
// Branch-free so that the loads issue together.
template <bool FI, int N>
__device__ __forceinline__ void gather(const OpArgs& a, const ColDesc& d, int k0, long long (&w)[N]) {
  const long long* in = reinterpret_cast<const long long*>(a.in);
  const long long m = FI ? (long long)0x8000000080000000ull : (long long)0x8000000000000000ull;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const int k = k0 + i;
    const bool seg1 = k >= a.g.K0;
    const int kk = seg1 ? (a.g.rev1 ? (a.g.K - 1 - k) : (k - a.g.K0)) : k;
    const long long base = seg1 ? d.in1 : d.in0;
    const bool live = d.valid && k < a.g.K && !(seg1 && d.sgn1 == 2);
    const long long v = live ? __ldg(in + base + (long long)kk * a.g.in_rs) : 0ll;
    w[i] = (seg1 && d.sgn1 == 1) ? (v ^ m) : v;
  }
}

// (hi, lo) float pair, packed like the mixed path's internal storage, of
// (a0 + a1 2^-8 + a2 2^-16 + a3 2^-24 + a4 2^-32) f1 f2 f3 (f1, f2, f3 powers of
// two).  a0 + a1 2^-8 + a2 2^-16 + a3 2^-24 (exact values) is summed with
// error-free transformations, so that the sum's only roundings are those of
// the low words and of a4 2^-32 (below 2^-48 of |a0|); summing a3 2^-24 in
// plain FP32 would cost about 2^-24 of it, more than the digit-sum-6 terms.
__device__ __forceinline__ long long fold_pair(float a0, float a1, float a2, float a3, float a4, float f1,
                                               float f2, float f3) {
  ff r = two_sum(a0, fm(a1, 0.00390625f));
  const ff q = two_sum(r.hi, fm(a2, 1.52587890625e-05f));
  const ff v = two_sum(q.hi, fm(a3, 5.9604644775390625e-08f));
  const float low = __fmaf_rn(a4, 2.3283064365386963e-10f, fa(fa(r.lo, q.lo), v.lo));
  r = fast_two_sum(v.hi, low);
  const float hi = fm(fm(fm(r.hi, f1), f2), f3), lo = fm(fm(fm(r.lo, f1), f2), f3);
  return (long long)(((unsigned long long)__float_as_uint(lo) << 32) | __float_as_uint(hi));
}

// 2^k as a float, k clamped to the normal range
__device__ __forceinline__ float pow2f(int k) {
  return __int_as_float((max(-126, min(127, k)) + 127) << 23);
}

// Digit slices of a float pair x = hi + lo (|lo| < ulp(hi), |x| < 2^E) on the
// FMA pipe.  Digit j has weight 2^(E - 7 - 8j) (the balanced base-256 digits
// of round(x 2^(47 - E))).  For a float v and each j the exact steps
//   d = rint(v / w_j) (one FFMA against 1.5 * 2^23),  v -= d w_j  (exact FFMA)
// give balanced digits |d| <= 128 of v; the last digit rounds like the
// fixed-point conversion.  lo contributes to digits 3..5 only (|lo| / w_2 < 1/2),
// so digit j is d_j(hi) + d_j(lo), |.| <= 256, an exact BF16 value; it is the
// same integer sum of weights as the rounded fixed point of hi plus that of lo.
// Requires -78 <= E <= 126 (every weight and inverse weight a normal float).
struct DigitScale {
  float w[kSlices], inv[kSlices];
};

__device__ __forceinline__ DigitScale digit_scale(int E) {
  DigitScale c;
#pragma unroll
  for (int j = 0; j < kSlices; ++j) {
    c.w[j] = __int_as_float((E - 7 - 8 * j + 127) << 23);
    c.inv[j] = __int_as_float((7 + 8 * j - E + 127) << 23);
  }
  return c;
}

__device__ __forceinline__ void digits_pair_f32(long long wbits, const DigitScale& c, float (&d)[kSlices]) {
  constexpr float M = 12582912.0f;  // 1.5 * 2^23
  float v = __int_as_float((int)(unsigned int)wbits);
  float u = __int_as_float((int)(unsigned int)((unsigned long long)wbits >> 32));
#pragma unroll
  for (int j = 0; j < kSlices; ++j) {
    d[j] = __fsub_rn(__fmaf_rn(v, c.inv[j], M), M);
    if (j < kSlices - 1) v = __fmaf_rn(-d[j], c.w[j], v);
  }
#pragma unroll
  for (int j = 3; j < kSlices; ++j) {
    const float e = __fsub_rn(__fmaf_rn(u, c.inv[j], M), M);
    if (j < kSlices - 1) u = __fmaf_rn(-e, c.w[j], u);
    d[j] = __fadd_rn(d[j], e);
  }
}

__device__ __forceinline__ void bar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_addr(b)) : "memory");
}

// STAGE: the launch is d_r (one operator class, all rows in one group): the
// epilogue stages the tile's outputs in shared memory and stores them as one
// contiguous block.
template <bool FI, int ROWS, bool STAGE = false>
__global__ void __launch_bounds__(TcCfg<ROWS>::kThreads) k_op_tc(TcBatch B, const int* __restrict__ exps,
                                                                 int pairing, int* __restrict__ flag) {
  using C = TcCfg<ROWS>;
  constexpr int S = C::kStages, KQ = C::kKQ;
  extern __shared__ __align__(128) unsigned char smtc[];
  __shared__ uint64_t xfull[S], wfull[S], empty[S], accf;
  __shared__ uint32_t tmem_base;
  __shared__ float rowF[ROWS];  // 2^E_row
  // operator class and azimuthal number of this CTA (blockIdx.y = class * nm + m)
  const int cls = B.nclass > 1 ? (int)blockIdx.y / B.nm : 0;
  OpArgs a = B.a[cls];
  TcOp W = B.W[cls];
  if ((long long)blockIdx.x >= B.tiles[cls] * W.ngroups) return;  // past this class's columns
  const int tid = threadIdx.x;
  const bool producer = tid < C::kProd;
  const long long tile = blockIdx.x / W.ngroups;
  const int grp = (int)(blockIdx.x - tile * W.ngroups);
  if (a.batched_m) {
    a.m = (int)blockIdx.y - cls * B.nm;
    W.w += (size_t)a.m * W.w_stride;
    W.rowexp += (size_t)a.m * W.rowexp_stride;
  }
  const int ctile = tid & (kTcCols - 1);        // column within the tile (producers)
  const int kq = (tid >> 7) * KQ;               // first k of this producer within a k-step
  const ColDesc col = make_col(a, tile * kTcCols + ctile);
  int ce = exps[col.fld];
  if (pairing) {
    // slot pairs (f, f ^ 1), f >= kPairedFrom, of the same stacked shell
    const int f = a.ns == 1 ? col.fld : col.fld / a.ns, sidx = col.fld - f * a.ns;
    if (f >= kPairedFrom) ce = max(ce, exps[(f ^ 1) * a.ns + sidx]);
  }
  const int E = ce - 1022 + B.eoff;
  // the row exponents are needed only by the epilogue: loaded here, stored
  // to shared memory before the barrier that ends the main loop
  const int rexp = tid < ROWS ? W.rowexp[grp * ROWS + tid] : 0;
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      tc::bar_init(&xfull[s], C::kProd);
      tc::bar_init(&wfull[s], 1);
      tc::bar_init(&empty[s], 1);
    }
    tc::bar_init(&accf, 1);
  }
  if (tid >= C::kProd) tc::alloc(&tmem_base, C::kTmemCols);  // the MMA warp
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tm = tmem_base;
  const int ksteps = W.ksteps;
  bool ok = true;

  if (producer) {
    // byte offset of this thread's row piece (column ctile, k kq..kq+KQ-1)
    const int xoff = (ctile >> 3) * 256 + (kq >> 3) * 128 + (ctile & 7) * 16 + (kq & 7) * 2;
    const bool fscale = E >= -78 && E <= 126;  // FMA-pipe slicing of float pairs
    const DigitScale dsc = digit_scale(fscale ? E : 0);
    // The loads of the next k-step are issued after the arrive on the
    // current stage: the proxy fence and the arrive's release wait for every
    // load the thread has in flight, so loads issued before them would hold
    // up this stage (measured: the first k-step's slices 0.7 us later).
    long long nxt[KQ];
    gather<FI, KQ>(a, col, kq, nxt);
    for (int ks = 0; ks < ksteps; ++ks) {
      const int s = ks % S;
      long long cur[KQ];
#pragma unroll
      for (int i = 0; i < KQ; ++i) cur[i] = nxt[i];
      if (ks >= S && ok) ok = pipe_wait(&empty[s], ((ks - S) / S) & 1, B.wait_ns);
      unsigned char* xs = smtc + s * C::kStage + xoff;
      uint32_t wd[kSlices][KQ / 2];
      if (FI && fscale && ks * 16 + kq < a.g.K) {
#pragma unroll
        for (int i = 0; i < KQ; i += 2) {
          float f0[kSlices], f1[kSlices];
          digits_pair_f32(cur[i], dsc, f0);
          digits_pair_f32(cur[i + 1], dsc, f1);
          // BF16 of an 8-bit integer float: its upper half
#pragma unroll
          for (int j = 0; j < kSlices; ++j)
            wd[j][i >> 1] = __byte_perm(__float_as_uint(f0[j]), __float_as_uint(f1[j]), 0x7632);
        }
      } else if (ks * 16 + kq < a.g.K) {
#pragma unroll
        for (int i = 0; i < KQ; i += 2) {
          unsigned int d0[kSlices], d1[kSlices];
          digits_bf16(raw_fixed47<FI>(cur[i], E), d0);
          digits_bf16(raw_fixed47<FI>(cur[i + 1], E), d1);
#pragma unroll
          for (int j = 0; j < kSlices; ++j) wd[j][i >> 1] = d0[j] | (d1[j] << 16);
        }
      } else {
#pragma unroll
        for (int j = 0; j < kSlices; ++j)
#pragma unroll
          for (int i = 0; i < KQ / 2; ++i) wd[j][i] = 0u;
      }
#pragma unroll
      for (int j = 0; j < kSlices; ++j) {
        if (KQ == 8)
          *reinterpret_cast<uint4*>(xs + j * kTcXSlice) = make_uint4(wd[j][0], wd[j][1], wd[j][2], wd[j][3]);
        else
          *reinterpret_cast<uint2*>(xs + j * kTcXSlice) = make_uint2(wd[j][0], wd[j][1]);
      }
      tc::fence_proxy_async();
      bar_arrive(&xfull[s]);
      if (ks + 1 < ksteps) gather<FI, KQ>(a, col, (ks + 1) * 16 + kq, nxt);
    }
    if (ok) ok = pipe_wait(&accf, 0, B.wait_ns);
  } else if (tid == C::kProd) {
    // MMA thread
    const unsigned char* wsrc =
        reinterpret_cast<const unsigned char*>(W.w) + (size_t)grp * ksteps * C::kWBytes;
    // the operator slices of a k-step; without the digit-sum-6 pairs the
    // last five (digits 1..5 times 2^-16) stay in global memory
    const uint32_t wcopy = B.sum6 ? C::kWBytes : (kTcWSlices - 5) * C::kWSlice;
    const uint32_t sbase = tc::smem_addr(smtc);
    for (int ks = 0; ks < S && ks < ksteps; ++ks) {
      tc::bar_expect_tx(&wfull[ks], wcopy);
      tc::bulk_g2s(smtc + ks * C::kStage + kTcXBytes, wsrc + (size_t)ks * C::kWBytes, wcopy, &wfull[ks]);
    }
    int copied = S < ksteps ? S : ksteps;  // operator k-steps whose copy has been issued
    for (int ks = 0; ks < ksteps && ok; ++ks) {
      const int s = ks % S;
      ok = pipe_wait(&wfull[s], (ks / S) & 1, B.wait_ns) && pipe_wait(&xfull[s], (ks / S) & 1, B.wait_ns);
      if (!ok) break;
      tc::fence_after();
      const uint32_t xa = sbase + s * C::kStage;
      const uint64_t dx = tc::desc_kmajor(xa, 128, 256);
      const uint64_t dw = tc::desc_kmajor(xa + kTcXBytes, 128, 256);
      constexpr uint32_t ID = tc::idesc_bf16_f32(kTcCols, ROWS);
      constexpr uint64_t XS = kTcXSlice >> 4, WS = C::kWSlice >> 4;  // slice strides, descriptor units
      // digit-sum <= 4 pairs of input slice j: the operator slices 0..4-j
      // are adjacent in shared memory and their accumulators acc_j..acc_4
      // adjacent in TMEM, so up to 256 / ROWS of them go into one MMA of
      // N = n ROWS (fewer re-reads of the input slice)
      constexpr int kMerge = 256 / ROWS;
#pragma unroll
      for (int j = 0; j < 5; ++j)
#pragma unroll
        for (int i = 0; i + j <= 4; i += kMerge) {
          const int n = (5 - j - i) < kMerge ? (5 - j - i) : kMerge;
          const uint32_t idn = tc::idesc_bf16_f32(kTcCols, n * ROWS);
          tc::mma(tm + (i + j) * ROWS, dx + j * XS, dw + i * WS, idn, (ks > 0 || j > 0) ? 1u : 0u);
        }
#pragma unroll
      for (int i = 0; i < 6; ++i) tc::mma(tm + 4 * ROWS, dx + (5 - i) * XS, dw + (5 + i) * WS, ID, 1u);
      if (B.sum6) {
#pragma unroll
        for (int i = 1; i < 6; ++i) tc::mma(tm + 4 * ROWS, dx + (6 - i) * XS, dw + (10 + i) * WS, ID, 1u);
      }
      tc::commit(&empty[s]);
      // refill the stage of k-step ks - 1 with the operator of k-step ks - 1 + S
      if (ks >= 1 && copied < ksteps) {
        const int sp = (ks - 1) % S;
        ok = pipe_wait(&empty[sp], ((ks - 1) / S) & 1, B.wait_ns);
        if (!ok) break;
        tc::bar_expect_tx(&wfull[sp], wcopy);
        tc::bulk_g2s(smtc + sp * C::kStage + kTcXBytes, wsrc + (size_t)copied * C::kWBytes, wcopy,
                     &wfull[sp]);
        ++copied;
      }
    }
    // accf completes once every MMA issued above has completed: then the
    // accumulators are final, or, after a wait gave up, no MMA still reads
    // shared memory or writes tensor memory
    tc::commit(&accf);
    if (!ok) {
      // let operator copies still in flight land, and the MMAs issued finish,
      // before the CTA's memory goes (the long bound: these always end)
      for (int c = (copied > S ? copied - S : 0); c < copied; ++c) tc::bar_wait(&wfull[c % S], (c / S) & 1, kTcWaitNs);
      tc::bar_wait(&accf, 0, kTcWaitNs);
    }
  }
  if (tid < ROWS) rowF[tid] = pow2f(rexp);
  ok = __syncthreads_and(ok);
  if (!ok && tid == 0) atomicOr(flag, 2);
  tc::fence_after();
  if (ok && producer) {
    // producer warp w reads TMEM lanes 32 (w % 4) .. + 31 (its columns) and
    // rows [g R, (g + 1) R) of every accumulator, g = w / 4, R = ROWS / (warps / 4)
    constexpr int R = ROWS / (C::kProd / 128);
    const int g = tid >> 7;
    const int prow = min(a.g.P - grp * ROWS, ROWS);  // valid rows of this group
    // d_r (all rows in one group): outputs staged in the free stage buffers
    // (every MMA and copy has completed) as [column][row]
    constexpr bool stage_out = STAGE;
    long long* out_tile = reinterpret_cast<long long*>(smtc);
    const uint32_t lane = tm + ((uint32_t)(((tid >> 5) & 3) * 32) << 16);
    // 2^(E_col - 14) as two factors (the second is 1 unless E_col - 14 is
    // below the float range, i.e. for outputs that underflow anyway)
    const int ec = E - 14;
    const float cf1 = pow2f(ec), cf2 = pow2f(ec - max(-126, min(127, ec)));
    // the group's rows of this thread's column, each folded result handed to
    // sink(row within the group, pair bits)
    auto rows_out = [&](auto&& sink) {
#pragma unroll 1
      for (int p0 = g * R; p0 < (g + 1) * R && p0 < prow; p0 += 8) {
        uint32_t v0[8], v1[8], v2[8], v3[8], v4[8];
        tc::ld8(lane + 0 * ROWS + p0, v0);
        tc::ld8(lane + 1 * ROWS + p0, v1);
        tc::ld8(lane + 2 * ROWS + p0, v2);
        tc::ld8(lane + 3 * ROWS + p0, v3);
        tc::ld8(lane + 4 * ROWS + p0, v4);
        tc::ld_wait(v0);
        tc::tie(v1);
        tc::tie(v2);
        tc::tie(v3);
        tc::tie(v4);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (p0 + j < prow)
            sink(p0 + j, fold_pair(__uint_as_float(v0[j]), __uint_as_float(v1[j]), __uint_as_float(v2[j]),
                                   __uint_as_float(v3[j]), __uint_as_float(v4[j]), rowF[p0 + j], cf1, cf2));
        }
      }
    };
    if constexpr (!stage_out)
      rows_out([&](int row, long long w) { store_elem(a, col, grp * ROWS + row, __longlong_as_double(w)); });
    else
      rows_out([&](int row, long long w) { out_tile[ctile * prow + row] = w; });
    if constexpr (stage_out) {
      // d_r: the tile's outputs (columns c of n_r rows each, out0 = c n_r)
      // are one contiguous block; after the producers' barrier it is copied
      // out with consecutive threads on consecutive words
      asm volatile("bar.sync 1, %0;" ::"r"(C::kProd) : "memory");
      const long long c0 = tile * kTcCols;
      const long long nc = min((long long)kTcCols, a.g.ncols - c0);
      long long* dst = reinterpret_cast<long long*>(a.out) + c0 * prow;
      for (long long e = tid; e < nc * prow; e += C::kProd) dst[e] = out_tile[e];
    }
  }
  tc::fence_before();
  __syncthreads();
  if (tid >= C::kProd) {
    tc::fence_after();
    tc::dealloc(tm, C::kTmemCols);
  }
}

// ---------------------------------------------------------------------------
// Host side

// Mixed path: one launch of the tcgen05 core over the classes of b (same row
// group size, same input storage), grid = (max tiles x row groups,
// classes x nm).
static int launch_batch(const cffyn_shell* sh, const TcBatch& b0, cudaStream_t st, int pairing, bool in_pairs,
                        const int* exps, int* flag = nullptr) {
  if (!flag) flag = sh->flag;
  TcBatch b = b0;
  b.wait_ns = sh->tc_wait_ns;
  long long gx = 0;
  for (int c = 0; c < b.nclass; ++c) gx = std::max(gx, b.tiles[c] * b.W[c].ngroups);
  if (gx == 0) return CFFYN_OK;
  const dim3 grid((unsigned)gx, (unsigned)(b.nclass * b.nm));
  // d_r (one class, one row group): the instance with the staged epilogue
  const bool stage = b.nclass == 1 && b.a[0].kind == OP_R && b.W[0].ngroups == 1;
#define CFFYN_LAUNCH_TC(R_, FI_, ST_) \
  k_op_tc<FI_, R_, ST_><<<grid, TcCfg<R_>::kThreads, TcCfg<R_>::kSmem, st>>>(b, exps, pairing, flag)
  if (b.W[0].rows == 48) {
    if (in_pairs)
      stage ? CFFYN_LAUNCH_TC(48, true, true) : CFFYN_LAUNCH_TC(48, true, false);
    else
      stage ? CFFYN_LAUNCH_TC(48, false, true) : CFFYN_LAUNCH_TC(48, false, false);
  } else {
    if (in_pairs)
      stage ? CFFYN_LAUNCH_TC(96, true, true) : CFFYN_LAUNCH_TC(96, true, false);
    else
      stage ? CFFYN_LAUNCH_TC(96, false, true) : CFFYN_LAUNCH_TC(96, false, false);
  }
#undef CFFYN_LAUNCH_TC
  count_launch();
  CF_CUDA(cudaGetLastError());
  return CFFYN_OK;
}

// FP64 core, or on the mixed path the tcgen05 core with the per-field
// exponents of the input at exps (op_prepare fills sh->exps); in_pairs: the
// input is pair-stored.  Mixed-path outputs are pair-stored.  flag: the
// status word a timed-out wait of the tcgen05 core marks (sh->flag if NULL).
static int launch(const cffyn_shell* sh, const OpArgs& a, const double* W64, const TcOp* Wt, dim3 extra,
                  cudaStream_t st, int pairing, bool in_pairs, const int* exps = nullptr, int eoff = 0,
                  int sum6 = 1, int* flag = nullptr) {
  if (a.g.ncols <= 0) return CFFYN_OK;
  if (sh->d.precision == CFFYN_FP64 || Wt == nullptr) {
    unsigned gx = (unsigned)((a.g.ncols + F64_QT - 1) / F64_QT);
    unsigned gy = (unsigned)((a.g.P + F64_PT - 1) / F64_PT);
    size_t smem = (size_t)(F64_PT * a.g.K + a.g.K * F64_QT) * sizeof(double);
    k_op_fp64<<<dim3(gx, gy, extra.y), 256, smem, st>>>(a, W64);
    count_launch();
    CF_CUDA(cudaGetLastError());
    return CFFYN_OK;
  }
  TcBatch b;
  memset(&b, 0, sizeof(b));
  b.a[0] = a;
  b.W[0] = *Wt;
  b.tiles[0] = (a.g.ncols + kTcCols - 1) / kTcCols;
  b.nclass = 1;
  b.nm = (int)extra.y;
  b.eoff = eoff;
  b.sum6 = sum6;
  return launch_batch(sh, b, st, pairing, in_pairs, exps ? exps : sh->exps, flag);
}

int set_op_smem_limits() {
  CF_CUDA(cudaFuncSetAttribute(k_op_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  CF_CUDA(cudaFuncSetAttribute(k_op_tc<true, 48>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcCfg<48>::kSmem));
  CF_CUDA(cudaFuncSetAttribute(k_op_tc<false, 48>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcCfg<48>::kSmem));
  CF_CUDA(cudaFuncSetAttribute(k_op_tc<true, 96>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcCfg<96>::kSmem));
  CF_CUDA(cudaFuncSetAttribute(k_op_tc<false, 96>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcCfg<96>::kSmem));
  CF_CUDA(cudaFuncSetAttribute(k_op_tc<true, 48, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               TcCfg<48>::kSmem));
  CF_CUDA(cudaFuncSetAttribute(k_op_tc<false, 48, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               TcCfg<48>::kSmem));
  CF_CUDA(cudaFuncSetAttribute(k_op_tc<true, 96, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               TcCfg<96>::kSmem));
  CF_CUDA(cudaFuncSetAttribute(k_op_tc<false, 96, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               TcCfg<96>::kSmem));
  return CFFYN_OK;
}

// Per-field exponents of nf fields of len values each into exps (max(nf, 64)
// words, zeroed here: they are atomicMax targets); in_pairs: pair-stored input.
static int field_exps(const double* in, bool in_pairs, int nf, long long len, int* exps, cudaStream_t st) {
  CF_CUDA(cudaMemsetAsync(exps, 0, sizeof(int) * std::max(nf, 64), st));
  const long long* x = reinterpret_cast<const long long*>(in);
  const unsigned bx = (unsigned)((len + kExpThreads * kExpPerThread - 1) / (kExpThreads * kExpPerThread));
  if (in_pairs)
    k_field_exp<true><<<dim3(bx, nf), kExpThreads, 0, st>>>(x, len, exps);
  else
    k_field_exp<false><<<dim3(bx, nf), kExpThreads, 0, st>>>(x, len, exps);
  count_launch();
  CF_CUDA(cudaGetLastError());
  return CFFYN_OK;
}

// Mixed path (no-op on the FP64 path): the per-field exponents of the next
// operator input into sh->exps.
int op_prepare(const cffyn_shell* sh, const double* in, bool in_pairs, int nf, long long len, int pairing,
               cudaStream_t st) {
  (void)pairing;  // pairing is applied by the operator kernel
  if (sh->d.precision != CFFYN_MIXED) return CFFYN_OK;
  return field_exps(in, in_pairs, nf, len, sh->exps, st);
}

static OpArgs base_args(const cffyn_shell* sh) {
  OpArgs a;
  memset(&a, 0, sizeof(a));
  a.n_r = sh->n_r;
  a.N = sh->N;
  a.J = sh->J;
  a.R = sh->R;
  a.L = sh->Lrows;  // row of b_1 minus 1 in the DFT coefficient layout
  a.ns = sh->ns;
  return a;
}

// d_r (which = 0), d_theta over the double cover (1), d_phi (2) of nf fields:
// in/out [nf][P]
static OpArgs deriv_args(const cffyn_shell* sh, int which, const double* in, double* out, int nf) {
  OpArgs a = base_args(sh);
  a.in = in;
  a.out = out;
  if (which == 0) {
    a.kind = OP_R;
    a.g.K = a.g.K0 = a.g.P = a.g.P0 = sh->n_r;
    a.g.in_rs = a.g.out_rs = 1;
    a.g.ncols = (long long)nf * sh->J * sh->N;
  } else if (which == 1) {
    a.kind = OP_THETA;
    a.g.K = a.g.P = 2 * sh->N;
    a.g.K0 = a.g.P0 = sh->N;
    a.g.rev1 = 1;
    a.g.in_rs = a.g.out_rs = sh->n_r;
    a.g.ncols = (long long)nf * (sh->J / 2) * sh->n_r;
  } else {
    a.kind = OP_ROWS;
    a.Q = sh->N * sh->n_r;
    a.in_bs = a.out_bs = (long long)sh->P;
    a.g.K = a.g.K0 = a.g.P = a.g.P0 = sh->J;
    a.g.in_rs = a.g.out_rs = a.Q;
    a.g.ncols = (long long)nf * a.Q;
  }
  return a;
}

int op_deriv_r(const cffyn_shell* sh, const double* in, double* out, int nfields, bool in_pairs,
               cudaStream_t st) {
  return launch(sh, deriv_args(sh, 0, in, out, nfields), sh->Dr, &sh->tDr, dim3(1, 1), st, 0, in_pairs);
}

int op_deriv_theta(const cffyn_shell* sh, const double* in, double* out, int nfields, bool in_pairs,
                   cudaStream_t st) {
  return launch(sh, deriv_args(sh, 1, in, out, nfields), sh->Dth2, &sh->tDth2, dim3(1, 1), st, 0, in_pairs);
}

int op_deriv_phi(const cffyn_shell* sh, const double* in, double* out, int nfields, bool in_pairs,
                 cudaStream_t st) {
  return launch(sh, deriv_args(sh, 2, in, out, nfields), sh->Dph, &sh->tDph, dim3(1, 1), st, 0, in_pairs);
}

// d_theta and d_phi of nf fields (same input; both operators have 2N rows):
// one launch of the tcgen05 core on the mixed path, so that the two share
// the last, partly filled wave of CTAs; two launches on the FP64 path.
int op_deriv_theta_phi(const cffyn_shell* sh, const double* in, double* out_th, double* out_ph, int nf,
                       bool in_pairs, cudaStream_t st) {
  if (sh->d.precision != CFFYN_MIXED || sh->tDth2.rows != sh->tDph.rows) {
    int rc = op_deriv_theta(sh, in, out_th, nf, in_pairs, st);
    return rc ? rc : op_deriv_phi(sh, in, out_ph, nf, in_pairs, st);
  }
  TcBatch b;
  memset(&b, 0, sizeof(b));
  b.a[0] = deriv_args(sh, 1, in, out_th, nf);
  b.W[0] = sh->tDth2;
  b.a[1] = deriv_args(sh, 2, in, out_ph, nf);
  b.W[1] = sh->tDph;
  for (int c = 0; c < 2; ++c) b.tiles[c] = (b.a[c].g.ncols + kTcCols - 1) / kTcCols;
  b.nclass = 2;
  b.nm = 1;
  b.sum6 = 1;
  return launch_batch(sh, b, st, 0, in_pairs, sh->exps);
}

static int op_rows(const cffyn_shell* sh, const double* in, double* out, int nb, int K, int P,
                   long long in_bs, long long out_bs, const double* W, const TcOp* Wt, cudaStream_t st,
                   int pairing, int eoff = 0, int fld0 = 0) {
  OpArgs a = base_args(sh);
  a.kind = OP_ROWS;
  a.fld0 = fld0;
  a.in = in;
  a.out = out;
  a.Q = sh->N * sh->n_r;
  a.in_bs = in_bs;
  a.out_bs = out_bs;
  a.g.K = a.g.K0 = K;
  a.g.P = a.g.P0 = P;
  a.g.in_rs = a.g.out_rs = a.Q;
  a.g.ncols = (long long)nb * a.Q;
  // the phi DFTs of the filter: digit sums up to 5 suffice (filter errors
  // stay near 1e-12 relative)
  return launch(sh, a, W, Wt, dim3(1, 1), st, pairing, true, nullptr, eoff, 0);
}

// phi analysis: S[f][j][i][k] -> C[f][row][i][k] (pair-stored input on the
// mixed path) of the nf arrays f0 .. f0 + nf - 1; pairing: the exponents of
// slot pairs (f, f ^ 1) are shared (the complex slots of the Yn filter)
int op_dft_fwd(const cffyn_shell* sh, const double* in, double* out, int nf, cudaStream_t st, int pairing,
               int f0) {
  long long Q = (long long)sh->N * sh->n_r;
  return op_rows(sh, in + (size_t)f0 * sh->J * Q, out + (size_t)f0 * sh->R * Q, nf, sh->J, sh->R,
                 (long long)sh->J * Q, (long long)sh->R * Q, sh->Fan, &sh->tFan, st, pairing, 0, f0);
}

// eoff: see TcBatch (the coefficients' exponents are bounds, not a scan)
int op_dft_inv(const cffyn_shell* sh, const double* in, double* out, int nf, cudaStream_t st, int pairing,
               int eoff, int f0) {
  long long Q = (long long)sh->N * sh->n_r;
  return op_rows(sh, in + (size_t)f0 * sh->R * Q, out + (size_t)f0 * sh->J * Q, nf, sh->R, sh->J,
                 (long long)sh->R * Q, (long long)sh->J * Q, sh->Fsy, &sh->tFsy, st, pairing, eoff, f0);
}

// Component-wise filters (Sec. 3.5): every field's coefficients projected
// with F^0_m, C -> C2: the Y filter at the retained degree L (one class), the
// graded Yg filter at L + d for the fields of spatial degree d (eq. nfofmu;
// one class per d), m = 0..Lrows; one launch on the mixed path.
int op_project_scalar(const cffyn_shell* sh, const double* C, double* C2, cudaStream_t st, int eoff) {
  const int N = sh->N;
  const bool graded = sh->d.filter_kind == CFFYN_FILTER_YG;
  const int nm = sh->Lrows + 1;
  OpArgs cls[4];
  const double* W64[4];
  const TcOp* Wt[4];
  int ncls = 0, off = 0;
  for (int d = 0; d < 4; ++d) {
    if (sh->ny[d] <= 0) continue;
    OpArgs a = base_args(sh);
    a.in = C;
    a.out = C2;
    a.kind = OP_PROJ0;
    a.slots = sh->yslots + off;
    a.nslots = sh->ny[d];
    a.batched_m = 1;
    a.w_stride = (long long)N * N;
    a.g.K = a.g.K0 = a.g.P = a.g.P0 = N;
    a.g.in_rs = a.g.out_rs = sh->n_r;
    a.g.ncols = (long long)sh->ny[d] * 2 * sh->n_r * sh->ns;
    off += sh->ny[d];
    cls[ncls] = a;
    W64[ncls] = graded ? sh->F0g + (size_t)d * nm * N * N : sh->Fproj0;
    Wt[ncls++] = graded ? &sh->tF0g[d] : &sh->tF0;
  }
  if (sh->d.precision == CFFYN_MIXED) {
    TcBatch bt;
    memset(&bt, 0, sizeof(bt));
    for (int c = 0; c < ncls; ++c) {
      bt.a[c] = cls[c];
      bt.W[c] = *Wt[c];
      bt.tiles[c] = (cls[c].g.ncols + kTcCols - 1) / kTcCols;
    }
    bt.nclass = ncls;
    bt.nm = nm;
    bt.eoff = eoff;
    bt.sum6 = 0;
    return launch_batch(sh, bt, st, 0, true, sh->exps);
  }
  for (int c = 0; c < ncls; ++c) {
    int rc = launch(sh, cls[c], W64[c], Wt[c], dim3(1, nm), st, 0, true);
    if (rc) return rc;
  }
  return CFFYN_OK;
}

// Projection of all spin classes, coefficients C -> C2 (same layout): every
// class and every m = 0..L in one launch on the mixed path, one launch per
// class on the FP64 path.
int op_project(const cffyn_shell* sh, const double* C, double* C2, const int* slots_r0, int n_r0,
               const int* const slots_c[3], const int n_c[3], cudaStream_t st, int eoff) {
  const int N = sh->N;
  const int nm = sh->L + 1;
  OpArgs cls[4];
  const double* W64[4];
  const TcOp* Wt[4];
  int ncls = 0;
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
    a.g.ncols = (long long)n_r0 * 2 * sh->n_r * sh->ns;
    cls[ncls] = a;
    W64[ncls] = sh->Fproj0;
    Wt[ncls++] = &sh->tF0;
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
    b.g.ncols = (long long)n_c[s] * 4 * sh->n_r * sh->ns;
    cls[ncls] = b;
    W64[ncls] = sh->FprojC + (size_t)s * nm * N * 2 * N;
    Wt[ncls++] = &sh->tFC[s];
  }
  if (sh->d.precision == CFFYN_MIXED) {
    // every class of the projection in one launch (all have N rows)
    TcBatch bt;
    memset(&bt, 0, sizeof(bt));
    for (int c = 0; c < ncls; ++c) {
      bt.a[c] = cls[c];
      bt.W[c] = *Wt[c];
      bt.tiles[c] = (cls[c].g.ncols + kTcCols - 1) / kTcCols;
    }
    bt.nclass = ncls;
    bt.nm = nm;
    bt.eoff = eoff;
    bt.sum6 = 0;
    return launch_batch(sh, bt, st, 1, true, sh->exps);
  }
  for (int c = 0; c < ncls; ++c) {
    int rc = launch(sh, cls[c], W64[c], Wt[c], dim3(1, nm), st, 1, true);
    if (rc) return rc;
  }
  return CFFYN_OK;
}

// Spherical derivatives of nf fields (FP64 input) into D = [3][nf][P], with the
// mixed path's per-field exponents (64 ints) at exps instead of the shell's
// workspace; exps is zeroed here on st (its words are atomicMax targets).
// A timed-out wait of the tcgen05 core sets bit 2 of *flag (not of the
// shell's own status word).  The FP64 path uses neither.  Same kernels and
// arithmetic as op_prepare followed by op_deriv_r / op_deriv_theta /
// op_deriv_phi.
int op_derivs_at(const cffyn_shell* sh, const double* u, double* D, int nf, int* exps, int* flag,
                 cudaStream_t st) {
  const long long P = (long long)sh->P;
  const bool mixed = sh->d.precision == CFFYN_MIXED;
  int rc;
  if (mixed && (rc = field_exps(u, false, nf, P, exps, st))) return rc;
  const double* W64[3] = {sh->Dr, sh->Dth2, sh->Dph};
  const TcOp* Wt[3] = {&sh->tDr, &sh->tDth2, &sh->tDph};
  for (int i = 0; i < 3; ++i)
    if ((rc = launch(sh, deriv_args(sh, i, u, D + i * nf * P, nf), W64[i], Wt[i], dim3(1, 1), st, 0, false,
                     exps, 0, 1, flag)))
      return rc;
  return CFFYN_OK;
}

}  // namespace cffyn
