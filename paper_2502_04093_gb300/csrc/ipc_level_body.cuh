// Reconstruction tile of the fused level kernels of libipcomp (sm_103a),
// shared by the units that instantiate its kernels (the plain reconstruction
// in ipc_level_kernels.cuh, the incremental and state-recording forms
// below, for ipc_level_delta.cu and ipc_level_delta_quad.cu). See
// ipc_level_kernels.cuh for the tile layout.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "ipc_device.cuh"
#include "ipc_internal.h"

namespace ipc {
namespace {
using namespace dev;

template <class T> struct Vec2;
template <> struct Vec2<float> { typedef float2 type; };
template <> struct Vec2<double> { typedef double2 type; };

struct CtaPos {
  int P, R0, R1, C0, C1;
  uint64_t rb, ct;
  int64_t pbase;  // element offset of lattice point (P, 0, 0)
  int64_t rs;     // element offset of one lattice row (c1 -> c1 + 1)
};

__device__ __forceinline__ CtaPos cta_pos(const LevelArgs& L, uint64_t cta, int BR, int BC) {
  CtaPos c;
  const uint32_t b = (uint32_t)cta, b1 = div_by(b, L.mct), p = div_by(b1, L.mrb);
  c.ct = b - b1 * (uint32_t)L.nct;
  c.rb = b1 - p * (uint32_t)L.nrb;
  c.P = (int)p;
  c.R0 = (int)c.rb * BR;
  c.R1 = (int)min(L.M[1], (int64_t)c.R0 + BR);
  c.C0 = (int)c.ct * BC;
  c.C1 = (int)min(L.M[2], (int64_t)c.C0 + BC);
  c.pbase = (int64_t)c.P * L.stride[0] * L.s;
  c.rs = L.stride[1] * L.s;
  return c;
}

// Quantize x against pred (Sec. 4.2.2); returns the code, writes xhat.
template <class T>
__device__ __forceinline__ int32_t quantize(T xv, T pred, const QuantArgs<T>& qa, T* rec,
                                            bool* outlier) {
  const T t = FP<T>::mul(FP<T>::sub(xv, pred), qa.inv2eb);
  *outlier = !FP<T>::abs_le(t, qa.R);
  *rec = xv;
  if (*outlier) return 0;
  int32_t qi;
  const T qf = FP<T>::rint_(t, &qi);
  const T rc = FP<T>::add(pred, FP<T>::mul(qf, qa.twoeb));
  if (FP<T>::abs_le(FP<T>::sub(xv, rc), qa.ebchk)) {
    *rec = rc;
    return qi;
  }
  *outlier = true;
  return 0;
}

__device__ __forceinline__ void record_outlier(const SweepOut& o, int stage, uint64_t ci,
                                               double v) {
  const unsigned long long slot = atomicAdd(o.outl_count, 1ULL);
  if (slot < o.outl_cap) {
    o.outl_key[slot] = ((unsigned long long)o.field << 48) | ((unsigned long long)stage << 40) |
                       (unsigned long long)ci;
    o.outl_val[slot] = v;
  }
}

// Segment of the stage's word grid owned by the CTA (see LevelStage).
__device__ __forceinline__ uint64_t seg_id(const LevelStage& S, uint64_t pi, uint64_t rb,
                                           uint64_t ct) {
  return (pi * S.nrb + rb) * S.nct + ct;
}

// Exact-value lookup of an outlier code (sorted index list of the stage).
// ZERO: the increment of an outlier (Algorithm 2) is zero -- its value is
// exact already -- so the lookup yields 0 instead of the value.
template <class T, bool ZERO = false>
__device__ __forceinline__ bool find_outlier(const LevelStage& S, const uint64_t* __restrict__ idx,
                                             const double* __restrict__ val, uint64_t ci, T* v) {
  uint64_t lo = S.out_begin, hi = S.out_end;
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    const uint64_t m = __ldg(idx + mid);
    if (m < ci) lo = mid + 1;
    else hi = mid;
  }
  if (lo < S.out_end && __ldg(idx + lo) == ci) {
    *v = ZERO ? (T)0 : (T)__ldg(val + lo);
    return true;
  }
  return false;
}

// ---------------------------------------------------------------------------
// Reconstruction of one level (Algorithm 1).
//
// Setup: warp 0 finds the planes to load (plane k >= b with nonzero words in
// the stage) and the top loaded plane; the CTA starts asynchronous copies,
// for the loaded planes of at most 13 segments (its own, and for halo
// targets the neighbouring segments: stage 1 left/right, stage 0 the 3x3
// block), of the group bitmap words, and notes the payload bases. A word's
// plane value is then found from its group's bitmap word alone (rank =
// population below its bit).
// Phase 1a (while the copies land): even value rows -- the sweep-0
//   predictions of an odd plane from the known planes P +- 1, P +- 3, or the
//   known points of an even plane; one column per thread.
// Phase 0: one thread per word of the tile's own code columns: load the
//   selected planes, undo the predictive XOR top-down, transpose (a 16-plane
//   window when the loaded planes span at most 16, else all 32) and store the
//   32 codes. The three halo code columns (one left, two right) are extracted
//   bit by bit from their words without a transpose.
// Phase 1b (odd planes): add the sweep-0 codes to the predictions -- the same
//   two operations, in the same order, as when they follow at once.
// Phase 2: odd value rows (sweep 1), one column per thread, the four row
//   neighbours kept in registers.
// Phase 3: sweep 2 fused with the output: each thread computes four odd
//   columns of a row and stores them with the five even columns around them
//   as one run of eight elements.
// ---------------------------------------------------------------------------
constexpr int kSlots = 13;
constexpr int kMaxBw = 4;  // bitmap words per segment (RB * CW <= 128)

// Code rows hold the tile's codes of one stage row. When the loaded planes
// of a level span at most 16 (the usual case; decided on the host per
// launch) a code is its 16-plane window value, stored in 16 bits (the
// window base is a shift applied on reading); otherwise the full 32 bits.
// Layout: blocks of 32 codes plus pad, so that one thread's 32 codes are
// conflict-free 16-byte stores and four consecutive codes one load.
template <bool W16> struct QCfg;
template <> struct QCfg<true> {
  typedef uint16_t QT;
  static constexpr int BLK = 40;  // codes + pad per block (80 bytes)
  static constexpr int NPL = 16;  // planes staged per segment
};
template <> struct QCfg<false> {
  typedef uint32_t QT;
  static constexpr int BLK = 36;  // 144 bytes
  static constexpr int NPL = 32;
};

template <int BR, int BC, bool W16>
struct RTile {
  static constexpr int HC = BC / 2;      // codes of one stage per tile row
  static constexpr int CWD = BC / 64;    // words per tile row
  static constexpr int QP = CWD * QCfg<W16>::BLK;  // code-row pitch
  static constexpr int VR = BR + 5;      // value rows: c1 in [R0-2, R0+BR+2]
  static constexpr int V0 = 4;           // value column of code column 0 (16-byte aligned)
  static constexpr int VP = HC + 8;      // value-row pitch: code columns -1 .. HC+1 (+ pad)
  static constexpr int H1 = BR / 2;      // stage-1 code rows (own odd c1)
  static constexpr int H0 = BR / 2 + 3;  // stage-0 code rows (even c1, with halo)
};

// Position of tile code column e in a code row.
template <bool W16>
__device__ __forceinline__ int qoff(int e) { return (e >> 5) * QCfg<W16>::BLK + (e & 31); }

// Four consecutive 32-bit codes.
__device__ __forceinline__ void load4(const uint32_t* p, int, uint32_t (&n)[4]) {
  const uint4 v = *reinterpret_cast<const uint4*>(p);
  n[0] = v.x;
  n[1] = v.y;
  n[2] = v.z;
  n[3] = v.w;
}

// Values of four codes: the small-code conversion when all four allow it.
__device__ __forceinline__ void code_values4(const uint32_t (&n)[4], float (&v)[4]) {
  int q[4];
  unsigned wide = 0u;
#pragma unroll
  for (int k = 0; k < 4; ++k) wide |= code_wide(n[k], &q[k]);
  if (wide == 0u) {
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = code_small(q[k]);
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = code_value(n[k], 0.0f);
  }
}
__device__ __forceinline__ void code_values4(const uint32_t (&n)[4], double (&v)[4]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) v[k] = code_value(n[k], 0.0);
}

// w[0] = p[-1] and w[1..8] = p[0..7], p 16-byte aligned (the value columns
// of code columns 4g-1 .. 4g+7 of one row).
template <class T>
__device__ __forceinline__ void lds9(const T* p, T (&w)[9]);
template <>
__device__ __forceinline__ void lds9<float>(const float* p, float (&w)[9]) {
  w[0] = p[-1];
  const float4 u = reinterpret_cast<const float4*>(p)[0], v = reinterpret_cast<const float4*>(p)[1];
  w[1] = u.x; w[2] = u.y; w[3] = u.z; w[4] = u.w;
  w[5] = v.x; w[6] = v.y; w[7] = v.z; w[8] = v.w;
}
template <>
__device__ __forceinline__ void lds9<double>(const double* p, double (&w)[9]) {
  w[0] = p[-1];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const double2 u = reinterpret_cast<const double2*>(p)[i];
    w[1 + 2 * i] = u.x;
    w[2 + 2 * i] = u.y;
  }
}

// Products code value x 2eb of the codes of a code row. A 16-bit row entry v
// holds the negabinary digits wb .. wb+15 of a code, whose value is then
// (-2)^wb times the 16-digit value of v. That sign is folded into the digit
// mask: swapping the masks of the odd and the even positions negates a digit
// string's value, so the code's value is 2^wb * z with z = (v ^ mask) - mask.
// z is exact in float (|z| < 2^16) and is formed by placing v ^ mask under
// the exponent of 1.5 * 2^23 and subtracting 1.5 * 2^23 + mask. The product
// z * (2eb 2^wb) is the same real number as value * 2eb, rounded once, so it
// is the same result (2eb 2^wb is exact: the host keeps it finite).
template <class T>
struct CodeScale {
  uint32_t zmask;  // digit mask in both 16-bit halves
  float zbias;     // 1.5 * 2^23 + the 16-bit mask
  T tw;            // 2eb * 2^wb (16-bit rows) or 2eb (32-bit rows)
};
template <class T>
__device__ __forceinline__ CodeScale<T> code_scale(T twoeb, int wb) {
  CodeScale<T> c;
  c.zmask = (wb & 1) ? 0x55555555u : 0xAAAAAAAAu;
  c.zbias = (wb & 1) ? 12604757.0f : 12626602.0f;
  c.tw = FP<T>::mul(twoeb, (T)(1u << wb));
  return c;
}
template <class T>
__device__ __forceinline__ void scaled_word(uint32_t x, const CodeScale<T>& cs, T* v) {
  const uint32_t t = x ^ cs.zmask;
  const float z0 = __fsub_rn(__int_as_float(__byte_perm(t, 0x4B40u, 0x5410)), cs.zbias);
  const float z1 = __fsub_rn(__int_as_float(__byte_perm(t, 0x4B40u, 0x5432)), cs.zbias);
  v[0] = FP<T>::mul((T)z0, cs.tw);
  v[1] = FP<T>::mul((T)z1, cs.tw);
}
// double: z in integer arithmetic and its exact double built the same way
// (no conversion instruction on the FP64 pipe)
template <>
__device__ __forceinline__ void scaled_word<double>(uint32_t x, const CodeScale<double>& cs,
                                                    double* v) {
  const uint32_t t = x ^ cs.zmask;
  const int m = (int)(cs.zmask & 0xFFFFu);
  v[0] = FP<double>::mul(exact_double((int)(t & 0xFFFFu) - m), cs.tw);
  v[1] = FP<double>::mul(exact_double((int)(t >> 16) - m), cs.tw);
}
template <class T>
__device__ __forceinline__ void scaled_pair(const uint16_t* p, const CodeScale<T>& cs, T (&v)[2]) {
  scaled_word(*reinterpret_cast<const uint32_t*>(p), cs, v);
}
template <class T>
__device__ __forceinline__ void scaled_pair(const uint32_t* p, const CodeScale<T>& cs, T (&v)[2]) {
  const uint2 u = *reinterpret_cast<const uint2*>(p);
  v[0] = FP<T>::mul(code_value(u.x, T()), cs.tw);
  v[1] = FP<T>::mul(code_value(u.y, T()), cs.tw);
}
template <class T>
__device__ __forceinline__ void scaled_quad(const uint16_t* p, const CodeScale<T>& cs, T (&v)[4]) {
  const uint2 u = *reinterpret_cast<const uint2*>(p);
  scaled_word(u.x, cs, v);
  scaled_word(u.y, cs, v + 2);
}
template <class T>
__device__ __forceinline__ void scaled_quad(const uint32_t* p, const CodeScale<T>& cs, T (&v)[4]) {
  uint32_t n[4];
  load4(p, 0, n);
  T c[4];
  code_values4(n, c);
#pragma unroll
  for (int k = 0; k < 4; ++k) v[k] = FP<T>::mul(c[k], cs.tw);
}

// Stores the values v[0..7] of lattice columns c2e .. c2e+7 of one row
// (element offset of lattice point (P, c1, 0) is `row`). At stride 1 they
// are consecutive elements; at stride 2 each value is written twice so that
// whole sectors are written (the element in between is a target of the next
// level and is never read as a known value); larger strides store singly.
// cs: evict-first ("streaming") stores for the runs at stride 1.
template <class T>
__device__ __forceinline__ void store_run(T* row, int64_t s, int64_t n2, int c2e, int C1,
                                          const T (&v)[8], bool cs = false) {
  typedef typename Vec2<T>::type V2;
  if (s == 1) {
    T* p = row + c2e;
    if (c2e + 8 <= C1 && ((uintptr_t)p & 15) == 0) {
      if (sizeof(T) == 4) {
        float4* q = reinterpret_cast<float4*>(p);
        const float4 a = make_float4((float)v[0], (float)v[1], (float)v[2], (float)v[3]);
        const float4 b = make_float4((float)v[4], (float)v[5], (float)v[6], (float)v[7]);
        if (cs) {
          __stcs(q, a);
          __stcs(q + 1, b);
        } else {
          q[0] = a;
          q[1] = b;
        }
      } else {
        V2* q = reinterpret_cast<V2*>(p);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          V2 t;
          t.x = v[2 * i];
          t.y = v[2 * i + 1];
          if (cs) __stcs(q + i, t);
          else q[i] = t;
        }
      }
      return;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if (c2e + i < C1) p[i] = v[i];
    return;
  }
  if (s == 2) {
    T* p = row + 2 * (int64_t)c2e;
    if (c2e + 8 <= C1 && 2 * (int64_t)(c2e + 7) + 1 < n2 && ((uintptr_t)p & 15) == 0) {
      if (sizeof(T) == 4) {
        float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
        for (int i = 0; i < 4; ++i)
          q[i] = make_float4((float)v[2 * i], (float)v[2 * i], (float)v[2 * i + 1],
                             (float)v[2 * i + 1]);
      } else {
        V2* q = reinterpret_cast<V2*>(p);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          V2 t;
          t.x = v[i];
          t.y = v[i];
          q[i] = t;
        }
      }
      return;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if (c2e + i < C1) p[2 * i] = v[i];
    return;
  }
#pragma unroll
  for (int i = 0; i < 8; ++i)
    if (c2e + i < C1) row[(int64_t)(c2e + i) * s] = v[i];
}

// Tile of a level launch: NS planes of the same parity side by side, each a
// sub-tile of BR rows and BC / NS lattice columns (NS > 1 only when the
// level's rows are at most BC / NS wide). Tiles enumerate (plane group,
// row block, column tile); with NS = 1 the groups are the planes in order.
__device__ __forceinline__ CtaPos sub_pos(const LevelArgs& L, uint64_t tile, int j, int NS, int BR,
                                          int BCs) {
  CtaPos c;
  const uint32_t t = (uint32_t)tile, t1 = div_by(t, L.mct), g = div_by(t1, L.mrb);
  c.ct = t - t1 * (uint32_t)L.nct;
  c.rb = t1 - g * (uint32_t)L.nrb;
  // groups alternate even / odd (an odd plane reads the known points of the
  // even planes around it while they are in L2); the even groups can be one
  // more than the odd ones
  const int64_t grp = g;
  const int64_t go = ((int)(L.M[0] >> 1) + NS - 1) / NS;
  const int64_t par = grp < 2 * go ? (grp & 1) : 0, idx = grp < 2 * go ? (grp >> 1) : go;
  c.P = (int)(2 * (idx * NS + j) + par);
  c.R0 = (int)c.rb * BR;
  c.R1 = (int)min(L.M[1], (int64_t)c.R0 + BR);
  c.C0 = (int)c.ct * BCs;
  c.C1 = (int)min(L.M[2], (int64_t)c.C0 + BCs);
  c.pbase = (int64_t)c.P * L.stride[0] * L.s;
  c.rs = L.stride[1] * L.s;
  return c;
}

// Forms of the reconstruction body:
//   kPlain  -- Algorithm 1: x^ from the selected planes;
//   kRecord -- the same, and for every own code word the decoded digits at
//              planes b and b + 1 go to the view's state (the prefix of a
//              later incremental refinement);
//   kDelta  -- Algorithm 2: only the planes [b, bo) are read, decoded with the
//              state's digits bo, bo + 1 as prefix; the increment Delta is
//              interpolated from zero (known points: the coarser level's
//              Delta; outliers: 0); the caller's array gets x^ += Delta where
//              Delta is not zero, and the state moves to digits b, b + 1.
constexpr int kPlain = 0, kRecord = 1, kDelta = 2;

// x^ += v over the run of eight elements of one output row (level 1 of an
// incremental refinement); elements whose increment is zero are left alone,
// a run of zeros is neither read nor written.
template <class T>
__device__ __forceinline__ void add_run(T* row, int c2e, int C1, const T (&v)[8]) {
  bool any = false;
#pragma unroll
  for (int i = 0; i < 8; ++i) any |= v[i] != (T)0;
  if (!any) return;
  T* p = row + c2e;
  if (c2e + 8 <= C1 && ((uintptr_t)p & 15) == 0) {
    typedef typename Vec2<T>::type V2;
    if (sizeof(T) == 4) {
      float4* q = reinterpret_cast<float4*>(p);
      float4 a = q[0], b = q[1];
      float o[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (v[i] != (T)0) o[i] = FP<float>::add(o[i], (float)v[i]);
      q[0] = make_float4(o[0], o[1], o[2], o[3]);
      q[1] = make_float4(o[4], o[5], o[6], o[7]);
    } else {
      V2* q = reinterpret_cast<V2*>(p);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        V2 t = q[i];
        if (v[2 * i] != (T)0) t.x = FP<T>::add(t.x, v[2 * i]);
        if (v[2 * i + 1] != (T)0) t.y = FP<T>::add(t.y, v[2 * i + 1]);
        q[i] = t;
      }
    }
    return;
  }
#pragma unroll
  for (int i = 0; i < 8; ++i)
    if (c2e + i < C1 && v[i] != (T)0) p[i] = FP<T>::add(p[i], v[i]);
}

// Q: the quadratic boundary forms of pred4 compiled in (interp 2 possible).
template <class T, int BR, int BC, bool W16, int NS, int MODE = kPlain, bool Q = false>
__device__ __forceinline__ void level_retrieve_body(const LevelArgs& L, T* out, T twoeb, int b,
                                                    const uint32_t* __restrict__ cap,
                                                    const uint32_t* __restrict__ bm,
                                                    const uint64_t* __restrict__ oidx,
                                                    const double* __restrict__ oval,
                                                    uint64_t tile, unsigned char* smem) {
  constexpr int BCs = BC / NS;  // lattice columns of a sub-tile
  typedef RTile<BR, BCs, W16> G;
  typedef typename QCfg<W16>::QT QT;
  constexpr int NPL = QCfg<W16>::NPL;
  constexpr int TS = 256 / NS;                 // threads of a sub-tile
  constexpr int BWS = kMaxBw / NS;             // bitmap words of a sub-tile's segment
  static_assert(G::HC * NS == 256, "one thread per code column of a tile row");
  constexpr size_t SUB = sizeof(T) * G::VR * G::VP + sizeof(QT) * (BR + G::H1 + G::H0) * G::QP +
                         16 * (G::H1 + G::H0);  // bytes of a sub-tile's dynamic smem
  // Segments a sub-tile reads: with one column tile per row (NS > 1) its
  // own stage-2 and stage-1 segments and the stage-0 segments of row blocks
  // rb-1..rb+1 (slots 0, 1, 2..4); otherwise also the column neighbours:
  // 0 = stage 2 own; 1..3 = stage 1 (ct-1, ct, ct+1); 4..12 = stage 0
  // (rb-1..rb+1) x (ct-1..ct+1).
  constexpr int KS = NS > 1 ? 5 : kSlots;
  __shared__ uint32_t SB[NS][KS][NPL][BWS];        // group bitmaps of the window's planes
  __shared__ const uint32_t* SP[NS][KS][NPL];      // payload base of (segment, plane)

  const int tid = threadIdx.x;
  const int sub = tid / TS, ltid = tid % TS;  // the thread's sub-tile
  auto VEof = [&](int s) { return reinterpret_cast<T*>(smem + s * SUB); };
  auto Q2of = [&](int s) { return reinterpret_cast<QT*>(VEof(s) + G::VR * G::VP); };
  auto Q1of = [&](int s) { return Q2of(s) + BR * G::QP; };
  auto Q0of = [&](int s) { return Q1of(s) + G::H1 * G::QP; };
  auto QHof = [&](int s) { return reinterpret_cast<uint32_t*>(Q0of(s) + G::H0 * G::QP); };
  const int interp = L.interp;
  const int M0 = (int)L.M[0], M1 = (int)L.M[1], M2 = (int)L.M[2];
  const LevelStage &S0 = L.st[0], &S1 = L.st[1], &S2 = L.st[2];

  // The thread's own sub-tile. The sub-tiles of a tile share rows, columns
  // and plane parity: sub-tile j holds plane P0 + 2j (sub-tile 0 always
  // holds a plane).
  const CtaPos c = sub_pos(L, tile, sub, NS, BR, BCs);
  const int P0 = c.P - 2 * sub;
  // Segments (the compression's tiles) are SR rows of stage 2 and SR / 2 of
  // stages 1 and 0; a tile of BR <= SR rows lies in segment row block rbseg.
  constexpr int SR = sizeof(T) == 4 ? kLevelRowsF32 : kLevelRowsF64;
  static_assert(SR % BR == 0, "a tile's rows lie in one segment");
  const int rbseg = c.R0 / SR;
  const bool live = c.P < M0;
  const bool podd = (c.P & 1) != 0;
  T* VE = VEof(sub);
  QT* Q2 = Q2of(sub);
  QT* Q1 = Q1of(sub);
  QT* Q0 = Q0of(sub);
  uint32_t* QH = QHof(sub);

  // Planes to load per stage (k >= b with nonzero words, from the host) and
  // the plane window: slot i of the staged tables is plane wb + i. With
  // 16-bit codes the loaded planes [b, ktop] lie in [wb, wb + 15] (checked
  // on the host for the level).
  const uint32_t km0 = podd ? L.sp[0].kmask : 0u, km1 = L.sp[1].kmask, km2 = L.sp[2].kmask;
  const int ktop = 31 - __clz((int)(km0 | km1 | km2));
  // (an increment's window starts at its lowest new plane b; the host keeps
  // bo - b <= 16 for 16-bit rows)
  const int wb = MODE == kDelta ? (W16 ? b : 0) : (W16 ? max(0, ktop - 15) : 0);
  const CodeScale<T> sc = code_scale<T>(twoeb, wb);
  // Staging, one (sub-tile, segment slot, window plane) per thread: the
  // payload base and asynchronous copies of the group bitmap words.
  for (int u = tid; u < NS * KS * NPL; u += 256) {
    const int s = u / (KS * NPL), r = u % (KS * NPL);
    const int sl = r / NPL, i = r % NPL, k = wb + i;
    int sx, drb, dct;
    if (sl == 0) { sx = 2; drb = 0; dct = 0; }
    else if (KS == 5) {
      sx = sl == 1 ? 1 : 0; drb = sl == 1 ? 0 : sl - 3; dct = 0;
    } else if (sl < 4) { sx = 1; drb = 0; dct = sl - 2; }
    else { sx = 0; drb = (sl - 4) / 3 - 1; dct = (sl - 4) % 3 - 1; }
    const uint32_t km = sx == 0 ? km0 : (sx == 1 ? km1 : km2);
    const int Ps = P0 + 2 * s;
    if (Ps >= M0 || k > 31 || !((km >> k) & 1u)) continue;
    const LevelStage& S = L.st[sx];
    const int64_t rbs = (int64_t)rbseg + drb, cts = (int64_t)c.ct + dct;
    if (rbs < 0 || (uint64_t)rbs >= S.nrb || cts < 0 || (uint64_t)cts >= S.nct) continue;
    const uint64_t pi = sx == 0 ? (uint64_t)((Ps - 1) >> 1) : (uint64_t)Ps;
    const uint64_t g = seg_id(S, pi, (uint64_t)rbs, (uint64_t)cts);
    const StagePlanes& SQ = L.sp[sx];
    const uint64_t cofs = SQ.cap0 + (uint64_t)k * SQ.pcap + g * (uint64_t)S.RB * S.CW;
    const uint64_t bofs = SQ.bm0 + (uint64_t)k * SQ.pbm + g * S.bw;
    SP[s][sl][i] = cap + cofs;
    const uint32_t* bp = bm + bofs;
    if (IPC_IN(L, cofs + (uint64_t)S.RB * S.CW - 1, L.lim_cap, kSiteStageCap) &&
        IPC_IN(L, bofs + S.bw - 1, L.lim_bm, kSiteStageBm)) {
      for (int v = 0; v < (int)S.bw; ++v) cp_async4(&SB[s][sl][i][v], bp + v);
    } else {
      for (int v = 0; v < (int)S.bw; ++v) SB[s][sl][i][v] = 0u;  // (checked build) nothing read
    }
  }

  // Phase 1a: even value rows -- the sweep-0 predictions of an odd plane
  // (its codes are added in phase 1b), or the known points of an even plane.
  // Own code columns go in pairs (2p, 2p+1) to the sub-tile's threads
  // p = ltid % (HC/2); the first half of them take the upper rows, the other
  // the lower rows. At stride 1 the two values of a pair (and the elements
  // between and after them) are one 16-byte load per plane. The three halo
  // columns are spread over the sub-tile's threads.
  const bool has0 = S0.out_end > S0.out_begin;
  constexpr int NP = G::HC / 2;                        // pairs per row
  const int pp = ltid % NP, jsp = 2 * pp;              // the pair's first code column
  const bool upper = ltid < NP;
  const int c2p = c.C0 + 2 * jsp;                      // its lattice column
  const bool pa = live && c2p < M2, pb = c2p + 2 < M2;  // columns present
  constexpr int H0A = (G::H0 + 1) / 2, H1A = G::H1 / 2;
  {
    // Known points come from the next coarser level's lattice, stored
    // densely: point (P', c1, c2) (all even) is kin[(P'/2) k0 + (c1/2) k1 +
    // c2/2]. `p` below points at plane P (even plane) or P - 1 (odd plane);
    // planes P + 1, P - 3, P + 3 are k0, -k0, 2 k0 away.
    typedef typename Vec2<T>::type V2;
    const T* kin = reinterpret_cast<const T*>(L.kin);
    const int64_t k0 = L.kst0, k1 = L.kst1;
    const bool r1 = c.P + 1 <= M0 - 1;
    // far planes read: Eq. 2 needs both, the quadratic the one that exists
    const bool r3 = interp != 0 && c.P - 3 >= 0 && c.P + 3 <= M0 - 1;
    const bool ra = Q && interp == 2 ? r1 && c.P - 3 >= 0 : r3;
    const bool rd = Q && interp == 2 ? c.P + 3 <= M0 - 1 : r3;
    // known-point loads (the checked build tests each against the lattice)
    auto kload = [&](const T* q) -> T {
      return IPC_IN(L, q - kin, L.lim_kin, kSiteKnown) ? __ldg(q) : (T)0;
    };
    auto kload2 = [&](const T* q) -> V2 {
      return IPC_IN(L, q + 1 - kin, L.lim_kin, kSiteKnown) ? __ldg(reinterpret_cast<const V2*>(q))
                                                           : V2{};
    };
    auto one = [&](const T* p) -> T {
      if (!podd) return kload(p);
      const T bb = kload(p);
      const T cc = r1 ? kload(p + k0) : bb;
      const T a = ra ? kload(p - k0) : bb;
      const T d = rd ? kload(p + 2 * k0) : bb;
      return pred4<T, Q>(a, bb, cc, d, c.P, M0, interp);
    };
    const T* kplane = kin + (int64_t)(c.P >> 1) * k0;
    if (pa) {
      const int jr0 = upper ? 0 : H0A, jr1 = upper ? H0A : G::H0;
      const T* colp = kplane + (c2p >> 1);
      // the pair's two known points are consecutive elements: one 8-byte
      // (16-byte for double) load per plane when every row and plane offset
      // keeps that alignment
      const bool vec = pb && (k1 & 1) == 0 && (k0 & 1) == 0 &&
                       ((uintptr_t)colp % (2 * sizeof(T))) == 0;
#pragma unroll
      for (int q = 0; q < H0A; ++q) {
        const int jr = jr0 + q;
        if (jr >= jr1) break;
        const int c1 = c.R0 - 2 + 2 * jr;
        if (c1 < 0 || c1 >= M1) continue;
        const T* p = colp + (int64_t)(c1 >> 1) * k1;
        V2 v2;
        if (vec) {
          if (!podd) {
            v2 = kload2(p);
          } else {
            const V2 bb = kload2(p);
            const V2 cc = r1 ? kload2(p + k0) : bb;
            const V2 a = ra ? kload2(p - k0) : bb;
            const V2 d = rd ? kload2(p + 2 * k0) : bb;
            v2.x = pred4<T, Q>(a.x, bb.x, cc.x, d.x, c.P, M0, interp);
            v2.y = pred4<T, Q>(a.y, bb.y, cc.y, d.y, c.P, M0, interp);
          }
        } else {
          v2.x = one(p);
          v2.y = pb ? one(p + 1) : v2.x;
        }
        *reinterpret_cast<V2*>(VE + (2 * jr) * G::VP + G::V0 + jsp) = v2;
      }
    }
    if (live && ltid < 3 * G::H0) {
      const int h = ltid / G::H0, jr = ltid - h * G::H0;
      const int js = h == 0 ? -1 : G::HC + h - 1;
      const int c1 = c.R0 - 2 + 2 * jr, c2 = c.C0 + 2 * js;
      if (c1 >= 0 && c1 < M1 && c2 >= 0 && c2 < M2 && c2 <= c.C1 + 2)
        VE[(2 * jr) * G::VP + G::V0 + js] = one(kplane + (int64_t)(c1 >> 1) * k1 + (c2 >> 1));
    }
  }
  cp_async_wait_all();
  __syncthreads();

  // Phase 0: decode the words of the sub-tiles' code columns (items of all
  // sub-tiles in one list).
  constexpr int MAXIT = (BR + G::H1 + G::H0) * G::CWD + 2 * (G::H1 + G::H0);
  for (int it = tid; it < NS * MAXIT; it += 256) {
    const int s = it / MAXIT, i = it % MAXIT;
    if (P0 + 2 * s >= M0) continue;
    const int cw0 = (int)c.ct * G::CWD;  // first own word of a row
    const int n2r = c.R1 - c.R0, n1r = (c.R1 - c.R0) >> 1;
    const bool st0 = S0.present && podd;
    const int nA = (S2.present && c.ct < S2.nct) ? n2r * G::CWD : 0;
    const int nB = S1.present ? n1r * G::CWD : 0;
    const int nC = st0 ? G::H0 * G::CWD : 0;
    const int nD1 = S1.present ? 2 * n1r : 0;
    const int nD0 = st0 ? 2 * G::H0 : 0;
    if (i >= nA + nB + nC + nD1 + nD0) continue;
    int sx, qrow, side, rr, j;  // side: -1 own word, 0 left / 1 right halo word
    if (i < nA) {
      sx = 2; qrow = i / G::CWD; j = cw0 + i % G::CWD; rr = c.R0 + qrow; side = -1;
    } else if (i < nA + nB) {
      const int u = i - nA;
      sx = 1; qrow = u / G::CWD; j = cw0 + u % G::CWD; rr = (c.R0 >> 1) + qrow; side = -1;
    } else if (i < nA + nB + nC) {
      const int u = i - nA - nB;
      sx = 0; qrow = u / G::CWD; j = cw0 + u % G::CWD; rr = (c.R0 >> 1) - 1 + qrow; side = -1;
    } else if (i < nA + nB + nC + nD1) {
      const int u = i - nA - nB - nC;
      sx = 1; qrow = u >> 1; side = u & 1; rr = (c.R0 >> 1) + qrow;
      j = side ? cw0 + G::CWD : cw0 - 1;
    } else {
      const int u = i - nA - nB - nC - nD1;
      sx = 0; qrow = u >> 1; side = u & 1; rr = (c.R0 >> 1) - 1 + qrow;
      j = side ? cw0 + G::CWD : cw0 - 1;
    }
    const LevelStage& S = L.st[sx];
    if (rr < 0 || (uint64_t)rr >= S.m1 || j < 0 || (uint64_t)j >= S.wr) continue;
    const int RB = sx == 2 ? SR : SR / 2;  // the segment's rows
    const int CW = (int)S.CW;  // G::CWD, or the whole (short) row when nct == 1
    const int ctw = CW == G::CWD ? (int)((unsigned)j / G::CWD) : 0;
    const int rbw = sx == 2 ? (int)((unsigned)rr / SR) : (int)((unsigned)rr / (SR / 2));
    int sl = 0;
    if (KS == 5) {
      if (sx == 1) sl = 1;
      else if (sx == 0) sl = 3 + (rbw - rbseg);
    } else {
      if (sx == 1) sl = 2 + (ctw - (int)c.ct);
      else if (sx == 0) sl = 4 + (rbw - rbseg + 1) * 3 + (ctw - (int)c.ct) + 1;
    }
    const int li = (rr - rbw * RB) * CW + (j - ctw * CW);
    const int wl = li >> 5;
    const uint32_t bit = 1u << (li & 31), below = bit - 1u;
    const uint32_t kmw = (sx == 0 ? km0 : (sx == 1 ? km1 : km2)) >> wb;  // bit i2: plane wb + i2 loaded
    const int bws = b - wb;  // window planes below bws are dropped
    const uint32_t* sb = &SB[s][sl][0][wl];
    const uint32_t* const* sp = SP[s][sl];
    const uint32_t off = (uint32_t)wl * 32;
    uint32_t* QHr = QHof(s) + (sx == 1 ? qrow : G::H1 + qrow) * 4;
    QT* Qr = (sx == 2 ? Q2of(s) : (sx == 1 ? Q1of(s) : Q0of(s))) + qrow * G::QP +
             (j - cw0) * QCfg<W16>::BLK;
    uint32_t a[NPL];
    uint32_t ax[2] = {0u, 0u};  // an increment's prefix digits just above the window
    uint32_t any = 0u;
#pragma unroll
    for (int i2 = 0; i2 < NPL; ++i2) {
      uint32_t w = 0u;
      if ((kmw >> i2) & 1u) {
        const uint32_t m = sb[i2 * BWS];
        if ((m & bit) && IPC_IN(L, (uint64_t)(sp[i2] - cap) + off + __popc(m & below), L.lim_cap,
                                 kSitePlaneWord))
          w = __ldcs(sp[i2] + off + __popc(m & below));  // read once: evict-first
      }
      a[i2] = w;
      any |= w;
    }
    // the word's place in the stage's word grid (the state is indexed by it)
    // and whether this tile owns it (the halo rows of stage 0 belong to the
    // row blocks above and below)
    const uint64_t gw = MODE == kPlain ? 0
        : ((sx == 0 ? (uint64_t)((P0 + 2 * s - 1) >> 1) : (uint64_t)(P0 + 2 * s)) * S.m1 +
           (uint64_t)rr) * S.wr + (uint64_t)j;
    const bool own = side < 0 && (sx != 0 || (2 * rr >= c.R0 && 2 * rr < c.R1));
    const int hi = MODE == kDelta ? L.bo - wb : 0;  // window index of plane bo
    if constexpr (MODE == kDelta) {
      if (L.bo > b) {
        const uint2 cw = *reinterpret_cast<const uint2*>(L.sp[sx].carry_in + 2 * gw);
        // (bit tests rather than index compares keep `a` in registers)
        const uint64_t m0 = 1ull << hi, m1 = 1ull << (hi + 1);
#pragma unroll
        for (int i2 = 0; i2 < NPL; ++i2)
          a[i2] |= (cw.x & (0u - (uint32_t)((m0 >> i2) & 1u))) |
                   (cw.y & (0u - (uint32_t)((m1 >> i2) & 1u)));
        ax[0] = hi == NPL ? cw.x : (hi + 1 == NPL ? cw.y : 0u);
        ax[1] = hi == NPL ? cw.y : (hi == NPL + 1 ? cw.x : 0u);
        any |= cw.x | cw.y;
      }
    }
    if (any == 0u) {
      // every loaded plane word is zero (common when few low planes are
      // loaded): the 32 codes are zero, with no XOR or transpose to undo
      // (and so are the state's new digits)
      if (MODE != kPlain && own && L.sp[sx].carry && (MODE == kRecord || L.bo > b))
        *reinterpret_cast<uint2*>(L.sp[sx].carry + 2 * gw) = make_uint2(0u, 0u);
      if (side < 0) {
        uint4* q = reinterpret_cast<uint4*>(Qr);
#pragma unroll
        for (int m = 0; m < (W16 ? 4 : 8); ++m) q[m] = make_uint4(0u, 0u, 0u, 0u);
      } else if (side) {
        QHr[1] = 0u;
        QHr[2] = 0u;
      } else {
        QHr[0] = 0u;
      }
      continue;
    }
    // inverse predictive XOR, top-down; planes below b are zero, planes
    // above the window are zero
    if constexpr (MODE == kDelta) {
      // only the new planes [b, bo) hold encoded bits; at hi and hi + 1 sit
      // the known digits bo, bo + 1, above them zeros
#pragma unroll
      for (int i2 = NPL - 1; i2 >= 0; --i2) {
        const uint32_t p1 = i2 + 1 < NPL ? a[i2 + 1] : ax[i2 + 1 - NPL];
        const uint32_t p2 = i2 + 2 < NPL ? a[i2 + 2] : ax[i2 + 2 - NPL];
        a[i2] = i2 < bws ? 0u : (i2 < hi ? (a[i2] ^ p1 ^ p2) : a[i2]);
      }
    } else {
#pragma unroll
      for (int i2 = NPL - 1; i2 >= 0; --i2) {
        const uint32_t p1 = i2 + 1 < NPL ? a[i2 + 1] : 0u, p2 = i2 + 2 < NPL ? a[i2 + 2] : 0u;
        a[i2] = i2 >= bws ? (a[i2] ^ p1 ^ p2) : 0u;
      }
    }
    if constexpr (MODE != kPlain) {
      // the state: the digits at planes b and b + 1 (the lowest loaded)
      if (own && L.sp[sx].carry) {
        uint32_t d0 = 0u, d1 = 0u;
        if constexpr (W16 && MODE == kDelta) {
          d0 = a[0];  // window base b (bo - b >= 1, so digit b + 1 is a[1])
          d1 = a[1];
        } else {
          const uint64_t m0 = 1ull << bws, m1 = 1ull << (bws + 1);  // bws <= 32
#pragma unroll
          for (int i2 = 0; i2 < NPL; ++i2) {
            d0 |= a[i2] & (0u - (uint32_t)((m0 >> i2) & 1u));
            d1 |= a[i2] & (0u - (uint32_t)((m1 >> i2) & 1u));
          }
        }
        *reinterpret_cast<uint2*>(L.sp[sx].carry + 2 * gw) = make_uint2(d0, d1);
      }
    }
    if constexpr (MODE == kDelta) {
      // the increment holds the new digits alone
#pragma unroll
      for (int i2 = 0; i2 < NPL; ++i2) a[i2] = i2 < hi ? a[i2] : 0u;
    }
    if (side < 0) {
      if constexpr (W16) {
        transpose16x2(a);
        // code i (i < 16) is the low half of a[i], code 16 + i the high half
        uint4* q = reinterpret_cast<uint4*>(Qr);
#pragma unroll
        for (int m = 0; m < 2; ++m)
          q[m] = make_uint4(__byte_perm(a[8 * m], a[8 * m + 1], 0x5410),
                            __byte_perm(a[8 * m + 2], a[8 * m + 3], 0x5410),
                            __byte_perm(a[8 * m + 4], a[8 * m + 5], 0x5410),
                            __byte_perm(a[8 * m + 6], a[8 * m + 7], 0x5410));
#pragma unroll
        for (int m = 0; m < 2; ++m)
          q[2 + m] = make_uint4(__byte_perm(a[8 * m], a[8 * m + 1], 0x7632),
                                __byte_perm(a[8 * m + 2], a[8 * m + 3], 0x7632),
                                __byte_perm(a[8 * m + 4], a[8 * m + 5], 0x7632),
                                __byte_perm(a[8 * m + 6], a[8 * m + 7], 0x7632));
      } else {
        transpose32(a);
        uint4* q = reinterpret_cast<uint4*>(Qr);
#pragma unroll
        for (int m = 0; m < 8; ++m) q[m] = make_uint4(a[4 * m], a[4 * m + 1], a[4 * m + 2], a[4 * m + 3]);
      }
    } else {
      uint32_t v0 = 0u, v1 = 0u;
      const int i0 = side ? 0 : 31;
#pragma unroll
      for (int i2 = 0; i2 < NPL; ++i2) {
        v0 |= ((a[i2] >> i0) & 1u) << i2;
        v1 |= ((a[i2] >> 1) & 1u) << i2;
      }
      if (side) {
        QHr[1] = v0 << wb;
        QHr[2] = v1 << wb;
      } else {
        QHr[0] = v0 << wb;
      }
    }
  }
  __syncthreads();

  // Phase 1b: the codes of sweep 0 (odd planes), over the items of phase 1a.
  if (podd) {
    auto fix = [&](int jr, int js, T* v) {
      const int c1 = c.R0 - 2 + 2 * jr, c2 = c.C0 + 2 * js;
      const uint64_t ci = ((uint64_t)((c.P - 1) >> 1) * S0.m1 + (uint64_t)(c1 >> 1)) * S0.m2 +
                          (uint64_t)(c2 >> 1);
      find_outlier<T, MODE == kDelta>(S0, oidx, oval, ci, v);
    };
    if (pa) {
      const int jr0 = upper ? 0 : H0A, jr1 = upper ? H0A : G::H0;
#pragma unroll
      for (int q = 0; q < H0A; ++q) {
        const int jr = jr0 + q;
        if (jr >= jr1) break;
        const int c1 = c.R0 - 2 + 2 * jr;
        if (c1 < 0 || c1 >= M1) continue;
        typedef typename Vec2<T>::type V2;
        V2* pv = reinterpret_cast<V2*>(VE + (2 * jr) * G::VP + G::V0 + jsp);
        V2 v = *pv;
        T cv[2];
        scaled_pair(Q0 + jr * G::QP + qoff<W16>(jsp), sc, cv);
        v.x = FP<T>::add(v.x, cv[0]);
        v.y = FP<T>::add(v.y, cv[1]);
        if (has0) {
          fix(jr, jsp, &v.x);
          if (pb) fix(jr, jsp + 1, &v.y);
        }
        *pv = v;
      }
    }
    if (live && ltid < 3 * G::H0) {
      const int h = ltid / G::H0, jr = ltid - h * G::H0;
      const int js = h == 0 ? -1 : G::HC + h - 1;
      const int c1 = c.R0 - 2 + 2 * jr, c2 = c.C0 + 2 * js;
      if (c1 >= 0 && c1 < M1 && c2 >= 0 && c2 < M2 && c2 <= c.C1 + 2) {
        T* p = VE + (2 * jr) * G::VP + G::V0 + js;
        T v = FP<T>::add(*p, FP<T>::mul(code_value(QH[(G::H1 + jr) * 4 + h], T()), twoeb));
        if (has0) fix(jr, js, &v);
        *p = v;
      }
    }
    __syncthreads();  // every thread of the tile sees the same parity
  }

  // Phase 2: sweep 1 on the odd rows, columns [C0-2, C1+2]; pairs of
  // columns as in phase 1, the four row neighbours kept in registers.
  {
    const bool has1 = S1.out_end > S1.out_begin;
    auto value = [&](T a, T bb, T cc, T d, int c1, int c2, T cv) {
      const T pred = pred4<T, Q>(a, bb, cc, d, c1, M1, interp);
      T v = FP<T>::add(pred, cv);
      if (has1) {
        const uint64_t ci = ((uint64_t)c.P * S1.m1 + (uint64_t)((c1 - 1) >> 1)) * S1.m2 +
                            (uint64_t)(c2 >> 1);
        find_outlier<T, MODE == kDelta>(S1, oidx, oval, ci, &v);
      }
      return v;
    };
    if (S1.present && live) {
      if (pa) {
        typedef typename Vec2<T>::type V2;
        const int jr0 = upper ? 0 : H1A, jr1 = upper ? H1A : G::H1;
        T* col = VE + G::V0 + jsp;
        V2 a = *reinterpret_cast<const V2*>(col + (2 * jr0) * G::VP);
        V2 bb = *reinterpret_cast<const V2*>(col + (2 * jr0 + 2) * G::VP);
        V2 cc = *reinterpret_cast<const V2*>(col + (2 * jr0 + 4) * G::VP);
        for (int jr = jr0; jr < jr1; ++jr) {
          const int c1 = c.R0 + 1 + 2 * jr;
          if (c1 >= c.R1) break;
          const V2 d = *reinterpret_cast<const V2*>(col + (2 * jr + 6) * G::VP);
          T cv[2];
          scaled_pair(Q1 + jr * G::QP + qoff<W16>(jsp), sc, cv);
          V2 v;
          v.x = value(a.x, bb.x, cc.x, d.x, c1, c2p, cv[0]);
          v.y = value(a.y, bb.y, cc.y, d.y, c1, c2p + 2, cv[1]);
          *reinterpret_cast<V2*>(col + (2 * jr + 3) * G::VP) = v;
          a = bb;
          bb = cc;
          cc = d;
        }
      }
      if (ltid < 3 * G::H1) {
        const int h = ltid / G::H1, jr = ltid - h * G::H1;
        const int js = h == 0 ? -1 : G::HC + h - 1;
        const int c1 = c.R0 + 1 + 2 * jr, c2 = c.C0 + 2 * js;
        if (c1 < c.R1 && c2 >= 0 && c2 < M2 && c2 <= c.C1 + 2) {
          const T* col = VE + G::V0 + js;
          VE[(2 * jr + 3) * G::VP + G::V0 + js] =
              value(col[(2 * jr) * G::VP], col[(2 * jr + 2) * G::VP], col[(2 * jr + 4) * G::VP],
                    col[(2 * jr + 6) * G::VP], c1, c2,
                    FP<T>::mul(code_value(QH[jr * 4 + h], T()), twoeb));
        }
      }
    }
  }
  __syncthreads();

  // Phase 3: sweep 2 and the output. Thread: four odd columns (code columns
  // 4g .. 4g+3) of the rows rq, rq+4, ... of its sub-tile.
  {
    const bool has2 = S2.out_end > S2.out_begin;
    constexpr int NG = G::HC / 4;  // four-column groups per row
    const int g = ltid % NG, rq = ltid / NG;
    const int c2e = c.C0 + 8 * g;  // first (even) lattice column of the run
    // per odd column k of the run: the form pred4 takes there (pred_rule),
    // RW bits each
    constexpr int RW = Q ? 3 : 2;
    uint32_t rule = 0u;
#pragma unroll
    for (int k = 0; k < 4; ++k) rule |= pred_rule<Q>(c2e + 2 * k + 1, M2, interp) << (RW * k);
    // a quadratic boundary form in the run (only runs at the ends of a row)
    const bool quad = Q && (rule & 04444u) != 0u;
    if (live && c2e < c.C1) {
      for (int lr = rq; lr < BR; lr += 4) {
        const int c1 = c.R0 + lr;
        if (c1 >= c.R1) break;
        T w[9];
        lds9<T>(VE + (lr + 2) * G::VP + G::V0 + 4 * g, w);
        T cv[4];
        scaled_quad(Q2 + lr * G::QP + qoff<W16>(4 * g), sc, cv);
        T v[8];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          // Eq. 2 and Eq. 1 side by side (same operations as pred4), then
          // the rule for this column; no lane takes a separate path (the
          // quadratic forms are redone below).
          const T u = FP<T>::add(w[k + 1], w[k + 2]);
          const T cub = FP<T>::template mul_pow2<-4>(
              FP<T>::sub(FP<T>::mul((T)9, u), FP<T>::add(w[k], w[k + 3])));
          const T lin = FP<T>::template mul_pow2<-1>(u);
          const uint32_t r = rule >> (RW * k) & ((1u << RW) - 1u);
          const T pred = r == 2u ? cub : (r == 1u ? lin : w[k + 1]);
          v[2 * k] = w[k + 1];
          v[2 * k + 1] = FP<T>::add(pred, cv[k]);
        }
        if (quad) {
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const uint32_t r = rule >> (RW * k) & 7u;
            if (r & 4u)
              v[2 * k + 1] =
                  FP<T>::add(quad3<T>(w[k], w[k + 1], w[k + 2], w[k + 3], r == 4u), cv[k]);
          }
        }
        if (has2) {
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int c2o = c2e + 2 * k + 1;
            if (c2o < c.C1) {
              const uint64_t ci =
                  ((uint64_t)c.P * S2.m1 + (uint64_t)c1) * S2.m2 + (uint64_t)((c2o - 1) >> 1);
              find_outlier<T, MODE == kDelta>(S2, oidx, oval, ci, &v[2 * k + 1]);
            }
          }
        }
        if (!IPC_IN(L, c.pbase + (int64_t)c1 * c.rs + (int64_t)(min(c.C1, c2e + 8) - 1) * L.s,
                    L.lim_out, kSiteOut))
          continue;
        if (MODE == kDelta && L.stream_out)
          add_run<T>(out + c.pbase + (int64_t)c1 * c.rs, c2e, c.C1, v);  // level 1: x^ += Delta
        else
          store_run<T>(out + c.pbase + (int64_t)c1 * c.rs, L.s, L.N[2], c2e, c.C1, v,
                       L.stream_out);
      }
    }
  }
}

// 16-bit code rows leave room for four CTAs per SM (three with four
// sub-tiles), 32-bit ones for three.
// Persistent: the grid holds as many CTAs as fit at once; CTA i takes tiles
// i, i + grid, ... (neighbouring CTAs stay on neighbouring tiles).
template <class T, int BR, bool W16>
__host__ __device__ constexpr int retrieve_ctas_per_sm() {
  return W16 || sizeof(T) * BR <= 32 ? 4 : 3;
}

template <class T, int BR, int BC, bool W16, int NS>
size_t smem_retrieve() {
  typedef RTile<BR, BC / NS, W16> G;
  return NS * (sizeof(T) * G::VR * G::VP +
               sizeof(typename QCfg<W16>::QT) * (BR + G::H1 + G::H0) * G::QP + 16 * (G::H1 + G::H0));
}

// CTAs of a persistent launch over `tiles` tiles: all that fit on the
// device at once (SM count of the current device, looked up once).
inline unsigned persistent_grid(uint64_t tiles, int per_sm) {
  static int sms = [] {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
      cudaGetLastError();
      n = 152;
    }
    return n;
  }();
  const uint64_t cap = (uint64_t)sms * per_sm;
  return (unsigned)(tiles < cap ? tiles : cap);
}
// CTAs per SM of a persistent grid: the shape's, within what fits.
inline int grid_per_sm(int want, int most) { return want > 0 && want < most ? want : most; }

// ---------------------------------------------------------------------------
// The recording and incremental forms (single-field launches), instantiated
// by ipc_level_delta.cu (Q = false) and ipc_level_delta_quad.cu (Q = true).
template <class T, int BR, int BC, bool W16, int NS, int MODE, bool Q>
__global__ void __launch_bounds__(256, retrieve_ctas_per_sm<T, BR, W16>()) k_level_retrieve_mode(
    LevelArgs L, T* out, T twoeb, int b, const uint32_t* __restrict__ cap,
    const uint32_t* __restrict__ bm, const uint64_t* __restrict__ oidx,
    const double* __restrict__ oval, uint64_t ntiles) {
  extern __shared__ __align__(16) unsigned char smem[];
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    level_retrieve_body<T, BR, BC, W16, NS, MODE, Q>(L, out, twoeb, b, cap, bm, oidx, oval, t, smem);
    __syncthreads();  // the next tile reuses shared memory
  }
}

template <class T, int BR, int BC, bool W16, int NS, int MODE, bool Q>
cudaError_t run_mode(const LevelArgs& L, void* out, double twoeb, int b, const uint32_t* cap,
                     const uint32_t* bm, const uint64_t* oidx, const double* oval, int per_sm,
                     cudaStream_t st) {
  static const cudaError_t setup = cudaFuncSetAttribute(
      k_level_retrieve_mode<T, BR, BC, W16, NS, MODE, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize,
      (int)smem_retrieve<T, BR, BC, W16, NS>());
  if (setup != cudaSuccess) return setup;
  const uint64_t tiles = retrieve_tiles(L, NS);
  if (tiles == 0) return cudaSuccess;
  k_level_retrieve_mode<T, BR, BC, W16, NS, MODE, Q>
      <<<persistent_grid(tiles, grid_per_sm(per_sm, retrieve_ctas_per_sm<T, BR, W16>())), 256,
         smem_retrieve<T, BR, BC, W16, NS>(), st>>>(L, (T*)out, (T)twoeb, b, cap, bm, oidx, oval,
                                                    tiles);
  return cudaGetLastError();
}

// BR16 / BR32: tile rows with 16-bit code rows / with 32-bit code rows and
// several planes per tile, as for the plain kernels.
template <class T, int BR16, int BR32, int BC, int MODE, bool Q>
cudaError_t dispatch_mode(const LevelArgs& L, void* out, double twoeb, int b, const uint32_t* cap,
                          const uint32_t* bm, const uint64_t* oidx, const double* oval, int w16,
                          int ns, int per_sm, cudaStream_t st) {
#define IPC_RM(R, W, N) \
  return run_mode<T, R, BC, W, N, MODE, Q>(L, out, twoeb, b, cap, bm, oidx, oval, per_sm, st)
  if (!w16) {
    if (ns == 4) IPC_RM(BR32, false, 4);
    if (ns == 2) IPC_RM(BR32, false, 2);
    IPC_RM(BR16, false, 1);
  }
  if (ns == 4) IPC_RM(BR16, true, 4);
  if (ns == 2) IPC_RM(BR16, true, 2);
  IPC_RM(BR16, true, 1);
#undef IPC_RM
}

template <bool Q>
cudaError_t level_retrieve_mode_impl(int dtype, const LevelArgs& L, void* out, double twoeb,
                                       int b, const uint32_t* cap, const uint32_t* bm,
                                       const uint64_t* oidx, const double* oval, int w16,
                                       RetrieveShape shape, int mode, cudaStream_t st) {
  const int ns = shape.ns ? shape.ns : retrieve_subtiles(L.M[2], w16);
  if (!retrieve_ns_ok(L.M[2], ns)) return cudaErrorInvalidValue;
  if (retrieve_tiles(L, ns) >= (1ULL << 32)) return cudaErrorInvalidValue;  // 32-bit tile ids
  if (mode != kRecord && mode != kDelta) return cudaErrorInvalidValue;
  if (dtype == 0) {
    if (mode == kRecord)
      return dispatch_mode<float, kLevelRowsF32, kLevelRowsF32 / 2, kLevelCols, kRecord, Q>(
          L, out, twoeb, b, cap, bm, oidx, oval, w16, ns, shape.per_sm, st);
    return dispatch_mode<float, kLevelRowsF32, kLevelRowsF32 / 2, kLevelCols, kDelta, Q>(
        L, out, twoeb, b, cap, bm, oidx, oval, w16, ns, shape.per_sm, st);
  }
  if (mode == kRecord)
    return dispatch_mode<double, kLevelRowsF64, kLevelRowsF64, kLevelCols, kRecord, Q>(
        L, out, twoeb, b, cap, bm, oidx, oval, w16, ns, shape.per_sm, st);
  return dispatch_mode<double, kLevelRowsF64, kLevelRowsF64, kLevelCols, kDelta, Q>(
      L, out, twoeb, b, cap, bm, oidx, oval, w16, ns, shape.per_sm, st);
}

}  // namespace
}  // namespace ipc
