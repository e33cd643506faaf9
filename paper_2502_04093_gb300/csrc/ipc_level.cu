// Fused per-level kernels of libipcomp (sm_103a).
//
// One launch per interpolation level l (stride s = 2^(l-1)) runs all of the
// level's sweeps (Sec. 4.1: along dimension 0, then 1, then 2). Work unit
// (one CTA, 256 threads): one plane P of the level lattice (coordinate c0),
// BR consecutive rows (c1) and BC lattice columns (c2). In lattice units
// the known points are those with every coordinate even; sweep 0 predicts
// (odd, even, even), sweep 1 (any, odd, even), sweep 2 (any, any, odd).
//
// The CTA keeps the plane tile in shared memory, split by column parity:
//   VE[c1][even c2] over rows [R0-2, R0+BR+2] and columns [C0-2, C0+BC+2]
//   VO[c1][odd  c2] over its own rows and columns.
// Phase 1: even rows of VE -- the sweep-0 targets of an odd plane (predicted
//          along c0 from the known planes P-3..P+3), or the known points of
//          an even plane.
// Phase 2: odd rows of VE -- sweep 1 (along c1 from phase 1).
// Phase 3: VO -- sweep 2 (along c2 from VE).
// Targets in the halo (rows and columns outside the CTA's own range) are
// recomputed exactly as their owner computes them (same inputs, same
// operations), so no CTA waits for another.
//
// Stream storage: per stage, the CTA's own codes form one "segment"
// (RB rows x CW words of the stage's word grid). Within a segment, every
// group of 32 words (one warp in phase 4) keeps, per plane, its zero-word
// bitmap word and its nonzero words compacted at the group's 32-word slot.
// Retrieval decodes words of its own segments plus the neighbouring
// segments' words that its halo targets need.
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


// Prediction from four lattice neighbours along one dimension (Eq. 1/2 with
// the boundary rule): i is the target's lattice coordinate, M the extent.
template <class T>
__device__ __forceinline__ T pred4(T a, T b, T c, T d, int i, int M, int cubic) {
  if (i + 1 > M - 1) return b;
  if (cubic && i - 3 >= 0 && i + 3 <= M - 1) {
    const T u = FP<T>::add(b, c);
    const T v = FP<T>::add(a, d);
    const T w = FP<T>::mul((T)9, u);
    const T z = FP<T>::sub(w, v);
    return FP<T>::mul(z, (T)0.0625);
  }
  return FP<T>::mul(FP<T>::add(b, c), (T)0.5);
}

// Quantize x against pred (Sec. 4.2.2); returns the code, writes xhat.
template <class T>
__device__ __forceinline__ int32_t quantize(T xv, T pred, const QuantArgs<T>& qa, T* rec,
                                            bool* outlier) {
  const T t = FP<T>::mul(FP<T>::sub(xv, pred), qa.inv2eb);
  *outlier = !(FP<T>::fabs_(t) <= qa.R);
  *rec = xv;
  if (*outlier) return 0;
  int32_t qi;
  const T qf = FP<T>::rint_(t, &qi);
  const T rc = FP<T>::add(pred, FP<T>::mul(qf, qa.twoeb));
  if (FP<T>::fabs_(FP<T>::sub(xv, rc)) <= qa.ebchk) {
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
template <class T>
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
    *v = (T)__ldg(val + lo);
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

template <class T, int BR, int BC, bool W16, int NS>
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
  const int cubic = L.cubic;
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
  const int wb = W16 ? max(0, ktop - 15) : 0;
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
    SP[s][sl][i] = cap + SQ.cap0 + (uint64_t)k * SQ.pcap + g * (uint64_t)S.RB * S.CW;
    const uint32_t* bp = bm + SQ.bm0 + (uint64_t)k * SQ.pbm + g * S.bw;
    for (int v = 0; v < (int)S.bw; ++v) cp_async4(&SB[s][sl][i][v], bp + v);
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
    const bool r3 = cubic && c.P - 3 >= 0 && c.P + 3 <= M0 - 1;
    auto one = [&](const T* p) -> T {
      if (!podd) return __ldg(p);
      const T bb = __ldg(p);
      const T cc = r1 ? __ldg(p + k0) : bb;
      const T a = r3 ? __ldg(p - k0) : bb;
      const T d = r3 ? __ldg(p + 2 * k0) : bb;
      return pred4<T>(a, bb, cc, d, c.P, M0, cubic);
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
          const V2* p2 = reinterpret_cast<const V2*>(p);
          if (!podd) {
            v2 = __ldg(p2);
          } else {
            const V2 bb = __ldg(p2);
            const V2 cc = r1 ? __ldg(reinterpret_cast<const V2*>(p + k0)) : bb;
            const V2 a = r3 ? __ldg(reinterpret_cast<const V2*>(p - k0)) : bb;
            const V2 d = r3 ? __ldg(reinterpret_cast<const V2*>(p + 2 * k0)) : bb;
            v2.x = pred4<T>(a.x, bb.x, cc.x, d.x, c.P, M0, cubic);
            v2.y = pred4<T>(a.y, bb.y, cc.y, d.y, c.P, M0, cubic);
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
    uint32_t any = 0u;
#pragma unroll
    for (int i2 = 0; i2 < NPL; ++i2) {
      uint32_t w = 0u;
      if ((kmw >> i2) & 1u) {
        const uint32_t m = sb[i2 * BWS];
        if (m & bit) w = __ldcs(sp[i2] + off + __popc(m & below));  // read once: evict-first
      }
      a[i2] = w;
      any |= w;
    }
    if (any == 0u) {
      // every loaded plane word is zero (common when few low planes are
      // loaded): the 32 codes are zero, with no XOR or transpose to undo
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
#pragma unroll
    for (int i2 = NPL - 1; i2 >= 0; --i2) {
      const uint32_t p1 = i2 + 1 < NPL ? a[i2 + 1] : 0u, p2 = i2 + 2 < NPL ? a[i2 + 2] : 0u;
      a[i2] = i2 >= bws ? (a[i2] ^ p1 ^ p2) : 0u;
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
      find_outlier<T>(S0, oidx, oval, ci, v);
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
      const T pred = pred4<T>(a, bb, cc, d, c1, M1, cubic);
      T v = FP<T>::add(pred, cv);
      if (has1) {
        const uint64_t ci = ((uint64_t)c.P * S1.m1 + (uint64_t)((c1 - 1) >> 1)) * S1.m2 +
                            (uint64_t)(c2 >> 1);
        find_outlier<T>(S1, oidx, oval, ci, &v);
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
    // per odd column k of the run: 2 = cubic, 1 = linear, 0 = copy (the
    // boundary rule of pred4), two bits each
    uint32_t rule = 0u;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int i = c2e + 2 * k + 1;
      const uint32_t r = i + 1 > M2 - 1 ? 0u : ((cubic && i - 3 >= 0 && i + 3 <= M2 - 1) ? 2u : 1u);
      rule |= r << (2 * k);
    }
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
          // the rule for this column; no lane takes a separate path.
          const T u = FP<T>::add(w[k + 1], w[k + 2]);
          const T cub = FP<T>::mul(FP<T>::sub(FP<T>::mul((T)9, u), FP<T>::add(w[k], w[k + 3])),
                                   (T)0.0625);
          const T lin = FP<T>::mul(u, (T)0.5);
          const uint32_t r = rule >> (2 * k) & 3u;
          const T pred = r == 2u ? cub : (r == 1u ? lin : w[k + 1]);
          v[2 * k] = w[k + 1];
          v[2 * k + 1] = FP<T>::add(pred, cv[k]);
        }
        if (has2) {
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int c2o = c2e + 2 * k + 1;
            if (c2o < c.C1) {
              const uint64_t ci =
                  ((uint64_t)c.P * S2.m1 + (uint64_t)c1) * S2.m2 + (uint64_t)((c2o - 1) >> 1);
              find_outlier<T>(S2, oidx, oval, ci, &v[2 * k + 1]);
            }
          }
        }
        store_run<T>(out + c.pbase + (int64_t)c1 * c.rs, L.s, L.N[2], c2e, c.C1, v, L.stream_out);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Compression of one level.
//
// Same tile and thread mappings as the reconstruction: value rows (even rows
// first, then the odd rows) hold the reconstructed values x^ of the tile and
// its halo; halo targets are recomputed exactly as their owner computes
// them. Codes of the CTA's own points go to code rows (32-bit, blocked).
// Phase 1: even value rows: sweep 0 of an odd plane (quantized against the
//   prediction from the known planes P +- 1, P +- 3) or the known points.
// Phase 2: odd value rows (sweep 1).
// Phase 3: sweep 2, four odd columns per thread; when the next level needs
//   them, the level's values are stored as runs of eight elements.
// Phase 4: per 32-code word, the bitplane transpose (two 16x16 transposes
//   when the warp's codes fit in 16 bits), the predictive XOR on the plane
//   words, and per 32-word group the zero-word bitmap and the compacted
//   nonzero words of every plane.
// ---------------------------------------------------------------------------
template <int BR, int BC>
struct CTile {
  static constexpr int HC = BC / 2;
  static constexpr int CWD = BC / 64;
  static constexpr int QP = CWD * 36;    // code-row pitch (32-bit codes, blocked)
  static constexpr int H0 = BR / 2 + 3;  // even value rows: c1 = R0-2+2j
  static constexpr int H1 = BR / 2;      // odd value rows: c1 = R0+1+2j
  static constexpr int V0 = 4;           // value column of code column 0
  static constexpr int VP = HC + 8;      // value-row pitch
  __device__ static int even_row(int j) { return j * VP; }
  __device__ static int odd_row(int j) { return (H0 + j) * VP; }
  // value row of lattice row c1 = R0 + lr (own rows)
  __device__ static int own_row(int lr) {
    return (lr & 1) ? odd_row((lr - 1) >> 1) : even_row((lr >> 1) + 1);
  }
};

template <class T, int BR, int BC>
__device__ __forceinline__ void level_compress_body(const LevelArgs& L, const T* __restrict__ x,
                                                    T* xh, int write_xh, const QuantArgs<T>& qa,
                                                    const SweepOut& o, const LevelDescs& D,
                                                    uint64_t cta, unsigned char* smem) {
  typedef CTile<BR, BC> G;
  typedef typename Vec2<T>::type V2;
  static_assert(G::HC == 256, "one thread per code column of a tile row");
  T* VE = reinterpret_cast<T*>(smem);                                // [H0 + H1][VP]
  uint32_t* E2 = reinterpret_cast<uint32_t*>(VE + (G::H0 + G::H1) * G::VP);  // [BR][QP]
  uint32_t* E1 = E2 + BR * G::QP;                                    // [H1][QP]
  uint32_t* E0 = E1 + G::H1 * G::QP;                                 // [BR/2][QP]

  const CtaPos c = cta_pos(L, cta, BR, BC);
  const bool podd = (c.P & 1) != 0;
  const int tid = threadIdx.x;
  const int cubic = L.cubic;
  const int M0 = (int)L.M[0], M1 = (int)L.M[1], M2 = (int)L.M[2];
  const LevelStage &S0 = L.st[0], &S1 = L.st[1], &S2 = L.st[2];
  uint32_t orN[3] = {0, 0, 0}, qmx[3] = {0, 0, 0};
  auto stat = [&](int st, int32_t q) {
    orN[st] |= negabinary(q);
    qmx[st] = max(qmx[st], (uint32_t)(q < 0 ? -q : q));
  };

  // codes outside the grid (edge tiles) must read as zero in phase 4
  if (c.R1 - c.R0 < BR || c.C1 - c.C0 < BC)
    for (int i = tid; i < (BR + G::H1 + BR / 2) * G::QP; i += 256) E2[i] = 0;
  __syncthreads();

  const int pp = tid & 127, jsp = 2 * pp;  // code-column pair of the thread
  const int c2p = c.C0 + 2 * jsp;
  const bool pa = c2p < M2, pb = c2p + 2 < M2;
  constexpr int H0A = (G::H0 + 1) / 2, H1A = G::H1 / 2;
  // 16-byte loads of x / x^ rows: float, stride 1, four elements inside the
  // row, rows and planes multiples of four elements apart
  const int64_t so = L.s * L.stride[0];
  const bool vec = sizeof(T) == 4 && L.s == 1 && c2p + 3 < M2 && (so & 3) == 0 &&
                   (c.rs & 3) == 0 && ((uintptr_t)(x + c.pbase + c2p) & 15) == 0;
  // Known points: the next coarser level's lattice stored densely, point
  // (P', c1, c2) (all even) at kin[(P'/2) k0 + (c1/2) k1 + c2/2]; `kp` points
  // at plane P (even plane) or P - 1 (odd plane) -- planes P + 1, P - 3,
  // P + 3 are k0, -k0, 2 k0 away.
  const T* kin = reinterpret_cast<const T*>(L.kin);
  const int64_t k0 = L.kst0, k1 = L.kst1;
  const T* kplane = kin + (int64_t)(c.P >> 1) * k0;
  const bool veck = pb && (k1 & 1) == 0 && (k0 & 1) == 0 &&
                    ((uintptr_t)(kplane + (c2p >> 1)) % (2 * sizeof(T))) == 0;

  // Phase 1: even value rows.
  {
    const bool r1 = c.P + 1 <= M0 - 1;
    const bool r3 = cubic && c.P - 3 >= 0 && c.P + 3 <= M0 - 1;
    // one point: value (quantized for an odd plane), code and bookkeeping
    auto point = [&](T pred, T xv, int c1, int c2, bool own, T* v) {
      bool outl;
      T rec;
      const int32_t q = quantize<T>(xv, pred, qa, &rec, &outl);
      *v = rec;
      if (own) {
        stat(0, q);
        E0[((c1 - c.R0) >> 1) * G::QP + qoff<false>((c2 - c.C0) >> 1)] = negabinary(q);
        if (outl)
          record_outlier(o, S0.t,
                         ((uint64_t)((c.P - 1) >> 1) * S0.m1 + (uint64_t)(c1 >> 1)) * S0.m2 +
                             (uint64_t)(c2 >> 1),
                         (double)xv);
      }
    };
    auto one = [&](int c1, int c2, bool own) -> T {
      const T* p = kplane + (int64_t)(c1 >> 1) * k1 + (c2 >> 1);
      if (!podd) return __ldg(p);
      const T bb = __ldg(p);
      const T cc = r1 ? __ldg(p + k0) : bb;
      const T a = r3 ? __ldg(p - k0) : bb;
      const T d = r3 ? __ldg(p + 2 * k0) : bb;
      T v;
      point(pred4<T>(a, bb, cc, d, c.P, M0, cubic),
            __ldg(x + c.pbase + (int64_t)c1 * c.rs + (int64_t)c2 * L.s), c1, c2, own, &v);
      return v;
    };
    if (pa) {
      const int jr0 = tid < 128 ? 0 : H0A, jr1 = tid < 128 ? H0A : G::H0;
#pragma unroll
      for (int q = 0; q < H0A; ++q) {
        const int jr = jr0 + q;
        if (jr >= jr1) break;
        const int c1 = c.R0 - 2 + 2 * jr;
        if (c1 < 0 || c1 >= M1) continue;
        const bool ownr = c1 >= c.R0 && c1 < c.R1;
        T va, vb;
        if (veck) {
          // the pair's known points: consecutive elements (one 8-byte load
          // per plane for float); x: one 16-byte load at stride 1
          const V2* p2 = reinterpret_cast<const V2*>(kplane + (int64_t)(c1 >> 1) * k1 + (c2p >> 1));
          if (!podd) {
            const V2 k = __ldg(p2);
            va = k.x;
            vb = k.y;
          } else {
            const V2 bb = __ldg(p2);
            const V2 cc = r1 ? __ldg(p2 + k0 / 2) : bb;
            const V2 a = r3 ? __ldg(p2 - k0 / 2) : bb;
            const V2 d = r3 ? __ldg(p2 + k0) : bb;
            const int64_t e = c.pbase + (int64_t)c1 * c.rs + (int64_t)c2p * L.s;
            T xa, xb;
            if (vec) {
              const float4 xv = __ldg(reinterpret_cast<const float4*>(reinterpret_cast<const float*>(x) + e));
              xa = (T)xv.x;
              xb = (T)xv.z;
            } else {
              xa = __ldg(x + e);
              xb = __ldg(x + e + 2 * L.s);
            }
            point(pred4<T>(a.x, bb.x, cc.x, d.x, c.P, M0, cubic), xa, c1, c2p, ownr, &va);
            point(pred4<T>(a.y, bb.y, cc.y, d.y, c.P, M0, cubic), xb, c1, c2p + 2, ownr, &vb);
          }
        } else {
          va = one(c1, c2p, ownr);
          vb = pb ? one(c1, c2p + 2, ownr) : va;
        }
        V2 v2;
        v2.x = va;
        v2.y = vb;
        *reinterpret_cast<V2*>(VE + G::even_row(jr) + G::V0 + jsp) = v2;
      }
    }
    if (tid < 3 * G::H0) {
      const int h = tid / G::H0, jr = tid - h * G::H0;
      const int js = h == 0 ? -1 : G::HC + h - 1;
      const int c1 = c.R0 - 2 + 2 * jr, c2 = c.C0 + 2 * js;
      if (c1 >= 0 && c1 < M1 && c2 >= 0 && c2 < M2 && c2 <= c.C1 + 2)
        VE[G::even_row(jr) + G::V0 + js] = one(c1, c2, false);
    }
  }
  __syncthreads();

  // Phase 2: sweep 1 on the odd rows, columns [C0-2, C1+2].
  if (S1.present) {
    auto point = [&](T a, T bb, T cc, T d, int c1, int c2, bool own, T xv) -> T {
      const T pred = pred4<T>(a, bb, cc, d, c1, M1, cubic);
      bool outl;
      T rec;
      const int32_t q = quantize<T>(xv, pred, qa, &rec, &outl);
      if (own) {
        stat(1, q);
        E1[((c1 - c.R0 - 1) >> 1) * G::QP + qoff<false>((c2 - c.C0) >> 1)] = negabinary(q);
        if (outl)
          record_outlier(o, S1.t,
                         ((uint64_t)c.P * S1.m1 + (uint64_t)((c1 - 1) >> 1)) * S1.m2 +
                             (uint64_t)(c2 >> 1),
                         (double)xv);
      }
      return rec;
    };
    if (pa) {
      const int jr0 = tid < 128 ? 0 : H1A, jr1 = tid < 128 ? H1A : G::H1;
      const T* col = VE + G::V0 + jsp;
      V2 a = *reinterpret_cast<const V2*>(col + G::even_row(jr0));
      V2 bb = *reinterpret_cast<const V2*>(col + G::even_row(jr0 + 1));
      V2 cc = *reinterpret_cast<const V2*>(col + G::even_row(jr0 + 2));
#pragma unroll
      for (int q = 0; q < (G::H1 + 1) / 2; ++q) {
        const int jr = jr0 + q;
        if (jr >= jr1) break;
        const int c1 = c.R0 + 1 + 2 * jr;
        if (c1 >= c.R1) break;
        const V2 d = *reinterpret_cast<const V2*>(col + G::even_row(jr + 3));
        const int64_t e = c.pbase + (int64_t)c1 * c.rs + (int64_t)c2p * L.s;
        T xa, xb;
        if (vec) {
          const float4 xv = __ldg(reinterpret_cast<const float4*>(reinterpret_cast<const float*>(x) + e));
          xa = (T)xv.x;
          xb = (T)xv.z;
        } else {
          xa = __ldg(x + e);
          xb = pb ? __ldg(x + e + 2 * L.s) : xa;
        }
        V2 v;
        v.x = point(a.x, bb.x, cc.x, d.x, c1, c2p, true, xa);
        v.y = pb ? point(a.y, bb.y, cc.y, d.y, c1, c2p + 2, true, xb) : v.x;
        *reinterpret_cast<V2*>(VE + G::odd_row(jr) + G::V0 + jsp) = v;
        a = bb;
        bb = cc;
        cc = d;
      }
    }
    if (tid < 3 * G::H1) {
      const int h = tid / G::H1, jr = tid - h * G::H1;
      const int js = h == 0 ? -1 : G::HC + h - 1;
      const int c1 = c.R0 + 1 + 2 * jr, c2 = c.C0 + 2 * js;
      if (c1 < c.R1 && c2 >= 0 && c2 < M2 && c2 <= c.C1 + 2) {
        const T* col = VE + G::V0 + js;
        VE[G::odd_row(jr) + G::V0 + js] =
            point(col[G::even_row(jr)], col[G::even_row(jr + 1)], col[G::even_row(jr + 2)],
                  col[G::even_row(jr + 3)], c1, c2, false,
                  __ldg(x + c.pbase + (int64_t)c1 * c.rs + (int64_t)c2 * L.s));
      }
    }
  }
  __syncthreads();

  // Phase 3: sweep 2 (four odd columns per thread) and the level's values.
  {
    const int g = tid & 63, rq = tid >> 6;
    const int c2e = c.C0 + 8 * g;
    uint32_t rule = 0u;  // per odd column: 2 cubic, 1 linear, 0 copy
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int i = c2e + 2 * k + 1;
      const uint32_t r = i + 1 > M2 - 1 ? 0u : ((cubic && i - 3 >= 0 && i + 3 <= M2 - 1) ? 2u : 1u);
      rule |= r << (2 * k);
    }
    const bool vec8 = vec && c2e + 8 <= M2 && ((uintptr_t)(x + c.pbase + c2e) & 15) == 0;
    if (c2e < c.C1) {
      for (int lr = rq; lr < BR; lr += 4) {
        const int c1 = c.R0 + lr;
        if (c1 >= c.R1) break;
        T w[9];
        lds9<T>(VE + G::own_row(lr) + G::V0 + 4 * g, w);
        const int64_t e = c.pbase + (int64_t)c1 * c.rs;
        T xo[4];
        if (vec8) {
          const float4* xp = reinterpret_cast<const float4*>(reinterpret_cast<const float*>(x) + e + c2e);
          const float4 u = __ldg(xp), v = __ldg(xp + 1);
          xo[0] = (T)u.y;
          xo[1] = (T)u.w;
          xo[2] = (T)v.y;
          xo[3] = (T)v.w;
        } else {
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int c2o = c2e + 2 * k + 1;
            xo[k] = c2o < c.C1 ? __ldg(x + e + (int64_t)c2o * L.s) : (T)0;
          }
        }
        T v[8];
        uint32_t n[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int c2o = c2e + 2 * k + 1;
          const T u = FP<T>::add(w[k + 1], w[k + 2]);
          const T cub = FP<T>::mul(FP<T>::sub(FP<T>::mul((T)9, u), FP<T>::add(w[k], w[k + 3])),
                                   (T)0.0625);
          const T lin = FP<T>::mul(u, (T)0.5);
          const uint32_t r = rule >> (2 * k) & 3u;
          const T pred = r == 2u ? cub : (r == 1u ? lin : w[k + 1]);
          bool outl;
          T rec;
          const int32_t q = quantize<T>(xo[k], pred, qa, &rec, &outl);
          v[2 * k] = w[k + 1];
          v[2 * k + 1] = rec;
          n[k] = 0u;
          if (c2o < c.C1) {
            n[k] = negabinary(q);
            stat(2, q);
            if (outl)
              record_outlier(o, S2.t,
                             ((uint64_t)c.P * S2.m1 + (uint64_t)c1) * S2.m2 + (uint64_t)((c2o - 1) >> 1),
                             (double)xo[k]);
          }
        }
        *reinterpret_cast<uint4*>(E2 + lr * G::QP + qoff<false>(4 * g)) = make_uint4(n[0], n[1], n[2], n[3]);
        if (write_xh) store_run<T>(xh + (int64_t)c.P * L.ost0 + (int64_t)c1 * L.ost1, 1, 0, c2e, c.C1, v);
      }
    }
  }
  __syncthreads();

  // Phase 4: bitplane transpose and compaction of the three segments.
  // Threads [0,128) words of stage 2, [128,192) stage 1, [192,256) stage 0.
  const int lane = tid & 31;
  int sidx, li;
  if (tid < 128) { sidx = 2; li = tid; }
  else if (tid < 192) { sidx = 1; li = tid - 128; }
  else { sidx = 0; li = tid - 192; }
  const LevelStage& S = L.st[sidx];
  int nrows;  // rows of this stage owned by the CTA
  if (sidx == 2) nrows = c.R1 - c.R0;
  else if (sidx == 1) nrows = (c.R1 - c.R0) >> 1;
  else nrows = podd ? (c.R1 - c.R0 + 1) >> 1 : 0;
  const int RB = sidx == 2 ? BR : BR / 2;
  const int CW = (int)S.CW;
  const bool active = S.present && nrows > 0 && c.rb < S.nrb && c.ct < S.nct;
  const int nwords = RB * CW;
  const bool mine = active && li < nwords;
  uint32_t cd[32];  // the word's codes, then its plane words
  uint32_t cor = 0u;
  {
    const uint32_t* Eb = sidx == 2 ? E2 : (sidx == 1 ? E1 : E0);
    const int lr = mine ? li / CW : 0, lj = mine ? li - lr * CW : 0;
    const uint4* src = reinterpret_cast<const uint4*>(Eb + lr * G::QP + lj * 36);
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const uint4 u = mine ? src[m] : make_uint4(0u, 0u, 0u, 0u);
      cd[4 * m] = u.x;
      cd[4 * m + 1] = u.y;
      cd[4 * m + 2] = u.z;
      cd[4 * m + 3] = u.w;
      cor |= u.x | u.y | u.z | u.w;
    }
  }
  const uint32_t wor = __reduce_or_sync(~0u, cor);  // top plane of the warp's words
  if ((wor >> 16) == 0u) {
    // codes below 2^16: planes 16..31 are zero
    uint32_t w[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) w[i] = cd[i] | (cd[16 + i] << 16);
    transpose16x2<false>(w);
#pragma unroll
    for (int k = 0; k < 16; ++k) cd[k] = w[k];
#pragma unroll
    for (int k = 16; k < 32; ++k) cd[k] = 0u;
  } else {
    transpose32<false>(cd);
  }
  xor_encode_planes(cd);
  const uint64_t pi = sidx == 0 ? (uint64_t)((c.P - 1) >> 1) : (uint64_t)c.P;
  const uint64_t gseg = active ? seg_id(S, pi, c.rb, c.ct) : 0;
  const uint32_t bwords = (uint32_t)((nwords + 31) / 32);
  const PlaneDesc* pds = D.s[sidx].p;
  const int wl = li >> 5;  // 32-word group of the segment (one warp)
  const bool wact = active && wl < (int)bwords;
  __shared__ uint32_t scnt[3][32];
  if (tid < 96) scnt[tid >> 5][tid & 31] = 0;
#pragma unroll
  for (int st = 0; st < 3; ++st) {
    const uint32_t a = __reduce_or_sync(~0u, orN[st]);
    const uint32_t m = __reduce_max_sync(~0u, qmx[st]);
    if (lane == 0) {
      if (a) atomicOr(o.stat + 2 * L.st[st].t, a);
      if (m) atomicMax(o.stat + 2 * L.st[st].t + 1, m);
    }
  }
  __syncthreads();
  const uint32_t lt = lanemask_lt();
  const uint64_t capg = gseg * (uint64_t)nwords + (uint64_t)wl * 32;
  const int ktop = wor ? 31 - __clz((int)wor) : -1;  // XOR encoding keeps the top plane
  uint32_t mybm = 0u;  // the bitmap word of plane `lane`
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    if (k > ktop) break;
    const uint32_t mk = __ballot_sync(~0u, cd[k] != 0u);
    if (lane == k) mybm = mk;
    if (wact && cd[k]) o.cap[pds[k].cap_off + capg + __popc(mk & lt)] = cd[k];
  }
  if (wact) {
    o.bm[pds[lane].bm_off + gseg * S.bw + wl] = mybm;
    if (mybm) atomicAdd(&scnt[sidx][lane], (uint32_t)__popc(mybm));
  }
  __syncthreads();
  if (tid < 96) {
    const uint32_t n = scnt[tid >> 5][tid & 31];
    if (n) atomicAdd(o.nnz + 32 * L.st[tid >> 5].t + (tid & 31), n);
  }
}

// Single-field kernels: arguments in the parameter space. Four CTAs of the
// compression fit per SM (64 registers, all of the SM's shared memory); the
// batched kernel, whose arguments come from global memory, keeps three.
template <class T, int BR, int BC>
__global__ void __launch_bounds__(256, 4) k_level_compress(LevelArgs L, const T* __restrict__ x,
                                                           T* xh, int write_xh, QuantArgs<T> qa,
                                                           SweepOut o, LevelDescs D) {
  extern __shared__ __align__(16) unsigned char smem[];
  level_compress_body<T, BR, BC>(L, x, xh, write_xh, qa, o, D, blockIdx.x, smem);
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
__global__ void __launch_bounds__(256, retrieve_ctas_per_sm<T, BR, W16>()) k_level_retrieve(
    LevelArgs L, T* out, T twoeb, int b, const uint32_t* __restrict__ cap,
    const uint32_t* __restrict__ bm, const uint64_t* __restrict__ oidx,
    const double* __restrict__ oval, uint64_t ntiles) {
  extern __shared__ __align__(16) unsigned char smem[];
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    level_retrieve_body<T, BR, BC, W16, NS>(L, out, twoeb, b, cap, bm, oidx, oval, t, smem);
    __syncthreads();  // the next tile reuses shared memory
  }
}

// Batched kernels: one grid covers the level's CTAs of every field of a
// batch; entry i owns CTAs [cta_begin_i, cta_begin_{i+1}).
template <class E>
__device__ __forceinline__ const E& find_entry(const E* __restrict__ ents, int n, uint64_t tile) {
  __shared__ int sel;
  if (threadIdx.x == 0) {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (ents[mid].cta_begin <= tile) lo = mid;
      else hi = mid;
    }
    sel = lo;
  }
  __syncthreads();
  return ents[sel];
}

template <class T, int BR, int BC>
__global__ void __launch_bounds__(256, 3) k_level_compress_batch(
    const CompressEntry* __restrict__ ents, int n) {
  extern __shared__ __align__(16) unsigned char smem[];
  const CompressEntry& e = find_entry(ents, n, blockIdx.x);
  level_compress_body<T, BR, BC>(e.L, (const T*)e.x, (T*)e.xh, e.write_xh,
                                 *reinterpret_cast<const QuantArgs<T>*>(e.quant), e.o, e.D,
                                 blockIdx.x - e.cta_begin, smem);
}

template <class T, int BR, int BC, bool W16, int NS>
__global__ void __launch_bounds__(256, retrieve_ctas_per_sm<T, BR, W16>()) k_level_retrieve_batch(
    const RetrieveEntry* __restrict__ ents, int n, uint64_t ntiles) {
  extern __shared__ __align__(16) unsigned char smem[];
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const RetrieveEntry& e = find_entry(ents, n, t);
    level_retrieve_body<T, BR, BC, W16, NS>(e.L, (T*)e.out, (T)e.twoeb, e.b, e.cap, e.bm, e.oidx,
                                            e.oval, t - e.cta_begin, smem);
    __syncthreads();  // the next tile reuses shared memory (and the entry index)
  }
}

template <class T, int BR, int BC>
size_t smem_compress() {
  typedef CTile<BR, BC> G;
  return sizeof(T) * (G::H0 + G::H1) * G::VP + 4 * (BR + G::H1 + BR / 2) * G::QP;
}
template <class T, int BR, int BC, bool W16, int NS>
size_t smem_retrieve() {
  typedef RTile<BR, BC / NS, W16> G;
  return NS * (sizeof(T) * G::VR * G::VP +
               sizeof(typename QCfg<W16>::QT) * (BR + G::H1 + G::H0) * G::QP + 16 * (G::H1 + G::H0));
}

template <class T, int BR, int BC, bool W16, int NS>
cudaError_t setup_retrieve() {
  cudaError_t r = cudaFuncSetAttribute(k_level_retrieve<T, BR, BC, W16, NS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem_retrieve<T, BR, BC, W16, NS>());
  if (r == cudaSuccess)
    r = cudaFuncSetAttribute(k_level_retrieve_batch<T, BR, BC, W16, NS>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_retrieve<T, BR, BC, W16, NS>());
  return r;
}

template <class T, int BR, int BC>
cudaError_t setup_once() {
  static cudaError_t e = [] {
    cudaError_t r = cudaFuncSetAttribute(k_level_compress<T, BR, BC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_compress<T, BR, BC>());
    if (r == cudaSuccess)
      r = cudaFuncSetAttribute(k_level_compress<T, BR, BC>,
                               cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared);
    if (r == cudaSuccess)
      r = cudaFuncSetAttribute(k_level_compress_batch<T, BR, BC>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem_compress<T, BR, BC>());
    if (r == cudaSuccess) r = setup_retrieve<T, BR, BC, true, 1>();
    if (r == cudaSuccess) r = setup_retrieve<T, BR, BC, true, 2>();
    if (r == cudaSuccess) r = setup_retrieve<T, BR, BC, true, 4>();
    constexpr int BR32 = sizeof(T) == 4 ? BR / 2 : BR;  // rows of 32-bit-code tiles, ns > 1
    if (r == cudaSuccess) r = setup_retrieve<T, BR, BC, false, 1>();
    if (r == cudaSuccess) r = setup_retrieve<T, BR32, BC, false, 2>();
    if (r == cudaSuccess) r = setup_retrieve<T, BR32, BC, false, 4>();
    return r;
  }();
  return e;
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

template <class T, int BR, int BC, bool W16, int NS>
void retrieve_kernel(const LevelArgs& L, void* out, double twoeb, int b, const uint32_t* cap,
                     const uint32_t* bm, const uint64_t* oidx, const double* oval, int per_sm,
                     cudaStream_t st) {
  const uint64_t tiles = retrieve_tiles(L, NS);
  if (tiles == 0) return;
  k_level_retrieve<T, BR, BC, W16, NS>
      <<<persistent_grid(tiles, grid_per_sm(per_sm, retrieve_ctas_per_sm<T, BR, W16>())), 256,
         smem_retrieve<T, BR, BC, W16, NS>(), st>>>(L, (T*)out, (T)twoeb, b, cap, bm, oidx, oval,
                                                    tiles);
}
template <class T, int BR, int BC, bool W16, int NS>
void retrieve_batch_kernel(const RetrieveEntry* ents, int n, uint64_t tiles, int per_sm,
                           cudaStream_t st) {
  k_level_retrieve_batch<T, BR, BC, W16, NS>
      <<<persistent_grid(tiles, grid_per_sm(per_sm, retrieve_ctas_per_sm<T, BR, W16>())), 256,
         smem_retrieve<T, BR, BC, W16, NS>(), st>>>(ents, n, tiles);
}

// BR16 / BR32: tile rows with 16-bit code rows / with 32-bit code rows and
// several planes per tile (one-plane 32-bit tiles keep BR16 rows).
template <class T, int BR16, int BR32, int BC>
void retrieve_dispatch(const LevelArgs& L, void* out, double twoeb, int b, const uint32_t* cap,
                       const uint32_t* bm, const uint64_t* oidx, const double* oval, int w16,
                       int ns, int per_sm, cudaStream_t st) {
#define IPC_RK(R, W, N) retrieve_kernel<T, R, BC, W, N>(L, out, twoeb, b, cap, bm, oidx, oval, per_sm, st)
  if (!w16) {
    if (ns == 4) IPC_RK(BR32, false, 4);
    else if (ns == 2) IPC_RK(BR32, false, 2);
    else IPC_RK(BR16, false, 1);
  } else if (ns == 4) IPC_RK(BR16, true, 4);
  else if (ns == 2) IPC_RK(BR16, true, 2);
  else IPC_RK(BR16, true, 1);
#undef IPC_RK
}
template <class T, int BR16, int BR32, int BC>
void retrieve_batch_dispatch(const RetrieveEntry* ents, int n, uint64_t tiles, int w16, int ns,
                             int per_sm, cudaStream_t st) {
#define IPC_RB(R, W, N) retrieve_batch_kernel<T, R, BC, W, N>(ents, n, tiles, per_sm, st)
  if (!w16) {
    if (ns == 4) IPC_RB(BR32, false, 4);
    else if (ns == 2) IPC_RB(BR32, false, 2);
    else IPC_RB(BR16, false, 1);
  } else if (ns == 4) IPC_RB(BR16, true, 4);
  else if (ns == 2) IPC_RB(BR16, true, 2);
  else IPC_RB(BR16, true, 1);
#undef IPC_RB
}

}  // namespace

int level_rows(int dtype) { return dtype == 0 ? kLevelRowsF32 : kLevelRowsF64; }

cudaError_t launch_level_compress(int dtype, const LevelArgs& L, const void* x, void* xh,
                                  int write_xh, const void* quant, const SweepOut& o,
                                  const LevelDescs& d, cudaStream_t st) {
  const uint64_t grid = (uint64_t)L.M[0] * L.nrb * L.nct;
  if (grid == 0) return cudaSuccess;
  if (grid >= (1ULL << 31)) return cudaErrorInvalidValue;  // grid x limit (tile ids are 32-bit)
  cudaError_t e;
  if (dtype == 0) {
    if ((e = setup_once<float, kLevelRowsF32, kLevelCols>()) != cudaSuccess) return e;
    k_level_compress<float, kLevelRowsF32, kLevelCols>
        <<<(unsigned)grid, 256, smem_compress<float, kLevelRowsF32, kLevelCols>(), st>>>(
            L, (const float*)x, (float*)xh, write_xh, *(const QuantArgs<float>*)quant, o, d);
  } else {
    if ((e = setup_once<double, kLevelRowsF64, kLevelCols>()) != cudaSuccess) return e;
    k_level_compress<double, kLevelRowsF64, kLevelCols>
        <<<(unsigned)grid, 256, smem_compress<double, kLevelRowsF64, kLevelCols>(), st>>>(
            L, (const double*)x, (double*)xh, write_xh, *(const QuantArgs<double>*)quant, o, d);
  }
  return cudaGetLastError();
}

cudaError_t launch_level_retrieve(int dtype, const LevelArgs& L, void* out, double twoeb, int b,
                                  const uint32_t* cap, const uint32_t* bm, const uint64_t* oidx,
                                  const double* oval, int w16, RetrieveShape shape,
                                  cudaStream_t st) {
  const int ns = shape.ns ? shape.ns : retrieve_subtiles(L.M[2], w16);
  if (!retrieve_ns_ok(L.M[2], ns)) return cudaErrorInvalidValue;
  const uint64_t tiles = retrieve_tiles(L, ns);
  if (tiles == 0) return cudaSuccess;
  if (tiles >= (1ULL << 32)) return cudaErrorInvalidValue;  // tile ids are 32-bit
  cudaError_t e;
  if (dtype == 0) {
    if ((e = setup_once<float, kLevelRowsF32, kLevelCols>()) != cudaSuccess) return e;
    retrieve_dispatch<float, kLevelRowsF32, kLevelRowsF32 / 2, kLevelCols>(L, out, twoeb, b, cap, bm, oidx, oval, w16, ns, shape.per_sm, st);
  } else {
    if ((e = setup_once<double, kLevelRowsF64, kLevelCols>()) != cudaSuccess) return e;
    retrieve_dispatch<double, kLevelRowsF64, kLevelRowsF64, kLevelCols>(L, out, twoeb, b, cap, bm, oidx, oval, w16, ns, shape.per_sm, st);
  }
  return cudaGetLastError();
}

cudaError_t launch_level_compress_batch(int dtype, const CompressEntry* ents, int n,
                                        uint64_t ctas, cudaStream_t st) {
  if (ctas == 0 || n == 0) return cudaSuccess;
  if (ctas >= (1ULL << 31)) return cudaErrorInvalidValue;
  cudaError_t e;
  if (dtype == 0) {
    if ((e = setup_once<float, kLevelRowsF32, kLevelCols>()) != cudaSuccess) return e;
    k_level_compress_batch<float, kLevelRowsF32, kLevelCols>
        <<<(unsigned)ctas, 256, smem_compress<float, kLevelRowsF32, kLevelCols>(), st>>>(ents, n);
  } else {
    if ((e = setup_once<double, kLevelRowsF64, kLevelCols>()) != cudaSuccess) return e;
    k_level_compress_batch<double, kLevelRowsF64, kLevelCols>
        <<<(unsigned)ctas, 256, smem_compress<double, kLevelRowsF64, kLevelCols>(), st>>>(ents, n);
  }
  return cudaGetLastError();
}

cudaError_t launch_level_retrieve_batch(int dtype, const RetrieveEntry* ents, int n,
                                        uint64_t tiles, int w16, int ns, int per_sm,
                                        cudaStream_t st) {
  if (tiles == 0 || n == 0) return cudaSuccess;
  if (tiles >= (1ULL << 32)) return cudaErrorInvalidValue;
  cudaError_t e;
  if (dtype == 0) {
    if ((e = setup_once<float, kLevelRowsF32, kLevelCols>()) != cudaSuccess) return e;
    retrieve_batch_dispatch<float, kLevelRowsF32, kLevelRowsF32 / 2, kLevelCols>(ents, n, tiles, w16, ns, per_sm, st);
  } else {
    if ((e = setup_once<double, kLevelRowsF64, kLevelCols>()) != cudaSuccess) return e;
    retrieve_batch_dispatch<double, kLevelRowsF64, kLevelRowsF64, kLevelCols>(ents, n, tiles, w16, ns, per_sm, st);
  }
  return cudaGetLastError();
}

}  // namespace ipc
