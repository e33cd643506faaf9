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

template <int BR, int BC>
struct Tile {
  static constexpr int HC = BC / 2;       // lattice columns of one parity
  static constexpr int CWD = BC / 64;     // words per row of a full tile
  static constexpr int PITCH = HC + CWD;  // code-row pitch (33 words per 32 codes)
  static constexpr int VR = BR + 5;       // VE rows: c1 in [R0-2, R0+BR+2]
  static constexpr int VEC = HC + 3;      // VE columns: even c2 in [C0-2, C0+BC+2]
  static constexpr int QEP = HC + 3 + (HC + 3) / 32 + 1;  // pitch of halo code rows
};

// Swizzled index of code column lc in a code row (one pad word per 32).
__device__ __forceinline__ int sw(int lc) { return lc + (lc >> 5); }

struct CtaPos {
  int P, R0, R1, C0, C1;
  uint64_t rb, ct;
  int64_t pbase;  // element offset of lattice point (P, 0, 0)
  int64_t rs;     // element offset of one lattice row (c1 -> c1 + 1)
};

__device__ __forceinline__ CtaPos cta_pos(const LevelArgs& L, uint64_t cta, int BR, int BC) {
  CtaPos c;
  uint64_t b = cta;
  c.ct = b % L.nct;
  b /= L.nct;
  c.rb = b % L.nrb;
  c.P = (int)(b / L.nrb);
  c.R0 = (int)c.rb * BR;
  c.R1 = (int)min(L.M[1], (int64_t)c.R0 + BR);
  c.C0 = (int)c.ct * BC;
  c.C1 = (int)min(L.M[2], (int64_t)c.C0 + BC);
  c.pbase = (int64_t)c.P * L.stride[0] * L.s;
  c.rs = L.stride[1] * L.s;
  return c;
}

// Element index of lattice point (P, c1, c2) of the CTA's plane.
__device__ __forceinline__ int64_t eidx(const LevelArgs& L, const CtaPos& c, int c1, int c2) {
  return c.pbase + (int64_t)c1 * c.rs + (int64_t)c2 * L.s;
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

// Writes the plane tile's lattice values (rows [R0, R1), columns [C0, C1))
// to the natural-layout array: the known values of the next level (compress)
// or the reconstruction (retrieve). At stride 1 a (even, odd) pair is one
// vector store; at stride 2 each value is stored twice so that whole sectors
// are written -- the element in between is a target of the next level and is
// never read as a known value.
template <class T, int BR, int HC, int VEC>
__device__ __forceinline__ void store_tile(const LevelArgs& L, const CtaPos& c, const T* VE,
                                           const T* VO, T* dst) {
  typedef typename Vec2<T>::type V2;
  const int ncol = c.C1 - c.C0;
  for (int it = threadIdx.x; it < BR * HC; it += 256) {
    const int lr = it / HC, jp = it - lr * HC;
    const int c1 = c.R0 + lr, c2 = c.C0 + 2 * jp;
    if (c1 >= c.R1 || 2 * jp >= ncol) continue;
    const T ve = VE[(lr + 2) * VEC + jp + 1];
    const int64_t e = eidx(L, c, c1, c2);
    const bool hasodd = 2 * jp + 1 < ncol;
    const T vo = hasodd ? VO[lr * HC + jp] : ve;
    if (L.vec && L.s == 1 && hasodd && (e & 1) == 0) {
      V2 v2;
      v2.x = ve;
      v2.y = vo;
      *reinterpret_cast<V2*>(dst + e) = v2;
    } else if (L.s == 2) {
      V2 v2;
      if (L.vec && (e & 1) == 0 && 2 * (int64_t)c2 + 1 < L.N[2]) {
        v2.x = ve;
        v2.y = ve;
        *reinterpret_cast<V2*>(dst + e) = v2;
      } else {
        dst[e] = ve;
      }
      if (hasodd) {
        if (L.vec && ((e + 2) & 1) == 0 && 2 * (int64_t)c2 + 3 < L.N[2]) {
          v2.x = vo;
          v2.y = vo;
          *reinterpret_cast<V2*>(dst + e + 2) = v2;
        } else {
          dst[e + 2] = vo;
        }
      }
    } else {
      dst[e] = ve;
      if (hasodd) dst[e + L.s] = vo;
    }
  }
}

// ---------------------------------------------------------------------------
// Compression of one level.
// ---------------------------------------------------------------------------
template <class T, int BR, int BC>
__device__ __forceinline__ void level_compress_body(const LevelArgs& L, const T* __restrict__ x,
                                                    T* xh, int write_xh, const QuantArgs<T>& qa,
                                                    const SweepOut& o, const LevelDescs& D,
                                                    uint64_t cta, unsigned char* smem) {
  typedef Tile<BR, BC> G;
  T* VE = reinterpret_cast<T*>(smem);                     // [VR][VEC]
  T* VO = VE + G::VR * G::VEC;                            // [BR][HC]
  uint32_t* E2 = reinterpret_cast<uint32_t*>(VO + BR * G::HC);  // [BR][PITCH]
  uint32_t* E1 = E2 + BR * G::PITCH;                      // [BR/2][PITCH]
  uint32_t* E0 = E1 + (BR / 2) * G::PITCH;                // [BR/2][PITCH]

  const CtaPos c = cta_pos(L, cta, BR, BC);
  const bool podd = (c.P & 1) != 0;
  const int tid = threadIdx.x;
  const int cubic = L.cubic;
  const int M0 = (int)L.M[0], M1 = (int)L.M[1], M2 = (int)L.M[2];
  uint32_t orN[3] = {0, 0, 0}, qmx[3] = {0, 0, 0};

  // codes outside the grid (edge tiles) must read as zero in phase 4
  if (c.R1 - c.R0 < BR || c.C1 - c.C0 < BC)
    for (int i = tid; i < 2 * BR * G::PITCH; i += 256) E2[i] = 0;  // E2, E1, E0
  __syncthreads();

  // Phase 1: even rows of VE.
  const LevelStage& S0 = L.st[0];
  const int64_t so = L.s * L.stride[0];
  const bool r1 = c.P + 1 <= M0 - 1;
  const bool r3 = cubic && c.P - 3 >= 0 && c.P + 3 <= M0 - 1;
#pragma unroll 2
  for (int it = tid; it < (BR / 2 + 3) * G::VEC; it += 256) {
    const int jr = it / G::VEC, je = it - jr * G::VEC;
    const int c1 = c.R0 - 2 + 2 * jr, c2 = c.C0 - 2 + 2 * je;
    if (c1 < 0 || c1 >= M1 || c2 < 0 || c2 >= M2 || c2 > c.C1 + 2) continue;
    const int64_t e = eidx(L, c, c1, c2);
    T v;
    if (!podd) {
      v = __ldg(xh + e);
    } else {
      const T b = __ldg(xh + e - so);
      const T cc = r1 ? __ldg(xh + e + so) : b;
      const T a = r3 ? __ldg(xh + e - 3 * so) : b;
      const T d = r3 ? __ldg(xh + e + 3 * so) : b;
      const T xv = __ldg(x + e);
      const T pred = pred4<T>(a, b, cc, d, c.P, M0, cubic);
      bool outl;
      T rec;
      const int32_t q = quantize<T>(xv, pred, qa, &rec, &outl);
      v = rec;
      if (c1 >= c.R0 && c1 < c.R1 && c2 >= c.C0 && c2 < c.C1) {
        const uint32_t N = negabinary(q);
        orN[0] |= N;
        qmx[0] = max(qmx[0], (uint32_t)(q < 0 ? -q : q));
        E0[((c1 - c.R0) >> 1) * G::PITCH + sw((c2 - c.C0) >> 1)] = N;
        if (outl)
          record_outlier(o, S0.t,
                         ((uint64_t)((c.P - 1) >> 1) * S0.m1 + (uint64_t)(c1 >> 1)) * S0.m2 +
                             (uint64_t)(c2 >> 1),
                         (double)xv);
      }
    }
    VE[(2 * jr) * G::VEC + je] = v;
  }
  __syncthreads();

  // Phase 2: sweep 1 on the odd rows of the CTA, columns [C0-2, C1+2].
  const LevelStage& S1 = L.st[1];
#pragma unroll 2
  for (int it = tid; it < (BR / 2) * G::VEC; it += 256) {
    const int jr = it / G::VEC, je = it - jr * G::VEC;
    const int c1 = c.R0 + 1 + 2 * jr, c2 = c.C0 - 2 + 2 * je;
    if (c1 >= c.R1 || c2 < 0 || c2 >= M2 || c2 > c.C1 + 2) continue;
    const T xv = __ldg(x + eidx(L, c, c1, c2));
    const T b = VE[(2 * jr + 2) * G::VEC + je];
    const T cc = VE[(2 * jr + 4) * G::VEC + je];
    const T a = VE[(2 * jr) * G::VEC + je];
    const T d = VE[(2 * jr + 6) * G::VEC + je];
    const T pred = pred4<T>(a, b, cc, d, c1, M1, cubic);
    bool outl;
    T rec;
    const int32_t q = quantize<T>(xv, pred, qa, &rec, &outl);
    VE[(2 * jr + 3) * G::VEC + je] = rec;
    if (c2 >= c.C0 && c2 < c.C1) {
      const uint32_t N = negabinary(q);
      orN[1] |= N;
      qmx[1] = max(qmx[1], (uint32_t)(q < 0 ? -q : q));
      E1[jr * G::PITCH + sw((c2 - c.C0) >> 1)] = N;
      if (outl)
        record_outlier(o, S1.t,
                       ((uint64_t)c.P * S1.m1 + (uint64_t)((c1 - 1) >> 1)) * S1.m2 +
                           (uint64_t)(c2 >> 1),
                       (double)xv);
    }
  }
  __syncthreads();

  // Phase 3: sweep 2 on the odd columns of the CTA's rows.
  const LevelStage& S2 = L.st[2];
#pragma unroll 4
  for (int it = tid; it < BR * G::HC; it += 256) {
    const int lr = it / G::HC, jo = it - lr * G::HC;
    const int c1 = c.R0 + lr, c2 = c.C0 + 1 + 2 * jo;
    if (c1 >= c.R1 || c2 >= c.C1) continue;
    const T xv = __ldg(x + eidx(L, c, c1, c2));
    const T* row = VE + (lr + 2) * G::VEC;
    const T pred = pred4<T>(row[jo], row[jo + 1], row[jo + 2], row[jo + 3], c2, M2, cubic);
    bool outl;
    T rec;
    const int32_t q = quantize<T>(xv, pred, qa, &rec, &outl);
    VO[lr * G::HC + jo] = rec;
    const uint32_t N = negabinary(q);
    orN[2] |= N;
    qmx[2] = max(qmx[2], (uint32_t)(q < 0 ? -q : q));
    E2[lr * G::PITCH + sw(jo)] = N;
    if (outl)
      record_outlier(o, S2.t,
                     ((uint64_t)c.P * S2.m1 + (uint64_t)c1) * S2.m2 + (uint64_t)((c2 - 1) >> 1),
                     (double)xv);
  }
  __syncthreads();

  // Phase 3b: the level's values for the next level (known points there).
  if (write_xh) store_tile<T, BR, G::HC, G::VEC>(L, c, VE, VO, xh);

  // Phase 4: bitplane transpose and compaction of the three segments.
  // Threads [0,128) words of stage 2, [128,192) stage 1, [192,256) stage 0.
  const int lane = tid & 31, wi = tid >> 5;
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
  uint32_t pw[32];
  {
    const uint32_t* Eb = sidx == 2 ? E2 : (sidx == 1 ? E1 : E0);
    const int lr = mine ? li / CW : 0, lj = mine ? li - lr * CW : 0;
#pragma unroll
    for (int i = 0; i < 32; ++i) pw[i] = mine ? Eb[lr * G::PITCH + lj * 33 + i] : 0u;
  }
  transpose32(pw);
  xor_encode_planes(pw);
  const uint64_t pi = sidx == 0 ? (uint64_t)((c.P - 1) >> 1) : (uint64_t)c.P;
  const uint64_t g = active ? seg_id(S, pi, c.rb, c.ct) : 0;
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
  const uint64_t capg = g * (uint64_t)nwords + (uint64_t)wl * 32;
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    const uint32_t mk = __ballot_sync(~0u, pw[k] != 0);
    if (wact) {
      if (lane == k) {
        o.bm[pds[k].bm_off + g * S.bw + wl] = mk;
        if (mk) atomicAdd(&scnt[sidx][k], (uint32_t)__popc(mk));
      }
      if (pw[k]) o.cap[pds[k].cap_off + capg + __popc(mk & lt)] = pw[k];
    }
  }
  __syncthreads();
  if (tid < 96) {
    const uint32_t n = scnt[tid >> 5][tid & 31];
    if (n) atomicAdd(o.nnz + 32 * L.st[tid >> 5].t + (tid & 31), n);
  }
}

// ---------------------------------------------------------------------------
// Reconstruction of one level (Algorithm 1).
// Words come from the CTA's own segments and, for halo targets, from the
// neighbouring segments (stage 1: left/right; stage 0: the 3x3 block) --
// at most 13 segments. Their group bitmap words of every selected plane are
// staged in shared memory first; a word's plane value is then found from
// its group's bitmap word alone (rank = population below its bit), so its
// 32 plane loads are independent of each other.
// ---------------------------------------------------------------------------
constexpr int kSlots = 13;
constexpr int kMaxBw = 4;  // bitmap words per segment (RB * CW <= 128)

template <class T, int BR, int BC>
__device__ __forceinline__ void level_retrieve_body(const LevelArgs& L, T* out, T twoeb, int b,
                                                    const uint32_t* __restrict__ cap,
                                                    const uint32_t* __restrict__ bm,
                                                    const uint64_t* __restrict__ oidx,
                                                    const double* __restrict__ oval,
                                                    const LevelDescs& D, uint64_t cta,
                                                    unsigned char* smem) {
  typedef Tile<BR, BC> G;
  T* VE = reinterpret_cast<T*>(smem);                           // [VR][VEC]
  T* VO = VE + G::VR * G::VEC;                                  // [BR][HC]
  uint32_t* Q2 = reinterpret_cast<uint32_t*>(VO + BR * G::HC);  // [BR][PITCH]
  uint32_t* Q1 = Q2 + BR * G::PITCH;                            // [BR/2][QEP]
  uint32_t* Q0 = Q1 + (BR / 2) * G::QEP;                        // [BR/2+3][QEP]
  __shared__ uint32_t SB[kSlots][32][kMaxBw];  // group bitmaps of the segments
  __shared__ unsigned long long SG[kSlots];    // segment id (or ~0 if absent)

  const CtaPos c = cta_pos(L, cta, BR, BC);
  const bool podd = (c.P & 1) != 0;
  const int tid = threadIdx.x;
  const int cubic = L.cubic;
  const int M0 = (int)L.M[0], M1 = (int)L.M[1], M2 = (int)L.M[2];
  const LevelStage &S0 = L.st[0], &S1 = L.st[1], &S2 = L.st[2];

  // slots: 0 = stage 2 own; 1..3 = stage 1 (ct-1, ct, ct+1);
  //        4..12 = stage 0 (rb-1..rb+1) x (ct-1..ct+1)
  if (tid < kSlots) {
    int sx, drb, dct;
    if (tid == 0) { sx = 2; drb = 0; dct = 0; }
    else if (tid < 4) { sx = 1; drb = 0; dct = tid - 2; }
    else { sx = 0; drb = (tid - 4) / 3 - 1; dct = (tid - 4) % 3 - 1; }
    const LevelStage& S = L.st[sx];
    const int64_t rbs = (int64_t)c.rb + drb, cts = (int64_t)c.ct + dct;
    const bool ok = S.present && (sx != 0 || podd) && rbs >= 0 && (uint64_t)rbs < S.nrb &&
                    cts >= 0 && (uint64_t)cts < S.nct;
    const uint64_t pi = sx == 0 ? (uint64_t)((c.P - 1) >> 1) : (uint64_t)c.P;
    SG[tid] = ok ? seg_id(S, pi, (uint64_t)rbs, (uint64_t)cts) : ~0ULL;
  }
  __syncthreads();
  for (int u = tid; u < kSlots * 32 * kMaxBw; u += 256) {
    const int slot = u / (32 * kMaxBw), k = (u / kMaxBw) & 31, v = u % kMaxBw;
    const int sx = slot == 0 ? 2 : (slot < 4 ? 1 : 0);
    const LevelStage& S = L.st[sx];
    const PlaneDesc& pd = D.s[sx].p[k];
    uint32_t w = 0;
    if (SG[slot] != ~0ULL && k >= b && pd.nnz && (uint64_t)v < S.bw)
      w = __ldg(bm + pd.bm_off + SG[slot] * S.bw + v);
    SB[slot][k][v] = w;
  }
  __syncthreads();

  // Phase 0: decode the words the CTA needs.
  //  stage 2: own rows x own words
  //  stage 1: own odd rows x words [C0/64 - 1, C0/64 + CWD] (halo columns)
  //  stage 0: even rows [R0-2, R1+2] x the same word range (odd planes)
  const int cw0 = c.C0 >> 6;  // first own word of a code row
  const int n2r = c.R1 - c.R0, n1r = (c.R1 - c.R0) >> 1;
  const int nw2 = (S2.present && c.ct < S2.nct && c.rb < S2.nrb) ? n2r * (int)S2.CW : 0;
  const int hw = G::CWD + 2;
  const int nw1 = S1.present ? n1r * hw : 0;
  const int nw0 = (S0.present && podd) ? (BR / 2 + 3) * hw : 0;
  for (int it = tid; it < nw2 + nw1 + nw0; it += 256) {
    int sx, lr;
    int64_t rr, j;
    if (it < nw2) {
      sx = 2;
      lr = it / (int)S2.CW;
      j = (int64_t)c.ct * S2.CW + (it - lr * (int)S2.CW);
      rr = c.R0 + lr;
    } else if (it < nw2 + nw1) {
      const int u = it - nw2;
      sx = 1;
      lr = u / hw;
      j = cw0 - 1 + (u - lr * hw);
      rr = (c.R0 >> 1) + lr;
    } else {
      const int u = it - nw2 - nw1;
      sx = 0;
      lr = u / hw;
      j = cw0 - 1 + (u - lr * hw);
      rr = (c.R0 >> 1) - 1 + lr;  // stage-0 row = c1 / 2 for c1 = R0 - 2 + 2 lr
    }
    const LevelStage& S = L.st[sx];
    if (rr < 0 || (uint64_t)rr >= S.m1 || j < 0 || (uint64_t)j >= S.wr) continue;
    const uint64_t rbw = (uint64_t)rr / S.RB, ctw = (uint64_t)j / S.CW;
    int slot = 0;
    if (sx == 1) slot = 2 + (int)((int64_t)ctw - (int64_t)c.ct);
    else if (sx == 0)
      slot = 4 + ((int)((int64_t)rbw - (int64_t)c.rb) + 1) * 3 + (int)((int64_t)ctw - (int64_t)c.ct) + 1;
    const uint64_t g = SG[slot];
    const uint32_t li = (uint32_t)(((uint64_t)rr % S.RB) * S.CW + ((uint64_t)j % S.CW));
    const uint32_t wl = li >> 5, bmask = (1u << (li & 31)) - 1u, bit = 1u << (li & 31);
    const uint64_t capg = g * (uint64_t)S.RB * S.CW + (uint64_t)wl * 32;
    const PlaneDesc* pds = D.s[sx].p;
    uint32_t nv[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      const uint32_t m = SB[slot][k][wl];  // zero for unselected / empty planes
      nv[k] = (m & bit) ? __ldg(cap + pds[k].cap_off + capg + __popc(m & bmask)) : 0u;
    }
    xor_decode_planes(nv, b);
    transpose32(nv);
    if (sx == 2) {
      const int lj = (int)(j - (int64_t)c.ct * S2.CW);
#pragma unroll
      for (int i = 0; i < 32; ++i) Q2[lr * G::PITCH + lj * 33 + i] = nv[i];
    } else {
      // keep the codes of the halo window: code column C0/2 - 1 + e, e < VEC
      uint32_t* Qr = (sx == 1 ? Q1 : Q0) + lr * G::QEP;
      const int base = (int)(j * 32 - ((c.C0 >> 1) - 1));
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const int e = base + i;
        if (e >= 0 && e < G::VEC) Qr[sw(e)] = nv[i];
      }
    }
  }
  __syncthreads();

  // Phase 1: even rows of VE (sweep 0 of an odd plane, else known points).
  const int64_t so = L.s * L.stride[0];
  const bool r1 = c.P + 1 <= M0 - 1;
  const bool r3 = cubic && c.P - 3 >= 0 && c.P + 3 <= M0 - 1;
#pragma unroll 2
  for (int it = tid; it < (BR / 2 + 3) * G::VEC; it += 256) {
    const int jr = it / G::VEC, je = it - jr * G::VEC;
    const int c1 = c.R0 - 2 + 2 * jr, c2 = c.C0 - 2 + 2 * je;
    if (c1 < 0 || c1 >= M1 || c2 < 0 || c2 >= M2 || c2 > c.C1 + 2) continue;
    const int64_t e = eidx(L, c, c1, c2);
    T v;
    if (!podd) {
      v = __ldg(out + e);
    } else {
      const T bb = __ldg(out + e - so);
      const T cc = r1 ? __ldg(out + e + so) : bb;
      const T a = r3 ? __ldg(out + e - 3 * so) : bb;
      const T d = r3 ? __ldg(out + e + 3 * so) : bb;
      const T pred = pred4<T>(a, bb, cc, d, c.P, M0, cubic);
      const int64_t q = negabinary_inv(Q0[jr * G::QEP + sw(je)]);
      v = FP<T>::add(pred, FP<T>::mul(FP<T>::from_code(q), twoeb));
      if (S0.out_end > S0.out_begin) {
        const uint64_t ci = ((uint64_t)((c.P - 1) >> 1) * S0.m1 + (uint64_t)(c1 >> 1)) * S0.m2 +
                            (uint64_t)(c2 >> 1);
        find_outlier<T>(S0, oidx, oval, ci, &v);
      }
    }
    VE[(2 * jr) * G::VEC + je] = v;
  }
  __syncthreads();

  // Phase 2: sweep 1.
#pragma unroll 2
  for (int it = tid; it < (BR / 2) * G::VEC; it += 256) {
    const int jr = it / G::VEC, je = it - jr * G::VEC;
    const int c1 = c.R0 + 1 + 2 * jr, c2 = c.C0 - 2 + 2 * je;
    if (c1 >= c.R1 || c2 < 0 || c2 >= M2 || c2 > c.C1 + 2) continue;
    const T bb = VE[(2 * jr + 2) * G::VEC + je];
    const T cc = VE[(2 * jr + 4) * G::VEC + je];
    const T a = VE[(2 * jr) * G::VEC + je];
    const T d = VE[(2 * jr + 6) * G::VEC + je];
    const T pred = pred4<T>(a, bb, cc, d, c1, M1, cubic);
    const int64_t q = negabinary_inv(Q1[jr * G::QEP + sw(je)]);
    T v = FP<T>::add(pred, FP<T>::mul(FP<T>::from_code(q), twoeb));
    if (S1.out_end > S1.out_begin) {
      const uint64_t ci = ((uint64_t)c.P * S1.m1 + (uint64_t)((c1 - 1) >> 1)) * S1.m2 +
                          (uint64_t)(c2 >> 1);
      find_outlier<T>(S1, oidx, oval, ci, &v);
    }
    VE[(2 * jr + 3) * G::VEC + je] = v;
  }
  __syncthreads();

  // Phase 3: sweep 2.
#pragma unroll 4
  for (int it = tid; it < BR * G::HC; it += 256) {
    const int lr = it / G::HC, jo = it - lr * G::HC;
    const int c1 = c.R0 + lr, c2 = c.C0 + 1 + 2 * jo;
    if (c1 >= c.R1 || c2 >= c.C1) continue;
    const T* row = VE + (lr + 2) * G::VEC;
    const T pred = pred4<T>(row[jo], row[jo + 1], row[jo + 2], row[jo + 3], c2, M2, cubic);
    const int64_t q = negabinary_inv(Q2[lr * G::PITCH + sw(jo)]);
    T v = FP<T>::add(pred, FP<T>::mul(FP<T>::from_code(q), twoeb));
    if (S2.out_end > S2.out_begin) {
      const uint64_t ci = ((uint64_t)c.P * S2.m1 + (uint64_t)c1) * S2.m2 + (uint64_t)((c2 - 1) >> 1);
      find_outlier<T>(S2, oidx, oval, ci, &v);
    }
    VO[lr * G::HC + jo] = v;
  }
  __syncthreads();

  // Phase 3b: write the plane tile (every lattice point of the CTA).
  store_tile<T, BR, G::HC, G::VEC>(L, c, VE, VO, out);
}

// Single-field kernels: arguments in the parameter space.
template <class T, int BR, int BC>
__global__ void __launch_bounds__(256, 3) k_level_compress(LevelArgs L, const T* __restrict__ x,
                                                           T* xh, int write_xh, QuantArgs<T> qa,
                                                           SweepOut o, LevelDescs D) {
  extern __shared__ __align__(16) unsigned char smem[];
  level_compress_body<T, BR, BC>(L, x, xh, write_xh, qa, o, D, blockIdx.x, smem);
}

template <class T, int BR, int BC>
__global__ void __launch_bounds__(256, 2) k_level_retrieve(LevelArgs L, T* out, T twoeb, int b,
                                                           const uint32_t* __restrict__ cap,
                                                           const uint32_t* __restrict__ bm,
                                                           const uint64_t* __restrict__ oidx,
                                                           const double* __restrict__ oval,
                                                           LevelDescs D) {
  extern __shared__ __align__(16) unsigned char smem[];
  level_retrieve_body<T, BR, BC>(L, out, twoeb, b, cap, bm, oidx, oval, D, blockIdx.x, smem);
}

// Batched kernels: one grid covers the level's CTAs of every field of a
// batch; entry i owns CTAs [cta_begin_i, cta_begin_{i+1}).
template <class E>
__device__ __forceinline__ const E& find_entry(const E* __restrict__ ents, int n) {
  __shared__ int sel;
  if (threadIdx.x == 0) {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (ents[mid].cta_begin <= blockIdx.x) lo = mid;
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
  const CompressEntry& e = find_entry(ents, n);
  level_compress_body<T, BR, BC>(e.L, (const T*)e.x, (T*)e.xh, e.write_xh,
                                 *reinterpret_cast<const QuantArgs<T>*>(e.quant), e.o, e.D,
                                 blockIdx.x - e.cta_begin, smem);
}

template <class T, int BR, int BC>
__global__ void __launch_bounds__(256, 2) k_level_retrieve_batch(
    const RetrieveEntry* __restrict__ ents, int n) {
  extern __shared__ __align__(16) unsigned char smem[];
  const RetrieveEntry& e = find_entry(ents, n);
  level_retrieve_body<T, BR, BC>(e.L, (T*)e.out, (T)e.twoeb, e.b, e.cap, e.bm, e.oidx, e.oval,
                                 e.D, blockIdx.x - e.cta_begin, smem);
}

template <class T, int BR, int BC>
size_t smem_compress() {
  typedef Tile<BR, BC> G;
  return sizeof(T) * (G::VR * G::VEC + BR * G::HC) + 4 * (2 * BR * G::PITCH);
}
template <class T, int BR, int BC>
size_t smem_retrieve() {
  typedef Tile<BR, BC> G;
  return sizeof(T) * (G::VR * G::VEC + BR * G::HC) +
         4 * (BR * G::PITCH + (BR / 2) * G::QEP + (BR / 2 + 3) * G::QEP);
}

template <class T, int BR, int BC>
cudaError_t setup_once() {
  static cudaError_t e = [] {
    cudaError_t r = cudaFuncSetAttribute(k_level_compress<T, BR, BC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_compress<T, BR, BC>());
    if (r == cudaSuccess)
      r = cudaFuncSetAttribute(k_level_retrieve<T, BR, BC>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem_retrieve<T, BR, BC>());
    if (r == cudaSuccess)
      r = cudaFuncSetAttribute(k_level_compress_batch<T, BR, BC>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem_compress<T, BR, BC>());
    if (r == cudaSuccess)
      r = cudaFuncSetAttribute(k_level_retrieve_batch<T, BR, BC>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem_retrieve<T, BR, BC>());
    return r;
  }();
  return e;
}

}  // namespace

int level_rows(int dtype) { return dtype == 0 ? kLevelRowsF32 : kLevelRowsF64; }

cudaError_t launch_level_compress(int dtype, const LevelArgs& L, const void* x, void* xh,
                                  int write_xh, const void* quant, const SweepOut& o,
                                  const LevelDescs& d, cudaStream_t st) {
  const uint64_t grid = (uint64_t)L.M[0] * L.nrb * L.nct;
  if (grid == 0) return cudaSuccess;
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
                                  const double* oval, const LevelDescs& d, cudaStream_t st) {
  const uint64_t grid = (uint64_t)L.M[0] * L.nrb * L.nct;
  if (grid == 0) return cudaSuccess;
  cudaError_t e;
  if (dtype == 0) {
    if ((e = setup_once<float, kLevelRowsF32, kLevelCols>()) != cudaSuccess) return e;
    k_level_retrieve<float, kLevelRowsF32, kLevelCols>
        <<<(unsigned)grid, 256, smem_retrieve<float, kLevelRowsF32, kLevelCols>(), st>>>(
            L, (float*)out, (float)twoeb, b, cap, bm, oidx, oval, d);
  } else {
    if ((e = setup_once<double, kLevelRowsF64, kLevelCols>()) != cudaSuccess) return e;
    k_level_retrieve<double, kLevelRowsF64, kLevelCols>
        <<<(unsigned)grid, 256, smem_retrieve<double, kLevelRowsF64, kLevelCols>(), st>>>(
            L, (double*)out, twoeb, b, cap, bm, oidx, oval, d);
  }
  return cudaGetLastError();
}

cudaError_t launch_level_compress_batch(int dtype, const CompressEntry* ents, int n,
                                        uint64_t ctas, cudaStream_t st) {
  if (ctas == 0 || n == 0) return cudaSuccess;
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
                                        uint64_t ctas, cudaStream_t st) {
  if (ctas == 0 || n == 0) return cudaSuccess;
  cudaError_t e;
  if (dtype == 0) {
    if ((e = setup_once<float, kLevelRowsF32, kLevelCols>()) != cudaSuccess) return e;
    k_level_retrieve_batch<float, kLevelRowsF32, kLevelCols>
        <<<(unsigned)ctas, 256, smem_retrieve<float, kLevelRowsF32, kLevelCols>(), st>>>(ents, n);
  } else {
    if ((e = setup_once<double, kLevelRowsF64, kLevelCols>()) != cudaSuccess) return e;
    k_level_retrieve_batch<double, kLevelRowsF64, kLevelCols>
        <<<(unsigned)ctas, 256, smem_retrieve<double, kLevelRowsF64, kLevelCols>(), st>>>(ents, n);
  }
  return cudaGetLastError();
}

}  // namespace ipc
