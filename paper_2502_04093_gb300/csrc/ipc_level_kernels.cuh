// Fused per-level kernels of libipcomp (sm_103a), templated on Q: Q = false
// for linear and cubic interpolation, Q = true for cubic interpolation with
// the three-point quadratic at the boundaries (its boundary forms cost the
// common case several percent when compiled in, so they are a variant of
// their own). Each variant is instantiated by a unit of its own
// (ipc_level.cu, ipc_level_quad.cu), compiled in parallel.
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
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "ipc_device.cuh"
#include "ipc_internal.h"
#include "ipc_level_body.cuh"

namespace ipc {
namespace {
using namespace dev;

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

template <class T, int BR, int BC, bool Q>
__device__ __forceinline__ void level_compress_body(const LevelArgs& L, const T* __restrict__ x,
                                                    T* xh, int write_xh, const QuantArgs<T>& qa,
                                                    const SweepOut& o,
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
  const int interp = L.interp;
  const int M0 = (int)L.M[0], M1 = (int)L.M[1], M2 = (int)L.M[2];
  const LevelStage &S0 = L.st[0], &S1 = L.st[1], &S2 = L.st[2];
  uint32_t orN[3] = {0, 0, 0}, qmx[3] = {0, 0, 0};
  auto stat = [&](int st, int32_t q) {
    orN[st] |= negabinary(q);
    qmx[st] = max(qmx[st], (uint32_t)(q < 0 ? -q : q));
  };

  // x loads (the checked build tests each index against the field)
  auto xld = [&](int64_t e) -> T { return IPC_IN(L, e, L.lim_x, kSiteX) ? __ldg(x + e) : (T)0; };
  auto xld4 = [&](int64_t e) -> float4 {
    return IPC_IN(L, e + 3, L.lim_x, kSiteX)
               ? __ldg(reinterpret_cast<const float4*>(reinterpret_cast<const float*>(x) + e))
               : make_float4(0.f, 0.f, 0.f, 0.f);
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
    // far planes read: Eq. 2 needs both, the quadratic the one that exists
    const bool r3 = interp != 0 && c.P - 3 >= 0 && c.P + 3 <= M0 - 1;
    const bool ra = Q && interp == 2 ? r1 && c.P - 3 >= 0 : r3;
    const bool rd = Q && interp == 2 ? c.P + 3 <= M0 - 1 : r3;
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
      const T a = ra ? __ldg(p - k0) : bb;
      const T d = rd ? __ldg(p + 2 * k0) : bb;
      T v;
      point(pred4<T, Q>(a, bb, cc, d, c.P, M0, interp),
            xld(c.pbase + (int64_t)c1 * c.rs + (int64_t)c2 * L.s), c1, c2, own, &v);
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
            const V2 a = ra ? __ldg(p2 - k0 / 2) : bb;
            const V2 d = rd ? __ldg(p2 + k0) : bb;
            const int64_t e = c.pbase + (int64_t)c1 * c.rs + (int64_t)c2p * L.s;
            T xa, xb;
            if (vec) {
              const float4 xv = xld4(e);
              xa = (T)xv.x;
              xb = (T)xv.z;
            } else {
              xa = xld(e);
              xb = xld(e + 2 * L.s);
            }
            point(pred4<T, Q>(a.x, bb.x, cc.x, d.x, c.P, M0, interp), xa, c1, c2p, ownr, &va);
            point(pred4<T, Q>(a.y, bb.y, cc.y, d.y, c.P, M0, interp), xb, c1, c2p + 2, ownr, &vb);
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
      const T pred = pred4<T, Q>(a, bb, cc, d, c1, M1, interp);
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
          const float4 xv = xld4(e);
          xa = (T)xv.x;
          xb = (T)xv.z;
        } else {
          xa = xld(e);
          xb = pb ? xld(e + 2 * L.s) : xa;
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
                  xld(c.pbase + (int64_t)c1 * c.rs + (int64_t)c2 * L.s));
      }
    }
  }
  __syncthreads();

  // Phase 3: sweep 2 (four odd columns per thread) and the level's values.
  {
    const int g = tid & 63, rq = tid >> 6;
    const int c2e = c.C0 + 8 * g;
    // per odd column: the form of pred4 (pred_rule), RW bits each
    constexpr int RW = Q ? 3 : 2;
    uint32_t rule = 0u;
#pragma unroll
    for (int k = 0; k < 4; ++k) rule |= pred_rule<Q>(c2e + 2 * k + 1, M2, interp) << (RW * k);
    const bool quad = Q && (rule & 04444u) != 0u;  // a quadratic boundary form in the run
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
          const float4 u = xld4(e + c2e), v = xld4(e + c2e + 4);
          xo[0] = (T)u.y;
          xo[1] = (T)u.w;
          xo[2] = (T)v.y;
          xo[3] = (T)v.w;
        } else {
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int c2o = c2e + 2 * k + 1;
            xo[k] = c2o < c.C1 ? xld(e + (int64_t)c2o * L.s) : (T)0;
          }
        }
        T v[8];
        uint32_t n[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int c2o = c2e + 2 * k + 1;
          const T u = FP<T>::add(w[k + 1], w[k + 2]);
          const T cub = FP<T>::template mul_pow2<-4>(
              FP<T>::sub(FP<T>::mul((T)9, u), FP<T>::add(w[k], w[k + 3])));
          const T lin = FP<T>::template mul_pow2<-1>(u);
          const uint32_t r = rule >> (RW * k) & ((1u << RW) - 1u);
          T pred = r == 2u ? cub : (r == 1u ? lin : w[k + 1]);
          if (quad && (r & 4u)) pred = quad3<T>(w[k], w[k + 1], w[k + 2], w[k + 3], r == 4u);
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
        if (write_xh && IPC_IN(L, (int64_t)c.P * L.ost0 + (int64_t)c1 * L.ost1 + min(c.C1, c2e + 8) - 1,
                               L.lim_out, kSiteXh))
          store_run<T>(xh + (int64_t)c.P * L.ost0 + (int64_t)c1 * L.ost1, 1, 0, c2e, c.C1, v);
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
  const StagePlanes& SP = L.sp[sidx];  // plane k: capacity SP.cap0 + k SP.pcap, bitmap alike
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
    if (wact && cd[k] &&
        IPC_IN(L, SP.cap0 + (uint64_t)k * SP.pcap + capg + __popc(mk & lt), L.lim_cap, kSiteCapStore))
      o.cap[SP.cap0 + (uint64_t)k * SP.pcap + capg + __popc(mk & lt)] = cd[k];
  }
  if (wact) {
    if (IPC_IN(L, SP.bm0 + (uint64_t)lane * SP.pbm + gseg * S.bw + wl, L.lim_bm, kSiteBmStore))
      o.bm[SP.bm0 + (uint64_t)lane * SP.pbm + gseg * S.bw + wl] = mybm;
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
template <class T, int BR, int BC, bool Q>
__global__ void __launch_bounds__(256, 4) k_level_compress(LevelArgs L, const T* __restrict__ x,
                                                           T* xh, int write_xh, QuantArgs<T> qa,
                                                           SweepOut o) {
  extern __shared__ __align__(16) unsigned char smem[];
  level_compress_body<T, BR, BC, Q>(L, x, xh, write_xh, qa, o, blockIdx.x, smem);
}

template <class T, int BR, int BC, bool W16, int NS, bool Q>
__global__ void __launch_bounds__(256, retrieve_ctas_per_sm<T, BR, W16>()) k_level_retrieve(
    LevelArgs L, T* out, T twoeb, int b, const uint32_t* __restrict__ cap,
    const uint32_t* __restrict__ bm, const uint64_t* __restrict__ oidx,
    const double* __restrict__ oval, uint64_t ntiles) {
  extern __shared__ __align__(16) unsigned char smem[];
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    level_retrieve_body<T, BR, BC, W16, NS, kPlain, Q>(L, out, twoeb, b, cap, bm, oidx, oval, t, smem);
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

template <class T, int BR, int BC, bool Q>
__global__ void __launch_bounds__(256, 3) k_level_compress_batch(
    const CompressEntry* __restrict__ ents, int n) {
  extern __shared__ __align__(16) unsigned char smem[];
  const CompressEntry& e = find_entry(ents, n, blockIdx.x);
  level_compress_body<T, BR, BC, Q>(e.L, (const T*)e.x, (T*)e.xh, e.write_xh,
                                 *reinterpret_cast<const QuantArgs<T>*>(e.quant), e.o,
                                 blockIdx.x - e.cta_begin, smem);
}

template <class T, int BR, int BC, bool W16, int NS, bool Q>
__global__ void __launch_bounds__(256, retrieve_ctas_per_sm<T, BR, W16>()) k_level_retrieve_batch(
    const RetrieveEntry* __restrict__ ents, int n, uint64_t ntiles) {
  extern __shared__ __align__(16) unsigned char smem[];
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const RetrieveEntry& e = find_entry(ents, n, t);
    level_retrieve_body<T, BR, BC, W16, NS, kPlain, Q>(e.L, (T*)e.out, (T)e.twoeb, e.b, e.cap, e.bm, e.oidx,
                                            e.oval, t - e.cta_begin, smem);
    __syncthreads();  // the next tile reuses shared memory (and the entry index)
  }
}

template <class T, int BR, int BC>
size_t smem_compress() {
  typedef CTile<BR, BC> G;
  return sizeof(T) * (G::H0 + G::H1) * G::VP + 4 * (BR + G::H1 + BR / 2) * G::QP;
}
template <class T, int BR, int BC, bool W16, int NS, bool Q>
cudaError_t setup_retrieve() {
  cudaError_t r = cudaFuncSetAttribute(k_level_retrieve<T, BR, BC, W16, NS, Q>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem_retrieve<T, BR, BC, W16, NS>());
  if (r == cudaSuccess)
    r = cudaFuncSetAttribute(k_level_retrieve_batch<T, BR, BC, W16, NS, Q>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_retrieve<T, BR, BC, W16, NS>());
  return r;
}

template <class T, int BR, int BC, bool Q>
cudaError_t setup_once() {
  static cudaError_t e = [] {
    cudaError_t r = cudaFuncSetAttribute(k_level_compress<T, BR, BC, Q>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_compress<T, BR, BC>());
    if (r == cudaSuccess)
      r = cudaFuncSetAttribute(k_level_compress<T, BR, BC, Q>,
                               cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared);
    if (r == cudaSuccess)
      r = cudaFuncSetAttribute(k_level_compress_batch<T, BR, BC, Q>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem_compress<T, BR, BC>());
    if (r == cudaSuccess) r = setup_retrieve<T, BR, BC, true, 1, Q>();
    if (r == cudaSuccess) r = setup_retrieve<T, BR, BC, true, 2, Q>();
    if (r == cudaSuccess) r = setup_retrieve<T, BR, BC, true, 4, Q>();
    constexpr int BR32 = sizeof(T) == 4 ? BR / 2 : BR;  // rows of 32-bit-code tiles, ns > 1
    if (r == cudaSuccess) r = setup_retrieve<T, BR, BC, false, 1, Q>();
    if (r == cudaSuccess) r = setup_retrieve<T, BR32, BC, false, 2, Q>();
    if (r == cudaSuccess) r = setup_retrieve<T, BR32, BC, false, 4, Q>();
    return r;
  }();
  return e;
}

template <class T, int BR, int BC, bool W16, int NS, bool Q>
void retrieve_kernel(const LevelArgs& L, void* out, double twoeb, int b, const uint32_t* cap,
                     const uint32_t* bm, const uint64_t* oidx, const double* oval, int per_sm,
                     cudaStream_t st) {
  const uint64_t tiles = retrieve_tiles(L, NS);
  if (tiles == 0) return;
  k_level_retrieve<T, BR, BC, W16, NS, Q>
      <<<persistent_grid(tiles, grid_per_sm(per_sm, retrieve_ctas_per_sm<T, BR, W16>())), 256,
         smem_retrieve<T, BR, BC, W16, NS>(), st>>>(L, (T*)out, (T)twoeb, b, cap, bm, oidx, oval,
                                                    tiles);
}
template <class T, int BR, int BC, bool W16, int NS, bool Q>
void retrieve_batch_kernel(const RetrieveEntry* ents, int n, uint64_t tiles, int per_sm,
                           cudaStream_t st) {
  k_level_retrieve_batch<T, BR, BC, W16, NS, Q>
      <<<persistent_grid(tiles, grid_per_sm(per_sm, retrieve_ctas_per_sm<T, BR, W16>())), 256,
         smem_retrieve<T, BR, BC, W16, NS>(), st>>>(ents, n, tiles);
}

// BR16 / BR32: tile rows with 16-bit code rows / with 32-bit code rows and
// several planes per tile (one-plane 32-bit tiles keep BR16 rows).
template <class T, int BR16, int BR32, int BC, bool Q>
void retrieve_dispatch(const LevelArgs& L, void* out, double twoeb, int b, const uint32_t* cap,
                       const uint32_t* bm, const uint64_t* oidx, const double* oval, int w16,
                       int ns, int per_sm, cudaStream_t st) {
#define IPC_RK(R, W, N) retrieve_kernel<T, R, BC, W, N, Q>(L, out, twoeb, b, cap, bm, oidx, oval, per_sm, st)
  if (!w16) {
    if (ns == 4) IPC_RK(BR32, false, 4);
    else if (ns == 2) IPC_RK(BR32, false, 2);
    else IPC_RK(BR16, false, 1);
  } else if (ns == 4) IPC_RK(BR16, true, 4);
  else if (ns == 2) IPC_RK(BR16, true, 2);
  else IPC_RK(BR16, true, 1);
#undef IPC_RK
}
template <class T, int BR16, int BR32, int BC, bool Q>
void retrieve_batch_dispatch(const RetrieveEntry* ents, int n, uint64_t tiles, int w16, int ns,
                             int per_sm, cudaStream_t st) {
#define IPC_RB(R, W, N) retrieve_batch_kernel<T, R, BC, W, N, Q>(ents, n, tiles, per_sm, st)
  if (!w16) {
    if (ns == 4) IPC_RB(BR32, false, 4);
    else if (ns == 2) IPC_RB(BR32, false, 2);
    else IPC_RB(BR16, false, 1);
  } else if (ns == 4) IPC_RB(BR16, true, 4);
  else if (ns == 2) IPC_RB(BR16, true, 2);
  else IPC_RB(BR16, true, 1);
#undef IPC_RB
}

template <bool Q>
cudaError_t level_compress_impl(int dtype, const LevelArgs& L, const void* x, void* xh,
                                  int write_xh, const void* quant, const SweepOut& o,
                                  cudaStream_t st) {
  const uint64_t grid = (uint64_t)L.M[0] * L.nrb * L.nct;
  if (grid == 0) return cudaSuccess;
  if (grid >= (1ULL << 31)) return cudaErrorInvalidValue;  // grid x limit (tile ids are 32-bit)
  cudaError_t e;
  if (dtype == 0) {
    if ((e = setup_once<float, kLevelRowsF32, kLevelCols, Q>()) != cudaSuccess) return e;
    k_level_compress<float, kLevelRowsF32, kLevelCols, Q>
        <<<(unsigned)grid, 256, smem_compress<float, kLevelRowsF32, kLevelCols>(), st>>>(
            L, (const float*)x, (float*)xh, write_xh, *(const QuantArgs<float>*)quant, o);
  } else {
    if ((e = setup_once<double, kLevelRowsF64, kLevelCols, Q>()) != cudaSuccess) return e;
    k_level_compress<double, kLevelRowsF64, kLevelCols, Q>
        <<<(unsigned)grid, 256, smem_compress<double, kLevelRowsF64, kLevelCols>(), st>>>(
            L, (const double*)x, (double*)xh, write_xh, *(const QuantArgs<double>*)quant, o);
  }
  return cudaGetLastError();
}

template <bool Q>
cudaError_t level_retrieve_impl(int dtype, const LevelArgs& L, void* out, double twoeb, int b,
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
    if ((e = setup_once<float, kLevelRowsF32, kLevelCols, Q>()) != cudaSuccess) return e;
    retrieve_dispatch<float, kLevelRowsF32, kLevelRowsF32 / 2, kLevelCols, Q>(L, out, twoeb, b, cap, bm, oidx, oval, w16, ns, shape.per_sm, st);
  } else {
    if ((e = setup_once<double, kLevelRowsF64, kLevelCols, Q>()) != cudaSuccess) return e;
    retrieve_dispatch<double, kLevelRowsF64, kLevelRowsF64, kLevelCols, Q>(L, out, twoeb, b, cap, bm, oidx, oval, w16, ns, shape.per_sm, st);
  }
  return cudaGetLastError();
}

template <bool Q>
cudaError_t level_compress_batch_impl(int dtype, const CompressEntry* ents, int n,
                                        uint64_t ctas, cudaStream_t st) {
  if (ctas == 0 || n == 0) return cudaSuccess;
  if (ctas >= (1ULL << 31)) return cudaErrorInvalidValue;
  cudaError_t e;
  if (dtype == 0) {
    if ((e = setup_once<float, kLevelRowsF32, kLevelCols, Q>()) != cudaSuccess) return e;
    k_level_compress_batch<float, kLevelRowsF32, kLevelCols, Q>
        <<<(unsigned)ctas, 256, smem_compress<float, kLevelRowsF32, kLevelCols>(), st>>>(ents, n);
  } else {
    if ((e = setup_once<double, kLevelRowsF64, kLevelCols, Q>()) != cudaSuccess) return e;
    k_level_compress_batch<double, kLevelRowsF64, kLevelCols, Q>
        <<<(unsigned)ctas, 256, smem_compress<double, kLevelRowsF64, kLevelCols>(), st>>>(ents, n);
  }
  return cudaGetLastError();
}

template <bool Q>
cudaError_t level_retrieve_batch_impl(int dtype, const RetrieveEntry* ents, int n,
                                        uint64_t tiles, int w16, int ns, int per_sm,
                                        cudaStream_t st) {
  if (tiles == 0 || n == 0) return cudaSuccess;
  if (tiles >= (1ULL << 32)) return cudaErrorInvalidValue;
  cudaError_t e;
  if (dtype == 0) {
    if ((e = setup_once<float, kLevelRowsF32, kLevelCols, Q>()) != cudaSuccess) return e;
    retrieve_batch_dispatch<float, kLevelRowsF32, kLevelRowsF32 / 2, kLevelCols, Q>(ents, n, tiles, w16, ns, per_sm, st);
  } else {
    if ((e = setup_once<double, kLevelRowsF64, kLevelCols, Q>()) != cudaSuccess) return e;
    retrieve_batch_dispatch<double, kLevelRowsF64, kLevelRowsF64, kLevelCols, Q>(ents, n, tiles, w16, ns, per_sm, st);
  }
  return cudaGetLastError();
}

}  // namespace
}  // namespace ipc
