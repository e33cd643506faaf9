// sm_103a kernels of libipcomp: range reduction, one compression launch per
// interpolation sweep (predict + quantize + negabinary/XOR + bitplane
// transpose + per-tile compaction), stream packing, and one reconstruction
// launch per sweep (plane fetch + transpose back + decode + predict).
//
// Floating point: every operation is an explicit round-to-nearest intrinsic
// (no FMA contraction; the library is also built with -fmad=false), in the
// same order as the method's definition, so results are bitwise reproducible.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ipc_internal.h"

namespace ipc {
namespace {

// ---------------------------------------------------------------------------
// Element-type arithmetic (round-to-nearest, no contraction).
// ---------------------------------------------------------------------------
template <class T> struct FP;
template <> struct FP<float> {
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float fabs_(float a) { return fabsf(a); }
  // Round-to-nearest-even of |t| <= 2^21 by adding 1.5*2^23: the sum lies in
  // [2^23, 2^24) where the spacing is 1, so the addition itself rounds. The
  // integer is the distance of the bit patterns; the sign of a zero result
  // follows t (as nearbyint does).
  static __device__ __forceinline__ float rint_(float t, int32_t* qi) {
    const float magic = 12582912.0f;
    float y = __fadd_rn(t, magic);
    *qi = __float_as_int(y) - 0x4B400000;
    return copysignf(__fsub_rn(y, magic), t);
  }
  static __device__ __forceinline__ float from_code(int64_t q) {
    return __int2float_rn((int)q);
  }
};
template <> struct FP<double> {
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double fabs_(double a) { return fabs(a); }
  static __device__ __forceinline__ double rint_(double t, int32_t* qi) {
    const double magic = 6755399441055744.0;  // 1.5 * 2^52
    double y = __dadd_rn(t, magic);
    *qi = (int32_t)(__double_as_longlong(y) - 0x4338000000000000LL);
    return copysign(__dsub_rn(y, magic), t);
  }
  static __device__ __forceinline__ double from_code(int64_t q) { return __ll2double_rn(q); }
};

// Interpolation along dimension d (Eq. 2 cubic when the +-3s neighbours are
// inside the line, Eq. 1 linear when i+s is inside, else copy of i-s).
template <class T>
__device__ __forceinline__ T predict(const T* __restrict__ xh, int64_t idx, int64_t id,
                                     int64_t s, int64_t Nd, int64_t sd, int cubic) {
  const int64_t o1 = s * sd;
  T b = __ldg(xh + idx - o1);
  if (id + s > Nd - 1) return b;
  T c = __ldg(xh + idx + o1);
  if (cubic && id - 3 * s >= 0 && id + 3 * s <= Nd - 1) {
    T a = __ldg(xh + idx - 3 * o1);
    T d = __ldg(xh + idx + 3 * o1);
    T u = FP<T>::add(b, c);
    T v = FP<T>::add(a, d);
    T w = FP<T>::mul((T)9, u);
    T z = FP<T>::sub(w, v);
    return FP<T>::mul(z, (T)0.0625);
  }
  T u = FP<T>::add(b, c);
  return FP<T>::mul(u, (T)0.5);
}

__device__ __forceinline__ uint32_t negabinary(int32_t q) {
  return ((uint32_t)q + 0xAAAAAAAAu) ^ 0xAAAAAAAAu;
}
__device__ __forceinline__ int64_t negabinary_inv(uint32_t n) {
  return (int64_t)(n ^ 0xAAAAAAAAu) - (int64_t)0xAAAAAAAAu;
}
// 2-prefix predictive XOR (Sec. 4.4.1): e = n ^ n>>1 ^ n>>2.
__device__ __forceinline__ uint32_t xor_encode(uint32_t n) { return n ^ (n >> 1) ^ (n >> 2); }
// Inverse: n = e * (1 + x + x^2)^-1 over GF(2) with x the right shift.
// (1 + x + x^2)^-1 = (1 + x) / (1 + x^3): a prefix XOR at stride 3 (four
// doubling steps reach shifts >= 32) followed by one XOR with the shift by 1.
__device__ __forceinline__ uint32_t xor_decode(uint32_t e) {
  uint32_t g = e;
  g ^= g >> 3;
  g ^= g >> 6;
  g ^= g >> 12;
  g ^= g >> 24;
  return g ^ (g >> 1);
}

// In-register transpose of a 32x32 bit matrix (row i = a[i], column k = bit
// k): afterwards bit i of a[k] is the former bit k of a[i]. Five rounds of
// block swaps (16, 8, 4, 2, 1).
template <int J, uint32_t M>
__device__ __forceinline__ void tround(uint32_t (&a)[32]) {
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    if ((i & J) == 0) {
      uint32_t t = ((a[i] >> J) ^ a[i + J]) & M;
      a[i + J] ^= t;
      a[i] ^= t << J;
    }
  }
}
__device__ __forceinline__ void transpose32(uint32_t (&a)[32]) {
  tround<16, 0x0000FFFFu>(a);
  tround<8, 0x00FF00FFu>(a);
  tround<4, 0x0F0F0F0Fu>(a);
  tround<2, 0x33333333u>(a);
  tround<1, 0x55555555u>(a);
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Row/word cursor over a stage's word space: word w = (row r, word j of the
// row); row r = (c0, c1) of the lattice. Advanced incrementally.
struct Cursor {
  uint64_t r, j, c0, c1;
  __device__ __forceinline__ void init(uint64_t w, const StageArgs& a) {
    r = w / a.wr;
    j = w - r * a.wr;
    c0 = r / (uint64_t)a.m[1];
    c1 = r - c0 * (uint64_t)a.m[1];
  }
  __device__ __forceinline__ void next(const StageArgs& a) {
    if (++j == a.wr) {
      j = 0;
      ++r;
      if (++c1 == (uint64_t)a.m[1]) { c1 = 0; ++c0; }
    }
  }
  __device__ __forceinline__ int64_t row_base(const StageArgs& a, int64_t* i0, int64_t* i1) const {
    *i0 = a.start[0] + (int64_t)c0 * a.step[0];
    *i1 = a.start[1] + (int64_t)c1 * a.step[1];
    return *i0 * a.stride[0] + *i1 * a.stride[1];
  }
};

// ---------------------------------------------------------------------------
// Range: min, max, max|x| over finite values (ordered-integer atomics).
// acc[0] = ordered key of min, acc[1] = ordered key of max, acc[2] = bits of
// max|x|, acc[3] = number of finite values.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long okey(double v) {
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ULL);
}

template <class T> struct Vec16;
template <> struct Vec16<float> { typedef float4 type; static constexpr int n = 4; };
template <> struct Vec16<double> { typedef double2 type; static constexpr int n = 2; };

template <class T>
struct RangeAcc {
  T mn, mx, ma;
  unsigned long long cnt;
  __device__ __forceinline__ void add(T v) {
    if (!isfinite(v)) return;
    mn = cnt ? (v < mn ? v : mn) : v;
    mx = cnt ? (v > mx ? v : mx) : v;
    const T a = FP<T>::fabs_(v);
    ma = cnt ? (a > ma ? a : ma) : a;
    ++cnt;
  }
};

// Min / max / max|x| in the element type (the values are exact, so no
// wider arithmetic is needed), 16-byte vector loads, then one ordered-key
// atomic per warp.
template <class T>
__global__ void __launch_bounds__(256) k_range(const T* __restrict__ x, uint64_t n,
                                               unsigned long long* acc) {
  typedef typename Vec16<T>::type V;
  constexpr int VN = Vec16<T>::n;
  RangeAcc<T> r{(T)0, (T)0, (T)0, 0ULL};
  const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
  // scalar head up to 16-byte alignment
  const uint64_t mis = ((uintptr_t)x & 15) / sizeof(T);
  const uint64_t head = mis ? ((uint64_t)VN - mis < n ? (uint64_t)VN - mis : n) : 0;
  if (tid < head) r.add(__ldg(x + tid));
  const uint64_t nv = (n - head) / VN;
  const V* xv = reinterpret_cast<const V*>(x + head);
  for (uint64_t i = tid; i < nv; i += nth) {
    const V v = __ldg(xv + i);
    const T* e = reinterpret_cast<const T*>(&v);
#pragma unroll
    for (int j = 0; j < VN; ++j) r.add(e[j]);
  }
  for (uint64_t i = head + nv * VN + tid; i < n; i += nth) r.add(__ldg(x + i));
  unsigned long long kmn = r.cnt ? okey((double)r.mn) : ~0ULL;
  unsigned long long kmx = r.cnt ? okey((double)r.mx) : 0ULL;
  unsigned long long kma = r.cnt ? (unsigned long long)__double_as_longlong((double)r.ma) : 0ULL;
  unsigned long long cnt = r.cnt;
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    kmn = min(kmn, __shfl_xor_sync(~0u, kmn, o));
    kmx = max(kmx, __shfl_xor_sync(~0u, kmx, o));
    kma = max(kma, __shfl_xor_sync(~0u, kma, o));
    cnt += __shfl_xor_sync(~0u, cnt, o);
  }
  if ((threadIdx.x & 31) == 0 && cnt) {
    atomicMin(acc + 0, kmn);
    atomicMax(acc + 1, kmx);
    atomicMax(acc + 2, kma);
    atomicAdd(acc + 3, cnt);
  }
}

// ---------------------------------------------------------------------------
// Compression of one sweep. CTA = 8 warps = one 256-word segment.
// Phase A (lane per code): warp wi walks its 32 words; lane L computes code
//   32j + L of word (r, j): prediction from xhat, quantization, xhat write,
//   negabinary + XOR -> E, stored to shared memory.
// Phase B (thread per word): the 32 codes of one word are read back and the
//   32x32 bit matrix transposed: pw[k] = plane-k word.
// Phase C: zero-word bitmap per plane (warp ballot), prefix of the warps'
//   nonzero counts, nonzero words stored compacted at the segment's start of
//   the plane's capacity array, per-plane nonzero counter.
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(256) k_compress(StageArgs a, const T* __restrict__ x,
                                                  T* xh, int write_xh, QuantArgs<T> qa,
                                                  int stage, SweepOut o, StageDescs ds) {
  __shared__ uint32_t Es[8][32][33];
  __shared__ uint32_t wcnt[32][8];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const uint64_t tile = blockIdx.x;
  const uint64_t wbase = tile * kTileWords + (uint64_t)wi * 32;
  const int d = a.d;
  const int64_t sd = a.stride[d];
  uint32_t orN = 0, qmax = 0;

  Cursor cur;
  cur.init(wbase < a.W ? wbase : 0, a);
  for (int i = 0; i < 32; ++i) {
    uint32_t E = 0;
    const uint64_t w = wbase + i;
    if (w < a.W) {
      const uint64_t p = cur.j * 32 + lane;
      if (p < (uint64_t)a.m[2]) {
        int64_t i0, i1;
        const int64_t rb = cur.row_base(a, &i0, &i1);
        const int64_t i2 = a.start[2] + (int64_t)p * a.step[2];
        const int64_t idx = rb + i2;
        const int64_t id = d == 0 ? i0 : (d == 1 ? i1 : i2);
        const T pred = predict<T>(xh, idx, id, a.s, a.N[d], sd, a.cubic);
        const T xv = __ldg(x + idx);
        const T diff = FP<T>::sub(xv, pred);
        const T t = FP<T>::mul(diff, qa.inv2eb);
        T rec = xv;
        int32_t q = 0;
        bool outlier = !(FP<T>::fabs_(t) <= qa.R);
        if (!outlier) {
          int32_t qi;
          const T qf = FP<T>::rint_(t, &qi);
          const T r = FP<T>::mul(qf, qa.twoeb);
          const T rc = FP<T>::add(pred, r);
          const T err = FP<T>::sub(xv, rc);
          if (FP<T>::fabs_(err) <= qa.ebchk) {
            q = qi;
            rec = rc;
          } else {
            outlier = true;
          }
        }
        if (outlier) {
          unsigned long long slot = atomicAdd(o.outl_count, 1ULL);
          if (slot < o.outl_cap) {
            o.outl_key[slot] = ((unsigned long long)stage << 40) |
                               (unsigned long long)(cur.r * (uint64_t)a.m[2] + p);
            o.outl_val[slot] = (double)xv;
          }
        }
        if (write_xh) xh[idx] = rec;
        const uint32_t N = negabinary(q);
        orN |= N;
        qmax = max(qmax, (uint32_t)(q < 0 ? -q : q));
        E = xor_encode(N);
      }
      cur.next(a);
    }
    Es[wi][i][lane] = E;
  }
  __syncwarp();

  uint32_t pw[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) pw[i] = Es[wi][lane][i];
  transpose32(pw);

  const uint32_t lt = lanemask_lt();
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    const uint32_t mk = __ballot_sync(~0u, pw[k] != 0);
    if (lane == k) {
      o.bm[ds.p[k].bm_off + tile * kTileBitmapWords + wi] = mk;
      wcnt[k][wi] = __popc(mk);
    }
  }
  orN = __reduce_or_sync(~0u, orN);
  qmax = __reduce_max_sync(~0u, qmax);
  if (lane == 0) {
    if (orN) atomicOr(o.stat + 2 * stage, orN);
    if (qmax) atomicMax(o.stat + 2 * stage + 1, qmax);
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int k = threadIdx.x;
    uint32_t run = 0;
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      const uint32_t c = wcnt[k][v];
      wcnt[k][v] = run;
      run += c;
    }
    if (run) atomicAdd(o.nnz + 32 * stage + k, run);
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    const uint32_t mk = __ballot_sync(~0u, pw[k] != 0);
    if (pw[k])
      o.cap[ds.p[k].cap_off + tile * kTileWords + wcnt[k][wi] + __popc(mk & lt)] = pw[k];
  }
}

// Block-wide exclusive scan of one value per thread (blockDim = 1024).
__device__ __forceinline__ uint32_t block_exscan(uint32_t v, uint32_t* total,
                                                 uint32_t* sh /* 33 */) {
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  uint32_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(~0u, inc, o);
    if (lane >= o) inc += t;
  }
  __syncthreads();
  if (lane == 31) sh[wi] = inc;
  __syncthreads();
  if (wi == 0) {
    uint32_t s = sh[lane];
    uint32_t si = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t t = __shfl_up_sync(~0u, si, o);
      if (lane >= o) si += t;
    }
    sh[lane] = si - s;
    if (lane == 31) sh[32] = si;
  }
  __syncthreads();
  *total = sh[32];
  return sh[wi] + inc - v;
}

// Per plane (blockIdx.x = k) of a sparse stream: exclusive prefix of the
// population of every 256-word segment. `packed` selects the bitmap source.
__global__ void __launch_bounds__(1024) k_seg_rank(StageArgs a, StageDescs ds, int packed,
                                                   const uint32_t* __restrict__ bm,
                                                   uint32_t* __restrict__ rank,
                                                   unsigned int* bad) {
  __shared__ uint32_t sh[33];
  const int k = blockIdx.x;
  const PlaneDesc pd = ds.p[k];
  if (pd.mode != 1) return;
  const uint64_t nbm = (a.W + 31) / 32;
  const uint32_t* src = packed ? bm + pd.pk_off + 1 : bm + pd.bm_off;
  uint32_t run = 0;
  for (uint64_t base = 0; base < a.ntiles; base += 1024) {
    const uint64_t t = base + threadIdx.x;
    uint32_t v = 0;
    if (t < a.ntiles) {
#pragma unroll
      for (int j = 0; j < kTileBitmapWords; ++j) {
        const uint64_t bw = t * kTileBitmapWords + j;
        if (bw < nbm) v += __popc(src[bw]);
      }
    }
    uint32_t tot;
    const uint32_t ex = block_exscan(v, &tot, sh);
    if (t < a.ntiles) rank[(uint64_t)k * a.ntiles + t] = run + ex;
    run += tot;
  }
  if (threadIdx.x == 0) {
    const uint32_t tail = (uint32_t)(a.W & 31);
    const bool extra = tail && (src[nbm - 1] >> tail) != 0;
    if (run != pd.nnz || extra) atomicOr(bad, 1u);
  }
}

// Segmented -> packed stream of one (segment, plane) (export). grid = (ntiles, 32).
__global__ void __launch_bounds__(256) k_pack(StageArgs a, StageDescs ds,
                                              const uint32_t* __restrict__ cap,
                                              const uint32_t* __restrict__ bm,
                                              const uint32_t* __restrict__ rank,
                                              uint32_t* __restrict__ blob) {
  __shared__ uint32_t sbm[8];
  __shared__ uint32_t pre[9];
  const int k = blockIdx.y;
  const uint64_t tile = blockIdx.x;
  const PlaneDesc pd = ds.p[k];
  if (tile == 0 && threadIdx.x == 0) blob[pd.pk_off] = pd.nnz;
  if (pd.mode == 0) return;
  const uint64_t W = a.W, nbm = (W + 31) / 32;
  if (threadIdx.x < 8) sbm[threadIdx.x] = bm[pd.bm_off + tile * kTileBitmapWords + threadIdx.x];
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int v = 0; v < 8; ++v) { pre[v] = run; run += __popc(sbm[v]); }
    pre[8] = run;
  }
  __syncthreads();
  const uint32_t* seg = cap + pd.cap_off + tile * kTileWords;
  if (pd.mode == 1) {
    if (threadIdx.x < 8) {
      const uint64_t bw = tile * kTileBitmapWords + threadIdx.x;
      if (bw < nbm) blob[pd.pk_off + 1 + bw] = sbm[threadIdx.x];
    }
    const uint32_t r0 = rank[(uint64_t)k * a.ntiles + tile];
    for (uint32_t i = threadIdx.x; i < pre[8]; i += blockDim.x)
      blob[pd.pk_off + 1 + nbm + r0 + i] = seg[i];
    return;
  }
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const uint64_t w = tile * kTileWords + threadIdx.x;
  if (w < W) {
    const uint32_t m = sbm[wi];
    blob[pd.pk_off + 1 + w] = ((m >> lane) & 1u) ? seg[pre[wi] + __popc(m & lanemask_lt())] : 0u;
  }
}

// Packed stream -> segmented (import). grid = (ntiles, 32). Flags payload
// words that are zero; counts the nonzero words of dense streams in chk.
__global__ void __launch_bounds__(256) k_unpack(StageArgs a, StageDescs ds,
                                                const uint32_t* __restrict__ blob,
                                                const uint32_t* __restrict__ rank,
                                                uint32_t* __restrict__ cap,
                                                uint32_t* __restrict__ bm, unsigned int* bad,
                                                unsigned int* chk) {
  __shared__ uint32_t sbm[8];
  __shared__ uint32_t pre[9];
  const int k = blockIdx.y;
  const uint64_t tile = blockIdx.x;
  const PlaneDesc pd = ds.p[k];
  const uint64_t W = a.W, nbm = (W + 31) / 32;
  uint32_t* seg = cap + pd.cap_off + tile * kTileWords;
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  if (pd.mode == 0) {
    if (threadIdx.x < 8) bm[pd.bm_off + tile * kTileBitmapWords + threadIdx.x] = 0u;
    return;
  }
  if (pd.mode == 1) {
    if (threadIdx.x < 8) {
      const uint64_t bw = tile * kTileBitmapWords + threadIdx.x;
      const uint32_t v = bw < nbm ? blob[pd.pk_off + 1 + bw] : 0u;
      sbm[threadIdx.x] = v;
      bm[pd.bm_off + bw] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t run = 0;
      for (int v = 0; v < 8; ++v) run += __popc(sbm[v]);
      pre[8] = run;
    }
    __syncthreads();
    const uint32_t r0 = rank[(uint64_t)k * a.ntiles + tile];
    for (uint32_t i = threadIdx.x; i < pre[8]; i += blockDim.x) {
      const uint64_t src = 1 + nbm + (uint64_t)r0 + i;
      const uint32_t v = src < 1 + nbm + pd.nnz ? blob[pd.pk_off + src] : 0u;
      if (v == 0) atomicOr(bad, 1u);
      seg[i] = v;
    }
    return;
  }
  const uint64_t w = tile * kTileWords + threadIdx.x;
  const uint32_t v = w < W ? blob[pd.pk_off + 1 + w] : 0u;
  const uint32_t m = __ballot_sync(~0u, v != 0);
  if (lane == 0) {
    sbm[wi] = m;
    bm[pd.bm_off + tile * kTileBitmapWords + wi] = m;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int q = 0; q < 8; ++q) { pre[q] = run; run += __popc(sbm[q]); }
    if (run) atomicAdd(chk + k, run);
  }
  __syncthreads();
  if (v) seg[pre[wi] + __popc(m & lanemask_lt())] = v;
}

// ---------------------------------------------------------------------------
// Reconstruction of one sweep (Algorithm 1). CTA = one 256-word segment.
// Thread per word: fetch the word of every selected plane (bitmap bit + rank
// inside the segment), transpose back to per-code E, undo the XOR, drop the
// unloaded digits, keep N in shared memory.
// Lane per code: q' = negabinary^-1(N), xhat' = P xhat' + q' 2eb.
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(256) k_retrieve(StageArgs a, T* out, T twoeb, StageDescs ds,
                                                  int b, const uint32_t* __restrict__ cap,
                                                  const uint32_t* __restrict__ bm) {
  __shared__ uint32_t Ns[8][32][33];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const uint64_t tile = blockIdx.x;
  const uint64_t W = a.W;
  const uint64_t wbase = tile * kTileWords + (uint64_t)wi * 32;
  const uint32_t lt = lanemask_lt();
  uint32_t pw[32];
#pragma unroll
  for (int k = 31; k >= 0; --k) {
    pw[k] = 0;
    if (k >= b && ds.p[k].nnz) {
      const uint32_t* bmp = bm + ds.p[k].bm_off + tile * kTileBitmapWords;
      const uint32_t m = __ldg(bmp + wi);
      uint32_t before = lane < wi ? __popc(__ldg(bmp + lane)) : 0u;
      before = __reduce_add_sync(~0u, before);
      if ((m >> lane) & 1u)
        pw[k] = __ldg(cap + ds.p[k].cap_off + tile * kTileWords + before + __popc(m & lt));
    }
  }
  transpose32(pw);
  const uint32_t keep = b >= 32 ? 0u : (0xFFFFFFFFu << b);
#pragma unroll
  for (int i = 0; i < 32; ++i) Ns[wi][lane][i] = xor_decode(pw[i] & keep) & keep;
  __syncwarp();

  const int d = a.d;
  const int64_t sd = a.stride[d];
  Cursor cur;
  cur.init(wbase < W ? wbase : 0, a);
  for (int i = 0; i < 32; ++i) {
    if (wbase + i >= W) break;
    const uint64_t p = cur.j * 32 + lane;
    if (p < (uint64_t)a.m[2]) {
      int64_t i0, i1;
      const int64_t rb = cur.row_base(a, &i0, &i1);
      const int64_t i2 = a.start[2] + (int64_t)p * a.step[2];
      const int64_t idx = rb + i2;
      const int64_t id = d == 0 ? i0 : (d == 1 ? i1 : i2);
      const T pred = predict<T>(out, idx, id, a.s, a.N[d], sd, a.cubic);
      const int64_t q = negabinary_inv(Ns[wi][i][lane]);
      const T r = FP<T>::mul(FP<T>::from_code(q), twoeb);
      out[idx] = FP<T>::add(pred, r);
    }
    cur.next(a);
  }
}

template <class T>
__global__ void k_outliers(StageArgs a, T* out, const uint64_t* __restrict__ idx,
                           const double* __restrict__ val, uint64_t n) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t ci = idx[i];
  const uint64_t r = ci / (uint64_t)a.m[2], p = ci - r * (uint64_t)a.m[2];
  const uint64_t c0 = r / (uint64_t)a.m[1], c1 = r - c0 * (uint64_t)a.m[1];
  const int64_t e = (a.start[0] + (int64_t)c0 * a.step[0]) * a.stride[0] +
                    (a.start[1] + (int64_t)c1 * a.step[1]) * a.stride[1] +
                    a.start[2] + (int64_t)p * a.step[2];
  out[e] = (T)val[i];
}

template <class T>
__global__ void k_anchor(T* out, double v) { out[0] = (T)v; }

unsigned grid_for(uint64_t n, unsigned block, unsigned cap) {
  uint64_t g = (n + block - 1) / block;
  if (g > cap) g = cap;
  return (unsigned)(g ? g : 1);
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
cudaError_t launch_range(int dtype, const void* x, uint64_t n, unsigned long long* acc,
                         cudaStream_t st) {
  const unsigned grid = grid_for(n / 4 + 1, 256, 152 * 8);
  if (dtype == 0) k_range<float><<<grid, 256, 0, st>>>((const float*)x, n, acc);
  else k_range<double><<<grid, 256, 0, st>>>((const double*)x, n, acc);
  return cudaGetLastError();
}

cudaError_t launch_compress_stage(int dtype, const StageArgs& a, const void* x, void* xh,
                                  int write_xh, const void* quant, int stage, const SweepOut& o,
                                  const StageDescs& d, cudaStream_t st) {
  const unsigned grid = (unsigned)a.ntiles;
  if (dtype == 0)
    k_compress<float><<<grid, 256, 0, st>>>(a, (const float*)x, (float*)xh, write_xh,
                                            *(const QuantArgs<float>*)quant, stage, o, d);
  else
    k_compress<double><<<grid, 256, 0, st>>>(a, (const double*)x, (double*)xh, write_xh,
                                             *(const QuantArgs<double>*)quant, stage, o, d);
  return cudaGetLastError();
}

cudaError_t launch_retrieve_stage(int dtype, const StageArgs& a, void* out, double twoeb,
                                  const StageDescs& d, int b, const uint32_t* cap,
                                  const uint32_t* bm, cudaStream_t st) {
  const unsigned grid = (unsigned)a.ntiles;
  if (dtype == 0)
    k_retrieve<float><<<grid, 256, 0, st>>>(a, (float*)out, (float)twoeb, d, b, cap, bm);
  else
    k_retrieve<double><<<grid, 256, 0, st>>>(a, (double*)out, twoeb, d, b, cap, bm);
  return cudaGetLastError();
}

cudaError_t launch_outlier_scatter(int dtype, const StageArgs& a, void* out,
                                   const uint64_t* idx, const double* val, uint64_t n,
                                   cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const unsigned grid = grid_for(n, 256, 1u << 30);
  if (dtype == 0) k_outliers<float><<<grid, 256, 0, st>>>(a, (float*)out, idx, val, n);
  else k_outliers<double><<<grid, 256, 0, st>>>(a, (double*)out, idx, val, n);
  return cudaGetLastError();
}

cudaError_t launch_set_anchor(int dtype, void* out, double v, cudaStream_t st) {
  if (dtype == 0) k_anchor<float><<<1, 1, 0, st>>>((float*)out, v);
  else k_anchor<double><<<1, 1, 0, st>>>((double*)out, v);
  return cudaGetLastError();
}

cudaError_t launch_seg_rank(const StageArgs& a, const StageDescs& d, int packed,
                            const uint32_t* bm, uint32_t* rank, unsigned int* bad,
                            cudaStream_t st) {
  k_seg_rank<<<32, 1024, 0, st>>>(a, d, packed, bm, rank, bad);
  return cudaGetLastError();
}

cudaError_t launch_pack(const StageArgs& a, const StageDescs& d, const uint32_t* cap,
                        const uint32_t* bm, const uint32_t* rank, uint32_t* blob,
                        cudaStream_t st) {
  k_pack<<<dim3((unsigned)a.ntiles, 32), 256, 0, st>>>(a, d, cap, bm, rank, blob);
  return cudaGetLastError();
}

cudaError_t launch_unpack(const StageArgs& a, const StageDescs& d, const uint32_t* blob,
                          const uint32_t* rank, uint32_t* cap, uint32_t* bm, unsigned int* bad,
                          unsigned int* chk, cudaStream_t st) {
  k_unpack<<<dim3((unsigned)a.ntiles, 32), 256, 0, st>>>(a, d, blob, rank, cap, bm, bad, chk);
  return cudaGetLastError();
}

}  // namespace ipc
