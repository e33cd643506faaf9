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

#include <algorithm>

#include "ipc_device.cuh"
#include "ipc_internal.h"
#include "ipc_table_kernels.h"

namespace ipc {
namespace {
using namespace dev;

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

// The range of up to kRangeBatch arrays in one launch: array j takes blocks
// blk[j] .. blk[j + 1] - 1 of a one-dimensional grid, in proportion to the
// arrays' sizes; its blocks reduce it as k_range does, and its first block
// also copies the array's first value (the anchor) as f64 bits into x0[j].
struct RangeBlocks {
  uint32_t blk[kRangeBatch + 1];
};

template <class T>
__global__ void __launch_bounds__(256) k_range_batch(RangeBatch rb, RangeBlocks bl, int narr) {
  int lo = 0, hi = narr - 1;  // the last j with blk[j] <= blockIdx.x
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (bl.blk[mid] <= blockIdx.x) lo = mid;
    else hi = mid - 1;
  }
  const int j = lo;
  const uint32_t b0 = bl.blk[j], nb = bl.blk[j + 1] - b0;
  const T* __restrict__ x = (const T*)rb.x[j];
  const uint64_t n = rb.n[j];
  unsigned long long* acc = rb.acc + 4 * j;
  if (blockIdx.x == b0 && threadIdx.x == 0 && n)
    rb.x0[j] = (unsigned long long)__double_as_longlong((double)__ldg(x));
  typedef typename Vec16<T>::type V;
  constexpr int VN = Vec16<T>::n;
  RangeAcc<T> r{(T)0, (T)0, (T)0, 0ULL};
  const uint64_t tid = (blockIdx.x - b0) * (uint64_t)blockDim.x + threadIdx.x;
  const uint64_t nth = (uint64_t)nb * blockDim.x;
  const uint64_t mis = ((uintptr_t)x & 15) / sizeof(T);
  const uint64_t head = mis ? ((uint64_t)VN - mis < n ? (uint64_t)VN - mis : n) : 0;
  if (tid < head) r.add(__ldg(x + tid));
  const uint64_t nv = (n - head) / VN;
  const V* xv = reinterpret_cast<const V*>(x + head);
  for (uint64_t i = tid; i < nv; i += nth) {
    const V v = __ldg(xv + i);
    const T* e = reinterpret_cast<const T*>(&v);
#pragma unroll
    for (int q = 0; q < VN; ++q) r.add(e[q]);
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

template <class T>
__global__ void k_anchor(T* out, double v) { out[0] = (T)v; }

template <class T>
__global__ void k_anchors(const AnchorEntry* __restrict__ a, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) ((T*)a[i].out)[0] = (T)a[i].v;
}

__global__ void k_set_quant(CompressEntry* __restrict__ e, int n, const uint4* __restrict__ q) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t f = e[i].o.field;
  uint4* d = reinterpret_cast<uint4*>(e[i].quant);
  d[0] = q[2 * f];
  d[1] = q[2 * f + 1];
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

// ---------------------------------------------------------------------------
// Segmented device streams <-> packed container streams.
// A word w of the stage's word grid is (row r = w / wr, column j = w % wr);
// r = plane * m1 + rr; its segment is (plane, rr / RB, j / CW) and its
// segment-local index is (rr % RB) * CW + j % CW.
// ---------------------------------------------------------------------------
struct Loc {
  uint64_t g;
  uint32_t li;
};
__device__ __forceinline__ Loc locate(const StageArgs& a, uint64_t w) {
  const uint64_t r = w / a.wr, j = w - r * a.wr;
  const uint64_t pl = r / a.m1, rr = r - pl * a.m1;
  Loc l;
  l.g = (pl * a.nrb + rr / a.RB) * a.nct + j / a.CW;
  l.li = (uint32_t)((rr % a.RB) * a.CW + j % a.CW);
  return l;
}
// Slot of a nonzero word in its segment: the words of every 32-word group
// are compacted at the group's own 32-word slot.
__device__ __forceinline__ uint32_t seg_rank(const uint32_t* segbm, uint32_t li) {
  return (li & ~31u) + __popc(segbm[li >> 5] & ((1u << (li & 31)) - 1u));
}

// Export step 1: packed bitmap word q of every plane (gathered from the
// segment bitmaps). grid = (ceil(nbm / 256), 32).
__global__ void k_pack_bits(StageArgs a, StageDescs ds, const uint32_t* __restrict__ bm,
                            uint32_t* __restrict__ bits) {
  const int k = blockIdx.y;
  const uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (q >= a.nbm) return;
  uint32_t v = 0;
  if (ds.p[k].mode != 0) {
    for (int i = 0; i < 32; ++i) {
      const uint64_t w = 32 * q + i;
      if (w >= a.W) break;
      const Loc l = locate(a, w);
      v |= ((bm[ds.p[k].bm_off + l.g * a.bw + (l.li >> 5)] >> (l.li & 31)) & 1u) << i;
    }
  }
  bits[(uint64_t)k * a.nbm + q] = v;
}

// Exclusive prefix of the population of the packed bitmap words, per plane
// (blockIdx.x = k); flags a population that differs from the stream's nnz.
__global__ void __launch_bounds__(1024) k_scan_bits(StageArgs a, StageDescs ds,
                                                    const uint32_t* __restrict__ bits,
                                                    uint32_t* __restrict__ rank,
                                                    unsigned int* bad) {
  __shared__ uint32_t sh[33];
  const int k = blockIdx.x;
  const PlaneDesc pd = ds.p[k];
  if (pd.mode == 0) return;
  uint32_t run = 0;
  for (uint64_t base = 0; base < a.nbm; base += 1024) {
    const uint64_t q = base + threadIdx.x;
    const uint32_t v = q < a.nbm ? __popc(bits[(uint64_t)k * a.nbm + q]) : 0u;
    uint32_t tot;
    const uint32_t ex = block_exscan(v, &tot, sh);
    if (q < a.nbm) rank[(uint64_t)k * a.nbm + q] = run + ex;
    run += tot;
  }
  if (threadIdx.x == 0 && bad && run != pd.nnz) atomicOr(bad, 1u);
}

// Export step 2: every word of every plane into its packed position.
// grid = (ceil(W / 256), 32).
__global__ void k_pack_words(StageArgs a, StageDescs ds, const uint32_t* __restrict__ cap,
                             const uint32_t* __restrict__ bm, const uint32_t* __restrict__ bits,
                             const uint32_t* __restrict__ rank, uint32_t* __restrict__ blob) {
  const int k = blockIdx.y;
  const PlaneDesc pd = ds.p[k];
  const uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (w == 0) blob[pd.pk_off] = pd.nnz;
  if (pd.mode == 0 || w >= a.W) return;
  const uint64_t q = w >> 5;
  const uint32_t bq = bits[(uint64_t)k * a.nbm + q];
  const uint32_t bit = (bq >> (w & 31)) & 1u;
  uint32_t v = 0;
  if (bit) {
    const Loc l = locate(a, w);
    const uint32_t* segbm = bm + pd.bm_off + l.g * a.bw;
    v = cap[pd.cap_off + l.g * (uint64_t)a.RB * a.CW + seg_rank(segbm, l.li)];
  }
  if (pd.mode == 2) {
    blob[pd.pk_off + 1 + w] = v;
    return;
  }
  if ((w & 31) == 0) blob[pd.pk_off + 1 + q] = bq;
  if (bit)
    blob[pd.pk_off + 1 + a.nbm + rank[(uint64_t)k * a.nbm + q] +
         __popc(bq & ((1u << (w & 31)) - 1u))] = v;
}

// Import step 1: packed bitmap of every plane (dense planes: from the
// values). grid = (ceil(nbm / 256), 32).
__global__ void k_unpack_bits(StageArgs a, StageDescs ds, const uint32_t* __restrict__ blob,
                              uint32_t* __restrict__ bits, unsigned int* bad) {
  const int k = blockIdx.y;
  const PlaneDesc pd = ds.p[k];
  const uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (q >= a.nbm) return;
  uint32_t v = 0;
  if (pd.mode == 1) {
    v = blob[pd.pk_off + 1 + q];
    const uint32_t tail = (uint32_t)(a.W & 31);
    if (q == a.nbm - 1 && tail && (v >> tail) != 0) atomicOr(bad, 1u);
  } else if (pd.mode == 2) {
    for (int i = 0; i < 32; ++i) {
      const uint64_t w = 32 * q + i;
      if (w >= a.W) break;
      v |= (blob[pd.pk_off + 1 + w] != 0 ? 1u : 0u) << i;
    }
  }
  bits[(uint64_t)k * a.nbm + q] = v;
}

// Import step 2: segment bitmaps. grid = (ceil(nseg * bw / 256), 32).
__global__ void k_unpack_segbits(StageArgs a, StageDescs ds, uint64_t nseg,
                                 const uint32_t* __restrict__ bits, uint32_t* __restrict__ bm,
                                 uint32_t kmask) {
  const int k = blockIdx.y;
  if (!((kmask >> k) & 1u)) return;  // a plane this upload leaves as it is
  const PlaneDesc pd = ds.p[k];
  const uint64_t u = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (u >= nseg * a.bw) return;
  const uint64_t g = u / a.bw;
  const uint32_t vw = (uint32_t)(u - g * a.bw);
  uint32_t word = 0;
  if (pd.mode != 0) {
    const uint64_t ct = g % a.nct, rest = g / a.nct;
    const uint64_t rb = rest % a.nrb, pl = rest / a.nrb;
    const uint32_t nw = a.RB * a.CW;
    for (int i = 0; i < 32; ++i) {
      const uint32_t li = vw * 32 + i;
      if (li >= nw) break;
      const uint64_t rr = rb * a.RB + li / a.CW, j = ct * a.CW + li % a.CW;
      if (rr >= a.m1 || j >= a.wr) continue;
      const uint64_t w = (pl * a.m1 + rr) * a.wr + j;
      word |= ((bits[(uint64_t)k * a.nbm + (w >> 5)] >> (w & 31)) & 1u) << i;
    }
  }
  bm[pd.bm_off + u] = word;
}

// Import step 3: every nonzero word into its segment slot. grid = (ceil(W / 256), 32).
__global__ void k_unpack_words(StageArgs a, StageDescs ds, const uint32_t* __restrict__ blob,
                               const uint32_t* __restrict__ bits,
                               const uint32_t* __restrict__ rank, const uint32_t* __restrict__ bm,
                               uint32_t* __restrict__ cap, unsigned int* bad) {
  const int k = blockIdx.y;
  const PlaneDesc pd = ds.p[k];
  const uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (pd.mode == 0 || w >= a.W) return;
  const uint64_t q = w >> 5;
  const uint32_t bq = bits[(uint64_t)k * a.nbm + q];
  if (!((bq >> (w & 31)) & 1u)) return;
  uint32_t v;
  if (pd.mode == 2) {
    v = blob[pd.pk_off + 1 + w];
  } else {
    const uint64_t p = (uint64_t)rank[(uint64_t)k * a.nbm + q] + __popc(bq & ((1u << (w & 31)) - 1u));
    if (p >= pd.nnz) {
      atomicOr(bad, 1u);
      return;
    }
    v = blob[pd.pk_off + 1 + a.nbm + p];
    if (v == 0) atomicOr(bad, 1u);
  }
  const Loc l = locate(a, w);
  const uint32_t* segbm = bm + pd.bm_off + l.g * a.bw;
  cap[pd.cap_off + l.g * (uint64_t)a.RB * a.CW + seg_rank(segbm, l.li)] = v;
}

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

// nmax is not needed: the blocks follow every array's own size.
cudaError_t launch_range_batch(int dtype, const RangeBatch& rb, int n, uint64_t /*nmax*/,
                               cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (n > kRangeBatch) return cudaErrorInvalidValue;
  // about 152 * 8 blocks over the batch in proportion to the arrays' sizes,
  // each array at least one and at most one per 1024 values
  RangeBlocks bl{};
  uint64_t tot = 0;
  for (int j = 0; j < n; ++j) tot += rb.n[j];
  const uint64_t target = 152 * 8;
  uint64_t b = 0;
  for (int j = 0; j < n; ++j) {
    bl.blk[j] = (uint32_t)b;
    uint64_t per = tot ? (rb.n[j] * target + tot - 1) / tot : 1;
    per = std::min<uint64_t>(per, (rb.n[j] + 1023) / 1024);
    b += std::max<uint64_t>(per, 1);
  }
  bl.blk[n] = (uint32_t)b;
  if (dtype == 0) k_range_batch<float><<<(unsigned)b, 256, 0, st>>>(rb, bl, n);
  else k_range_batch<double><<<(unsigned)b, 256, 0, st>>>(rb, bl, n);
  return cudaGetLastError();
}

cudaError_t launch_set_anchor(int dtype, void* out, double v, cudaStream_t st) {
  if (dtype == 0) k_anchor<float><<<1, 1, 0, st>>>((float*)out, v);
  else k_anchor<double><<<1, 1, 0, st>>>((double*)out, v);
  return cudaGetLastError();
}

cudaError_t launch_set_anchors(int dtype, const AnchorEntry* a, int n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)((n + 127) / 128);
  if (dtype == 0) k_anchors<float><<<grid, 128, 0, st>>>(a, n);
  else k_anchors<double><<<grid, 128, 0, st>>>(a, n);
  return cudaGetLastError();
}

cudaError_t launch_set_quant(CompressEntry* e, int n, const unsigned char* q, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_set_quant<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(e, n, reinterpret_cast<const uint4*>(q));
  return cudaGetLastError();
}

cudaError_t launch_pack(const StageArgs& a, const StageDescs& d, const uint32_t* cap,
                        const uint32_t* bm, uint32_t* tmp, uint32_t* blob, cudaStream_t st) {
  uint32_t* bits = tmp;
  uint32_t* rank = tmp + 32 * a.nbm;
  k_pack_bits<<<dim3(grid_for(a.nbm, 256, 1u << 30), 32), 256, 0, st>>>(a, d, bm, bits);
  k_scan_bits<<<32, 1024, 0, st>>>(a, d, bits, rank, nullptr);
  k_pack_words<<<dim3(grid_for(a.W, 256, 1u << 30), 32), 256, 0, st>>>(a, d, cap, bm, bits, rank,
                                                                        blob);
  return cudaGetLastError();
}

cudaError_t launch_unpack(const StageArgs& a, const StageDescs& d, uint64_t nseg,
                          const uint32_t* blob, uint32_t* tmp, uint32_t* cap, uint32_t* bm,
                          unsigned int* flags, uint32_t kmask, cudaStream_t st) {
  uint32_t* bits = tmp;
  uint32_t* rank = tmp + 32 * a.nbm;
  k_unpack_bits<<<dim3(grid_for(a.nbm, 256, 1u << 30), 32), 256, 0, st>>>(a, d, blob, bits, flags);
  k_scan_bits<<<32, 1024, 0, st>>>(a, d, bits, rank, flags);
  k_unpack_segbits<<<dim3(grid_for(nseg * a.bw, 256, 1u << 30), 32), 256, 0, st>>>(a, d, nseg, bits,
                                                                                   bm, kmask);
  k_unpack_words<<<dim3(grid_for(a.W, 256, 1u << 30), 32), 256, 0, st>>>(a, d, blob, bits, rank, bm,
                                                                          cap, flags);
  return cudaGetLastError();
}

}  // namespace ipc
