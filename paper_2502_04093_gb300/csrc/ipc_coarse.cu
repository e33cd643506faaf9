// The coarse levels of a reconstruction in one CTA per field (sm_103a).
//
// A level's launch of the tile kernels (ipc_level_kernels.cuh) costs a
// dependent chain of global loads per tile (bitmaps, plane words, known
// points) whatever the level's size, so the small coarse levels take
// several microseconds each for a few
// thousand points. Here one CTA reconstructs levels K .. Lc together in
// shared memory (Algorithm 1), Lc chosen by the host so that the level-Lc
// lattice and the codes of every stage of those levels fit:
//   phase A: every code word of every stage is decoded at once (its loaded
//     planes read through the zero-word bitmaps, the predictive XOR undone
//     top-down, transposed) into a code buffer -- the codes do not depend on
//     the values, so all of the loads are in flight together;
//   phase B: the stages in order (coarse to fine, dimension 0..2), each
//     target predicted from the values of earlier stages (pred4: Eq. 1 /
//     Eq. 2 with the boundary rule, the compressor's operation order), plus its code's
//     value times 2e_q, or the outlier's exact value;
//   the level-Lc lattice is then written densely: the known points of level
//   Lc - 1, or the caller's array when Lc = 1.
// Values live in a dense array of the level-Lc lattice; a level-l point is
// the level-Lc point at 2^(l - Lc) times its coordinates.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ipc_device.cuh"
#include "ipc_internal.h"

namespace ipc {
namespace {
using namespace dev;

constexpr int kCoarseThreads = 512;

// The exact value of an outlier code (sorted code indices of the stage).
template <class T>
__device__ __forceinline__ void outlier_value(const CoarseStage& S, const uint64_t* __restrict__ idx,
                                              const double* __restrict__ val, uint64_t ci, T* v) {
  uint64_t lo = S.out_begin, hi = S.out_end;
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    if (__ldg(idx + mid) < ci) lo = mid + 1;
    else hi = mid;
  }
  if (lo < S.out_end && __ldg(idx + lo) == ci) *v = (T)__ldg(val + lo);
}

// pred4 on the dense level-Lc lattice: idx the target, st the lattice
// stride of one level-l step along the sweep; a far neighbour is read only
// where it lies on the lattice and the form uses it.
template <class T>
__device__ __forceinline__ T coarse_pred(const T* v, int64_t idx, int64_t st, int i, int M,
                                         int interp) {
  const T b = v[idx - st];
  if (i + 1 > M - 1) return b;
  const T c = v[idx + st];
  const bool left = i - 3 >= 0, right = i + 3 <= M - 1;
  // far neighbours: both for Eq. 2, the one that exists for the quadratic
  const bool far = interp == 2 || (interp != 0 && left && right);
  const T a = far && left ? v[idx - 3 * st] : b;
  const T d = far && right ? v[idx + 3 * st] : b;
  return pred4<T>(a, b, c, d, i, M, interp);
}

template <class T>
__device__ void coarse_body(const CoarseArgs& a, unsigned char* smem) {
  T* val = reinterpret_cast<T*>(smem);
  const int64_t nval = a.ML[0] * a.ML[1] * a.ML[2];
  uint32_t* code = reinterpret_cast<uint32_t*>(smem + ((nval * sizeof(T) + 15) & ~(int64_t)15));
  const int tid = threadIdx.x;

  // Phase A: decode every word of every stage, the words of all stages in
  // one index space (a thread takes about one word in all).
  uint32_t total = 0;
  for (int t = 0; t < a.nst; ++t) total += (uint32_t)a.st[t].words;
  for (uint32_t u = tid; u < total; u += blockDim.x) {
    int t = 0;
    uint32_t w = u;
    while (w >= (uint32_t)a.st[t].words) {
      w -= (uint32_t)a.st[t].words;
      ++t;
    }
    const CoarseStage& S = a.st[t];
    // (the coarse stages are small: their indices fit 32 bits)
    const uint32_t wr = (uint32_t)S.wr, m1 = (uint32_t)S.m[1];
    {
      const uint32_t r = w / wr, j = w - r * wr;
      const uint32_t pi = r / m1, rr = r - pi * m1;
      const uint32_t rb = rr / S.RB, ct = j / S.CW;
      const uint64_t g = ((uint64_t)pi * S.nrb + rb) * S.nct + ct;
      const uint32_t li = (rr - rb * S.RB) * S.CW + (j - ct * S.CW);
      const uint32_t wl = li >> 5, bit = 1u << (li & 31), below = bit - 1u;
      const uint32_t* bmp = a.bm + S.bm0 + g * S.bw + wl;
      const uint32_t* cp = a.cap + S.cap0 + g * (uint64_t)S.RB * S.CW + wl * 32u;
      // all the bitmap words first, then all the plane words: 32 loads in
      // flight at a time instead of a chain of 32 dependent pairs
      uint32_t p[32];
#pragma unroll
      for (int k = 0; k < 32; ++k)
        p[k] = ((S.kmask >> k) & 1u) ? __ldg(bmp + (uint64_t)k * S.pbm) : 0u;
      uint32_t any = 0u;
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        const uint32_t m = p[k];
        p[k] = (m & bit) ? __ldg(cp + (uint64_t)k * S.pcap + __popc(m & below)) : 0u;
        any |= p[k];
      }
      uint32_t* dst = code + S.code_off + (uint64_t)r * S.m[2] + 32 * j;
      const int nc = (int)min((int64_t)32, S.m[2] - 32 * (int64_t)j);
      if (any == 0u) {
        for (int i = 0; i < nc; ++i) dst[i] = 0u;
        continue;  // the next word
      }
#pragma unroll
      for (int k = 31; k >= 0; --k) {
        const uint32_t p1 = k + 1 < 32 ? p[k + 1] : 0u, p2 = k + 2 < 32 ? p[k + 2] : 0u;
        p[k] = k >= S.b ? (p[k] ^ p1 ^ p2) : 0u;
      }
      transpose32(p);
#pragma unroll
      for (int i = 0; i < 32; ++i)
        if (i < nc) dst[i] = p[i];
    }
  }
  if (tid == 0) val[0] = (T)a.anchor;
  __syncthreads();

  // Phase B: the stages in order.
  const int64_t s2 = 1, s1 = a.ML[2], s0 = a.ML[1] * a.ML[2];
  const T twoeb = (T)a.twoeb;
  for (int t = 0; t < a.nst; ++t) {
    const CoarseStage& S = a.st[t];
    const int f = S.level - a.Lc;  // level-l coordinates scale by 2^f into the Lc lattice
    const int d = S.dim;
    const int64_t M = ((a.ML[d] - 1) >> f) + 1;  // the level's extent along d
    const int64_t sd = (d == 0 ? s0 : (d == 1 ? s1 : s2)) << f;
    const uint32_t n = (uint32_t)(S.m[0] * S.m[1] * S.m[2]);
    const uint32_t m2 = (uint32_t)S.m[2], m1 = (uint32_t)S.m[1];
    const bool has_out = S.out_end > S.out_begin;
    for (uint32_t ci = tid; ci < n; ci += blockDim.x) {
      const uint32_t c01 = ci / m2, c2 = ci - c01 * m2;
      const uint32_t c0 = c01 / m1, c1 = c01 - c0 * m1;
      // level-l lattice coordinates of the target
      const int64_t p0 = d == 0 ? 2 * (int64_t)c0 + 1 : (int64_t)c0;
      const int64_t p1 = d == 1 ? 2 * (int64_t)c1 + 1 : (d < 1 ? 2 * (int64_t)c1 : (int64_t)c1);
      const int64_t p2 = d == 2 ? 2 * (int64_t)c2 + 1 : 2 * (int64_t)c2;
      const int64_t idx = ((p0 << f) * s0) + ((p1 << f) * s1) + (p2 << f);
      const int i = (int)(d == 0 ? p0 : (d == 1 ? p1 : p2));
      const T pred = coarse_pred<T>(val, idx, sd, i, (int)M, a.interp);
      T v = FP<T>::add(pred, FP<T>::mul(code_value(code[S.code_off + ci], T()), twoeb));
      if (has_out) outlier_value<T>(S, a.oidx, a.oval, ci, &v);
      val[idx] = v;
    }
    __syncthreads();
  }

  // The level-Lc lattice, densely.
  T* out = reinterpret_cast<T*>(a.out);
  for (int64_t i = tid; i < nval; i += blockDim.x) out[i] = val[i];
}

template <class T>
__global__ void __launch_bounds__(kCoarseThreads, 1)
    k_coarse(const __grid_constant__ CoarseArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  coarse_body<T>(a, smem);
}

template <class T>
__global__ void __launch_bounds__(kCoarseThreads, 1)
    k_coarse_batch(const CoarseArgs* __restrict__ args) {
  extern __shared__ __align__(16) unsigned char smem[];
  coarse_body<T>(args[blockIdx.x], smem);
}

template <class T>
cudaError_t setup_coarse() {
  static const cudaError_t e = [] {
    cudaError_t r = cudaFuncSetAttribute(k_coarse<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kCoarseSmem);
    if (r == cudaSuccess)
      r = cudaFuncSetAttribute(k_coarse_batch<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kCoarseSmem);
    return r;
  }();
  return e;
}

}  // namespace

cudaError_t launch_coarse(int dtype, const CoarseArgs& a, cudaStream_t st) {
  const size_t smem = coarse_smem(a);
  if (smem > kCoarseSmem) return cudaErrorInvalidValue;
  cudaError_t e;
  if (dtype == 0) {
    if ((e = setup_coarse<float>()) != cudaSuccess) return e;
    k_coarse<float><<<1, kCoarseThreads, smem, st>>>(a);
  } else {
    if ((e = setup_coarse<double>()) != cudaSuccess) return e;
    k_coarse<double><<<1, kCoarseThreads, smem, st>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_coarse_batch(int dtype, const CoarseArgs* d_args, int n, size_t smem,
                                cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (smem > kCoarseSmem) return cudaErrorInvalidValue;
  cudaError_t e;
  if (dtype == 0) {
    if ((e = setup_coarse<float>()) != cudaSuccess) return e;
    k_coarse_batch<float><<<n, kCoarseThreads, smem, st>>>(d_args);
  } else {
    if ((e = setup_coarse<double>()) != cudaSuccess) return e;
    k_coarse_batch<double><<<n, kCoarseThreads, smem, st>>>(d_args);
  }
  return cudaGetLastError();
}

}  // namespace ipc
