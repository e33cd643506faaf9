// Allocation-free variant of the range reduction (min, max, max|x| and the
// finite count of device arrays), for callers that may not allocate device
// memory: a process whose device memory is all handed out by another pool or
// allocator, or a loop that must keep a fixed memory footprint.
//
// The reduction's accumulators live in one fixed device array of this file
// (kMaxFields sets of 4 words, 32 KiB). Every GPU that loads the library
// holds it until the process exits. Host code cannot use the array's name as
// a device address, so every call looks the address up (with the calling
// thread's current device, before any work is queued) and passes it to the
// kernels; a looked-up address therefore never outlives a context reset.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>
#include <mutex>

#include "ipc.h"
#include "ipc_internal.h"

namespace {

constexpr int kMaxFields = IPC_NOALLOC_MAX_FIELDS;
constexpr int kMaxDevices = 64;

// Scratch of the reduction: per field [ordered key of min, ordered key of
// max, bits of max|x|, finite count].
static __device__ __align__(256) unsigned long long g_range_scratch[4 * kMaxFields];

std::mutex g_mu;  // one call at a time in this process (they share the array)

__device__ __forceinline__ unsigned long long okey(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ULL);
}

double okey_to_double(unsigned long long k) {
  const unsigned long long b = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFULL) : ~k;
  double v;
  std::memcpy(&v, &b, 8);
  return v;
}

__global__ void k_range_init(unsigned long long* acc, int nfields) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nfields) {
    acc[4 * i + 0] = ~0ULL;
    acc[4 * i + 1] = 0ULL;
    acc[4 * i + 2] = 0ULL;
    acc[4 * i + 3] = 0ULL;
  }
}

// Grid-stride reduction of one array into acc[0..3] (one atomic per warp).
template <class T>
__global__ void __launch_bounds__(256) k_range_noalloc(const T* __restrict__ x, uint64_t n,
                                                       unsigned long long* acc) {
  T mn = 0, mx = 0, ma = 0;
  unsigned long long cnt = 0;
  const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = tid; i < n; i += nth) {
    const T v = __ldg(x + i);
    if (!isfinite(v)) continue;
    const T a = fabs(v);  // +0 for -0: the bits of max|x| are compared as integers
    mn = cnt ? (v < mn ? v : mn) : v;
    mx = cnt ? (v > mx ? v : mx) : v;
    ma = cnt ? (a > ma ? a : ma) : a;
    ++cnt;
  }
  unsigned long long kmn = cnt ? okey((double)mn) : ~0ULL;
  unsigned long long kmx = cnt ? okey((double)mx) : 0ULL;
  unsigned long long kma = cnt ? (unsigned long long)__double_as_longlong((double)ma) : 0ULL;
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

}  // namespace

extern "C" int ipc_range_noalloc(int nfields, const void* const* d_in, const uint64_t* n,
                                 int dtype, void* stream, double* out) {
  using ipc::set_last_error;
  if (nfields < 0 || (nfields > 0 && (!d_in || !n || !out))) {
    set_last_error("ipc_range_noalloc: null argument or negative count");
    return IPC_EINVAL;
  }
  if (nfields > kMaxFields) {  // beyond the fixed scratch
    set_last_error("ipc_range_noalloc: more arrays than IPC_NOALLOC_MAX_FIELDS");
    return IPC_EINVAL;
  }
  if (dtype != IPC_F32 && dtype != IPC_F64) {
    set_last_error("ipc_range_noalloc: dtype must be IPC_F32 or IPC_F64");
    return IPC_EINVAL;
  }
  if (nfields == 0) return IPC_OK;
  for (int i = 0; i < nfields; ++i)
    if (!d_in[i] && n[i]) {
      set_last_error("ipc_range_noalloc: null array with a nonzero size");
      return IPC_EINVAL;
    }
  cudaStream_t st = (cudaStream_t)stream;
  // The call ends with a host wait on `stream`, which a capturing stream
  // does not allow: refuse before anything is queued, so the caller's
  // capture stays intact.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
    cudaGetLastError();
    set_last_error("ipc_range_noalloc: cudaStreamIsCapturing failed");
    return IPC_ECUDA;
  }
  if (cap != cudaStreamCaptureStatusNone) {
    set_last_error("ipc_range_noalloc: the stream is being captured; the call waits on it");
    return IPC_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    set_last_error("ipc_range_noalloc: no current device");
    return IPC_ECUDA;
  }
  // The array's device address, with this device current (a host-side
  // lookup; it allocates nothing).
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_range_scratch) != cudaSuccess || !p) {
    cudaGetLastError();
    set_last_error("ipc_range_noalloc: cudaGetSymbolAddress failed");
    return IPC_ECUDA;
  }
  unsigned long long* acc = (unsigned long long*)p;
  // the array keeps the previous call's contents: reset the used part
  k_range_init<<<(nfields + 127) / 128, 128, 0, st>>>(acc, nfields);
  for (int i = 0; i < nfields; ++i) {
    if (n[i] == 0) continue;
    uint64_t g = (n[i] + 1023) / 1024;
    if (g > 152 * 8) g = 152 * 8;
    if (dtype == IPC_F32)
      k_range_noalloc<float><<<(unsigned)g, 256, 0, st>>>((const float*)d_in[i], n[i], acc + 4 * i);
    else
      k_range_noalloc<double><<<(unsigned)g, 256, 0, st>>>((const double*)d_in[i], n[i],
                                                            acc + 4 * i);
  }
  // the results land in the caller's array (4 words per field), decoded in place
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, acc, 32 * (size_t)nfields, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return IPC_ECUDA;
  }
  for (int i = 0; i < nfields; ++i) {
    unsigned long long w[4];
    std::memcpy(w, out + 4 * i, 32);
    const bool any = w[3] > 0;
    double ma = 0;
    std::memcpy(&ma, &w[2], 8);
    out[4 * i + 0] = any ? okey_to_double(w[0]) : 0.0;
    out[4 * i + 1] = any ? okey_to_double(w[1]) : 0.0;
    out[4 * i + 2] = any ? ma : 0.0;
    out[4 * i + 3] = (double)w[3];
  }
  return IPC_OK;
}
