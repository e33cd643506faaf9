// Recording and incremental forms of the level reconstruction (sm_103a).
//
// kRecord: Algorithm 1 as in ipc_level.cu, and the view's state -- the
//   digits of every code at its two lowest loaded planes -- is written.
// kDelta: Algorithm 2 (Sec. 4.3). Only the planes [b, bo) of each stage are
//   read; each new digit is decoded from its encoded bit and the two more
//   significant digits (Sec. 4.4.1), the top two from the state. The
//   increment is interpolated from zero level by level (the coarser
//   level's increments are the known points) and added to the caller's
//   array at level 1.
// Single-field launches only; a unit of its own so that it compiles in
// parallel with the plain kernels.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ipc_device.cuh"
#include "ipc_internal.h"
#include "ipc_level_body.cuh"

namespace ipc {
namespace {

template <class T, int BR, int BC, bool W16, int NS, int MODE>
__global__ void __launch_bounds__(256, retrieve_ctas_per_sm<T, BR, W16>()) k_level_retrieve_mode(
    LevelArgs L, T* out, T twoeb, int b, const uint32_t* __restrict__ cap,
    const uint32_t* __restrict__ bm, const uint64_t* __restrict__ oidx,
    const double* __restrict__ oval, uint64_t ntiles) {
  extern __shared__ __align__(16) unsigned char smem[];
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    level_retrieve_body<T, BR, BC, W16, NS, MODE>(L, out, twoeb, b, cap, bm, oidx, oval, t, smem);
    __syncthreads();  // the next tile reuses shared memory
  }
}

template <class T, int BR, int BC, bool W16, int NS, int MODE>
cudaError_t run_mode(const LevelArgs& L, void* out, double twoeb, int b, const uint32_t* cap,
                     const uint32_t* bm, const uint64_t* oidx, const double* oval, int per_sm,
                     cudaStream_t st) {
  static const cudaError_t setup = cudaFuncSetAttribute(
      k_level_retrieve_mode<T, BR, BC, W16, NS, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
      (int)smem_retrieve<T, BR, BC, W16, NS>());
  if (setup != cudaSuccess) return setup;
  const uint64_t tiles = retrieve_tiles(L, NS);
  if (tiles == 0) return cudaSuccess;
  k_level_retrieve_mode<T, BR, BC, W16, NS, MODE>
      <<<persistent_grid(tiles, grid_per_sm(per_sm, retrieve_ctas_per_sm<T, BR, W16>())), 256,
         smem_retrieve<T, BR, BC, W16, NS>(), st>>>(L, (T*)out, (T)twoeb, b, cap, bm, oidx, oval,
                                                    tiles);
  return cudaGetLastError();
}

// BR16 / BR32: tile rows with 16-bit code rows / with 32-bit code rows and
// several planes per tile, as for the plain kernels.
template <class T, int BR16, int BR32, int BC, int MODE>
cudaError_t dispatch_mode(const LevelArgs& L, void* out, double twoeb, int b, const uint32_t* cap,
                          const uint32_t* bm, const uint64_t* oidx, const double* oval, int w16,
                          int ns, int per_sm, cudaStream_t st) {
#define IPC_RM(R, W, N) \
  return run_mode<T, R, BC, W, N, MODE>(L, out, twoeb, b, cap, bm, oidx, oval, per_sm, st)
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

}  // namespace

cudaError_t launch_level_retrieve_mode(int dtype, const LevelArgs& L, void* out, double twoeb,
                                       int b, const uint32_t* cap, const uint32_t* bm,
                                       const uint64_t* oidx, const double* oval, int w16,
                                       RetrieveShape shape, int mode, cudaStream_t st) {
  const int ns = shape.ns ? shape.ns : retrieve_subtiles(L.M[2], w16);
  if (!retrieve_ns_ok(L.M[2], ns)) return cudaErrorInvalidValue;
  if (retrieve_tiles(L, ns) >= (1ULL << 32)) return cudaErrorInvalidValue;  // 32-bit tile ids
  if (mode != kRecord && mode != kDelta) return cudaErrorInvalidValue;
  if (dtype == 0) {
    if (mode == kRecord)
      return dispatch_mode<float, kLevelRowsF32, kLevelRowsF32 / 2, kLevelCols, kRecord>(
          L, out, twoeb, b, cap, bm, oidx, oval, w16, ns, shape.per_sm, st);
    return dispatch_mode<float, kLevelRowsF32, kLevelRowsF32 / 2, kLevelCols, kDelta>(
        L, out, twoeb, b, cap, bm, oidx, oval, w16, ns, shape.per_sm, st);
  }
  if (mode == kRecord)
    return dispatch_mode<double, kLevelRowsF64, kLevelRowsF64, kLevelCols, kRecord>(
        L, out, twoeb, b, cap, bm, oidx, oval, w16, ns, shape.per_sm, st);
  return dispatch_mode<double, kLevelRowsF64, kLevelRowsF64, kLevelCols, kDelta>(
      L, out, twoeb, b, cap, bm, oidx, oval, w16, ns, shape.per_sm, st);
}

}  // namespace ipc
