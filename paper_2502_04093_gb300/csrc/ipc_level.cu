// The level kernels for linear and cubic interpolation (interp 0, 1); a
// level of a field with quadratic boundaries (interp 2) goes to the
// variant in ipc_level_quad.cu.
#include "ipc_level_kernels.cuh"

namespace ipc {

int level_rows(int dtype) { return dtype == 0 ? kLevelRowsF32 : kLevelRowsF64; }

cudaError_t launch_level_compress(int dtype, const LevelArgs& L, const void* x, void* xh,
                                  int write_xh, const void* quant, const SweepOut& o,
                                  cudaStream_t st) {
  if (L.interp == 2) return launch_level_compress_quad(dtype, L, x, xh, write_xh, quant, o, st);
  return level_compress_impl<false>(dtype, L, x, xh, write_xh, quant, o, st);
}

cudaError_t launch_level_retrieve(int dtype, const LevelArgs& L, void* out, double twoeb, int b,
                                  const uint32_t* cap, const uint32_t* bm, const uint64_t* oidx,
                                  const double* oval, int w16, RetrieveShape shape,
                                  cudaStream_t st) {
  if (L.interp == 2)
    return launch_level_retrieve_quad(dtype, L, out, twoeb, b, cap, bm, oidx, oval, w16, shape, st);
  return level_retrieve_impl<false>(dtype, L, out, twoeb, b, cap, bm, oidx, oval, w16, shape, st);
}

cudaError_t launch_level_compress_batch(int dtype, const CompressEntry* ents, int n,
                                        uint64_t ctas, int quad, cudaStream_t st) {
  if (quad) return launch_level_compress_batch_quad(dtype, ents, n, ctas, st);
  return level_compress_batch_impl<false>(dtype, ents, n, ctas, st);
}

cudaError_t launch_level_retrieve_batch(int dtype, const RetrieveEntry* ents, int n,
                                        uint64_t tiles, int w16, int ns, int per_sm, int quad,
                                        cudaStream_t st) {
  if (quad) return launch_level_retrieve_batch_quad(dtype, ents, n, tiles, w16, ns, per_sm, st);
  return level_retrieve_batch_impl<false>(dtype, ents, n, tiles, w16, ns, per_sm, st);
}

}  // namespace ipc
