// The level kernels with the quadratic boundary forms compiled in (Q =
// true): fields compressed with cubic interpolation and quadratic
// boundaries (interp 2), and batches that hold one.
#include "ipc_level_kernels.cuh"

namespace ipc {

cudaError_t launch_level_compress_quad(int dtype, const LevelArgs& L, const void* x, void* xh,
                                       int write_xh, const void* quant, const SweepOut& o,
                                       cudaStream_t st) {
  return level_compress_impl<true>(dtype, L, x, xh, write_xh, quant, o, st);
}

cudaError_t launch_level_retrieve_quad(int dtype, const LevelArgs& L, void* out, double twoeb,
                                       int b, const uint32_t* cap, const uint32_t* bm,
                                       const uint64_t* oidx, const double* oval, int w16,
                                       RetrieveShape shape, cudaStream_t st) {
  return level_retrieve_impl<true>(dtype, L, out, twoeb, b, cap, bm, oidx, oval, w16, shape, st);
}

cudaError_t launch_level_compress_batch_quad(int dtype, const CompressEntry* ents, int n,
                                             uint64_t ctas, cudaStream_t st) {
  return level_compress_batch_impl<true>(dtype, ents, n, ctas, st);
}

cudaError_t launch_level_retrieve_batch_quad(int dtype, const RetrieveEntry* ents, int n,
                                             uint64_t tiles, int w16, int ns, int per_sm,
                                             cudaStream_t st) {
  return level_retrieve_batch_impl<true>(dtype, ents, n, tiles, w16, ns, per_sm, st);
}

}  // namespace ipc
