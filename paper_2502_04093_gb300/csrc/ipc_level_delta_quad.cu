// The recording and incremental level reconstructions with the quadratic
// boundary forms compiled in (interp 2); see ipc_level_delta.cu.
#include "ipc_level_body.cuh"

namespace ipc {

cudaError_t launch_level_retrieve_mode_quad(int dtype, const LevelArgs& L, void* out,
                                            double twoeb, int b, const uint32_t* cap,
                                            const uint32_t* bm, const uint64_t* oidx,
                                            const double* oval, int w16, RetrieveShape shape,
                                            int mode, cudaStream_t st) {
  return level_retrieve_mode_impl<true>(dtype, L, out, twoeb, b, cap, bm, oidx, oval, w16, shape,
                                        mode, st);
}

}  // namespace ipc
