// Recording and incremental forms of the level reconstruction (sm_103a).
//
// kRecord: Algorithm 1 as in the plain level kernels, and the view's state -- the
//   digits of every code at its two lowest loaded planes -- is written.
// kDelta: Algorithm 2 (Sec. 4.3). Only the planes [b, bo) of each stage are
//   read; each new digit is decoded from its encoded bit and the two more
//   significant digits (Sec. 4.4.1), the top two from the state. The
//   increment is interpolated from zero level by level (the coarser
//   level's increments are the known points) and added to the caller's
//   array at level 1.
// Single-field launches only. The kernels are in ipc_level_body.cuh; this
// unit instantiates them for interp 0 and 1 and ipc_level_delta_quad.cu for
// interp 2, each compiled in parallel with the plain kernels.
#include "ipc_level_body.cuh"

namespace ipc {

cudaError_t launch_level_retrieve_mode(int dtype, const LevelArgs& L, void* out, double twoeb,
                                       int b, const uint32_t* cap, const uint32_t* bm,
                                       const uint64_t* oidx, const double* oval, int w16,
                                       RetrieveShape shape, int mode, cudaStream_t st) {
  if (L.interp == 2)
    return launch_level_retrieve_mode_quad(dtype, L, out, twoeb, b, cap, bm, oidx, oval, w16,
                                           shape, mode, st);
  return level_retrieve_mode_impl<false>(dtype, L, out, twoeb, b, cap, bm, oidx, oval, w16,
                                         shape, mode, st);
}

}  // namespace ipc
