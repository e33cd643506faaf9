// Launchers of the small table kernels of ipc_kernels.cu that the batched
// compression uses (host side: ipc_host.cu).
#pragma once

#include <cuda_runtime.h>

#include "ipc_internal.h"

namespace ipc {

// Entry i of a compression table takes the quantizer arguments of its field:
// the 32 bytes at q + 32 * e[i].o.field (q 16-byte aligned).
cudaError_t launch_set_quant(CompressEntry* e, int n, const unsigned char* q, cudaStream_t st);

}  // namespace ipc
