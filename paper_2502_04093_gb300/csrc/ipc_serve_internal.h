// Library-internal hooks the serving loop uses (defined in ipc_host.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "ipc.h"

// Selection for a target (constrained to b <= *upper when upper != null).
// rparts (optional): the rounding and truncation parts of its cost.
int ipc_internal_select(ipc_field* f, ipc_target tg, const std::vector<int>* upper,
                        std::vector<int>* b, uint64_t* bytes, double* bound,
                        uint64_t* rparts = nullptr);
// A host view of field f with selection b, as a retrieval leaves it (no
// recorded state), refining in `mode`; freed with ipc_free.
ipc_view* ipc_internal_view_make(ipc_field* f, const std::vector<int>& b, uint64_t bytes,
                                 double bound, uint64_t racc, int mode);
// The selection of a host view.
void ipc_internal_view_selection(const ipc_view* v, std::vector<int>* b, uint64_t* bytes,
                                 double* bound);
// The refinement form a view of f takes for `mode` (IPC_REFINE_AUTO
// resolved by the element type).
int ipc_internal_refine_mode(const ipc_field* f, int mode);
// Element count and dtype of a field.
void ipc_internal_field_shape(const ipc_field* f, uint64_t* n, int* dtype);
// One reconstruction per field with the single-field kernels.
int ipc_internal_reconstruct_each(const std::vector<ipc_field*>& fs,
                                  const std::vector<std::vector<int>>& bs,
                                  const std::vector<void*>& outs, cudaStream_t st);
// Batched reconstruction (one launch per level per element type); the
// device tables to free once the stream has passed are appended to `tabs`.
int ipc_internal_reconstruct_batch(const std::vector<ipc_field*>& fs,
                                   const std::vector<std::vector<int>>& bs,
                                   const std::vector<void*>& outs, cudaStream_t st,
                                   std::vector<void*>* tabs);
