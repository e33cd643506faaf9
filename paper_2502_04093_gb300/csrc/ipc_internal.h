// Internal declarations of libipcomp shared by its host and device units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

namespace ipc {

// Words of a compaction tile: one CTA of the sweep kernels owns 256
// consecutive plane words (8 warps x 32 words, 8192 codes) of a stage.
constexpr int kTileWords = 256;
constexpr int kTileBitmapWords = kTileWords / 32;

// One non-empty (level, dimension) sweep over the padded 3-D index space.
// Targets are the lattice start[e] + c_e * step[e], c_e < m[e]; codes are in
// row-major lattice order, a row being a line along the last dimension.
struct StageGeo {
  int level;          // 1..K
  int dim3;           // sweep dimension (padded index 0..2)
  int64_t start[3], step[3], m[3];
  uint64_t ncodes, rows, wr, words, ntiles;
};

struct Geo {
  int ndim;
  int64_t N[3];  // padded extents (leading 1s)
  int K;
  uint64_t n;
  std::vector<StageGeo> stages;
};
bool build_geo(int ndim, const int64_t* dims, Geo* g);

// Kernel-side view of a stage (passed by value).
struct StageArgs {
  int64_t N[3];
  int64_t stride[3];
  int64_t start[3], step[3], m[3];
  int64_t s;       // level stride 2^(l-1)
  uint64_t W, wr, ntiles;
  int d;           // sweep dimension
  int cubic;
};
StageArgs stage_args(const Geo& g, const StageGeo& sg, int cubic);

template <class T>
struct QuantArgs {
  T inv2eb, twoeb, ebchk, R;
};

// Scratch of one compression (library workspace).
struct CompressScratch {
  uint32_t* cap;        // per plane: ntiles*256 candidate words (compacted per tile)
  uint32_t* bitmap;     // per plane: ntiles*8 words
  uint32_t* tilecnt;    // per plane: ntiles counts
  unsigned long long* outl_key;  // (stage << 40) | code index
  double* outl_val;
  unsigned long long* outl_count;
  uint64_t outl_cap;
  uint32_t* stat;       // per stage: [OR of negabinary codes, max |q|]
};

// Retrieval descriptor of one plane stream.
struct PlaneDesc {
  uint64_t off;      // word offset of the stream's nnz word in the field blob
  uint64_t rank_off; // offset of the stream's tile-rank index
  uint32_t nnz;
  uint32_t mode;     // 0 empty, 1 sparse (bitmap + payload), 2 dense
};
struct StageDescs {
  PlaneDesc p[32];
};

// Stream mode and byte size from (nnz, W) (format definition).
inline uint32_t stream_mode(uint64_t nnz, uint64_t W) {
  if (nnz == 0) return 0;
  uint64_t nbm = (W + 31) / 32;
  return (nbm + nnz < W) ? 1u : 2u;
}
inline uint64_t stream_bytes(uint64_t nnz, uint64_t W) {
  uint32_t m = stream_mode(nnz, W);
  if (m == 0) return 4;
  if (m == 1) return 4 + 4 * ((W + 31) / 32 + nnz);
  return 4 + 4 * W;
}

// ---- kernel launchers (ipc_kernels.cu) ------------------------------------
cudaError_t launch_range(int dtype, const void* x, uint64_t n, unsigned long long* acc,
                         cudaStream_t st);
cudaError_t launch_compress_stage(int dtype, const StageArgs& a, const void* x, void* xh,
                                  int write_xh, const void* quant, int stage,
                                  const CompressScratch& sc, uint64_t cap_off,
                                  uint64_t bm_off, uint64_t cnt_off, cudaStream_t st);
cudaError_t launch_scan_stage(const StageArgs& a, const CompressScratch& sc, uint64_t cnt_off,
                              uint32_t* rank_out, uint32_t* nnz_out, cudaStream_t st);
cudaError_t launch_pack_stage(const StageArgs& a, const CompressScratch& sc, uint64_t cap_off,
                              uint64_t bm_off, uint64_t cnt_off, const uint32_t* rank,
                              const StageDescs& d, uint32_t* blob, cudaStream_t st);
cudaError_t launch_retrieve_stage(int dtype, const StageArgs& a, void* out, double twoeb,
                                  const StageDescs& d, int b, const uint32_t* blob,
                                  const uint32_t* rank, cudaStream_t st);
cudaError_t launch_outlier_scatter(int dtype, const StageArgs& a, void* out,
                                   const uint64_t* idx, const double* val, uint64_t n,
                                   cudaStream_t st);
cudaError_t launch_set_anchor(int dtype, void* out, double v, cudaStream_t st);
cudaError_t launch_build_rank(const StageArgs& a, const StageDescs& d, const uint32_t* blob,
                              uint32_t* rank, unsigned int* bad, cudaStream_t st);

}  // namespace ipc
