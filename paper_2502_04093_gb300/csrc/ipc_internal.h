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

// Outputs of the compression sweeps. The plane streams of a device-resident
// field are kept "segmented": per (stage, plane) a capacity array of
// ntiles * 256 words in which every 256-word segment stores its nonzero words
// compacted at the segment's own start, plus the zero-word bitmap of the
// whole plane (ntiles * 8 words). The packed container form is produced only
// by export.
struct SweepOut {
  uint32_t* cap;        // field capacity arrays
  uint32_t* bm;         // field bitmaps
  uint32_t* nnz;        // 32 counters per stage (nonzero words per plane)
  unsigned long long* outl_key;  // (stage << 40) | code index
  double* outl_val;
  unsigned long long* outl_count;
  uint64_t outl_cap;
  uint32_t* stat;       // per stage: [OR of negabinary codes, max |q|]
};

// Per-plane descriptor of a device-resident stream.
struct PlaneDesc {
  uint64_t cap_off;  // word offset of the plane's capacity array (segmented)
  uint64_t bm_off;   // word offset of the plane's bitmap
  uint64_t pk_off;   // word offset of the stream (nnz word) in a packed blob
  uint32_t nnz;
  uint32_t mode;     // 0 empty, 1 sparse, 2 dense (packed container modes)
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
                                  int write_xh, const void* quant, int stage, const SweepOut& o,
                                  const StageDescs& d, cudaStream_t st);
cudaError_t launch_retrieve_stage(int dtype, const StageArgs& a, void* out, double twoeb,
                                  const StageDescs& d, int b, const uint32_t* cap,
                                  const uint32_t* bm, cudaStream_t st);
cudaError_t launch_outlier_scatter(int dtype, const StageArgs& a, void* out,
                                   const uint64_t* idx, const double* val, uint64_t n,
                                   cudaStream_t st);
cudaError_t launch_set_anchor(int dtype, void* out, double v, cudaStream_t st);
// Exclusive prefix, per plane, of the population of each 256-word segment of
// a bitmap (bm = segmented bitmaps when packed == 0, the packed blob's sparse
// bitmaps when packed != 0); flags bitmaps whose population differs from nnz.
cudaError_t launch_seg_rank(const StageArgs& a, const StageDescs& d, int packed,
                            const uint32_t* bm, uint32_t* rank, unsigned int* bad,
                            cudaStream_t st);
// Segmented -> packed container streams (export) and back (import).
cudaError_t launch_pack(const StageArgs& a, const StageDescs& d, const uint32_t* cap,
                        const uint32_t* bm, const uint32_t* rank, uint32_t* blob,
                        cudaStream_t st);
// chk: 32 counters per stage (nonzero words of dense streams); bad: flag.
cudaError_t launch_unpack(const StageArgs& a, const StageDescs& d, const uint32_t* blob,
                          const uint32_t* rank, uint32_t* cap, uint32_t* bm, unsigned int* bad,
                          unsigned int* chk, cudaStream_t st);

}  // namespace ipc
