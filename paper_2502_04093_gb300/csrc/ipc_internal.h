// Internal declarations of libipcomp shared by its host and device units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

namespace ipc {

// Work unit of the fused level kernels: one plane of the level lattice,
// kLevelRows rows and kLevelCols lattice columns (a multiple of 64, so a
// tile's codes of one column parity fill whole 32-code words).
constexpr int kLevelRowsF32 = 16;
constexpr int kLevelRowsF64 = 8;
constexpr int kLevelCols = 512;

// One non-empty (level, dimension) sweep over the padded 3-D index space.
// Targets are the lattice start[e] + c_e * step[e], c_e < m[e]; codes are in
// row-major lattice order, a row being a line along the last dimension.
// Device storage is split into segments: the words one level-kernel CTA
// owns, RB rows x CW words of the stage's word grid (rows x wr), numbered
// (plane, row block, column tile).
struct StageGeo {
  int level;          // 1..K
  int dim3;           // sweep dimension (padded index 0..2)
  int64_t start[3], step[3], m[3];
  uint64_t ncodes, rows, wr, words;
  uint32_t RB, CW;    // segment: rows x words
  uint64_t nrb, nct;  // row blocks per stage plane, column tiles per row
  uint64_t nseg, bw;  // segments; bitmap words per segment
};

struct Geo {
  int ndim;
  int64_t N[3];  // padded extents (leading 1s)
  int K;
  uint64_t n;
  std::vector<StageGeo> stages;
  std::vector<int> level_stage[3];  // per level (index l-1) the stage of sweep d, or -1
};
bool build_geo(int ndim, const int64_t* dims, int dtype, Geo* g);

// Kernel-side view of one sweep of a level (passed by value).
struct LevelStage {
  int present;
  int t;              // stage index
  uint32_t RB, CW;
  uint64_t nrb, nct, bw;
  uint64_t m1, m2, wr;  // stage lattice: rows per plane, codes per row, words per row
  uint64_t out_begin, out_end;  // outlier range of the stage (reconstruction)
};
// Reconstruction view of a sweep's plane streams: word offsets of plane 0's
// capacity array and bitmap, the per-plane strides (plane k lies k strides
// further), and the planes to load (bit k: k >= b and the plane has nonzero
// words).
struct StagePlanes {
  uint64_t cap0, pcap, bm0, pbm;
  uint32_t kmask;
  // State of an incremental view (Algorithm 2): per word of the stage's word
  // grid, the digits of its 32 codes at the two lowest loaded planes (two
  // words, word-grid order). Written (`carry`) by recording and incremental
  // reconstructions; an incremental one reads the previous state from a
  // second buffer (`carry_in`), since a tile reads its neighbours' words for
  // its halo while their owners write theirs. Null otherwise.
  uint32_t* carry;
  const uint32_t* carry_in;
};
struct LevelArgs {
  int64_t N[3], stride[3], M[3];  // extents, element strides, lattice extents
  int64_t s;
  int interp;         // 0 linear, 1 cubic, 2 cubic with quadratic boundaries
  int vec;            // output base aligned to two elements (paired stores allowed)
  int stream_out;     // reconstruction: the output is the caller's array, written
                      // with evict-first stores (kept out of L2's way)
  uint64_t nrb, nct;  // CTA row blocks per plane, column tiles
  uint64_t mrb, mct;  // div_magic(nrb), div_magic(nct): tile -> (plane, row block, column tile)
  LevelStage st[3];
  // the known points of the level: the next coarser level's lattice stored
  // densely (plane and row strides in elements)
  const void* kin;
  int64_t kst0, kst1;
  // compression: plane and row strides of the level's own dense lattice
  // (its reconstructed values, the next finer level's known points)
  int64_t ost0, ost1;
  StagePlanes sp[3];  // plane offsets (both); the planes to load and the state (reconstruction)
  int bo;             // incremental reconstruction: planes >= bo are loaded already
#ifdef IPC_DEBUG_BOUNDS
  // Bounds-checking build: the extents (elements / words) the level's
  // accesses must stay within, and the device record of the first access
  // outside them ([0] count, [1] site, [2] index, [3] limit).
  uint64_t lim_cap, lim_bm, lim_kin, lim_out, lim_x;
  unsigned long long* bounds;
#endif
};

// The coarse levels K .. Lc of a reconstruction in one CTA (ipc_coarse.cu):
// per stage of those levels (execution order), its lattice, word grid,
// segments, the planes to load and where its codes go in shared memory.
constexpr int kCoarseMaxStages = 32;
constexpr size_t kCoarseSmem = 96 * 1024;  // shared memory the host may plan for
struct CoarseStage {
  int level, dim;          // dim: sweep dimension in the padded index space
  int b;                   // planes dropped
  uint32_t kmask;          // planes to load (k >= b with nonzero words)
  int64_t m[3];            // stage lattice extents
  uint64_t wr, words;      // words per row, words of the stage
  uint32_t RB, CW;         // segment rows x words
  uint64_t nrb, nct, bw;
  uint64_t cap0, pcap, bm0, pbm;
  uint64_t out_begin, out_end;
  uint64_t code_off;       // first code of the stage in the shared code buffer
};
struct CoarseArgs {
  int nst, K, Lc, interp;
  int esz;                 // element bytes
  int64_t ML[3];           // level-Lc lattice extents
  double anchor, twoeb;
  void* out;               // the level-Lc lattice, dense
  const uint32_t* cap;
  const uint32_t* bm;
  const uint64_t* oidx;
  const double* oval;
  CoarseStage st[kCoarseMaxStages];
};
// Shared memory of a coarse launch: the level-Lc lattice (16-byte aligned)
// and the codes of every stage.
inline size_t coarse_smem(const CoarseArgs& a) {
  const size_t v = (size_t)(a.ML[0] * a.ML[1] * a.ML[2]) * (size_t)a.esz;
  size_t c = 0;
  for (int t = 0; t < a.nst; ++t)
    c += (size_t)(a.st[t].m[0] * a.st[t].m[1] * a.st[t].m[2]) * 4;
  return ((v + 15) & ~(size_t)15) + c;
}
cudaError_t launch_coarse(int dtype, const CoarseArgs& a, cudaStream_t st);
cudaError_t launch_coarse_batch(int dtype, const CoarseArgs* d_args, int n, size_t smem,
                                cudaStream_t st);

// Division of a 32-bit n by a divisor 1 <= d < 2^32 as the high half of n * m,
// m = ceil(2^64 / d) (0 for d = 1): n m / 2^64 exceeds n / d by less than
// 2^-32 < 1/d, which never carries it past the next integer.
inline uint64_t div_magic(uint64_t d) { return d <= 1 ? 0 : UINT64_MAX / d + 1; }

// Kernel-side view of a stage's word grid and segments (pack / unpack).
struct StageArgs {
  uint64_t W, wr, m1;   // words, words per row, rows per stage plane
  uint32_t RB, CW;
  uint64_t nrb, nct, bw, nbm;  // nbm = packed bitmap words = ceil(W / 32)
};
StageArgs stage_args(const StageGeo& sg);

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
  uint32_t field;       // batch index (tags outlier keys)
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

// One field's share of a batched level launch (device memory).
struct CompressEntry {
  LevelArgs L;  // L.sp: the planes' capacity and bitmap offsets
  SweepOut o;
  const void* x;
  void* xh;
  alignas(16) unsigned char quant[32];  // QuantArgs<T>
  int write_xh;
  uint64_t cta_begin;
};
struct RetrieveEntry {
  LevelArgs L;
  void* out;
  const uint32_t* cap;
  const uint32_t* bm;
  const uint64_t* oidx;
  const double* oval;
  double twoeb;
  int b;
  uint64_t cta_begin;
};

struct AnchorEntry {
  void* out;
  double v;
};

// ---- kernel launchers -------------------------------------------------------
cudaError_t launch_range(int dtype, const void* x, uint64_t n, unsigned long long* acc,
                         cudaStream_t st);
// The range of up to kRangeBatch arrays in one launch (arguments by value):
// acc[4 j ..] as launch_range, x0[j] = the f64 bits of array j's first value.
constexpr int kRangeBatch = 128;
struct RangeBatch {
  const void* x[kRangeBatch];
  uint64_t n[kRangeBatch];
  unsigned long long* acc;
  unsigned long long* x0;
};
cudaError_t launch_range_batch(int dtype, const RangeBatch& rb, int n, uint64_t nmax,
                               cudaStream_t st);
cudaError_t launch_set_anchor(int dtype, void* out, double v, cudaStream_t st);
cudaError_t launch_set_anchors(int dtype, const AnchorEntry* a, int n, cudaStream_t st);
// Fused level kernels (ipc_level.cu; the variants with the quadratic
// boundary forms, for interp 2, in ipc_level_quad.cu and
// ipc_level_delta_quad.cu -- the single-field launchers pick them by
// L.interp, the batched ones by `quad`: some entry has interp 2).
cudaError_t launch_level_compress(int dtype, const LevelArgs& L, const void* x, void* xh,
                                  int write_xh, const void* quant, const SweepOut& o,
                                  cudaStream_t st);
// Retrieve tiles of a level: levels whose lattice rows hold at most
// kLevelCols/2 (kLevelCols/4) columns put 2 (4) planes of the same parity
// side by side in one tile.
// Tiles enumerate (plane group, row block, column tile), the groups
// alternating even and odd planes.
inline int retrieve_subtiles(int64_t M2, int) {
  return M2 <= kLevelCols / 4 ? 4 : (M2 <= kLevelCols / 2 ? 2 : 1);
}
inline uint64_t retrieve_tiles(const LevelArgs& L, int ns) {
  const int64_t ne = (L.M[0] + 1) / 2, no = L.M[0] / 2;
  const uint64_t groups = (uint64_t)((ne + ns - 1) / ns + (no + ns - 1) / ns);
  return groups * L.nrb * L.nct;
}
// Launch shape of a level reconstruction (results do not depend on it):
// planes per tile (1, 2 or 4; 0 = the most the level's rows allow) and CTAs
// per SM of the persistent grid (0 = as many as fit).
struct RetrieveShape {
  int ns = 0;
  int per_sm = 0;
};
inline bool retrieve_ns_ok(int64_t M2, int ns) {
  return ns == 1 || (ns == 2 && M2 <= kLevelCols / 2) || (ns == 4 && M2 <= kLevelCols / 4);
}
// Rows of a reconstruction tile: the compressed segment's rows, except for
// f32 tiles of several planes (ns > 1) with 32-bit code rows, which take half
// a segment (8 rows) so that four CTAs fit per SM. (One-plane tiles keep 16
// rows: with 8, the halo rows' share of the work costs more than the fourth
// CTA gains.)
inline int retrieve_rows(int dtype, int w16, int ns) {
  return dtype == 0 ? (w16 || ns == 1 ? kLevelRowsF32 : kLevelRowsF32 / 2) : kLevelRowsF64;
}
// Most CTAs of a level reconstruction resident per SM.
inline int retrieve_max_per_sm(int dtype, int w16, int ns) {
  return w16 || (dtype == 0 && ns > 1) ? 4 : 3;
}
// w16: the planes loaded at the level span at most 16 (16-bit code rows).
// The recording (mode 1) and incremental (mode 2) forms of the level
// reconstruction (single field); mode 2 reads only the planes [b, L.bo).
cudaError_t launch_level_retrieve_mode(int dtype, const LevelArgs& L, void* out, double twoeb,
                                       int b, const uint32_t* cap, const uint32_t* bm,
                                       const uint64_t* oidx, const double* oval, int w16,
                                       RetrieveShape shape, int mode, cudaStream_t st);
cudaError_t launch_level_retrieve(int dtype, const LevelArgs& L, void* out, double twoeb, int b,
                                  const uint32_t* cap, const uint32_t* bm, const uint64_t* oidx,
                                  const double* oval, int w16, RetrieveShape shape,
                                  cudaStream_t st);
int level_rows(int dtype);
// Batched level launches: `ents` (device memory) sorted by cta_begin.
cudaError_t launch_level_compress_batch(int dtype, const CompressEntry* ents, int n,
                                        uint64_t ctas, int quad, cudaStream_t st);
// Batched: `tiles` over all entries, each entry's tiles counted with `ns`.
cudaError_t launch_level_retrieve_batch(int dtype, const RetrieveEntry* ents, int n,
                                        uint64_t tiles, int w16, int ns, int per_sm, int quad,
                                        cudaStream_t st);
cudaError_t launch_level_compress_quad(int dtype, const LevelArgs& L, const void* x, void* xh,
                                       int write_xh, const void* quant, const SweepOut& o,
                                       cudaStream_t st);
cudaError_t launch_level_retrieve_quad(int dtype, const LevelArgs& L, void* out, double twoeb,
                                       int b, const uint32_t* cap, const uint32_t* bm,
                                       const uint64_t* oidx, const double* oval, int w16,
                                       RetrieveShape shape, cudaStream_t st);
cudaError_t launch_level_compress_batch_quad(int dtype, const CompressEntry* ents, int n,
                                             uint64_t ctas, cudaStream_t st);
cudaError_t launch_level_retrieve_batch_quad(int dtype, const RetrieveEntry* ents, int n,
                                             uint64_t tiles, int w16, int ns, int per_sm,
                                             cudaStream_t st);
cudaError_t launch_level_retrieve_mode_quad(int dtype, const LevelArgs& L, void* out,
                                            double twoeb, int b, const uint32_t* cap,
                                            const uint32_t* bm, const uint64_t* oidx,
                                            const double* oval, int w16, RetrieveShape shape,
                                            int mode, cudaStream_t st);
// Segmented <-> packed container streams of one stage (export / import).
// tmp: 2 * 32 * nbm words of scratch; flags[0] = corruption flag,
// flags[1 + k] = nonzero words found in plane k (import).
cudaError_t launch_pack(const StageArgs& a, const StageDescs& d, const uint32_t* cap,
                        const uint32_t* bm, uint32_t* tmp, uint32_t* blob, cudaStream_t st);
// kmask: the planes this upload writes (the others keep their words).
cudaError_t launch_unpack(const StageArgs& a, const StageDescs& d, uint64_t nseg,
                          const uint32_t* blob, uint32_t* tmp, uint32_t* cap, uint32_t* bm,
                          unsigned int* flags, uint32_t kmask, cudaStream_t st);

// Sets the message ipc_last_error() returns on the calling thread.
void set_last_error(const char* what);

}  // namespace ipc
