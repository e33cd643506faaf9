// Host side of libipcomp: the C ABI of include/ipc.h, the container format,
// the optimized loader (Sec. 5) and the launch sequences of compression and
// reconstruction. Every step of the data path runs in the kernels of
// ipc_kernels.cu; this file only plans, allocates and orders them.
#include <cuda_runtime.h>
#include <stdint.h>

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <unistd.h>

#include <array>
#include <atomic>
#include <cfloat>
#include <cmath>
#include <condition_variable>
#include <functional>
#include <cstdio>
#include <cstring>
#include <exception>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "ipc.h"
#include "ipc_internal.h"
#include "ipc_select.h"
#include "ipc_serve_internal.h"
#include "ipc_table_kernels.h"

using namespace ipc;

namespace {

thread_local std::string g_err;

int fail(int code, const char* what) {
  g_err = what;
  return code;
}
int cuda_fail(cudaError_t e, const char* where) {
  g_err = std::string(where) + ": " + cudaGetErrorString(e);
  return IPC_ECUDA;
}
#define CU(call)                                         \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
  } while (0)

// ---------------------------------------------------------------------------
// Kernel profiler: CUDA events recorded on the launching stream around every
// kernel launch (when enabled), accumulated per kernel kind together with the
// algorithmic bytes of each launch. The launch counter always runs.
// ---------------------------------------------------------------------------
struct ProfRec {
  int kind;
  cudaEvent_t a, b;
  double bytes;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof_pending;
std::vector<cudaEvent_t> g_prof_pool;
struct ProfAcc {
  uint64_t launches;
  double ms, bytes;
} g_prof_acc[IPC_KERNEL_KINDS];
std::atomic<unsigned long long> g_launches{0};

cudaEvent_t prof_event() {
  if (!g_prof_pool.empty()) {
    cudaEvent_t e = g_prof_pool.back();
    g_prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}
// Returns a handle for prof_end (or -1 when the profiler is off).
// NVTX ranges (host timeline) around the library's calls and level launches,
// while enabled (ipc_nvtx_enable): a profiler can then select the kernels of
// one level (`ncu --nvtx --nvtx-include "ipc retrieve/level 1/"`). The header-only
// NVTX costs a relaxed load per range when no tool is attached.
std::atomic<bool> g_nvtx{false};
struct Nvtx {
  bool on;
  explicit Nvtx(const char* name) : on(g_nvtx.load(std::memory_order_relaxed)) {
    if (on) nvtxRangePushA(name);
  }
  Nvtx(const char* fmt, int a) : on(g_nvtx.load(std::memory_order_relaxed)) {
    if (on) {
      char b[48];
      std::snprintf(b, sizeof b, fmt, a);
      nvtxRangePushA(b);
    }
  }
  ~Nvtx() {
    if (on) nvtxRangePop();
  }
  Nvtx(const Nvtx&) = delete;
  Nvtx& operator=(const Nvtx&) = delete;
};

long prof_begin(int kind, cudaStream_t st) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (!g_prof_on) return -1;
  ProfRec r{kind, prof_event(), prof_event(), 0.0};
  if (!r.a || !r.b) return -1;
  cudaEventRecord(r.a, st);
  g_prof_pending.push_back(r);
  return (long)g_prof_pending.size() - 1;
}
void prof_end(long h, cudaStream_t st, double bytes) {
  if (h < 0) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if ((size_t)h >= g_prof_pending.size()) return;
  g_prof_pending[h].bytes = bytes;
  cudaEventRecord(g_prof_pending[h].b, st);
}
void prof_set_bytes(long h, double bytes) {
  if (h < 0) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if ((size_t)h < g_prof_pending.size()) g_prof_pending[h].bytes = bytes;
}
void prof_drain() {  // caller holds g_prof_mu
  for (ProfRec& r : g_prof_pending) {
    float ms = 0;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      ProfAcc& a = g_prof_acc[r.kind];
      a.launches += 1;
      a.ms += ms;
      a.bytes += r.bytes;
    }
    cudaGetLastError();
    g_prof_pool.push_back(r.a);
    g_prof_pool.push_back(r.b);
  }
  g_prof_pending.clear();
}

const uint32_t kMagic = 0x31435049u;  // "IPC1"
const uint32_t kVersion = 1u;
const uint32_t kFieldTag = 0x46435049u, kViewTag = 0x56435049u, kPlanTag = 0x50435049u;
const uint32_t kDeadTag = 0xDEADDEADu;

}  // namespace

// ---------------------------------------------------------------------------
// Geometry (Sec. 4.1): dims padded to 3-D; level l = K..1 has stride
// s = 2^(l-1); sweep d over the points whose coordinate d is an odd multiple
// of s, coordinates before d multiples of s, after d multiples of 2s.
// ---------------------------------------------------------------------------
namespace ipc {
bool build_geo(int ndim, const int64_t* dims, int dtype, Geo* g) {
  if (ndim < 1 || ndim > 3 || !dims) return false;
  g->ndim = ndim;
  g->N[0] = g->N[1] = g->N[2] = 1;
  uint64_t n = 1;
  for (int e = 0; e < ndim; ++e) {
    if (dims[e] < 1 || dims[e] > (int64_t(1) << 31) - 1) return false;
    g->N[3 - ndim + e] = dims[e];
    n *= (uint64_t)dims[e];
    if (n > (uint64_t(1) << 42)) return false;
  }
  g->n = n;
  const int64_t mx = std::max(g->N[0], std::max(g->N[1], g->N[2]));
  int K = 0;
  while ((int64_t(1) << K) < mx) ++K;
  g->K = K;
  g->stages.clear();
  for (int d = 0; d < 3; ++d) g->level_stage[d].assign(K, -1);
  const uint32_t BR = (uint32_t)level_rows(dtype), CWD = (uint32_t)(kLevelCols / 64);
  for (int l = K; l >= 1; --l) {
    const int64_t s = int64_t(1) << (l - 1);
    for (int d = 0; d < 3; ++d) {
      StageGeo sg{};
      sg.level = l;
      sg.dim3 = d;
      bool empty = false;
      for (int e = 0; e < 3; ++e) {
        sg.start[e] = e == d ? s : 0;
        sg.step[e] = e < d ? s : 2 * s;
        sg.m[e] = g->N[e] > sg.start[e] ? 1 + (g->N[e] - 1 - sg.start[e]) / sg.step[e] : 0;
        empty = empty || sg.m[e] == 0;
      }
      if (empty) continue;
      sg.rows = (uint64_t)sg.m[0] * (uint64_t)sg.m[1];
      sg.ncodes = sg.rows * (uint64_t)sg.m[2];
      sg.wr = ((uint64_t)sg.m[2] + 31) / 32;
      sg.words = sg.rows * sg.wr;
      // segments = the words of one level-kernel CTA (see ipc_level_kernels.cuh)
      sg.RB = d == 2 ? BR : BR / 2;
      sg.CW = (uint32_t)std::min<uint64_t>(CWD, sg.wr);
      sg.nrb = ((uint64_t)sg.m[1] + sg.RB - 1) / sg.RB;
      sg.nct = (sg.wr + sg.CW - 1) / sg.CW;
      sg.nseg = (uint64_t)sg.m[0] * sg.nrb * sg.nct;
      sg.bw = ((uint64_t)sg.RB * sg.CW + 31) / 32;
      g->level_stage[d][l - 1] = (int)g->stages.size();
      g->stages.push_back(sg);
    }
  }
  return true;
}

StageArgs stage_args(const StageGeo& sg) {
  StageArgs a{};
  a.W = sg.words;
  a.wr = sg.wr;
  a.m1 = (uint64_t)sg.m[1];
  a.RB = sg.RB;
  a.CW = sg.CW;
  a.nrb = sg.nrb;
  a.nct = sg.nct;
  a.bw = sg.bw;
  a.nbm = (sg.words + 31) / 32;
  return a;
}
}  // namespace ipc

// ---------------------------------------------------------------------------
// Objects
// ---------------------------------------------------------------------------
struct StageTab {
  int32_t H;
  uint32_t Q;
  std::vector<uint64_t> out_idx;
  std::vector<double> out_val;
  uint64_t nnz[32], size[32];  // by plane
};

// One device allocation shared by several fields' plane streams.
struct SharedStreams {
  void* p;
  std::atomic<int> refs;
};

struct ipc_field {
  uint32_t tag;
  int device;
  int dtype, interp, bound, eb_mode;
  double eb_user, eb, xmin, xmax, xmaxabs, anchor;
  Geo g;
  std::vector<StageTab> st;
  uint64_t mandatory;     // header + tables + outliers
  uint64_t stream_bytes;  // packed streams of the container
  // device: segmented plane streams, outliers
  uint32_t* d_cap;
  uint32_t* d_bm;
  // the fields of a large compressed batch hold their streams in one
  // allocation, freed with the last of them (null: d_cap is its own)
  struct SharedStreams* shared = nullptr;
  uint64_t cap_words, bm_words;
  uint64_t* d_oidx;       // outliers: code indices, per stage contiguous
  double* d_oval;
  std::vector<StageDescs> desc;   // per stage
  std::vector<uint64_t> out_off;  // per stage offset into d_oidx/d_oval
  SelInput sel;                   // the selector's input, prepared once
  // Planes held on the device: per level, planes k >= rb[l-1] (a field
  // imported from part of a container); empty: every plane.
  std::vector<int> rb;
};

struct ipc_view {
  uint32_t tag;
  ipc_field* f;
  std::vector<int> b;
  uint64_t bytes;
  double bound;
  // Refinement form (IPC_REFINE_*). An incremental view keeps, per code word
  // of every stage, the digits of its 32 codes at the two lowest loaded
  // planes (`d_state`, two words per word, stage by stage), and the rounding
  // allowance of its current reconstruction (units of eb * 2^-16).
  int mode = IPC_REFINE_CANONICAL;
  int state_device = 0;           // the device of d_state
  uint32_t* d_state = nullptr;    // two buffers of state_words words each
  uint64_t state_words = 0;
  int state_cur = 0;              // the buffer that holds the current state
  std::vector<uint64_t> state_off;  // per stage, word offset into a buffer
  bool state_valid = false;
  uint64_t racc = 0;
  int last_incremental = 0;   // the last refinement added an increment
  uint64_t last_stream_bytes = 0;  // plane-stream bytes that refinement read
};

struct ipc_plan {
  uint32_t tag;
  int device;
  void* d_tab;              // entries + anchors (device)
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  uint64_t launches;        // kernels per replay
};

namespace {

// Persistent host worker threads for the per-field work of large batches
// (selection, launch-table preparation): run(n, fn) calls fn(i) for every i
// in [0, n) on the calling thread and the workers that join in, and returns
// when all calls have finished. One job at a time; the caller claims indices
// too, so a job completes even if no worker ever wakes (after a fork, say).
// An exception thrown by a call (on any thread) stops the job's remaining
// calls and is rethrown on the calling thread, as a serial loop would.
class HostPool {
 public:
  static HostPool& get() {
    static std::mutex mu;
    static HostPool* p = nullptr;
    static pid_t owner = 0;
    std::lock_guard<std::mutex> lk(mu);
    if (!p || owner != getpid()) {  // a forked child starts a pool of its own
      p = new HostPool();           // never freed: its workers outlive main
      owner = getpid();
    }
    return *p;
  }
  void run(int n, const std::function<void(int)>& fn) {
    if (in_job()) {  // a job's own calls run serially (no nested jobs)
      for (int i = 0; i < n; ++i) fn(i);
      return;
    }
    std::lock_guard<std::mutex> one(job_mu_);
    start_workers();
    std::atomic<int> next{0};
    {
      std::lock_guard<std::mutex> lk(mu_);
      fn_ = &fn;
      n_ = n;
      next_ = &next;
      ++gen_;
    }
    cv_.notify_all();
    claim(fn, n, next);
    std::exception_ptr err;
    {
      std::unique_lock<std::mutex> lk(mu_);
      done_.wait(lk, [&] { return active_ == 0; });
      fn_ = nullptr;  // a worker that wakes late finds no job
      next_ = nullptr;
      std::swap(err, err_);
    }
    if (err) std::rethrow_exception(err);
  }

 private:
  static bool& in_job() {
    thread_local bool b = false;
    return b;
  }
  void claim(const std::function<void(int)>& fn, int n, std::atomic<int>& next) {
    in_job() = true;
    try {
      for (int i; (i = next.fetch_add(1, std::memory_order_relaxed)) < n;) fn(i);
    } catch (...) {
      next.store(n);  // the others stop claiming
      std::lock_guard<std::mutex> lk(mu_);
      if (!err_) err_ = std::current_exception();
    }
    in_job() = false;
  }
  void start_workers() {
    if (started_) return;
    started_ = true;
    const unsigned hc = std::thread::hardware_concurrency();
    const int nw = (int)std::min<unsigned>(8, std::max(1u, hc / 2)) - 1;
    for (int k = 0; k < nw; ++k) {
      try {
        std::thread([this] { loop(); }).detach();
      } catch (...) {
        break;  // fewer workers: the caller takes the rest
      }
    }
  }
  void loop() {
    uint64_t seen = 0;
    std::unique_lock<std::mutex> lk(mu_);
    for (;;) {
      cv_.wait(lk, [&] { return gen_ != seen && fn_; });
      seen = gen_;
      const std::function<void(int)>* fn = fn_;
      std::atomic<int>* next = next_;
      const int n = n_;
      ++active_;
      lk.unlock();
      claim(*fn, n, *next);
      lk.lock();
      if (--active_ == 0) done_.notify_all();
    }
  }
  std::mutex job_mu_, mu_;
  std::condition_variable cv_, done_;
  const std::function<void(int)>* fn_ = nullptr;
  std::atomic<int>* next_ = nullptr;
  std::exception_ptr err_;  // the job's first exception
  int n_ = 0, active_ = 0;
  uint64_t gen_ = 0;
  bool started_ = false;
};

// ---------------------------------------------------------------------------
// Workspace: scratch of compression, one per device, grown on demand.
// ---------------------------------------------------------------------------
struct Workspace {
  std::mutex mu;
  void* xh = nullptr;
  uint64_t xh_bytes = 0;
  unsigned long long* okey = nullptr;
  double* oval = nullptr;
  uint64_t ocap = 0;
  unsigned long long* small = nullptr;  // range acc[4] per field + outlier count
  uint64_t small_words = 0;
  uint32_t* stat = nullptr;             // 2 per stage
  uint64_t stat_words = 0;
  uint32_t* nnz = nullptr;              // 32 per stage
  uint64_t nnz_words = 0;
};
Workspace g_ws[64];

template <class P>
int grow(P** p, uint64_t* have, uint64_t need, uint64_t elem) {
  if (*have >= need && *p) return IPC_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *have = 0;
  uint64_t n = std::max<uint64_t>(need, 1);
  cudaError_t e = cudaMalloc((void**)p, n * elem);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(IPC_ENOMEM, "workspace allocation failed");
  }
  *have = n;
  return IPC_OK;
}

// Little-endian serialisation helpers.
void put32(std::vector<uint8_t>& b, uint32_t v) {
  for (int i = 0; i < 4; ++i) b.push_back(uint8_t(v >> (8 * i)));
}
void put64(std::vector<uint8_t>& b, uint64_t v) {
  for (int i = 0; i < 8; ++i) b.push_back(uint8_t(v >> (8 * i)));
}
void putd(std::vector<uint8_t>& b, double v) {
  uint64_t u;
  std::memcpy(&u, &v, 8);
  put64(b, u);
}

// Header + stage table + size table + outliers (the "mandatory" bytes).
std::vector<uint8_t> header_bytes(const ipc_field* f) {
  std::vector<uint8_t> h;
  const Geo& g = f->g;
  put32(h, kMagic);
  put32(h, kVersion);
  put32(h, (uint32_t)f->dtype);
  put32(h, (uint32_t)f->interp);
  put32(h, (uint32_t)f->bound);
  put32(h, (uint32_t)g.ndim);
  for (int e = 0; e < 3; ++e) put64(h, e < g.ndim ? (uint64_t)g.N[3 - g.ndim + e] : 0);
  put32(h, (uint32_t)f->eb_mode);
  put32(h, (uint32_t)g.K);
  putd(h, f->eb_user);
  putd(h, f->eb);
  putd(h, f->xmin);
  putd(h, f->xmax);
  putd(h, f->xmaxabs);
  putd(h, f->anchor);
  put32(h, (uint32_t)g.stages.size());
  put32(h, 0);
  for (size_t t = 0; t < g.stages.size(); ++t) {
    const StageGeo& sg = g.stages[t];
    put32(h, (uint32_t)sg.level);
    put32(h, (uint32_t)(sg.dim3 - (3 - g.ndim)));
    put64(h, sg.ncodes);
    put32(h, (uint32_t)f->st[t].H);
    put32(h, f->st[t].Q);
    put64(h, f->st[t].out_idx.size());
  }
  for (size_t t = 0; t < g.stages.size(); ++t)
    for (int k = 31; k >= 0; --k) put64(h, f->st[t].size[k]);
  for (size_t t = 0; t < g.stages.size(); ++t)
    for (size_t i = 0; i < f->st[t].out_idx.size(); ++i) {
      put64(h, f->st[t].out_idx[i]);
      putd(h, f->st[t].out_val[i]);
    }
  return h;
}

SelInput sel_input(const ipc_field* f);

#ifdef IPC_DEBUG_BOUNDS
// Bounds-checking build: the device record of the first out-of-bounds
// access, one per device ([0] count, [1] site, [2] index, [3] limit).
std::mutex g_bounds_mu;
unsigned long long* g_bounds_rec[64] = {};
unsigned long long* bounds_record() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_bounds_mu);
  if (!g_bounds_rec[dev] && cudaMalloc((void**)&g_bounds_rec[dev], 32) == cudaSuccess)
    cudaMemset(g_bounds_rec[dev], 0, 32);
  return g_bounds_rec[dev];
}
#endif

uint32_t get32le(const uint8_t* p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

// Bytes of header_bytes(f) without building it: 112-byte fixed part, per
// stage a 32-byte record and 32 plane sizes, 16 bytes per outlier.
uint64_t header_size(const ipc_field* f) {
  uint64_t nout = 0;
  for (const auto& s : f->st) nout += s.out_idx.size();
  return 112 + 288 * (uint64_t)f->g.stages.size() + 16 * nout;
}

void dfree(void* p) {
  if (p) cudaFreeAsync(p, cudaStreamLegacy);
}

void free_field_device(ipc_field* f) {
  if (f->shared) {  // the batch's allocation goes with its last field
    if (f->shared->refs.fetch_sub(1) == 1) {
      dfree(f->shared->p);
      delete f->shared;
    }
    f->shared = nullptr;
  } else {
    dfree(f->d_cap);  // the bitmaps share its allocation
  }
  dfree(f->d_oidx);  // the outlier values share its allocation
  f->d_cap = nullptr;
  f->d_bm = nullptr;
  f->d_oidx = nullptr;
  f->d_oval = nullptr;
}

int dalloc(void** p, uint64_t bytes, cudaStream_t st) {
  *p = nullptr;
  if (cudaMallocAsync(p, std::max<uint64_t>(bytes, 16), st) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(IPC_ENOMEM, "device allocation failed");
  }
  return IPC_OK;
}

// Pinned host staging of the tables that batched launches read from device
// memory (a pageable source makes every upload a staged, blocking copy): a
// ring of buffers per device, each reused only after the event recorded
// behind its previous copy has completed. `fill` writes the bytes.
constexpr int kStageSlots = 4;
struct StageRing {
  std::mutex mu;
  void* buf[kStageSlots] = {};
  size_t cap[kStageSlots] = {};
  cudaEvent_t ev[kStageSlots] = {};
  bool pending[kStageSlots] = {};
  int next = 0;
};
StageRing g_stage[64];

template <class Fill>
int upload_staged(void* d_dst, size_t bytes, cudaStream_t st, Fill fill) {
  if (bytes == 0) return IPC_OK;
  int dev = 0;
  CU(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(IPC_EINVAL, "device index out of range");
  StageRing& r = g_stage[dev];
  std::lock_guard<std::mutex> lk(r.mu);
  const int s = r.next;
  r.next = (s + 1) % kStageSlots;
  if (r.pending[s]) {
    CU(cudaEventSynchronize(r.ev[s]));
    r.pending[s] = false;
  }
  if (!r.ev[s]) CU(cudaEventCreateWithFlags(&r.ev[s], cudaEventDisableTiming));
  if (r.cap[s] < bytes) {
    if (r.buf[s]) cudaFreeHost(r.buf[s]);
    r.buf[s] = nullptr;
    r.cap[s] = 0;
    const size_t c = std::max<size_t>(bytes + bytes / 2, 1 << 16);
    if (cudaMallocHost(&r.buf[s], c) != cudaSuccess) {
      cudaGetLastError();
      r.buf[s] = nullptr;
      return fail(IPC_ENOMEM, "pinned host allocation failed");
    }
    r.cap[s] = c;
  }
  fill((uint8_t*)r.buf[s]);
  CU(cudaMemcpyAsync(d_dst, r.buf[s], bytes, cudaMemcpyHostToDevice, st));
  CU(cudaEventRecord(r.ev[s], st));
  r.pending[s] = true;
  return IPC_OK;
}

// Keeps freed pool memory for reuse instead of returning it to the driver
// (process-local setting of the device's default pool).
void keep_pool(int dev) {
  static std::once_flag once[64];
  if (dev < 0 || dev >= 64) return;
  std::call_once(once[dev], [dev]() {
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = ~uint64_t(0);
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
  });
}

// Segmented layout of the device streams (independent of the data): per
// stage and plane, nseg segments of RB*CW capacity words and bw bitmap words.
// The planes of a stage follow one another at a fixed stride (the level
// kernels address plane k from plane 0 and that stride).
void stream_layout(ipc_field* f) {
  const Geo& g = f->g;
  f->desc.assign(g.stages.size(), StageDescs{});
  uint64_t cw = 0, bw = 0;
  for (size_t t = 0; t < g.stages.size(); ++t) {
    const StageGeo& sg = g.stages[t];
    const uint64_t pc = sg.nseg * (uint64_t)sg.RB * sg.CW, pb = sg.nseg * sg.bw;
    for (int k = 0; k < 32; ++k) {
      PlaneDesc& pd = f->desc[t].p[k];
      pd.cap_off = cw + (uint64_t)k * pc;
      pd.bm_off = bw + (uint64_t)k * pb;
    }
    cw += 32 * pc;
    bw += 32 * pb;
  }
  f->cap_words = cw;
  f->bm_words = bw;
}

int plan_field(ipc_field* f, cudaStream_t st) {
  stream_layout(f);
  // capacity arrays and bitmaps in one allocation (bitmaps behind)
  const int rc = dalloc((void**)&f->d_cap, (f->cap_words + f->bm_words) * 4, st);
  if (rc) {
    free_field_device(f);
    return rc;
  }
  f->d_bm = f->d_cap + f->cap_words;
  return IPC_OK;
}

// The streams of a batch's fields in one allocation (each field's at a
// 256-byte boundary).
int plan_fields_shared(const std::vector<ipc_field*>& fs, cudaStream_t st) {
  uint64_t words = 0;
  std::vector<uint64_t> at(fs.size());
  for (size_t i = 0; i < fs.size(); ++i) {
    stream_layout(fs[i]);
    at[i] = words;
    words += (fs[i]->cap_words + fs[i]->bm_words + 63) & ~uint64_t(63);
  }
  SharedStreams* sh = new (std::nothrow) SharedStreams();
  if (!sh) return fail(IPC_ENOMEM, "host allocation");
  uint32_t* p = nullptr;
  const int rc = dalloc((void**)&p, words * 4, st);
  if (rc) {
    delete sh;
    return rc;
  }
  sh->p = p;
  sh->refs.store((int)fs.size());
  for (size_t i = 0; i < fs.size(); ++i) {
    fs[i]->shared = sh;
    fs[i]->d_cap = p + at[i];
    fs[i]->d_bm = fs[i]->d_cap + fs[i]->cap_words;
  }
  return IPC_OK;
}

// Kernel arguments of level l (1..K).
LevelArgs level_args(const ipc_field* f, int l) {
  const Geo& g = f->g;
  LevelArgs L{};
  const int64_t s = int64_t(1) << (l - 1);
  for (int e = 0; e < 3; ++e) {
    L.N[e] = g.N[e];
    L.M[e] = (g.N[e] - 1) / s + 1;
  }
  L.stride[2] = 1;
  L.stride[1] = g.N[2];
  L.stride[0] = g.N[1] * g.N[2];
  L.s = s;
  L.interp = f->interp;
  const int BR = level_rows(f->dtype);
  L.nrb = ((uint64_t)L.M[1] + BR - 1) / BR;
  L.nct = ((uint64_t)L.M[2] + kLevelCols - 1) / kLevelCols;
  L.mrb = div_magic(L.nrb);
  L.mct = div_magic(L.nct);
  for (int d = 0; d < 3; ++d) {
    LevelStage& S = L.st[d];
    const int t = g.level_stage[d][l - 1];
    S.present = t >= 0;
    S.t = t;
    if (t < 0) continue;
    const StageGeo& sg = g.stages[t];
    S.RB = sg.RB;
    S.CW = sg.CW;
    S.nrb = sg.nrb;
    S.nct = sg.nct;
    S.bw = sg.bw;
    S.m1 = (uint64_t)sg.m[1];
    S.m2 = (uint64_t)sg.m[2];
    S.wr = sg.wr;
    if (!f->out_off.empty()) {
      S.out_begin = f->out_off[t];
      S.out_end = f->out_off[t + 1];
    }
  }
#ifdef IPC_DEBUG_BOUNDS
  L.lim_cap = f->cap_words;
  L.lim_bm = f->bm_words;
  L.lim_x = (uint64_t)g.N[0] * g.N[1] * g.N[2];
  L.bounds = bounds_record();
#endif
  return L;
}

// Row blocks of a level's reconstruction tiles (their rows depend on the
// code width, see retrieve_rows).
void retrieve_tiling(LevelArgs* L, int dtype, int w16, int ns) {
  const int R = retrieve_rows(dtype, w16, ns);
  L->nrb = ((uint64_t)L->M[1] + R - 1) / R;
  L->mrb = div_magic(L->nrb);
}

// Reconstruction view of level l's plane streams with b_l = b: where plane
// 0 of each stage lies, the plane strides, and the planes to load.
// Offsets of the planes of level l's stages: plane k's capacity array at
// cap0 + k pcap, its bitmap at bm0 + k pbm (words).
void plane_offsets(const ipc_field* f, int l, LevelArgs* L) {
  for (int d = 0; d < 3; ++d) {
    const int t = f->g.level_stage[d][l - 1];
    if (t < 0) continue;
    const StageGeo& sg = f->g.stages[t];
    StagePlanes& S = L->sp[d];
    S.cap0 = f->desc[t].p[0].cap_off;
    S.bm0 = f->desc[t].p[0].bm_off;
    S.pcap = sg.nseg * (uint64_t)sg.RB * sg.CW;
    S.pbm = sg.nseg * sg.bw;
  }
}

void retrieve_planes(const ipc_field* f, int l, int b, LevelArgs* L) {
  plane_offsets(f, l, L);
  for (int d = 0; d < 3; ++d) {
    const int t = f->g.level_stage[d][l - 1];
    StagePlanes& S = L->sp[d];
    S.kmask = 0;
    if (t < 0) continue;
    for (int k = std::max(b, 0); k < 32; ++k)
      if (f->st[t].nnz[k]) S.kmask |= 1u << k;
  }
}

// Container layout from the per-plane nnz: stream sizes and modes, packed
// offsets (stage-major, plane 31..0), mandatory bytes, the selector's tables
// (host only).
void finish_layout(ipc_field* f) {
  const Geo& g = f->g;
  uint64_t word = 0;
  for (size_t t = 0; t < g.stages.size(); ++t) {
    const StageGeo& sg = g.stages[t];
    for (int k = 31; k >= 0; --k) {
      StageTab& s = f->st[t];
      PlaneDesc& pd = f->desc[t].p[k];
      pd.nnz = (uint32_t)s.nnz[k];
      pd.mode = stream_mode(s.nnz[k], sg.words);
      pd.pk_off = word;
      s.size[k] = stream_bytes(s.nnz[k], sg.words);
      word += s.size[k] / 4;
    }
  }
  f->stream_bytes = word * 4;
  uint64_t nout = 0;
  f->out_off.assign(g.stages.size() + 1, 0);
  for (size_t t = 0; t < g.stages.size(); ++t) {
    f->out_off[t] = nout;
    nout += f->st[t].out_idx.size();
  }
  f->out_off[g.stages.size()] = nout;
  f->mandatory = header_size(f);
  f->sel = sel_input(f);
  prepare_selection(&f->sel);
}

// The field's outlier arrays to the device.
int upload_outliers(ipc_field* f, cudaStream_t st) {
  const uint64_t nout = f->out_off.empty() ? 0 : f->out_off.back();
  if (nout == 0) return IPC_OK;  // no outlier arrays (kernels read them only for outliers)
  // indices, then values, in one allocation, from pinned staging
  const int rc = dalloc((void**)&f->d_oidx, nout * 16, st);
  if (rc) return rc;
  f->d_oval = reinterpret_cast<double*>(f->d_oidx + nout);
  return upload_staged(f->d_oidx, nout * 16, st, [&](uint8_t* h) {
    uint64_t* idx = reinterpret_cast<uint64_t*>(h);
    double* val = reinterpret_cast<double*>(h + nout * 8);
    for (auto& s : f->st) {
      std::memcpy(idx, s.out_idx.data(), s.out_idx.size() * 8);
      std::memcpy(val, s.out_val.data(), s.out_val.size() * 8);
      idx += s.out_idx.size();
      val += s.out_val.size();
    }
  });
}

int finish_field(ipc_field* f, cudaStream_t st) {
  finish_layout(f);
  return upload_outliers(f, st);
}

double okey_to_double(unsigned long long k) {
  unsigned long long b = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFULL) : ~k;
  double v;
  std::memcpy(&v, &b, 8);
  return v;
}

// Quantizer half bin (Sec. 4.2.2): eb less 4u(max|x| + eb), the allowance
// for the two roundings of pred + q*bin in the element type, at least eb/2.
double half_bin(double eb, double xmaxabs, int dtype) {
  const double u = dtype == 0 ? 1.0 / 16777216.0 : 1.0 / 9007199254740992.0;
  double eq = eb - 4.0 * u * (xmaxabs + eb);
  if (!(eq >= 0.5 * eb)) eq = 0.5 * eb;
  return eq;
}
double bin_width(const ipc_field* f) {
  const double eq = half_bin(f->eb, f->xmaxabs, f->dtype);
  return f->dtype == 0 ? (double)(float)(2.0 * eq) : 2.0 * eq;
}

template <class T>
void quant_args(double eb, double xmaxabs, void* out) {
  QuantArgs<T> q;
  const double eq = half_bin(eb, xmaxabs, sizeof(T) == 4 ? 0 : 1);
  q.inv2eb = (T)(1.0 / (2.0 * eq));
  q.twoeb = (T)(2.0 * eq);
  const double shrink = sizeof(T) == 4 ? 1.0 - 1.0 / 1048576.0 : 1.0 - 1.0 / 1125899906842624.0;
  q.ebchk = (T)(eb * shrink);
  q.R = (T)(sizeof(T) == 4 ? 2097152.0 : 1073741824.0);
  std::memcpy(out, &q, sizeof(q));
}

// Compression of a batch of fields of one element type (a single field is
// a batch of one): one range launch per field and one host sync; then, for
// every level from the coarsest, ONE launch covering that level's CTAs of
// every field (entry table in device memory); one sync to read the
// per-stage statistics, plane populations and outliers back.
// Level ladders: level l >= 2 of a reconstruction (of a compression) writes
// its whole lattice densely (row major over its extents) to a scratch array,
// which holds the known points of level l - 1; level K + 1 is the anchor
// alone. Only level 1 writes the caller's array (compression: nothing).
// ladder() returns the scratch bytes and the byte offset of each level's
// array (256-byte aligned).
uint64_t lattice_elems(const Geo& g, int l) {
  uint64_t n = 1;
  for (int e = 0; e < 3; ++e) n *= (uint64_t)(((g.N[e] - 1) >> (l - 1)) + 1);
  return n;
}
uint64_t ladder(const Geo& g, size_t esz, std::vector<uint64_t>* off) {
  off->assign(g.K + 2, 0);
  uint64_t tot = 0;
  for (int l = 2; l <= g.K + 1; ++l) {
    (*off)[l] = tot;
    tot += (lattice_elems(g, l) * esz + 255) & ~uint64_t(255);
  }
  return tot;
}
// Level l's layout in a reconstruction: dense lattice strides for its
// output, the known points read from level l + 1's dense lattice `kin`.
void retrieve_layout(LevelArgs* L, const void* kin) {
  for (int e = 0; e < 3; ++e) L->N[e] = L->M[e];
  L->stride[2] = 1;
  L->stride[1] = L->M[2];
  L->stride[0] = L->M[1] * L->M[2];
  L->s = 1;
  L->kin = kin;
  L->kst1 = ((L->M[2] - 1) >> 1) + 1;
  L->kst0 = (((L->M[1] - 1) >> 1) + 1) * L->kst1;
#ifdef IPC_DEBUG_BOUNDS
  L->lim_kin = (uint64_t)(((L->M[0] - 1) >> 1) + 1) * L->kst0;
  L->lim_out = (uint64_t)L->M[0] * L->M[1] * L->M[2];
#endif
}

// Level l's layout in a compression: x is read in its natural layout, the
// known points from level l + 1's dense lattice `kin`, and the level's own
// values go densely to its ladder array.
void compress_layout(LevelArgs* L, const void* kin) {
  L->kin = kin;
  L->kst1 = ((L->M[2] - 1) >> 1) + 1;
  L->kst0 = (((L->M[1] - 1) >> 1) + 1) * L->kst1;
  L->ost1 = L->M[2];
  L->ost0 = L->M[1] * L->M[2];
#ifdef IPC_DEBUG_BOUNDS
  L->lim_kin = (uint64_t)(((L->M[0] - 1) >> 1) + 1) * L->kst0;
  L->lim_out = (uint64_t)L->M[0] * L->M[1] * L->M[2];
#endif
}

int compress_fields(std::vector<ipc_field*>& fs, const std::vector<const void*>& ins,
                    cudaStream_t st) {
  int dev = 0;
  CU(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(IPC_EINVAL, "device index out of range");
  keep_pool(dev);
  Workspace& ws = g_ws[dev];
  std::lock_guard<std::mutex> lock(ws.mu);
  const size_t nf = fs.size();
  if (nf == 0) return IPC_OK;
  if (nf > 65535) return fail(IPC_EINVAL, "too many fields in one batch");
  const int dtype = fs[0]->dtype;
  const size_t esz = dtype == 0 ? 4 : 8;
  // per-field offsets into the shared scratch
  // per field: its level ladder of reconstructed values (byte offsets)
  std::vector<uint64_t> xo(nf + 1, 0), so(nf + 1, 0);
  std::vector<std::vector<uint64_t>> xl(nf);
  int Kmax = 0;
  for (size_t i = 0; i < nf; ++i) {
    xo[i + 1] = xo[i] + ladder(fs[i]->g, esz, &xl[i]);
    so[i + 1] = so[i] + std::max<size_t>(fs[i]->g.stages.size(), 1);
    Kmax = std::max(Kmax, fs[i]->g.K);
  }
  int rc;
  uint64_t dummy = 0;
  if ((rc = grow(&ws.xh, &ws.xh_bytes, xo[nf], 1)) ||
      (rc = grow(&ws.stat, &ws.stat_words, 2 * so[nf], 4)) ||
      (rc = grow(&ws.nnz, &ws.nnz_words, 32 * so[nf], 4)))
    return rc;
  if (ws.small_words < 5 * nf + 1) {
    if (ws.small) cudaFree(ws.small);
    ws.small = nullptr;
    ws.small_words = 0;
    if ((rc = grow(&ws.small, &dummy, 5 * nf + 1, 8))) return rc;
    ws.small_words = 5 * nf + 1;
  }
  // small: [range accumulators, 4 per field | first values, 1 per field | outlier count]
  if (ws.ocap == 0) {
    uint64_t oc = 0;
    if ((rc = grow(&ws.okey, &oc, 1 << 16, 8)) || (rc = grow(&ws.oval, &oc, 1 << 16, 8)))
      return rc;
    ws.ocap = 1 << 16;
  }
  unsigned long long* acc = ws.small;          // 4 per field
  unsigned long long* x0d = ws.small + 4 * nf;  // f64 bits of each field's first value
  unsigned long long* ocount = ws.small + 5 * nf;

  // a0: range over finite values, and the anchor: one launch per
  // kRangeBatch fields, accumulators initialised from pinned staging
  if ((rc = upload_staged(acc, 32 * nf, st, [&](uint8_t* h) {
         unsigned long long* a = reinterpret_cast<unsigned long long*>(h);
         for (size_t i = 0; i < nf; ++i) {
           a[4 * i] = ~0ULL;
           a[4 * i + 1] = a[4 * i + 2] = a[4 * i + 3] = 0ULL;
         }
       })))
    return rc;
  for (size_t i0 = 0; i0 < nf; i0 += kRangeBatch) {
    const int nb = (int)std::min<size_t>(kRangeBatch, nf - i0);
    RangeBatch rb{};
    double by = 0;
    for (int j = 0; j < nb; ++j) {
      rb.x[j] = ins[i0 + j];
      rb.n[j] = fs[i0 + j]->g.n;
      by += (double)(rb.n[j] * esz);
    }
    rb.acc = acc + 4 * i0;
    rb.x0 = x0d + i0;
    const long ph = prof_begin(IPC_KERNEL_RANGE, st);
    CU(launch_range_batch(dtype, rb, nb, 0, st));
    prof_end(ph, st, by);
  }
  // While the range runs: the fields' device streams, and the entry table
  // of every level (coarsest first), uploaded without the quantizer
  // arguments, which wait for the range.
  if (nf >= 8) {
    if ((rc = plan_fields_shared(fs, st))) return rc;
  } else {
    for (size_t i = 0; i < nf; ++i)
      if ((rc = plan_field(fs[i], st))) return rc;
  }
  std::vector<std::array<unsigned char, 32>> quant(nf);
  for (auto& q : quant) q.fill(0);
  std::vector<uint64_t> lev_off(Kmax + 1, 0), lev_ctas(Kmax + 1, 0);
  std::vector<CompressEntry> ents;
  std::vector<std::pair<size_t, int>> who;  // (field, level) of each entry
  bool table = false;  // some level has several fields (the batched kernel)
  // entry positions: level-major (coarsest first), fields in order within
  // a level; the entries themselves are filled per field (large batches on
  // the host pool), the CTA offsets then per level
  std::vector<size_t> pos(nf * (size_t)(Kmax + 1), 0);
  size_t ne = 0;
  for (int l = Kmax; l >= 1; --l) {
    lev_off[l] = ne;
    for (size_t i = 0; i < nf; ++i)
      if (l <= fs[i]->g.K) pos[i * (Kmax + 1) + l] = ne++;
    if (ne - lev_off[l] > 1) table = true;
  }
  ents.resize(ne);
  who.resize(ne);
  auto field_entries = [&](int i) {
    ipc_field* f = fs[i];
    for (int l = 1; l <= f->g.K; ++l) {
      const size_t q = pos[i * (Kmax + 1) + l];
      CompressEntry& e = ents[q];
      e = CompressEntry{};
      e.L = level_args(f, l);
      e.L.vec = 1;  // the scratch is allocated aligned
      plane_offsets(f, l, &e.L);
      e.o = SweepOut{f->d_cap, f->d_bm, ws.nnz + 32 * so[i], ws.okey, ws.oval, ocount,
                     ws.ocap, ws.stat + 2 * so[i], (uint32_t)i};
      compress_layout(&e.L, (uint8_t*)ws.xh + xo[i] + xl[i][l + 1]);
      e.x = ins[i];
      e.xh = l > 1 ? (uint8_t*)ws.xh + xo[i] + xl[i][l] : nullptr;
      std::memcpy(e.quant, quant[i].data(), 32);
      e.write_xh = l > 1;  // the finest level's values are never read again
      who[q] = {(size_t)i, l};
    }
  };
  auto build_entries = [&]() {
    if (nf >= 8)
      HostPool::get().run((int)nf, field_entries);
    else
      for (size_t i = 0; i < nf; ++i) field_entries((int)i);
    for (int l = Kmax; l >= 1; --l) {
      uint64_t cta = 0;
      const size_t end = l > 1 ? lev_off[l - 1] : ne;
      for (size_t q = lev_off[l]; q < end; ++q) {
        ents[q].cta_begin = cta;
        cta += (uint64_t)ents[q].L.M[0] * ents[q].L.nrb * ents[q].L.nct;
      }
      lev_ctas[l] = cta;
    }
  };
  build_entries();
  // device table: [entries | anchors | quantizer arguments per field]
  const size_t eby = ents.size() * sizeof(CompressEntry), aby = nf * sizeof(AnchorEntry);
  CompressEntry* d_ents = nullptr;
  if ((rc = dalloc((void**)&d_ents, eby + aby + 32 * nf, st))) return rc;
  struct EntGuard {
    CompressEntry*& p;
    cudaStream_t s;
    ~EntGuard() { if (p) cudaFreeAsync(p, s); }
  } eguard{d_ents, st};
  AnchorEntry* d_anch = reinterpret_cast<AnchorEntry*>((uint8_t*)d_ents + eby);
  unsigned char* d_quant = (uint8_t*)d_ents + eby + aby;
  auto upload_entries = [&]() {
    return upload_staged(d_ents, eby, st, [&](uint8_t* h) {
      const size_t chunk = 64 << 10, nc = (eby + chunk - 1) / chunk;
      auto part = [&](int c) {
        const size_t o = c * chunk;
        std::memcpy(h + o, (const uint8_t*)ents.data() + o, std::min(chunk, eby - o));
      };
      if (nc >= 4)
        HostPool::get().run((int)nc, part);
      else
        for (size_t c = 0; c < nc; ++c) part((int)c);
    });
  };
  if (table && (rc = upload_entries())) return rc;

  std::vector<unsigned long long> hacc(5 * nf);
  CU(cudaMemcpyAsync(hacc.data(), acc, 40 * nf, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  std::vector<AnchorEntry> anch;  // the origin of level K + 1 is x[0], stored exactly
  anch.reserve(nf);
  for (size_t i = 0; i < nf; ++i) {
    ipc_field* f = fs[i];
    const unsigned long long* a4 = &hacc[4 * i];
    const bool any = a4[3] > 0;
    f->xmin = any ? okey_to_double(a4[0]) : 0.0;
    f->xmax = any ? okey_to_double(a4[1]) : 0.0;
    double ma = 0;
    std::memcpy(&ma, &a4[2], 8);
    f->xmaxabs = any ? ma : 0.0;
    double eb = f->eb_user;
    if (f->eb_mode == IPC_EB_REL) {
      if (!any) return fail(IPC_EINVAL, "relative error bound on a field without finite values");
      const double r = f->xmax - f->xmin;
      eb = r > 0 ? f->eb_user * r : f->eb_user;
    }
    if (!(eb > 0) || !std::isfinite(eb)) return fail(IPC_EINVAL, "error bound must be > 0 and finite");
    f->eb = eb;
    std::memcpy(&f->anchor, &hacc[4 * nf + i], 8);
    if (dtype == 0) quant_args<float>(eb, f->xmaxabs, quant[i].data());
    else quant_args<double>(eb, f->xmaxabs, quant[i].data());
    if (f->g.K > 0) anch.push_back(AnchorEntry{(uint8_t*)ws.xh + xo[i] + xl[i][f->g.K + 1], f->anchor});
  }
  // the host's entries take the quantizer arguments too (single-field
  // launches pass theirs by value, a retry uploads them whole)
  for (size_t q = 0; q < ents.size(); ++q) std::memcpy(ents[q].quant, quant[who[q].first].data(), 32);
  if ((rc = upload_staged(d_anch, aby + 32 * nf, st, [&](uint8_t* h) {
         std::memcpy(h, anch.data(), anch.size() * sizeof(AnchorEntry));
         for (size_t i = 0; i < nf; ++i) std::memcpy(h + aby + 32 * i, quant[i].data(), 32);
       })))
    return rc;

  std::vector<long> level_prof(Kmax + 1, -1);
  unsigned long long nout = 0;
  std::vector<uint32_t> stat(2 * so[nf]), nnz(32 * so[nf]);
  for (int attempt = 0; attempt < 2; ++attempt) {
    if (attempt > 0 && table && (rc = upload_entries())) return rc;
    if (!anch.empty()) CU(launch_set_anchors(dtype, d_anch, (int)anch.size(), st));
    if (table) CU(launch_set_quant(d_ents, (int)ents.size(), d_quant, st));
    CU(cudaMemsetAsync(ws.stat, 0, 2 * so[nf] * 4, st));
    CU(cudaMemsetAsync(ws.nnz, 0, 32 * so[nf] * 4, st));
    CU(cudaMemsetAsync(ocount, 0, 8, st));
    for (int l = Kmax; l >= 1; --l) {
      Nvtx nv("level %d", l);
      const int n_l = (int)((l > 1 ? lev_off[l - 1] : ents.size()) - lev_off[l]);
      const long ph = prof_begin(IPC_KERNEL_COMPRESS_LEVEL, st);
      if (n_l == 1) {  // one field: arguments in the parameter space
        const CompressEntry& e = ents[lev_off[l]];
        CU(launch_level_compress(dtype, e.L, e.x, e.xh, e.write_xh, e.quant, e.o, st));
      } else {
        int quad = 0;  // a field of the level with quadratic boundaries
        for (int q = 0; q < n_l; ++q) quad |= ents[lev_off[l] + q].L.interp == 2;
        CU(launch_level_compress_batch(dtype, d_ents + lev_off[l], n_l, lev_ctas[l], quad, st));
      }
      uint64_t nc = 0;
      for (int q = 0; q < n_l; ++q) {
        const ipc_field* f = fs[who[lev_off[l] + q].first];
        for (int d = 0; d < 3; ++d)
          if (f->g.level_stage[d][l - 1] >= 0) nc += f->g.stages[f->g.level_stage[d][l - 1]].ncodes;
      }
      prof_end(ph, st, (double)(nc * esz));
      level_prof[l] = ph;
    }
    CU(cudaMemcpyAsync(&nout, ocount, 8, cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(stat.data(), ws.stat, 8 * so[nf], cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(nnz.data(), ws.nnz, 128 * so[nf], cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (nout <= ws.ocap) break;
    if (attempt == 1) return fail(IPC_ECUDA, "outlier count changed between passes");
    // grow the outlier buffers to the exact count and run the levels again
    cudaFree(ws.okey);
    cudaFree(ws.oval);
    ws.okey = nullptr;
    ws.oval = nullptr;
    ws.ocap = 0;
    uint64_t oc = 0;
    if ((rc = grow(&ws.okey, &oc, nout, 8)) || (rc = grow(&ws.oval, &oc, nout, 8))) return rc;
    ws.ocap = nout;
    build_entries();
  }

  // outliers sorted by key: (field, stage, code index), so each field's are
  // one run, its stages in order
  std::vector<unsigned long long> key(nout);
  std::vector<double> val(nout);
  std::vector<uint64_t> order(nout), obeg(nf + 1, nout);
  if (nout) {
    CU(cudaMemcpyAsync(key.data(), ws.okey, nout * 8, cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(val.data(), ws.oval, nout * 8, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    for (uint64_t i = 0; i < nout; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](uint64_t a, uint64_t b) { return key[a] < key[b]; });
    for (uint64_t q = nout; q-- > 0;) {
      const size_t fi = (size_t)(key[order[q]] >> 48);
      if (fi >= nf) return fail(IPC_ECUDA, "outlier of an unknown field");
      obeg[fi] = q;
    }
    for (size_t i = nf; i-- > 0;) obeg[i] = std::min(obeg[i], obeg[i + 1]);
  }
  // per field (large batches on the host pool): the stage statistics, its
  // outliers, then the container layout and the selector's tables
  auto finish = [&](int i) {
    ipc_field* f = fs[i];
    const size_t S = f->g.stages.size();
    f->st.assign(S, StageTab{});
    for (size_t t = 0; t < S; ++t) {
      uint32_t orv = stat[2 * (so[i] + t)];
      int h = -1;
      while (orv) { ++h; orv >>= 1; }
      f->st[t].H = h;
      f->st[t].Q = stat[2 * (so[i] + t) + 1];
      for (int k = 0; k < 32; ++k) f->st[t].nnz[k] = nnz[32 * (so[i] + t) + k];
    }
    for (uint64_t q = obeg[i]; q < obeg[i + 1]; ++q) {
      const uint64_t j = order[q];
      const size_t t = (size_t)((key[j] >> 40) & 0xFF);
      f->st[t].out_idx.push_back(key[j] & ((1ULL << 40) - 1));
      f->st[t].out_val.push_back(val[j]);
    }
    finish_layout(f);
  };
  if (nf >= 8)
    HostPool::get().run((int)nf, finish);
  else
    for (size_t i = 0; i < nf; ++i) finish((int)i);
  for (size_t i = 0; i < nf; ++i)
    if ((rc = upload_outliers(fs[i], st))) return rc;
  // algorithmic bytes of each level launch: input values + produced streams
  for (int l = 1; l <= Kmax; ++l) {
    double by = 0;
    for (size_t i = 0; i < nf; ++i) {
      const ipc_field* f = fs[i];
      if (l > f->g.K) continue;
      for (int d = 0; d < 3; ++d) {
        const int t = f->g.level_stage[d][l - 1];
        if (t < 0) continue;
        by += (double)(f->g.stages[t].ncodes * esz);
        for (int k = 0; k < 32; ++k) by += (double)f->st[t].size[k];
      }
    }
    prof_set_bytes(level_prof[l], by);
  }
  return IPC_OK;
}

// Per-field choice of the interpolation (IPC_INTERP_AUTO): the mode whose
// container is smallest on the centred block of extents min(N_d, c),
// c = 2^20 / 1024 / 128 for 1 / 2 / 3 dimensions (first index
// floor((N_d - e_d) / 2)), compressed with the whole field's absolute error
// bound; the lower mode on a tie. The whole fields' ranges (relative
// bounds) take one range launch per element type, the blocks are copied
// out with strided copies, and every block's three trial compressions run
// as one batch per element type.
struct AutoItem {
  const void* d_in;
  int dtype, ndim;
  int64_t dims[3];
  int eb_mode, bound;
  double eb;
  int mode;  // out: the chosen interpolation
};

int resolve_auto(std::vector<AutoItem>& v, cudaStream_t st) {
  const size_t na = v.size();
  if (na == 0) return IPC_OK;
  int rc;
  struct DevFree {
    void* p = nullptr;
    cudaStream_t s;
    ~DevFree() { if (p) cudaFreeAsync(p, s); }
  };
  // the absolute bound of every field
  std::vector<double> eb_abs(na);
  std::vector<size_t> order;  // relative-bound fields, by element type
  for (int dt = 0; dt < 2; ++dt)
    for (size_t i = 0; i < na; ++i)
      if (v[i].dtype == dt && v[i].eb_mode == IPC_EB_REL) order.push_back(i);
  for (size_t i = 0; i < na; ++i)
    if (v[i].eb_mode != IPC_EB_REL) eb_abs[i] = v[i].eb;
  if (!order.empty()) {
    const size_t nr = order.size();
    DevFree acc{nullptr, st};
    if ((rc = dalloc(&acc.p, 40 * nr, st))) return rc;
    unsigned long long* a = (unsigned long long*)acc.p;  // [4 per field | first value per field]
    if ((rc = upload_staged(a, 32 * nr, st, [&](uint8_t* h) {
           unsigned long long* w = reinterpret_cast<unsigned long long*>(h);
           for (size_t k = 0; k < nr; ++k) {
             w[4 * k] = ~0ULL;
             w[4 * k + 1] = w[4 * k + 2] = w[4 * k + 3] = 0ULL;
           }
         })))
      return rc;
    for (size_t k0 = 0; k0 < nr;) {
      const int dt = v[order[k0]].dtype;
      RangeBatch rb{};
      int nb = 0;
      while (k0 + nb < nr && nb < kRangeBatch && v[order[k0 + nb]].dtype == dt) {
        const AutoItem& it = v[order[k0 + nb]];
        rb.x[nb] = it.d_in;
        rb.n[nb] = (uint64_t)it.dims[0] * (uint64_t)(it.ndim > 1 ? it.dims[1] : 1) *
                   (uint64_t)(it.ndim > 2 ? it.dims[2] : 1);
        ++nb;
      }
      rb.acc = a + 4 * k0;
      rb.x0 = a + 4 * nr + k0;
      CU(launch_range_batch(dt, rb, nb, 0, st));
      k0 += nb;
    }
    std::vector<unsigned long long> h(4 * nr);
    CU(cudaMemcpyAsync(h.data(), a, 32 * nr, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    for (size_t k = 0; k < nr; ++k) {
      if (h[4 * k + 3] == 0)
        return fail(IPC_EINVAL, "relative error bound on a field without finite values");
      const double r = okey_to_double(h[4 * k + 1]) - okey_to_double(h[4 * k]);
      const size_t i = order[k];
      eb_abs[i] = r > 0 ? v[i].eb * r : v[i].eb;
    }
  }
  for (size_t i = 0; i < na; ++i)
    if (!(eb_abs[i] > 0) || !std::isfinite(eb_abs[i]))
      return fail(IPC_EINVAL, "error bound must be > 0 and finite");
  // the blocks, one after another in one allocation
  std::vector<std::array<int64_t, 3>> ext(na);
  std::vector<uint64_t> boff(na);
  uint64_t tot = 0;
  for (size_t i = 0; i < na; ++i) {
    const AutoItem& it = v[i];
    const int64_t cap = it.ndim == 1 ? (int64_t)1 << 20 : it.ndim == 2 ? 1024 : 128;
    uint64_t n = it.dtype == IPC_F32 ? 4 : 8;
    for (int d = 0; d < it.ndim; ++d) {
      ext[i][d] = std::min<int64_t>(it.dims[d], cap);
      n *= (uint64_t)ext[i][d];
    }
    boff[i] = tot;
    tot += (n + 255) & ~uint64_t(255);
  }
  DevFree blocks{nullptr, st};
  if ((rc = dalloc(&blocks.p, tot, st))) return rc;
  for (size_t i = 0; i < na; ++i) {
    const AutoItem& it = v[i];
    const size_t esz = it.dtype == IPC_F32 ? 4 : 8;
    int64_t N[3] = {1, 1, 1}, e[3] = {1, 1, 1}, o[3] = {0, 0, 0};
    for (int d = 0; d < it.ndim; ++d) {
      N[3 - it.ndim + d] = it.dims[d];
      e[3 - it.ndim + d] = ext[i][d];
      o[3 - it.ndim + d] = (it.dims[d] - ext[i][d]) / 2;
    }
    const uint8_t* src = (const uint8_t*)it.d_in;
    uint8_t* dst = (uint8_t*)blocks.p + boff[i];
    if (e[0] == 1 && e[1] == 1) {  // one row (a 1-D field): a plain copy
      CU(cudaMemcpyAsync(dst, src + (size_t)((o[0] * N[1] + o[1]) * N[2] + o[2]) * esz,
                         (size_t)e[2] * esz, cudaMemcpyDeviceToDevice, st));
      continue;
    }
    for (int64_t i0 = 0; i0 < e[0]; ++i0)
      CU(cudaMemcpy2DAsync(dst + (size_t)(i0 * e[1] * e[2]) * esz, (size_t)e[2] * esz,
                           src + (size_t)(((o[0] + i0) * N[1] + o[1]) * N[2] + o[2]) * esz,
                           (size_t)N[2] * esz, (size_t)e[2] * esz, (size_t)e[1],
                           cudaMemcpyDeviceToDevice, st));
  }
  // three trial compressions per block, one batch per element type
  std::vector<ipc_field*> trial(3 * na, nullptr);
  struct TrialFree {
    std::vector<ipc_field*>& t;
    ~TrialFree() {
      for (auto* f : t)
        if (f) {
          free_field_device(f);
          f->tag = kDeadTag;
          delete f;
        }
    }
  } tguard{trial};
  int dev = 0;
  CU(cudaGetDevice(&dev));
  for (size_t i = 0; i < na; ++i)
    for (int m = 0; m < 3; ++m) {
      ipc_field* f = new (std::nothrow) ipc_field();
      if (!f) return fail(IPC_ENOMEM, "host allocation");
      trial[3 * i + m] = f;
      f->tag = kFieldTag;
      if (!build_geo(v[i].ndim, ext[i].data(), v[i].dtype, &f->g)) return fail(IPC_EINVAL, "shape");
      f->device = dev;
      f->dtype = v[i].dtype;
      f->interp = m;
      f->bound = v[i].bound;
      f->eb_mode = IPC_EB_ABS;
      f->eb_user = eb_abs[i];
    }
  for (int dt = 0; dt < 2; ++dt) {
    std::vector<ipc_field*> fs;
    std::vector<const void*> ins;
    for (size_t i = 0; i < na; ++i)
      if (v[i].dtype == dt)
        for (int m = 0; m < 3; ++m) {
          fs.push_back(trial[3 * i + m]);
          ins.push_back((const uint8_t*)blocks.p + boff[i]);
        }
    if (!fs.empty() && (rc = compress_fields(fs, ins, st))) return rc;
  }
  for (size_t i = 0; i < na; ++i) {
    v[i].mode = 0;
    uint64_t best = 0;
    for (int m = 0; m < 3; ++m) {
      const ipc_field* f = trial[3 * i + m];
      const uint64_t bytes = f->mandatory + f->stream_bytes;
      if (m == 0 || bytes < best) {
        best = bytes;
        v[i].mode = m;
      }
    }
  }
  return IPC_OK;
}

// ---------------------------------------------------------------------------
// Optimized loader (Sec. 5.2 / 5.3): the field's stage statistics and plane
// sizes go to the host selector (ipc_select.cu).
// ---------------------------------------------------------------------------
SelInput sel_input(const ipc_field* f) {
  SelInput in;
  in.K = f->g.K;
  in.dtype = f->dtype;
  in.interp = f->interp;
  in.bound = f->bound;
  in.eb_mode = f->eb_mode;
  in.eb = f->eb;
  in.bin = bin_width(f) / f->eb;
  in.xmin = f->xmin;
  in.xmax = f->xmax;
  in.xmaxabs = f->xmaxabs;
  in.n = f->g.n;
  in.mandatory = f->mandatory;
  in.st.resize(f->g.stages.size());
  for (size_t t = 0; t < in.st.size(); ++t) {
    SelStage& s = in.st[t];
    s.level = f->g.stages[t].level;
    s.H = f->st[t].H;
    s.Q = f->st[t].Q;
    std::memcpy(s.size, f->st[t].size, sizeof(s.size));
  }
  return in;
}

int select(const ipc_field* f, ipc_target tg, const std::vector<int>* upper, std::vector<int>* b,
           uint64_t* bytes, double* bound, uint64_t* rparts = nullptr) {
  const char* why = "";
  const int rc =
      select_planes(f->sel, tg.kind, tg.value, upper, b, bytes, bound, &why, rparts);
  return rc ? fail(rc, why) : IPC_OK;
}

// Whether the planes loaded at level l (k >= b with nonzero words in one of
// the level's stages) span at most 16: the kernel then keeps 16-bit codes.
bool level_w16(const ipc_field* f, int l, int b) {
  int ktop = -1;
  for (int d = 0; d < 3; ++d) {
    const int t = f->g.level_stage[d][l - 1];
    if (t < 0) continue;
    for (int k = 31; k > ktop && k >= b; --k)
      if (f->st[t].nnz[k]) {
        ktop = k;
        break;
      }
  }
  // 16-bit rows scale 2eb by up to 2^16 (the product must stay finite)
  const double lim = f->dtype == 0 ? (double)FLT_MAX : DBL_MAX;
  return ktop - b <= 15 && bin_width(f) * 65536.0 <= lim;
}

// Launch shapes chosen by measurement (ipc_autotune_retrieve), per element
// type, code width and level lattice extents; process-wide.
struct ShapeKey {
  int dtype, w16;
  int64_t M0, M1, M2;
  bool operator<(const ShapeKey& o) const {
    if (dtype != o.dtype) return dtype < o.dtype;
    if (w16 != o.w16) return w16 < o.w16;
    if (M0 != o.M0) return M0 < o.M0;
    if (M1 != o.M1) return M1 < o.M1;
    return M2 < o.M2;
  }
};
std::mutex g_shape_mu;
std::map<ShapeKey, RetrieveShape> g_shapes;

ShapeKey shape_key(int dtype, int w16, const LevelArgs& L) {
  return ShapeKey{dtype, w16 ? 1 : 0, L.M[0], L.M[1], L.M[2]};
}
// The tuned shape of a level launch, or the default (ns = per_sm = 0).
RetrieveShape tuned_shape(const ShapeKey& k) {
  std::lock_guard<std::mutex> lk(g_shape_mu);
  auto it = g_shapes.find(k);
  return it == g_shapes.end() ? RetrieveShape{} : it->second;
}

// State of an incremental view: per stage, two words per code word.
uint64_t state_words(const Geo& g, std::vector<uint64_t>* off) {
  off->assign(g.stages.size(), 0);
  uint64_t tot = 0;
  for (size_t t = 0; t < g.stages.size(); ++t) {
    (*off)[t] = tot;
    tot += 2 * g.stages[t].words;
  }
  return tot;
}

// The coarse levels K .. Lc of a reconstruction with selection b, for one
// CTA (ipc_coarse.cu): the smallest Lc whose lattice and codes fit its shared
// memory. Returns false when not even level K fits.
bool coarse_plan(const ipc_field* f, const std::vector<int>& b, void* out, CoarseArgs* a) {
  const Geo& g = f->g;
  if (g.K < 1) return false;
  std::memset(a, 0, sizeof(*a));
  a->K = g.K;
  a->interp = f->interp;
  a->esz = f->dtype == 0 ? 4 : 8;
  a->anchor = f->anchor;
  a->twoeb = bin_width(f);
  a->out = out;
  a->cap = f->d_cap;
  a->bm = f->d_bm;
  a->oidx = f->d_oidx;
  a->oval = f->d_oval;
  int best = 0;
  for (int Lc = g.K; Lc >= 1; --Lc) {
    CoarseArgs t = *a;
    t.Lc = Lc;
    for (int e = 0; e < 3; ++e) t.ML[e] = ((g.N[e] - 1) >> (Lc - 1)) + 1;
    int n = 0;
    bool ok = true;
    for (size_t s = 0; s < g.stages.size() && ok; ++s) {
      const StageGeo& sg = g.stages[s];
      if (sg.level < Lc) continue;
      if (n == kCoarseMaxStages) { ok = false; break; }
      CoarseStage& S = t.st[n++];
      S.level = sg.level;
      S.dim = sg.dim3;
      S.b = b[sg.level - 1];
      for (int e = 0; e < 3; ++e) S.m[e] = sg.m[e];
      S.wr = sg.wr;
      S.words = sg.words;
      S.RB = sg.RB;
      S.CW = sg.CW;
      S.nrb = sg.nrb;
      S.nct = sg.nct;
      S.bw = sg.bw;
      S.cap0 = f->desc[s].p[0].cap_off;
      S.bm0 = f->desc[s].p[0].bm_off;
      S.pcap = sg.nseg * (uint64_t)sg.RB * sg.CW;
      S.pbm = sg.nseg * sg.bw;
      S.kmask = 0;
      for (int k = std::max(S.b, 0); k < 32; ++k)
        if (f->st[s].nnz[k]) S.kmask |= 1u << k;
      S.out_begin = f->out_off[s];
      S.out_end = f->out_off[s + 1];
    }
    if (!ok) break;
    t.nst = n;
    uint64_t off = 0;
    for (int i = 0; i < n; ++i) {
      t.st[i].code_off = off;
      off += (uint64_t)(t.st[i].m[0] * t.st[i].m[1] * t.st[i].m[2]);
    }
    if (coarse_smem(t) > kCoarseSmem) break;
    *a = t;
    best = Lc;
  }
  return best > 0;
}

// Algorithm 1 on the device: the anchor, then one fused launch per level
// (coarse to fine); outliers are applied inside the level kernels. The
// coarse levels that fit one CTA's shared memory run together in one launch
// (ipc_coarse.cu). With a view state (`state`, per-stage offsets `soff`)
// every level takes the level kernels, which also record the digits of
// every code at its two lowest loaded planes.
int reconstruct(ipc_field* f, const std::vector<int>& b, void* d_out, cudaStream_t st,
                uint32_t* state = nullptr, const std::vector<uint64_t>* soff = nullptr) {
  const Geo& g = f->g;
  const size_t esz = f->dtype == 0 ? 4 : 8;
  std::vector<uint64_t> off;
  uint8_t* scr = nullptr;
  if (g.K > 0) {
    int rc = dalloc((void**)&scr, ladder(g, esz, &off), st);
    if (rc) return rc;
  }
  struct Free {  // stream-ordered after the launches
    uint8_t* p;
    cudaStream_t s;
    ~Free() { if (p) cudaFreeAsync(p, s); }
  } guard{scr, st};
  int ltop = g.K;  // the finest level not done yet
  {
    CoarseArgs ca;
    if (!state && coarse_plan(f, b, nullptr, &ca)) {
      ca.out = ca.Lc == 1 ? d_out : (void*)(scr + off[ca.Lc]);
      double by = 0;
      uint64_t nc = 0;
      for (int i = 0; i < ca.nst; ++i) {
        const int t = g.level_stage[ca.st[i].dim][ca.st[i].level - 1];
        nc += g.stages[t].ncodes;
        for (int k = ca.st[i].b; k < 32; ++k) by += (double)f->st[t].size[k];
      }
      const long ph = prof_begin(IPC_KERNEL_COARSE, st);
      CU(launch_coarse(f->dtype, ca, st));
      prof_end(ph, st, by + (double)(nc * esz));
      ltop = ca.Lc - 1;
    }
  }
  if (ltop == g.K) {
    const long ph = prof_begin(IPC_KERNEL_ANCHOR, st);
    CU(launch_set_anchor(f->dtype, g.K > 0 ? (void*)(scr + off[g.K + 1]) : d_out, f->anchor, st));
    prof_end(ph, st, 8);
  }
  const double twoeb = bin_width(f);
  for (int l = ltop; l >= 1; --l) {
    Nvtx nv("level %d", l);
    LevelArgs L = level_args(f, l);
    retrieve_layout(&L, scr + off[l + 1]);
    retrieve_planes(f, l, b[l - 1], &L);
    L.stream_out = l == 1;
    void* o = l == 1 ? d_out : (void*)(scr + off[l]);
    double by = 0;
    uint64_t nc = 0;
    for (int d = 0; d < 3; ++d) {
      const int t = g.level_stage[d][l - 1];
      if (t < 0) continue;
      nc += g.stages[t].ncodes;
      for (int k = b[l - 1]; k < 32; ++k) by += (double)f->st[t].size[k];
    }
    const int w16 = level_w16(f, l, b[l - 1]) ? 1 : 0;
    RetrieveShape sh = tuned_shape(shape_key(f->dtype, w16, L));
    if (!sh.ns) sh.ns = retrieve_subtiles(L.M[2], w16);
    retrieve_tiling(&L, f->dtype, w16, sh.ns);
    const long ph = prof_begin(IPC_KERNEL_RETRIEVE_LEVEL, st);
    if (state) {
      for (int d = 0; d < 3; ++d) {
        const int t = g.level_stage[d][l - 1];
        L.sp[d].carry = t >= 0 ? state + (*soff)[t] : nullptr;
        L.sp[d].carry_in = nullptr;
      }
      CU(launch_level_retrieve_mode(f->dtype, L, o, twoeb, b[l - 1], f->d_cap, f->d_bm,
                                    f->d_oidx, f->d_oval, w16, sh, 1, st));
    } else {
      CU(launch_level_retrieve(f->dtype, L, o, twoeb, b[l - 1], f->d_cap, f->d_bm, f->d_oidx,
                               f->d_oval, w16, sh, st));
    }
    prof_end(ph, st, by + (double)(nc * esz));
  }
  return IPC_OK;
}

// Algorithm 2 on the device: from selection bo to bn (bn <= bo), read only
// the planes [bn_l, bo_l) of every level, decode them with the view's state
// as prefix, interpolate the increment from zero and add it to d_out (which
// holds the current reconstruction). Levels coarser than the coarsest one
// that loads planes have a zero increment and are skipped: the known points
// of that level are zeros. *stream_bytes: the plane-stream bytes read.
// The state is read from `state_in` and written to `state_out` (whole: the
// words of levels that load no new planes are copied).
int reconstruct_increment(ipc_field* f, const std::vector<int>& bo, const std::vector<int>& bn,
                          void* d_out, const uint32_t* state_in, uint32_t* state_out,
                          const std::vector<uint64_t>& soff, cudaStream_t st,
                          uint64_t* stream_bytes) {
  const Geo& g = f->g;
  const size_t esz = f->dtype == 0 ? 4 : 8;
  *stream_bytes = 0;
  int lc = 0;
  for (int l = 1; l <= g.K; ++l)
    if (bn[l - 1] < bo[l - 1]) lc = l;
  if (lc == 0) return IPC_OK;
  std::vector<uint64_t> off;
  uint8_t* scr = nullptr;
  int rc = dalloc((void**)&scr, ladder(g, esz, &off), st);
  if (rc) return rc;
  struct Free {  // stream-ordered after the launches
    uint8_t* p;
    cudaStream_t s;
    ~Free() { if (p) cudaFreeAsync(p, s); }
  } guard{scr, st};
  // the increments of level lc's known points (level lc + 1, or the anchor)
  CU(cudaMemsetAsync(scr + off[lc + 1], 0, lattice_elems(g, lc + 1) * esz, st));
  // the state of the stages whose level loads no new planes is carried over
  for (size_t t = 0; t < g.stages.size(); ++t) {
    const int l = g.stages[t].level;
    if (bn[l - 1] < bo[l - 1]) continue;
    CU(cudaMemcpyAsync(state_out + soff[t], state_in + soff[t], 8 * g.stages[t].words,
                       cudaMemcpyDeviceToDevice, st));
  }
  const double twoeb = bin_width(f);
  const double lim = f->dtype == 0 ? (double)FLT_MAX : DBL_MAX;
  for (int l = lc; l >= 1; --l) {
    Nvtx nv("level %d", l);
    const int b0 = bo[l - 1], b1 = bn[l - 1];
    LevelArgs L = level_args(f, l);
    retrieve_layout(&L, scr + off[l + 1]);
    retrieve_planes(f, l, b1, &L);
    double by = 0;
    uint64_t nc = 0, nw = 0;
    for (int d = 0; d < 3; ++d) {
      const int t = g.level_stage[d][l - 1];
      L.sp[d].carry = t >= 0 ? state_out + soff[t] : nullptr;
      L.sp[d].carry_in = t >= 0 ? state_in + soff[t] : nullptr;
      if (t < 0) continue;
      // only the new planes [b1, b0)
      L.sp[d].kmask &= b0 >= 32 ? ~0u : ((1u << b0) - 1u);
      nc += g.stages[t].ncodes;
      nw += g.stages[t].words;
      for (int k = b1; k < b0; ++k) by += (double)f->st[t].size[k];
    }
    *stream_bytes += (uint64_t)by;
    L.bo = b0;
    L.stream_out = l == 1;
    void* o = l == 1 ? d_out : (void*)(scr + off[l]);
    const int w16 = (b0 - b1 <= 16 && bin_width(f) * 65536.0 <= lim) ? 1 : 0;
    RetrieveShape sh = tuned_shape(shape_key(f->dtype, w16, L));
    if (!sh.ns) sh.ns = retrieve_subtiles(L.M[2], w16);
    retrieve_tiling(&L, f->dtype, w16, sh.ns);
    const long ph = prof_begin(IPC_KERNEL_INCREMENT_LEVEL, st);
    CU(launch_level_retrieve_mode(f->dtype, L, o, twoeb, b1, f->d_cap, f->d_bm, f->d_oidx,
                                  f->d_oval, w16, sh, 2, st));
    const double state_bytes = b0 > b1 ? 16.0 * (double)nw : 0.0;
    // level 1 reads and writes the whole output; coarser levels write their
    // targets' increments
    prof_end(ph, st, by + state_bytes + (l == 1 ? 2.0 * (double)g.n * (double)esz
                                                 : (double)(nc * esz)));
  }
  return IPC_OK;
}

// Batched reconstruction of fields of one element type: the anchors in one
// launch, then ONE launch per level over that level's CTAs of every field.
// The entry table and the fields' scratch ladders are one device allocation
// (`tab`); the entries carry scratch offsets until upload_table turns them
// into pointers. When `plan` is set the launches go to a capturing stream
// and no profiler events are recorded.
struct BatchTable {
  std::vector<RetrieveEntry> ents;
  std::vector<AnchorEntry> anchors;
  std::vector<int64_t> kin_off, out_off, anch_off;  // scratch offsets (-1: caller's array)
  // fields whose coarse levels run in one CTA each (ipc_coarse.cu): their
  // arguments, where each writes its level-Lc lattice (-1: the caller's
  // array), and the most shared memory one of them takes
  std::vector<CoarseArgs> coarse;
  std::vector<int64_t> coarse_off;
  size_t coarse_smem = 0;
  // One launch per (level, code width): a level's entries whose loaded
  // planes span at most 16 go to the 16-bit kernel, the others to the
  // 32-bit one, coarse levels first.
  struct Launch {
    uint64_t off = 0;   // first entry
    int n = 0;          // entries
    uint64_t ctas = 0;  // tiles over the entries
    int w16 = 1;        // 16-bit code rows
    int ns = 1;         // sub-tiles per tile
    int psm = 0;        // CTAs per SM (0: as many as fit)
    int quad = 0;       // some entry interpolates with quadratic boundaries
  };
  std::vector<Launch> launches;
  uint64_t scratch = 0;      // bytes of the fields' scratch ladders
  int Kmax = 0;
  double alg_bytes = 0;
};

// What a batched reconstruction needs of one field, independent of the
// other fields: its scratch ladder, its coarse-level plan, and per level
// it runs in the level kernels the kernel arguments (layout and planes;
// the row tiling waits for the launch's sub-tile count) and the code width.
struct FieldPrep {
  uint64_t scratch = 0;
  std::vector<uint64_t> off;  // ladder offsets per level
  bool coarse = false;
  CoarseArgs ca;
  int ltop = 0;                  // the finest level the level kernels start at
  std::vector<LevelArgs> las;    // index l - 1, levels 1..ltop
  std::vector<uint8_t> w16;      // index l - 1
  std::vector<double> lbytes;    // algorithmic bytes per level, index l - 1
  double coarse_bytes = 0;
};

void prepare_field(const ipc_field* f, const std::vector<int>& b, FieldPrep* P) {
  const Geo& g = f->g;
  const size_t esz = f->dtype == 0 ? 4 : 8;
  P->scratch = g.K > 0 ? ladder(g, esz, &P->off) : 0;
  P->coarse = coarse_plan(f, b, nullptr, &P->ca);
  P->ltop = P->coarse ? P->ca.Lc - 1 : g.K;
  if (P->coarse)
    for (int j = 0; j < P->ca.nst; ++j) {
      const int t = g.level_stage[P->ca.st[j].dim][P->ca.st[j].level - 1];
      P->coarse_bytes += (double)(g.stages[t].ncodes * esz);
      for (int k = P->ca.st[j].b; k < 32; ++k) P->coarse_bytes += (double)f->st[t].size[k];
    }
  P->las.resize(P->ltop);
  P->w16.resize(P->ltop);
  P->lbytes.assign(P->ltop, 0.0);
  for (int l = 1; l <= P->ltop; ++l) {
    const int bl = b[l - 1];
    LevelArgs& L = P->las[l - 1];
    L = level_args(f, l);
    retrieve_layout(&L, nullptr);
    retrieve_planes(f, l, bl, &L);
    L.stream_out = l == 1;
    P->w16[l - 1] = level_w16(f, l, bl) ? 1 : 0;
    for (int d = 0; d < 3; ++d) {
      const int t = g.level_stage[d][l - 1];
      if (t < 0) continue;
      P->lbytes[l - 1] += (double)(g.stages[t].ncodes * esz);
      for (int k = bl; k < 32; ++k) P->lbytes[l - 1] += (double)f->st[t].size[k];
    }
  }
}

void build_retrieve_table(const std::vector<ipc_field*>& fs, const std::vector<std::vector<int>>& bs,
                          const std::vector<void*>& outs, BatchTable* T) {
  const size_t nf = fs.size();
  T->Kmax = 0;
  for (auto* f : fs) T->Kmax = std::max(T->Kmax, f->g.K);
  T->launches.clear();
  T->ents.clear();
  T->anchors.clear();
  T->kin_off.clear();
  T->out_off.clear();
  T->anch_off.clear();
  T->coarse.clear();
  T->coarse_off.clear();
  T->coarse_smem = 0;
  T->alg_bytes = 0;
  T->ents.reserve(fs.size() * (size_t)T->Kmax);
  T->kin_off.reserve(fs.size() * (size_t)T->Kmax);
  T->out_off.reserve(fs.size() * (size_t)T->Kmax);
  T->coarse.reserve(fs.size());
  // the fields' own preparation is independent: large batches spread it
  // over the host pool
  std::vector<FieldPrep> P(nf);
  if (nf >= 8)
    HostPool::get().run((int)nf, [&](int i) { prepare_field(fs[i], bs[i], &P[i]); });
  else
    for (size_t i = 0; i < nf; ++i) prepare_field(fs[i], bs[i], &P[i]);
  // each field's scratch ladder, one after the other
  std::vector<uint64_t> base(nf, 0);
  T->scratch = 0;
  for (size_t i = 0; i < nf; ++i) {
    base[i] = T->scratch;
    T->scratch += P[i].scratch;
  }
  for (size_t i = 0; i < nf; ++i) {
    const int K = fs[i]->g.K;
    if (P[i].coarse) {
      const CoarseArgs& ca = P[i].ca;
      T->coarse.push_back(ca);
      T->coarse_off.push_back(ca.Lc == 1 ? -1 : (int64_t)(base[i] + P[i].off[ca.Lc]));
      if (ca.Lc == 1) T->coarse.back().out = outs[i];
      T->coarse_smem = std::max(T->coarse_smem, coarse_smem(ca));
      T->alg_bytes += P[i].coarse_bytes;
      continue;
    }
    T->anchors.push_back(AnchorEntry{outs[i], fs[i]->anchor});
    T->anch_off.push_back(K > 0 ? (int64_t)(base[i] + P[i].off[K + 1]) : -1);
  }
  std::vector<size_t> group[2];  // a level's fields by code width (index: w16)
  for (int l = T->Kmax; l >= 1; --l) {
    group[0].clear();
    group[1].clear();
    for (size_t i = 0; i < nf; ++i)
      if (l <= P[i].ltop) group[P[i].w16[l - 1]].push_back(i);
    for (int w16 : {1, 0}) {
      if (group[w16].empty()) continue;
      BatchTable::Launch ln;
      ln.off = T->ents.size();
      ln.n = (int)group[w16].size();
      ln.w16 = w16;
      // the tile shape holds for every entry; a tuned shape applies when
      // every entry's level has the same key
      int ns = 4;
      bool same = true;
      ShapeKey key{};
      int seen = 0;
      for (size_t i : group[w16]) {
        const LevelArgs& La = P[i].las[l - 1];
        ln.quad |= fs[i]->interp == IPC_CUBIC_QUAD;
        ns = std::min(ns, retrieve_subtiles(La.M[2], w16));
        const ShapeKey k = shape_key(fs[i]->dtype, w16, La);
        if (seen++ && (k < key || key < k)) same = false;
        key = k;
      }
      if (same) {
        const RetrieveShape sh = tuned_shape(key);
        if (sh.ns && sh.ns <= ns) ns = sh.ns;
        ln.psm = sh.per_sm;
      }
      ln.ns = ns;
      uint64_t cta = 0;
      for (size_t i : group[w16]) {
        ipc_field* f = fs[i];
        RetrieveEntry e{};
        e.L = P[i].las[l - 1];
        retrieve_tiling(&e.L, f->dtype, w16, ns);
        e.out = outs[i];
        e.cap = f->d_cap;
        e.bm = f->d_bm;
        e.oidx = f->d_oidx;
        e.oval = f->d_oval;
        e.twoeb = bin_width(f);
        e.b = bs[i][l - 1];
        e.cta_begin = cta;
        cta += retrieve_tiles(e.L, ns);
        T->ents.push_back(e);
        T->kin_off.push_back((int64_t)(base[i] + P[i].off[l + 1]));
        T->out_off.push_back(l == 1 ? -1 : (int64_t)(base[i] + P[i].off[l]));
        T->alg_bytes += P[i].lbytes[l - 1];
      }
      ln.ctas = cta;
      T->launches.push_back(ln);
    }
  }
}

// Table layout: [scratch ladders | entries | anchors]; the scratch comes
// first so that it keeps the allocation's alignment.
uint64_t table_scratch(const BatchTable& T) { return (T.scratch + 255) & ~uint64_t(255); }

int launch_retrieve_table(int dtype, const BatchTable& T, void* tab, cudaStream_t st,
                          bool profile, uint64_t* launches) {
  RetrieveEntry* d_ents = (RetrieveEntry*)((uint8_t*)tab + table_scratch(T));
  AnchorEntry* d_anch = (AnchorEntry*)((uint8_t*)d_ents + T.ents.size() * sizeof(RetrieveEntry));
  CoarseArgs* d_coarse = (CoarseArgs*)((uint8_t*)d_anch + T.anchors.size() * sizeof(AnchorEntry));
  uint64_t nl = 0;
  if (!T.anchors.empty()) {
    const long ph = profile ? prof_begin(IPC_KERNEL_ANCHOR, st) : -1;
    CU(launch_set_anchors(dtype, d_anch, (int)T.anchors.size(), st));
    if (profile) prof_end(ph, st, 16.0 * T.anchors.size());
    ++nl;
  }
  if (!T.coarse.empty()) {
    const long ph = profile ? prof_begin(IPC_KERNEL_COARSE, st) : -1;
    CU(launch_coarse_batch(dtype, d_coarse, (int)T.coarse.size(), T.coarse_smem, st));
    if (profile) prof_end(ph, st, 0.0);
    ++nl;
  }
  // the algorithmic bytes of the whole batch are reported with its last launch
  for (size_t j = 0; j < T.launches.size(); ++j) {
    Nvtx nv("launch %d", (int)j);
    const BatchTable::Launch& ln = T.launches[j];
    const long ph = profile ? prof_begin(IPC_KERNEL_RETRIEVE_LEVEL, st) : -1;
    CU(launch_level_retrieve_batch(dtype, d_ents + ln.off, ln.n, ln.ctas, ln.w16, ln.ns, ln.psm,
                                   ln.quad, st));
    if (profile) prof_end(ph, st, j + 1 == T.launches.size() ? T.alg_bytes : 0.0);
    ++nl;
  }
  if (!profile) g_launches.fetch_add(nl, std::memory_order_relaxed);
  if (launches) *launches = nl;
  return IPC_OK;
}

int upload_table(const BatchTable& T, void** tab, cudaStream_t st, bool pooled) {
  const uint64_t sb = table_scratch(T);
  const size_t eb = T.ents.size() * sizeof(RetrieveEntry) + T.anchors.size() * sizeof(AnchorEntry);
  const size_t bytes = eb + T.coarse.size() * sizeof(CoarseArgs);
  int rc;
  if (pooled) {
    if ((rc = dalloc(tab, sb + bytes, st))) return rc;
  } else if (cudaMalloc(tab, std::max<size_t>(sb + bytes, 16)) != cudaSuccess) {
    cudaGetLastError();
    return fail(IPC_ENOMEM, "device allocation failed");
  }
  uint8_t* base = (uint8_t*)*tab;
  // the entries with their scratch offsets turned into addresses, written
  // straight into pinned staging
  rc = upload_staged(base + sb, bytes, st, [&](uint8_t* h) {
    RetrieveEntry* ents = reinterpret_cast<RetrieveEntry*>(h);
    std::memcpy(ents, T.ents.data(), T.ents.size() * sizeof(RetrieveEntry));
    for (size_t i = 0; i < T.ents.size(); ++i) {
      ents[i].L.kin = base + T.kin_off[i];
      if (T.out_off[i] >= 0) ents[i].out = base + T.out_off[i];
    }
    AnchorEntry* anch = reinterpret_cast<AnchorEntry*>(h + T.ents.size() * sizeof(RetrieveEntry));
    std::memcpy(anch, T.anchors.data(), T.anchors.size() * sizeof(AnchorEntry));
    for (size_t i = 0; i < T.anchors.size(); ++i)
      if (T.anch_off[i] >= 0) anch[i].out = base + T.anch_off[i];
    CoarseArgs* co = reinterpret_cast<CoarseArgs*>(h + eb);
    if (!T.coarse.empty()) std::memcpy(co, T.coarse.data(), T.coarse.size() * sizeof(CoarseArgs));
    for (size_t i = 0; i < T.coarse.size(); ++i)
      if (T.coarse_off[i] >= 0) co[i].out = base + T.coarse_off[i];
  });
  if (rc) return rc;
  if (!pooled) CU(cudaStreamSynchronize(st));
  return IPC_OK;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace

// ===========================================================================
// C ABI
// Little-endian reads of the container.
uint32_t get32(const uint8_t* p) {
  uint32_t v = 0;
  for (int i = 0; i < 4; ++i) v |= uint32_t(p[i]) << (8 * i);
  return v;
}
uint64_t get64(const uint8_t* p) {
  uint64_t v = 0;
  for (int i = 0; i < 8; ++i) v |= uint64_t(p[i]) << (8 * i);
  return v;
}

// Reads the container header, the stage table and the plane-size table into
// the host fields of f (geometry, statistics). On success *pos is the offset
// of the outlier lists, nout[t] the outliers of stage t and size[32 t + k]
// the stream bytes of plane k of stage t.
int parse_head(const uint8_t* p, uint64_t len, ipc_field* f, uint64_t* pos_out,
               std::vector<uint64_t>* nout, std::vector<uint64_t>* size, const char** why) {
  uint64_t pos = 0;
  bool ok = true;
  auto need = [&](uint64_t k) {
    if (pos + k > len || pos + k < pos) ok = false;
    return ok;
  };
  auto g32 = [&]() -> uint32_t {
    if (!need(4)) return 0;
    const uint32_t v = get32(p + pos);
    pos += 4;
    return v;
  };
  auto g64 = [&]() -> uint64_t {
    if (!need(8)) return 0;
    const uint64_t v = get64(p + pos);
    pos += 8;
    return v;
  };
  auto gd = [&]() {
    const uint64_t u = g64();
    double d;
    std::memcpy(&d, &u, 8);
    return d;
  };
  if (!p || g32() != kMagic || g32() != kVersion || !ok) {
    *why = "bad magic/version";
    return IPC_ECORRUPT;
  }
  f->dtype = (int)g32();
  f->interp = (int)g32();
  f->bound = (int)g32();
  const int ndim = (int)g32();
  int64_t dims[3];
  for (int e = 0; e < 3; ++e) dims[e] = (int64_t)g64();
  f->eb_mode = (int)g32();
  const int K = (int)g32();
  f->eb_user = gd();
  f->eb = gd();
  f->xmin = gd();
  f->xmax = gd();
  f->xmaxabs = gd();
  f->anchor = gd();
  const uint32_t S = g32();
  g32();
  if (!ok || f->dtype < 0 || f->dtype > 1 || f->interp < 0 || f->interp > 2 || f->bound < 0 ||
      f->bound > 1 || f->eb_mode < 0 || f->eb_mode > 1 || !(f->eb > 0) || !std::isfinite(f->eb)) {
    *why = "bad header fields";
    return IPC_ECORRUPT;
  }
  if (ndim < 1 || ndim > 3 || !build_geo(ndim, dims, f->dtype, &f->g) || f->g.K != K ||
      f->g.stages.size() != S) {
    *why = "bad geometry";
    return IPC_ECORRUPT;
  }
  f->st.assign(S, StageTab{});
  nout->assign(S, 0);
  for (uint32_t t = 0; t < S; ++t) {
    const StageGeo& sg = f->g.stages[t];
    const uint32_t lv = g32(), dm = g32();
    const uint64_t nc = g64();
    f->st[t].H = (int32_t)g32();
    f->st[t].Q = g32();
    (*nout)[t] = g64();
    if (!ok || (int)lv != sg.level || (int)dm != sg.dim3 - (3 - ndim) || nc != sg.ncodes ||
        f->st[t].H < -1 || f->st[t].H > 31 || (*nout)[t] > nc) {
      *why = "bad stage table";
      return IPC_ECORRUPT;
    }
  }
  size->assign(32 * (size_t)S, 0);
  for (uint32_t t = 0; t < S; ++t)
    for (int k = 31; k >= 0; --k) (*size)[32 * t + k] = g64();
  if (!ok) {
    *why = "truncated tables";
    return IPC_ECORRUPT;
  }
  *pos_out = pos;
  return IPC_OK;
}

namespace ipc {
void set_last_error(const char* what) { g_err = what; }
}  // namespace ipc

// ===========================================================================
extern "C" {

const char* ipc_last_error(void) { return g_err.c_str(); }

int ipc_compress(const void* d_in, int dtype, int ndim, const int64_t* dims, int eb_mode,
                 double eb, int interp, int bound, void* stream, ipc_field** out) {
  g_err.clear();
  Nvtx nv_call("ipc compress");
  if (!d_in || !out) return fail(IPC_EINVAL, "null argument");
  if (dtype != IPC_F32 && dtype != IPC_F64) return fail(IPC_EINVAL, "dtype");
  if (interp < IPC_LINEAR || interp > IPC_INTERP_AUTO) return fail(IPC_EINVAL, "interp");
  if (bound != IPC_BOUND_STRICT && bound != IPC_BOUND_PAPER) return fail(IPC_EINVAL, "bound");
  if (eb_mode != IPC_EB_ABS && eb_mode != IPC_EB_REL) return fail(IPC_EINVAL, "eb_mode");
  if (!std::isfinite(eb) || !(eb > 0)) return fail(IPC_EINVAL, "eb must be > 0 and finite");
  ipc_field* f = new (std::nothrow) ipc_field();
  if (!f) return fail(IPC_ENOMEM, "host allocation");
  f->tag = kFieldTag;
  if (!build_geo(ndim, dims, dtype, &f->g)) {
    delete f;
    return fail(IPC_EINVAL, "shape");
  }
  if (interp == IPC_INTERP_AUTO) {
    std::vector<AutoItem> a(1, AutoItem{d_in, dtype, ndim, {1, 1, 1}, eb_mode, bound, eb, -1});
    for (int d = 0; d < ndim; ++d) a[0].dims[d] = dims[d];
    const int rc = resolve_auto(a, (cudaStream_t)stream);
    if (rc) {
      delete f;
      return rc;
    }
    interp = a[0].mode;
  }
  cudaGetDevice(&f->device);
  f->dtype = dtype;
  f->interp = interp;
  f->bound = bound;
  f->eb_mode = eb_mode;
  f->eb_user = eb;
  std::vector<ipc_field*> fs{f};
  std::vector<const void*> ins{d_in};
  int rc = compress_fields(fs, ins, (cudaStream_t)stream);
  if (rc) {
    free_field_device(f);
    f->tag = kDeadTag;
    delete f;
    return rc;
  }
  *out = f;
  return IPC_OK;
}

int ipc_retrieve(ipc_field* f, ipc_target target, void* d_out, void* stream, ipc_view** out) {
  return ipc_retrieve_ex(f, target, d_out, stream, IPC_REFINE_CANONICAL, out);
}

int ipc_retrieve_ex(ipc_field* f, ipc_target target, void* d_out, void* stream, int refine_mode,
                    ipc_view** out) {
  g_err.clear();
  Nvtx nv_call("ipc retrieve");
  if (!f || f->tag != kFieldTag || !d_out) return fail(IPC_EINVAL, "null or invalid argument");
  if (refine_mode < IPC_REFINE_CANONICAL || refine_mode > IPC_REFINE_AUTO)
    return fail(IPC_EINVAL, "unknown refine mode");
  refine_mode = ipc_internal_refine_mode(f, refine_mode);
  DeviceGuard dg(f->device);
  std::vector<int> b;
  uint64_t bytes = 0;
  double bound = 0;
  uint64_t rparts[2] = {0, 0};
  int rc = select(f, target, nullptr, &b, &bytes, &bound, rparts);
  if (rc) return rc;
  ipc_view* v = nullptr;
  if (out) {
    v = new (std::nothrow) ipc_view();
    if (!v) return fail(IPC_ENOMEM, "host allocation");
    v->tag = kViewTag;
    v->f = f;
    v->mode = refine_mode;
    v->state_device = f->device;
  }
  // the incremental form records its state during this reconstruction
  const bool record = v && refine_mode == IPC_REFINE_INCREMENTAL;
  if (record) {
    v->state_words = std::max<uint64_t>(state_words(f->g, &v->state_off), 2);
    if (cudaMalloc((void**)&v->d_state, 2 * v->state_words * 4) != cudaSuccess) {
      cudaGetLastError();
      delete v;
      return fail(IPC_ENOMEM, "device allocation of the view state");
    }
  }
  rc = reconstruct(f, b, d_out, (cudaStream_t)stream, record ? v->d_state : nullptr,
                   record ? &v->state_off : nullptr);
  if (rc) {
    if (v && v->d_state) cudaFree(v->d_state);
    delete v;
    return rc;
  }
  if (out) {
    v->b = b;
    v->bytes = bytes;
    v->bound = bound;
    v->racc = rparts[0];
    v->state_valid = record;
    *out = v;
  }
  return IPC_OK;
}

int ipc_autotune_retrieve(ipc_field* f, ipc_target target, void* d_out, void* stream, int reps,
                          int* nshapes) {
  g_err.clear();
  if (!f || f->tag != kFieldTag || !d_out) return fail(IPC_EINVAL, "null or invalid argument");
  if (reps < 1 || reps > 100) return fail(IPC_EINVAL, "reps must be 1..100");
  DeviceGuard dg(f->device);
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<int> b;
  uint64_t bytes = 0;
  double bound = 0;
  int rc = select(f, target, nullptr, &b, &bytes, &bound);
  if (rc) return rc;
  const Geo& g = f->g;
  const size_t esz = f->dtype == 0 ? 4 : 8;
  std::vector<uint64_t> off;
  uint8_t* scr = nullptr;
  if (g.K > 0 && (rc = dalloc((void**)&scr, ladder(g, esz, &off), st))) return rc;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  struct Guard {
    uint8_t* p;
    cudaStream_t s;
    cudaEvent_t& a;
    cudaEvent_t& b;
    ~Guard() {
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
      if (p) cudaFreeAsync(p, s);
    }
  } guard{scr, st, e0, e1};
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  CU(launch_set_anchor(f->dtype, g.K > 0 ? (void*)(scr + off[g.K + 1]) : d_out, f->anchor, st));
  const double twoeb = bin_width(f);
  // level l's launch with shape sh (its inputs: level l + 1's output)
  std::vector<LevelArgs> La(g.K + 2);
  std::vector<int> W(g.K + 2, 0);
  std::vector<RetrieveShape> chosen(g.K + 2);
  for (int l = g.K; l >= 1; --l) {
    La[l] = level_args(f, l);
    retrieve_layout(&La[l], scr + off[l + 1]);
    retrieve_planes(f, l, b[l - 1], &La[l]);
    La[l].stream_out = l == 1;
    W[l] = level_w16(f, l, b[l - 1]) ? 1 : 0;
  }
  auto run = [&](int l, RetrieveShape sh) {
    void* o = l == 1 ? d_out : (void*)(scr + off[l]);
    if (!sh.ns) sh.ns = retrieve_subtiles(La[l].M[2], W[l]);
    LevelArgs Lt = La[l];
    retrieve_tiling(&Lt, f->dtype, W[l], sh.ns);
    return launch_level_retrieve(f->dtype, Lt, o, twoeb, b[l - 1], f->d_cap, f->d_bm,
                                 f->d_oidx, f->d_oval, W[l], sh, st);
  };
  for (int l = g.K; l >= 1; --l) {
    // Each shape is timed `reps` times, each time right after level l + 1
    // ran again (as in a reconstruction, level l reads what level l + 1 just
    // wrote); the median decides. A shape replaces the default only when it
    // is faster by more than 3 %. Every shape gives the same values, so the
    // level's output is right after any of the launches.
    std::vector<float> t(reps);
    auto timed = [&](RetrieveShape sh, float* med) -> int {
      CU(run(l, sh));  // warm-up
      for (int r = 0; r < reps; ++r) {
        if (l < g.K) CU(run(l + 1, chosen[l + 1]));
        CU(cudaEventRecord(e0, st));
        CU(run(l, sh));
        CU(cudaEventRecord(e1, st));
        CU(cudaEventSynchronize(e1));
        CU(cudaEventElapsedTime(&t[r], e0, e1));
      }
      std::sort(t.begin(), t.end());
      *med = t[reps / 2];
      return IPC_OK;
    };
    float def_ms = 0, best_ms = 0;
    if ((rc = timed(RetrieveShape{}, &def_ms))) return rc;
    RetrieveShape best{};
    best_ms = def_ms;
    for (int ns : {1, 2, 4}) {
      if (!retrieve_ns_ok(La[l].M[2], ns)) continue;
      for (int psm = 1; psm <= retrieve_max_per_sm(f->dtype, W[l], ns); ++psm) {
        float ms = 0;
        if ((rc = timed(RetrieveShape{ns, psm}, &ms))) return rc;
        if (ms < best_ms && ms < 0.97f * def_ms) {
          best = RetrieveShape{ns, psm};
          best_ms = ms;
        }
      }
    }
    chosen[l] = best;
    std::lock_guard<std::mutex> lk(g_shape_mu);
    g_shapes[shape_key(f->dtype, W[l], La[l])] = best;
  }
  CU(cudaStreamSynchronize(st));
  if (nshapes) {
    std::lock_guard<std::mutex> lk(g_shape_mu);
    *nshapes = (int)g_shapes.size();
  }
  return IPC_OK;
}

int ipc_autotune_clear(void) {
  std::lock_guard<std::mutex> lk(g_shape_mu);
  g_shapes.clear();
  return IPC_OK;
}

int ipc_autotune_entry(int i, int* dtype, int* w16, int64_t* M, int* ns, int* per_sm) {
  g_err.clear();
  std::lock_guard<std::mutex> lk(g_shape_mu);
  if (i < 0 || i >= (int)g_shapes.size()) return fail(IPC_EINVAL, "no such entry");
  auto it = g_shapes.begin();
  std::advance(it, i);
  if (dtype) *dtype = it->first.dtype;
  if (w16) *w16 = it->first.w16;
  if (M) {
    M[0] = it->first.M0;
    M[1] = it->first.M1;
    M[2] = it->first.M2;
  }
  if (ns) *ns = it->second.ns;
  if (per_sm) *per_sm = it->second.per_sm;
  return IPC_OK;
}

int ipc_error_metrics_host(const void* x, const void* y, int dtype, uint64_t n,
                           ipc_error_metrics* out) {
  g_err.clear();
  if (!out || (n && (!x || !y))) return fail(IPC_EINVAL, "null argument");
  if (dtype != IPC_F32 && dtype != IPC_F64) return fail(IPC_EINVAL, "dtype");
  struct Part {
    double maxe = 0, sse = 0, mn = 0, mx = 0;
    uint64_t fin = 0, bad = 0, cnt = 0;  // cnt: pairs in the sums
  };
  constexpr uint64_t kChunk = uint64_t(1) << 16;
  const uint64_t nc = (n + kChunk - 1) / kChunk;
  std::vector<Part> part(nc);
  auto chunk = [&](int c) {
    Part p;
    const uint64_t a = (uint64_t)c * kChunk, b = std::min(n, a + kChunk);
    for (uint64_t i = a; i < b; ++i) {
      const double xv = dtype == IPC_F32 ? (double)((const float*)x)[i] : ((const double*)x)[i];
      const double yv = dtype == IPC_F32 ? (double)((const float*)y)[i] : ((const double*)y)[i];
      if (!std::isfinite(xv)) {
        const bool same = std::isnan(xv) ? std::isnan(yv) : yv == xv;
        if (!same) ++p.bad;
        continue;
      }
      if (p.fin == 0) p.mn = p.mx = xv;
      p.mn = std::min(p.mn, xv);
      p.mx = std::max(p.mx, xv);
      ++p.fin;
      if (!std::isfinite(yv)) {
        ++p.bad;
        p.maxe = HUGE_VAL;
        continue;
      }
      const double d = xv - yv;
      p.maxe = std::max(p.maxe, std::fabs(d));
      p.sse += d * d;
      ++p.cnt;
    }
    part[c] = p;
  };
  if (nc >= 8)
    HostPool::get().run((int)nc, chunk);
  else
    for (uint64_t c = 0; c < nc; ++c) chunk((int)c);
  Part t;
  for (const Part& p : part) {  // in chunk order
    if (p.fin) {
      t.mn = t.fin ? std::min(t.mn, p.mn) : p.mn;
      t.mx = t.fin ? std::max(t.mx, p.mx) : p.mx;
    }
    t.fin += p.fin;
    t.bad += p.bad;
    t.cnt += p.cnt;
    t.maxe = std::max(t.maxe, p.maxe);
    t.sse += p.sse;
  }
  out->finite = t.fin;
  out->nonfinite_mismatch = t.bad;
  out->max_abs_err = t.maxe;
  out->range = t.fin ? t.mx - t.mn : 0.0;
  out->mse = t.cnt ? t.sse / (double)t.cnt : 0.0;
  if (out->mse == 0.0) out->psnr = HUGE_VAL;
  else if (out->range == 0.0) out->psnr = -HUGE_VAL;
  else out->psnr = 20.0 * std::log10(out->range / std::sqrt(out->mse));
  return IPC_OK;
}

int ipc_autotune_set(int dtype, int w16, const int64_t* M, int ns, int per_sm) {
  g_err.clear();
  if (!M) return fail(IPC_EINVAL, "null argument");
  if ((dtype != IPC_F32 && dtype != IPC_F64) || (w16 != 0 && w16 != 1))
    return fail(IPC_EINVAL, "dtype or code width");
  if (M[0] < 1 || M[1] < 1 || M[2] < 1) return fail(IPC_EINVAL, "extents");
  const bool dflt = ns == 0 && per_sm == 0;
  if (!dflt && ((ns != 1 && ns != 2 && ns != 4) || !retrieve_ns_ok(M[2], ns) || per_sm < 1 ||
                per_sm > retrieve_max_per_sm(dtype, w16, ns)))
    return fail(IPC_EINVAL, "not a shape the tuner records");
  std::lock_guard<std::mutex> lk(g_shape_mu);
  g_shapes[ShapeKey{dtype, w16, M[0], M[1], M[2]}] = RetrieveShape{ns, per_sm};
  return IPC_OK;
}

int ipc_refine(ipc_view* v, ipc_target target, void* d_out, void* stream) {
  g_err.clear();
  Nvtx nv_call("ipc refine");
  if (!v || v->tag != kViewTag || !d_out) return fail(IPC_EINVAL, "null or invalid argument");
  ipc_field* f = v->f;
  DeviceGuard dg(f->device);
  std::vector<int> b;
  uint64_t bytes = 0;
  double bound = 0;
  uint64_t rparts[2] = {0, 0};
  int rc = select(f, target, &v->b, &b, &bytes, &bound, rparts);
  if (rc == IPC_EBUDGET && target.kind == IPC_TARGET_BITRATE) {
    g_err.clear();
    return IPC_OK;
  }
  if (rc) return rc;
  if (b == v->b) return IPC_OK;
  const cudaStream_t st = (cudaStream_t)stream;
  if (v->mode == IPC_REFINE_INCREMENTAL && v->state_valid) {
    uint64_t racc = 0;
    const double Gd =
        incremental_bound(f->sel, v->b, v->bound, v->racc, b, bound, rparts, &racc);
    double E = target.value;
    if (f->eb_mode == IPC_EB_REL && f->xmax - f->xmin > 0) E = target.value * (f->xmax - f->xmin);
    if (target.kind == IPC_TARGET_BITRATE || Gd <= E) {
      uint64_t sb = 0;
      uint32_t* cur = v->d_state + (uint64_t)v->state_cur * v->state_words;
      uint32_t* nxt = v->d_state + (uint64_t)(1 - v->state_cur) * v->state_words;
      rc = reconstruct_increment(f, v->b, b, d_out, cur, nxt, v->state_off, st, &sb);
      if (rc) {
        v->state_valid = false;  // d_out may be half updated
        return rc;
      }
      v->state_cur = 1 - v->state_cur;
      v->b = b;
      v->bytes = bytes;
      v->bound = Gd;
      v->racc = racc;
      v->last_incremental = 1;
      v->last_stream_bytes = sb;
      return IPC_OK;
    }
  }
  // canonical form (an incremental view records its state on the way)
  const bool record = v->mode == IPC_REFINE_INCREMENTAL;
  if (record && !v->d_state) {
    v->state_words = std::max<uint64_t>(state_words(f->g, &v->state_off), 2);
    if (cudaMalloc((void**)&v->d_state, 2 * v->state_words * 4) != cudaSuccess) {
      cudaGetLastError();
      return fail(IPC_ENOMEM, "device allocation of the view state");
    }
  }
  rc = reconstruct(f, b, d_out, st,
                   record ? v->d_state + (uint64_t)v->state_cur * v->state_words : nullptr,
                   record ? &v->state_off : nullptr);
  if (rc) {
    v->state_valid = false;
    return rc;
  }
  v->b = b;
  v->bytes = bytes;
  v->bound = bound;
  v->racc = rparts[0];
  v->state_valid = record;
  v->last_incremental = 0;
  v->last_stream_bytes = bytes - f->mandatory;
  return IPC_OK;
}

int ipc_view_set_refine_mode(ipc_view* v, int refine_mode) {
  g_err.clear();
  if (!v || v->tag != kViewTag) return fail(IPC_EINVAL, "null or invalid view");
  if (refine_mode < IPC_REFINE_CANONICAL || refine_mode > IPC_REFINE_AUTO)
    return fail(IPC_EINVAL, "unknown refine mode");
  refine_mode = ipc_internal_refine_mode(v->f, refine_mode);
  if (refine_mode != v->mode) v->state_valid = false;
  v->mode = refine_mode;
  return IPC_OK;
}

int ipc_refine_info(const ipc_view* v, int* incremental, uint64_t* stream_bytes) {
  g_err.clear();
  if (!v || v->tag != kViewTag) return fail(IPC_EINVAL, "null or invalid view");
  if (incremental) *incremental = v->last_incremental;
  if (stream_bytes) *stream_bytes = v->last_stream_bytes;
  return IPC_OK;
}

int ipc_free(void* handle) {
  if (!handle) return IPC_OK;
  uint32_t tag;
  std::memcpy(&tag, handle, 4);
  if (tag == kFieldTag) {
    ipc_field* f = (ipc_field*)handle;
    DeviceGuard dg(f->device);
    free_field_device(f);
    f->tag = kDeadTag;
    delete f;
    return IPC_OK;
  }
  if (tag == kViewTag) {
    ipc_view* v = (ipc_view*)handle;
    if (v->d_state) {
      DeviceGuard dg(v->state_device);
      cudaFree(v->d_state);
    }
    v->tag = kDeadTag;
    delete v;
    return IPC_OK;
  }
  if (tag == kPlanTag) {
    ipc_plan* p = (ipc_plan*)handle;
    DeviceGuard dg(p->device);
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->d_tab) cudaFree(p->d_tab);
    p->tag = kDeadTag;
    delete p;
    return IPC_OK;
  }
  return fail(IPC_EINVAL, "not a live ipc handle");
}

int ipc_select_container(const void* buf, uint64_t len, ipc_target target, int* b_per_level,
                         int* nlevels, uint64_t* bytes, double* guaranteed_bound) {
  g_err.clear();
  if (!buf) return fail(IPC_EINVAL, "null argument");
  ipc_field f{};
  uint64_t pos = 0;
  std::vector<uint64_t> nout, size;
  const char* why = "";
  if (parse_head((const uint8_t*)buf, len, &f, &pos, &nout, &size, &why))
    return fail(IPC_ECORRUPT, why);
  uint64_t mand = pos;  // the outlier lists count, whether present or not
  for (size_t t = 0; t < f.st.size(); ++t) {
    mand += 16 * nout[t];
    const uint64_t W = f.g.stages[t].words, nbm = (W + 31) / 32;
    for (int k = 0; k < 32; ++k) {
      const uint64_t z = size[32 * t + k];
      // a stream size is 4 (empty), 4 + 4 W (dense) or 4 + 4 (nbm + nnz)
      // with nnz >= 1 and nbm + nnz < W (sparse)
      bool valid = z == 4 || z == 4 + 4 * W;
      if (!valid && z > 4 && z % 4 == 0 && (z - 4) / 4 > nbm) {
        const uint64_t nnz = (z - 4) / 4 - nbm;
        valid = stream_bytes(nnz, W) == z;
      }
      if (!valid) return fail(IPC_ECORRUPT, "bad plane size");
      f.st[t].size[k] = z;
    }
  }
  f.mandatory = mand;
  std::vector<int> b;
  uint64_t y = 0;
  double bound = 0;
  SelInput in = sel_input(&f);
  prepare_selection(&in);  // the tables as a device-resident field keeps them
  const int rc = select_planes(in, target.kind, target.value, nullptr, &b, &y, &bound, &why);
  if (rc) return fail(rc, why);
  if (nlevels) *nlevels = (int)b.size();
  if (b_per_level)
    for (size_t i = 0; i < b.size(); ++i) b_per_level[i] = b[i];
  if (bytes) *bytes = y;
  if (guaranteed_bound) *guaranteed_bound = bound;
  return IPC_OK;
}

int ipc_selection(const ipc_view* v, int* b_per_level, int* nlevels, uint64_t* bytes,
                  double* guaranteed_bound) {
  if (!v || v->tag != kViewTag) return fail(IPC_EINVAL, "invalid view");
  if (nlevels) *nlevels = (int)v->b.size();
  if (b_per_level)
    for (size_t i = 0; i < v->b.size(); ++i) b_per_level[i] = v->b[i];
  if (bytes) *bytes = v->bytes;
  if (guaranteed_bound) *guaranteed_bound = v->bound;
  return IPC_OK;
}

int ipc_compressed_size(const ipc_field* f, uint64_t* bytes) {
  if (!f || f->tag != kFieldTag || !bytes) return fail(IPC_EINVAL, "invalid argument");
  *bytes = f->mandatory + f->stream_bytes;
  return IPC_OK;
}

int ipc_export(const ipc_field* f, void* host_buf, uint64_t* len) {
  if (!f || f->tag != kFieldTag || !len) return fail(IPC_EINVAL, "invalid argument");
  if (!f->rb.empty()) return fail(IPC_EINVAL, "the field holds only some of its planes");
  const uint64_t total = f->mandatory + f->stream_bytes;
  if (!host_buf) {
    *len = total;
    return IPC_OK;
  }
  if (*len < total) return fail(IPC_EINVAL, "buffer too small");
  DeviceGuard dg(f->device);
  std::vector<uint8_t> h = header_bytes(f);
  std::memcpy(host_buf, h.data(), h.size());
  const Geo& g = f->g;
  if (f->stream_bytes) {
    cudaStream_t st = nullptr;
    CU(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    uint32_t *blob = nullptr, *tmp = nullptr;
    uint64_t tw = 0;
    for (auto& sg : g.stages) tw = std::max<uint64_t>(tw, 2 * 32 * ((sg.words + 31) / 32));
    int rc = IPC_OK;
    if ((rc = dalloc((void**)&blob, f->stream_bytes, st)) || (rc = dalloc((void**)&tmp, tw * 4, st))) {
      dfree(blob);
      cudaStreamDestroy(st);
      return rc;
    }
    cudaError_t e = cudaSuccess;
    for (size_t t = 0; t < g.stages.size() && e == cudaSuccess; ++t) {
      const long ph = prof_begin(IPC_KERNEL_PACK, st);
      e = launch_pack(stage_args(g.stages[t]), f->desc[t], f->d_cap, f->d_bm, tmp, blob, st);
      prof_end(ph, st, 0);
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync((uint8_t*)host_buf + h.size(), blob, f->stream_bytes,
                          cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFreeAsync(blob, st);
    cudaFreeAsync(tmp, st);
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    if (e != cudaSuccess) return cuda_fail(e, "export");
  }
  *len = total;
  return IPC_OK;
}

}  // extern "C"

namespace {

// nnz of a stream from its size alone (a plane whose stream is not loaded):
// exact for empty and sparse streams; a dense one is known only to have
// nonzero words (W stands in until the stream is loaded).
uint64_t nnz_from_size(uint64_t z, uint64_t W) {
  const uint64_t nbm = (W + 31) / 32;
  if (z == 4) return 0;
  if (z == 4 + 4 * W) return W;
  return (z - 4) / 4 - nbm;
}

// Uploads `len` bytes of streams (stage order, planes descending within a
// stage, the planes of stage t at level l being [lo_l, hi_l)) and unpacks
// them into the field's segmented layout; `nzs` holds their nnz (read from
// the streams by the caller). Synchronises.
int unpack_streams(ipc_field* f, const uint8_t* p, uint64_t len, const std::vector<int>& lo,
                   const std::vector<int>& hi, const std::vector<uint32_t>& nzs, cudaStream_t st) {
  uint32_t *blob = nullptr, *tmp = nullptr;
  unsigned int* flags = nullptr;  // [0] corruption flag
  uint64_t tw = 0;
  for (auto& sg : f->g.stages) tw = std::max<uint64_t>(tw, 2 * 32 * ((sg.words + 31) / 32));
  int rc;
  if ((rc = dalloc((void**)&blob, std::max<uint64_t>(len, 4), st)) ||
      (rc = dalloc((void**)&tmp, tw * 4, st)) || (rc = dalloc((void**)&flags, 4, st))) {
    dfree(blob);
    dfree(tmp);
    return rc;
  }
  cudaError_t e = cudaSuccess;
  if (len) e = cudaMemcpyAsync(blob, p, len, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(flags, 0, 4, st);
  uint64_t word = 0;  // word offset of the next stream in the blob
  size_t j = 0;
  const uint32_t S = (uint32_t)f->g.stages.size();
  for (uint32_t t = 0; t < S && e == cudaSuccess; ++t) {
    const int l = f->g.stages[t].level;
    const uint64_t W = f->g.stages[t].words;
    StageDescs d = f->desc[t];
    uint32_t kmask = 0;
    for (int k = 31; k >= 0; --k) {
      PlaneDesc& pd = d.p[k];
      if (k >= lo[l - 1] && k < hi[l - 1]) {
        pd.nnz = nzs[j++];
        pd.mode = stream_mode(pd.nnz, W);
        pd.pk_off = word;
        word += stream_bytes(pd.nnz, W) / 4;
        kmask |= 1u << k;
      } else {
        pd.mode = 0;  // not in this upload: left as it is
      }
    }
    if (!kmask) continue;
    const long ph = prof_begin(IPC_KERNEL_UNPACK, st);
    e = launch_unpack(stage_args(f->g.stages[t]), d, f->g.stages[t].nseg, blob, tmp, f->d_cap,
                      f->d_bm, flags, kmask, st);
    prof_end(ph, st, 0);
  }
  unsigned int hbad = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, flags, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(blob, st);
  cudaFreeAsync(tmp, st);
  cudaFreeAsync(flags, st);
  if (e != cudaSuccess) return cuda_fail(e, "stream upload");
  if (hbad) return fail(IPC_ECORRUPT, "stream contents disagree with their nnz / bitmap");
  return IPC_OK;
}

// A device field from container bytes: the leading tables, then for each
// stage the streams of its planes k >= res_l (every plane when res is null).
int import_core(const uint8_t* p, uint64_t len, const int* res, int nres, cudaStream_t st,
                ipc_field** out) {
  ipc_field* f = new (std::nothrow) ipc_field();
  if (!f) return fail(IPC_ENOMEM, "host allocation");
  f->tag = kFieldTag;
  cudaGetDevice(&f->device);
  keep_pool(f->device);
  auto drop = [&](int code, const char* why) {
    free_field_device(f);
    f->tag = kDeadTag;
    delete f;
    return code == IPC_ECUDA || !why ? code : fail(code, why);
  };
  uint64_t pos = 0;
  std::vector<uint64_t> nout, size;
  const char* why = "";
  if (parse_head(p, len, f, &pos, &nout, &size, &why)) return drop(IPC_ECORRUPT, why);
  const int K = f->g.K;
  std::vector<int> lo(K, 0), hi(K, 32);
  if (res) {
    if (nres != K) return drop(IPC_EINVAL, "resident planes: one entry per level");
    for (int l = 0; l < K; ++l) {
      if (res[l] < 0 || res[l] > 32) return drop(IPC_EINVAL, "resident planes out of range");
      lo[l] = res[l];
    }
  }
  const uint32_t S = (uint32_t)f->g.stages.size();
  for (uint32_t t = 0; t < S; ++t) {
    if (pos + nout[t] * 16 > len) return drop(IPC_ECORRUPT, "truncated outliers");
    for (uint64_t i = 0; i < nout[t]; ++i) {
      const uint64_t idx = get64(p + pos);
      double v;
      const uint64_t vb = get64(p + pos + 8);
      std::memcpy(&v, &vb, 8);
      pos += 16;
      if (idx >= f->g.stages[t].ncodes || (i && idx <= f->st[t].out_idx.back()))
        return drop(IPC_ECORRUPT, "bad outlier list");
      f->st[t].out_idx.push_back(idx);
      f->st[t].out_val.push_back(v);
    }
  }
  const uint64_t mand = pos;
  uint64_t spos = pos;
  std::vector<uint32_t> nzs;
  for (uint32_t t = 0; t < S; ++t) {
    const uint64_t W = f->g.stages[t].words;
    const int l = f->g.stages[t].level;
    for (int k = 31; k >= 0; --k) {
      const uint64_t z = size[32 * t + k];
      if (k < lo[l - 1]) {  // not loaded: what the size tells
        if (z < 4 || stream_bytes(nnz_from_size(z, W), W) != z) return drop(IPC_ECORRUPT, "bad stream size");
        f->st[t].nnz[k] = nnz_from_size(z, W);
        continue;
      }
      if (spos + 4 > len) return drop(IPC_ECORRUPT, "truncated streams");
      uint32_t nz = 0;
      for (int i = 0; i < 4; ++i) nz |= uint32_t(p[spos + i]) << (8 * i);
      if (nz > W || z != stream_bytes(nz, W)) return drop(IPC_ECORRUPT, "bad stream size");
      f->st[t].nnz[k] = nz;
      nzs.push_back(nz);
      spos += z;
      if (spos > len) return drop(IPC_ECORRUPT, "truncated streams");
    }
  }
  if (spos != len) return drop(IPC_ECORRUPT, "trailing bytes");
  DeviceGuard dg(f->device);
  int rc = plan_field(f, st);
  if (rc) return drop(rc, "allocation");
  rc = finish_field(f, st);
  if (rc) return drop(rc, "allocation");
  if (f->mandatory != mand) return drop(IPC_ECORRUPT, "table size mismatch");
  if (res) {
    bool any = false;
    for (int l = 0; l < K; ++l) any |= lo[l] > 0;
    if (any) {
      f->rb = lo;
      f->sel.lower = lo;
    }
  }
  rc = unpack_streams(f, p + mand, spos - mand, lo, hi, nzs, st);
  if (rc) return drop(rc, nullptr);
  *out = f;
  return IPC_OK;
}

// The streams of planes [lo_l, hi_l) of every stage: byte ranges of the
// container (stage order, planes descending: each stage's span is one run).
void stream_ranges(const ipc_field& f, uint64_t mand, const std::vector<uint64_t>& size,
                   const int* lo, const int* hi, std::vector<std::pair<uint64_t, uint64_t>>* r) {
  uint64_t pos = mand;
  for (size_t t = 0; t < f.g.stages.size(); ++t) {
    const int l = f.g.stages[t].level;
    uint64_t a = pos, b = pos;
    for (int k = 31; k >= 0; --k) {
      const uint64_t z = size[32 * t + k];
      if (k >= hi[l - 1]) a += z;
      if (k >= lo[l - 1]) b += z;
      pos += z;
    }
    if (b > a) {
      if (!r->empty() && r->back().first + r->back().second == a) r->back().second += b - a;
      else r->push_back({a, b - a});
    }
  }
}

}  // namespace

extern "C" {

int ipc_import(const void* host_buf, uint64_t len, void* stream, ipc_field** out) {
  g_err.clear();
  Nvtx nv_call("ipc import");
  if (!out || (!host_buf && len)) return fail(IPC_EINVAL, "null argument");
  if (len >= 4 && get32le((const uint8_t*)host_buf) == 0x5A435049u) {  // coded form: decode first
    uint64_t raw = 0;
    int rc = ipc_decode_container(host_buf, len, nullptr, &raw, 0);
    if (rc) return rc;
    std::vector<uint8_t> dec;
    try {
      dec.resize(raw);
    } catch (...) {
      return fail(IPC_ENOMEM, "host allocation");
    }
    if ((rc = ipc_decode_container(host_buf, len, dec.data(), &raw, 0))) return rc;
    if (raw >= 4 && get32le(dec.data()) == 0x5A435049u) return fail(IPC_ECORRUPT, "nested coding");
    return ipc_import(dec.data(), raw, stream, out);
  }
  return import_core((const uint8_t*)host_buf, len, nullptr, 0, (cudaStream_t)stream, out);
}

int ipc_container_ranges(const void* head, uint64_t head_len, const int* b_new, const int* b_old,
                         int nlevels, uint64_t* ranges, int* nranges) {
  g_err.clear();
  if (!head || !b_new || !nranges) return fail(IPC_EINVAL, "null argument");
  ipc_field f{};
  uint64_t pos = 0;
  std::vector<uint64_t> nout, size;
  const char* why = "";
  if (parse_head((const uint8_t*)head, head_len, &f, &pos, &nout, &size, &why))
    return fail(IPC_ECORRUPT, why);
  const int K = f.g.K;
  if (nlevels != K) return fail(IPC_EINVAL, "one entry per level");
  std::vector<int> hi(K, 32);
  for (int l = 0; l < K; ++l) {
    if (b_old) hi[l] = b_old[l];
    if (b_new[l] < 0 || hi[l] > 32 || b_new[l] > hi[l]) return fail(IPC_EINVAL, "plane bounds");
  }
  uint64_t mand = pos;
  for (uint64_t n : nout) mand += 16 * n;
  std::vector<std::pair<uint64_t, uint64_t>> r;
  if (!b_old) r.push_back({0, mand});
  stream_ranges(f, mand, size, b_new, hi.data(), &r);
  const int cap = *nranges;
  *nranges = (int)r.size();
  if (!ranges) return IPC_OK;
  if ((int)r.size() > cap) return fail(IPC_EINVAL, "range capacity too small");
  for (size_t i = 0; i < r.size(); ++i) {
    ranges[2 * i] = r[i].first;
    ranges[2 * i + 1] = r[i].second;
  }
  return IPC_OK;
}

int ipc_import_partial(const void* parts, uint64_t len, const int* b_per_level, int nlevels,
                       void* stream, ipc_field** out) {
  g_err.clear();
  Nvtx nv_call("ipc import partial");
  if (!out || !parts || !b_per_level) return fail(IPC_EINVAL, "null argument");
  return import_core((const uint8_t*)parts, len, b_per_level, nlevels, (cudaStream_t)stream, out);
}

int ipc_field_load_planes(ipc_field* f, const void* parts, uint64_t len, const int* b_new,
                          int nlevels, void* stream) {
  g_err.clear();
  Nvtx nv_call("ipc load planes");
  if (!f || f->tag != kFieldTag || !b_new || (!parts && len)) return fail(IPC_EINVAL, "invalid argument");
  const int K = f->g.K;
  if (nlevels != K) return fail(IPC_EINVAL, "one entry per level");
  if (f->rb.empty()) return len ? fail(IPC_EINVAL, "the field holds every plane") : IPC_OK;
  std::vector<int> lo(K), hi = f->rb;
  for (int l = 0; l < K; ++l) {
    if (b_new[l] < 0 || b_new[l] > f->rb[l]) return fail(IPC_EINVAL, "plane bounds");
    lo[l] = b_new[l];
  }
  const uint8_t* p = (const uint8_t*)parts;
  uint64_t pos = 0;
  std::vector<uint32_t> nzs;
  std::vector<std::pair<int, int>> at;  // (stage, plane) of each stream
  for (size_t t = 0; t < f->g.stages.size(); ++t) {
    const int l = f->g.stages[t].level;
    const uint64_t W = f->g.stages[t].words;
    for (int k = hi[l - 1] - 1; k >= lo[l - 1]; --k) {
      const uint64_t z = f->st[t].size[k];
      if (pos + 4 > len) return fail(IPC_ECORRUPT, "truncated streams");
      uint32_t nz = 0;
      for (int i = 0; i < 4; ++i) nz |= uint32_t(p[pos + i]) << (8 * i);
      if (nz > W || z != stream_bytes(nz, W)) return fail(IPC_ECORRUPT, "bad stream size");
      nzs.push_back(nz);
      at.push_back({(int)t, k});
      pos += z;
      if (pos > len) return fail(IPC_ECORRUPT, "truncated streams");
    }
  }
  if (pos != len) return fail(IPC_ECORRUPT, "trailing bytes");
  DeviceGuard dg(f->device);
  const int rc = unpack_streams(f, p, len, lo, hi, nzs, (cudaStream_t)stream);
  if (rc) return rc;
  for (size_t i = 0; i < at.size(); ++i) {
    const int t = at[i].first, k = at[i].second;
    f->st[t].nnz[k] = nzs[i];
    f->desc[t].p[k].nnz = nzs[i];
  }
  bool any = false;
  for (int l = 0; l < K; ++l) any |= lo[l] > 0;
  f->rb = any ? lo : std::vector<int>();
  f->sel.lower = f->rb;
  return IPC_OK;
}

int ipc_field_resident(const ipc_field* f, int* b_per_level, int* nlevels) {
  if (!f || f->tag != kFieldTag) return fail(IPC_EINVAL, "invalid field");
  if (nlevels) *nlevels = f->g.K;
  if (b_per_level)
    for (int l = 0; l < f->g.K; ++l) b_per_level[l] = f->rb.empty() ? 0 : f->rb[l];
  return IPC_OK;
}

}  // extern "C"

// ---- hooks of the serving loop (ipc_serve.cu) ---------------------------------
int ipc_internal_refine_mode(const ipc_field* f, int mode) {
  if (mode != IPC_REFINE_AUTO) return mode;
  return f->dtype == IPC_F64 ? IPC_REFINE_INCREMENTAL : IPC_REFINE_CANONICAL;
}

int ipc_internal_select(ipc_field* f, ipc_target tg, const std::vector<int>* upper,
                        std::vector<int>* b, uint64_t* bytes, double* bound, uint64_t* rparts) {
  return select(f, tg, upper, b, bytes, bound, rparts);
}

ipc_view* ipc_internal_view_make(ipc_field* f, const std::vector<int>& b, uint64_t bytes,
                                 double bound, uint64_t racc, int mode) {
  ipc_view* v = new (std::nothrow) ipc_view();
  if (!v) return nullptr;
  v->tag = kViewTag;
  v->f = f;
  v->b = b;
  v->bytes = bytes;
  v->bound = bound;
  v->racc = racc;
  v->mode = mode;
  v->state_device = f->device;
  return v;
}

void ipc_internal_view_selection(const ipc_view* v, std::vector<int>* b, uint64_t* bytes,
                                 double* bound) {
  *b = v->b;
  *bytes = v->bytes;
  *bound = v->bound;
}

void ipc_internal_field_shape(const ipc_field* f, uint64_t* n, int* dtype) {
  *n = f->g.n;
  *dtype = f->dtype;
}

int ipc_internal_reconstruct_each(const std::vector<ipc_field*>& fs,
                                  const std::vector<std::vector<int>>& bs,
                                  const std::vector<void*>& outs, cudaStream_t st) {
  for (size_t i = 0; i < fs.size(); ++i) {
    const int rc = reconstruct(fs[i], bs[i], outs[i], st);
    if (rc) return rc;
  }
  return IPC_OK;
}

int ipc_internal_reconstruct_batch(const std::vector<ipc_field*>& fs,
                                   const std::vector<std::vector<int>>& bs,
                                   const std::vector<void*>& outs, cudaStream_t st,
                                   std::vector<void*>* tabs) {
  for (int dt = 0; dt < 2; ++dt) {
    std::vector<ipc_field*> f2;
    std::vector<std::vector<int>> b2;
    std::vector<void*> o2;
    for (size_t i = 0; i < fs.size(); ++i)
      if (fs[i]->dtype == dt) {
        f2.push_back(fs[i]);
        b2.push_back(bs[i]);
        o2.push_back(outs[i]);
      }
    if (f2.empty()) continue;
    BatchTable T;
    build_retrieve_table(f2, b2, o2, &T);
    void* tab = nullptr;
    int rc = upload_table(T, &tab, st, true);
    if (tab) tabs->push_back(tab);
    if (!rc) rc = launch_retrieve_table(dt, T, tab, st, true, nullptr);
    if (rc) return rc;
  }
  return IPC_OK;
}

extern "C" {

int ipc_compress_batch(int nfields, const ipc_batch_item* items, void* stream, ipc_field** outs) {
  g_err.clear();
  Nvtx nv_call("ipc compress batch");
  if (nfields < 0 || (nfields > 0 && (!items || !outs))) return fail(IPC_EINVAL, "null argument");
  std::vector<ipc_field*> all(nfields, nullptr);
  int dev = 0;
  cudaGetDevice(&dev);
  auto cleanup = [&](int rc) {
    for (auto* f : all)
      if (f) {
        free_field_device(f);
        f->tag = kDeadTag;
        delete f;
      }
    return rc;
  };
  for (int i = 0; i < nfields; ++i) {
    const ipc_batch_item& it = items[i];
    if (!it.d_in || (it.dtype != IPC_F32 && it.dtype != IPC_F64) ||
        it.interp < IPC_LINEAR || it.interp > IPC_INTERP_AUTO ||
        (it.bound != IPC_BOUND_STRICT && it.bound != IPC_BOUND_PAPER) ||
        (it.eb_mode != IPC_EB_ABS && it.eb_mode != IPC_EB_REL) || !std::isfinite(it.eb) ||
        !(it.eb > 0))
      return cleanup(fail(IPC_EINVAL, "invalid batch item"));
    ipc_field* f = new (std::nothrow) ipc_field();
    if (!f) return cleanup(fail(IPC_ENOMEM, "host allocation"));
    all[i] = f;
    f->tag = kFieldTag;
    f->device = dev;
    f->dtype = it.dtype;
    f->interp = it.interp;
    f->bound = it.bound;
    f->eb_mode = it.eb_mode;
    f->eb_user = it.eb;
  }
  // the fields' geometries (large batches on the host pool)
  std::vector<char> geo_ok(nfields, 0);
  auto geo = [&](int i) {
    try {
      geo_ok[i] = build_geo(items[i].ndim, items[i].dims, items[i].dtype, &all[i]->g) ? 1 : 0;
    } catch (const std::bad_alloc&) {
      geo_ok[i] = 0;
    }
  };
  if (nfields >= 8)
    HostPool::get().run(nfields, geo);
  else
    for (int i = 0; i < nfields; ++i) geo(i);
  for (int i = 0; i < nfields; ++i)
    if (!geo_ok[i]) return cleanup(fail(IPC_EINVAL, "shape"));
  // the per-field interpolation choices, all in one pass
  {
    std::vector<AutoItem> a;
    std::vector<int> who;
    for (int i = 0; i < nfields; ++i)
      if (items[i].interp == IPC_INTERP_AUTO) {
        const ipc_batch_item& it = items[i];
        a.push_back(AutoItem{it.d_in, it.dtype, it.ndim, {1, 1, 1}, it.eb_mode, it.bound, it.eb, -1});
        for (int d = 0; d < it.ndim; ++d) a.back().dims[d] = it.dims[d];
        who.push_back(i);
      }
    const int rc = resolve_auto(a, (cudaStream_t)stream);
    if (rc) return cleanup(rc);
    for (size_t k = 0; k < a.size(); ++k) all[who[k]]->interp = a[k].mode;
  }
  for (int dt = 0; dt < 2; ++dt) {
    std::vector<ipc_field*> fs;
    std::vector<const void*> ins;
    for (int i = 0; i < nfields; ++i)
      if (items[i].dtype == dt) {
        fs.push_back(all[i]);
        ins.push_back(items[i].d_in);
      }
    if (fs.empty()) continue;
    const int rc = compress_fields(fs, ins, (cudaStream_t)stream);
    if (rc) return cleanup(rc);
  }
  for (int i = 0; i < nfields; ++i) outs[i] = all[i];
  return IPC_OK;
}

namespace {
// Shared front end of the batched retrieval and its plan: validation and
// selection of every field, grouped by element type.
int batch_select(int n, ipc_field* const* fields, const ipc_target* targets, void* const* d_outs,
                 std::vector<std::vector<int>>* bs, std::vector<uint64_t>* bytes,
                 std::vector<double>* bounds) {
  if (n < 0 || (n > 0 && (!fields || !targets || !d_outs))) return fail(IPC_EINVAL, "null argument");
  bs->assign(n, {});
  bytes->assign(n, 0);
  bounds->assign(n, 0.0);
  for (int i = 0; i < n; ++i)
    if (!fields[i] || fields[i]->tag != kFieldTag || !d_outs[i])
      return fail(IPC_EINVAL, "invalid field or output");
  // the fields' selections are independent: large batches spread them over
  // the host pool (the first failure in field order is reported)
  std::vector<int> rcs(n, IPC_OK);
  std::vector<const char*> why(n, "");
  auto one = [&](int i) {
    try {
      rcs[i] = select_planes(fields[i]->sel, targets[i].kind, targets[i].value, nullptr,
                             &(*bs)[i], &(*bytes)[i], &(*bounds)[i], &why[i]);
    } catch (const std::bad_alloc&) {
      rcs[i] = IPC_ENOMEM;
      why[i] = "host allocation";
    }
  };
  if (n >= 16)
    HostPool::get().run(n, one);
  else
    for (int i = 0; i < n; ++i) one(i);
  for (int i = 0; i < n; ++i)
    if (rcs[i]) return fail(rcs[i], why[i]);
  return IPC_OK;
}
}  // namespace

int ipc_retrieve_batch(int n, ipc_field* const* fields, const ipc_target* targets,
                       void* const* d_outs, void* stream, ipc_view** outs) {
  g_err.clear();
  Nvtx nv_call("ipc retrieve batch");
  std::vector<std::vector<int>> bs;
  std::vector<uint64_t> bytes;
  std::vector<double> bounds;
  int rc = batch_select(n, fields, targets, d_outs, &bs, &bytes, &bounds);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<ipc_view*> views;
  if (outs) {
    for (int i = 0; i < n; ++i) {
      ipc_view* v = new (std::nothrow) ipc_view();
      if (!v) {
        for (auto* w : views) delete w;
        return fail(IPC_ENOMEM, "host allocation");
      }
      v->tag = kViewTag;
      v->f = fields[i];
      v->b = bs[i];
      v->bytes = bytes[i];
      v->bound = bounds[i];
      views.push_back(v);
    }
  }
  for (int dt = 0; dt < 2; ++dt) {
    std::vector<ipc_field*> fs;
    std::vector<std::vector<int>> b2;
    std::vector<void*> o2;
    for (int i = 0; i < n; ++i)
      if (fields[i]->dtype == dt) {
        fs.push_back(fields[i]);
        b2.push_back(bs[i]);
        o2.push_back(d_outs[i]);
      }
    if (fs.empty()) continue;
    BatchTable T;
    build_retrieve_table(fs, b2, o2, &T);
    void* tab = nullptr;
    rc = upload_table(T, &tab, st, true);
    if (!rc) rc = launch_retrieve_table(dt, T, tab, st, true, nullptr);
    if (tab) cudaFreeAsync(tab, st);
    if (rc) {
      for (auto* w : views) delete w;
      return rc;
    }
  }
  if (outs)
    for (int i = 0; i < n; ++i) outs[i] = views[i];
  return IPC_OK;
}

int ipc_plan_retrieve_batch(int n, ipc_field* const* fields, const ipc_target* targets,
                            void* const* d_outs, void* stream, ipc_plan** out) {
  g_err.clear();
  if (!out) return fail(IPC_EINVAL, "null argument");
  std::vector<std::vector<int>> bs;
  std::vector<uint64_t> bytes;
  std::vector<double> bounds;
  int rc = batch_select(n, fields, targets, d_outs, &bs, &bytes, &bounds);
  if (rc) return rc;
  for (int i = 1; i < n; ++i)
    if (fields[i]->dtype != fields[0]->dtype) return fail(IPC_EINVAL, "a plan takes one element type");
  ipc_plan* p = new (std::nothrow) ipc_plan();
  if (!p) return fail(IPC_ENOMEM, "host allocation");
  p->tag = kPlanTag;
  cudaGetDevice(&p->device);
  std::vector<ipc_field*> fs(fields, fields + n);
  std::vector<void*> o2(d_outs, d_outs + n);
  BatchTable T;
  build_retrieve_table(fs, bs, o2, &T);
  cudaStream_t st = (cudaStream_t)stream;
  rc = upload_table(T, &p->d_tab, st, false);
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaSuccess;
  if (!rc) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (!rc && e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (!rc && e == cudaSuccess) {
    rc = launch_retrieve_table(n ? fields[0]->dtype : 0, T, p->d_tab, cs, false, &p->launches);
    g_launches.fetch_sub(p->launches, std::memory_order_relaxed);  // counted at replay
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess) e = e2;
    p->graph = g;
    if (!rc && e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, g, 0);
  }
  if (cs) cudaStreamDestroy(cs);
  if (rc || e != cudaSuccess) {
    if (e != cudaSuccess) cuda_fail(e, "graph capture");
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->d_tab) cudaFree(p->d_tab);
    delete p;
    return rc ? rc : IPC_ECUDA;
  }
  *out = p;
  return IPC_OK;
}

int ipc_plan_launch(ipc_plan* p, void* stream) {
  if (!p || p->tag != kPlanTag) return fail(IPC_EINVAL, "invalid plan");
  CU(cudaGraphLaunch(p->exec, (cudaStream_t)stream));
  g_launches.fetch_add(p->launches, std::memory_order_relaxed);
  return IPC_OK;
}

int ipc_debug_bounds(uint64_t* rec, int reset) {
#ifdef IPC_DEBUG_BOUNDS
  if (!rec) return fail(IPC_EINVAL, "null argument");
  unsigned long long* d = bounds_record();
  if (!d) return fail(IPC_ENOMEM, "bounds record");
  CU(cudaDeviceSynchronize());
  unsigned long long h[4];
  CU(cudaMemcpy(h, d, 32, cudaMemcpyDeviceToHost));
  for (int i = 0; i < 4; ++i) rec[i] = h[i];
  if (reset) CU(cudaMemset(d, 0, 32));
  return IPC_OK;
#else
  (void)rec;
  (void)reset;
  return fail(IPC_EINVAL, "not a bounds-checking build");
#endif
}

int ipc_nvtx_enable(int on) {
  g_nvtx.store(on != 0, std::memory_order_relaxed);
  return IPC_OK;
}

int ipc_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_on = on != 0;
  return IPC_OK;
}

int ipc_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  prof_drain();
  for (auto& a : g_prof_acc) a = ProfAcc{0, 0.0, 0.0};
  return IPC_OK;
}

int ipc_profile_read(int kind, uint64_t* launches, double* total_ms, double* alg_bytes) {
  if (kind < 0 || kind >= IPC_KERNEL_KINDS) return fail(IPC_EINVAL, "kernel kind");
  std::lock_guard<std::mutex> lk(g_prof_mu);
  prof_drain();
  if (launches) *launches = g_prof_acc[kind].launches;
  if (total_ms) *total_ms = g_prof_acc[kind].ms;
  if (alg_bytes) *alg_bytes = g_prof_acc[kind].bytes;
  return IPC_OK;
}

uint64_t ipc_launch_count(void) { return g_launches.load(); }

int ipc_field_info(const ipc_field* f, int* dtype, int* ndim, int64_t* dims, int* K, int* S,
                   double* eb, double* xmin, double* xmax) {
  if (!f || f->tag != kFieldTag) return fail(IPC_EINVAL, "invalid field");
  if (dtype) *dtype = f->dtype;
  if (ndim) *ndim = f->g.ndim;
  if (dims)
    for (int e = 0; e < 3; ++e) dims[e] = e < f->g.ndim ? f->g.N[3 - f->g.ndim + e] : 0;
  if (K) *K = f->g.K;
  if (S) *S = (int)f->g.stages.size();
  if (eb) *eb = f->eb;
  if (xmin) *xmin = f->xmin;
  if (xmax) *xmax = f->xmax;
  return IPC_OK;
}

}  // extern "C"
