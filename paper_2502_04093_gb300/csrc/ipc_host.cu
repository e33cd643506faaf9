// Host side of libipcomp: the C ABI of include/ipc.h, the container format,
// the optimized loader (Sec. 5) and the launch sequences of compression and
// reconstruction. Every step of the data path runs in the kernels of
// ipc_kernels.cu; this file only plans, allocates and orders them.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "ipc.h"
#include "ipc_internal.h"

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

const uint32_t kMagic = 0x31435049u;  // "IPC1"
const uint32_t kVersion = 1u;
const uint32_t kFieldTag = 0x46435049u, kViewTag = 0x56435049u, kDeadTag = 0xDEADDEADu;
const uint64_t kSaturate = 1ull << 62;

}  // namespace

// ---------------------------------------------------------------------------
// Geometry (Sec. 4.1): dims padded to 3-D; level l = K..1 has stride
// s = 2^(l-1); sweep d over the points whose coordinate d is an odd multiple
// of s, coordinates before d multiples of s, after d multiples of 2s.
// ---------------------------------------------------------------------------
namespace ipc {
bool build_geo(int ndim, const int64_t* dims, Geo* g) {
  if (ndim < 1 || ndim > 3 || !dims) return false;
  g->ndim = ndim;
  g->N[0] = g->N[1] = g->N[2] = 1;
  uint64_t n = 1;
  for (int e = 0; e < ndim; ++e) {
    if (dims[e] < 1 || dims[e] > (int64_t(1) << 40)) return false;
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
      sg.ntiles = (sg.words + kTileWords - 1) / kTileWords;
      g->stages.push_back(sg);
    }
  }
  return true;
}

StageArgs stage_args(const Geo& g, const StageGeo& sg, int cubic) {
  StageArgs a{};
  for (int e = 0; e < 3; ++e) {
    a.N[e] = g.N[e];
    a.start[e] = sg.start[e];
    a.step[e] = sg.step[e];
    a.m[e] = sg.m[e];
  }
  a.stride[2] = 1;
  a.stride[1] = g.N[2];
  a.stride[0] = g.N[1] * g.N[2];
  a.s = int64_t(1) << (sg.level - 1);
  a.W = sg.words;
  a.wr = sg.wr;
  a.ntiles = sg.ntiles;
  a.d = sg.dim3;
  a.cubic = cubic;
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

struct ipc_field {
  uint32_t tag;
  int device;
  int dtype, interp, bound, eb_mode;
  double eb_user, eb, xmin, xmax, xmaxabs, anchor;
  Geo g;
  std::vector<StageTab> st;
  uint64_t mandatory;  // header + tables + outliers
  uint64_t stream_bytes;
  // device
  uint32_t* d_blob;    // every stream, in container order (32-bit words)
  uint32_t* d_rank;    // tile-rank index of every (stage, plane)
  uint64_t* d_oidx;    // outliers: code indices, per stage contiguous
  double* d_oval;
  std::vector<StageDescs> desc;       // per stage
  std::vector<uint64_t> out_off;      // per stage offset into d_oidx/d_oval
};

struct ipc_view {
  uint32_t tag;
  ipc_field* f;
  std::vector<int> b;
  uint64_t bytes;
  double bound;
};

namespace {

// ---------------------------------------------------------------------------
// Workspace: scratch of compression, one per device, grown on demand.
// ---------------------------------------------------------------------------
struct Workspace {
  std::mutex mu;
  void* xh = nullptr;
  uint64_t xh_bytes = 0;
  uint32_t* cap = nullptr;
  uint64_t cap_words = 0;
  uint32_t* bitmap = nullptr;
  uint64_t bitmap_words = 0;
  uint32_t* tilecnt = nullptr;
  uint64_t tilecnt_words = 0;
  unsigned long long* okey = nullptr;
  double* oval = nullptr;
  uint64_t ocap = 0;
  unsigned long long* small = nullptr;  // range acc[4] + outlier count
  uint32_t* stat = nullptr;
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

void free_field_device(ipc_field* f) {
  if (f->d_blob) cudaFree(f->d_blob);
  if (f->d_rank) cudaFree(f->d_rank);
  if (f->d_oidx) cudaFree(f->d_oidx);
  if (f->d_oval) cudaFree(f->d_oval);
  f->d_blob = nullptr;
  f->d_rank = nullptr;
  f->d_oidx = nullptr;
  f->d_oval = nullptr;
}

// Lays out the streams (container order: stage-major, plane 31..0) and the
// rank index from the per-plane nnz; allocates the device buffers.
int layout_field(ipc_field* f) {
  const Geo& g = f->g;
  uint64_t word = 0, rank = 0;
  f->desc.assign(g.stages.size(), StageDescs{});
  for (size_t t = 0; t < g.stages.size(); ++t) {
    const StageGeo& sg = g.stages[t];
    for (int k = 31; k >= 0; --k) {
      StageTab& s = f->st[t];
      PlaneDesc& pd = f->desc[t].p[k];
      pd.off = word;
      pd.nnz = (uint32_t)s.nnz[k];
      pd.mode = stream_mode(s.nnz[k], sg.words);
      s.size[k] = stream_bytes(s.nnz[k], sg.words);
      word += s.size[k] / 4;
    }
    for (int k = 0; k < 32; ++k) f->desc[t].p[k].rank_off = rank + (uint64_t)k * sg.ntiles;
    rank += 32 * sg.ntiles;
  }
  f->stream_bytes = word * 4;
  uint64_t nout = 0;
  f->out_off.assign(g.stages.size() + 1, 0);
  for (size_t t = 0; t < g.stages.size(); ++t) {
    f->out_off[t] = nout;
    nout += f->st[t].out_idx.size();
  }
  f->out_off[g.stages.size()] = nout;
  f->mandatory = header_bytes(f).size();
  if (cudaMalloc((void**)&f->d_blob, std::max<uint64_t>(word, 1) * 4) != cudaSuccess ||
      cudaMalloc((void**)&f->d_rank, std::max<uint64_t>(rank, 1) * 4) != cudaSuccess ||
      cudaMalloc((void**)&f->d_oidx, std::max<uint64_t>(nout, 1) * 8) != cudaSuccess ||
      cudaMalloc((void**)&f->d_oval, std::max<uint64_t>(nout, 1) * 8) != cudaSuccess) {
    cudaGetLastError();
    free_field_device(f);
    return fail(IPC_ENOMEM, "field allocation failed");
  }
  return IPC_OK;
}

int upload_outliers(ipc_field* f, cudaStream_t st) {
  const uint64_t n = f->out_off.back();
  if (n == 0) return IPC_OK;
  std::vector<uint64_t> idx;
  std::vector<double> val;
  idx.reserve(n);
  val.reserve(n);
  for (auto& s : f->st) {
    idx.insert(idx.end(), s.out_idx.begin(), s.out_idx.end());
    val.insert(val.end(), s.out_val.begin(), s.out_val.end());
  }
  CU(cudaMemcpyAsync(f->d_oidx, idx.data(), n * 8, cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(f->d_oval, val.data(), n * 8, cudaMemcpyHostToDevice, st));
  CU(cudaStreamSynchronize(st));
  return IPC_OK;
}

double okey_to_double(unsigned long long k) {
  unsigned long long b = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFULL) : ~k;
  double v;
  std::memcpy(&v, &b, 8);
  return v;
}

template <class T>
void quant_args(double eb, void* out) {
  QuantArgs<T> q;
  q.inv2eb = (T)(1.0 / (2.0 * eb));
  q.twoeb = (T)(2.0 * eb);
  const double shrink = sizeof(T) == 4 ? 1.0 - 1.0 / 1048576.0 : 1.0 - 1.0 / 1125899906842624.0;
  q.ebchk = (T)(eb * shrink);
  q.R = (T)(sizeof(T) == 4 ? 2097152.0 : 1073741824.0);
  std::memcpy(out, &q, sizeof(q));
}

int compress_impl(const void* d_in, ipc_field* f, cudaStream_t st) {
  int dev = 0;
  CU(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(IPC_EINVAL, "device index out of range");
  Workspace& ws = g_ws[dev];
  std::lock_guard<std::mutex> lock(ws.mu);
  const Geo& g = f->g;
  const size_t esz = f->dtype == 0 ? 4 : 8;
  const size_t S = g.stages.size();

  // scratch sizes
  uint64_t capw = 0, bmw = 0, cntw = 0;
  for (auto& sg : g.stages) {
    capw += 32 * sg.ntiles * kTileWords;
    bmw += 32 * sg.ntiles * kTileBitmapWords;
    cntw += 32 * sg.ntiles;
  }
  int rc;
  if ((rc = grow(&ws.xh, &ws.xh_bytes, g.n * esz, 1)) ||
      (rc = grow(&ws.cap, &ws.cap_words, capw, 4)) ||
      (rc = grow(&ws.bitmap, &ws.bitmap_words, bmw, 4)) ||
      (rc = grow(&ws.tilecnt, &ws.tilecnt_words, cntw, 4)) ||
      (rc = grow(&ws.stat, &ws.stat_words, 2 * std::max<size_t>(S, 1), 4)) ||
      (rc = grow(&ws.nnz, &ws.nnz_words, 32 * std::max<size_t>(S, 1), 4)))
    return rc;
  uint64_t dummy = 0;
  if (!ws.small && (rc = grow(&ws.small, &dummy, 8, 8))) return rc;
  if (ws.ocap == 0) {
    uint64_t oc = 0;
    if ((rc = grow(&ws.okey, &oc, 1 << 16, 8)) || (rc = grow(&ws.oval, &oc, 1 << 16, 8)))
      return rc;
    ws.ocap = 1 << 16;
  }

  // a0: range over finite values
  unsigned long long init[5] = {~0ULL, 0ULL, 0ULL, 0ULL, 0ULL};
  CU(cudaMemcpyAsync(ws.small, init, sizeof(init), cudaMemcpyHostToDevice, st));
  CU(launch_range(f->dtype, d_in, g.n, ws.small, st));
  unsigned long long acc[5];
  CU(cudaMemcpyAsync(acc, ws.small, sizeof(acc), cudaMemcpyDeviceToHost, st));
  double x0 = 0;
  if (f->dtype == 0) {
    float v;
    CU(cudaMemcpyAsync(&v, d_in, 4, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    x0 = v;
  } else {
    CU(cudaMemcpyAsync(&x0, d_in, 8, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
  }
  const bool any = acc[3] > 0;
  f->xmin = any ? okey_to_double(acc[0]) : 0.0;
  f->xmax = any ? okey_to_double(acc[1]) : 0.0;
  {
    double ma = 0;
    std::memcpy(&ma, &acc[2], 8);
    f->xmaxabs = any ? ma : 0.0;
  }
  double eb = f->eb_user;
  if (f->eb_mode == IPC_EB_REL) {
    if (!any) return fail(IPC_EINVAL, "relative error bound on a field without finite values");
    const double r = f->xmax - f->xmin;
    eb = r > 0 ? f->eb_user * r : f->eb_user;
  }
  if (!(eb > 0) || !std::isfinite(eb)) return fail(IPC_EINVAL, "error bound must be > 0 and finite");
  f->eb = eb;
  f->anchor = x0;
  alignas(16) unsigned char qbuf[64];
  if (f->dtype == 0) quant_args<float>(eb, qbuf);
  else quant_args<double>(eb, qbuf);

  for (int attempt = 0; attempt < 2; ++attempt) {
    CU(cudaMemsetAsync(ws.stat, 0, 2 * std::max<size_t>(S, 1) * 4, st));
    CU(cudaMemsetAsync(ws.small + 4, 0, 8, st));
    CompressScratch sc{ws.cap, ws.bitmap, ws.tilecnt, ws.okey, ws.oval, ws.small + 4, ws.ocap,
                       ws.stat};
    // the anchor is known exactly; xh[0] = x[0]
    CU(cudaMemcpyAsync(ws.xh, d_in, esz, cudaMemcpyDeviceToDevice, st));
    uint64_t capo = 0, bmo = 0, cnto = 0;
    for (size_t t = 0; t < S; ++t) {
      const StageGeo& sg = g.stages[t];
      StageArgs a = stage_args(g, sg, f->interp == IPC_CUBIC);
      const int write_xh = t + 1 < S;  // the last sweep's values are never read
      CU(launch_compress_stage(f->dtype, a, d_in, ws.xh, write_xh, qbuf, (int)t, sc, capo, bmo,
                               cnto, st));
      capo += 32 * sg.ntiles * kTileWords;
      bmo += 32 * sg.ntiles * kTileBitmapWords;
      cnto += 32 * sg.ntiles;
    }
    unsigned long long nout = 0;
    CU(cudaMemcpyAsync(&nout, ws.small + 4, 8, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (nout <= ws.ocap) break;
    if (attempt == 1) return fail(IPC_ECUDA, "outlier count changed between passes");
    // grow the outlier buffers to the exact count and run the sweeps again
    cudaFree(ws.okey);
    cudaFree(ws.oval);
    ws.okey = nullptr;
    ws.oval = nullptr;
    ws.ocap = 0;
    uint64_t oc = 0;
    if ((rc = grow(&ws.okey, &oc, nout, 8)) || (rc = grow(&ws.oval, &oc, nout, 8)))
      return rc;
    ws.ocap = nout;
  }

  // statistics and outliers
  f->st.assign(S, StageTab{});
  if (S) {
    std::vector<uint32_t> stat(2 * S);
    CU(cudaMemcpyAsync(stat.data(), ws.stat, 8 * S, cudaMemcpyDeviceToHost, st));
    unsigned long long nout = 0;
    CU(cudaMemcpyAsync(&nout, ws.small + 4, 8, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    for (size_t t = 0; t < S; ++t) {
      uint32_t orv = stat[2 * t];
      int h = -1;
      while (orv) { ++h; orv >>= 1; }
      f->st[t].H = h;
      f->st[t].Q = stat[2 * t + 1];
    }
    if (nout) {
      std::vector<unsigned long long> key(nout);
      std::vector<double> val(nout);
      CU(cudaMemcpyAsync(key.data(), ws.okey, nout * 8, cudaMemcpyDeviceToHost, st));
      CU(cudaMemcpyAsync(val.data(), ws.oval, nout * 8, cudaMemcpyDeviceToHost, st));
      CU(cudaStreamSynchronize(st));
      std::vector<uint64_t> order(nout);
      for (uint64_t i = 0; i < nout; ++i) order[i] = i;
      std::sort(order.begin(), order.end(), [&](uint64_t a, uint64_t b) { return key[a] < key[b]; });
      for (uint64_t i : order) {
        const size_t t = (size_t)(key[i] >> 40);
        f->st[t].out_idx.push_back(key[i] & ((1ULL << 40) - 1));
        f->st[t].out_val.push_back(val[i]);
      }
    }
  }

  // per-plane nnz and tile ranks
  uint64_t cnto = 0, rank_total = 0;
  for (auto& sg : g.stages) rank_total += 32 * sg.ntiles;
  uint32_t* d_rank = nullptr;
  if (cudaMalloc((void**)&d_rank, std::max<uint64_t>(rank_total, 1) * 4) != cudaSuccess) {
    cudaGetLastError();
    return fail(IPC_ENOMEM, "rank index allocation failed");
  }
  {
    uint64_t ro = 0;
    for (size_t t = 0; t < S; ++t) {
      const StageGeo& sg = g.stages[t];
      StageArgs a = stage_args(g, sg, 0);
      cudaError_t e = launch_scan_stage(a, CompressScratch{nullptr, nullptr, ws.tilecnt}, cnto,
                                        d_rank + ro, ws.nnz + 32 * t, st);
      if (e != cudaSuccess) { cudaFree(d_rank); return cuda_fail(e, "scan"); }
      cnto += 32 * sg.ntiles;
      ro += 32 * sg.ntiles;
    }
    std::vector<uint32_t> nnz(32 * std::max<size_t>(S, 1));
    cudaError_t e = cudaMemcpyAsync(nnz.data(), ws.nnz, 32 * S * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { cudaFree(d_rank); return cuda_fail(e, "nnz readback"); }
    for (size_t t = 0; t < S; ++t)
      for (int k = 0; k < 32; ++k) f->st[t].nnz[k] = nnz[32 * t + k];
  }
  rc = layout_field(f);
  if (rc) { cudaFree(d_rank); return rc; }
  cudaFree(f->d_rank);
  f->d_rank = d_rank;

  // pack the streams into the field blob
  uint64_t capo = 0, bmo = 0;
  cnto = 0;
  for (size_t t = 0; t < S; ++t) {
    const StageGeo& sg = g.stages[t];
    StageArgs a = stage_args(g, sg, 0);
    CompressScratch sc{ws.cap, ws.bitmap, ws.tilecnt};
    CU(launch_pack_stage(a, sc, capo, bmo, cnto, f->d_rank + f->desc[t].p[0].rank_off, f->desc[t],
                         f->d_blob, st));
    capo += 32 * sg.ntiles * kTileWords;
    bmo += 32 * sg.ntiles * kTileBitmapWords;
    cnto += 32 * sg.ntiles;
  }
  CU(cudaStreamSynchronize(st));
  return upload_outliers(f, st);
}

// ---------------------------------------------------------------------------
// Optimized loader (Sec. 5.2 / 5.3): exact knapsack over the levels on the
// Pareto frontier of (error cost, loaded bytes).
// Cost of dropping b planes at level l, in units of eb * 2^-16:
//   M(t, b) = 0 (b = 0) | U(b) (b <= H_t) | Q_t (b > H_t), U the negabinary
//   uncertainty of b digits (Sec. 4.4.2).
//   strict: sum_{t in l} ceil(p^(S-1-t) * M * bin * 2^16) + [b > 0] rho_l,
//           rho_l = ceil(kappa * u * (A / eb) * 2^16 * sum_{t: level <= l} p^(S-1-t))
//   paper : ceil(p^(l-1) * max_{t in l} M * bin * 2^16)   (Theorem 1)
// with bin = fl(2eb) / eb, kappa = 24 (cubic) / 12 (linear), u the unit
// roundoff of the element type, A a bound on the magnitudes involved.
// ---------------------------------------------------------------------------
uint64_t sadd(uint64_t a, uint64_t b) {
  const uint64_t c = a + b;
  return (c < a || c > kSaturate) ? kSaturate : c;
}
uint64_t units(double v) {
  if (!(v < (double)kSaturate)) return kSaturate;
  return v <= 0 ? 0 : (uint64_t)std::ceil(v);
}
uint64_t uncert(int b) {
  if (b <= 0) return 0;
  const uint64_t p = uint64_t(1) << (b + 1);
  return (b & 1) ? (p - 1) / 3 : (p - 2) / 3;
}

struct Tables {
  int K;
  std::vector<uint64_t> cost, bytes;  // [l-1][b]
};

void build_tables(const ipc_field* f, double A, Tables* T) {
  const Geo& g = f->g;
  const int K = g.K, S = (int)g.stages.size();
  const bool cubic = f->interp == IPC_CUBIC, strict = f->bound == IPC_BOUND_STRICT;
  const double p = cubic ? 1.25 : 1.0;
  std::vector<double> pw(std::max(S, K) + 1);
  pw[0] = 1.0;
  for (size_t i = 1; i < pw.size(); ++i) pw[i] = pw[i - 1] * p;
  const double twoeb = f->dtype == 0 ? (double)(float)(2.0 * f->eb) : 2.0 * f->eb;
  const double bin = twoeb / f->eb;
  const double u = f->dtype == 0 ? 1.0 / 16777216.0 : 1.0 / 9007199254740992.0;
  const double kappa = cubic ? 24.0 : 12.0;
  T->K = K;
  T->cost.assign((size_t)K * 33, 0);
  T->bytes.assign((size_t)K * 33, 0);
  for (int l = 1; l <= K; ++l) {
    double asum = 0;
    for (int t = 0; t < S; ++t)
      if (g.stages[t].level <= l) asum += (strict && cubic) ? pw[S - 1 - t] : 1.0;
    const uint64_t rho = units(kappa * u * (A / f->eb) * 65536.0 * asum);
    for (int b = 0; b <= 32; ++b) {
      uint64_t c = 0, y = 0, mmax = 0;
      for (int t = 0; t < S; ++t) {
        if (g.stages[t].level != l) continue;
        const StageTab& s = f->st[t];
        const uint64_t M = b <= 0 ? 0 : (b <= s.H ? uncert(b) : (uint64_t)s.Q);
        if (strict) c = sadd(c, units((cubic ? pw[S - 1 - t] : 1.0) * (double)M * bin * 65536.0));
        else mmax = std::max(mmax, M);
        for (int k = b; k < 32; ++k) y += s.size[k];
      }
      if (strict) {
        if (b > 0) c = sadd(c, rho);
      } else {
        c = units(pw[l - 1] * (double)mmax * bin * 65536.0);
      }
      T->cost[(size_t)(l - 1) * 33 + b] = c;
      T->bytes[(size_t)(l - 1) * 33 + b] = y;
    }
  }
}

// Pareto frontier DP, levels 1..K (finest first). Each label keeps its
// parent so the prefix (b_1..b_j) can be rebuilt for lexicographic ties.
struct Label {
  uint64_t c, y;
  int parent;
  int b;
};

void prefix_of(const std::vector<std::vector<Label>>& L, int level, int i, std::vector<int>* out) {
  out->assign(level + 1, 0);
  for (int j = level; j >= 0; --j) {
    (*out)[j] = L[j][i].b;
    i = L[j][i].parent;
  }
}

int solve(const Tables& T, int kind, uint64_t limit, const std::vector<int>* upper,
          std::vector<int>* best) {
  const int K = T.K;
  if (K == 0) { best->clear(); return IPC_OK; }
  std::vector<std::vector<Label>> L(K);
  std::vector<int> pa, pb;
  for (int l = 0; l < K; ++l) {
    std::vector<Label> cand;
    const int bmax = upper ? (*upper)[l] : 32;
    const size_t nprev = l == 0 ? 1 : L[l - 1].size();
    for (size_t i = 0; i < nprev; ++i) {
      const uint64_t c0 = l == 0 ? 0 : L[l - 1][i].c, y0 = l == 0 ? 0 : L[l - 1][i].y;
      for (int b = 0; b <= bmax; ++b) {
        Label n{sadd(c0, T.cost[(size_t)l * 33 + b]), y0 + T.bytes[(size_t)l * 33 + b], (int)i, b};
        if ((kind == 0 && n.c > limit) || (kind == 1 && n.y > limit)) continue;
        cand.push_back(n);
      }
    }
    if (cand.empty()) return kind == 0 ? IPC_EBOUND : IPC_EBUDGET;
    L[l] = cand;  // temporarily, so prefixes can be rebuilt while sorting
    std::vector<int> order(cand.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::sort(order.begin(), order.end(), [&](int a, int b) {
      const Label &x = cand[a], &z = cand[b];
      if (x.c != z.c) return x.c < z.c;
      if (x.y != z.y) return x.y < z.y;
      prefix_of(L, l, a, &pa);
      prefix_of(L, l, b, &pb);
      return pa > pb;  // lexicographically larger (b_1, b_2, ...) first
    });
    std::vector<Label> keep;
    for (int i : order) {
      if (keep.empty() || cand[i].y < keep.back().y) keep.push_back(cand[i]);
    }
    L[l] = keep;
  }
  // cost increases and bytes decrease along the frontier
  const int pick = kind == 0 ? (int)L[K - 1].size() - 1 : 0;
  prefix_of(L, K - 1, pick, best);
  return IPC_OK;
}

uint64_t loaded(const ipc_field* f, const std::vector<int>& b) {
  uint64_t y = f->mandatory;
  for (size_t t = 0; t < f->g.stages.size(); ++t)
    for (int k = b[f->g.stages[t].level - 1]; k < 32; ++k) y += f->st[t].size[k];
  return y;
}
uint64_t cost_of(const Tables& T, const std::vector<int>& b) {
  uint64_t c = 0;
  for (size_t l = 0; l < b.size(); ++l) c = sadd(c, T.cost[l * 33 + b[l]]);
  return c;
}

int select(const ipc_field* f, ipc_target tg, const std::vector<int>* upper, std::vector<int>* b,
           uint64_t* bytes, double* bound) {
  if (!std::isfinite(tg.value)) return fail(IPC_EINVAL, "target must be finite");
  const double range = f->xmax - f->xmin;
  Tables T;
  if (tg.kind == IPC_TARGET_EB) {
    double E = tg.value;
    if (f->eb_mode == IPC_EB_REL) E = range > 0 ? tg.value * range : tg.value;
    if (!(E >= f->eb)) return fail(IPC_EBOUND, "target error bound is below the compression bound");
    build_tables(f, f->xmaxabs + E, &T);
    const double Bd = std::floor(((E - f->eb) / f->eb) * 65536.0);
    const uint64_t B = Bd >= (double)kSaturate ? kSaturate : (uint64_t)Bd;
    int rc = solve(T, 0, B, upper, b);
    if (rc) return fail(rc, "no selection meets the error bound");
    *bytes = loaded(f, *b);
    *bound = f->eb + (double)cost_of(T, *b) * f->eb / 65536.0;
    return IPC_OK;
  }
  if (tg.kind == IPC_TARGET_BITRATE) {
    if (!(tg.value >= 0)) return fail(IPC_EINVAL, "bitrate must be >= 0");
    const double Sd = std::floor(tg.value * (double)f->g.n / 8.0);
    const uint64_t Sb = Sd >= 1.8e19 ? ~uint64_t(0) : (uint64_t)Sd;
    if (f->mandatory > Sb) return fail(IPC_EBUDGET, "bitrate below the mandatory bytes");
    double A = f->xmaxabs + std::max(range, f->eb);
    build_tables(f, A, &T);
    int rc = solve(T, 1, Sb - f->mandatory, upper, b);
    if (rc) return fail(rc, "no selection fits the bitrate");
    *bytes = loaded(f, *b);
    double G = f->eb + (double)cost_of(T, *b) * f->eb / 65536.0;
    for (int it = 0; it < 16 && G > A - f->xmaxabs; ++it) {
      A = f->xmaxabs + G;
      build_tables(f, A, &T);
      G = f->eb + (double)cost_of(T, *b) * f->eb / 65536.0;
    }
    *bound = G;
    return IPC_OK;
  }
  return fail(IPC_EINVAL, "unknown target kind");
}

// Algorithm 1 on the device: anchor, then one reconstruction launch per
// sweep (coarse to fine), each followed by its outlier scatter.
int reconstruct(ipc_field* f, const std::vector<int>& b, void* d_out, cudaStream_t st) {
  const Geo& g = f->g;
  CU(launch_set_anchor(f->dtype, d_out, f->anchor, st));
  const double twoeb = f->dtype == 0 ? (double)(float)(2.0 * f->eb) : 2.0 * f->eb;
  for (size_t t = 0; t < g.stages.size(); ++t) {
    const StageGeo& sg = g.stages[t];
    StageArgs a = stage_args(g, sg, f->interp == IPC_CUBIC);
    CU(launch_retrieve_stage(f->dtype, a, d_out, twoeb, f->desc[t], b[sg.level - 1], f->d_blob,
                             f->d_rank, st));
    const uint64_t no = f->out_off[t + 1] - f->out_off[t];
    if (no)
      CU(launch_outlier_scatter(f->dtype, a, d_out, f->d_oidx + f->out_off[t],
                                f->d_oval + f->out_off[t], no, st));
  }
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
// ===========================================================================
extern "C" {

const char* ipc_last_error(void) { return g_err.c_str(); }

int ipc_compress(const void* d_in, int dtype, int ndim, const int64_t* dims, int eb_mode,
                 double eb, int interp, int bound, void* stream, ipc_field** out) {
  g_err.clear();
  if (!d_in || !out) return fail(IPC_EINVAL, "null argument");
  if (dtype != IPC_F32 && dtype != IPC_F64) return fail(IPC_EINVAL, "dtype");
  if (interp != IPC_LINEAR && interp != IPC_CUBIC) return fail(IPC_EINVAL, "interp");
  if (bound != IPC_BOUND_STRICT && bound != IPC_BOUND_PAPER) return fail(IPC_EINVAL, "bound");
  if (eb_mode != IPC_EB_ABS && eb_mode != IPC_EB_REL) return fail(IPC_EINVAL, "eb_mode");
  if (!std::isfinite(eb) || !(eb > 0)) return fail(IPC_EINVAL, "eb must be > 0 and finite");
  ipc_field* f = new (std::nothrow) ipc_field();
  if (!f) return fail(IPC_ENOMEM, "host allocation");
  f->tag = kFieldTag;
  if (!build_geo(ndim, dims, &f->g)) {
    delete f;
    return fail(IPC_EINVAL, "shape");
  }
  cudaGetDevice(&f->device);
  f->dtype = dtype;
  f->interp = interp;
  f->bound = bound;
  f->eb_mode = eb_mode;
  f->eb_user = eb;
  int rc = compress_impl(d_in, f, (cudaStream_t)stream);
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
  g_err.clear();
  if (!f || f->tag != kFieldTag || !d_out) return fail(IPC_EINVAL, "null or invalid argument");
  DeviceGuard dg(f->device);
  std::vector<int> b;
  uint64_t bytes = 0;
  double bound = 0;
  int rc = select(f, target, nullptr, &b, &bytes, &bound);
  if (rc) return rc;
  ipc_view* v = nullptr;
  if (out) {
    v = new (std::nothrow) ipc_view();
    if (!v) return fail(IPC_ENOMEM, "host allocation");
  }
  rc = reconstruct(f, b, d_out, (cudaStream_t)stream);
  if (rc) {
    delete v;
    return rc;
  }
  if (out) {
    v->tag = kViewTag;
    v->f = f;
    v->b = b;
    v->bytes = bytes;
    v->bound = bound;
    *out = v;
  }
  return IPC_OK;
}

int ipc_refine(ipc_view* v, ipc_target target, void* d_out, void* stream) {
  g_err.clear();
  if (!v || v->tag != kViewTag || !d_out) return fail(IPC_EINVAL, "null or invalid argument");
  ipc_field* f = v->f;
  DeviceGuard dg(f->device);
  std::vector<int> b;
  uint64_t bytes = 0;
  double bound = 0;
  int rc = select(f, target, &v->b, &b, &bytes, &bound);
  if (rc == IPC_EBUDGET && target.kind == IPC_TARGET_BITRATE) {
    g_err.clear();
    return IPC_OK;
  }
  if (rc) return rc;
  if (b == v->b) return IPC_OK;
  rc = reconstruct(f, b, d_out, (cudaStream_t)stream);
  if (rc) return rc;
  v->b = b;
  v->bytes = bytes;
  v->bound = bound;
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
    v->tag = kDeadTag;
    delete v;
    return IPC_OK;
  }
  return fail(IPC_EINVAL, "not a live ipc handle");
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
  const uint64_t total = f->mandatory + f->stream_bytes;
  if (!host_buf) {
    *len = total;
    return IPC_OK;
  }
  if (*len < total) return fail(IPC_EINVAL, "buffer too small");
  DeviceGuard dg(f->device);
  std::vector<uint8_t> h = header_bytes(f);
  std::memcpy(host_buf, h.data(), h.size());
  if (f->stream_bytes)
    CU(cudaMemcpy((uint8_t*)host_buf + h.size(), f->d_blob, f->stream_bytes,
                  cudaMemcpyDeviceToHost));
  *len = total;
  return IPC_OK;
}

int ipc_import(const void* host_buf, uint64_t len, void* stream, ipc_field** out) {
  g_err.clear();
  if (!out || (!host_buf && len)) return fail(IPC_EINVAL, "null argument");
  const uint8_t* p = (const uint8_t*)host_buf;
  uint64_t pos = 0;
  bool ok = true;
  auto need = [&](uint64_t k) {
    if (pos + k > len || pos + k < pos) ok = false;
    return ok;
  };
  auto g32 = [&]() -> uint32_t {
    if (!need(4)) return 0;
    uint32_t v = 0;
    for (int i = 0; i < 4; ++i) v |= uint32_t(p[pos + i]) << (8 * i);
    pos += 4;
    return v;
  };
  auto g64 = [&]() -> uint64_t {
    if (!need(8)) return 0;
    uint64_t v = 0;
    for (int i = 0; i < 8; ++i) v |= uint64_t(p[pos + i]) << (8 * i);
    pos += 8;
    return v;
  };
  auto gd = [&]() {
    uint64_t u = g64();
    double d;
    std::memcpy(&d, &u, 8);
    return d;
  };
  if (g32() != kMagic || g32() != kVersion || !ok) return fail(IPC_ECORRUPT, "bad magic/version");
  ipc_field* f = new (std::nothrow) ipc_field();
  if (!f) return fail(IPC_ENOMEM, "host allocation");
  f->tag = kFieldTag;
  cudaGetDevice(&f->device);
  auto bad = [&](const char* why) {
    free_field_device(f);
    f->tag = kDeadTag;
    delete f;
    return fail(IPC_ECORRUPT, why);
  };
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
  if (!ok || f->dtype < 0 || f->dtype > 1 || f->interp < 0 || f->interp > 1 || f->bound < 0 ||
      f->bound > 1 || f->eb_mode < 0 || f->eb_mode > 1 || !(f->eb > 0) || !std::isfinite(f->eb))
    return bad("bad header fields");
  if (ndim < 1 || ndim > 3 || !build_geo(ndim, dims, &f->g) || f->g.K != K ||
      f->g.stages.size() != S)
    return bad("bad geometry");
  f->st.assign(S, StageTab{});
  std::vector<uint64_t> nout(S);
  for (uint32_t t = 0; t < S; ++t) {
    const StageGeo& sg = f->g.stages[t];
    const uint32_t lv = g32(), dm = g32();
    const uint64_t nc = g64();
    f->st[t].H = (int32_t)g32();
    f->st[t].Q = g32();
    nout[t] = g64();
    if (!ok || (int)lv != sg.level || (int)dm != sg.dim3 - (3 - ndim) || nc != sg.ncodes ||
        f->st[t].H < -1 || f->st[t].H > 31 || nout[t] > nc)
      return bad("bad stage table");
  }
  std::vector<uint64_t> size(32 * (size_t)S);
  for (uint32_t t = 0; t < S; ++t)
    for (int k = 31; k >= 0; --k) size[32 * t + k] = g64();
  for (uint32_t t = 0; t < S; ++t) {
    if (!need(nout[t] * 16)) return bad("truncated outliers");
    for (uint64_t i = 0; i < nout[t]; ++i) {
      const uint64_t idx = g64();
      const double v = gd();
      if (idx >= f->g.stages[t].ncodes || (i && idx <= f->st[t].out_idx.back()))
        return bad("bad outlier list");
      f->st[t].out_idx.push_back(idx);
      f->st[t].out_val.push_back(v);
    }
  }
  if (!ok) return bad("truncated tables");
  const uint64_t mand = pos;
  // stream layout: read each nnz word and check the size follows from it
  uint64_t spos = pos;
  for (uint32_t t = 0; t < S; ++t) {
    const uint64_t W = f->g.stages[t].words;
    for (int k = 31; k >= 0; --k) {
      if (spos + 4 > len) return bad("truncated streams");
      uint32_t nnz = 0;
      for (int i = 0; i < 4; ++i) nnz |= uint32_t(p[spos + i]) << (8 * i);
      if (nnz > W || size[32 * t + k] != stream_bytes(nnz, W)) return bad("bad stream size");
      f->st[t].nnz[k] = nnz;
      spos += size[32 * t + k];
      if (spos > len) return bad("truncated streams");
    }
  }
  if (spos != len) return bad("trailing bytes");
  DeviceGuard dg(f->device);
  int rc = layout_field(f);
  if (rc) {
    f->tag = kDeadTag;
    delete f;
    return rc;
  }
  if (f->mandatory != mand) return bad("table size mismatch");
  cudaStream_t st = (cudaStream_t)stream;
  unsigned int* d_bad = nullptr;
  cudaError_t e = cudaSuccess;
  if (f->stream_bytes)
    e = cudaMemcpyAsync(f->d_blob, p + mand, f->stream_bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMalloc((void**)&d_bad, 4);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_bad, 0, 4, st);
  for (uint32_t t = 0; t < S && e == cudaSuccess; ++t) {
    StageArgs a = stage_args(f->g, f->g.stages[t], 0);
    e = launch_build_rank(a, f->desc[t], f->d_blob, f->d_rank, d_bad, st);
  }
  unsigned int hbad = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, d_bad, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (d_bad) cudaFree(d_bad);
  if (e != cudaSuccess) {
    free_field_device(f);
    f->tag = kDeadTag;
    delete f;
    return cuda_fail(e, "import");
  }
  if (hbad) return bad("bitmap population differs from the stream's nnz");
  rc = upload_outliers(f, st);
  if (rc) {
    free_field_device(f);
    f->tag = kDeadTag;
    delete f;
    return rc;
  }
  *out = f;
  return IPC_OK;
}

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
