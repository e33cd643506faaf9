/*
 * IPComp CPU ORACLE -- test infrastructure, not part of the product.
 *
 * Plain, slow, single-threaded restatement of the IPComp method
 * (arXiv 2502.04093). It is compiled with -O2 -ffp-contract=off so that every
 * floating-point operation below is one IEEE operation in the element type T,
 * in the order written. Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark load it; it shares no code with the CUDA library.
 *
 * Readings of the paper that this file fixes (the paper is silent or
 * ambiguous on them) are stated next to the code that implements them.
 *
 * Parity pins: every function here is pinned by a CPU test that does not
 * re-type its formula (brute force, closed forms, invariants, an independent
 * pure-Python restatement on tiny grids). See tests/test_oracle_*.py.
 */
#include "ipcomp_oracle.h"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

namespace {

/* ------------------------------------------------------------------------ */
/* Constants of the quantizer (Sec. 4.2.2): outlier radius R, the shrink of  */
/* the error check, and the unit roundoff u used by the strict bound.        */
/* ------------------------------------------------------------------------ */
template <class T> struct Prec;
template <> struct Prec<float> {
  static double radius() { return 2097152.0; }              /* 2^21 */
  static double shrink() { return 1.0 - 1.0 / 1048576.0; }  /* 1 - 2^-20 */
  static double unit() { return 1.0 / 16777216.0; }         /* 2^-24 */
};
template <> struct Prec<double> {
  static double radius() { return 1073741824.0; }                   /* 2^30 */
  static double shrink() { return 1.0 - 1.0 / 1125899906842624.0; } /* 1-2^-50 */
  static double unit() { return 1.0 / 9007199254740992.0; }         /* 2^-53 */
};

const uint32_t kMagic = 0x31435049u; /* "IPC1" */
const uint32_t kVersion = 1u;
const uint64_t kSat = (uint64_t)1 << 62; /* saturation of integer costs */

/* ------------------------------------------------------------------------ */
/* Geometry: levels and stages (Sec. 4.1, Fig. 3; Sec. 4.2.2).               */
/* Reading: dims are padded to 3 with leading 1s. K = ceil(log2 max N).      */
/* Level l (K..1) has stride s = 2^(l-1); inside a level one sweep per       */
/* dimension d = 0..2 (slowest first). Sweep d predicts the points whose     */
/* coordinate d is an odd multiple of s, whose coordinates e < d are         */
/* multiples of s, and whose coordinates e > d are multiples of 2s. Empty    */
/* sweeps are skipped. The origin is the anchor, stored exactly.             */
/* ------------------------------------------------------------------------ */
struct StageGeom {
  int level;
  int dim3;             /* sweep dimension in the padded 3-D index space */
  int64_t start[3], step[3], m[3];
  uint64_t ncodes, rows, wr, words;
};

struct Geometry {
  int ndim;
  int64_t N[3];
  int K;
  uint64_t n;
  std::vector<StageGeom> stages;
};

bool make_geometry(int ndim, const int64_t* dims, Geometry* g) {
  if (ndim < 1 || ndim > 3 || dims == nullptr) return false;
  g->ndim = ndim;
  for (int e = 0; e < 3; ++e) g->N[e] = 1;
  uint64_t n = 1;
  for (int e = 0; e < ndim; ++e) {
    if (dims[e] < 1) return false;
    g->N[3 - ndim + e] = dims[e];
    n *= (uint64_t)dims[e];
  }
  g->n = n;
  int64_t maxN = std::max(g->N[0], std::max(g->N[1], g->N[2]));
  int K = 0;
  while (((int64_t)1 << K) < maxN) ++K;
  g->K = K;
  g->stages.clear();
  for (int l = K; l >= 1; --l) {
    int64_t s = (int64_t)1 << (l - 1);
    for (int d = 0; d < 3; ++d) {
      StageGeom st;
      st.level = l;
      st.dim3 = d;
      uint64_t cnt = 1;
      for (int e = 0; e < 3; ++e) {
        if (e == d) { st.start[e] = s; st.step[e] = 2 * s; }
        else if (e < d) { st.start[e] = 0; st.step[e] = s; }
        else { st.start[e] = 0; st.step[e] = 2 * s; }
        st.m[e] = g->N[e] > st.start[e]
                      ? (g->N[e] - 1 - st.start[e]) / st.step[e] + 1 : 0;
        cnt *= (uint64_t)st.m[e];
      }
      if (cnt == 0) continue;
      st.ncodes = cnt;
      st.rows = (uint64_t)st.m[0] * (uint64_t)st.m[1];
      st.wr = ((uint64_t)st.m[2] + 31) / 32;
      st.words = st.rows * st.wr;
      g->stages.push_back(st);
    }
  }
  return true;
}

/* ------------------------------------------------------------------------ */
/* Interpolation predictor, Eq. 1 (linear) and Eq. 2 (cubic).                */
/* Reading at boundaries: cubic needs both i-3s and i+3s inside the line;    */
/* otherwise linear (Eq. 1) if i+s is inside; otherwise the left neighbour   */
/* is copied. Every rule has infinity-norm <= p (Sec. 5.1, p = 1 or 1.25).   */
/* Op order (fixed): u = b + c; v = a + d; w = 9u; z = w - v; pred = z/16.   */
/* interp 2 (cubic with quadratic boundaries, a predictor beyond the paper's */
/* two): where cubic lacks one outer neighbour, the quadratic through the    */
/* three points that exist -- (3b + 6c - d)/8 at the left end (i - 3s       */
/* outside), (-a + 6b + 3c)/8 at the right end -- instead of Eq. 1. Its      */
/* infinity-norm is (3 + 6 + 1)/8 = 1.25 = p of the cubic mode. Op order:    */
/* u = 3b; v = 6c; w = u + v; z = w - d; pred = z/8 (left), and u = 6b;      */
/* v = 3c; w = u + v; z = w - a; pred = z/8 (right).                         */
/* ------------------------------------------------------------------------ */
template <class T>
T predict(const T* xh, int64_t base, int64_t stride, int64_t i, int64_t s,
          int64_t N, int interp) {
  T b = xh[base + (i - s) * stride];
  if (i + s > N - 1) return b;
  T c = xh[base + (i + s) * stride];
  const bool left = i - 3 * s >= 0, right = i + 3 * s <= N - 1;
  if (interp >= 1 && left && right) {
    T a = xh[base + (i - 3 * s) * stride];
    T d = xh[base + (i + 3 * s) * stride];
    T u = b + c;
    T v = a + d;
    T w = (T)9 * u;
    T z = w - v;
    return z * (T)0.0625;
  }
  if (interp == 2 && right) {
    T d = xh[base + (i + 3 * s) * stride];
    T u = (T)3 * b;
    T v = (T)6 * c;
    T w = u + v;
    T z = w - d;
    return z * (T)0.125;
  }
  if (interp == 2 && left) {
    T a = xh[base + (i - 3 * s) * stride];
    T u = (T)6 * b;
    T v = (T)3 * c;
    T w = u + v;
    T z = w - a;
    return z * (T)0.125;
  }
  T u = b + c;
  return u * (T)0.5;
}

/* ------------------------------------------------------------------------ */
/* Negabinary (Sec. 4.4.2) and 2-prefix predictive XOR (Sec. 4.4.1).         */
/* ------------------------------------------------------------------------ */
uint32_t negabinary(int32_t q) {
  return ((uint32_t)q + 0xAAAAAAAAu) ^ 0xAAAAAAAAu;
}
int64_t negabinary_inv(uint32_t n) {
  return (int64_t)(n ^ 0xAAAAAAAAu) - (int64_t)0xAAAAAAAAu;
}
/* encoded bit k = n_k xor n_{k+1} xor n_{k+2}; missing prefix bits are 0. */
uint32_t xor_encode(uint32_t n) {
  uint32_t e = 0;
  for (int k = 31; k >= 0; --k) {
    uint32_t nk = (n >> k) & 1u;
    uint32_t p1 = k + 1 <= 31 ? (n >> (k + 1)) & 1u : 0u;
    uint32_t p2 = k + 2 <= 31 ? (n >> (k + 2)) & 1u : 0u;
    e |= (nk ^ p1 ^ p2) << k;
  }
  return e;
}
/* decode top-down: the two more significant digits are already known. */
uint32_t xor_decode(uint32_t e) {
  uint32_t n = 0;
  for (int k = 31; k >= 0; --k) {
    uint32_t ek = (e >> k) & 1u;
    uint32_t p1 = k + 1 <= 31 ? (n >> (k + 1)) & 1u : 0u;
    uint32_t p2 = k + 2 <= 31 ? (n >> (k + 2)) & 1u : 0u;
    n |= (ek ^ p1 ^ p2) << k;
  }
  return n;
}
uint32_t plane_mask(int b) { /* keep planes >= b */
  return b >= 32 ? 0u : ~((1u << b) - 1u);
}
int msb_index(uint32_t v) {
  int h = -1;
  for (int k = 0; k < 32; ++k)
    if ((v >> k) & 1u) h = k;
  return h;
}

/* Uncertainty of d dropped negabinary digits (Sec. 4.4.2): the largest
 * |value| that d digits can hold, (2/3)2^d - 1/3 (d odd), (2/3)2^d - 2/3
 * (d even). */
uint64_t uncertainty(int d) {
  if (d <= 0) return 0;
  uint64_t p = (uint64_t)1 << (d + 1);
  return (d % 2 == 1) ? (p - 1) / 3 : (p - 2) / 3;
}

/* Half bin width of the quantizer. Reading of Sec. 4.2.2: |y - yhat| <= eb
 * must hold for the value reconstructed in the element type, whose two
 * roundings (q*bin and pred + r) add up to about 3u(max|x| + eb); the half
 * bin is eb shrunk by 4u(max|x| + eb), but never below eb/2 (where the
 * shrink would pass eb/2, the outlier check takes over). */
double half_bin(double eb, double xmaxabs, int dtype) {
  const double u = dtype == 0 ? Prec<float>::unit() : Prec<double>::unit();
  double eq = eb - 4.0 * u * (xmaxabs + eb);
  if (!(eq >= 0.5 * eb)) eq = 0.5 * eb;
  return eq;
}

/* ------------------------------------------------------------------------ */
/* Little-endian byte writer/reader for the container.                       */
/* ------------------------------------------------------------------------ */
struct Writer {
  std::vector<uint8_t> buf;
  void u32(uint32_t v) { for (int i = 0; i < 4; ++i) buf.push_back((uint8_t)(v >> (8 * i))); }
  void u64(uint64_t v) { for (int i = 0; i < 8; ++i) buf.push_back((uint8_t)(v >> (8 * i))); }
  void f64(double v) { uint64_t u; std::memcpy(&u, &v, 8); u64(u); }
};
struct Reader {
  const uint8_t* p;
  uint64_t len, pos;
  bool ok;
  bool need(uint64_t k) { if (pos + k > len || pos + k < pos) { ok = false; return false; } return true; }
  uint32_t u32() { if (!need(4)) return 0; uint32_t v = 0; for (int i = 0; i < 4; ++i) v |= (uint32_t)p[pos + i] << (8 * i); pos += 4; return v; }
  uint64_t u64() { if (!need(8)) return 0; uint64_t v = 0; for (int i = 0; i < 8; ++i) v |= (uint64_t)p[pos + i] << (8 * i); pos += 8; return v; }
  double f64() { uint64_t u = u64(); double v; std::memcpy(&v, &u, 8); return v; }
};

/* ------------------------------------------------------------------------ */
/* Plane stream (replaces zstd of Sec. 6.2.1): u32 nnz, then nothing        */
/* (nnz = 0), a zero-word bitmap + the nonzero words (when that is smaller   */
/* than W words), else all W words.                                          */
/* ------------------------------------------------------------------------ */
void encode_stream(const std::vector<uint32_t>& words, Writer* w) {
  uint64_t W = words.size(), nnz = 0;
  for (uint32_t v : words) nnz += (v != 0);
  w->u32((uint32_t)nnz);
  if (nnz == 0) return;
  uint64_t bm = (W + 31) / 32;
  if (bm + nnz < W) {
    for (uint64_t j = 0; j < bm; ++j) {
      uint32_t bits = 0;
      for (uint64_t i = 0; i < 32 && 32 * j + i < W; ++i)
        if (words[32 * j + i] != 0) bits |= 1u << i;
      w->u32(bits);
    }
    for (uint32_t v : words)
      if (v != 0) w->u32(v);
  } else {
    for (uint32_t v : words) w->u32(v);
  }
}

bool decode_stream(const uint8_t* p, uint64_t size, uint64_t W,
                   std::vector<uint32_t>* words) {
  Reader r{p, size, 0, true};
  words->assign(W, 0);
  uint64_t nnz = r.u32();
  if (!r.ok || nnz > W) return false;
  if (nnz == 0) return size == 4;
  uint64_t bm = (W + 31) / 32;
  if (bm + nnz < W) {
    if (size != 4 + 4 * (bm + nnz)) return false;
    std::vector<uint32_t> bits(bm);
    for (uint64_t j = 0; j < bm; ++j) bits[j] = r.u32();
    uint64_t cnt = 0;
    for (uint64_t w = 0; w < W; ++w) {
      if ((bits[w / 32] >> (w % 32)) & 1u) {
        if (cnt == nnz) return false;
        (*words)[w] = r.u32();
        if ((*words)[w] == 0) return false;
        ++cnt;
      }
    }
    return cnt == nnz && r.ok;
  }
  if (size != 4 + 4 * W) return false;
  uint64_t cnt = 0;
  for (uint64_t w = 0; w < W; ++w) {
    (*words)[w] = r.u32();
    cnt += ((*words)[w] != 0);
  }
  return cnt == nnz && r.ok;
}

}  // namespace

/* ------------------------------------------------------------------------ */
/* The compressed field.                                                     */
/* ------------------------------------------------------------------------ */
struct StageData {
  int32_t H;
  uint32_t Q;
  std::vector<std::pair<uint64_t, double>> outliers; /* (code index, value) */
  uint64_t size[32];                                 /* indexed by plane k */
  uint64_t offset[32];                               /* into `bytes` */
};

struct ipco_field {
  int dtype, interp, bound, eb_mode;
  double eb_user, eb, xmin, xmax, xmaxabs, anchor;
  Geometry g;
  std::vector<StageData> st;
  std::vector<uint8_t> bytes; /* the whole container */
  uint64_t mandatory;
  std::vector<std::vector<int32_t>> codes; /* kept after compress (tests) */
  /* Which bound on |q - q'_b| the cost tables use: 0 the closed form of
   * stage_M (the container's model), 1 the data maximum `mdata` (a study of
   * the table Sec. 5.1 says can be precomputed; needs `codes`). */
  int delta_model = 0;
  std::vector<std::vector<uint64_t>> mdata; /* per stage, b = 0..32 */
};

struct ipco_view {
  const ipco_field* f;
  std::vector<int> b; /* b[l-1] */
  uint64_t bytes;
  double bound;
  /* State of Algorithm 2: per stage, the loaded negabinary digits of every
   * code (planes >= b_l, the others zero), and the rounding allowance, in
   * units of eb * 2^-16, that the current reconstruction carries against the
   * compressor's values (the rounding margins of a fresh selection, plus
   * the margin of every incremental step since). */
  std::vector<std::vector<uint32_t>> N;
  uint64_t racc = 0;
};

namespace {

/* Element-type specific compression: range, quantized sweeps, streams. */
template <class T>
int compress_t(const T* x, ipco_field* f) {
  const Geometry& g = f->g;
  /* Range over finite values (Sec. 3.1.1: value range used by PSNR and by
   * relative error bounds). */
  double mn = 0, mx = 0, ma = 0;
  bool any = false;
  for (uint64_t i = 0; i < g.n; ++i) {
    double v = (double)x[i];
    if (!std::isfinite(v)) continue;
    if (!any) { mn = mx = v; any = true; }
    mn = std::min(mn, v);
    mx = std::max(mx, v);
    ma = std::max(ma, std::fabs(v));
  }
  f->xmin = mn; f->xmax = mx; f->xmaxabs = ma;
  double eb = f->eb_user;
  if (f->eb_mode == 1) {
    if (!any) return IPCO_EINVAL;
    double range = mx - mn;
    eb = range > 0 ? f->eb_user * range : f->eb_user;
  }
  if (!(eb > 0) || !std::isfinite(eb)) return IPCO_EINVAL;
  f->eb = eb;
  f->anchor = (double)x[0];

  /* Quantizer constants (Sec. 4.2.2): the reconstructed value in T must be
   * within eb of x, so the bin is 2 e_q with e_q = eb minus the rounding of
   * pred + q*bin in T (see half_bin). */
  const double eq = half_bin(eb, ma, sizeof(T) == 4 ? 0 : 1);
  const T inv2eb = (T)(1.0 / (2.0 * eq));
  const T twoeb = (T)(2.0 * eq);
  const T ebchk = (T)(eb * Prec<T>::shrink());
  const T R = (T)Prec<T>::radius();
  const bool cubic = f->interp >= 1;  /* p = 1.25, kappa 24 */

  std::vector<T> xh(g.n);
  xh[0] = x[0];
  const int64_t stride[3] = {g.N[1] * g.N[2], g.N[2], 1};
  f->codes.assign(g.stages.size(), {});
  f->st.assign(g.stages.size(), StageData());
  for (size_t t = 0; t < g.stages.size(); ++t) {
    const StageGeom& sg = g.stages[t];
    const int d = sg.dim3;
    const int64_t s = (int64_t)1 << (sg.level - 1);
    std::vector<int32_t>& q = f->codes[t];
    q.assign(sg.ncodes, 0);
    StageData& sd = f->st[t];
    uint64_t ci = 0;
    for (int64_t c0 = 0; c0 < sg.m[0]; ++c0)
      for (int64_t c1 = 0; c1 < sg.m[1]; ++c1)
        for (int64_t c2 = 0; c2 < sg.m[2]; ++c2, ++ci) {
          int64_t i[3] = {sg.start[0] + c0 * sg.step[0],
                          sg.start[1] + c1 * sg.step[1],
                          sg.start[2] + c2 * sg.step[2]};
          int64_t idx = i[0] * stride[0] + i[1] * stride[1] + i[2];
          int64_t base = idx - i[d] * stride[d];
          T pred = predict<T>(xh.data(), base, stride[d], i[d], s, g.N[d], f->interp);
          /* y = x - P xhat; quantize to the nearest multiple of 2eb. */
          T xv = x[idx];
          T diff = xv - pred;
          T tq = diff * inv2eb;
          bool outlier = !(std::fabs(tq) <= R);
          T rec = xv;
          int32_t code = 0;
          if (!outlier) {
            T qf = std::nearbyint(tq);
            T r = qf * twoeb;
            rec = pred + r;
            T err = xv - rec;
            if (!(std::fabs(err) <= ebchk)) outlier = true;
            else code = (int32_t)qf;
          }
          if (outlier) {
            rec = xv;
            code = 0;
            sd.outliers.push_back({ci, (double)xv});
          }
          xh[idx] = rec;
          q[ci] = code;
        }
  }

  /* Per-stage statistics for the error bound (Sec. 5.1): H = msb of the OR
   * of all negabinary codes, Q = max |q|. */
  for (size_t t = 0; t < g.stages.size(); ++t) {
    uint32_t orv = 0, qmax = 0;
    for (int32_t v : f->codes[t]) {
      orv |= negabinary(v);
      uint32_t a = v < 0 ? (uint32_t)(-(int64_t)v) : (uint32_t)v;
      qmax = std::max(qmax, a);
    }
    f->st[t].H = msb_index(orv);
    f->st[t].Q = qmax;
  }
  return IPCO_OK;
}

/* Build the word array of plane k of stage t (Sec. 4.3: the bits of the same
 * position across the integers form a plane). Word (r, j) bit i holds code
 * (r, 32j + i) of the row-major code order; a row's last word is zero-padded.*/
void plane_words(const StageGeom& sg, const std::vector<uint32_t>& E, int k,
                 std::vector<uint32_t>* out) {
  out->assign(sg.words, 0);
  const uint64_t m = (uint64_t)sg.m[2];
  for (uint64_t r = 0; r < sg.rows; ++r)
    for (uint64_t j = 0; j < sg.wr; ++j) {
      uint32_t w = 0;
      for (uint64_t i = 0; i < 32; ++i) {
        uint64_t p = 32 * j + i;
        if (p >= m) break;
        w |= ((E[r * m + p] >> k) & 1u) << i;
      }
      (*out)[r * sg.wr + j] = w;
    }
}

void serialize(ipco_field* f) {
  const Geometry& g = f->g;
  const uint32_t S = (uint32_t)g.stages.size();
  Writer w;
  w.u32(kMagic); w.u32(kVersion);
  w.u32((uint32_t)f->dtype); w.u32((uint32_t)f->interp);
  w.u32((uint32_t)f->bound); w.u32((uint32_t)g.ndim);
  for (int e = 0; e < 3; ++e)
    w.u64(e < g.ndim ? (uint64_t)g.N[3 - g.ndim + e] : 0);
  w.u32((uint32_t)f->eb_mode); w.u32((uint32_t)g.K);
  w.f64(f->eb_user); w.f64(f->eb);
  w.f64(f->xmin); w.f64(f->xmax); w.f64(f->xmaxabs); w.f64(f->anchor);
  w.u32(S); w.u32(0);
  /* Stream bytes are produced first so the size table can be written. */
  std::vector<std::vector<uint8_t>> streams(S * 32);
  std::vector<uint32_t> words, E;
  for (uint32_t t = 0; t < S; ++t) {
    /* the predictively coded negabinary form of every code of the stage */
    E.resize(f->codes[t].size());
    for (size_t c = 0; c < E.size(); ++c) E[c] = xor_encode(negabinary(f->codes[t][c]));
    for (int k = 31; k >= 0; --k) {
      plane_words(g.stages[t], E, k, &words);
      Writer sw;
      encode_stream(words, &sw);
      f->st[t].size[k] = sw.buf.size();
      streams[t * 32 + (31 - k)] = std::move(sw.buf);
    }
  }
  for (uint32_t t = 0; t < S; ++t) {
    const StageGeom& sg = g.stages[t];
    w.u32((uint32_t)sg.level);
    w.u32((uint32_t)(sg.dim3 - (3 - g.ndim)));
    w.u64(sg.ncodes);
    w.u32((uint32_t)f->st[t].H);
    w.u32(f->st[t].Q);
    w.u64(f->st[t].outliers.size());
  }
  for (uint32_t t = 0; t < S; ++t)
    for (int k = 31; k >= 0; --k) w.u64(f->st[t].size[k]);
  for (uint32_t t = 0; t < S; ++t)
    for (auto& o : f->st[t].outliers) { w.u64(o.first); w.f64(o.second); }
  f->mandatory = w.buf.size();
  for (uint32_t t = 0; t < S; ++t)
    for (int k = 31; k >= 0; --k) {
      f->st[t].offset[k] = w.buf.size();
      auto& sb = streams[t * 32 + (31 - k)];
      w.buf.insert(w.buf.end(), sb.begin(), sb.end());
    }
  f->bytes = std::move(w.buf);
}

/* ------------------------------------------------------------------------ */
/* Error cost of a per-level choice (Theorem 1, Sec. 5.1-5.2).               */
/* M[t][b] bounds |q - q'_b| over the codes of stage t when its b low planes */
/* are dropped: 0 for b = 0; the uncertainty U(b) while b <= H; the stored   */
/* maximum |q| once every nonzero digit is dropped (b > H).                  */
/* Strict mode amplifies stage t by p^(S-1-t) (each later sweep is one more  */
/* application of an interpolation of norm p) and adds a rounding margin.   */
/* Paper mode uses p^(l-1) times the largest stage term of level l.          */
/* Costs are integers in units of eb * 2^-16.                                */
/* ------------------------------------------------------------------------ */
uint64_t sat_add(uint64_t a, uint64_t b) { uint64_t c = a + b; return (c < a || c > kSat) ? kSat : c; }
uint64_t ceil_units(double v) {
  if (!(v < (double)kSat)) return kSat;
  if (v <= 0) return 0;
  return (uint64_t)std::ceil(v);
}

uint64_t stage_M(const StageData& sd, int b) {
  if (b <= 0) return 0;
  if (b <= sd.H) return uncertainty(b);
  return sd.Q;
}

/* The data maximum of |q - q'_b| over a stage's codes, b = 0..32. Since a
 * negabinary value is the sum of its digits' values, q - q'_b is the value
 * of the b dropped low digits alone: per code, the partial sums of
 * digit_k * (-2)^k, k < b, and their largest magnitude over the codes. */
void delta_data(const std::vector<int32_t>& q, std::vector<uint64_t>* out) {
  out->assign(33, 0);
  for (int32_t v : q) {
    const uint32_t n = negabinary(v);
    int64_t low = 0, w = 1; /* value of digits 0 .. k; w = (-2)^k */
    for (int k = 0; k < 32; ++k) {
      if ((n >> k) & 1u) low += w;
      w *= -2;
      const uint64_t a = (uint64_t)(low < 0 ? -low : low);
      if (a > (*out)[k + 1]) (*out)[k + 1] = a;
    }
  }
}

uint64_t stage_M(const ipco_field* f, int t, int b) {
  if (f->delta_model == 1) return b <= 0 ? 0 : f->mdata[t][b];
  return stage_M(f->st[t], b);
}

struct Options {
  std::vector<uint64_t> cost;  /* K x 33 */
  std::vector<uint64_t> bytes; /* K x 33 */
  std::vector<uint64_t> rho;   /* K: the rounding margin in cost(l, b > 0) */
};

void option_tables(const ipco_field* f, double A, Options* o) {
  const Geometry& g = f->g;
  const int K = g.K, S = (int)g.stages.size();
  const bool cubic = f->interp >= 1;  /* p = 1.25, kappa 24 */
  const double p = cubic ? 1.25 : 1.0;
  std::vector<double> P(std::max(S, K) + 1);
  P[0] = 1.0;
  for (size_t i = 1; i < P.size(); ++i) P[i] = P[i - 1] * p;
  const double eq = half_bin(f->eb, f->xmaxabs, f->dtype);
  double twoeb_T = f->dtype == 0 ? (double)(float)(2.0 * eq) : 2.0 * eq;
  double bin = twoeb_T / f->eb;
  double u = f->dtype == 0 ? Prec<float>::unit() : Prec<double>::unit();
  /* kappa bounds the rounding of one stage, in units of u * A, summed over
   * the two computations whose difference it covers (compressor and
   * retriever). With |a|,|b|,|c|,|d| <= A: u = b + c and v = a + d round by
   * at most 2A u each, w = 9u by 18A u, z = w - v by 20A u; the u-error
   * enters w nine times. pred = z / 16 is exact, so the stencil's rounding
   * reaches pred divided by 16: (9*2 + 2 + 18 + 20) A u / 16 < 3.7 A u. The
   * scaled code r = q * bin (|r| <= 2.25A, x - pred with |pred| <= 1.25A)
   * and xhat = pred + r (|xhat| <= A) add 2.25 A u and A u: 6.9 A u per
   * computation, 13.8 A u for the two. kappa = 24 keeps a 1.7x headroom.
   * Linear: b + c rounds by 2A u, halved by the exact * 0.5, then r (2A u)
   * and xhat (A u): 4A u per computation, 8A u for two; kappa = 12 keeps a
   * 1.5x headroom. */
  double kappa = cubic ? 24.0 : 12.0;
  o->cost.assign((size_t)K * 33, 0);
  o->bytes.assign((size_t)K * 33, 0);
  o->rho.assign((size_t)K, 0);
  for (int l = 1; l <= K; ++l) {
    /* rounding margin: every stage at this level or finer recomputes. */
    double asum = 0;
    for (int t = 0; t < S; ++t)
      if (g.stages[t].level <= l) asum += (f->bound == 0 && cubic) ? P[S - 1 - t] : 1.0;
    uint64_t rho = ceil_units(kappa * u * (A / f->eb) * 65536.0 * asum);
    o->rho[l - 1] = f->bound == 0 ? rho : 0;
    for (int b = 0; b <= 32; ++b) {
      uint64_t c = 0, y = 0;
      uint64_t mmax = 0;
      for (int t = 0; t < S; ++t) {
        if (g.stages[t].level != l) continue;
        uint64_t M = stage_M(f, t, b);
        if (f->bound == 0) {
          double a = cubic ? P[S - 1 - t] : 1.0;
          c = sat_add(c, ceil_units(a * (double)M * bin * 65536.0));
        } else {
          mmax = std::max(mmax, M);
        }
        for (int k = b; k < 32; ++k) y += f->st[t].size[k];
      }
      if (f->bound == 0) {
        if (b > 0) c = sat_add(c, rho);
      } else {
        c = ceil_units(P[l - 1] * (double)mmax * bin * 65536.0);
      }
      o->cost[(size_t)(l - 1) * 33 + b] = c;
      o->bytes[(size_t)(l - 1) * 33 + b] = y;
    }
  }
}

/* Exact knapsack over levels (Sec. 5.2 eb mode, Sec. 5.3 bitrate mode),
 * solved on the Pareto frontier of (cost, bytes) instead of a discretised
 * error grid. Ties: fewer bytes (eb) / smaller cost (bitrate), then the other
 * objective, then the lexicographically larger (b_1, b_2, ...). */
struct Entry {
  uint64_t c, y;
  std::vector<int> b; /* b_1 .. b_j */
};
bool lex_greater(const std::vector<int>& a, const std::vector<int>& b) {
  for (size_t i = 0; i < a.size() && i < b.size(); ++i)
    if (a[i] != b[i]) return a[i] > b[i];
  return false;
}

int select_levels(const Options& o, int K, int kind, uint64_t limit,
                  const std::vector<int>* upper, std::vector<int>* best) {
  std::vector<Entry> F(1);
  F[0].c = 0; F[0].y = 0;
  for (int l = 1; l <= K; ++l) {
    std::vector<Entry> G;
    int bmax = upper ? (*upper)[l - 1] : 32;
    for (const Entry& e : F)
      for (int b = 0; b <= bmax; ++b) {
        Entry n;
        n.c = sat_add(e.c, o.cost[(size_t)(l - 1) * 33 + b]);
        n.y = e.y + o.bytes[(size_t)(l - 1) * 33 + b];
        if (kind == 0 && n.c > limit) continue;
        if (kind == 1 && n.y > limit) continue;
        n.b = e.b;
        n.b.push_back(b);
        G.push_back(std::move(n));
      }
    std::sort(G.begin(), G.end(), [](const Entry& a, const Entry& b) {
      if (a.c != b.c) return a.c < b.c;
      if (a.y != b.y) return a.y < b.y;
      return lex_greater(a.b, b.b);
    });
    F.clear();
    for (Entry& e : G)
      if (F.empty() || e.y < F.back().y) F.push_back(std::move(e));
    if (F.empty()) return kind == 0 ? IPCO_EBOUND : IPCO_EBUDGET;
  }
  /* Frontier: cost strictly increasing, bytes strictly decreasing. */
  *best = kind == 0 ? F.back().b : F.front().b;
  return IPCO_OK;
}

uint64_t loaded_bytes(const ipco_field* f, const std::vector<int>& b) {
  uint64_t y = f->mandatory;
  for (size_t t = 0; t < f->g.stages.size(); ++t)
    for (int k = b[f->g.stages[t].level - 1]; k < 32; ++k) y += f->st[t].size[k];
  return y;
}

uint64_t total_cost(const Options& o, const std::vector<int>& b) {
  uint64_t c = 0;
  for (size_t l = 0; l < b.size(); ++l) c = sat_add(c, o.cost[l * 33 + b[l]]);
  return c;
}

double range_of(const ipco_field* f) { return f->xmax - f->xmin; }

/* Choose a selection for a target. Returns the selection, bytes and the
 * guaranteed L-inf bound (absolute). upper != null constrains b'_l <= b_l. */
uint64_t rounding_part(const Options& o, const std::vector<int>& b) {
  uint64_t r = 0;
  for (size_t l = 0; l < b.size(); ++l)
    if (b[l] > 0) r = sat_add(r, o.rho[l]);
  return r;
}

/* rparts (optional): [0] = the rounding margins in the selection's cost
 * (sum of rho_l over levels with b_l > 0), [1] = the rest (truncation). */
int choose(const ipco_field* f, int kind, double value,
           const std::vector<int>* upper, std::vector<int>* b,
           uint64_t* bytes, double* bound, uint64_t* rparts = nullptr) {
  const int K = f->g.K;
  if (!std::isfinite(value)) return IPCO_EINVAL;
  Options o;
  if (kind == 0) {
    double E = value;
    if (f->eb_mode == 1) { double r = range_of(f); E = r > 0 ? value * r : value; }
    if (!(E >= f->eb)) return IPCO_EBOUND;
    double A = f->xmaxabs + E;
    option_tables(f, A, &o);
    double Bd = std::floor(((E - f->eb) / f->eb) * 65536.0);
    uint64_t B = Bd >= (double)kSat ? kSat : (uint64_t)Bd;
    int rc = select_levels(o, K, 0, B, upper, b);
    if (rc) return rc;
    *bytes = loaded_bytes(f, *b);
    *bound = f->eb + (double)total_cost(o, *b) * f->eb / 65536.0;
    if (rparts) { rparts[0] = rounding_part(o, *b); rparts[1] = total_cost(o, *b) - rparts[0]; }
    return IPCO_OK;
  }
  if (kind == 1) {
    if (!(value >= 0)) return IPCO_EINVAL;
    double Sd = std::floor(value * (double)f->g.n / 8.0);
    uint64_t Sb = Sd >= 1.8e19 ? ~(uint64_t)0 : (uint64_t)Sd;
    if (f->mandatory > Sb) return IPCO_EBUDGET;
    double A = f->xmaxabs + std::max(range_of(f), f->eb);
    option_tables(f, A, &o);
    int rc = select_levels(o, K, 1, Sb - f->mandatory, upper, b);
    if (rc) return rc;
    *bytes = loaded_bytes(f, *b);
    double G = f->eb + (double)total_cost(o, *b) * f->eb / 65536.0;
    /* The rounding margin assumed |values| <= xmaxabs + range; widen A until
     * it covers the reported bound. */
    for (int it = 0; it < 16 && G > A - f->xmaxabs; ++it) {
      A = f->xmaxabs + G;
      option_tables(f, A, &o);
      G = f->eb + (double)total_cost(o, *b) * f->eb / 65536.0;
    }
    *bound = G;
    if (rparts) { rparts[0] = rounding_part(o, *b); rparts[1] = total_cost(o, *b) - rparts[0]; }
    return IPCO_OK;
  }
  return IPCO_EINVAL;
}

/* Reconstruction (Algorithm 1) from the container bytes: decode the selected
 * planes of every stage, undo the predictive XOR top-down, zero the dropped
 * digits, map negabinary back to q', and rebuild xhat' = P xhat' + q' 2eb in
 * the compressor's op order. Outliers take their stored value. */
template <class T>
int reconstruct_t(const ipco_field* f, const std::vector<int>& bsel, T* out) {
  const Geometry& g = f->g;
  const T twoeb = (T)(2.0 * half_bin(f->eb, f->xmaxabs, f->dtype));
  const bool cubic = f->interp >= 1;  /* p = 1.25, kappa 24 */
  const int64_t stride[3] = {g.N[1] * g.N[2], g.N[2], 1};
  out[0] = (T)f->anchor;
  std::vector<uint32_t> words;
  for (size_t t = 0; t < g.stages.size(); ++t) {
    const StageGeom& sg = g.stages[t];
    const StageData& sd = f->st[t];
    const int b = bsel[sg.level - 1];
    const uint64_t m = (uint64_t)sg.m[2];
    std::vector<uint32_t> E(sg.ncodes, 0);
    for (int k = 31; k >= b; --k) {
      if (!decode_stream(f->bytes.data() + sd.offset[k], sd.size[k], sg.words, &words))
        return IPCO_ECORRUPT;
      for (uint64_t r = 0; r < sg.rows; ++r)
        for (uint64_t j = 0; j < sg.wr; ++j) {
          uint32_t w = words[r * sg.wr + j];
          for (uint64_t i = 0; i < 32 && 32 * j + i < m; ++i)
            E[r * m + 32 * j + i] |= ((w >> i) & 1u) << k;
        }
    }
    const int d = sg.dim3;
    const int64_t s = (int64_t)1 << (sg.level - 1);
    size_t oi = 0;
    uint64_t ci = 0;
    for (int64_t c0 = 0; c0 < sg.m[0]; ++c0)
      for (int64_t c1 = 0; c1 < sg.m[1]; ++c1)
        for (int64_t c2 = 0; c2 < sg.m[2]; ++c2, ++ci) {
          int64_t i[3] = {sg.start[0] + c0 * sg.step[0],
                          sg.start[1] + c1 * sg.step[1],
                          sg.start[2] + c2 * sg.step[2]};
          int64_t idx = i[0] * stride[0] + i[1] * stride[1] + i[2];
          if (oi < sd.outliers.size() && sd.outliers[oi].first == ci) {
            out[idx] = (T)sd.outliers[oi].second;
            ++oi;
            continue;
          }
          int64_t base = idx - i[d] * stride[d];
          T pred = predict<T>(out, base, stride[d], i[d], s, g.N[d], f->interp);
          uint32_t N = xor_decode(E[ci]) & plane_mask(b);
          int64_t qv = negabinary_inv(N);
          T r = (T)qv * twoeb;
          out[idx] = pred + r;
        }
  }
  return IPCO_OK;
}

int reconstruct(const ipco_field* f, const std::vector<int>& b, void* out) {
  if (f->dtype == 0) return reconstruct_t<float>(f, b, (float*)out);
  return reconstruct_t<double>(f, b, (double*)out);
}

/* ------------------------------------------------------------------------ */
/* Incremental reconstruction (Algorithm 2, Sec. 4.3).                       */
/* Reading: a refinement loads only the encoded planes b'_l .. b_l - 1 of   */
/* each level. Each new digit is decoded from its encoded bit and the two   */
/* more significant digits (Sec. 4.4.1); for the top two new planes those   */
/* are the lowest two loaded digits, which the view keeps. The increment of */
/* a code, dq, is the value of its new digits; it is dequantized            */
/* (dq * 2e_q) and interpolated level by level from zero -- the Delta of    */
/* Algorithm 2, zero at outliers, whose values are exact already -- and     */
/* x^new = x^old + Delta wherever Delta is not zero.                        */
/* ------------------------------------------------------------------------ */

/* The loaded digits (planes >= b) of every code of stage t. */
int loaded_digits(const ipco_field* f, size_t t, int b, std::vector<uint32_t>* N) {
  const StageGeom& sg = f->g.stages[t];
  const StageData& sd = f->st[t];
  const uint64_t m = (uint64_t)sg.m[2];
  std::vector<uint32_t> E(sg.ncodes, 0), words;
  for (int k = 31; k >= b; --k) {
    if (!decode_stream(f->bytes.data() + sd.offset[k], sd.size[k], sg.words, &words))
      return IPCO_ECORRUPT;
    for (uint64_t r = 0; r < sg.rows; ++r)
      for (uint64_t j = 0; j < sg.wr; ++j)
        for (uint64_t i = 0; i < 32 && 32 * j + i < m; ++i)
          E[r * m + 32 * j + i] |= ((words[r * sg.wr + j] >> i) & 1u) << k;
  }
  N->assign(sg.ncodes, 0);
  for (uint64_t ci = 0; ci < sg.ncodes; ++ci) (*N)[ci] = xor_decode(E[ci]) & plane_mask(b);
  return IPCO_OK;
}

int all_loaded_digits(const ipco_field* f, const std::vector<int>& b,
                      std::vector<std::vector<uint32_t>>* N) {
  N->assign(f->g.stages.size(), {});
  for (size_t t = 0; t < f->g.stages.size(); ++t) {
    int rc = loaded_digits(f, t, b[f->g.stages[t].level - 1], &(*N)[t]);
    if (rc) return rc;
  }
  return IPCO_OK;
}

/* Digits bn .. bo-1 of one code, from its encoded bits e (only those planes
 * are read) and its loaded digits nold (planes >= bo, the rest zero),
 * decoded top-down. Returns the new digits alone. */
uint32_t decode_window(uint32_t e, uint32_t nold, int bn, int bo) {
  uint32_t n = nold;
  for (int k = bo - 1; k >= bn; --k) {
    const uint32_t ek = (e >> k) & 1u;
    const uint32_t p1 = k + 1 <= 31 ? (n >> (k + 1)) & 1u : 0u;
    const uint32_t p2 = k + 2 <= 31 ? (n >> (k + 2)) & 1u : 0u;
    n |= (ek ^ p1 ^ p2) << k;
  }
  return n & plane_mask(bn) & ~plane_mask(bo);
}

/* Algorithm 2 on the host: Delta from the new planes, then out += Delta.
 * On success N holds the digits of the new selection. */
template <class T>
int delta_t(const ipco_field* f, const std::vector<int>& bold, const std::vector<int>& bnew,
            std::vector<std::vector<uint32_t>>* N, T* out) {
  const Geometry& g = f->g;
  const T twoeb = (T)(2.0 * half_bin(f->eb, f->xmaxabs, f->dtype));
  const bool cubic = f->interp >= 1;  /* p = 1.25, kappa 24 */
  const int64_t stride[3] = {g.N[1] * g.N[2], g.N[2], 1};
  std::vector<T> D(g.n, (T)0);  /* Delta; the anchor never changes */
  std::vector<std::vector<uint32_t>> Nn = *N;
  std::vector<uint32_t> words;
  for (size_t t = 0; t < g.stages.size(); ++t) {
    const StageGeom& sg = g.stages[t];
    const StageData& sd = f->st[t];
    const int bo = bold[sg.level - 1], bn = bnew[sg.level - 1];
    const uint64_t m = (uint64_t)sg.m[2];
    /* the encoded bits of the new planes only */
    std::vector<uint32_t> E(sg.ncodes, 0);
    for (int k = bo - 1; k >= bn; --k) {
      if (!decode_stream(f->bytes.data() + sd.offset[k], sd.size[k], sg.words, &words))
        return IPCO_ECORRUPT;
      for (uint64_t r = 0; r < sg.rows; ++r)
        for (uint64_t j = 0; j < sg.wr; ++j)
          for (uint64_t i = 0; i < 32 && 32 * j + i < m; ++i)
            E[r * m + 32 * j + i] |= ((words[r * sg.wr + j] >> i) & 1u) << k;
    }
    const int d = sg.dim3;
    const int64_t s = (int64_t)1 << (sg.level - 1);
    size_t oi = 0;
    uint64_t ci = 0;
    for (int64_t c0 = 0; c0 < sg.m[0]; ++c0)
      for (int64_t c1 = 0; c1 < sg.m[1]; ++c1)
        for (int64_t c2 = 0; c2 < sg.m[2]; ++c2, ++ci) {
          int64_t i[3] = {sg.start[0] + c0 * sg.step[0],
                          sg.start[1] + c1 * sg.step[1],
                          sg.start[2] + c2 * sg.step[2]};
          int64_t idx = i[0] * stride[0] + i[1] * stride[1] + i[2];
          if (oi < sd.outliers.size() && sd.outliers[oi].first == ci) {
            D[idx] = (T)0;  /* an outlier's value is exact: no increment */
            ++oi;
            continue;
          }
          int64_t base = idx - i[d] * stride[d];
          T pred = predict<T>(D.data(), base, stride[d], i[d], s, g.N[d], f->interp);
          uint32_t nd = bn < bo ? decode_window(E[ci], (*N)[t][ci], bn, bo) : 0u;
          int64_t dq = negabinary_inv(nd);  /* value of the new digits */
          T r = (T)dq * twoeb;
          D[idx] = pred + r;
          Nn[t][ci] |= nd;
        }
  }
  for (uint64_t i = 0; i < g.n; ++i)
    if (D[i] != (T)0) out[i] = out[i] + D[i];
  *N = std::move(Nn);
  return IPCO_OK;
}

/* Guaranteed bound of an incremental result (strict mode). Relative to the
 * compressor's values, x^old + Delta differs from the truncated exact
 * reconstruction of the new selection by the old result's rounding (the
 * view's allowance), the rounding of Delta and that of the final addition.
 * Delta is interpolated from zero, so it is exactly zero above the coarsest
 * changed level l_c; below, each stage rounds by at most (kappa / 2) u D in
 * the worst case (the per-computation share of the margin kappa, with D =
 * G_old + G_new bounding |Delta|), amplified like any stage error (a_t).
 * The addition rounds by u (max|x| + 2D) at most. Paper mode carries no
 * rounding model: the bound is the selection's. */
void delta_bound(const ipco_field* f, const ipco_view* v, const std::vector<int>& b,
                 double Gnew, const uint64_t* rparts, double* Gd, uint64_t* racc) {
  if (f->bound != 0) { *Gd = Gnew; *racc = 0; return; }
  const Geometry& g = f->g;
  const int S = (int)g.stages.size();
  const bool cubic = f->interp >= 1;  /* p = 1.25, kappa 24 */
  int lc = 0;
  for (int l = 1; l <= g.K; ++l)
    if (b[l - 1] < v->b[l - 1]) lc = l;
  std::vector<double> P(S + 1);
  P[0] = 1.0;
  for (int i = 1; i <= S; ++i) P[i] = P[i - 1] * (cubic ? 1.25 : 1.0);
  double asum = 0;
  for (int t = 0; t < S; ++t)
    if (g.stages[t].level <= lc) asum += P[S - 1 - t];
  const double u = f->dtype == 0 ? Prec<float>::unit() : Prec<double>::unit();
  const double D = v->bound + Gnew;
  const double half_kappa = cubic ? 12.0 : 6.0;
  const uint64_t eps = sat_add(ceil_units(half_kappa * u * (D / f->eb) * 65536.0 * asum),
                               ceil_units(u * ((f->xmaxabs + 2.0 * D) / f->eb) * 65536.0));
  *racc = sat_add(v->racc, eps);
  *Gd = f->eb + (double)sat_add(rparts[1], *racc) * f->eb / 65536.0;
}

/* Absolute error target of an eb-mode request. */
double target_abs(const ipco_field* f, double value) {
  if (f->eb_mode == 1) { double r = range_of(f); return r > 0 ? value * r : value; }
  return value;
}

/* Parse a container (import) and rebuild the per-stage tables. */
int parse(const uint8_t* p, uint64_t len, ipco_field* f) {
  Reader r{p, len, 0, true};
  if (r.u32() != kMagic || r.u32() != kVersion) return IPCO_ECORRUPT;
  f->dtype = (int)r.u32(); f->interp = (int)r.u32(); f->bound = (int)r.u32();
  int ndim = (int)r.u32();
  int64_t dims[3];
  for (int e = 0; e < 3; ++e) dims[e] = (int64_t)r.u64();
  f->eb_mode = (int)r.u32();
  int K = (int)r.u32();
  f->eb_user = r.f64(); f->eb = r.f64();
  f->xmin = r.f64(); f->xmax = r.f64(); f->xmaxabs = r.f64(); f->anchor = r.f64();
  uint32_t S = r.u32(); r.u32();
  if (!r.ok || f->dtype < 0 || f->dtype > 1 || f->interp < 0 || f->interp > 2 ||
      f->bound < 0 || f->bound > 1 || f->eb_mode < 0 || f->eb_mode > 1)
    return IPCO_ECORRUPT;
  for (int e = 0; e < ndim && e < 3; ++e)
    if (dims[e] < 1 || dims[e] > ((int64_t)1 << 40)) return IPCO_ECORRUPT;
  if (!make_geometry(ndim, dims, &f->g)) return IPCO_ECORRUPT;
  if (f->g.K != K || f->g.stages.size() != S || !(f->eb > 0)) return IPCO_ECORRUPT;
  f->st.assign(S, StageData());
  std::vector<uint64_t> nout(S);
  for (uint32_t t = 0; t < S; ++t) {
    const StageGeom& sg = f->g.stages[t];
    uint32_t lv = r.u32(), dm = r.u32();
    uint64_t nc = r.u64();
    f->st[t].H = (int32_t)r.u32();
    f->st[t].Q = r.u32();
    nout[t] = r.u64();
    if (!r.ok || (int)lv != sg.level || (int)dm != sg.dim3 - (3 - ndim) ||
        nc != sg.ncodes || f->st[t].H < -1 || f->st[t].H > 31 || nout[t] > nc)
      return IPCO_ECORRUPT;
  }
  for (uint32_t t = 0; t < S; ++t)
    for (int k = 31; k >= 0; --k) f->st[t].size[k] = r.u64();
  for (uint32_t t = 0; t < S; ++t) {
    if (!r.need(nout[t] * 16)) return IPCO_ECORRUPT;
    uint64_t prev = 0;
    for (uint64_t i = 0; i < nout[t]; ++i) {
      uint64_t idx = r.u64();
      double v = r.f64();
      if (idx >= f->g.stages[t].ncodes || (i > 0 && idx <= prev)) return IPCO_ECORRUPT;
      prev = idx;
      f->st[t].outliers.push_back({idx, v});
    }
  }
  if (!r.ok) return IPCO_ECORRUPT;
  f->mandatory = r.pos;
  uint64_t pos = r.pos;
  for (uint32_t t = 0; t < S; ++t)
    for (int k = 31; k >= 0; --k) {
      uint64_t sz = f->st[t].size[k];
      if (sz < 4 || pos + sz > len || pos + sz < pos) return IPCO_ECORRUPT;
      f->st[t].offset[k] = pos;
      pos += sz;
    }
  if (pos != len) return IPCO_ECORRUPT;
  f->bytes.assign(p, p + len);
  /* Validate every stream and rebuild the codes (full-plane decode). */
  f->codes.assign(S, {});
  std::vector<uint32_t> words;
  for (uint32_t t = 0; t < S; ++t) {
    const StageGeom& sg = f->g.stages[t];
    std::vector<uint32_t> E(sg.ncodes, 0);
    for (int k = 31; k >= 0; --k) {
      if (!decode_stream(p + f->st[t].offset[k], f->st[t].size[k], sg.words, &words))
        return IPCO_ECORRUPT;
      const uint64_t m = (uint64_t)sg.m[2];
      for (uint64_t rr = 0; rr < sg.rows; ++rr)
        for (uint64_t j = 0; j < sg.wr; ++j) {
          uint32_t w = words[rr * sg.wr + j];
          for (uint64_t i = 0; i < 32; ++i) {
            if (32 * j + i >= m) { if ((w >> i) & 1u) return IPCO_ECORRUPT; continue; }
            E[rr * m + 32 * j + i] |= ((w >> i) & 1u) << k;
          }
        }
    }
    f->codes[t].resize(sg.ncodes);
    for (uint64_t c = 0; c < sg.ncodes; ++c)
      f->codes[t][c] = (int32_t)negabinary_inv(xor_decode(E[c]));
  }
  return IPCO_OK;
}

}  // namespace

/* ======================================================================== */
/* C API                                                                     */
/* ======================================================================== */
namespace {

/* Per-field choice of the interpolation (interp 3): the mode whose container
 * is smallest on a sample of the field. This build's reading of the
 * per-field form of the interpolation tuning that the QoZ line of
 * compressors applies (the paper fixes cubic, Sec. 4.1): the sample is the
 * centred block of extents min(N_d, c) with c = 2^20, 1024, 128 for 1, 2, 3
 * dimensions (first index floor((N_d - e_d) / 2)); each mode compresses it
 * with the absolute error bound of the whole field (a relative bound times
 * the whole field's finite range); the smallest container wins, the lower
 * mode on a tie. */
template <class T>
int auto_mode_t(const T* x, int ndim, const int64_t* dims, int eb_mode, double eb, int bound,
                int* mode) {
  uint64_t n = 1;
  for (int d = 0; d < ndim; ++d) n *= (uint64_t)dims[d];
  double eb_abs = eb;
  if (eb_mode == 1) {
    double mn = 0, mx = 0;
    bool any = false;
    for (uint64_t i = 0; i < n; ++i) {
      const double v = (double)x[i];
      if (!std::isfinite(v)) continue;
      if (!any) { mn = mx = v; any = true; }
      mn = std::min(mn, v);
      mx = std::max(mx, v);
    }
    if (!any) return IPCO_EINVAL;
    const double range = mx - mn;
    eb_abs = range > 0 ? eb * range : eb;
  }
  if (!(eb_abs > 0) || !std::isfinite(eb_abs)) return IPCO_EINVAL;
  const int64_t cap = ndim == 1 ? (int64_t)1 << 20 : ndim == 2 ? 1024 : 128;
  int64_t N[3] = {1, 1, 1}, e[3] = {1, 1, 1}, o[3] = {0, 0, 0};
  for (int d = 0; d < ndim; ++d) {
    N[3 - ndim + d] = dims[d];
    e[3 - ndim + d] = std::min<int64_t>(dims[d], cap);
    o[3 - ndim + d] = (dims[d] - e[3 - ndim + d]) / 2;
  }
  std::vector<T> sample((size_t)(e[0] * e[1] * e[2]));
  size_t k = 0;
  for (int64_t i0 = 0; i0 < e[0]; ++i0)
    for (int64_t i1 = 0; i1 < e[1]; ++i1)
      for (int64_t i2 = 0; i2 < e[2]; ++i2)
        sample[k++] = x[((o[0] + i0) * N[1] + (o[1] + i1)) * N[2] + (o[2] + i2)];
  int64_t sd[3];
  for (int d = 0; d < ndim; ++d) sd[d] = e[3 - ndim + d];
  uint64_t best = 0;
  for (int m = 0; m < 3; ++m) {
    ipco_field* f = nullptr;
    const int rc = ipco_compress(sample.data(), sizeof(T) == 4 ? 0 : 1, ndim, sd, 0, eb_abs, m,
                                 bound, &f);
    if (rc) return rc;
    const uint64_t bytes = f->bytes.size();
    ipco_free_field(f);
    if (m == 0 || bytes < best) {
      best = bytes;
      *mode = m;
    }
  }
  return IPCO_OK;
}

}  // namespace

extern "C" {

int ipco_auto_interp(const void* x, int dtype, int ndim, const int64_t* dims, int eb_mode,
                     double eb, int bound, int* mode) {
  if (!x || !mode || !dims || ndim < 1 || ndim > 3 || dtype < 0 || dtype > 1 || bound < 0 ||
      bound > 1 || eb_mode < 0 || eb_mode > 1 || !std::isfinite(eb) || !(eb > 0))
    return IPCO_EINVAL;
  for (int d = 0; d < ndim; ++d)
    if (dims[d] < 1) return IPCO_EINVAL;
  return dtype == 0 ? auto_mode_t((const float*)x, ndim, dims, eb_mode, eb, bound, mode)
                    : auto_mode_t((const double*)x, ndim, dims, eb_mode, eb, bound, mode);
}

int ipco_compress(const void* x, int dtype, int ndim, const int64_t* dims,
                  int eb_mode, double eb, int interp, int bound,
                  ipco_field** out) {
  if (!x || !out || dtype < 0 || dtype > 1 || interp < 0 || interp > 3 ||
      bound < 0 || bound > 1 || eb_mode < 0 || eb_mode > 1 || !std::isfinite(eb) ||
      !(eb > 0))
    return IPCO_EINVAL;
  if (interp == 3) {  /* the per-field choice, then that mode's container */
    const int rc = ipco_auto_interp(x, dtype, ndim, dims, eb_mode, eb, bound, &interp);
    if (rc) return rc;
  }
  ipco_field* f = new (std::nothrow) ipco_field();
  if (!f) return IPCO_ENOMEM;
  if (!make_geometry(ndim, dims, &f->g)) { delete f; return IPCO_EINVAL; }
  f->dtype = dtype; f->interp = interp; f->bound = bound; f->eb_mode = eb_mode;
  f->eb_user = eb;
  int rc = dtype == 0 ? compress_t<float>((const float*)x, f)
                      : compress_t<double>((const double*)x, f);
  if (rc) { delete f; return rc; }
  serialize(f);
  *out = f;
  return IPCO_OK;
}

int ipco_export(const ipco_field* f, void* buf, uint64_t* len) {
  if (!f || !len) return IPCO_EINVAL;
  if (!buf) { *len = f->bytes.size(); return IPCO_OK; }
  if (*len < f->bytes.size()) return IPCO_EINVAL;
  std::memcpy(buf, f->bytes.data(), f->bytes.size());
  *len = f->bytes.size();
  return IPCO_OK;
}

int ipco_import(const void* buf, uint64_t len, ipco_field** out) {
  if (!buf || !out) return IPCO_EINVAL;
  ipco_field* f = new (std::nothrow) ipco_field();
  if (!f) return IPCO_ENOMEM;
  int rc = parse((const uint8_t*)buf, len, f);
  if (rc) { delete f; return rc; }
  *out = f;
  return IPCO_OK;
}

int ipco_free_field(ipco_field* f) { delete f; return IPCO_OK; }
int ipco_free_view(ipco_view* v) { delete v; return IPCO_OK; }

int ipco_retrieve(const ipco_field* f, int kind, double value, void* out,
                  ipco_view** view) {
  if (!f || !out) return IPCO_EINVAL;
  std::vector<int> b;
  uint64_t bytes = 0;
  double bound = 0;
  uint64_t rp[2] = {0, 0};
  int rc = choose(f, kind, value, nullptr, &b, &bytes, &bound, rp);
  if (rc) return rc;
  rc = reconstruct(f, b, out);
  if (rc) return rc;
  if (view) {
    ipco_view* v = new (std::nothrow) ipco_view();
    if (!v) return IPCO_ENOMEM;
    v->f = f; v->b = b; v->bytes = bytes; v->bound = bound;
    v->racc = rp[0];
    rc = all_loaded_digits(f, b, &v->N);
    if (rc) { delete v; return rc; }
    *view = v;
  }
  return IPCO_OK;
}

int ipco_refine(ipco_view* v, int kind, double value, void* out) {
  if (!v || !out) return IPCO_EINVAL;
  std::vector<int> b;
  uint64_t bytes = 0;
  double bound = 0;
  uint64_t rp[2] = {0, 0};
  int rc = choose(v->f, kind, value, &v->b, &b, &bytes, &bound, rp);
  /* A target that the current selection already meets (or, in bitrate
   * mode, one below what is already loaded) leaves the view unchanged. */
  if (rc == IPCO_EBUDGET && kind == 1) return IPCO_OK;
  if (rc) return rc;
  if (b == v->b) return IPCO_OK;
  rc = reconstruct(v->f, b, out);
  if (rc) return rc;
  std::vector<std::vector<uint32_t>> N;
  rc = all_loaded_digits(v->f, b, &N);
  if (rc) return rc;
  v->b = b; v->bytes = bytes; v->bound = bound;
  v->N = std::move(N);
  v->racc = rp[0];
  return IPCO_OK;
}

int ipco_refine_delta(ipco_view* v, int kind, double value, void* out, int* incremental) {
  if (!v || !out) return IPCO_EINVAL;
  if (incremental) *incremental = 0;
  const ipco_field* f = v->f;
  std::vector<int> b;
  uint64_t bytes = 0;
  double bound = 0;
  uint64_t rp[2] = {0, 0};
  int rc = choose(f, kind, value, &v->b, &b, &bytes, &bound, rp);
  if (rc == IPCO_EBUDGET && kind == 1) return IPCO_OK;
  if (rc) return rc;
  if (b == v->b) return IPCO_OK;
  double Gd = 0;
  uint64_t racc = 0;
  delta_bound(f, v, b, bound, rp, &Gd, &racc);
  /* the incremental result is taken when its bound meets the target (an
   * error target) or always (a bitrate target); otherwise the refinement
   * reconstructs from scratch */
  if (kind == 1 || Gd <= target_abs(f, value)) {
    rc = f->dtype == 0 ? delta_t<float>(f, v->b, b, &v->N, (float*)out)
                       : delta_t<double>(f, v->b, b, &v->N, (double*)out);
    if (rc) return rc;
    v->b = b; v->bytes = bytes; v->bound = Gd; v->racc = racc;
    if (incremental) *incremental = 1;
    return IPCO_OK;
  }
  rc = reconstruct(f, b, out);
  if (rc) return rc;
  std::vector<std::vector<uint32_t>> N;
  rc = all_loaded_digits(f, b, &N);
  if (rc) return rc;
  v->b = b; v->bytes = bytes; v->bound = bound;
  v->N = std::move(N);
  v->racc = rp[0];
  return IPCO_OK;
}

uint32_t ipco_decode_window(uint32_t e, uint32_t nold, int bn, int bo) {
  if (bn < 0 || bo > 32 || bn > bo) return 0;
  return decode_window(e, nold, bn, bo);
}

int ipco_reconstruct(const ipco_field* f, const int* b, void* out) {
  if (!f || !b || !out) return IPCO_EINVAL;
  std::vector<int> bv(b, b + f->g.K);
  for (int v : bv)
    if (v < 0 || v > 32) return IPCO_EINVAL;
  return reconstruct(f, bv, out);
}

int ipco_selection(const ipco_view* v, int* b, int* nlevels, uint64_t* bytes,
                   double* bound) {
  if (!v) return IPCO_EINVAL;
  if (nlevels) *nlevels = (int)v->b.size();
  if (b) for (size_t i = 0; i < v->b.size(); ++i) b[i] = v->b[i];
  if (bytes) *bytes = v->bytes;
  if (bound) *bound = v->bound;
  return IPCO_OK;
}

int ipco_field_info(const ipco_field* f, int* K, int* S, uint64_t* n,
                    double* eb, double* xmin, double* xmax, double* xmaxabs,
                    uint64_t* mandatory_bytes) {
  if (!f) return IPCO_EINVAL;
  if (K) *K = f->g.K;
  if (S) *S = (int)f->g.stages.size();
  if (n) *n = f->g.n;
  if (eb) *eb = f->eb;
  if (xmin) *xmin = f->xmin;
  if (xmax) *xmax = f->xmax;
  if (xmaxabs) *xmaxabs = f->xmaxabs;
  if (mandatory_bytes) *mandatory_bytes = f->mandatory;
  return IPCO_OK;
}

int ipco_stage_info(const ipco_field* f, int t, int* level, int* dim,
                    uint64_t* ncodes, int* H, uint32_t* Q, uint64_t* noutliers) {
  if (!f || t < 0 || t >= (int)f->g.stages.size()) return IPCO_EINVAL;
  const StageGeom& sg = f->g.stages[t];
  if (level) *level = sg.level;
  if (dim) *dim = sg.dim3 - (3 - f->g.ndim);
  if (ncodes) *ncodes = sg.ncodes;
  if (H) *H = f->st[t].H;
  if (Q) *Q = f->st[t].Q;
  if (noutliers) *noutliers = f->st[t].outliers.size();
  return IPCO_OK;
}

int ipco_delta_table(const ipco_field* f, int t, uint64_t* out) {
  if (!f || !out || t < 0 || (size_t)t >= f->codes.size()) return IPCO_EINVAL;
  std::vector<uint64_t> m;
  delta_data(f->codes[t], &m);
  for (int b = 0; b <= 32; ++b) out[b] = m[b];
  return IPCO_OK;
}

int ipco_set_delta_model(ipco_field* f, int model) {
  if (!f || model < 0 || model > 1) return IPCO_EINVAL;
  if (model == 1) {
    if (f->codes.size() != f->g.stages.size()) return IPCO_EINVAL; /* imported: no codes */
    f->mdata.resize(f->codes.size());
    for (size_t t = 0; t < f->codes.size(); ++t) delta_data(f->codes[t], &f->mdata[t]);
  }
  f->delta_model = model;
  return IPCO_OK;
}

int ipco_stage_codes(const ipco_field* f, int t, int32_t* q) {
  if (!f || !q || t < 0 || t >= (int)f->codes.size()) return IPCO_EINVAL;
  std::memcpy(q, f->codes[t].data(), f->codes[t].size() * sizeof(int32_t));
  return IPCO_OK;
}

int ipco_stream_size(const ipco_field* f, int t, int k, uint64_t* bytes) {
  if (!f || !bytes || t < 0 || t >= (int)f->st.size() || k < 0 || k > 31)
    return IPCO_EINVAL;
  *bytes = f->st[t].size[k];
  return IPCO_OK;
}

int ipco_point_stage(int ndim, const int64_t* dims, int32_t* sp) {
  Geometry g;
  if (!sp || !make_geometry(ndim, dims, &g)) return IPCO_EINVAL;
  const int64_t stride[3] = {g.N[1] * g.N[2], g.N[2], 1};
  for (uint64_t i = 0; i < g.n; ++i) sp[i] = -2;
  sp[0] = -1;
  for (size_t t = 0; t < g.stages.size(); ++t) {
    const StageGeom& sg = g.stages[t];
    for (int64_t c0 = 0; c0 < sg.m[0]; ++c0)
      for (int64_t c1 = 0; c1 < sg.m[1]; ++c1)
        for (int64_t c2 = 0; c2 < sg.m[2]; ++c2) {
          int64_t idx = (sg.start[0] + c0 * sg.step[0]) * stride[0] +
                        (sg.start[1] + c1 * sg.step[1]) * stride[1] +
                        (sg.start[2] + c2 * sg.step[2]);
          /* a point produced twice is reported as -3 */
          sp[idx] = sp[idx] == -2 ? (int32_t)t : -3;
        }
  }
  return IPCO_OK;
}

int ipco_option_tables(const ipco_field* f, double E_abs, uint64_t* cost,
                       uint64_t* bytes) {
  if (!f || !cost || !bytes) return IPCO_EINVAL;
  Options o;
  double A = E_abs > 0 ? f->xmaxabs + E_abs
                       : f->xmaxabs + std::max(range_of(f), f->eb);
  option_tables(f, A, &o);
  std::memcpy(cost, o.cost.data(), o.cost.size() * 8);
  std::memcpy(bytes, o.bytes.data(), o.bytes.size() * 8);
  return IPCO_OK;
}

uint32_t ipco_negabinary(int32_t q) { return negabinary(q); }
int64_t ipco_negabinary_inv(uint32_t n) { return negabinary_inv(n); }
uint32_t ipco_xor_encode(uint32_t n) { return xor_encode(n); }
uint32_t ipco_xor_decode(uint32_t e) { return xor_decode(e); }

uint64_t ipco_xor_check(uint64_t start, uint64_t count, uint64_t step) {
  /* Checks, for n = start + i*step (mod 2^32), that the bitwise decoder
   * inverts the word form e = n ^ n>>1 ^ n>>2, that the bitwise encoder
   * equals that word form, and the progressive property: the planes >= b of
   * e decode to the digits >= b of n. Returns the number of failures. */
  uint64_t fails = 0;
  for (uint64_t i = 0; i < count; ++i) {
    uint32_t n = (uint32_t)(start + i * step);
    uint32_t e = n ^ (n >> 1) ^ (n >> 2);
    if (xor_encode(n) != e) ++fails;
    if (xor_decode(e) != n) ++fails;
    int b = (int)(i % 33u);
    uint32_t mk = plane_mask(b);
    if ((xor_decode(e & mk) & mk) != (n & mk)) ++fails;
  }
  return fails;
}

}  // extern "C"
