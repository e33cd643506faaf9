// Host-side plane selection of libipcomp (Sec. 5.1-5.3). See ipc_select.h.
#include "ipc_select.h"

#include <algorithm>
#include <cmath>
#include <cstring>

#include "ipc.h"

namespace ipc {
namespace {

const uint64_t kSat = 1ull << 62;  // saturation of integer costs

uint64_t sadd(uint64_t a, uint64_t b) {
  const uint64_t c = a + b;
  return (c < a || c > kSat) ? kSat : c;
}
uint64_t units(double v) {
  if (!(v < (double)kSat)) return kSat;
  return v <= 0 ? 0 : (uint64_t)std::ceil(v);
}
// Largest |value| of b dropped negabinary digits (Sec. 4.4.2).
uint64_t uncert(int b) {
  if (b <= 0) return 0;
  const uint64_t p = uint64_t(1) << (b + 1);
  return (b & 1) ? (p - 1) / 3 : (p - 2) / 3;
}

// Option tables: cost[l-1][b] (error cost of dropping b planes at level l,
// in units of eb * 2^-16) and bytes[l-1][b] (stream bytes loaded).
// Strict mode: stage t of S is amplified by p^(S-1-t) (every later sweep is
// one more interpolation of infinity-norm <= p) and a rounding margin
// kappa * u * A / eb is added per recomputed stage. Paper mode: p^(l-1)
// times the largest stage term of the level (Theorem 1).
struct Tables {
  int K;
  std::vector<uint64_t> cost, bytes;
  std::vector<uint64_t> rho;  // per level: the rounding margin inside cost(l, b > 0)
  std::vector<int> lo;        // per level: the smallest b allowed
};

// The target-independent parts of the tables: base[l-1][b] (strict: the sum
// of the stage terms; paper: the whole cost), ybytes[l-1][b], asum[l-1].
void prepare_tables(const SelInput& in, std::vector<uint64_t>* base, std::vector<uint64_t>* ybytes,
                    std::vector<double>* asum_out) {
  const int K = in.K, S = (int)in.st.size();
  const bool cubic = in.interp != IPC_LINEAR, strict = in.bound == IPC_BOUND_STRICT;
  const double p = cubic ? 1.25 : 1.0;
  std::vector<double> pw(std::max(S, K) + 1);
  pw[0] = 1.0;
  for (size_t i = 1; i < pw.size(); ++i) pw[i] = pw[i - 1] * p;
  base->assign((size_t)K * 33, 0);
  ybytes->assign((size_t)K * 33, 0);
  asum_out->assign((size_t)K, 0.0);
  // the stages of each level (stage order), and the bytes of planes >= b of
  // each stage (suffix sums), so a level's options cost O(33 x its stages)
  std::vector<int> by_level(S), first(K + 2, 0);
  for (int t = 0; t < S; ++t) ++first[in.st[t].level + 1];
  for (int l = 1; l <= K + 1; ++l) first[l] += first[l - 1];
  {
    std::vector<int> fill(first.begin(), first.end());
    for (int t = 0; t < S; ++t) by_level[fill[in.st[t].level]++] = t;
  }
  std::vector<uint64_t> ysuf((size_t)S * 33);
  for (int t = 0; t < S; ++t) {
    ysuf[(size_t)t * 33 + 32] = 0;
    for (int k = 31; k >= 0; --k) ysuf[(size_t)t * 33 + k] = ysuf[(size_t)t * 33 + k + 1] + in.st[t].size[k];
  }
  for (int l = 1; l <= K; ++l) {
    double asum = 0;  // a_t over the stages of levels <= l, in stage order
    for (int t = 0; t < S; ++t)
      if (in.st[t].level <= l) asum += (strict && cubic) ? pw[S - 1 - t] : 1.0;
    (*asum_out)[l - 1] = asum;
    for (int b = 0; b <= 32; ++b) {
      uint64_t c = 0, y = 0, mmax = 0;
      for (int j = first[l]; j < first[l + 1]; ++j) {
        const int t = by_level[j];
        const SelStage& s = in.st[t];
        const uint64_t M = b <= 0 ? 0 : (b <= s.H ? uncert(b) : (uint64_t)s.Q);
        if (strict) c = sadd(c, units((cubic ? pw[S - 1 - t] : 1.0) * (double)M * in.bin * 65536.0));
        else mmax = std::max(mmax, M);
        y += ysuf[(size_t)t * 33 + b];
      }
      if (!strict) c = units(pw[l - 1] * (double)mmax * in.bin * 65536.0);
      (*base)[(size_t)(l - 1) * 33 + b] = c;
      (*ybytes)[(size_t)(l - 1) * 33 + b] = y;
    }
  }
}

// Option tables for the magnitude bound A (strict: rho_l from A, added to
// every b > 0).
void build_tables(const SelInput& in, double A, Tables* T) {
  std::vector<uint64_t> lb, ly;
  std::vector<double> la;
  const bool prepared = !in.base.empty();
  if (!prepared) prepare_tables(in, &lb, &ly, &la);
  const std::vector<uint64_t>& base = prepared ? in.base : lb;
  const std::vector<double>& asum = prepared ? in.asum : la;
  const int K = in.K;
  const bool cubic = in.interp != IPC_LINEAR, strict = in.bound == IPC_BOUND_STRICT;
  const double u = in.dtype == IPC_F32 ? 1.0 / 16777216.0 : 1.0 / 9007199254740992.0;
  const double kappa = cubic ? 24.0 : 12.0;
  T->K = K;
  T->bytes = prepared ? in.ybytes : ly;
  T->lo.assign((size_t)K, 0);
  if (in.lower.size() == (size_t)K) T->lo = in.lower;
  T->cost.assign((size_t)K * 33, 0);
  T->rho.assign((size_t)K, 0);
  for (int l = 1; l <= K; ++l) {
    const uint64_t rho = units(kappa * u * (A / in.eb) * 65536.0 * asum[l - 1]);
    T->rho[l - 1] = strict ? rho : 0;
    for (int b = 0; b <= 32; ++b) {
      const uint64_t c = base[(size_t)(l - 1) * 33 + b];
      T->cost[(size_t)(l - 1) * 33 + b] = strict && b > 0 ? sadd(c, rho) : c;
    }
  }
}

uint64_t cost_of(const Tables& T, const std::vector<int>& b) {
  uint64_t c = 0;
  for (size_t l = 0; l < b.size(); ++l) c = sadd(c, T.cost[l * 33 + b[l]]);
  return c;
}

// A feasible selection found greedily; its objective value (bytes in eb
// mode, cost in bitrate mode) bounds the optimum's, and so every partial
// sum of the optimum. Returns ~0 when the greedy start is infeasible.
uint64_t greedy_bound(const Tables& T, int kind, uint64_t limit, const std::vector<int>* upper) {
  const int K = T.K;
  std::vector<int> b(K);
  uint64_t c = 0, y = 0;
  for (int l = 0; l < K; ++l) {
    b[l] = kind == 0 ? T.lo[l] : (upper ? (*upper)[l] : 32);
    if (b[l] < T.lo[l] || (upper && b[l] > (*upper)[l])) return ~uint64_t(0);  // no option
    c = sadd(c, T.cost[(size_t)l * 33 + b[l]]);
    y += T.bytes[(size_t)l * 33 + b[l]];
  }
  if ((kind == 0 && c > limit) || (kind == 1 && y > limit)) return ~uint64_t(0);
  // Each step takes the move of best ratio over all levels. A level's best
  // move depends only on its own b and on the slack left (cost in eb mode,
  // bytes in bitrate mode), and the slack only shrinks: so a level's best is
  // recomputed only after it moved, or when the slack no longer admits it
  // (the best of a subset that still holds the old best is the old best).
  auto level_best = [&](int l, int* v_out) -> double {
    const uint64_t c0 = T.cost[(size_t)l * 33 + b[l]], y0 = T.bytes[(size_t)l * 33 + b[l]];
    double best = 0;
    *v_out = -1;
    if (kind == 0) {  // drop more planes: fewer bytes for more cost
      const int bmax = upper ? (*upper)[l] : 32;
      for (int v = b[l] + 1; v <= bmax; ++v) {
        const uint64_t c1 = T.cost[(size_t)l * 33 + v], y1 = T.bytes[(size_t)l * 33 + v];
        if (c1 < c0 || sadd(c - c0, c1) > limit || y1 >= y0) continue;
        const double r = (double)(y0 - y1) / (double)(c1 - c0 + 1);
        if (r > best) { best = r; *v_out = v; }
      }
    } else {  // load more planes: less cost for more bytes
      for (int v = b[l] - 1; v >= T.lo[l]; --v) {
        const uint64_t c1 = T.cost[(size_t)l * 33 + v], y1 = T.bytes[(size_t)l * 33 + v];
        if (c1 >= c0 || y - y0 + y1 > limit) continue;
        const double r = (double)(c0 - c1) / (double)(y1 - y0 + 1);
        if (r > best) { best = r; *v_out = v; }
      }
    }
    return best;
  };
  auto fits = [&](int l, int v) {
    const uint64_t c0 = T.cost[(size_t)l * 33 + b[l]], y0 = T.bytes[(size_t)l * 33 + b[l]];
    const uint64_t c1 = T.cost[(size_t)l * 33 + v], y1 = T.bytes[(size_t)l * 33 + v];
    return kind == 0 ? sadd(c - c0, c1) <= limit : y - y0 + y1 <= limit;
  };
  std::vector<double> lr(K);
  std::vector<int> lv(K);
  for (int l = 0; l < K; ++l) lr[l] = level_best(l, &lv[l]);
  for (;;) {
    int bl = -1, bb = -1;
    double best = 0;
    for (int l = 0; l < K; ++l) {
      if (lv[l] >= 0 && !fits(l, lv[l])) lr[l] = level_best(l, &lv[l]);
      if (lv[l] >= 0 && lr[l] > best) { best = lr[l]; bl = l; bb = lv[l]; }
    }
    if (bl < 0) break;
    c = sadd(c - T.cost[(size_t)bl * 33 + b[bl]], T.cost[(size_t)bl * 33 + bb]);
    y = y - T.bytes[(size_t)bl * 33 + b[bl]] + T.bytes[(size_t)bl * 33 + bb];
    b[bl] = bb;
    lr[bl] = level_best(bl, &lv[bl]);
  }
  return kind == 0 ? y : c;
}

// Exact solver (meet in the middle). Every option of a level is a point
// (cost, bytes); bytes fall strictly with b (each stream is >= 4 bytes), so an
// option with a larger-b alternative of no greater cost can never be part of
// an optimum and is dropped. The levels are split in two halves; each half's
// Pareto frontier (cost ascending, bytes descending; equal points keep the
// lexicographically larger part-vector) is built level by level, and the two
// frontiers are joined with a binary search per entry of the first half.
// Partial sums beyond the greedy bound are dropped (costs and bytes only
// grow), so the optimum and its ties are kept.
// Ties: eb mode -> fewer bytes, then smaller cost, then the lexicographically
// larger (b_1, b_2, ...); bitrate mode -> smaller cost, then fewer bytes,
// then the same lexicographic rule.
constexpr int kKeySlots = 16;  // levels per half (K <= 32)
typedef unsigned __int128 Key;

struct Part {
  uint64_t c, y;
  Key key;  // the half's b-vector, 6 bits per level, first level most significant
};

inline Key key_put(Key k, int i, int b) { return k | ((Key)(unsigned)b << (6 * (kKeySlots - 1 - i))); }
inline int key_get(Key k, int i) { return (int)((k >> (6 * (kKeySlots - 1 - i))) & 63u); }

void half_frontier(const Tables& T, int l0, int l1, int kind, uint64_t limit, uint64_t gbound,
                   const std::vector<int>* upper, std::vector<Part>* out) {
  std::vector<Part> F(1), G;
  F[0] = Part{0, 0, 0};
  for (int l = l0; l < l1; ++l) {
    const int bmax = upper ? (*upper)[l] : 32;
    int opt[33];
    int nopt = 0;
    uint64_t best = ~uint64_t(0);
    for (int b = bmax; b >= T.lo[l]; --b) {  // staircase: keep b only if strictly cheaper
      const uint64_t c = T.cost[(size_t)l * 33 + b];
      if (c < best) {
        opt[nopt++] = b;
        best = c;
      }
    }
    // F extended by option i is F shifted by a constant: still sorted (but
    // where saturated costs tie). The nopt runs are merged (heap on their
    // heads) in the order of `before`; should a run not be sorted, the merge
    // is sorted after all. Then the Pareto filter.
    auto before = [](const Part& x, const Part& z) {
      if (x.c != z.c) return x.c < z.c;
      if (x.y != z.y) return x.y < z.y;
      return x.key > z.key;
    };
    auto entry = [&](int i, size_t j, Part* out) {  // run i, position j; false: pruned
      const int b = opt[i];
      const Part& e = F[j];
      const uint64_t c = sadd(e.c, T.cost[(size_t)l * 33 + b]);
      const uint64_t y = e.y + T.bytes[(size_t)l * 33 + b];
      if (kind == 0 ? (c > limit || y > gbound) : (y > limit || c > gbound)) return false;
      *out = Part{c, y, key_put(e.key, l - l0, b)};
      return true;
    };
    struct Head {
      Part p;
      int run;
      size_t pos;
    };
    Head heap[33];
    int nh = 0;
    auto push = [&](const Head& h) {  // binary min-heap on `before`
      int i = nh++;
      while (i > 0 && before(h.p, heap[(i - 1) / 2].p)) {
        heap[i] = heap[(i - 1) / 2];
        i = (i - 1) / 2;
      }
      heap[i] = h;
    };
    auto pop = [&]() {
      const Head top = heap[0];
      const Head last = heap[--nh];
      int i = 0;
      for (;;) {
        int c = 2 * i + 1;
        if (c >= nh) break;
        if (c + 1 < nh && before(heap[c + 1].p, heap[c].p)) ++c;
        if (!before(heap[c].p, last.p)) break;
        heap[i] = heap[c];
        i = c;
      }
      if (nh > 0) heap[i] = last;
      return top;
    };
    // next unpruned entry of run i at or after position j
    auto advance = [&](int i, size_t j) {
      Part p;
      for (; j < F.size(); ++j)
        if (entry(i, j, &p)) {
          push(Head{p, i, j});
          return;
        }
    };
    for (int i = 0; i < nopt; ++i) advance(i, 0);
    G.clear();
    bool sorted = true;
    while (nh > 0) {
      const Head h = pop();
      if (!G.empty() && before(h.p, G.back())) sorted = false;
      G.push_back(h.p);
      advance(h.run, h.pos + 1);
    }
    if (!sorted) std::sort(G.begin(), G.end(), before);
    F.clear();
    for (const Part& e : G)
      if (F.empty() || e.y < F.back().y) F.push_back(e);
    if (F.empty()) break;
  }
  *out = std::move(F);
}

int solve(const Tables& T, int kind, uint64_t limit, const std::vector<int>* upper,
          std::vector<int>* best) {
  const int K = T.K;
  if (K == 0) {
    best->clear();
    return IPC_OK;
  }
  if (K > 2 * kKeySlots) return IPC_EINVAL;
  const uint64_t gb = greedy_bound(T, kind, limit, upper);
  const int h = K / 2;
  std::vector<Part> A, B;
  half_frontier(T, 0, h, kind, limit, gb, upper, &A);
  half_frontier(T, h, K, kind, limit, gb, upper, &B);
  if (A.empty() || B.empty()) return kind == 0 ? IPC_EBOUND : IPC_EBUDGET;
  // B: cost ascending, bytes descending.
  bool found = false;
  uint64_t bc = 0, by = 0;
  const Part *ba = nullptr, *bb = nullptr;
  for (const Part& a : A) {
    const Part* m = nullptr;
    if (kind == 0) {
      if (a.c > limit) continue;
      const uint64_t lim = limit - a.c;  // largest cost <= lim has the fewest bytes
      size_t lo = 0, hi = B.size();
      while (lo < hi) {
        const size_t mid = (lo + hi) / 2;
        if (B[mid].c <= lim) lo = mid + 1;
        else hi = mid;
      }
      if (lo == 0) continue;
      m = &B[lo - 1];
    } else {
      if (a.y > limit) continue;
      const uint64_t lim = limit - a.y;  // first entry with bytes <= lim: least cost
      size_t lo = 0, hi = B.size();
      while (lo < hi) {
        const size_t mid = (lo + hi) / 2;
        if (B[mid].y > lim) lo = mid + 1;
        else hi = mid;
      }
      if (lo == B.size()) continue;
      m = &B[lo];
    }
    const uint64_t c = sadd(a.c, m->c), y = a.y + m->y;
    bool better;
    if (!found) {
      better = true;
    } else {
      const bool lex = a.key > ba->key || (a.key == ba->key && m->key > bb->key);
      if (kind == 0) better = y < by || (y == by && c < bc) || (y == by && c == bc && lex);
      else better = c < bc || (c == bc && y < by) || (c == bc && y == by && lex);
    }
    if (better) {
      found = true;
      bc = c;
      by = y;
      ba = &a;
      bb = m;
    }
  }
  if (!found) return kind == 0 ? IPC_EBOUND : IPC_EBUDGET;
  best->assign(K, 0);
  for (int l = 0; l < h; ++l) (*best)[l] = key_get(ba->key, l);
  for (int l = h; l < K; ++l) (*best)[l] = key_get(bb->key, l - h);
  return IPC_OK;
}

// The selection's cost split into its rounding margins (rho_l of every
// level with b_l > 0) and the rest (the truncation terms).
void cost_parts(const Tables& T, const std::vector<int>& b, uint64_t* rparts) {
  uint64_t r = 0;
  for (size_t l = 0; l < b.size(); ++l)
    if (b[l] > 0) r = sadd(r, T.rho[l]);
  rparts[0] = r;
  rparts[1] = cost_of(T, b) - r;
}

uint64_t loaded(const SelInput& in, const std::vector<int>& b) {
  uint64_t y = in.mandatory;
  for (const SelStage& s : in.st)
    for (int k = b[s.level - 1]; k < 32; ++k) y += s.size[k];
  return y;
}

}  // namespace

void prepare_selection(SelInput* in) { prepare_tables(*in, &in->base, &in->ybytes, &in->asum); }

int select_planes(const SelInput& in, int kind, double value, const std::vector<int>* upper,
                  std::vector<int>* b, uint64_t* bytes, double* bound, const char** why,
                  uint64_t* rparts) {
  *why = "";
  if (!std::isfinite(value)) {
    *why = "target must be finite";
    return IPC_EINVAL;
  }
  const double range = in.xmax - in.xmin;
  Tables T;
  if (kind == IPC_TARGET_EB) {
    double E = value;
    if (in.eb_mode == IPC_EB_REL) E = range > 0 ? value * range : value;
    if (!(E >= in.eb)) {
      *why = "target error bound is below the compression bound";
      return IPC_EBOUND;
    }
    build_tables(in, in.xmaxabs + E, &T);
    const double Bd = std::floor(((E - in.eb) / in.eb) * 65536.0);
    const uint64_t B = Bd >= (double)kSat ? kSat : (uint64_t)Bd;
    const int rc = solve(T, 0, B, upper, b);
    if (rc) {
      *why = "no selection meets the error bound";
      return rc;
    }
    *bytes = loaded(in, *b);
    *bound = in.eb + (double)cost_of(T, *b) * in.eb / 65536.0;
    if (rparts) cost_parts(T, *b, rparts);
    return IPC_OK;
  }
  if (kind == IPC_TARGET_BITRATE) {
    if (!(value >= 0)) {
      *why = "bitrate must be >= 0";
      return IPC_EINVAL;
    }
    const double Sd = std::floor(value * (double)in.n / 8.0);
    const uint64_t Sb = Sd >= 1.8e19 ? ~uint64_t(0) : (uint64_t)Sd;
    if (in.mandatory > Sb) {
      *why = "bitrate below the mandatory bytes";
      return IPC_EBUDGET;
    }
    double A = in.xmaxabs + std::max(range, in.eb);
    build_tables(in, A, &T);
    const int rc = solve(T, 1, Sb - in.mandatory, upper, b);
    if (rc) {
      *why = "no selection fits the bitrate";
      return rc;
    }
    *bytes = loaded(in, *b);
    // The rounding margin assumed |values| <= max|x| + range; widen A until
    // it covers the reported bound.
    double G = in.eb + (double)cost_of(T, *b) * in.eb / 65536.0;
    for (int it = 0; it < 16 && G > A - in.xmaxabs; ++it) {
      A = in.xmaxabs + G;
      build_tables(in, A, &T);
      G = in.eb + (double)cost_of(T, *b) * in.eb / 65536.0;
    }
    *bound = G;
    if (rparts) cost_parts(T, *b, rparts);
    return IPC_OK;
  }
  *why = "unknown target kind";
  return IPC_EINVAL;
}

double incremental_bound(const SelInput& in, const std::vector<int>& bold, double Gold,
                         uint64_t racc_old, const std::vector<int>& bnew, double Gnew,
                         const uint64_t* rparts, uint64_t* racc_new) {
  if (in.bound != IPC_BOUND_STRICT) {
    *racc_new = 0;
    return Gnew;
  }
  const int S = (int)in.st.size();
  const bool cubic = in.interp != IPC_LINEAR;
  int lc = 0;  // coarsest level that loads new planes
  for (int l = 1; l <= in.K; ++l)
    if (bnew[l - 1] < bold[l - 1]) lc = l;
  // a_t = p^(S-1-t), products formed in order as in the option tables
  std::vector<double> pw(S + 1);
  pw[0] = 1.0;
  for (int i = 1; i <= S; ++i) pw[i] = pw[i - 1] * (cubic ? 1.25 : 1.0);
  double asum = 0;
  for (int t = 0; t < S; ++t)
    if (in.st[t].level <= lc) asum += pw[S - 1 - t];
  const double u = in.dtype == IPC_F32 ? 1.0 / 16777216.0 : 1.0 / 9007199254740992.0;
  const double D = Gold + Gnew;  // bounds |Delta|
  const double half_kappa = cubic ? 12.0 : 6.0;
  const uint64_t eps = sadd(units(half_kappa * u * (D / in.eb) * 65536.0 * asum),
                            units(u * ((in.xmaxabs + 2.0 * D) / in.eb) * 65536.0));
  *racc_new = sadd(racc_old, eps);
  return in.eb + (double)sadd(rparts[1], *racc_new) * in.eb / 65536.0;
}

}  // namespace ipc
