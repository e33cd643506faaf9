// Host-side plane selection of libipcomp (Sec. 5.1-5.3): the per-level
// option tables (error cost, loaded bytes) and the exact knapsack over the
// levels. Host code only: it needs nothing but the stage statistics and the
// plane sizes of a field, so it also runs on a container header alone.
#pragma once
#include <stdint.h>

#include <vector>

namespace ipc {

struct SelStage {
  int level;          // 1..K
  int32_t H;          // highest nonzero negabinary digit of the stage (-1: none)
  uint32_t Q;         // max |q| over the stage's non-outlier codes
  uint64_t size[32];  // packed stream bytes of plane k
};

struct SelInput {
  int K;
  int dtype, interp, bound, eb_mode;
  double eb;       // absolute compression bound
  double bin;      // quantization bin width in the element type, divided by eb
  double xmin, xmax, xmaxabs;
  uint64_t n;          // values
  uint64_t mandatory;  // container bytes always loaded (header, tables, outliers)
  std::vector<SelStage> st;
  // Optional, filled by prepare_selection: the parts of the option tables
  // that do not depend on the target (per level l and b: the cost terms of
  // the stages, the loaded stream bytes; per level: the sum of a_t over the
  // stages of levels <= l). Without them every selection computes them.
  std::vector<uint64_t> base, ybytes;
  std::vector<double> asum;
  // Optional lower bounds on b_l (a field that holds only the planes
  // k >= lower_l of each level); empty: none.
  std::vector<int> lower;
};

// Fills in.base, in.ybytes and in.asum (for inputs selected many times).
void prepare_selection(SelInput* in);

// Selection for a target (kind 0: error bound in the field's eb mode, kind 1:
// bitrate in bits/value). upper (optional) bounds b_l from above (refine).
// Returns 0 or a negative IPC_* status; `why` names the failure.
// rparts (optional): [0] = the rounding margins inside the selection's cost
// (rho_l of each level with b_l > 0), [1] = the rest (truncation terms); both
// in units of eb * 2^-16.
int select_planes(const SelInput& in, int kind, double value, const std::vector<int>* upper,
                  std::vector<int>* b, uint64_t* bytes, double* bound, const char** why,
                  uint64_t* rparts = nullptr);

// Guaranteed bound of an incremental refinement (Algorithm 2) from selection
// bold (bound Gold, rounding allowance racc_old) to bnew (whose fresh
// reconstruction would have bound Gnew and cost parts rparts). Relative to
// the compressor's values, x^old + Delta adds to the truncation of bnew the
// old result's rounding and the increment's: Delta is zero above the
// coarsest changed level l_c, each stage at or below it rounds by at most
// (kappa / 2) u D (D = Gold + Gnew bounds |Delta|), amplified like any stage
// error, and the final addition rounds by u (max|x| + 2D). Returns the bound
// and the new allowance (units of eb * 2^-16). Paper mode: Gnew, allowance 0.
double incremental_bound(const SelInput& in, const std::vector<int>& bold, double Gold,
                         uint64_t racc_old, const std::vector<int>& bnew, double Gnew,
                         const uint64_t* rparts, uint64_t* racc_new);

}  // namespace ipc
