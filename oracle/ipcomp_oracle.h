/*
 * IPComp CPU ORACLE -- test infrastructure, not part of the product.
 *
 * A plain, slow, single-threaded C++ restatement of what the IPComp paper
 * (arXiv 2502.04093) computes: the interpolation predictor with
 * error-bounded quantization (Sec. 4.1, Eq. 1-2, Sec. 4.2.2 Eq. 4), the
 * per-level 32-bitplane split (Sec. 4.3), predictive negabinary coding
 * (Sec. 4.4), the Theorem-1 error bound (Sec. 5.1) and the two knapsack
 * loaders (Sec. 5.2, 5.3), plus reconstruction (Algorithm 1) and refinement
 * (Algorithm 2).
 *
 * Only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load this library. It shares no code with the CUDA library.
 *
 * All pointers are host pointers. Return value 0 = success; the negative
 * codes are the same numbers the product header uses.
 */
#ifndef IPCOMP_ORACLE_H
#define IPCOMP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { IPCO_OK = 0, IPCO_EINVAL = -1, IPCO_EBOUND = -2, IPCO_EBUDGET = -3,
       IPCO_ENOMEM = -4, IPCO_ECORRUPT = -5 };

typedef struct ipco_field ipco_field;
typedef struct ipco_view ipco_view;

/* Compress x (dtype 0 = f32, 1 = f64; row-major, last dim fastest).
 * eb_mode 0 = absolute, 1 = relative to (max - min). interp 0 linear,
 * 1 cubic, 2 cubic with quadratic boundaries (see the predictor in the
 * .cpp), 3 the per-field choice of ipco_auto_interp (the container records
 * the chosen mode). bound 0 strict, 1 paper. */
int ipco_compress(const void* x, int dtype, int ndim, const int64_t* dims,
                  int eb_mode, double eb, int interp, int bound,
                  ipco_field** out);
/* The interpolation mode (0..2) whose container is smallest on a centred
 * sample of the field (extents min(N_d, c), c = 2^20 / 1024 / 128 for 1 / 2
 * / 3 dimensions), compressed with the whole field's absolute error bound;
 * the lower mode on a tie. */
int ipco_auto_interp(const void* x, int dtype, int ndim, const int64_t* dims, int eb_mode,
                     double eb, int bound, int* mode);
/* Container bytes: len query when buf == NULL. */
int ipco_export(const ipco_field* f, void* buf, uint64_t* len);
int ipco_import(const void* buf, uint64_t len, ipco_field** out);
int ipco_free_field(ipco_field* f);

/* kind 0 = error bound (in the field's eb mode), 1 = bitrate (bits/value). */
int ipco_retrieve(const ipco_field* f, int kind, double value, void* out,
                  ipco_view** view);
/* Canonical refinement: selection constrained to b'_l <= b_l. */
int ipco_refine(ipco_view* v, int kind, double value, void* out);
/* Incremental refinement (Algorithm 2): `out` must hold the view's current
 * reconstruction. The same constrained selection as ipco_refine; only the
 * new planes are read, and out += Delta. The incremental result is used when
 * its guaranteed bound (which adds the rounding of the increment) meets an
 * error target, or for a bitrate target; otherwise the refinement
 * reconstructs from scratch. *incremental (optional) tells which ran. */
int ipco_refine_delta(ipco_view* v, int kind, double value, void* out, int* incremental);
/* The digits bn..bo-1 of a code from its encoded bits e and its loaded
 * digits nold (planes >= bo), decoded top-down (for the coding pins). */
uint32_t ipco_decode_window(uint32_t e, uint32_t nold, int bn, int bo);
/* Reconstruction for an explicit per-level selection b[0..K-1]
 * (b[l-1] = planes dropped at level l). */
int ipco_reconstruct(const ipco_field* f, const int* b, void* out);
int ipco_selection(const ipco_view* v, int* b, int* nlevels, uint64_t* bytes,
                   double* bound);
int ipco_free_view(ipco_view* v);

/* ---- introspection used by the tests ---- */
/* K, S, n, absolute eb, xmin, xmax, xmaxabs, mandatory bytes. */
int ipco_field_info(const ipco_field* f, int* K, int* S, uint64_t* n,
                    double* eb, double* xmin, double* xmax, double* xmaxabs,
                    uint64_t* mandatory_bytes);
/* Stage t: level, native dim, code count, H (msb of the OR of the
 * negabinary codes, -1 if all zero), Q (max |q|), outlier count. */
int ipco_stage_info(const ipco_field* f, int t, int* level, int* dim,
                    uint64_t* ncodes, int* H, uint32_t* Q,
                    uint64_t* noutliers);
/* The quantized codes of stage t in code order (0 at outliers). */
int ipco_stage_codes(const ipco_field* f, int t, int32_t* q);
/* The data maximum of |q - q'_b| over stage t's codes, b = 0..32 (out[33]);
 * fields compressed here only (the codes are kept). */
int ipco_delta_table(const ipco_field* f, int t, uint64_t* out);
/* Bound on |q - q'_b| in the cost tables: 0 the closed form (U(b) up to the
 * top digit H, then Q; the container's model), 1 the data maximum (a
 * study: it is not stored in the container). */
int ipco_set_delta_model(ipco_field* f, int model);
/* Byte size of stream (t, plane k). */
int ipco_stream_size(const ipco_field* f, int t, int k, uint64_t* bytes);
/* For every point (row-major), the stage that produces it (-1 = anchor). */
int ipco_point_stage(int ndim, const int64_t* dims, int32_t* stage_of_point);
/* Integer error cost (units of eb * 2^-16) and loaded bytes of every
 * option b = 0..32 at every level, for an eb-mode target E (absolute)
 * or, when E <= 0, for the bitrate-mode magnitude bound. */
int ipco_option_tables(const ipco_field* f, double E_abs, uint64_t* cost,
                       uint64_t* bytes);
/* Negabinary / predictive-XOR primitives (for the coding pins). */
uint32_t ipco_negabinary(int32_t q);
int64_t ipco_negabinary_inv(uint32_t n);
uint32_t ipco_xor_encode(uint32_t n);
uint32_t ipco_xor_decode(uint32_t e);
/* For n = start + i*step (mod 2^32), i < count: checks decode(encode(n)) == n
 * and that decoding the planes >= b of encode(n) gives the digits >= b of n.
 * Returns the number of failures. */
uint64_t ipco_xor_check(uint64_t start, uint64_t count, uint64_t step);

#ifdef __cplusplus
}
#endif
#endif
