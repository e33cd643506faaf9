/*
 * ipc.h -- C ABI of libipcomp, a GB300 (sm_103a) implementation of IPComp,
 * the interpolation-based progressive lossy compressor of arXiv 2502.04093.
 *
 * Compression (Sec. 3.2, Fig. 2): a coarse-to-fine multi-level interpolation
 * predictor (Sec. 4.1, Eq. 1 linear / Eq. 2 cubic) with error-bounded
 * quantization of the residuals (Sec. 4.2.2), then the per-level bitplane
 * split of the 32-bit codes (Sec. 4.3) with negabinary sign coding and 2-bit
 * prefix predictive XOR (Sec. 4.4). Retrieval: the optimized loader
 * (Sec. 5.2 error-bound mode, Sec. 5.3 bitrate mode) picks per level how many
 * low planes to drop, then reconstruction (Algorithm 1) decodes the selected
 * planes and rebuilds the field by interpolation. Refinement (Algorithm 2)
 * adds planes to an earlier retrieval.
 *
 * Conventions (all entry points):
 *  - Pointers named d_* are CUDA device pointers owned by the caller; other
 *    pointers are host pointers. Arrays are dense row-major, last dimension
 *    fastest, 1 <= ndim <= 3.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream). Work is
 *    ordered on that stream. ipc_compress and ipc_import synchronise with it
 *    before returning; ipc_retrieve / ipc_refine return as soon as their
 *    kernels are queued (d_out is valid once the stream reaches that point).
 *  - ipc_field and ipc_view objects are owned by the library until
 *    ipc_free. A view refers to its field: free views before their field.
 *  - Every function returns IPC_OK (0) or a negative status; on error no
 *    output argument is written and no object is leaked. ipc_last_error()
 *    returns a short description of the calling thread's last failure.
 *  - Calls on one field or view must not overlap; different fields may be
 *    used from different threads. Compressions on one device are serialised
 *    internally (they share a scratch workspace).
 */
#ifndef IPCOMP_IPC_H
#define IPCOMP_IPC_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
enum {
  IPC_OK = 0,
  IPC_EINVAL = -1,   /* bad shape / dtype / error bound / argument           */
  IPC_EBOUND = -2,   /* requested error bound below the compression bound    */
  IPC_EBUDGET = -3,  /* bitrate below the mandatory (header + tables) bytes  */
  IPC_ENOMEM = -4,   /* host or device allocation failed                     */
  IPC_ECORRUPT = -5, /* container failed validation on import                */
  IPC_ECUDA = -6,    /* a CUDA call failed (see ipc_last_error)              */
  IPC_ETIMEOUT = -7, /* a bounded wait ran out                               */
  IPC_EBUSY = -8     /* resource in use (server slots, pending work)         */
};

typedef enum { IPC_F32 = 0, IPC_F64 = 1 } ipc_dtype;
/* Eq. 1 (linear, p = 1) or Eq. 2 (cubic, p = 1.25), Sec. 4.1; a cubic
 * target missing one far neighbour takes Eq. 1 (IPC_CUBIC) or the
 * three-point quadratic through its two near neighbours and the far one
 * that exists (IPC_CUBIC_QUAD: weights 3/8, 6/8, -1/8, infinity norm 1.25,
 * so p and the error model are the cubic ones).
 * IPC_INTERP_AUTO (compression only) chooses one of the three per field:
 * the mode whose container is smallest on the centred block of extents
 * min(N_d, c), c = 2^20 / 1024 / 128 for 1 / 2 / 3 dimensions (first index
 * floor((N_d - e_d) / 2)), compressed with the whole field's absolute error
 * bound; the lower mode on a tie. The container records the chosen mode. It
 * costs a range pass (relative bounds) and three compressions of the block. */
typedef enum { IPC_LINEAR = 0, IPC_CUBIC = 1, IPC_CUBIC_QUAD = 2, IPC_INTERP_AUTO = 3 } ipc_interp;
/* Error bound absolute, or relative to the value range (max - min). */
typedef enum { IPC_EB_ABS = 0, IPC_EB_REL = 1 } ipc_eb_mode;
/* Error model of the loader (Sec. 5.1, Theorem 1): STRICT amplifies every
 * sweep by p and adds a floating-point rounding margin (a rigorous bound);
 * PAPER applies p once per level as Theorem 1 states. */
typedef enum { IPC_BOUND_STRICT = 0, IPC_BOUND_PAPER = 1 } ipc_bound;
/* Retrieval target: kind 0 = L-inf error bound (in the field's eb mode,
 * Sec. 5.2), kind 1 = bitrate in bits per value (Sec. 5.3). */
typedef struct {
  int kind;
  double value;
} ipc_target;
enum { IPC_TARGET_EB = 0, IPC_TARGET_BITRATE = 1 };

typedef struct ipc_field ipc_field; /* compressed field: device streams + host tables */
typedef struct ipc_view ipc_view;   /* a retrieval: per-level selection (for refine) */

/* ipc_compress -- Sec. 4.1-4.4 (compression workflow of Sec. 3.2).
 *  d_in   : device array of prod(dims) elements of `dtype` (not modified).
 *  dims   : host array of ndim extents, each >= 1.
 *  eb     : error bound (> 0, finite) in `eb_mode` units. Every
 *           reconstructed value with all planes loaded is within eb of the
 *           input (Eq. 4); non-finite inputs and values whose residual
 *           exceeds the code range are stored exactly.
 *  out    : receives the new field.
 * Errors: IPC_EINVAL (shape, dtype, eb, relative eb on an all-non-finite
 * input), IPC_ENOMEM, IPC_ECUDA. Synchronises `stream`. */
int ipc_compress(const void* d_in, int dtype, int ndim, const int64_t* dims,
                 int eb_mode, double eb, int interp, int bound, void* stream,
                 ipc_field** out);

/* ipc_retrieve -- Sec. 5.2/5.3 selection + Algorithm 1 reconstruction.
 *  d_out : device array of prod(dims) elements of the field's dtype,
 *          overwritten with the reconstruction.
 *  out   : receives a view (NULL allowed when no refinement will follow).
 * The result satisfies max|x - x_out| <= the guaranteed bound reported by
 * ipc_selection (<= target in eb mode). Errors: IPC_EINVAL, IPC_EBOUND
 * (target below the compression eb), IPC_EBUDGET (bitrate below the
 * mandatory bytes), IPC_ENOMEM, IPC_ECUDA. Asynchronous on `stream`. */
int ipc_retrieve(ipc_field* f, ipc_target target, void* d_out, void* stream,
                 ipc_view** out);

/* ipc_autotune_retrieve -- launch-shape tuning of the reconstruction kernel
 * (no counterpart in the paper; the values it computes do not depend on the
 * shape). Selects as ipc_retrieve does, then reconstructs level by level,
 * timing every shape of each level's launch -- planes per tile 1, 2 or 4
 * where the level's rows allow, persistent grids of 1 .. the most CTAs per
 * SM that fit -- `reps` times each (1..100) with CUDA events on `stream`,
 * each time right after the next coarser level ran again, and records per
 * (element type, code width, level lattice extents) the shape with the
 * smallest median time (the default one unless another is faster by more
 * than 3 %) in a process-wide table. Later ipc_retrieve / ipc_refine calls, and batched
 * retrievals whose fields share a level's extents, launch with the recorded
 * shapes. d_out (device, prod(dims) elements) receives the reconstruction.
 * nshapes (optional) receives the table's size. Synchronizes `stream`.
 * Errors: those of ipc_retrieve, IPC_EINVAL for reps out of range. */
int ipc_autotune_retrieve(ipc_field* f, ipc_target target, void* d_out, void* stream, int reps,
                          int* nshapes);
/* ipc_autotune_clear -- empties the table (default shapes again). */
int ipc_autotune_clear(void);
/* ipc_autotune_entry -- entry i (0 .. size-1) of the table: element type,
 * code width (1: 16-bit), level lattice extents M[3], planes per tile and
 * CTAs per SM (0, 0: the default shape measured fastest). IPC_EINVAL when i
 * is out of range. Any output pointer may be NULL. */
int ipc_autotune_entry(int i, int* dtype, int* w16, int64_t* M, int* ns, int* per_sm);
/* ipc_autotune_set -- records a shape in the table as ipc_autotune_retrieve
 * would (replacing the entry of the same key), so that a table saved from
 * ipc_autotune_entry can be restored in another process. Accepted shapes are
 * those the tuner can record: (ns, per_sm) = (0, 0), or ns in {1, 2, 4} with
 * ns = 2 only for M[2] <= 256 and ns = 4 only for M[2] <= 128, and
 * 1 <= per_sm <= 4 (16-bit codes, or f32 with ns > 1) or 3 (otherwise).
 * Host only. Errors: IPC_EINVAL (null M, dtype, w16, extents < 1, shape). */
int ipc_autotune_set(int dtype, int w16, const int64_t* M, int ns, int per_sm);

/* Refinement forms of a view (Algorithm 2, Sec. 4.3).
 *  IPC_REFINE_CANONICAL   : a refinement reconstructs from the union of the
 *      selected planes; the result is bitwise equal to a fresh retrieval of
 *      the same planes (the default).
 *  IPC_REFINE_INCREMENTAL : a refinement reads only the newly selected planes
 *      of each level, plus a per-view state of two bits per code (the digits
 *      at the two lowest loaded planes, the prefix that decodes the next
 *      plane down, Sec. 4.4.1), and adds the interpolated increment to the
 *      array that holds the view's current reconstruction: x += Delta. Its
 *      guaranteed bound adds the increment's worst-case rounding to the
 *      canonical one; when that bound misses an error target, the refinement
 *      runs in the canonical form instead (ipc_refine_info tells which). */
/*  IPC_REFINE_AUTO        : incremental for f64 fields, canonical for f32 ones.
 *      In f32 the increment's rounding margin (u = 2^-24) misses most error
 *      targets past the first few planes, so the refinement would fall back
 *      to a reconstruction and the recorded state would cost without use;
 *      in f64 the increment nearly always applies. */
enum { IPC_REFINE_CANONICAL = 0, IPC_REFINE_INCREMENTAL = 1, IPC_REFINE_AUTO = 2 };

/* ipc_refine -- Algorithm 2. The new selection only adds planes (b'_l <= b_l
 * at every level) and minimises the added bytes. d_out: device array of
 * prod(dims) elements. Canonical form: d_out is rewritten with a
 * reconstruction bitwise equal to a fresh retrieval of the same planes.
 * Incremental form: d_out must hold the view's current reconstruction (the
 * output of its last retrieve or refine, unmodified); it is updated in place.
 * A target the view already meets (or, in bitrate mode, a budget below what
 * is loaded) leaves the view and d_out unchanged and returns IPC_OK.
 * Errors: IPC_EINVAL, IPC_EBOUND, IPC_ENOMEM, IPC_ECUDA. Asynchronous on
 * `stream`. */
int ipc_refine(ipc_view* v, ipc_target target, void* d_out, void* stream);

/* ipc_retrieve_ex -- ipc_retrieve whose view refines in `refine_mode`; in the
 * incremental form the reconstruction also records the view's state (two
 * bits per code of device memory, held until ipc_free). Errors: those of
 * ipc_retrieve; IPC_EINVAL for an unknown mode. */
int ipc_retrieve_ex(ipc_field* f, ipc_target target, void* d_out, void* stream, int refine_mode,
                    ipc_view** out);

/* ipc_view_set_refine_mode -- switches a view's refinement form. A view
 * switched to the incremental form records its state during its next
 * refinement, which therefore runs in the canonical form. */
int ipc_view_set_refine_mode(ipc_view* v, int refine_mode);

/* ipc_refine_info -- about the view's last refinement that loaded planes:
 * whether it added an increment (1) or reconstructed (0), and the plane-stream
 * bytes it read (the new planes alone for an increment; every selected plane
 * for a reconstruction). Any output pointer may be NULL. */
int ipc_refine_info(const ipc_view* v, int* incremental, uint64_t* stream_bytes);

/* ipc_free -- frees a field, a view or a plan (NULL is accepted). No work
 * that uses the handle may still be pending on any stream. */
int ipc_free(void* handle);

/* ipc_selection -- the view's per-level selection b_per_level[l-1] = planes
 * dropped at level l (host array of at least 64 ints, may be NULL), level
 * count, loaded bytes (mandatory + selected streams) and the guaranteed
 * absolute L-inf bound (Sec. 5.1). Any output pointer may be NULL. */
int ipc_selection(const ipc_view* v, int* b_per_level, int* nlevels,
                  uint64_t* bytes, double* guaranteed_bound);

/* ipc_select_container -- the selection of ipc_retrieve (Sec. 5.2 eb mode,
 * Sec. 5.3 bitrate mode) computed on the host from a container's leading
 * bytes alone: the header, the stage table and the plane-size table (the
 * outlier lists need not be present). No device work and no device needed;
 * it tells which plane streams of a stored container a retrieval reads.
 * Outputs as for ipc_selection (b_per_level: at least 64 ints, may be NULL).
 * Errors: IPC_EINVAL (null buffer, bad target), IPC_ECORRUPT (the leading
 * bytes are not a valid header or are too short), IPC_EBOUND, IPC_EBUDGET. */
int ipc_select_container(const void* buf, uint64_t len, ipc_target target, int* b_per_level,
                         int* nlevels, uint64_t* bytes, double* guaranteed_bound);

/* ipc_compressed_size -- bytes of the exported container. */
int ipc_compressed_size(const ipc_field* f, uint64_t* bytes);

/* ipc_export -- writes the container to host memory. host_buf == NULL:
 * *len receives the size. Otherwise *len is the capacity on entry (must be
 * >= size) and the size on return. Synchronous. */
int ipc_export(const ipc_field* f, void* host_buf, uint64_t* len);

/* ipc_import -- builds a device-resident field from container bytes (host
 * memory). Errors: IPC_ECORRUPT (bad magic/version/tables/stream layout),
 * IPC_ENOMEM, IPC_ECUDA. Synchronises `stream`. */
int ipc_import(const void* host_buf, uint64_t len, void* stream,
               ipc_field** out);

/* ---- progressive loading (Sec. 5: only the selected bitplanes are read) --- */
/* ipc_container_ranges -- the byte ranges of a container that hold, for
 * each level l, the streams of planes b_new[l-1] <= k < b_old[l-1] of its
 * stages, and, when b_old == NULL (nothing loaded yet), the leading tables
 * and the planes k >= b_new[l-1]. Computed from the container's leading
 * bytes (as ipc_select_container: header, stage records, plane sizes).
 * Streams are stored stage by stage, planes 31 .. 0, so each stage gives
 * one run; adjacent runs are merged. ranges: (offset, length) pairs;
 * *nranges: capacity on entry (pairs), count on return (ranges == NULL:
 * count only). Errors: IPC_ECORRUPT (tables), IPC_EINVAL (nlevels != the
 * container's level count, bounds outside 0 <= b_new <= b_old <= 32,
 * capacity). */
int ipc_container_ranges(const void* head, uint64_t head_len, const int* b_new, const int* b_old,
                         int nlevels, uint64_t* ranges, int* nranges);

/* ipc_import_partial -- a device-resident field from the bytes of those
 * ranges for b_old == NULL, concatenated in order: it holds the planes
 * k >= b_per_level[l-1] of each level. Every retrieval and refinement of it
 * selects among the planes it holds (Sec. 5.2 / 5.3 with b_l >= the
 * resident bound): a target those planes cannot meet fails with IPC_EBOUND
 * (IPC_EBUDGET for a bitrate). ipc_export refuses such a field (IPC_EINVAL)
 * until every plane is loaded. Errors as ipc_import. */
int ipc_import_partial(const void* parts, uint64_t len, const int* b_per_level, int nlevels,
                       void* stream, ipc_field** out);

/* ipc_field_load_planes -- adds the planes b_new[l-1] <= k < resident[l-1]
 * of each level to a partially loaded field, from the bytes of
 * ipc_container_ranges(b_new, resident) concatenated in order. b_new <=
 * resident per level. Synchronises `stream`; views of the field keep their
 * selections (the new planes serve later retrievals and refinements).
 * Errors: IPC_EINVAL, IPC_ECORRUPT (the streams do not match the tables),
 * IPC_ENOMEM, IPC_ECUDA. */
int ipc_field_load_planes(ipc_field* f, const void* parts, uint64_t len, const int* b_new,
                          int nlevels, void* stream);

/* ipc_field_resident -- per level, the lowest plane the field holds (all 0
 * for a field with every plane); *nlevels = K. */
int ipc_field_resident(const ipc_field* f, int* b_per_level, int* nlevels);

/* ---- lossless backend (host) --------------------------------------------- */
/* ipc_encode_container -- the lossless stage after predictive coding (Sec.
 * 6.2.1, where the paper runs zstd over the plane streams): a byte string,
 * normally an exported container, cut into blocks of 2^block_log2 bytes
 * (0: 2^20; 12..26), each coded by an order-0 range asymmetric numeral
 * system (rANS, 12-bit symbol frequencies, 32-bit state) or stored when
 * coding does not shrink it. Host memory only; blocks run on up to
 * `nthreads` host threads (0: the host's cores, at most 16). The coded
 * form: u32 magic "IPCZ", u32 version 2, u64 raw length, u32 block_log2,
 * u32 block count, u32 record size per block, the records (u8 mode 0 +
 * raw bytes, or u8 mode 2 + 256 u16 frequencies + the bytes of two rANS
 * states that code the symbols in turn -- symbol i with state i mod 2 --
 * over one stream, the two final encoder states first); little-endian.
 * Deterministic: equal inputs give equal bytes on every host.
 * out == NULL: *out_len receives an upper bound of the coded size.
 * Otherwise *out_len is the capacity on entry and the size on return.
 * Errors: IPC_EINVAL (null pointer, block size, capacity too small). */
int ipc_encode_container(const void* raw, uint64_t raw_len, int block_log2, void* out,
                         uint64_t* out_len, int nthreads);

/* ipc_decode_container -- inverse of ipc_encode_container; version 1
 * containers (mode 1 records: one state) are read too. out == NULL:
 * *out_len receives the decoded size (read from the header). Otherwise
 * *out_len is the capacity on entry and the size on return. Errors:
 * IPC_ECORRUPT (magic, version, block table, or a block that does not
 * decode to exactly its length), IPC_EINVAL. ipc_import also accepts the
 * coded form and decodes it first. */
int ipc_decode_container(const void* coded, uint64_t coded_len, void* out, uint64_t* out_len,
                         int nthreads);

/* ---- error metrics (Sec. 3.1.1 definitions; host, FP64) ------------------- */
/* Deviation of a reconstruction y from the original x (n host values of
 * `dtype`, compared in FP64). Over the positions where x is finite:
 * max_abs_err = max |x - y| (the L-inf error), mse = mean (x - y)^2 over
 * those where y is finite too (0 when there are none),
 * range = max(x) - min(x), psnr = 20 log10(range / sqrt(mse)) (+inf when
 * mse = 0, -inf when range = 0 < mse). A non-finite y there counts in
 * `nonfinite_mismatch` and leaves the sums (max_abs_err is then +inf).
 * Where x is not finite, y must hold the same class (NaN, +Inf, -Inf) --
 * the container stores those values exactly -- else it counts in
 * `nonfinite_mismatch`. `finite` = the finite positions of x. Sums run in
 * fixed chunks combined in order, so the result does not depend on the
 * number of host threads. Errors: IPC_EINVAL (null pointer with n > 0,
 * dtype). */
typedef struct {
  double max_abs_err, mse, psnr, range;
  uint64_t finite, nonfinite_mismatch;
} ipc_error_metrics;
int ipc_error_metrics_host(const void* x, const void* y, int dtype, uint64_t n,
                           ipc_error_metrics* out);

/* ---- batches (uneven fields in one launch per level) --------------------- */
/* One field of a batched compression; the fields are the same as ipc_compress
 * arguments. dims[] holds ndim extents. */
typedef struct {
  const void* d_in;
  int dtype;
  int ndim;
  int64_t dims[3];
  int eb_mode;
  double eb;
  int interp;
  int bound;
} ipc_batch_item;

/* ipc_compress_batch -- compresses nfields fields of any shapes (Sec. 4.1-4.4
 * applied to each). Per element type: one range launch over every field and
 * one host sync, then ONE kernel launch per interpolation level covering
 * that level's work of every field, and one sync for the statistics. The
 * output of field i is byte-identical to ipc_compress of that field alone.
 * outs: host array of nfields handles. On error nothing is returned.
 * A batch of 8 or more fields keeps its fields' plane streams in one device
 * allocation, released when the last of those handles is freed.
 * Synchronises `stream`. */
int ipc_compress_batch(int nfields, const ipc_batch_item* items, void* stream,
                       ipc_field** outs);

/* ipc_retrieve_batch -- Sec. 5.2/5.3 selection per field, then Algorithm 1
 * for all of them with one anchor launch and ONE launch per level over every
 * field of an element type. d_outs[i] receives field i's reconstruction,
 * bitwise equal to ipc_retrieve of that field alone. outs (may be NULL)
 * receives one view per field. Asynchronous on `stream`. */
int ipc_retrieve_batch(int n, ipc_field* const* fields, const ipc_target* targets,
                       void* const* d_outs, void* stream, ipc_view** outs);

/* A captured batched retrieval (CUDA graph) that can be replayed. */
typedef struct ipc_plan ipc_plan;
/* ipc_plan_retrieve_batch -- selects as ipc_retrieve_batch does (one element
 * type per plan), uploads the launch tables and captures the launches into a
 * CUDA graph. The fields and outputs must outlive the plan. Synchronises
 * `stream` once (table upload). Free with ipc_free. */
int ipc_plan_retrieve_batch(int n, ipc_field* const* fields, const ipc_target* targets,
                            void* const* d_outs, void* stream, ipc_plan** out);
/* ipc_plan_launch -- replays the plan's launches on `stream`. */
int ipc_plan_launch(ipc_plan* p, void* stream);

/* ---- serving: continuous batching of retrievals ---------------------------- */
typedef struct ipc_server ipc_server;
typedef struct {
  uint64_t mem_budget;   /* bytes of output buffers the server may hold         */
  uint64_t hbm_reserve;  /* free device memory a new output must leave untouched */
  int max_batch;         /* requests per launched batch (<= 0: unlimited)       */
  int max_inflight;      /* batches on the device at once (>= 1)                */
  int nstreams;          /* streams the batches rotate over (1..16)             */
  int plain;             /* 1: single-field launches per request (a baseline)   */
  uint64_t max_batch_values; /* values (output elements) per batch; a request past
                                the limit waits for the next batch, a larger one
                                runs alone (0: unlimited)                        */
  int refine_mode;       /* IPC_REFINE_*: the form of REFINE requests; in the
                            incremental form a view's refines run through its
                            own increment path (single-field launches on the
                            batch's stream), not in the batched launch      */
} ipc_server_cfg;
enum { IPC_REQ_RETRIEVE = 0, IPC_REQ_REFINE = 1, IPC_REQ_RELEASE = 2 };
/* RETRIEVE(field, target): a new view with a server-owned output buffer.
 * REFINE(view_id, target): Algorithm 2 on that view (planes only added).
 * RELEASE(view_id): frees the view and its buffer. */
typedef struct {
  int kind;
  ipc_field* field;
  uint64_t view_id;
  ipc_target target;
  uint64_t user_tag;
} ipc_request;
typedef struct {
  uint64_t ticket, user_tag;
  int status;            /* IPC_OK or the request's error                       */
  uint64_t view_id;      /* view created / refined / released                   */
  void* d_out;           /* the view's reconstruction (valid until released)    */
  uint64_t bytes;        /* loaded bytes of the view's selection                */
  double bound;          /* guaranteed L-inf bound of the selection             */
  double latency_us;     /* submit -> completion seen by the server             */
  double queue_us;       /* submit -> launch                                    */
} ipc_completion;

/* ipc_server_create -- starts a server on the current device: a worker
 * thread admits submitted requests in arrival order while output memory
 * (mem_budget, and free HBM above hbm_reserve) and the batch limits allow,
 * groups everything it admitted into one batched reconstruction
 * (ipc_retrieve_batch's launches; a batch of one takes ipc_retrieve's)
 * and rotates batches over `nstreams` streams, so requests that arrive
 * while others run are launched and overlap on the device. A request's
 * reconstruction is bitwise equal to the same request served alone. A
 * retrieve larger than mem_budget completes with IPC_ENOMEM. */
int ipc_server_create(const ipc_server_cfg* cfg, ipc_server** out);
/* ipc_server_submit -- queues a request; returns its ticket. Fields must
 * outlive the server. IPC_EBUSY after destroy began. */
int ipc_server_submit(ipc_server* s, const ipc_request* r, uint64_t* ticket);
/* ipc_server_poll -- up to `max` completions; waits up to timeout_us for
 * the first one (0: no wait). IPC_ETIMEOUT when the wait ran out. */
int ipc_server_poll(ipc_server* s, ipc_completion* out, int max, int* n, int timeout_us);
/* ipc_server_stats -- batches launched, requests launched, output bytes held. */
int ipc_server_stats(ipc_server* s, uint64_t* batches, uint64_t* requests, uint64_t* mem_used);
/* ipc_server_stop -- shuts the server down but keeps it pollable: later
 * submissions return IPC_EBUSY; work in flight finishes; what can still be
 * admitted runs; queued requests that cannot (e.g. a retrieve waiting for
 * memory) complete with IPC_EBUSY. Returns when the worker has exited. */
int ipc_server_stop(ipc_server* s);
/* ipc_server_destroy -- ipc_server_stop, then frees every view, the streams
 * and the server. */
int ipc_server_destroy(ipc_server* s);

/* ---- introspection ------------------------------------------------------- */
/* ipc_field_info -- dtype, ndim, dims (host array of 3), K (levels), S
 * (non-empty sweeps), absolute eb, and the value range over finite inputs.
 * Any output pointer may be NULL. */
int ipc_field_info(const ipc_field* f, int* dtype, int* ndim, int64_t* dims,
                   int* K, int* S, double* eb, double* xmin, double* xmax);

/* ---- allocation-free range reduction -------------------------------------- */
/* No counterpart in the paper: an entry point for callers that must not
 * allocate device memory -- a process whose device memory is all owned by
 * another pool or allocator, or a loop that must keep a fixed footprint. It
 * computes, for each of nfields device arrays of n[i] elements of `dtype`,
 * the minimum, maximum and maximum |x| over the finite values and their
 * count (the range step of ipc_compress), writing out[4*i + 0..3] = {min,
 * max, max|x|, count} (host array; all zero when an array has no finite
 * value; max|x| of signed zeros is +0). It allocates nothing: the
 * reduction's accumulators are a fixed 32 KiB device array inside the
 * library, sized for IPC_NOALLOC_MAX_FIELDS arrays per call; more arrays
 * are rejected with IPC_EINVAL. Every GPU that loads the library holds that
 * array until the process exits. Each call looks up the array's address for
 * the current device before it queues any work. The results are decoded on
 * the host, so the call waits for `stream` before it returns; a stream that
 * is being captured is refused with IPC_EINVAL before anything is queued.
 * Calls share the array: this process serialises them, but work that
 * overlaps on the GPU through other means (another process loading the
 * library runs on its own copy) would race on it. */
#define IPC_NOALLOC_MAX_FIELDS 1024
int ipc_range_noalloc(int nfields, const void* const* d_in, const uint64_t* n, int dtype,
                      void* stream, double* out);

/* ---- kernel profiler (not part of the method; measurement support) ------ */
/* Kinds of kernels the library launches. */
enum {
  IPC_KERNEL_RANGE = 0,           /* min / max / max|x| reduction               */
  IPC_KERNEL_COMPRESS_LEVEL = 1,  /* all sweeps of one level, compression       */
  IPC_KERNEL_RETRIEVE_LEVEL = 2,  /* all sweeps of one level, reconstruction    */
  IPC_KERNEL_ANCHOR = 3,          /* anchor store                               */
  IPC_KERNEL_PACK = 4,            /* device streams -> container (export)       */
  IPC_KERNEL_UNPACK = 5,          /* container -> device streams (import)       */
  IPC_KERNEL_INCREMENT_LEVEL = 6, /* all sweeps of one level, increment (Alg. 2) */
  IPC_KERNEL_COARSE = 7,          /* the coarse levels of a reconstruction, one CTA */
  IPC_KERNEL_KINDS = 8
};
/* ipc_profile_enable -- when on, every later launch is bracketed by CUDA
 * events recorded on its stream. */
int ipc_profile_enable(int on);
/* ipc_nvtx_enable -- when on, the library pushes NVTX ranges (host
 * timeline) around its calls ("ipc compress", "ipc retrieve", "ipc refine",
 * "ipc compress batch", "ipc retrieve batch", "ipc import", ...) and around
 * each level's launches inside them ("level <l>", "launch <j>" for a batch),
 * so that a profiler can select one level's kernels. Off by default. */
int ipc_nvtx_enable(int on);
/* ipc_debug_bounds -- in the bounds-checking build (compiled with
 * -DIPC_DEBUG_BOUNDS, libipcomp_bounds.so), every global access of the level
 * kernels (plane words, bitmaps, known points, outputs, the input, the
 * written streams) is tested against its array's extent; an access outside
 * it is skipped and the first one recorded. rec[4] receives (count, site,
 * index, limit) after a device synchronisation; reset clears the record.
 * Sites: 1 staged plane words, 2 staged bitmaps, 3 plane word, 4 known
 * point, 5 output, 6 input, 7 written plane word, 8 written bitmap, 9 level
 * values of a compression. The regular build returns IPC_EINVAL. */
int ipc_debug_bounds(uint64_t* rec, int reset);
/* ipc_profile_read -- waits for the recorded events and returns, for one
 * kernel kind, the number of timed launches, their summed device time (ms)
 * and their summed algorithmic bytes (compress level: input values of its
 * targets + the compacted streams it produced; retrieve level: selected
 * stream bytes + its output values; increment level: the new planes' stream
 * bytes + the state words read and written + its output values (at level 1
 * read and written); range: input bytes). */
int ipc_profile_read(int kind, uint64_t* launches, double* total_ms, double* alg_bytes);
/* ipc_profile_reset -- clears the accumulated figures. */
int ipc_profile_reset(void);
/* ipc_launch_count -- number of kernels this library has launched. */
uint64_t ipc_launch_count(void);

/* ipc_last_error -- NUL-terminated description of the calling thread's last
 * failure (empty string if none). Owned by the library. */
const char* ipc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
