/*
 * ps.h -- C ABI of the GB300 (sm_103a) Proportional Similarity library.
 *
 * Computes the 2-way and 3-way Proportional Similarity (Czekanowski)
 * metrics of Joubert, Nance, Weighill and Jacobson, "Parallel Accelerated
 * Vector Similarity Calculations for Genomics Applications" (arXiv
 * 1705.08210):
 *
 *   Section 2.1:  c2(u,v) = 2 n2(u,v) / d2(u,v),
 *                 n2 = sum_q min(u_q, v_q),  d2 = sum_q u_q + sum_q v_q
 *   Section 2.2:  c3(u,v,w) = (3/2) n3(u,v,w) / d3(u,v,w),   eq. (1):
 *                 n3 = n2(u,v) + n2(u,w) + n2(v,w) - n3'(u,v,w),
 *                 n3' = sum_q min(u_q, v_q, w_q),  d3 = sum_q (u_q+v_q+w_q)
 *
 * The numerators are computed as a "min-product" matrix product
 * M = V^T (min) V (Section 3.1); the 3-way term as B_j = X_j^T (min) V with
 * X_j = min(V, v_j) (Section 3.2).  Only non-redundant blocks are computed:
 * the upper triangle for pairs, the i<j<k tetrahedron for triples.
 *
 * ---------------------------------------------------------------------------
 * Conventions shared by every entry point
 *
 * Matrix V.  nv vectors of nf fields each, values finite and >= 0 (the paper
 *   assumes v_{i,q} >= 0, Section 2.1; negative or NaN input is undefined).
 *   layout PS_LAYOUT_FIELD_MAJOR  : element (i,q) at data[i + q*ld], ld >= nv
 *                                   ("column-major nv x nf"; default)
 *   layout PS_LAYOUT_VECTOR_MAJOR : element (i,q) at data[q + i*ld], ld >= nf
 *                                   (the paper's column-major n_f x n_v file)
 *   dtype PS_F32 or PS_F64.  FP64 input is rounded to FP32 for the numerator
 *   products of the FP32 paths; the denominators always use the original
 *   values summed in FP64.
 *
 * Pointers.  Every data pointer may be DEVICE memory (cudaMalloc, torch CUDA
 *   tensors, managed memory) or HOST memory (pinned or pageable).  The kind
 *   is detected with cudaPointerGetAttributes.  Host buffers are staged
 *   through library-owned device memory inside the call, and a call that
 *   touches any host buffer synchronises `stream` before returning.  The FP32
 *   2-way path with a host output either lets the kernel write the metrics
 *   straight into it (pinned or registered memory, n_f >= 256; see
 *   ps_config.host_direct) or computes in row bands and copies each
 *   finished band while the next one computes.  A call
 *   on device buffers only is asynchronous on `stream`.  The caller owns all
 *   buffers it passes; the library owns only its workspace (grown on demand,
 *   freed by ps_destroy).
 *
 * Errors.  Every entry point returns a ps_status.  Argument errors are
 *   detected before any launch and leave outputs untouched.  CUDA errors are
 *   reported as PS_ERR_CUDA; ps_last_error() gives the message.  No
 *   exception, abort or exit crosses this boundary.  Every wait inside a
 *   kernel is bounded (ps_config.wait_limit_ns, 2 s by default); a TMA-fed
 *   min-product kernel whose pipeline
 *   wait timed out raises a word in the handle's mapped host memory and
 *   returns, leaving that call's output incomplete: the call reports
 *   PS_ERR_TIMEOUT itself when it synchronises (host buffers), otherwise the
 *   next ps_metrics_2way / ps_metrics_2way_part / ps_metrics_3way /
 *   ps_threshold_3way call on the handle does, once.
 *
 * Threads.  A handle may be used by one host thread at a time.  Calls that
 *   overlap on the GPU (different streams, same handle) race on the handle's
 *   workspace: serialise them or use one handle per stream.
 *
 * Readings where the paper is silent:
 *   - a pair/triple whose denominator is 0 (all-zero vectors) gets metric 0;
 *   - FP32 outputs are round-to-nearest of the ratio; on integer-valued input
 *     whose sums stay below 2^24 every FP32 output equals the FP32 rounding
 *     of the exact FP64 ratio (2*n2)/(S_i+S_j) or (1.5*n3)/((S_i+S_j)+S_k).
 */
#ifndef PS_H
#define PS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t (struct CUstream_st*).  NULL means the legacy default
 * stream. */
struct CUstream_st;
typedef struct CUstream_st* ps_stream;

typedef struct ps_ctx* ps_handle;

typedef enum {
  PS_OK = 0,
  PS_ERR_INVALID_ARG = 1,
  PS_ERR_OOM = 2,
  PS_ERR_CUDA = 3,
  PS_ERR_CAPACITY = 4,
  PS_ERR_TIMEOUT = 5,
  PS_ERR_UNSUPPORTED = 6
} ps_status;

/* PS_U8 is an output type only (ps_metrics_2way and ps_metrics_2way_part,
 * paths PS_PATH_FP32 and PS_PATH_THERMO): the one-byte metric code of the
 * realistic sample problem of Section 6.8 (one unsigned byte per metric,
 * about 2.5 significant figures).  code = rint(255 * c2), round half to even,
 * evaluated in FP32 on the FP32 metric; decode c2 ~ code / 255, absolute
 * error <= 1/510 plus the FP32 error of c2.
 *
 * PS_B1 is an input type: a bit-packed 0/1 matrix (Section 2.3, where the
 * metric is the Sorenson metric).  Layout must be PS_LAYOUT_VECTOR_MAJOR;
 * field q of vector i is bit (q % 32) of the 32-bit word data[i*ld + q/32]
 * (ld in words, ld >= ceil(nf/32)); bits at q >= nf are ignored.  With
 * PS_PATH_THERMO the bits are the tensor-core operand directly (no
 * quantization; `levels` is ignored) and the result is exact; every other
 * path and call unpacks the bits to 0.0 / 1.0 first. */
typedef enum { PS_F32 = 0, PS_F64 = 1, PS_U8 = 2, PS_B1 = 3 } ps_dtype;

typedef enum {
  /* FP32 min + FP32 add on the CUDA cores, chunked and compensated
   * accumulation (relative error <= ~4e-6). */
  PS_PATH_FP32 = 0,
  /* FP64 min + FP64 add on the CUDA cores (small problems). */
  PS_PATH_FP64 = 1,
  /* Quantize to `levels` levels, thermometer-encode, and run the numerator
   * product on the tensor cores (exact on the quantized data). */
  PS_PATH_THERMO = 2,
  /* Values scaled by a power of two and rounded to FP16, pairs of fields
   * packed as half2: one packed min (min.f16x2) for two comparisons, both
   * halves added to FP32 accumulators (relative error <= ~5e-4 from the FP16
   * rounding of the inputs; exact on integers below 2048). */
  PS_PATH_HALF2 = 3
} ps_path;

typedef enum { PS_LAYOUT_FIELD_MAJOR = 0, PS_LAYOUT_VECTOR_MAJOR = 1 } ps_layout;

/* Field matrix descriptor (see "Matrix V" above). */
typedef struct {
  const void* data;
  int64_t nv;     /* number of vectors   (n_v in the paper) */
  int64_t nf;     /* fields per vector   (n_f in the paper) */
  int64_t ld;     /* leading dimension in elements */
  int32_t dtype;  /* ps_dtype */
  int32_t layout; /* ps_layout */
} ps_matrix;

/* One thresholded 2-way result: indices i<j and c2 (FP32). */
typedef struct {
  int32_t i, j;
  float value;
} ps_pair;

/* One thresholded 3-way result: indices i<j<k and c3 (FP32). */
typedef struct {
  int32_t i, j, k;
  float value;
} ps_triple;

/* ---------------------------------------------------------------------------
 * Handle configuration.  The paper fixes its precision (SP or DP) and its
 * decomposition sizes at build or job-launch time (Sections 5 and 6.5); here
 * they are per-handle run-time settings.  Every field has a default (what
 * ps_config_init writes; 0 means "automatic" in every kernel-choice field),
 * and no kernel choice depends on anything outside this struct.  Results are
 * the same, bit for bit, under every kernel choice (only speed differs).
 *
 *   precision      : arithmetic of the calls that take no path argument
 *                    (ps_metrics_2way_part, ps_metrics_batched and the 3-way
 *                    calls): PS_PATH_FP32 (default).  PS_PATH_FP64 is the
 *                    paper's DP build: ps_metrics_2way_part then computes on
 *                    the FP64 path, and the calls with no FP64 kernel (3-way,
 *                    thresholded, batched) return PS_ERR_UNSUPPORTED.
 *   debug_checks   : 1 = every call first checks that the input values are
 *                    finite and >= 0 (one extra pass over V, synchronising)
 *                    and returns PS_ERR_INVALID_ARG otherwise; 0 (default) =
 *                    such input is undefined, as the paper assumes v >= 0.
 *   wait_limit_ns  : bound of every wait inside a kernel (pipeline barriers,
 *                    grid-wide meetings, the batched launch's dependency
 *                    waits).  A wait that runs out makes the call return
 *                    PS_ERR_TIMEOUT (see "Errors" above).  Default 2e9 (2 s);
 *                    must be in [1e3, 6e10].
 *   autotune_cache : path of the JSON-lines file of ps_autotune_batched,
 *                    used when that call's cache_path is NULL, and read by
 *                    ps_metrics_batched for batch shapes the handle has not
 *                    tuned itself.  NULL = none.  The string is copied.
 *   Kernel choices of the FP32 min-product (0 = automatic):
 *   mgemm_feed     : 2-way operand feed: 1 = TMA ring (automatic),
 *                    2 = per-thread cp.async.
 *   mgemm3_feed    : 3-way operand feed: 1 = TMA ring (automatic), 2 = cp.async.
 *   mgemm_tile     : 64 or 128 (automatic) vectors per tile side of the
 *                    cp.async kernels (the TMA kernels use 128).
 *   mgemm_warps    : 8 or 16 warps per 128 x 128 tile of the cp.async
 *                    kernels (automatic: 16 for 2-way, 8 for 3-way).
 *   mgemm_unroll   : 4, 8 (automatic) or 16 k-steps per loop iteration of
 *                    the cp.async kernels.
 *   mgemm_add      : add form of the FP32 accumulators (identical values).
 *                    cp.async kernels: packed add.rn.f32x2 (automatic, 1,
 *                    3) or scalar adds (2; 8-warp 128 x 128 tiles).  TMA
 *                    2-way kernel: half of each lane's columns packed, half
 *                    scalar (automatic, 3), all packed (1) or all scalar (2;
 *                    these two with 32-field slices).  The TMA 3-way and
 *                    batched kernels always use the mixed form.
 *   mgemm_band     : tile rows per band of the 2-way tile walk, 1..64
 *                    (automatic 16).
 *   tma_slice      : fields per TMA slice, 16, 32 or 64 (automatic: 16 up
 *                    to n_f = 32; the 2-way kernel 64 above n_f = 256 and
 *                    32 between; the 3-way kernel 16 or 32 up to n_f = 16
 *                    or 32, else 64).
 *   tma_unroll     : k-steps per loop iteration of the TMA kernels, 8, 16
 *                    (automatic) or 32.
 *   tma_stages     : ring depth of 32-field TMA slices, 3, 4 (automatic) or 6.
 *   tma_schedule   : tiles of the TMA 2-way kernel: 1 = claimed from a
 *                    grid-wide counter (automatic), 2 = static round-robin.
 *   tma_meet       : with the static schedule, slices between grid-wide
 *                    meetings of the TMA producers (0 = never, automatic).
 *   mgemm3_schedule: work items of the TMA 3-way kernel: 1 = claimed from a
 *                    grid-wide counter (automatic), 2 = static round-robin.
 *   thermo_tile_m  : rows of the thermometer tensor-core tile, 128 or 256
 *                    (automatic: by the operand width).
 *   thermo_meet_kb : k-blocks between grid-wide meetings of the thermometer
 *                    GEMM's producers; 0 = automatic (960), -1 = never.
 *   mgemm_narrow   : FP32 / one-byte 2-way metrics with n_f <= 64: 1 = the
 *                    narrow kernel, whose warps write each tile's metrics
 *                    while they compute the next tile, each store
 *                    instruction writing 32 consecutive metrics of a row
 *                    (automatic); 2 = the general TMA kernel.  (The narrow
 *                    kernel needs the automatic tma_schedule, tma_meet and
 *                    tma_slice.)
 *   tma_lookahead  : slices (tiles, in the narrow kernel) the producer of the
 *                    2-way TMA kernels loads ahead of the one its warps
 *                    compute, 1..7, capped at the ring depth minus one;
 *                    0 = automatic.
 *   host_direct    : FP32 2-way calls (ps_metrics_2way, PS_PATH_FP32) whose
 *                    output is host memory pinned or registered with CUDA:
 *                    0 (default) = for n_f >= 256 the kernel writes the
 *                    metrics straight into it through its device mapping
 *                    (no staging buffer, no copy); 1 = always stage in the
 *                    workspace and copy (in row bands that overlap the
 *                    compute).
 *   test_batched_stall : testing aid for the timeout path, 0 by default.
 *                    1 = the next ps_metrics_batched call (persistent mode)
 *                    raises one dependency target by one item that does not
 *                    exist (the first 3-way problem's n2 table with the
 *                    TMA-fed kernel, problem 0's sums with the cp.async
 *                    kernels), so that the launch's dependency wait runs out
 *                    after wait_limit_ns and the call returns PS_ERR_TIMEOUT;
 *                    the setting then clears itself.  No kernel is altered:
 *                    the wait is an ordinary bounded wait on a count that
 *                    nothing completes. */
typedef struct {
  int32_t precision;
  int32_t debug_checks;
  int64_t wait_limit_ns;
  const char* autotune_cache;
  int32_t mgemm_feed;
  int32_t mgemm3_feed;
  int32_t mgemm_tile;
  int32_t mgemm_warps;
  int32_t mgemm_unroll;
  int32_t mgemm_add;
  int32_t mgemm_band;
  int32_t tma_slice;
  int32_t tma_unroll;
  int32_t tma_stages;
  int32_t tma_schedule;
  int32_t tma_meet;
  int32_t mgemm3_schedule;
  int32_t thermo_tile_m;
  int32_t thermo_meet_kb;
  int32_t test_batched_stall;
  int32_t mgemm_narrow;
  int32_t tma_lookahead;
  int32_t host_direct;
} ps_config;

/* Defaults: precision PS_PATH_FP32, no debug checks, 2 s wait limit, no
 * autotune cache, every kernel choice automatic (0). */
void ps_config_init(ps_config* cfg);

/* ---------------------------------------------------------------------------
 * Handle.  ps_create binds a handle to CUDA device `device` (the device is
 * made current inside each call) with configuration `cfg` (copied; NULL =
 * ps_config_init's defaults).  Returns PS_ERR_INVALID_ARG for a null `out`,
 * an invalid device or a configuration field outside the ranges above,
 * PS_ERR_CUDA if the device cannot be used. */
ps_status ps_create(ps_handle* out, int device, const ps_config* cfg);
/* Current configuration of `h` (autotune_cache points at the handle's copy,
 * valid until the next ps_set_config or ps_destroy). */
ps_status ps_get_config(ps_handle h, ps_config* cfg);
/* Replaces the configuration of `h` (validated as in ps_create); applies to
 * later calls.  Synchronises the device first, so no queued call of the
 * handle runs under the old settings. */
ps_status ps_set_config(ps_handle h, const ps_config* cfg);
/* Frees the handle and its workspace (synchronises the device first).
 * NULL is accepted. */
ps_status ps_destroy(ps_handle h);

/* Static string for a status code (never NULL). */
const char* ps_status_string(ps_status s);
/* Message of the last failing call on `h` ("" if none); valid until the next
 * call on `h`.  NULL handle gives the last message of any handle. */
const char* ps_last_error(ps_handle h);
/* Library version string. */
const char* ps_version(void);

/* ---------------------------------------------------------------------------
 * Per-vector sums S_i = sum_q v_{i,q} in FP64 (Section 2.1: the denominator
 * d2 = S_i + S_j needs only these O(n_f n_v) adds; Section 2.2: d3 likewise).
 *   S : nv doubles, device or host.
 * Errors: PS_ERR_INVALID_ARG for a null/invalid matrix or null S. */
ps_status ps_vector_sums(ps_handle h, const ps_matrix* V, double* S,
                         ps_stream stream);

/* ---------------------------------------------------------------------------
 * All 2-way metrics c2(v_i, v_j), i < j (Section 2.1; the numerators are the
 * strict upper triangle of M = V^T (min) V, Section 3.1).
 *   path      : ps_path.
 *   levels    : PS_PATH_THERMO only, number of quantization levels L in
 *               [2, 16]; ignored otherwise.
 *   out       : nv*(nv-1)/2 values of out_dtype (PS_F32, PS_F64, or PS_U8
 *               codes with PS_PATH_FP32 / PS_PATH_THERMO), packed
 *               strict upper triangle, row-major:
 *                 out[i*(2*nv-i-1)/2 + (j-i-1)] = c2(v_i, v_j),  i < j.
 *               For PS_PATH_THERMO the metric is that of the quantized
 *               levels (the scale cancels in the ratio).
 * Errors: PS_ERR_INVALID_ARG for nv < 2, nf < 0, a bad ld/layout/dtype/path,
 *   levels out of range, or null pointers; PS_ERR_OOM if the workspace
 *   cannot grow. */
ps_status ps_metrics_2way(ps_handle h, const ps_matrix* V, int32_t path,
                          int32_t levels, void* out, int32_t out_dtype,
                          ps_stream stream);

/* Size in elements of the pivot slab [j_begin, j_end) written by
 * ps_metrics_3way: sum over j of j*(nv-1-j).  Returns -1 on bad arguments. */
int64_t ps_slab_size(int64_t nv, int64_t j_begin, int64_t j_end);

/* ---------------------------------------------------------------------------
 * 3-way metrics c3(v_i, v_j, v_k), i < j < k, for the pivots j in
 * [j_begin, j_end) (Section 2.2 eq. (1); n3' via B_j = X_j^T (min) V with
 * X_j = min(V, v_j), Section 3.2, computing only i < j < k).
 *   out_slab : ps_slab_size(nv, j_begin, j_end) floats.  Pivot j owns a
 *              j x (nv-1-j) row-major block (rows i in [0,j), columns k in
 *              (j,nv)); blocks follow in increasing j:
 *                out_slab[off(j) + i*(nv-1-j) + (k-j-1)] = c3(v_i,v_j,v_k),
 *                off(j) = ps_slab_size(nv, j_begin, j).
 *              Computing a campaign in slabs is the paper's staging
 *              (Section 4.2): a run can resume from any pivot.
 * Only PS_PATH_FP32 arithmetic is used (FP32 min/add, FP64 sums).
 * Errors: PS_ERR_INVALID_ARG for nv < 3, 0 <= j_begin <= j_end <= nv
 *   violated, or null pointers. */
ps_status ps_metrics_3way(ps_handle h, const ps_matrix* V, int64_t j_begin,
                          int64_t j_end, float* out_slab, ps_stream stream);

/* ---------------------------------------------------------------------------
 * Thresholded 3-way search: every triple i<j<k with c3 >= tau, sorted
 * lexicographically by (i,j,k).
 *   use_proposal : 0 = exhaustive over all 128-tile blocks (I<=J<=K);
 *                  1 = only the blocks the trained encoder proposes
 *                      (ps_proposal_train; vectors reordered by its
 *                      clusters; falls back to exhaustive when more than 60%
 *                      of the blocks are proposed); recall < 1 is possible;
 *                  2 = only blocks that the bound
 *                      c3 <= 1.5 min(n2ij+n2ik+n2jk, n2jk+S_i, n2ik+S_j,
 *                      n2ij+S_k) / d3 (from min(a,b,c) >= min(a,b) +
 *                      min(a,c) - a) cannot rule out: lossless; reordered by
 *                      the encoder when one is trained for this nf.
 *                  Every reported value equals the exhaustive one bit for
 *                  bit (eq. (1) is summed in original index order).
 *   out          : `capacity` ps_triple slots (device or host).
 *   count        : one int64 (device or host) receiving the total number of
 *                  triples found, also when it exceeds `capacity`.
 * Returns PS_ERR_CAPACITY when the total exceeds `capacity`; the first
 * `capacity` triples in sorted order are then written.
 * Synchronous: returns once the result and count are written.
 * Errors: PS_ERR_INVALID_ARG for nv < 3 or nv > 2^21, capacity < 0, null
 *   pointers, use_proposal outside 0..2, or use_proposal 1 without a trained
 *   encoder for this nf. */
ps_status ps_threshold_3way(ps_handle h, const ps_matrix* V, float tau,
                            int32_t use_proposal, ps_triple* out,
                            int64_t capacity, int64_t* count,
                            ps_stream stream);

/* ---------------------------------------------------------------------------
 * Thresholded 2-way metrics: every pair i < j with c2(v_i, v_j) >= tau
 * (Section 2.1's metric; thresholding the output, as Section 6.8's
 * discussion of the metric data volume suggests, instead of writing all
 * nv(nv-1)/2 values).  Values are bit-identical to ps_metrics_2way with
 * PS_PATH_FP32 and PS_F32 output; pairs are sorted by (i, j).
 *   out      : `capacity` ps_pair slots (device or host).
 *   count    : one int64 (device or host) receiving the total number of
 *              pairs found, also when it exceeds `capacity`.
 * Returns PS_ERR_CAPACITY when the total exceeds `capacity`; the first
 * `capacity` pairs in sorted order are then written.
 * Synchronous: returns once the result and count are written.
 * Errors: PS_ERR_INVALID_ARG for nv < 2 or nv > 2^31 - 1, capacity < 0 or
 *   null pointers; PS_ERR_OOM if the hit buffer cannot grow. */
ps_status ps_threshold_2way(ps_handle h, const ps_matrix* V, float tau,
                            ps_pair* out, int64_t capacity, int64_t* count,
                            ps_stream stream);

/* ---------------------------------------------------------------------------
 * Sharding over several GPUs (one process per GPU; V replicated, no
 * collective on the data path).  The paper splits the vector axis over nodes
 * with circulant exchanges (Section 4.1); with V resident on every GPU the
 * unique outputs are simply split into equal-work contiguous ranges.
 *
 * ps_partition: host-only (no GPU needed).  way 2: rows [begin, end) of the
 *   packed triangle (128-row bands, ~1/nparts of the pairs each); their
 *   outputs are packed entries [out_begin, out_end).  way 3: pivots
 *   [begin, end) (pass them to ps_metrics_3way), slab entries
 *   [out_begin, out_end) of the full pivot range.  out_begin / out_end may
 *   be NULL.  Parts are disjoint and cover everything.
 * ps_metrics_2way_part: the pairs of rows [begin, end) of part `part`,
 *   written at their packed positions of the full nv*(nv-1)/2 DEVICE array
 *   `out` (other entries untouched); FP32 path, or the FP64 path under a
 *   handle whose ps_config.precision is PS_PATH_FP64.
 * Errors: PS_ERR_INVALID_ARG for bad sizes or part indices. */
ps_status ps_partition(int64_t nv, int32_t way, int32_t nparts, int32_t part,
                       int64_t* begin, int64_t* end, int64_t* out_begin,
                       int64_t* out_end);
ps_status ps_metrics_2way_part(ps_handle h, const ps_matrix* V, int32_t nparts,
                               int32_t part, void* out, int32_t out_dtype,
                               ps_stream stream);

/* ---------------------------------------------------------------------------
 * Batched uneven instances (not in the paper, whose unit of work is one
 * large decomposed problem, Section 4).  Each problem: */
typedef struct {
  ps_matrix V;       /* PS_F32, PS_LAYOUT_FIELD_MAJOR, ld % 4 == 0, 16-byte
                        aligned DEVICE memory; 2-way nv >= 2, 3-way nv >= 3,
                        nv <= 2^20 */
  int32_t way;       /* 2 or 3 */
  int32_t out_dtype; /* 2-way: PS_F32 or PS_F64; 3-way: PS_F32 */
  void* out;         /* DEVICE memory: 2-way nv*(nv-1)/2 packed pairs (as
                        ps_metrics_2way); 3-way ps_slab_size(nv, 0, nv) floats
                        (all pivots, as ps_metrics_3way) */
} ps_problem;

#define PS_BATCH_PERSISTENT 0   /* one persistent launch, CUDA graph */
#define PS_BATCH_PER_INSTANCE 1 /* one ps_metrics_2way/3way call each */

/* All problems of the batch.  PS_BATCH_PERSISTENT: one CUDA graph holding
 * the per-vector sums of every problem and one persistent kernel whose CTAs
 * take work items (2-way tiles, n2-table tiles, 3-way pivot tiles of every
 * problem, longest first) from an atomic queue; a 3-way epilogue waits for
 * its problem's n2 table, whose tiles sit earlier in the queue.  Default
 * kernel: TMA-fed (tensor maps per problem, mbarrier ring); the autotuner's
 * other candidates are cp.async kernels that also take the sum blocks from
 * the queue.  The graph is captured once per batch (same shapes, pointers,
 * kernel variant and wait limit), kept in the handle and replayed on later
 * calls; the handle also keeps that batch's device state (sums, n2 tables,
 * work list) until ps_destroy.  Results are bit-identical to
 * PS_BATCH_PER_INSTANCE, which is the comparison point.  The kernel variant
 * is the one ps_autotune_batched chose for these shapes (or the configured
 * autotune cache holds), else the default.  Synchronises `stream` (it reads
 * the launch's error flag).
 * Errors: PS_ERR_INVALID_ARG for a problem outside the limits above;
 *   PS_ERR_TIMEOUT if a dependency wait inside the launch ran out
 *   (ps_config.wait_limit_ns; the handle stays usable);
 *   PS_ERR_UNSUPPORTED under FP64 precision. */
ps_status ps_metrics_batched(ps_handle h, const ps_problem* probs, int32_t n,
                             int32_t mode, ps_stream stream);

/* Autotuner of the batched launch: times every kernel configuration (the
 * TMA-fed kernel; cp.async kernels with tile 128 x 128 and 8 or 16 warps or
 * 64 x 64 with 2 warps, k-unroll depth 16, 8 or 4) on these problems, keeps the fastest for this batch shape in the
 * handle and appends {"shape_signature", "variant", "ms"} as one JSON line to
 * cache_path (NULL: the handle's ps_config.autotune_cache, if any).  If that
 * file already holds this shape signature, its variant is used without
 * measuring.  choice (if not NULL)
 * receives a readable description of the chosen configuration.
 * Errors: as ps_metrics_batched. */
ps_status ps_autotune_batched(ps_handle h, const ps_problem* probs, int32_t n,
                              const char* cache_path, char* choice,
                              int32_t choice_len, ps_stream stream);

/* ---------------------------------------------------------------------------
 * Learned block proposal for ps_threshold_3way (not in the paper).
 * Encoder: e_i = W2 relu(W1 x_i + b1) + b2, x_iq = log1p(v_iq n_f / S_i) (d_in = n_f
 * inputs, 256 hidden, 64 outputs), BF16 weights in the products, FP32
 * accumulation, FP32 master weights; p_i = softmax(e_i) is a soft
 * assignment to 64 learned clusters and a pair is scored
 * P_ij = p_i . p_j (probability of sharing a cluster).
 * Parameters (FP32, this order): W1[256][d_in], b1[256], W2[64][256], b2[64].
 * The encoder lives in the handle.
 *
 * ps_proposal_init: allocates and initialises (Glorot-uniform weights from a
 *   seeded host generator, zero biases).
 * ps_proposal_param_count: number of parameters (-1 without an encoder).
 * ps_proposal_params: set != 0 copies `params` into the encoder (and, with a
 *   non-NULL theta, marks it trained with that proposal threshold);
 *   set == 0 copies the parameters (and theta) out.  Host or device memory.
 * ps_proposal_pair_grad: embeddings E (nv x 64, row-major) of an FP32
 *   field-major DEVICE matrix with nf = d_in, and, when grad is not NULL, the
 *   gradient of the mean binary cross-entropy of P (clamped to
 *   [1e-6, 1-1e-6]) over `npairs` pairs (pairs[2p],
 *   pairs[2p+1] vector indices, labels 0/1; device memory) in parameter
 *   order, and the loss.  Synchronises `stream`.
 * ps_proposal_train: for every training matrix (FP32 field-major DEVICE,
 *   one common nf, ld % 4 == 0; typically small random subsets of the
 *   vectors to be searched, which share their population's structure) runs
 *   the exact thresholded search at `tau`,
 *   labels a pair positive when it belongs to a triple with c3 >= tau, adds
 *   4 random negatives per positive, then takes `steps` Adam steps (rate lr)
 *   on the pair loss, cycling through the matrices, and sets the
 *   proposal threshold theta to the (1 - target_recall) quantile of the
 *   positive pair scores.  final_loss (may be NULL) receives the last loss.
 * ps_proposal_last_stats: fraction of the 128-tile blocks (I<=J<=K) that
 *   the last ps_threshold_3way call searched, and their number.
 * Errors: PS_ERR_INVALID_ARG for bad sizes or a missing encoder. */
ps_status ps_proposal_init(ps_handle h, int32_t d_in, uint64_t seed);
int64_t ps_proposal_param_count(ps_handle h);
ps_status ps_proposal_params(ps_handle h, int32_t set, float* params,
                             int64_t n, float* theta);
ps_status ps_proposal_pair_grad(ps_handle h, const ps_matrix* V,
                                const int32_t* pairs, const float* labels,
                                int64_t npairs, float* E_out, float* grad,
                                double* loss, ps_stream stream);
ps_status ps_proposal_train(ps_handle h, const ps_matrix* train,
                            int32_t ntrain, float tau, int32_t steps, float lr,
                            float target_recall, uint64_t seed,
                            double* final_loss, ps_stream stream);
ps_status ps_proposal_last_stats(ps_handle h, double* kept_fraction,
                                 int64_t* blocks);

/* ---------------------------------------------------------------------------
 * Quantizer of the thermometer path (not in the paper).
 *   P      : the nearest-rank 99.9th percentile of the nonzero entries
 *            (rank ceil(0.999*m) of m nonzeros, ascending, 1-based);
 *            0 if all entries are zero.
 *   level  : 0 for a zero entry, else
 *            min(L-1, floor(fl32(fl32(x * r) + 0.5))),  r = fl32((L-1)/P),
 *            all in IEEE single precision.
 *   P_out  : one float (device or host).
 *   q_out  : nv*nf bytes, field-major with leading dimension nv (device or
 *            host); may be NULL to compute P only.
 * Errors: PS_ERR_INVALID_ARG for levels outside [2,16] or null P_out. */
ps_status ps_quantize(ps_handle h, const ps_matrix* V, int32_t levels,
                      float* P_out, uint8_t* q_out, ps_stream stream);

/* ---------------------------------------------------------------------------
 * Kernel timing for benchmarks (no counterpart in the paper, which reads
 * kernel times from the CUDA profiler, Section 6.2).  While enabled, every
 * launch of a library kernel is bracketed by two CUDA events recorded on the
 * stream the kernel is launched on.  ps_timing_enable clears the records
 * (it waits for recorded events first).
 * ps_timing_read synchronises on the recorded events of `kernel` and returns
 * their number and summed duration.  Kernel names: "vector_sums", "pack",
 * "mgemm2", "mgemm2_f64", "mgemm2_half", "mgemm2_n2", "mgemm3", "quantize",
 * "thermo_encode", "b1_encode", "thermo_gemm", "threshold2", "threshold3",
 * "sort", "batched", "proposal_encode", "proposal_score", "proposal_bound";
 * and two regions of ps_proposal_train: "proposal_labels" (the exact
 * thresholded search of one training matrix, one record each) and
 * "proposal_steps" (all training steps, one record).
 * Errors: PS_ERR_INVALID_ARG for null arguments. */
ps_status ps_timing_enable(ps_handle h, int32_t enable);
ps_status ps_timing_read(ps_handle h, const char* kernel, int64_t* launches,
                         double* total_ms);

/* ---------------------------------------------------------------------------
 * Measured CUDA-core issue rate of the paper's inner operation (one min plus
 * one add per element pair, Section 3.1), from a register-only kernel of
 * independent min/add chains over the whole GPU.  variant 0: scalar FP32
 * min + scalar FP32 add; variant 1: FP32 min + packed f32x2 add; variant 2:
 * the half2 path's operation, one packed FP16 min (two comparisons) and two
 * FP32 adds of its halves; variant 3: the min as the signed-integer min of
 * the bit patterns (equal for non-negative floats) + scalar FP32 add;
 * variant 4: FP32 min, half the chains with scalar adds and half with
 * packed f32x2 adds.
 *   cmp_per_s : comparisons (min+add pairs) per second.
 * Synchronises the device.  Errors: PS_ERR_INVALID_ARG for a bad variant. */
ps_status ps_probe_minadd_peak(ps_handle h, int32_t variant,
                               double* cmp_per_s);

/* ---------------------------------------------------------------------------
 * 2-way metrics without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot let a library call
 * cudaMalloc -- services whose device memory is owned in full by their own
 * allocator or by a fixed budget set at start-up (a framework caching
 * allocator that must account for every byte, a long-running service that
 * forbids cudaMalloc/cudaFree after warm-up because they can synchronise the
 * device and fragment memory).
 *
 * Same result as ps_metrics_2way(..., PS_PATH_FP32, ...) on the current CUDA
 * device, with these limits:
 *   - V must be PS_F32, PS_LAYOUT_FIELD_MAJOR, ld a multiple of 4, data
 *     16-byte aligned, 2 <= nv <= PS_STATIC_MAX_NV (65536);
 *   - V->data and out must be DEVICE memory (no host staging);
 *   - out: nv*(nv-1)/2 values of out_dtype (PS_F32 or PS_F64), packed as in
 *     ps_metrics_2way.
 * Its only scratch (nv FP64 sums) lives in a 512 KiB array inside the
 * library's device image, held on every GPU that loads the library until the
 * process exits.  No handle is used and nothing is allocated.  Every call
 * looks up that array's device address (cudaGetSymbolAddress, a host-side
 * query); the first call on a device also loads the library's kernels there
 * and sets kernel attributes, so make that first call before any stream
 * capture.  The call always runs the 16-warp 128 x 128 cp.async min-product
 * kernel under the default configuration (no handle, so no ps_config
 * applies); its values equal those of ps_metrics_2way's default TMA-fed
 * kernel bit for bit.
 * All calls share the array and it keeps the last call's contents; every call
 * rewrites the entries it reads, so nothing needs clearing.  Calls that
 * overlap on the GPU (other streams or host threads) race on the array:
 * serialise them.  Asynchronous on `stream`.
 * Errors: PS_ERR_INVALID_ARG for any violated limit (message via
 * ps_last_error(NULL)); PS_ERR_CUDA for a CUDA failure. */
#define PS_STATIC_MAX_NV 65536
ps_status ps_metrics_2way_static(const ps_matrix* V, void* out,
                                 int32_t out_dtype, ps_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* PS_H */
