/*
 * hc.h -- C ABI of libhc.so: HSZp-style error-bounded compression with
 * multi-stage partial decompression and homomorphic analytical operations on
 * the intermediate stages, for one NVIDIA GB300 (sm_103a) GPU.
 *
 * Paper: "HSZ" (arXiv 2603.25206).  Problem statement, Section III-A: a
 * compressor C, decompression stages D_1..D_m and operations Q_i run on the
 * intermediate representation d^(i) = D_i(...D_1(c)).  Stages follow Table 1:
 *   1 = D_m (block metadata), 2 = D_p (decorrelated integers),
 *   3 = D_q (quantization integers), 4 = D_f (decompressed floats).
 *
 * Conventions for every call:
 *  - Pointers named d_* are DEVICE pointers on the current CUDA device; all
 *    other pointers are host pointers.  The library never allocates or frees
 *    device memory: callers pass outputs and a workspace sized by the
 *    *_workspace_bytes queries.  Device buffers must be 16-byte aligned.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls marked ASYNC only enqueue kernels on it and return; their
 *    results are valid once the stream has been synchronised.  Calls marked
 *    SYNC wait for the stream before returning.
 *  - Return value: HC_OK, or an error code with a message readable through
 *    hc_last_error() (thread-local).  Argument errors are detected on the
 *    host before anything is enqueued.  A corrupt stream found by a kernel is
 *    reported through a device status word: the `status` field of an
 *    hc_scalar result, or the first int32 of the workspace for field results
 *    (read it with hc_workspace_status).  Kernels never read outside the
 *    stream, whatever its content.
 *  - A host hc_header passed by the caller (hc_decompress_to_stage, an
 *    hc_stage of kind HC_STAGE_COMPRESSED, hc_autotune, hc_batch_plan,
 *    hc_shard_plan) is
 *    checked on the host before anything is enqueued: its section offsets,
 *    sizes, block or box extents, width, eps and max |q| must follow from
 *    its shape and block size, else HC_ERR_CORRUPT.  The header must still
 *    describe the device stream passed with it (hc_read_header of that
 *    stream, or the one hc_compress returned).
 *  - No C++ exception crosses this interface.
 */
#ifndef HC_H
#define HC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define HC_API __attribute__((visibility("default")))
#else
#define HC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HC_OK = 0,
  HC_ERR_INVALID_ARG = 1,  /* bad pointer, size, shape, dtype, or mismatch with the stream header */
  HC_ERR_RANGE = 2,        /* a code |q| >= 2^30, or a non-finite input value */
  HC_ERR_CORRUPT = 3,      /* the stream violates its layout */
  HC_ERR_UNSUPPORTED = 4,  /* operation not defined at this stage (Section V-B) */
  HC_ERR_CUDA = 5,         /* a CUDA runtime call failed */
  HC_ERR_NOMEM = 6,        /* the caller's buffer or workspace is too small */
  HC_ERR_TIMEOUT = 7       /* a bounded wait ran out */
} hc_status;

typedef enum { HC_F32 = 0, HC_F64 = 1, HC_I32 = 2, HC_I64 = 3 } hc_dtype;
typedef enum {
  HC_OP_MEAN = 0,
  HC_OP_VARIANCE = 1,
  HC_OP_DERIVATIVE = 2,
  HC_OP_GRADMAG = 3,
  HC_OP_LAPLACIAN = 4,
  HC_OP_MULTI = 5 /* every operation in one pass (hc_op_multi) */
} hc_op;
typedef enum { HC_EB_ABS = 0, HC_EB_REL = 1 } hc_eb_mode;
/* Decorrelation (Section IV).  DELTA: the block's first code is metadata and
 * p_k = q_k - q_{k-1} inside the block (HSZp with SZp-style block heads).
 * MEAN: the block mean M_b (nearest integer to the code sum over the block
 * size, ties toward zero) is metadata and p_k = q_k - M_b (HSZx).
 * The two global predictors keep no block metadata (heads are 0) and predict
 * across block boundaries; blocks only group residuals for the encoder:
 *   LORENZO (HSZp-nd): the multidimensional Lorenzo residual over the
 *     field's axes -- 1-D p_i = q_i - q_{i-1}; 2-D p_{i,j} = q_{i,j} -
 *     q_{i,j-1} - q_{i-1,j} + q_{i-1,j-1}; 3-D the eight-term form -- with
 *     codes before the field taken as 0;
 *   GLOBAL_DELTA (HSZp): p_i = q_i - q_{i-1} over the row-major flattened
 *     field (p_0 = q_0), whatever its ndim.
 * So q is the prefix sum of D_p over every prediction axis (the field's axes
 * for LORENZO, the flattened field for GLOBAL_DELTA).  A global-predictor
 * residual must satisfy |p| < 2^31 (else HC_ERR_RANGE at compression). */
typedef enum {
  HC_PRED_DELTA = 0,
  HC_PRED_MEAN = 1,
  HC_PRED_LORENZO = 2,
  HC_PRED_GLOBAL_DELTA = 3,
  HC_PRED_MEAN_ND = 4 /* HSZx-nd: block means over boxes of codes (hc_compress_nd) */
} hc_predictor;
typedef enum {
  HC_STAGE_COMPRESSED = 0, /* the stream itself (operations fuse decoding in) */
  HC_STAGE_M = 1,          /* D_m: heads int32[nb] */
  HC_STAGE_P = 2,          /* D_p: int32[N], block head in each block's first slot */
  HC_STAGE_Q = 3,          /* D_q: int32[N] */
  HC_STAGE_F = 4           /* D_f: float32 or float64 [N] */
} hc_stage_kind;

/* Host copy of a stream header (layout: 256-byte little-endian header followed
 * by widths u8[nb], heads i32[nb], chunk index u64[nchunks+1] and payload
 * u32 words, each section 16-byte aligned; see the stream layout notes in the
 * library source).  Filled by hc_read_header. */
typedef struct hc_header {
  int32_t dtype;     /* HC_F32 or HC_F64: the type of the original field */
  int32_t ndim;      /* 1..3 */
  int64_t dims[3];   /* (n0, n1, n2) row-major, n2 fastest, leading ones for ndim < 3 */
  int32_t S;         /* block size, 1..4096 */
  int32_t G;         /* blocks per chunk = max(1, 4096 / S) */
  double eps;        /* absolute error bound used by the quantizer */
  double eb;         /* error bound as given */
  int32_t eb_mode;   /* HC_EB_ABS or HC_EB_REL */
  uint32_t qmax;     /* max |q| over the field */
  int64_t N, nb, nchunks, payload_words;
  int64_t off_widths, off_heads, off_chunks, off_payload, total_bytes;
  uint32_t wmax;     /* largest block width */
  uint32_t pred;     /* hc_predictor the stream was written with */
  uint32_t block[3]; /* HC_PRED_MEAN_ND: box extents (b0, b1, b2) along (n0, n1, n2), leading ones;
                        S = b0 b1 b2.  0 for the other predictors */
} hc_header;

/* An input of an operation: the stream (fused decode + operation) or a
 * materialized stage array. */
typedef struct hc_stage {
  int32_t kind;          /* hc_stage_kind */
  int32_t level;         /* COMPRESSED only: the stage the fused kernel works at,
                            HC_STAGE_P (Section V, "Operation with D_p") or
                            HC_STAGE_Q ("Operation with D_q") */
  const void* d_data;    /* stream bytes, or the stage array */
  const hc_header* hdr;  /* COMPRESSED: header of d_data (from hc_read_header) */
  int32_t dtype;         /* F: HC_F32 / HC_F64 */
  int32_t S;             /* P: block size of the stream the array came from */
  int64_t n;             /* P / Q / F: element count */
  uint32_t qmax;         /* P / Q: an upper bound on |q|, 0 if unknown */
  uint32_t pred;         /* M / P arrays: hc_predictor of the stream they came from */
} hc_stage;

/* Device-resident result of a statistic.  Integer stages carry the exact
 * sums; the float stage (plain path) carries zeros there and exact = 0. */
typedef struct hc_scalar {
  double mean;       /* (sum q / N) * 2 eps                         (Section V-A) */
  double variance;   /* (N s2 - s1^2) / (N (N-1)) * (2 eps)^2        (Eq. var_q) */
  double std;        /* sqrt(variance)                               (Eq. var)   */
  int64_t n;         /* N */
  int64_t s1;        /* sum q, exact */
  uint64_t s2_lo;    /* sum q^2, exact, low 64 bits  (variance only) */
  uint64_t s2_hi;    /* sum q^2, high 64 bits */
  int32_t status;    /* HC_OK or the error a kernel found */
  int32_t exact;     /* 1 when s1 / s2 are exact integer sums */
} hc_scalar;

/* ----------------------------------------------------------- diagnostics */
HC_API const char* hc_status_str(int status);
HC_API const char* hc_last_error(void);
HC_API int hc_version(void);

/* ------------------------------------------------------------ sizing (host) */
/* Upper bound of the stream size for N elements at block size S (every block
 * at width 31).  Returns 0 for invalid arguments. */
HC_API size_t hc_compress_bound(int64_t n, int S);
/* Workspace of hc_compress for N elements at block size S. */
HC_API size_t hc_compress_workspace_bytes(int64_t n, int S);
/* Workspace of any hc_decompress_to_stage / hc_op_* call on a DELTA or MEAN
 * stream or on a stage array (one size fits all). */
HC_API size_t hc_workspace_bytes(void);
/* Workspace of any call on the stream `hdr` describes: hc_workspace_bytes()
 * for DELTA and MEAN streams; for the global predictors (LORENZO,
 * GLOBAL_DELTA) hc_workspace_bytes() plus scratch for a rebuilt D_q and the
 * prefix sums (about 12.3 bytes per element); for MEAN_ND streams
 * hc_workspace_bytes() plus 4 bytes per element (a stage in field order).
 * 0 for a NULL header, or one whose ndim, extents (>= 1, product N), box
 * extents or predictor are invalid. */
HC_API size_t hc_workspace_bytes_for(const hc_header* hdr);
/* Bytes of a materialized stage (M, P, Q or F; F in the header's dtype). */
HC_API size_t hc_stage_bytes(const hc_header* hdr, int kind);

/* ------------------------------------------------------------ compression */
/* C (Algorithm 1, Section IV): quantize q = floor(x / (2 eps) + 0.5) (IEEE
 * double), partition into blocks of S, keep each block's first code as
 * metadata, delta-code inside the block, and encode every block at the bit
 * width of its largest |p| with the sign bits first.
 *   d_x: float32 or float64 field (dtype), row-major dims[0..ndim).
 *   eb, eb_mode: absolute bound, or eb * (max - min) (Section VI-B); a
 *     constant field with a relative bound uses eps = eb.
 *   d_stream, cap: output buffer of at least hc_compress_bound(N, S) bytes.
 *   d_ws, ws_bytes: hc_compress_workspace_bytes(N, S) bytes of scratch.
 *   out_bytes, hdr_out (host, hdr_out may be NULL): stream size and header.
 * SYNC.  HC_ERR_RANGE if a code would not fit in (-2^30, 2^30). */
HC_API int hc_compress(const void* d_x, int dtype, int ndim, const int64_t* dims, double eb, int eb_mode, int S,
                void* d_stream, size_t cap, void* d_ws, size_t ws_bytes, size_t* out_bytes,
                hc_header* hdr_out, void* stream);

/* Encoder on given codes (the steps of Algorithm 1 after quantization):
 * d_q int32[N] with |q| < 2^30; eps/eb/eb_mode/dtype are recorded in the
 * header.  SYNC.  Produces the same bytes as hc_compress on the field. */
HC_API int hc_compress_codes(const int32_t* d_q, int dtype, int ndim, const int64_t* dims, double eps, double eb,
                      int eb_mode, int S, void* d_stream, size_t cap, void* d_ws, size_t ws_bytes,
                      size_t* out_bytes, hc_header* hdr_out, void* stream);

/* hc_compress / hc_compress_codes with a choice of decorrelation
 * (hc_predictor): HC_PRED_DELTA gives the same bytes as hc_compress,
 * HC_PRED_MEAN writes an HSZx stream (block means as metadata, p = q - M_b;
 * Section IV, "HSZx").  SYNC. */
HC_API int hc_compress_ex(const void* d_x, int dtype, int ndim, const int64_t* dims, double eb, int eb_mode, int S,
                          int predictor, void* d_stream, size_t cap, void* d_ws, size_t ws_bytes, size_t* out_bytes,
                          hc_header* hdr_out, void* stream);
HC_API int hc_compress_codes_ex(const int32_t* d_q, int dtype, int ndim, const int64_t* dims, double eps, double eb,
                                int eb_mode, int S, int predictor, void* d_stream, size_t cap, void* d_ws,
                                size_t ws_bytes, size_t* out_bytes, hc_header* hdr_out, void* stream);

/* HSZx-nd (Section IV, "HSZx-nd"): the field is partitioned into boxes of
 * block[0] x ... x block[ndim-1] codes (one extent per axis, product S <=
 * 4096) and each box is decorrelated by its integer mean, p = q - M_b (M_b the
 * nearest integer to the box's code sum over its true size, ties toward zero;
 * a box cut by the end of the field has the true size of its clipped extents
 * and zero in the slots outside the field).  Boxes are stored in row-major
 * order of the box grid ceil(n_a / b_a), the S slots of a box row-major inside
 * it; header byte 140 = HC_PRED_MEAN_ND and bytes 144..155 the extents.
 * Sizing: hc_compress_bound_nd / hc_compress_workspace_bytes_nd.  SYNC. */
HC_API size_t hc_compress_bound_nd(int ndim, const int64_t* dims, const int32_t* block);
HC_API size_t hc_compress_workspace_bytes_nd(int ndim, const int64_t* dims, const int32_t* block);
HC_API int hc_compress_nd(const void* d_x, int dtype, int ndim, const int64_t* dims, const int32_t* block, double eb,
                          int eb_mode, void* d_stream, size_t cap, void* d_ws, size_t ws_bytes, size_t* out_bytes,
                          hc_header* hdr_out, void* stream);
HC_API int hc_compress_codes_nd(const int32_t* d_q, int dtype, int ndim, const int64_t* dims, const int32_t* block,
                                double eps, double eb, int eb_mode, void* d_stream, size_t cap, void* d_ws,
                                size_t ws_bytes, size_t* out_bytes, hc_header* hdr_out, void* stream);

/* Copy the 256-byte header of a device-resident stream to the host and
 * validate it (magic, version, shape, section offsets, total size against
 * `bytes`).  SYNC. */
HC_API int hc_read_header(const void* d_stream, size_t bytes, hc_header* hdr_out, void* stream);
/* The same checks on a stream held in HOST memory (a file read back, a
 * buffer received from another process): h_stream holds `bytes` bytes of the
 * stream, at least its 256-byte header.  No device access; the stream is the
 * persistent form of the compressed field (Section III-A: c = C(d, eps)),
 * so saving it is writing its total_bytes and loading it is this check
 * followed by a copy to the device.  Errors as hc_read_header. */
HC_API int hc_read_header_host(const void* h_stream, size_t bytes, hc_header* hdr_out);

/* ---------------------------------------------------------- decompression */
/* D_i ... D_1 (Algorithm 2): decode the whole stream to stage `kind`:
 *   HC_STAGE_M -> int32 heads[nb] (HC_PRED_MEAN / MEAN_ND: the block or box
 *   means, boxes in grid order; the global predictors have no stage 1:
 *   HC_ERR_UNSUPPORTED); MEAN_ND stages 2-4 are in field order;
 *   HC_STAGE_P -> int32[N] (HC_PRED_DELTA: head in each block's first slot,
 *   so q is the in-block prefix sum; HC_PRED_MEAN: p = q - M_b; the global
 *   predictors: their residuals); HC_STAGE_Q -> int32[N] (global
 *   predictors: prefix sums of D_p along every prediction axis); HC_STAGE_F
 *   -> out_dtype HC_F32 ((float)q * (float)(2 eps)) or HC_F64 ((double)q *
 *   2 eps).
 * d_out holds hc_stage_bytes(hdr, kind) bytes (8 per element for F64).
 * ws_bytes >= hc_workspace_bytes_for(hdr).
 * ASYNC; corruption is reported in the workspace status word. */
HC_API int hc_decompress_to_stage(const hc_header* hdr, const void* d_stream, int kind, void* d_out, int out_dtype,
                           void* d_ws, size_t ws_bytes, void* stream);

/* Status word a kernel left in a workspace (HC_OK when clean); resets it.  SYNC. */
HC_API int hc_workspace_status(void* d_ws, void* stream);

/* ------------------------------------------------------------- operations */
/* Statistics (Section V-A).  `in`: the stream (fused) at a level, or a
 * materialized M, P, Q or F array.  eps and dims must match the stream header
 * for the fused form.  d_out: one hc_scalar in device memory.  hc_op_mean
 * fills mean (and s1); hc_op_variance and hc_op_std fill every field.
 *   level Q: exact s1 = sum q, s2 = sum q^2, Eq. var_q.
 *   level P, HC_PRED_DELTA: the mean from the block-weighted sum
 *     sum_i (S_b - i + 1) p_i (no prefix sum); the variance through the eta
 *     accumulator (exact, as level Q).
 *   level P, HC_PRED_MEAN: the mean from sum p + M_b S_b (exact); the
 *     variance of Section V-A about the integer mean mu~ = round(T / N),
 *     T = sum_b M_b S_b (nearest, ties toward zero):
 *     variance = sum (p + M_b - mu~)^2 / (N - 1) * (2 eps)^2, std its root;
 *     s1 = sum q exact and s2 = sum (q - mu~)^2 exact; exact = 0 because
 *     this variance is the paper's approximation, not Eq. var_q.
 *   level M (HC_PRED_MEAN streams, or an M array with pred = HC_PRED_MEAN,
 *     S and n set): the mean of Eq. mean_m, (T / N) 2 eps, from the block
 *     means alone; s1 = T, exact = 0; mean only (the variance needs the codes).
 *     HC_PRED_DELTA heads support no statistic (HC_ERR_UNSUPPORTED).
 *   MEAN_ND streams: as MEAN with the true box sizes S_b (stage 1: Eq.
 *     mean_m; stage 2: the exact mean and the deviation about mu~; stage 3:
 *     exact), fused with the decode.
 *   Global predictors (stream inputs; ws_bytes >= hc_workspace_bytes_for):
 *     level P mean: sum q = sum_i p_i (L0 - z)(L1 - y)(L2 - x), (z, y, x)
 *     the position of p_i in the prediction shape L (the field's shape for
 *     LORENZO, (1, 1, N) for GLOBAL_DELTA; Section V-A's HSZp-2d and HSZp
 *     weighted sums), fused with the decode, no prefix sum, exact;
 *     level P variance (Algorithm 4: q rebuilt by prefix sums, s1 and s2
 *     accumulated) and level Q: D_q rebuilt in the workspace, then the
 *     exact stage-3 sums.  Arrays of their D_p are refused (operate on the
 *     stream); levels M are HC_ERR_UNSUPPORTED.
 * ASYNC. */
HC_API int hc_op_mean(const hc_stage* in, double eps, int ndim, const int64_t* dims, hc_scalar* d_out, void* d_ws,
               size_t ws_bytes, void* stream);
HC_API int hc_op_variance(const hc_stage* in, double eps, int ndim, const int64_t* dims, hc_scalar* d_out, void* d_ws,
                   size_t ws_bytes, void* stream);
HC_API int hc_op_std(const hc_stage* in, double eps, int ndim, const int64_t* dims, hc_scalar* d_out, void* d_ws,
              size_t ws_bytes, void* stream);

/* Allocation-free fused variance (the paper has no counterpart: this is an
 * interface for callers, not a method step).  For callers that cannot
 * allocate device memory when they need the statistic -- allocation-free
 * real-time loops, whose latency budget leaves no room for an allocator call,
 * and plugins handed only a stream and pointers by a host application that
 * owns all device memory and gives out no allocator -- it computes what
 * hc_op_variance computes for a compressed-stream input (level P or Q), but
 * takes no workspace: its scratch is a static device array inside libhc.so of
 * 64 KiB + 256 bytes (one ticket counter and 2048 per-CTA partial sums), held
 * by every GPU that loads the library until the process exits.
 *   in: a HC_STAGE_COMPRESSED stage (other kinds: HC_ERR_UNSUPPORTED);
 *   d_out: one hc_scalar in device memory (every field filled, as
 *   hc_op_variance does).  A launch that would need more than 2048 partial
 *   slots is refused with HC_ERR_NOMEM.
 * It calls no allocating routine.  The first call on each device looks up the
 * device address of the static array (with that device current); make that
 * first call before any stream capture.  Every call clears the ticket it needs
 * and reuses the same array, so calls whose kernels overlap on the GPU (for
 * example on two concurrent streams) race and must not be issued.  ASYNC. */
HC_API int hc_op_variance_noalloc(const hc_stage* in, double eps, int ndim, const int64_t* dims, hc_scalar* d_out,
                                  void* stream);

/* Numerical differentiation (Section V-B, "Operation with D_q").  Inputs: the
 * stream (fused, level Q), or a materialized Q or F array.  A stage-P input
 * returns HC_ERR_UNSUPPORTED: a 1-D block partition does not keep the
 * multidimensional layout (Section V-B) -- except for HC_PRED_LORENZO
 * (HSZp-nd) streams at level P: the derivative along axis a is the box sum of
 * D_p over the other axes at slices a = i and i + 1 (Eq. derivative_Dp and
 * the sum form above it), the Laplacian the sum over axes of differences of
 * such box sums (Eq. laplacian_Dp), computed from D_p by prefix sums over
 * the other axes only, never forming D_q; the gradient magnitude is not
 * offered there (HC_ERR_UNSUPPORTED) -- and for HC_PRED_MEAN_ND (HSZx-nd)
 * streams at level P: Section V-B's HSZx-2d formulas on every axis, the
 * differences of D_p plus the box means' difference where a neighbour lies
 * in another box (derivative, gradient magnitude and Laplacian; D_p in field
 * order is formed in the workspace, D_q never).  Global-predictor streams at level Q
 * rebuild D_q in the workspace and take the stage-3 operation on it
 * (ws_bytes >= hc_workspace_bytes_for).  `axis` is a user axis in
 * [0, ndim), 0 the slowest.  d_out: N elements of out_dtype:
 *   HC_F32 / HC_F64  the scaled value (eps * D, eps * |grad|, 2 eps * L),
 *   HC_I64           the exact integer numerator (D or L; integer inputs).
 * Interior derivative D = q[i+1] - q[i-1]; at a domain edge D = 2 (q[1] -
 * q[0]) (one-sided); an axis of length 1 gives 0.  The Laplacian replicates
 * edge values.  ASYNC. */
HC_API int hc_op_derivative(const hc_stage* in, double eps, int ndim, const int64_t* dims, int axis, void* d_out,
                     int out_dtype, void* d_ws, size_t ws_bytes, void* stream);
HC_API int hc_op_gradmag(const hc_stage* in, double eps, int ndim, const int64_t* dims, void* d_out, int out_dtype,
                  void* d_ws, size_t ws_bytes, void* stream);
HC_API int hc_op_laplacian(const hc_stage* in, double eps, int ndim, const int64_t* dims, void* d_out, int out_dtype,
                    void* d_ws, size_t ws_bytes, void* stream);

/* Divergence and curl of a vector field (Section V-C, "Multivariate
 * Derivation"), stage Q, fused: one compressed stream per component, all of
 * the same shape and block size, each read straight from its stream.
 *   hc_op_divergence: ncomp == ndim components; component c is
 *     differentiated along user axis c; value = (sum_c D_c) eps.
 *   hc_op_curl: a 2-D field (u, v), ncomp == 2; with i the first and j the
 *     second index, value = (D_u along j - D_v along i) eps.
 * D is the derivative numerator of hc_op_derivative (one-sided and doubled at
 * an edge).  Components quantized with different eps are scaled one by one,
 * sum_c eps_c D_c in double (the paper assumes one eps); an HC_I64 output
 * (the exact integer numerator) needs one eps for all components.
 *   comps: ncomp HC_STAGE_COMPRESSED stages, all at level HC_STAGE_Q (or all
 *   at HC_STAGE_P for HSZp-nd / HSZx-nd components, see below).
 *   d_out: N outputs of out_dtype (HC_F32, HC_F64 or HC_I64), 16-byte aligned.
 * Rows longer than about a million codes are HC_ERR_UNSUPPORTED.  ASYNC. */
/* Components of other predictors, of different block sizes, or at level P
 * (HSZp-nd and HSZx-nd: Section V-C's stage-2 divergence and curl, each
 * component's derivative taken by its stage-2 path -- Eq. derivative_Dp for
 * HSZp-nd, the box-border form for HSZx-nd -- then added): each component's
 * integer derivative numerators are formed in turn in the workspace, summed
 * exactly, and scaled as above (the same values as the fused kernel).  Then
 * ws_bytes >= hc_vector_workspace_bytes(comps, ncomp) (the largest
 * component workspace + 16 bytes per element); otherwise hc_workspace_bytes()
 * suffices. */
HC_API size_t hc_vector_workspace_bytes(const hc_stage* comps, int ncomp);
HC_API int hc_op_divergence(const hc_stage* comps, int ncomp, int ndim, const int64_t* dims, void* d_out,
                            int out_dtype, void* d_ws, size_t ws_bytes, void* stream);
HC_API int hc_op_curl(const hc_stage* comps, int ncomp, int ndim, const int64_t* dims, void* d_out, int out_dtype,
                      void* d_ws, size_t ws_bytes, void* stream);

/* All operations of one field in one pass ("decompress once, many ops",
 * Section VI's remark that a decompressed representation serves several
 * analyses).  Fused on a stream input (level Q): the codes are decoded once
 * and every wanted output is written from the same neighbourhood -- the
 * derivative along each user axis, the gradient magnitude, the Laplacian
 * (values exactly as hc_op_derivative / hc_op_gradmag / hc_op_laplacian
 * produce them) and the stage-Q statistics (as hc_op_variance at level Q:
 * exact s1, s2, mean, variance, std).  Where the one-pass kernel does not
 * apply (block size other than 32, |q| >= 2^15, rows not a multiple of 4
 * codes, unaligned outputs) and for array inputs, the same results come from
 * the one-operation entry points in turn.  ASYNC. */
typedef struct hc_multi_out {
  void* d_derivative[3];  /* per user axis (the first ndim used): N outputs, or NULL */
  void* d_gradmag;        /* N outputs, or NULL */
  void* d_laplacian;      /* N outputs, or NULL */
  hc_scalar* d_stats;     /* or NULL */
  int32_t out_dtype;      /* HC_F32 or HC_F64 for every field output */
  int32_t reserved;
} hc_multi_out;
HC_API int hc_op_multi(const hc_stage* in, double eps, int ndim, const int64_t* dims, const hc_multi_out* out,
                       void* d_ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------- batched fused launch */
/* Many compressed fields, each with its own operations, decoded and operated
 * on by ONE persistent kernel: decoding and operation fused, no stage
 * materialized (Section V's homomorphic operations, batched; the batching
 * itself has no counterpart in the paper).  Statistics are taken at stage Q
 * ("Operation with D_q", Section V-A: exact s1 = sum q, s2 = sum q^2 and the
 * final scaling of Eq. var_q); stencils follow Section V-B exactly as
 * hc_op_derivative / hc_op_gradmag / hc_op_laplacian do on a stream.  A field
 * with both a stencil and statistics is read once: the stencil pass also
 * accumulates the sums.
 *
 * Use: hc_batch_plan (host only) writes a plan into caller host memory; the
 * caller copies those plan bytes unchanged into a 16-byte aligned device
 * buffer; hc_batch_run launches the kernel (ASYNC, capturable in a CUDA
 * graph), or hc_batch_graph_create captures it once and hc_batch_graph_launch
 * replays it.  The device plan, the streams and the outputs must stay valid
 * while launches that use them run.
 *
 * Workspace (hc_batch_workspace_bytes(n), 16-byte aligned, device): must be
 * zero-filled before its first use; every launch leaves it zeroed again
 * except the status word.  One workspace serves one launch at a time:
 * concurrent launches need separate workspaces.  Errors found by the kernel
 * (a corrupt stream) go to the field's hc_scalar.status and to the status
 * word read by hc_batch_status. */
typedef enum {
  HC_BATCH_MEAN = 1,        /* d_scalar: mean; exact s1 */
  HC_BATCH_VARIANCE = 2,    /* d_scalar: mean, variance, std; exact s1, s2 */
  HC_BATCH_DERIVATIVE = 4,  /* d_field: derivative along `axis` */
  HC_BATCH_GRADMAG = 8,     /* d_field: gradient magnitude */
  HC_BATCH_LAPLACIAN = 16,  /* d_field: Laplacian */
  HC_BATCH_DIVERGENCE = 32, /* d_field: divergence of the item's components (Section V-C) */
  HC_BATCH_CURL = 64        /* d_field: 2-D curl of the item's two components (Section V-C) */
} hc_batch_op;

/* A batch item is one field, or (DIVERGENCE / CURL) one vector field given
 * by its component streams: the values are exactly those of hc_op_divergence
 * / hc_op_curl on the same components at stage Q (one fused tile reads every
 * component's stream).  A vector item has that one operation and no other;
 * its components are block-head or block-mean streams (HC_PRED_DELTA or
 * HC_PRED_MEAN) of one shape and block size (other predictors:
 * HC_ERR_UNSUPPORTED, use hc_op_divergence / hc_op_curl); DIVERGENCE takes
 * ndim components, CURL a 2-D field's two. */
typedef struct hc_batch_item {
  const void* d_stream;  /* device: the compressed stream, 16-byte aligned (unused by vector items) */
  hc_header hdr;         /* host copy of its header (hc_read_header / hc_compress; unused by vector items) */
  uint32_t ops;          /* OR of hc_batch_op, with at most one field operation */
  int32_t axis;          /* HC_BATCH_DERIVATIVE: user axis in [0, ndim) */
  hc_scalar* d_scalar;   /* device: statistics result, or NULL without MEAN / VARIANCE */
  void* d_field;         /* device: N outputs of field_dtype, or NULL without a field op */
  int32_t field_dtype;   /* HC_F32, HC_F64, or HC_I64 (exact numerators; not GRADMAG; one eps for
                            every component of a vector item) */
  int32_t ncomp;         /* DIVERGENCE / CURL: components in comps; 0 otherwise */
  const hc_stage* comps; /* DIVERGENCE / CURL: HOST array of ncomp HC_STAGE_COMPRESSED stages at level
                            HC_STAGE_Q (streams 16-byte aligned, headers as for d_stream / hdr), read
                            by hc_batch_plan only; NULL otherwise */
} hc_batch_item;

/* Launch shape of the batch kernel (GPU tiling choices, no counterpart in
 * the paper).  Zero fields take the defaults. */
typedef struct hc_batch_tune {
  int32_t threads;      /* threads per CTA: 128, 256 (default) or 512 */
  int32_t ty;           /* largest stencil tile height in rows; 0: no limit.  Each field takes the largest
                           height up to it (the whole plane when it has at most 128 rows, else 128, 64, 32,
                           16, 8, 4, 2 or 1) whose tile fits three CTAs per SM */
  int64_t unit_elems;   /* output points per stencil work unit; 0: about six units per CTA */
  int32_t ctas_per_sm;  /* upper limit on resident CTAs per SM; 0: occupancy limit */
  int32_t reserved;
} hc_batch_tune;

/* Bytes of a plan / of the workspace for n items (0 for n < 1). */
HC_API size_t hc_batch_plan_bytes(int n_items);
HC_API size_t hc_batch_workspace_bytes(int n_items);
/* Validate the items and build the plan in h_plan (host memory, cap bytes);
 * *used receives its size.  Host only, but it queries the current device's
 * occupancy and sets the kernel's shared-memory limit.  Errors:
 * HC_ERR_INVALID_ARG (bad item or tune), HC_ERR_CORRUPT (inconsistent
 * header), HC_ERR_NOMEM (cap too small), HC_ERR_UNSUPPORTED (a tile does not
 * fit in shared memory, or GRADMAG with HC_I64). */
HC_API int hc_batch_plan(const hc_batch_item* items, int n_items, const hc_batch_tune* tune, void* h_plan,
                         size_t cap, size_t* used);
/* Launch the batch on `stream`.  h_plan: the host plan; d_plan: its device
 * copy.  ASYNC. */
HC_API int hc_batch_run(const void* h_plan, const void* d_plan, void* d_ws, size_t ws_bytes, void* stream);
/* Capture one hc_batch_run into an instantiated CUDA graph (*graph_exec,
 * owned by the caller: hc_batch_graph_destroy), replayed by
 * hc_batch_graph_launch on any stream.  SYNC for the capture itself. */
HC_API int hc_batch_graph_create(const void* h_plan, const void* d_plan, void* d_ws, size_t ws_bytes,
                                 void** graph_exec);
HC_API int hc_batch_graph_launch(void* graph_exec, void* stream);
HC_API int hc_batch_graph_destroy(void* graph_exec);
/* Read and clear the batch workspace's status word (first error of any
 * launch since the last call).  SYNC on `stream`. */
HC_API int hc_batch_status(void* d_ws, void* stream);

/* ---------------------------------------------------------------- shards */
/* A contiguous range of whole chunks of a stream as a stream of its own, so
 * that ranks can each reduce a part of one field (no counterpart in the
 * paper: with block heads (HC_PRED_DELTA) or block means (HC_PRED_MEAN) every
 * block decodes alone, so the exact sums of Section V-A add over any
 * partition of the blocks).  The shard of chunks [c0, c1) is a 1-D field of
 * the elements those blocks hold, in row-major order from element `first`;
 * every statistic of hc_op_mean / hc_op_variance runs on it unchanged, and
 * the ranks' exact s1 and s2 add up to the whole field's.  Stencils need
 * neighbours across the range and are not offered on shards.
 *
 * hc_shard_plan (host only, no device access) takes the full stream's
 * header and a host copy of its chunk index (nchunks + 1 uint64 words, from
 * byte hdr->off_chunks of the stream) and fills `out`: the shard's header,
 * its 256-byte image, the three byte ranges to copy from the full stream
 * (widths, heads, payload) and where they go, and in chunks_out (c1 - c0 + 1
 * uint64) the shard's chunk index, rebased to its first payload word.  The
 * caller builds the shard in a zeroed device buffer of hdr.total_bytes:
 * header_bytes at 0, the three copies, chunks_out at chunks_off.
 * The shard keeps the full stream's max width and max |q| as upper bounds.
 * Errors: HC_ERR_INVALID_ARG (null pointer, c0 < 0, c1 <= c0 or c1 >
 * nchunks), HC_ERR_CORRUPT (an inconsistent header, or a chunk index that
 * is not ascending or does not end at the payload size), HC_ERR_UNSUPPORTED
 * (a global-predictor or HSZx-nd stream: their blocks do not decode
 * alone). */
typedef struct hc_shard {
  hc_header hdr;            /* the shard's header (ndim 1, N = its elements) */
  uint8_t header_bytes[256];/* its image: the first 256 bytes of the shard */
  int64_t src_off[3];       /* byte offsets in the full stream of the widths, heads and payload copied */
  int64_t dst_off[3];       /* their byte offsets in the shard */
  int64_t nbytes[3];        /* their sizes in bytes */
  int64_t chunks_off;       /* byte offset of the shard's chunk index */
  int64_t first;            /* the shard's first element in the full field (row-major) */
} hc_shard;
HC_API int hc_shard_plan(const hc_header* full, const uint64_t* h_chunks, int64_t c0, int64_t c1, hc_shard* out,
                         uint64_t* chunks_out);

/* The final scaling of Eq. var_q (Section V-A) on the host, from exact sums:
 * s1 = sum q (int64) and s2 = sum q^2 (128 bits: s2_hi * 2^64 + s2_lo) over
 * n codes quantized with bound eps -- for example the totals of several
 * shards' hc_scalar results, added exactly.  Fills *out (HOST memory) as a
 * fused statistic's device finish does, with the same integer arithmetic and
 * the same roundings, so the values are bit-equal to a one-launch result:
 *   mean = ((double)s1 / N) * 2 eps,
 *   variance = ((double)(N s2 - s1^2) / (N (N - 1))) * (2 eps)^2, the
 *     128-bit numerator converted once (round to nearest even),
 *   std = sqrt(variance); variance and std are NaN for N = 1;
 *   n, s1, s2_lo, s2_hi copied; status = HC_OK; exact = 1.
 * No device access.  Errors: HC_ERR_INVALID_ARG for out == NULL, n < 1, or
 * eps not positive and finite (nothing written then). */
HC_API int hc_finalize(int64_t n, int64_t s1, uint64_t s2_lo, uint64_t s2_hi, double eps, hc_scalar* out);

/* ---------------------------------------------------------------- tuning */
/* Autotuner of the fused stencil kernel (no counterpart in the paper: a GPU
 * tiling choice).  For a compressed-stream input and op (HC_OP_DERIVATIVE,
 * HC_OP_GRADMAG or HC_OP_LAPLACIAN) and output type, times every tile height
 * the kernel can use on this field, each with the grid sized for one and for
 * two waves of resident CTAs (each 1 warm-up + 3 runs, writing d_out, which
 * must hold the op's output) and keeps the fastest pair for all later calls
 * on fields of the same shape, max width, op and output type in this
 * process.  *chosen receives the tile height (0: the general kernel applies
 * and nothing was tuned; statistics ops have nothing to tune).  HC_OP_MULTI
 * tunes hc_op_multi's one-pass kernel: d_out must then hold (ndim + 2) * N
 * outputs (the derivative along each axis, the gradient magnitude and the
 * Laplacian, one after the other).  SYNC: call it before capturing work in a
 * CUDA graph. */
HC_API int hc_autotune(const hc_stage* in, int op, int out_dtype, void* d_out, void* d_ws, size_t ws_bytes,
                       void* stream, int* chosen);

/* The autotuner's choices as text, so that a later process (a server that
 * restarts, a job on another GPU of the same kind) can reuse them instead of
 * timing every tile again (no counterpart in the paper: a GPU tiling choice).
 * The text is JSON:
 *   {"format": "hc-autotune", "version": 1, "entries": [
 *     {"n0": 512, "n1": 512, "n2": 512, "wmax": 9, "op": "multi", "out": "float32",
 *      "tile_rows": 8, "waves": 1}, ...]}
 * one entry per choice hc_autotune kept in this process: (n0, n1, n2) the shape
 * the fused stencils walk (a 2-D field (n1, n2) is walked as (n1, 1, n2)), wmax
 * the stream's largest block width, op one of "derivative", "gradmag",
 * "laplacian", "multi", out one of "float32", "float64", "int64", tile_rows
 * the tile height and waves the plane ranges (1 or 2 waves of resident CTAs).
 * A choice is a launch shape only: every choice gives the same results, and a
 * tile that does not fit a later field of the same key falls back to another
 * kernel of the same results.
 *
 * hc_autotune_export: writes the text, NUL-terminated, into buf (cap bytes)
 * and its length without the NUL into *len.  buf == NULL: only *len is set
 * (a size query).  Errors: HC_ERR_INVALID_ARG for len == NULL; HC_ERR_NOMEM
 * when cap <= *len (nothing written to buf).  Host only, no device access. */
HC_API int hc_autotune_export(char* buf, size_t cap, size_t* len);

/* hc_autotune_import: reads text in the export format (NUL-terminated; keys in
 * any order, whitespace anywhere between tokens) and keeps its choices for the
 * later calls of this process, replacing a kept choice of the same key;
 * *count receives the number of entries read.  Errors (nothing kept then,
 * *count = 0): HC_ERR_INVALID_ARG for a NULL argument, text that is not in the
 * format (an unknown, missing or repeated key, another format name or
 * version, trailing characters, string escapes, negative or over-long
 * numbers), or an entry out of range (a dimension outside 1..2^40, wmax
 * above 32, tile_rows outside 1..255, waves outside 1..2, an int64 gradient
 * magnitude or one-pass entry).  Host only, no device access. */
HC_API int hc_autotune_import(const char* text, int* count);

#ifdef __cplusplus
}
#endif
#endif /* HC_H */
