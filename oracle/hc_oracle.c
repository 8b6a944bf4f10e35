/*
 * hc_oracle.c -- TEST INFRASTRUCTURE, NOT PRODUCT CODE.
 *
 * A plain, serial, deliberately slow CPU reference ("oracle") for the
 * HSZp-style multi-stage decompression framework and its homomorphic
 * analytical operations (paper: "HSZ", Sections III-V).  Only the test suite,
 * __graft_entry__.smoke() and bench.py's CPU-baseline / reference arm may load
 * it.  It shares no code, header, table or constant with the CUDA library in
 * paper_2603_25206_gb300/csrc; both sides implement the stream layout below
 * independently.
 *
 * Every function names the passage of the paper it follows.  Where the paper
 * is silent, the reading that is applied is stated in the comment.
 *
 * Stream layout (all little-endian):
 *   header, 256 bytes:
 *     0 u32 magic 'HCZ1'   4 u16 version 1   6 u8 dtype (0 f32, 1 f64)
 *     7 u8 ndim            8 i64[3] shape (n0, n1, n2), leading ones
 *    32 u32 S (block size) 36 u32 G = max(1, 4096 / S) blocks per chunk
 *    40 f64 eps (absolute bound used)  48 f64 eb (as given)
 *    56 u32 eb mode (0 abs, 1 rel)     60 u32 max |q|
 *    64 i64 N  72 i64 nb  80 i64 nchunks  88 i64 payload words
 *    96 i64 off widths  104 i64 off heads  112 i64 off chunks
 *   120 i64 off payload 128 i64 total bytes  136 u32 max width
 *   140 u32 predictor: 0 = delta inside the block (HSZp with SZp-style block
 *       heads), 1 = block mean (HSZx), 2 = Lorenzo over the field's axes
 *       (HSZp-nd), 3 = delta across blocks over the flattened field (HSZp),
 *       4 = block mean over multidimensional blocks (HSZx-nd)
 *   144 u32[3] block extents (b0, b1, b2) along (n0, n1, n2) for predictor 4,
 *       S = b0 b1 b2 (zero for the other predictors); rest zero
 *   widths u8[nb] at 256; heads i32[nb], chunk index u64[nchunks + 1] and
 *   payload u32 words each start on the next 16-byte boundary; the stream
 *   ends 16..31 zero bytes after the payload (total rounded to 16).
 *   chunk[c] = payload word of the first block of chunk c, chunk[nchunks] =
 *   payload words.  A block of width w > 0 holds ceil(S/32) sign words (bit
 *   k%32 of word k/32 set iff p_k < 0) followed by ceil(S*w/32) magnitude
 *   words in which |p_k| occupies bits [k*w, (k+1)*w) of the word sequence
 *   read least-significant bit first.  Predictor 0: heads[b] is the block's
 *   first code, p_k = q_k - q_{k-1} and p_0 = 0.  Predictor 1: heads[b] is
 *   the block mean M_b (the integer nearest to the block's code sum over its
 *   true size, ties toward zero) and p_k = q_k - M_b for every k.
 *   Predictors 2 and 3: heads[b] = 0 and every slot holds the residual of a
 *   prediction that runs over the whole field (below, "global predictors").
 *   The padding
 *   slots of a short last block are 0.  A block of width 0 has no payload
 *   words.
 *
 * Integers: codes q are int32 with |q| < 2^30; sums of q are int64; sums of
 * q^2 and the variance numerator are 128-bit (__int128).  Floating point is
 * IEEE double unless the stored field type is float.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared (no -march flags:
 * the same source must give the same bytes on x86-64 and aarch64).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* status values (same meaning as the library's public enum) */
#define ORC_OK 0
#define ORC_ERR_INVALID_ARG 1
#define ORC_ERR_RANGE 2
#define ORC_ERR_CORRUPT 3
#define ORC_ERR_UNSUPPORTED 4

/* stream layout constants (layout in the file header) */
#define ORC_MAGIC 0x315A4348u /* bytes 'H' 'C' 'Z' '1' */
#define ORC_VERSION 1u
#define ORC_HEADER_BYTES 256
#define ORC_CHUNK_ELEMS 4096 /* G = max(1, 4096 / S) blocks per chunk */
#define ORC_QLIMIT (1 << 30) /* |q| must be < 2^30 */
#define ORC_MAX_S 4096

typedef __int128 i128;
typedef unsigned __int128 u128;

/* ------------------------------------------------------------------ */
/* little-endian byte access (explicit, independent of host order)     */
/* ------------------------------------------------------------------ */
static void put_u8(uint8_t *b, int64_t off, uint32_t v) { b[off] = (uint8_t)v; }
static void put_u16(uint8_t *b, int64_t off, uint32_t v) {
  b[off] = (uint8_t)(v & 0xff);
  b[off + 1] = (uint8_t)((v >> 8) & 0xff);
}
static void put_u32(uint8_t *b, int64_t off, uint32_t v) {
  for (int i = 0; i < 4; i++) b[off + i] = (uint8_t)((v >> (8 * i)) & 0xff);
}
static void put_u64(uint8_t *b, int64_t off, uint64_t v) {
  for (int i = 0; i < 8; i++) b[off + i] = (uint8_t)((v >> (8 * i)) & 0xff);
}
static void put_f64(uint8_t *b, int64_t off, double v) {
  uint64_t u;
  memcpy(&u, &v, 8);
  put_u64(b, off, u);
}
static uint32_t get_u8(const uint8_t *b, int64_t off) { return b[off]; }
static uint32_t get_u16(const uint8_t *b, int64_t off) {
  return (uint32_t)b[off] | ((uint32_t)b[off + 1] << 8);
}
static uint32_t get_u32(const uint8_t *b, int64_t off) {
  uint32_t v = 0;
  for (int i = 0; i < 4; i++) v |= (uint32_t)b[off + i] << (8 * i);
  return v;
}
static uint64_t get_u64(const uint8_t *b, int64_t off) {
  uint64_t v = 0;
  for (int i = 0; i < 8; i++) v |= (uint64_t)b[off + i] << (8 * i);
  return v;
}
static double get_f64(const uint8_t *b, int64_t off) {
  uint64_t u = get_u64(b, off);
  double v;
  memcpy(&v, &u, 8);
  return v;
}

static int64_t align16(int64_t x) { return (x + 15) & ~(int64_t)15; }

/* ------------------------------------------------------------------ */
/* Parsed header                                                       */
/* ------------------------------------------------------------------ */
typedef struct {
  int dtype; /* 0 = float32, 1 = float64 */
  int ndim;
  int64_t dims[3]; /* (n0, n1, n2), leading ones for ndim < 3 */
  int S;           /* block size */
  int G;           /* blocks per chunk */
  double eps;      /* absolute error bound actually used */
  double eb;       /* error bound as given */
  int eb_mode;     /* 0 absolute, 1 value-range relative */
  int64_t qmax;    /* max |q| */
  int64_t N, nb, nchunks, payload_words;
  int64_t off_widths, off_heads, off_chunks, off_payload, total_bytes;
  int wmax;
  int pred;      /* the predictor (header byte 140) */
  int64_t bd[3]; /* predictor 4: block extents (b0, b1, b2); zero otherwise */
} orc_header;

static int64_t chunk_blocks(int S) {
  int64_t g = ORC_CHUNK_ELEMS / S;
  return g < 1 ? 1 : g;
}

/* blocks of a multidimensional partition: the grid ceil(n_a / b_a) */
static int64_t grid_blocks(const int64_t *dims, const int64_t *bd) {
  int64_t nb = 1;
  for (int a = 0; a < 3; a++) nb *= (dims[a] + bd[a] - 1) / bd[a];
  return nb;
}

/* Section offsets follow from (N, S) alone, or from the block grid for
 * predictor 4. */
static void layout(orc_header *h) {
  h->nb = h->bd[0] > 0 ? grid_blocks(h->dims, h->bd) : (h->N + h->S - 1) / h->S;
  h->G = (int)chunk_blocks(h->S);
  h->nchunks = (h->nb + h->G - 1) / h->G;
  h->off_widths = ORC_HEADER_BYTES;
  h->off_heads = align16(h->off_widths + h->nb);
  h->off_chunks = align16(h->off_heads + 4 * h->nb);
  h->off_payload = align16(h->off_chunks + 8 * (h->nchunks + 1));
}

/* ------------------------------------------------------------------ */
/* Error bound (Section VI-B: value-range-relative bounds)              */
/* ------------------------------------------------------------------ */
static double load_x(const void *x, int dtype, int64_t i) {
  if (dtype == 0) return (double)((const float *)x)[i];
  return ((const double *)x)[i];
}

/* epsilon = eb (absolute) or eb * (max - min) (value-range relative).
 * Reading: a constant field (max == min) falls back to epsilon = eb. */
int orc_eps(const void *x, int dtype, int64_t n, double eb, int eb_mode, double *eps_out) {
  if (!(eb > 0.0) || !isfinite(eb) || n < 1) return ORC_ERR_INVALID_ARG;
  double eps = eb;
  if (eb_mode == 1) {
    double mn = load_x(x, dtype, 0), mx = mn;
    for (int64_t i = 1; i < n; i++) {
      double v = load_x(x, dtype, i);
      if (v < mn) mn = v;
      if (v > mx) mx = v;
    }
    if (!isfinite(mn) || !isfinite(mx)) return ORC_ERR_RANGE;
    if (mx > mn) eps = eb * (mx - mn);
  } else if (eb_mode != 0) {
    return ORC_ERR_INVALID_ARG;
  }
  if (!(eps > 0.0) || !isfinite(eps)) return ORC_ERR_INVALID_ARG;
  *eps_out = eps;
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Quantization (Section IV "Quantization"; Algorithm 1, quantize step) */
/* q = round(d / (2 eps)).  Reading: round(t) = floor(t + 0.5) in IEEE  */
/* double with a true division, the only rule that reproduces the       */
/* worked example of Section IV (HSZx-nd, 2x4 array Y, eps = 0.1).      */
/* ------------------------------------------------------------------ */
int orc_quantize(const void *x, int dtype, int64_t n, double eps, int32_t *q) {
  double two_eps = 2.0 * eps;
  for (int64_t i = 0; i < n; i++) {
    double t = load_x(x, dtype, i) / two_eps;
    double r = floor(t + 0.5);
    if (!(fabs(r) < (double)ORC_QLIMIT)) return ORC_ERR_RANGE; /* also NaN */
    q[i] = (int32_t)r;
  }
  return ORC_OK;
}

/* bit length of a non-negative value: smallest w with v < 2^w */
static int bit_length(uint32_t v) {
  int w = 0;
  while (v != 0) {
    w++;
    v >>= 1;
  }
  return w;
}

static int64_t block_words(int S, int w) {
  if (w == 0) return 0;
  return (int64_t)(S + 31) / 32 + ((int64_t)S * w + 31) / 32;
}

int64_t orc_compress_bound(int64_t n, int S) {
  if (n < 1 || S < 1 || S > ORC_MAX_S) return -1;
  orc_header h;
  memset(&h, 0, sizeof h);
  h.N = n;
  h.S = S;
  layout(&h);
  return align16(h.off_payload + 4 * h.nb * block_words(S, 31) + 16);
}

/* ------------------------------------------------------------------ */
/* Compression: Algorithm 1 (quantize -> partition -> metadata ->       */
/* decorrelate -> encode), SZp variant with the first code of each     */
/* block kept as metadata (Section IV "Metadata Collection",            */
/* "Decorrelation") and the block-wise fixed-rate encoder of Section IV */
/* "Encoding": per block the signs are gathered first, then the         */
/* magnitudes in order at the width set by the largest magnitude.       */
/* ------------------------------------------------------------------ */
/* Integer mean of HSZx: the integer nearest to a / d (d > 0), ties toward
 * zero.  Reading: Section V-D bounds the rounding error of the block means by
 * 1/2 (so: nearest), and the worked example of Section IV rounds 22/4 = 5.5
 * to 5 (so: the tie goes toward zero). */
static int64_t nearest_ratio(int64_t a, int64_t d) {
  i128 m = a < 0 ? -(i128)a : (i128)a;
  i128 r = (2 * m + d - 1) / (2 * (i128)d);
  return (int64_t)(a < 0 ? -r : r);
}

/* ------------------------------------------------------------------ */
/* Global predictors (Section IV, "HSZp" and "HSZp-nd").                */
/* The prediction runs over the whole field, across block boundaries;  */
/* blocks only group residuals for the fixed-length encoder.  Codes     */
/* outside the field count as 0, so the first residual is the code.     */
/*   predictor 2 (HSZp-nd): the multidimensional Lorenzo residual over   */
/*     the field's axes: 1-D p_i = q_i - q_{i-1}; 2-D p_{i,j} = q_{i,j} - */
/*     q_{i,j-1} - q_{i-1,j} + q_{i-1,j-1}; 3-D the eight-term form.     */
/*   predictor 3 (HSZp): p_i = q_i - q_{i-1} over the row-major          */
/*     flattened field, whatever its ndim.                               */
/* Both are the Lorenzo residual over "prediction dimensions" L: the    */
/* field's (n0, n1, n2) for predictor 2, (1, 1, N) for predictor 3.      */
/* Reading: the paper's HSZp-nd also partitions the field into          */
/* multidimensional blocks for encoding; here the residuals are grouped */
/* into 1-D blocks of S in row-major order like every other predictor   */
/* (the grouping changes the widths, not any value of D_p or D_q).      */
/* ------------------------------------------------------------------ */
static void global_dims(const int64_t *dims3, int64_t n, int pred, int64_t *L) {
  if (pred == 3) {
    L[0] = 1;
    L[1] = 1;
    L[2] = n;
  } else {
    L[0] = dims3[0];
    L[1] = dims3[1];
    L[2] = dims3[2];
  }
}

static int64_t code_at(const int32_t *q, const int64_t *L, int64_t z, int64_t y, int64_t x) {
  if (z < 0 || y < 0 || x < 0) return 0;
  return q[(z * L[1] + y) * L[2] + x];
}

/* Lorenzo residual at flat index i, written term by term as in Section IV
 * (the 3-D form; with leading axes of length 1 the terms that reach before
 * the field vanish and the 2-D and 1-D forms remain). */
static int64_t lorenzo_residual(const int32_t *q, const int64_t *L, int64_t i) {
  int64_t x = i % L[2], y = (i / L[2]) % L[1], z = i / (L[2] * L[1]);
  int64_t v = code_at(q, L, z, y, x) - code_at(q, L, z, y, x - 1) - code_at(q, L, z, y - 1, x) -
              code_at(q, L, z - 1, y, x) + code_at(q, L, z, y - 1, x - 1) + code_at(q, L, z - 1, y, x - 1) +
              code_at(q, L, z - 1, y - 1, x) - code_at(q, L, z - 1, y - 1, x - 1);
  return v;
}

static void encode_block(uint8_t *out, const orc_header *h, int64_t word, const int32_t *p, int w);
static void finish_stream(uint8_t *out, orc_header *hp, int64_t word);

int orc_compress_codes_pred(const int32_t *q, int dtype, int ndim, const int64_t *dims_in, double eps,
                            double eb, int eb_mode, int S, int pred, uint8_t *out, int64_t cap,
                            int64_t *out_bytes) {
  if (ndim < 1 || ndim > 3 || S < 1 || S > ORC_MAX_S || !(eps > 0.0)) return ORC_ERR_INVALID_ARG;
  if (pred < 0 || pred > 3) return ORC_ERR_INVALID_ARG;
  if (dtype != 0 && dtype != 1) return ORC_ERR_INVALID_ARG;
  orc_header h;
  memset(&h, 0, sizeof h);
  h.dims[0] = h.dims[1] = h.dims[2] = 1;
  int64_t n = 1;
  for (int a = 0; a < ndim; a++) {
    if (dims_in[a] < 1) return ORC_ERR_INVALID_ARG;
    h.dims[3 - ndim + a] = dims_in[a];
    n *= dims_in[a];
  }
  h.N = n;
  h.S = S;
  layout(&h);
  int64_t bound = orc_compress_bound(n, S);
  if (cap < bound) return ORC_ERR_INVALID_ARG;
  memset(out, 0, (size_t)bound);

  for (int64_t i = 0; i < n; i++)
    if (!(q[i] > -ORC_QLIMIT && q[i] < ORC_QLIMIT)) return ORC_ERR_RANGE;

  int32_t *p = (int32_t *)malloc(sizeof(int32_t) * (size_t)S);
  if (!p) return ORC_ERR_INVALID_ARG;
  int64_t L[3];
  global_dims(h.dims, n, pred, L);
  int64_t word = 0; /* running payload word index */
  int64_t qmax = 0;
  int wmax = 0;
  for (int64_t b = 0; b < h.nb; b++) {
    int64_t first = b * S;
    int64_t Sb = (first + S <= n) ? S : n - first; /* true size of the last block */
    if (b % h.G == 0) put_u64(out, h.off_chunks + 8 * (b / h.G), (uint64_t)word);
    int32_t head;
    uint32_t maxmag = 0;
    if (pred == 0) {
      /* metadata: the first code of the block; decorrelation inside the
       * block: p_k = q_k - q_{k-1}, p_0 = 0 */
      head = q[first];
      for (int64_t k = 0; k < S; k++) {
        if (k == 0 || k >= Sb) {
          p[k] = 0;
        } else {
          p[k] = q[first + k] - q[first + k - 1];
          uint32_t m = (uint32_t)(p[k] < 0 ? -(int64_t)p[k] : p[k]);
          if (m > maxmag) maxmag = m;
        }
      }
    } else if (pred >= 2) {
      /* HSZp-nd / HSZp: no block metadata; each slot holds the residual of
       * the prediction over the whole field */
      head = 0;
      for (int64_t k = 0; k < S; k++) {
        if (k >= Sb) {
          p[k] = 0;
        } else {
          /* reading: a residual must fit the 31-bit magnitude of the
           * encoder (|p| < 2^31); a field whose residual does not is
           * rejected like a code out of range */
          int64_t v = lorenzo_residual(q, L, first + k);
          if (v <= -((int64_t)1 << 31) || v >= ((int64_t)1 << 31)) {
            free(p);
            return ORC_ERR_RANGE;
          }
          p[k] = (int32_t)v;
          uint32_t m = (uint32_t)(p[k] < 0 ? -(int64_t)p[k] : p[k]);
          if (m > maxmag) maxmag = m;
        }
      }
    } else {
      /* HSZx (Section IV, "HSZx"): metadata M_b = mean of the block's codes
       * as an integer; decorrelation p_k = q_k - M_b */
      int64_t sum = 0;
      for (int64_t k = 0; k < Sb; k++) sum += q[first + k];
      head = (int32_t)nearest_ratio(sum, Sb);
      for (int64_t k = 0; k < S; k++) {
        if (k >= Sb) {
          p[k] = 0;
        } else {
          p[k] = q[first + k] - head;
          uint32_t m = (uint32_t)(p[k] < 0 ? -(int64_t)p[k] : p[k]);
          if (m > maxmag) maxmag = m;
        }
      }
    }
    put_u32(out, h.off_heads + 4 * b, (uint32_t)head);
    /* the padding slots k >= Sb of a short last block are zero */
    for (int64_t k = 0; k < Sb; k++) {
      int64_t a = q[first + k] < 0 ? -(int64_t)q[first + k] : q[first + k];
      if (a > qmax) qmax = a;
    }
    int w = bit_length(maxmag);
    if (w > wmax) wmax = w;
    put_u8(out, h.off_widths + b, (uint32_t)w);
    if (w == 0) continue;
    encode_block(out, &h, word, p, w);
    word += block_words(S, w);
  }
  free(p);
  h.qmax = qmax;
  h.wmax = wmax;
  h.eps = eps;
  h.eb = eb;
  h.eb_mode = eb_mode;
  h.dtype = dtype;
  h.ndim = ndim;
  h.pred = pred;
  finish_stream(out, &h, word);
  *out_bytes = h.total_bytes;
  return ORC_OK;
}

/* Encoder (Section IV, "Encoding"): sign words, then the magnitudes at w bits
 * each, least-significant bit first, for the S slots p[0..S) of one block
 * whose payload starts at word `word`. */
static void encode_block(uint8_t *out, const orc_header *h, int64_t word, const int32_t *p, int w) {
  int S = h->S;
  int64_t nsw = (S + 31) / 32;
  for (int64_t k = 0; k < S; k++) {
    if (p[k] < 0) {
      int64_t byte = h->off_payload + 4 * (word + k / 32) + (k % 32) / 8;
      out[byte] |= (uint8_t)(1u << (k % 8));
    }
  }
  int64_t mword = word + nsw;
  for (int64_t k = 0; k < S; k++) {
    uint32_t m = (uint32_t)(p[k] < 0 ? -(int64_t)p[k] : p[k]);
    for (int j = 0; j < w; j++) {
      if ((m >> j) & 1u) {
        int64_t bit = k * w + j; /* position in the magnitude bit string */
        int64_t byte = h->off_payload + 4 * (mword + bit / 32) + (bit % 32) / 8;
        out[byte] |= (uint8_t)(1u << (bit % 8));
      }
    }
  }
}

/* The chunk index end, the totals and the 256-byte header of a stream whose
 * payload holds `word` words. */
static void finish_stream(uint8_t *out, orc_header *hp, int64_t word) {
  orc_header h = *hp;
  h.nchunks = (h.nb + h.G - 1) / h.G;
  put_u64(out, h.off_chunks + 8 * h.nchunks, (uint64_t)word);
  h.payload_words = word;
  h.total_bytes = align16(h.off_payload + 4 * word + 16);
  int S = h.S;
  int dtype = h.dtype, ndim = h.ndim, eb_mode = h.eb_mode, pred = h.pred, wmax = h.wmax;
  double eps = h.eps, eb = h.eb;
  int64_t qmax = h.qmax;

  put_u32(out, 0, ORC_MAGIC);
  put_u16(out, 4, ORC_VERSION);
  put_u8(out, 6, (uint32_t)dtype);
  put_u8(out, 7, (uint32_t)ndim);
  put_u64(out, 8, (uint64_t)h.dims[0]);
  put_u64(out, 16, (uint64_t)h.dims[1]);
  put_u64(out, 24, (uint64_t)h.dims[2]);
  put_u32(out, 32, (uint32_t)S);
  put_u32(out, 36, (uint32_t)h.G);
  put_f64(out, 40, eps);
  put_f64(out, 48, eb);
  put_u32(out, 56, (uint32_t)eb_mode);
  put_u32(out, 60, (uint32_t)qmax);
  put_u64(out, 64, (uint64_t)h.N);
  put_u64(out, 72, (uint64_t)h.nb);
  put_u64(out, 80, (uint64_t)h.nchunks);
  put_u64(out, 88, (uint64_t)h.payload_words);
  put_u64(out, 96, (uint64_t)h.off_widths);
  put_u64(out, 104, (uint64_t)h.off_heads);
  put_u64(out, 112, (uint64_t)h.off_chunks);
  put_u64(out, 120, (uint64_t)h.off_payload);
  put_u64(out, 128, (uint64_t)h.total_bytes);
  put_u32(out, 136, (uint32_t)wmax);
  put_u32(out, 140, (uint32_t)pred);
  for (int a = 0; a < 3; a++) put_u32(out, 144 + 4 * a, (uint32_t)h.bd[a]);
  *hp = h;
}

/* ------------------------------------------------------------------ */
/* HSZx-nd (Section IV, "HSZx-nd"): the field is partitioned into boxes  */
/* of b0 x b1 x b2 codes (the multidimensional partition of HSZp-nd), and */
/* each box is decorrelated by its own integer mean, p = q - M_b.        */
/* Readings: boxes are stored in row-major order of the box grid          */
/* ceil(n_a / b_a), the S = b0 b1 b2 slots of a box row-major inside it; */
/* a box cut by the end of the field has its true size S_b (the product   */
/* of its clipped extents) for the mean and zero in the slots outside    */
/* the field; M_b is the nearest integer to the sum over S_b, ties toward */
/* zero, as for HSZx.                                                     */
/* ------------------------------------------------------------------ */
typedef struct {
  int64_t g[3];  /* box grid */
  int64_t k[3];  /* box coordinates of the current box */
} nd_grid;

static void nd_box(const int64_t *dims, const int64_t *bd, int64_t b, nd_grid *G) {
  for (int a = 0; a < 3; a++) G->g[a] = (dims[a] + bd[a] - 1) / bd[a];
  G->k[2] = b % G->g[2];
  G->k[1] = (b / G->g[2]) % G->g[1];
  G->k[0] = b / (G->g[2] * G->g[1]);
}

/* field index of slot s of the box, or -1 for a slot outside the field */
static int64_t nd_slot_index(const int64_t *dims, const int64_t *bd, const nd_grid *G, int64_t s) {
  int64_t c[3];
  c[2] = s % bd[2];
  c[1] = (s / bd[2]) % bd[1];
  c[0] = s / (bd[2] * bd[1]);
  for (int a = 0; a < 3; a++) {
    c[a] += G->k[a] * bd[a];
    if (c[a] >= dims[a]) return -1;
  }
  return (c[0] * dims[1] + c[1]) * dims[2] + c[2];
}

/* true size of box b */
static int64_t nd_box_size(const int64_t *dims, const int64_t *bd, int64_t b) {
  nd_grid G;
  nd_box(dims, bd, b, &G);
  int64_t n = 1;
  for (int a = 0; a < 3; a++) {
    int64_t rest = dims[a] - G.k[a] * bd[a];
    n *= rest < bd[a] ? rest : bd[a];
  }
  return n;
}

/* box holding field position (z, y, x) */
static int64_t nd_box_of(const int64_t *dims, const int64_t *bd, int64_t z, int64_t y, int64_t x) {
  int64_t g1 = (dims[1] + bd[1] - 1) / bd[1], g2 = (dims[2] + bd[2] - 1) / bd[2];
  return ((z / bd[0]) * g1 + y / bd[1]) * g2 + x / bd[2];
}

static int nd_setup(int ndim, const int64_t *dims_in, const int64_t *block_in, orc_header *h) {
  if (ndim < 1 || ndim > 3) return ORC_ERR_INVALID_ARG;
  memset(h, 0, sizeof *h);
  int64_t n = 1, S = 1;
  for (int a = 0; a < 3; a++) {
    h->dims[a] = 1;
    h->bd[a] = 1;
  }
  for (int a = 0; a < ndim; a++) {
    if (dims_in[a] < 1 || block_in[a] < 1) return ORC_ERR_INVALID_ARG;
    h->dims[3 - ndim + a] = dims_in[a];
    h->bd[3 - ndim + a] = block_in[a];
    n *= dims_in[a];
    S *= block_in[a];
  }
  if (S > ORC_MAX_S) return ORC_ERR_INVALID_ARG;
  h->N = n;
  h->S = (int)S;
  layout(h);
  return ORC_OK;
}

int64_t orc_compress_bound_nd(int ndim, const int64_t *dims, const int64_t *block) {
  orc_header h;
  if (nd_setup(ndim, dims, block, &h)) return -1;
  return align16(h.off_payload + 4 * h.nb * block_words(h.S, 31) + 16);
}

int orc_compress_codes_nd(const int32_t *q, int dtype, int ndim, const int64_t *dims_in, const int64_t *block_in,
                          double eps, double eb, int eb_mode, uint8_t *out, int64_t cap, int64_t *out_bytes) {
  if (!(eps > 0.0) || (dtype != 0 && dtype != 1)) return ORC_ERR_INVALID_ARG;
  orc_header h;
  int st = nd_setup(ndim, dims_in, block_in, &h);
  if (st) return st;
  int64_t bound = align16(h.off_payload + 4 * h.nb * block_words(h.S, 31) + 16);
  if (cap < bound) return ORC_ERR_INVALID_ARG;
  memset(out, 0, (size_t)bound);
  for (int64_t i = 0; i < h.N; i++)
    if (!(q[i] > -ORC_QLIMIT && q[i] < ORC_QLIMIT)) return ORC_ERR_RANGE;
  int S = h.S;
  int32_t *p = (int32_t *)malloc(sizeof(int32_t) * (size_t)S);
  if (!p) return ORC_ERR_INVALID_ARG;
  int64_t word = 0, qmax = 0;
  int wmax = 0;
  for (int64_t b = 0; b < h.nb; b++) {
    if (b % h.G == 0) put_u64(out, h.off_chunks + 8 * (b / h.G), (uint64_t)word);
    nd_grid G;
    nd_box(h.dims, h.bd, b, &G);
    /* metadata: the box mean over its true size */
    int64_t sum = 0, Sb = 0;
    for (int64_t k = 0; k < S; k++) {
      int64_t i = nd_slot_index(h.dims, h.bd, &G, k);
      if (i < 0) continue;
      sum += q[i];
      Sb++;
      int64_t a = q[i] < 0 ? -(int64_t)q[i] : q[i];
      if (a > qmax) qmax = a;
    }
    int32_t M = (int32_t)nearest_ratio(sum, Sb);
    put_u32(out, h.off_heads + 4 * b, (uint32_t)M);
    uint32_t maxmag = 0;
    for (int64_t k = 0; k < S; k++) {
      int64_t i = nd_slot_index(h.dims, h.bd, &G, k);
      p[k] = i < 0 ? 0 : q[i] - M;
      uint32_t m = (uint32_t)(p[k] < 0 ? -(int64_t)p[k] : p[k]);
      if (m > maxmag) maxmag = m;
    }
    int w = bit_length(maxmag);
    if (w > wmax) wmax = w;
    put_u8(out, h.off_widths + b, (uint32_t)w);
    if (w == 0) continue;
    encode_block(out, &h, word, p, w);
    word += block_words(S, w);
  }
  free(p);
  h.qmax = qmax;
  h.wmax = wmax;
  h.eps = eps;
  h.eb = eb;
  h.eb_mode = eb_mode;
  h.dtype = dtype;
  h.ndim = ndim;
  h.pred = 4;
  finish_stream(out, &h, word);
  *out_bytes = h.total_bytes;
  return ORC_OK;
}

int orc_compress_nd(const void *x, int dtype, int ndim, const int64_t *dims, const int64_t *block, double eb,
                    int eb_mode, uint8_t *out, int64_t cap, int64_t *out_bytes, double *eps_out) {
  if (ndim < 1 || ndim > 3) return ORC_ERR_INVALID_ARG;
  int64_t n = 1;
  for (int a = 0; a < ndim; a++) {
    if (dims[a] < 1) return ORC_ERR_INVALID_ARG;
    n *= dims[a];
  }
  double eps;
  int st = orc_eps(x, dtype, n, eb, eb_mode, &eps);
  if (st) return st;
  int32_t *q = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  if (!q) return ORC_ERR_INVALID_ARG;
  st = orc_quantize(x, dtype, n, eps, q);
  if (!st) st = orc_compress_codes_nd(q, dtype, ndim, dims, block, eps, eb, eb_mode, out, cap, out_bytes);
  free(q);
  if (eps_out) *eps_out = eps;
  return st;
}

int orc_compress_codes(const int32_t *q, int dtype, int ndim, const int64_t *dims_in, double eps,
                       double eb, int eb_mode, int S, uint8_t *out, int64_t cap,
                       int64_t *out_bytes) {
  return orc_compress_codes_pred(q, dtype, ndim, dims_in, eps, eb, eb_mode, S, 0, out, cap, out_bytes);
}

int orc_compress_pred(const void *x, int dtype, int ndim, const int64_t *dims, double eb, int eb_mode,
                      int S, int pred, uint8_t *out, int64_t cap, int64_t *out_bytes, double *eps_out) {
  if (ndim < 1 || ndim > 3) return ORC_ERR_INVALID_ARG;
  int64_t n = 1;
  for (int a = 0; a < ndim; a++) {
    if (dims[a] < 1) return ORC_ERR_INVALID_ARG;
    n *= dims[a];
  }
  double eps;
  int st = orc_eps(x, dtype, n, eb, eb_mode, &eps);
  if (st) return st;
  int32_t *q = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  if (!q) return ORC_ERR_INVALID_ARG;
  st = orc_quantize(x, dtype, n, eps, q);
  if (!st) st = orc_compress_codes_pred(q, dtype, ndim, dims, eps, eb, eb_mode, S, pred, out, cap, out_bytes);
  free(q);
  if (eps_out) *eps_out = eps;
  return st;
}

int orc_compress(const void *x, int dtype, int ndim, const int64_t *dims, double eb, int eb_mode,
                 int S, uint8_t *out, int64_t cap, int64_t *out_bytes, double *eps_out) {
  return orc_compress_pred(x, dtype, ndim, dims, eb, eb_mode, S, 0, out, cap, out_bytes, eps_out);
}

/* ------------------------------------------------------------------ */
/* Header parsing with the structural checks a reader must make         */
/* ------------------------------------------------------------------ */
static int parse(const uint8_t *s, int64_t bytes, orc_header *h) {
  if (bytes < ORC_HEADER_BYTES) return ORC_ERR_CORRUPT;
  if (get_u32(s, 0) != ORC_MAGIC || get_u16(s, 4) != ORC_VERSION) return ORC_ERR_CORRUPT;
  memset(h, 0, sizeof *h);
  h->dtype = (int)get_u8(s, 6);
  h->ndim = (int)get_u8(s, 7);
  for (int a = 0; a < 3; a++) h->dims[a] = (int64_t)get_u64(s, 8 + 8 * a);
  h->S = (int)get_u32(s, 32);
  h->eps = get_f64(s, 40);
  h->eb = get_f64(s, 48);
  h->eb_mode = (int)get_u32(s, 56);
  h->qmax = get_u32(s, 60);
  h->N = (int64_t)get_u64(s, 64);
  if (h->dtype > 1 || h->ndim < 1 || h->ndim > 3 || h->S < 1 || h->S > ORC_MAX_S) return ORC_ERR_CORRUPT;
  if (h->dims[0] < 1 || h->dims[1] < 1 || h->dims[2] < 1) return ORC_ERR_CORRUPT;
  if (h->dims[0] * h->dims[1] * h->dims[2] != h->N) return ORC_ERR_CORRUPT;
  int64_t bprod = 1;
  for (int a = 0; a < 3; a++) {
    h->bd[a] = (int64_t)get_u32(s, 144 + 4 * a);
    bprod *= h->bd[a];
  }
  if ((int)get_u32(s, 140) == 4) {
    if (bprod != h->S) return ORC_ERR_CORRUPT;
  } else if (bprod != 0 || h->bd[0] || h->bd[1] || h->bd[2]) {
    return ORC_ERR_CORRUPT;
  }
  orc_header ref = *h;
  layout(&ref);
  h->nb = ref.nb;
  h->G = ref.G;
  h->nchunks = ref.nchunks;
  h->off_widths = ref.off_widths;
  h->off_heads = ref.off_heads;
  h->off_chunks = ref.off_chunks;
  h->off_payload = ref.off_payload;
  if ((int64_t)get_u32(s, 36) != h->G || (int64_t)get_u64(s, 72) != h->nb ||
      (int64_t)get_u64(s, 80) != h->nchunks || (int64_t)get_u64(s, 96) != h->off_widths ||
      (int64_t)get_u64(s, 104) != h->off_heads || (int64_t)get_u64(s, 112) != h->off_chunks ||
      (int64_t)get_u64(s, 120) != h->off_payload)
    return ORC_ERR_CORRUPT;
  h->payload_words = (int64_t)get_u64(s, 88);
  h->total_bytes = (int64_t)get_u64(s, 128);
  h->wmax = (int)get_u32(s, 136);
  h->pred = (int)get_u32(s, 140);
  if (h->pred < 0 || h->pred > 4) return ORC_ERR_CORRUPT;
  if (h->total_bytes != align16(h->off_payload + 4 * h->payload_words + 16)) return ORC_ERR_CORRUPT;
  if (h->total_bytes > bytes) return ORC_ERR_CORRUPT;
  if (!(h->eps > 0.0)) return ORC_ERR_CORRUPT;
  return ORC_OK;
}

/* exported view of the header: 20 int64 fields + 2 doubles */
int orc_read_header(const uint8_t *s, int64_t bytes, int64_t *ints, double *dbls) {
  orc_header h;
  int st = parse(s, bytes, &h);
  if (st) return st;
  ints[0] = h.dtype;
  ints[1] = h.ndim;
  ints[2] = h.dims[0];
  ints[3] = h.dims[1];
  ints[4] = h.dims[2];
  ints[5] = h.S;
  ints[6] = h.G;
  ints[7] = h.eb_mode;
  ints[8] = h.qmax;
  ints[9] = h.N;
  ints[10] = h.nb;
  ints[11] = h.nchunks;
  ints[12] = h.payload_words;
  ints[13] = h.total_bytes;
  ints[14] = h.wmax;
  ints[15] = h.off_payload;
  ints[16] = h.pred;
  ints[17] = h.bd[0];
  ints[18] = h.bd[1];
  ints[19] = h.bd[2];
  dbls[0] = h.eps;
  dbls[1] = h.eb;
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Multi-stage partial decompression: Algorithm 2.                      */
/* decode() returns D_p for one block; recorrelate() undoes the          */
/* within-block delta; dequantize() multiplies by 2 eps.                 */
/* ------------------------------------------------------------------ */

/* decode(c_b): signs and magnitudes of block b -> p_k for k < S.
 * Returns the block's width or -1 when the stream is inconsistent. */
static int decode_block(const uint8_t *s, const orc_header *h, int64_t b, int64_t word,
                        int32_t *p) {
  int w = (int)get_u8(s, h->off_widths + b);
  if (w > 31) return -1;
  for (int k = 0; k < h->S; k++) p[k] = 0;
  if (w == 0) return 0;
  int64_t nsw = (h->S + 31) / 32;
  if (word + block_words(h->S, w) > h->payload_words) return -1;
  for (int k = 0; k < h->S; k++) {
    uint32_t m = 0;
    for (int j = 0; j < w; j++) {
      int64_t bit = (int64_t)k * w + j;
      int64_t byte = h->off_payload + 4 * (word + nsw + bit / 32) + (bit % 32) / 8;
      if ((s[byte] >> (bit % 8)) & 1u) m |= 1u << j;
    }
    int64_t sbyte = h->off_payload + 4 * (word + k / 32) + (k % 32) / 8;
    int neg = (s[sbyte] >> (k % 8)) & 1u;
    p[k] = neg ? -(int32_t)m : (int32_t)m;
  }
  return w;
}

/* Walk all blocks; per block call back with (b, first index, Sb, head, p).
 * The payload word offset of each block is the running sum of block sizes,
 * checked against the stored chunk index at every chunk start. */
typedef void (*block_fn)(void *ctx, int pred, int64_t b, int64_t first, int64_t Sb, int32_t head,
                         const int32_t *p);

static int walk(const uint8_t *s, int64_t bytes, block_fn fn, void *ctx, orc_header *hout) {
  orc_header h;
  int st = parse(s, bytes, &h);
  if (st) return st;
  int32_t *p = (int32_t *)malloc(sizeof(int32_t) * (size_t)h.S);
  if (!p) return ORC_ERR_INVALID_ARG;
  int64_t word = 0;
  for (int64_t b = 0; b < h.nb; b++) {
    if (b % h.G == 0 && (int64_t)get_u64(s, h.off_chunks + 8 * (b / h.G)) != word) {
      free(p);
      return ORC_ERR_CORRUPT;
    }
    int w = decode_block(s, &h, b, word, p);
    if (w < 0) {
      free(p);
      return ORC_ERR_CORRUPT;
    }
    int64_t first = b * h.S;
    int64_t Sb = (first + h.S <= h.N) ? h.S : h.N - first;
    int32_t head = (int32_t)get_u32(s, h.off_heads + 4 * b);
    fn(ctx, h.pred, b, first, Sb, head, p);
    word += block_words(h.S, w);
  }
  free(p);
  if (word != h.payload_words ||
      (int64_t)get_u64(s, h.off_chunks + 8 * h.nchunks) != h.payload_words)
    return ORC_ERR_CORRUPT;
  if (hout) *hout = h;
  return ORC_OK;
}

/* Stage 2 (D_p).  Predictor 0 -- reading: the materialized D_p carries the
 * block's head in the slot of its first element, so that q is the inclusive
 * prefix sum of D_p inside every block (the form q_i = sum_{t<=i} p_t of
 * Section V-A).  Predictor 1: D_p = q - M_b in every slot (Section IV,
 * "HSZx"). */
static void put_p(void *ctx, int pred, int64_t b, int64_t first, int64_t Sb, int32_t head,
                  const int32_t *p) {
  (void)b;
  int32_t *dp = (int32_t *)ctx;
  if (pred != 0) { /* every slot holds a residual (HSZx and the global predictors) */
    for (int64_t k = 0; k < Sb; k++) dp[first + k] = p[k];
    return;
  }
  dp[first] = head;
  for (int64_t k = 1; k < Sb; k++) dp[first + k] = p[k];
}
/* HSZx-nd: the slots of box b go back to their field positions (slots
 * outside the field are dropped); stage 2 holds p, stage 3 M_b + p. */
typedef struct {
  const orc_header *h;
  int32_t *out;
  int add_mean;
} nd_ctx;
static void put_nd(void *ctx, int pred, int64_t b, int64_t first, int64_t Sb, int32_t head, const int32_t *p) {
  (void)pred;
  (void)first;
  (void)Sb;
  nd_ctx *c = (nd_ctx *)ctx;
  nd_grid G;
  nd_box(c->h->dims, c->h->bd, b, &G);
  for (int64_t k = 0; k < c->h->S; k++) {
    int64_t i = nd_slot_index(c->h->dims, c->h->bd, &G, k);
    if (i >= 0) c->out[i] = c->add_mean ? head + p[k] : p[k];
  }
}
static int decode_nd(const uint8_t *s, int64_t bytes, int32_t *out, int add_mean) {
  orc_header h;
  int st = parse(s, bytes, &h);
  if (st) return st;
  nd_ctx c = {&h, out, add_mean};
  return walk(s, bytes, put_nd, &c, NULL);
}

int orc_decode_p(const uint8_t *s, int64_t bytes, int32_t *dp) {
  orc_header h;
  int st = parse(s, bytes, &h);
  if (st) return st;
  if (h.pred == 4) return decode_nd(s, bytes, dp, 0);
  return walk(s, bytes, put_p, dp, NULL);
}

/* Stage 3 (D_q).  Predictor 0: recorrelate q_k = q_{k-1} + p_k from the
 * head.  Predictor 1: q_k = M_b + p_k. */
static void put_q(void *ctx, int pred, int64_t b, int64_t first, int64_t Sb, int32_t head,
                  const int32_t *p) {
  (void)b;
  int32_t *dq = (int32_t *)ctx;
  if (pred == 1) {
    for (int64_t k = 0; k < Sb; k++) dq[first + k] = head + p[k];
    return;
  }
  int32_t q = head;
  dq[first] = q;
  for (int64_t k = 1; k < Sb; k++) {
    q = q + p[k];
    dq[first + k] = q;
  }
}
/* Global predictors: q is the inclusive prefix sum of D_p over every
 * prediction axis, rebuilt plane by plane with the row-wise recurrence of
 * Algorithm 4 (HSZp-2d): a prefix sum runs along the row, a column buffer
 * accumulates it down the plane (colSum), and, for a 3-D field, the plane
 * below is added (q_{k,i,j} = q_{k-1,i,j} + colSum_j).  In place. */
static void lorenzo_rebuild(int32_t *a, const int64_t *L) {
  int64_t *col = (int64_t *)calloc((size_t)L[2], sizeof(int64_t));
  for (int64_t z = 0; z < L[0]; z++) {
    for (int64_t x = 0; x < L[2]; x++) col[x] = 0;
    for (int64_t y = 0; y < L[1]; y++) {
      int64_t pref = 0;
      for (int64_t x = 0; x < L[2]; x++) {
        int64_t i = (z * L[1] + y) * L[2] + x;
        pref += a[i];
        col[x] += pref;
        int64_t below = z > 0 ? a[i - L[1] * L[2]] : 0;
        a[i] = (int32_t)(below + col[x]);
      }
    }
  }
  free(col);
}

int orc_decode_q(const uint8_t *s, int64_t bytes, int32_t *dq) {
  orc_header h;
  int st = parse(s, bytes, &h);
  if (st) return st;
  if (h.pred == 4) return decode_nd(s, bytes, dq, 1);
  if (h.pred < 2) return walk(s, bytes, put_q, dq, NULL);
  st = walk(s, bytes, put_p, dq, NULL);
  if (st) return st;
  int64_t L[3];
  global_dims(h.dims, h.N, h.pred, L);
  lorenzo_rebuild(dq, L);
  return ORC_OK;
}

/* Stage 1 (D_m): the block metadata (heads, or the block means of HSZx). */
static void put_m(void *ctx, int pred, int64_t b, int64_t first, int64_t Sb, int32_t head,
                  const int32_t *p) {
  (void)pred;
  (void)first;
  (void)Sb;
  (void)p;
  ((int32_t *)ctx)[b] = head;
}
int orc_decode_m(const uint8_t *s, int64_t bytes, int32_t *heads) {
  orc_header h;
  int st = parse(s, bytes, &h);
  if (st) return st;
  /* the global predictors keep no block metadata (Table 2: stages 2-4) */
  if (h.pred == 2 || h.pred == 3) return ORC_ERR_UNSUPPORTED;
  return walk(s, bytes, put_m, heads, NULL);
}

/* Stage 4 (D_f): dequantize d' = 2 eps q.  Reading: a float32 field is
 * reconstructed in float32 arithmetic, (float)q * (float)(2 eps); a float64
 * field as (double)q * (2 eps). */
int orc_dequantize(const int32_t *q, int64_t n, double eps, int dtype, void *f) {
  double two_eps = 2.0 * eps;
  if (dtype == 0) {
    float te = (float)two_eps;
    float *o = (float *)f;
    for (int64_t i = 0; i < n; i++) {
      float qf = (float)q[i];
      o[i] = qf * te;
    }
  } else {
    double *o = (double *)f;
    for (int64_t i = 0; i < n; i++) o[i] = (double)q[i] * two_eps;
  }
  return ORC_OK;
}

int orc_decode_f(const uint8_t *s, int64_t bytes, void *f) {
  orc_header h;
  int st = parse(s, bytes, &h);
  if (st) return st;
  int32_t *q = (int32_t *)malloc(sizeof(int32_t) * (size_t)h.N);
  if (!q) return ORC_ERR_INVALID_ARG;
  st = orc_decode_q(s, bytes, q);
  if (!st) st = orc_dequantize(q, h.N, h.eps, h.dtype, f);
  free(q);
  return st;
}

/* ------------------------------------------------------------------ */
/* Statistics                                                           */
/* ------------------------------------------------------------------ */

/* Stage 3 mean / standard deviation inputs: exact sum(q) and sum(q^2)
 * (Section V-A, "Operation with D_q" and Eq. var_q). */
int orc_sums_q(const int32_t *q, int64_t n, int64_t *s1, uint64_t *s2_lo, uint64_t *s2_hi) {
  int64_t a = 0;
  u128 b = 0;
  for (int64_t i = 0; i < n; i++) {
    a += q[i];
    b += (u128)((int64_t)q[i] * (int64_t)q[i]);
  }
  *s1 = a;
  *s2_lo = (uint64_t)b;
  *s2_hi = (uint64_t)(b >> 64);
  return ORC_OK;
}

/* Stage 2 mean for HSZp-style blocks (Section V-A, "Operation with D_p"):
 * the block sum of q is sum_{i=1}^{S_b} (S_b - i + 1) p_i, with p_1 the head
 * (first slot of the materialized D_p).  No prefix sum is formed. */
int orc_mean_p_sum(const int32_t *dp, int64_t n, int S, int64_t *s1) {
  int64_t total = 0;
  for (int64_t first = 0; first < n; first += S) {
    int64_t Sb = (first + S <= n) ? S : n - first;
    for (int64_t i = 1; i <= Sb; i++) total += (Sb - i + 1) * (int64_t)dp[first + i - 1];
  }
  *s1 = total;
  return ORC_OK;
}

/* Stage 2 standard deviation for HSZp-style blocks (Section V-A): a running
 * accumulator eta = sum_{j<=i} p_j rebuilds q inside each block and feeds
 * s1 += eta, s2 += eta^2.  With within-block prediction eta restarts at every
 * block (reading: the paper gives eta for inter-block prediction; with the
 * head kept as block metadata the accumulator starts again at each head). */
int orc_var_p_sums(const int32_t *dp, int64_t n, int S, int64_t *s1, uint64_t *s2_lo,
                   uint64_t *s2_hi) {
  int64_t a = 0;
  u128 b = 0;
  for (int64_t first = 0; first < n; first += S) {
    int64_t Sb = (first + S <= n) ? S : n - first;
    int64_t eta = 0;
    for (int64_t i = 0; i < Sb; i++) {
      eta += dp[first + i];
      a += eta;
      b += (u128)(eta * eta);
    }
  }
  *s1 = a;
  *s2_lo = (uint64_t)b;
  *s2_hi = (uint64_t)(b >> 64);
  return ORC_OK;
}

/* Stage 1 mean of HSZx (Eq. mean_m): T = sum_b M_b * S_b from the block
 * means alone; mu = (T / N) * 2 eps.  S_b is the true size of block b. */
int orc_mean_m_sum(const int32_t *M, int64_t nb, int S, int64_t n, int64_t *T) {
  int64_t t = 0;
  for (int64_t b = 0; b < nb; b++) {
    int64_t first = b * S;
    int64_t Sb = (first + S <= n) ? S : n - first;
    t += (int64_t)M[b] * Sb;
  }
  *T = t;
  return ORC_OK;
}

/* Stage 2 mean of HSZx (Section V-A, "Operation with D_p"): the block sum of
 * q is sum_{p in block} p + M_b S_b. */
int orc_mean_p_sum_x(const int32_t *dp, const int32_t *M, int64_t n, int S, int64_t *s1) {
  int64_t total = 0;
  for (int64_t first = 0, b = 0; first < n; first += S, b++) {
    int64_t Sb = (first + S <= n) ? S : n - first;
    for (int64_t k = 0; k < Sb; k++) total += dp[first + k];
    total += (int64_t)M[b] * Sb;
  }
  *s1 = total;
  return ORC_OK;
}

/* Stage 2 standard deviation of HSZx (Section V-A): with the integer mean
 * mu~ = round(T / N) (T as in orc_mean_m_sum; the same rounding as the block
 * means: nearest, ties toward zero, in exact integer arithmetic), each
 * deviation is split
 * as (q - M_b) + (M_b - mu~) = p + M_b - mu~, and
 *   sigma = sqrt(sum (p + M_b - mu~)^2 / (N - 1)) * 2 eps.
 * Returns mu~, the exact 128-bit sum of squares and sigma (NaN for N = 1). */
int orc_std_p_x(const int32_t *dp, const int32_t *M, int64_t n, int S, double eps, int64_t *mu_tilde,
                uint64_t *ss_lo, uint64_t *ss_hi, double *sigma) {
  int64_t nb = (n + S - 1) / S, T;
  orc_mean_m_sum(M, nb, S, n, &T);
  int64_t mt = nearest_ratio(T, n);
  u128 ss = 0;
  for (int64_t first = 0, b = 0; first < n; first += S, b++) {
    int64_t Sb = (first + S <= n) ? S : n - first;
    for (int64_t k = 0; k < Sb; k++) {
      int64_t d = (int64_t)dp[first + k] + M[b] - mt;
      ss += (u128)((i128)d * d);
    }
  }
  *mu_tilde = mt;
  *ss_lo = (uint64_t)ss;
  *ss_hi = (uint64_t)(ss >> 64);
  *sigma = n < 2 ? NAN : sqrt((double)ss / (double)(n - 1)) * (2.0 * eps);
  return ORC_OK;
}

/* Final scaling of the exact sums (Eq. var and Eq. var_q):
 *   mean     = (s1 / N) * 2 eps
 *   variance = ((N s2 - s1^2) / (N (N - 1))) * (2 eps)^2
 * The numerator N s2 - s1^2 equals N (s2 - s1^2 / N) of Eq. var_q and is
 * formed exactly in 128-bit integers (reading: the paper's floating-point
 * s2 - s1^2/N cancels catastrophically).  N = 1 gives variance NaN. */
int orc_finalize(int64_t n, int64_t s1, uint64_t s2_lo, uint64_t s2_hi, double eps,
                 double *mean, double *var, double *sd) {
  double two_eps = 2.0 * eps;
  *mean = ((double)s1 / (double)n) * two_eps;
  if (n < 2) {
    *var = NAN;
    *sd = NAN;
    return ORC_OK;
  }
  u128 s2 = ((u128)s2_hi << 64) | (u128)s2_lo;
  i128 num = (i128)n * (i128)s2 - (i128)s1 * (i128)s1;
  double numd = (double)num;
  double den = (double)n * (double)(n - 1);
  *var = (numd / den) * (two_eps * two_eps);
  *sd = sqrt(*var);
  return ORC_OK;
}

/* Generic flow on D_f (Eq. var): mean by compensated (Neumaier) summation,
 * sample variance by a second compensated pass over (d - mean)^2. */
int orc_stats_f(const void *f, int dtype, int64_t n, double *mean, double *var) {
  double s = 0.0, c = 0.0;
  for (int64_t i = 0; i < n; i++) {
    double v = load_x(f, dtype, i);
    double t = s + v;
    if (fabs(s) >= fabs(v))
      c += (s - t) + v;
    else
      c += (v - t) + s;
    s = t;
  }
  double mu = (s + c) / (double)n;
  *mean = mu;
  if (n < 2) {
    *var = NAN;
    return ORC_OK;
  }
  s = 0.0;
  c = 0.0;
  for (int64_t i = 0; i < n; i++) {
    double d = load_x(f, dtype, i) - mu;
    double v = d * d;
    double t = s + v;
    if (fabs(s) >= fabs(v))
      c += (s - t) + v;
    else
      c += (v - t) + s;
    s = t;
  }
  *var = (s + c) / (double)(n - 1);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Stage 2 of the global predictors (predictors 2 and 3).  L is the      */
/* prediction shape (L0, L1, L2): the field's (n0, n1, n2) for HSZp-nd,  */
/* (1, 1, N) for HSZp.  q at (z, y, x) is the sum of D_p over the box    */
/* [0..z] x [0..y] x [0..x].                                            */
/* ------------------------------------------------------------------ */

/* Mean (Section V-A, "Operation with D_p", the HSZp-2d weighted sum and the
 * HSZp identity sum q_i = sum (S - i + 1) p_i with the prediction running
 * over the whole field): every p is counted once for each code of the box
 * that starts at it, so sum q = sum p (L0 - z)(L1 - y)(L2 - x). */
int orc_lorenzo_mean_p(const int32_t *dp, const int64_t *L, int64_t *s1) {
  i128 t = 0;
  for (int64_t z = 0; z < L[0]; z++)
    for (int64_t y = 0; y < L[1]; y++)
      for (int64_t x = 0; x < L[2]; x++) {
        int64_t i = (z * L[1] + y) * L[2] + x;
        t += (i128)dp[i] * (L[0] - z) * (L[1] - y) * (L[2] - x);
      }
  *s1 = (int64_t)t;
  return ORC_OK;
}

/* Standard deviation inputs (Section V-A): Algorithm 4's column buffer and
 * row prefix rebuild each q in turn (for a 3-D field on top of the same
 * position of the plane below, for HSZp the single row's running sum eta),
 * and s1 += q, s2 += q^2 are accumulated without storing D_q. */
int orc_lorenzo_var_p(const int32_t *dp, const int64_t *L, int64_t *s1, uint64_t *s2_lo, uint64_t *s2_hi) {
  int64_t *col = (int64_t *)calloc((size_t)L[2], sizeof(int64_t));
  int64_t *below = (int64_t *)calloc((size_t)(L[1] * L[2]), sizeof(int64_t));
  if (!col || !below) {
    free(col);
    free(below);
    return ORC_ERR_INVALID_ARG;
  }
  int64_t a = 0;
  u128 b = 0;
  for (int64_t z = 0; z < L[0]; z++) {
    for (int64_t x = 0; x < L[2]; x++) col[x] = 0;
    for (int64_t y = 0; y < L[1]; y++) {
      int64_t pref = 0;
      for (int64_t x = 0; x < L[2]; x++) {
        pref += dp[(z * L[1] + y) * L[2] + x];
        col[x] += pref;
        int64_t qv = below[y * L[2] + x] + col[x];
        below[y * L[2] + x] = qv;
        a += qv;
        b += (u128)(qv * qv);
      }
    }
  }
  free(col);
  free(below);
  *s1 = a;
  *s2_lo = (uint64_t)b;
  *s2_hi = (uint64_t)(b >> 64);
  return ORC_OK;
}

/* inclusive prefix sum of a (int64, shape L) along internal axis ax */
static void prefix_along(int64_t *a, const int64_t *L, int ax) {
  int64_t st = ax == 2 ? 1 : (ax == 1 ? L[2] : L[1] * L[2]);
  for (int64_t z = 0; z < L[0]; z++)
    for (int64_t y = 0; y < L[1]; y++)
      for (int64_t x = 0; x < L[2]; x++) {
        int64_t c = ax == 0 ? z : (ax == 1 ? y : x);
        if (c == 0) continue;
        int64_t i = (z * L[1] + y) * L[2] + x;
        a[i] += a[i - st];
      }
}

static int64_t dp_at(const int32_t *dp, const int64_t *L, int64_t z, int64_t y, int64_t x) {
  return dp[(z * L[1] + y) * L[2] + x];
}

/* Derivative numerators on D_p of HSZp-nd (Section V-B, Eq. derivative_Dp
 * and the sum form above it): q[i+1] - q[i-1] along axis a is the box sum
 * of p over the other axes, taken at the two slices a = i and a = i + 1,
 * i.e. D_a = P_other(r) with r(i) = p(i) + p(i + e_a); the recursion of
 * Eq. derivative_Dp is this prefix sum written incrementally (eta along the
 * row, the column accumulators across rows).  Edges (the reading of the
 * stage-3 operation): at a = 0, 2 (q_1 - q_0) = 2 P_other(p(i + e_a)); at
 * the last slice, 2 (q_{n-1} - q_{n-2}) = 2 P_other(p(i)); an axis of
 * length 1 gives 0.  dims3 = the field's (n0, n1, n2); axis internal. */
int orc_lorenzo_deriv_p(const int32_t *dp, const int64_t *dims3, int axis, int64_t *D) {
  const int64_t *L = dims3;
  for (int64_t z = 0; z < L[0]; z++)
    for (int64_t y = 0; y < L[1]; y++)
      for (int64_t x = 0; x < L[2]; x++) {
        int64_t c[3] = {z, y, x};
        int64_t len = L[axis], k = c[axis];
        int64_t nx[3] = {z, y, x};
        nx[axis] = k + 1;
        int64_t r;
        if (len == 1)
          r = 0;
        else if (k == 0)
          r = 2 * dp_at(dp, L, nx[0], nx[1], nx[2]);
        else if (k == len - 1)
          r = 2 * dp_at(dp, L, z, y, x);
        else
          r = dp_at(dp, L, z, y, x) + dp_at(dp, L, nx[0], nx[1], nx[2]);
        D[(z * L[1] + y) * L[2] + x] = r;
      }
  for (int ax = 0; ax < 3; ax++)
    if (ax != axis) prefix_along(D, L, ax);
  return ORC_OK;
}

/* Laplacian numerators on D_p of HSZp-nd (Section V-B, Eq. laplacian_Dp):
 * per axis, (q[i+1] - q[i]) - (q[i] - q[i-1]) is the difference of two box
 * sums of p over the other axes (the xi prefix sums of the paper): with
 * t_a(i) = [i_a < n_a - 1] p(i + e_a) - [i_a > 0] p(i) (a missing neighbour
 * replicates the edge value, so its difference is 0), L = sum_a P_other(t_a).
 * dims3 = the field's (n0, n1, n2). */
int orc_lorenzo_lap_p(const int32_t *dp, const int64_t *dims3, int64_t *Lout) {
  const int64_t *L = dims3;
  int64_t n = L[0] * L[1] * L[2];
  int64_t *t = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  if (!t) return ORC_ERR_INVALID_ARG;
  for (int64_t i = 0; i < n; i++) Lout[i] = 0;
  for (int a = 0; a < 3; a++) {
    for (int64_t z = 0; z < L[0]; z++)
      for (int64_t y = 0; y < L[1]; y++)
        for (int64_t x = 0; x < L[2]; x++) {
          int64_t c[3] = {z, y, x};
          int64_t nx[3] = {z, y, x};
          nx[a] = c[a] + 1;
          int64_t v = 0;
          if (c[a] < L[a] - 1) v += dp_at(dp, L, nx[0], nx[1], nx[2]);
          if (c[a] > 0) v -= dp_at(dp, L, z, y, x);
          t[(z * L[1] + y) * L[2] + x] = v;
        }
    for (int ax = 0; ax < 3; ax++)
      if (ax != a) prefix_along(t, L, ax);
    for (int64_t i = 0; i < n; i++) Lout[i] += t[i];
  }
  free(t);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* HSZx-nd operations (Sections V-A and V-B) on D_p in field order and   */
/* the box means M (row-major over the box grid).  bd = (b0, b1, b2).    */
/* ------------------------------------------------------------------ */

/* Stage 1 mean (Eq. mean_m): T = sum_b M_b S_b with the true box sizes. */
int orc_xnd_mean_m(const int32_t *M, const int64_t *dims3, const int64_t *bd, int64_t *T) {
  int64_t nb = grid_blocks(dims3, bd), t = 0;
  for (int64_t b = 0; b < nb; b++) t += (int64_t)M[b] * nd_box_size(dims3, bd, b);
  *T = t;
  return ORC_OK;
}

/* Stage 2 mean (Section V-A): sum q = sum_b (sum_{p in B_b} p + M_b S_b). */
int orc_xnd_mean_p(const int32_t *dp, const int32_t *M, const int64_t *dims3, const int64_t *bd, int64_t *s1) {
  int64_t t = 0;
  orc_xnd_mean_m(M, dims3, bd, &t);
  int64_t n = dims3[0] * dims3[1] * dims3[2];
  for (int64_t i = 0; i < n; i++) t += dp[i];
  *s1 = t;
  return ORC_OK;
}

/* Stage 2 standard deviation (Section V-A): about the integer mean
 * mu~ = round(T / N) of stage 1 (nearest, ties toward zero),
 * sigma = sqrt(sum (p + M_b - mu~)^2 / (N - 1)) 2 eps; the exact 128-bit
 * sum of squares is returned too. */
int orc_xnd_std_p(const int32_t *dp, const int32_t *M, const int64_t *dims3, const int64_t *bd, double eps,
                  int64_t *mu_tilde, uint64_t *s2_lo, uint64_t *s2_hi, double *sigma) {
  int64_t n = dims3[0] * dims3[1] * dims3[2];
  int64_t T;
  orc_xnd_mean_m(M, dims3, bd, &T);
  int64_t mu = nearest_ratio(T, n);
  u128 acc = 0;
  for (int64_t z = 0; z < dims3[0]; z++)
    for (int64_t y = 0; y < dims3[1]; y++)
      for (int64_t x = 0; x < dims3[2]; x++) {
        int64_t i = (z * dims3[1] + y) * dims3[2] + x;
        int64_t d = (int64_t)dp[i] + M[nd_box_of(dims3, bd, z, y, x)] - mu;
        acc += (u128)(d * d);
      }
  *mu_tilde = mu;
  *s2_lo = (uint64_t)acc;
  *s2_hi = (uint64_t)(acc >> 64);
  double v = n >= 2 ? (double)acc / (double)(n - 1) : NAN;
  *sigma = sqrt(v) * 2.0 * eps;
  return ORC_OK;
}

static int64_t xnd_p(const int32_t *dp, const int64_t *d, const int64_t *c) {
  return dp[(c[0] * d[1] + c[1]) * d[2] + c[2]];
}
static int64_t xnd_m(const int32_t *M, const int64_t *d, const int64_t *bd, const int64_t *c) {
  return M[nd_box_of(d, bd, c[0], c[1], c[2])];
}

/* Stage 2 derivative numerators of HSZx-nd (Section V-B, "Operation with
 * D_p", HSZx-2d, written for every axis of a 3-D field): inside a box
 * D = p[i+e] - p[i-e]; where a neighbour lies in another box the difference
 * of the box means is added, D = p[i+e] - p[i-e] + (M_{box(i+e)} -
 * M_{box(i-e)}).  Domain edges as at stage 3: one-sided and doubled, 0 on an
 * axis of length 1. */
int orc_xnd_deriv_p(const int32_t *dp, const int32_t *M, const int64_t *dims3, const int64_t *bd, int axis,
                    int64_t *D) {
  const int64_t *d = dims3;
  for (int64_t z = 0; z < d[0]; z++)
    for (int64_t y = 0; y < d[1]; y++)
      for (int64_t x = 0; x < d[2]; x++) {
        int64_t c[3] = {z, y, x}, lo[3] = {z, y, x}, hi[3] = {z, y, x};
        int64_t len = d[axis], k = c[axis], e = 1;
        if (len == 1) {
          D[(z * d[1] + y) * d[2] + x] = 0;
          continue;
        }
        if (k == 0) {
          hi[axis] = 1;
          e = 2;
        } else if (k == len - 1) {
          lo[axis] = k - 1;
          e = 2;
        } else {
          lo[axis] = k - 1;
          hi[axis] = k + 1;
        }
        int64_t v = xnd_p(dp, d, hi) - xnd_p(dp, d, lo);
        if (nd_box_of(d, bd, hi[0], hi[1], hi[2]) != nd_box_of(d, bd, lo[0], lo[1], lo[2]))
          v += xnd_m(M, d, bd, hi) - xnd_m(M, d, bd, lo); /* border: the box means' difference */
        D[(z * d[1] + y) * d[2] + x] = v * e;
      }
  return ORC_OK;
}

/* Stage 2 Laplacian numerators of HSZx-nd (Section V-B, HSZx-2d: the
 * neighbours' p minus 2 ndim p, corrected at box borders by the neighbour
 * box's mean minus the centre box's), with replicated edges: a missing
 * neighbour repeats the centre (its term is 0). */
int orc_xnd_lap_p(const int32_t *dp, const int32_t *M, const int64_t *dims3, const int64_t *bd, int64_t *L) {
  const int64_t *d = dims3;
  for (int64_t z = 0; z < d[0]; z++)
    for (int64_t y = 0; y < d[1]; y++)
      for (int64_t x = 0; x < d[2]; x++) {
        int64_t c[3] = {z, y, x};
        int64_t pc = xnd_p(dp, d, c), mc = xnd_m(M, d, bd, c), v = 0;
        for (int a = 0; a < 3; a++)
          for (int sgn = -1; sgn <= 1; sgn += 2) {
            int64_t nb[3] = {z, y, x};
            nb[a] += sgn;
            if (nb[a] < 0 || nb[a] >= d[a]) continue; /* replicated edge: term 0 */
            v += xnd_p(dp, d, nb) - pc;
            if (nd_box_of(d, bd, nb[0], nb[1], nb[2]) != nd_box_of(d, bd, z, y, x)) v += xnd_m(M, d, bd, nb) - mc;
          }
        L[(z * d[1] + y) * d[2] + x] = v;
      }
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Numerical differentiation on codes (Section V-B, "Operation with      */
/* D_q"): integer numerators, scaled at the end.                         */
/*   derivative  (d_{i+1} - d_{i-1}) / 2 = eps (q_{i+1} - q_{i-1})       */
/*   Laplacian   sum of the 2*ndim neighbours - 2*ndim*d = 2 eps L        */
/* Readings (the paper is silent on edges): one-sided differences at the  */
/* domain edge,                                                           */
/* D = 2 (q_1 - q_0) (numpy.gradient, edge_order=1); an axis of length 1  */
/* has D = 0; the Laplacian replicates the edge value (mode 'nearest').   */
/* Shapes are (n0, n1, n2) row-major, n2 fastest; a field of ndim < 3 has */
/* leading axes of length 1.                                              */
/* ------------------------------------------------------------------ */
static int64_t idx3(const int64_t *d, int64_t i0, int64_t i1, int64_t i2) {
  return (i0 * d[1] + i1) * d[2] + i2;
}

static int64_t deriv_num(const int32_t *q, const int64_t *d, int64_t i0, int64_t i1, int64_t i2,
                         int axis) {
  int64_t c[3] = {i0, i1, i2};
  int64_t na = d[axis];
  if (na < 2) return 0;
  int64_t lo[3] = {i0, i1, i2}, hi[3] = {i0, i1, i2};
  if (c[axis] == 0) {
    hi[axis] = 1;
    return 2 * ((int64_t)q[idx3(d, hi[0], hi[1], hi[2])] - q[idx3(d, i0, i1, i2)]);
  }
  if (c[axis] == na - 1) {
    lo[axis] = na - 2;
    return 2 * ((int64_t)q[idx3(d, i0, i1, i2)] - q[idx3(d, lo[0], lo[1], lo[2])]);
  }
  lo[axis] = c[axis] - 1;
  hi[axis] = c[axis] + 1;
  return (int64_t)q[idx3(d, hi[0], hi[1], hi[2])] - q[idx3(d, lo[0], lo[1], lo[2])];
}

/* integer derivative numerators D along internal axis (0, 1 or 2) */
int orc_deriv_q(const int32_t *q, const int64_t *dims3, int axis, int64_t *D) {
  if (axis < 0 || axis > 2) return ORC_ERR_INVALID_ARG;
  for (int64_t i0 = 0; i0 < dims3[0]; i0++)
    for (int64_t i1 = 0; i1 < dims3[1]; i1++)
      for (int64_t i2 = 0; i2 < dims3[2]; i2++)
        D[idx3(dims3, i0, i1, i2)] = deriv_num(q, dims3, i0, i1, i2, axis);
  return ORC_OK;
}

/* Divergence of a vector field (Section V-C, "Multivariate Derivation",
 * Eq. divergence on D_q): component c differentiated along internal axis
 * axes[c] with the derivative numerators above; num = sum_c D_c.  The value
 * is num * eps when every component has the same eps (the paper's form);
 * otherwise (reading: components quantized with different bounds) each term
 * carries its own eps, sum_c eps_c D_c in component order. */
int orc_divergence_q(const int32_t *const *q, int ncomp, const int64_t *d, const int *axes, const double *eps,
                     int64_t *num, double *val) {
  if (ncomp < 1 || ncomp > 3) return ORC_ERR_INVALID_ARG;
  int same = 1;
  for (int c = 1; c < ncomp; c++) same &= eps[c] == eps[0];
  for (int64_t i0 = 0; i0 < d[0]; i0++)
    for (int64_t i1 = 0; i1 < d[1]; i1++)
      for (int64_t i2 = 0; i2 < d[2]; i2++) {
        int64_t n = 0;
        double v = 0.0;
        for (int c = 0; c < ncomp; c++) {
          int64_t D = deriv_num(q[c], d, i0, i1, i2, axes[c]);
          n += D;
          v += (double)D * eps[c];
        }
        num[idx3(d, i0, i1, i2)] = n;
        val[idx3(d, i0, i1, i2)] = same ? (double)n * eps[0] : v;
      }
  return ORC_OK;
}

/* Curl of a 2-D field F = (u, v) (Section V-C, Eq. curl on D_q): with i the
 * first and j the second index, (q^u_{i,j+1} - q^u_{i,j-1}) - (q^v_{i+1,j} -
 * q^v_{i-1,j}), times eps; axis_i / axis_j are the internal axes of i and j.
 * The same edge rule and the same reading for different bounds as the
 * divergence. */
int orc_curl2_q(const int32_t *qu, const int32_t *qv, const int64_t *d, int axis_i, int axis_j, double eps_u,
                double eps_v, int64_t *num, double *val) {
  for (int64_t i0 = 0; i0 < d[0]; i0++)
    for (int64_t i1 = 0; i1 < d[1]; i1++)
      for (int64_t i2 = 0; i2 < d[2]; i2++) {
        int64_t du = deriv_num(qu, d, i0, i1, i2, axis_j);
        int64_t dv = deriv_num(qv, d, i0, i1, i2, axis_i);
        num[idx3(d, i0, i1, i2)] = du - dv;
        val[idx3(d, i0, i1, i2)] = eps_u == eps_v ? (double)(du - dv) * eps_u : (double)du * eps_u - (double)dv * eps_v;
      }
  return ORC_OK;
}

/* integer Laplacian numerator at one point (replicated edges) */
static int64_t lap_num(const int32_t *q, const int64_t *d, int64_t i0, int64_t i1, int64_t i2) {
  int64_t c[3] = {i0, i1, i2};
  int64_t center = q[idx3(d, i0, i1, i2)];
  int64_t acc = 0;
  for (int a = 0; a < 3; a++) {
    int64_t m[3] = {i0, i1, i2}, p[3] = {i0, i1, i2};
    m[a] = c[a] > 0 ? c[a] - 1 : 0;
    p[a] = c[a] < d[a] - 1 ? c[a] + 1 : d[a] - 1;
    acc += (int64_t)q[idx3(d, m[0], m[1], m[2])] + q[idx3(d, p[0], p[1], p[2])] - 2 * center;
  }
  return acc;
}

/* integer Laplacian numerators L */
int orc_lap_q(const int32_t *q, const int64_t *d, int64_t *L) {
  for (int64_t i0 = 0; i0 < d[0]; i0++)
    for (int64_t i1 = 0; i1 < d[1]; i1++)
      for (int64_t i2 = 0; i2 < d[2]; i2++) L[idx3(d, i0, i1, i2)] = lap_num(q, d, i0, i1, i2);
  return ORC_OK;
}

/* The same numerators and scaled values at m flat indices only (sampled
 * checks of fields too large to evaluate whole):
 *   kind 0: num = D along axis, val = eps * D
 *   kind 1: num = 0,            val = eps * sqrt(sum_a D_a^2)
 *   kind 2: num = L,            val = 2 eps * L */
int orc_stencil_at(const int32_t *q, const int64_t *d, int kind, int axis, double eps, const int64_t *idx,
                   int64_t m, int64_t *num, double *val) {
  if (kind < 0 || kind > 2 || axis < 0 || axis > 2) return ORC_ERR_INVALID_ARG;
  for (int64_t k = 0; k < m; k++) {
    int64_t i = idx[k];
    if (i < 0 || i >= d[0] * d[1] * d[2]) return ORC_ERR_INVALID_ARG;
    int64_t i2 = i % d[2], i1 = (i / d[2]) % d[1], i0 = i / (d[1] * d[2]);
    if (kind == 0) {
      num[k] = deriv_num(q, d, i0, i1, i2, axis);
      val[k] = (double)num[k] * eps;
    } else if (kind == 1) {
      u128 acc = 0;
      for (int a = 0; a < 3; a++) {
        int64_t t = deriv_num(q, d, i0, i1, i2, a);
        uint64_t u = (uint64_t)(t < 0 ? -t : t);
        acc += (u128)u * u;
      }
      num[k] = 0;
      val[k] = sqrt((double)acc) * eps;
    } else {
      num[k] = lap_num(q, d, i0, i1, i2);
      val[k] = (double)num[k] * (2.0 * eps);
    }
  }
  return ORC_OK;
}

/* scaled values of the homomorphic results, in double:
 *   kind 0: derivative along axis -> eps * D
 *   kind 1: gradient magnitude   -> eps * sqrt(sum_a D_a^2)
 *   kind 2: Laplacian            -> 2 eps * L */
int orc_stencil_q(const int32_t *q, const int64_t *d, int kind, int axis, double eps, double *out) {
  int64_t n = d[0] * d[1] * d[2];
  int64_t *t = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  if (!t) return ORC_ERR_INVALID_ARG;
  int st = ORC_OK;
  if (kind == 0) {
    st = orc_deriv_q(q, d, axis, t);
    for (int64_t i = 0; i < n && !st; i++) out[i] = (double)t[i] * eps;
  } else if (kind == 1) {
    for (int64_t i = 0; i < n; i++) out[i] = 0.0;
    u128 *acc = (u128 *)calloc((size_t)n, sizeof(u128));
    if (!acc) {
      free(t);
      return ORC_ERR_INVALID_ARG;
    }
    for (int a = 0; a < 3; a++) {
      orc_deriv_q(q, d, a, t);
      for (int64_t i = 0; i < n; i++) {
        uint64_t m = (uint64_t)(t[i] < 0 ? -t[i] : t[i]);
        acc[i] += (u128)m * m;
      }
    }
    for (int64_t i = 0; i < n; i++) out[i] = sqrt((double)acc[i]) * eps;
    free(acc);
  } else if (kind == 2) {
    orc_lap_q(q, d, t);
    for (int64_t i = 0; i < n; i++) out[i] = (double)t[i] * (2.0 * eps);
  } else {
    st = ORC_ERR_INVALID_ARG;
  }
  free(t);
  return st;
}

/* Generic flow on D_f (Eq. derivatives and Eq. laplacian written for any
 * number of axes), in double: the "full decompression, then operate" result. */
int orc_stencil_f(const void *f, int dtype, const int64_t *d, int kind, int axis, double *out) {
  if (kind < 0 || kind > 2 || axis < 0 || axis > 2) return ORC_ERR_INVALID_ARG;
  for (int64_t i0 = 0; i0 < d[0]; i0++)
    for (int64_t i1 = 0; i1 < d[1]; i1++)
      for (int64_t i2 = 0; i2 < d[2]; i2++) {
        int64_t c[3] = {i0, i1, i2};
        double center = load_x(f, dtype, idx3(d, i0, i1, i2));
        double g[3];
        double lap = 0.0;
        for (int a = 0; a < 3; a++) {
          int64_t m[3] = {i0, i1, i2}, p[3] = {i0, i1, i2};
          m[a] = c[a] > 0 ? c[a] - 1 : 0;
          p[a] = c[a] < d[a] - 1 ? c[a] + 1 : d[a] - 1;
          double vm = load_x(f, dtype, idx3(d, m[0], m[1], m[2]));
          double vp = load_x(f, dtype, idx3(d, p[0], p[1], p[2]));
          lap += vm + vp - 2.0 * center;
          if (d[a] < 2)
            g[a] = 0.0;
          else if (c[a] == 0 || c[a] == d[a] - 1)
            g[a] = vp - vm; /* one-sided: neighbours are (c, c+1) or (c-1, c) */
          else
            g[a] = (vp - vm) / 2.0;
        }
        double r;
        if (kind == 0)
          r = g[axis];
        else if (kind == 1)
          r = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
        else
          r = lap;
        out[idx3(d, i0, i1, i2)] = r;
      }
  return ORC_OK;
}
