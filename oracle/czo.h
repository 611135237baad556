/*
 * czo.h -- CPU oracle for the CubismZ stage-1 wavelet codec (test infrastructure).
 *
 * This is a plain, slow, sequential C implementation of what the GPU path
 * computes.  It exists only to check the GPU library: the test-suite, the
 * smoke check and the benchmark's CPU-baseline leg are its only callers.  It
 * shares no code, header, table or constant with the CUDA library and it is
 * never linked into it.
 *
 * Arithmetic is done in the field's own precision T (float or double), which
 * the paper makes a compile-time option of the codec ("precision (float,
 * double)", program summary).  Every sum is evaluated left to right exactly as
 * written in the comments of czo_real.inc; the file must be built with
 * -ffp-contract=off so that no multiply-add is fused.
 *
 * Readings of the paper used here (the paper names the wavelets, Sec. 2.3
 * "Wavelet types", and cites Donoho 1992 and Cohen-Daubechies-Vial 1993, but
 * prints no filter, boundary rule, level count or stream layout):
 *   - W4    : interpolating wavelet, 4-point Lagrange (Deslauriers-Dubuc)
 *             prediction, one-sided stencils on the interval.
 *   - W4li  : W4 prediction followed by a lifting update that gives every
 *             synthesis wavelet two vanishing moments (interior weight 1/4).
 *   - W3ai  : average-interpolating wavelet: quadratic matching three coarse
 *             cell averages.
 *   - full dyadic decomposition of a B^3 block down to a 4^3 coarse cube,
 *     axes x then y then z at every level.
 *   - keep a detail iff !(|d| < t), t = eps * (max - min) of the whole field.
 *   - stream: header, (nblocks+1) u64 chunk offsets, one chunk per block;
 *     optional stage 2 = byte shuffle + zero run-length coding per chunk.
 *   - aggregate chunks (Sec. 3, Exp. 2 and 3: the stage-1 output of several
 *     blocks is concatenated and the buffer coded by the lossless substage
 *     as one stream): with a group flag, G consecutive blocks (x-fastest
 *     block order; the last group may hold fewer) share one chunk and one
 *     table entry.  The chunk is [nnz of each block | ntok | tokens |
 *     literals] over the byte shuffle of the concatenated payloads.
 */
#ifndef CZO_H
#define CZO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { CZO_W4 = 0, CZO_W4LI = 1, CZO_W3AI = 2 };
enum { CZO_F32 = 0, CZO_F64 = 1 };
enum { CZO_EPS_REL = 0, CZO_EPS_ABS = 1 };
enum { CZO_BOUND_PAPER = 0, CZO_BOUND_STRICT = 1 };

/* return codes (mirrors the numeric meaning of the library's codes) */
enum {
  CZO_OK = 0,
  CZO_ERR_ARG = -1,
  CZO_ERR_CAPACITY = -2,
  CZO_ERR_CORRUPT = -3
};

#define CZO_HEADER_BYTES 128
/* bit zeroing (Sec. 3, Exp. 2): the 4 / 8 least significant bits of every
 * kept detail coefficient are cleared before the lossless substage */
enum { CZO_FLAG_ZERO4 = 2, CZO_FLAG_ZERO8 = 4 };
/* aggregate chunks (Sec. 3, Exp. 2): a two-bit field, G = 2 << code
 * consecutive blocks per chunk (code 0: one chunk per block); stage 2 only */
enum { CZO_FLAG_GROUP4 = 8, CZO_FLAG_GROUP8 = 16, CZO_FLAG_GROUP16 = 24, CZO_GROUP_MASK = 24 };
#define CZO_MAGIC 0x315A4343u /* bytes "CCZ1" */
#define CZO_ZMIN_WORDS 2      /* shortest zero run coded as a run (32-bit words) */

typedef struct czo_params {
  int32_t nx, ny, nz; /* field dims in elements, C order [nz][ny][nx]        */
  int32_t block;      /* cubic block edge B: 8, 16, 32 or 64                   */
  int32_t dtype;      /* CZO_F32 / CZO_F64                                     */
  int32_t kind;       /* CZO_W4 / CZO_W4LI / CZO_W3AI                          */
  int32_t eps_mode;   /* CZO_EPS_REL: t = eps*range ; CZO_EPS_ABS: t = eps     */
  int32_t stage2;     /* 1: byte shuffle + zero-RLE per chunk                  */
  int32_t bound_mode; /* CZO_BOUND_PAPER: threshold t ; CZO_BOUND_STRICT:
                         threshold t / C (see czo_synthesis_norm)             */
  int32_t flags;      /* CZO_FLAG_ZERO4 / CZO_FLAG_ZERO8: bit zeroing of the
                         kept details; CZO_FLAG_GROUP*: aggregate chunks;
                         other bits (library build options) are ignored      */
  double eps;
  double range;       /* >= 0: use this range ; < 0: compute max - min         */
} czo_params;

/* ---- one level of the 1D transform, in place, interleaved (coarse at even
 *      local index, detail at odd); n = 2m samples spaced by `stride`, m >= 4 */
int czo_fwd1d_f32(int kind, float *f, int n, ptrdiff_t stride);
int czo_inv1d_f32(int kind, float *f, int n, ptrdiff_t stride);
int czo_fwd1d_f64(int kind, double *f, int n, ptrdiff_t stride);
int czo_inv1d_f64(int kind, double *f, int n, ptrdiff_t stride);

/* ---- full dyadic 3D transform of one B^3 block (x fastest), in place ---- */
int czo_fwd3d_f32(int kind, float *blk, int B);
int czo_inv3d_f32(int kind, float *blk, int B);
int czo_fwd3d_f64(int kind, double *blk, int B);
int czo_inv3d_f64(int kind, double *blk, int B);

/* ---- one block: raw values -> chunk bytes (returns length or < 0) ------- */
int64_t czo_encode_block_f32(int kind, int B, float t, int stage2,
                             const float *blk, uint8_t *out, size_t cap);
int64_t czo_encode_block_f64(int kind, int B, double t, int stage2,
                             const double *blk, uint8_t *out, size_t cap);
/* the same with the zbits (0, 4 or 8) least significant bits of every kept
 * detail cleared */
int64_t czo_encode_block_z_f32(int kind, int B, float t, int stage2, int zbits,
                               const float *blk, uint8_t *out, size_t cap);
int64_t czo_encode_block_z_f64(int kind, int B, double t, int stage2, int zbits,
                               const double *blk, uint8_t *out, size_t cap);
/* chunk bytes -> reconstructed block values */
int czo_decode_block_f32(int kind, int B, int stage2, const uint8_t *chunk,
                         size_t n, float *blk);
int czo_decode_block_f64(int kind, int B, int stage2, const uint8_t *chunk,
                         size_t n, double *blk);

/* ---- whole field <-> stream ---------------------------------------------- */
int czo_compress_bound(const czo_params *p, size_t *bytes);
int czo_compress(const czo_params *p, const void *field, uint8_t *out,
                 size_t cap, size_t *out_bytes);
int czo_decompress(const uint8_t *in, size_t n, void *field, size_t field_cap);
/* header fields as plain values; returns 0 or < 0 */
int czo_read_header(const uint8_t *in, size_t n, czo_params *p,
                    double *t, double *mn, double *mx, uint64_t *total);

/* ---- a0: min / max ignoring NaN (both +inf/-inf if nothing counted) ----- */
void czo_minmax_f32(const float *x, size_t n, double *mn, double *mx);
void czo_minmax_f64(const double *x, size_t n, double *mn, double *mx);
/* threshold t = eps*range (REL) or eps (ABS), formed in double */
double czo_threshold(double eps, int eps_mode, double range);

/* C = max over the positions i of a B^3 block of sum_j |S_ij| over the
 * detail columns j of the block synthesis operator S (decoder = S applied to
 * the kept coefficients).  Dropping details smaller than t / C therefore
 * changes no value by more than t (the bound Sec. 2.3 states for the
 * threshold).  Computed from the 1D level syntheses: a level-l detail is
 * rebuilt by the syntheses of levels l..0 only, whose composition is the
 * Kronecker cube of a B x (B >> l) matrix m_l, so its columns' row sums
 * are products of the 1D row sums R_l (all columns) and E_l (even columns,
 * which are coarse values, not details):
 *   C = max_i sum_l ( R_l(ix) R_l(iy) R_l(iz) - E_l(ix) E_l(iy) E_l(iz) ).
 * Returns a negative value for an unsupported (kind, B). */
double czo_synthesis_norm(int kind, int B);

/* blocks per chunk of a flags word: 1, 4, 8 or 16 */
int czo_group_blocks(int32_t flags);

/* ---- stage 2 primitives ---------------------------------------------------- */
void czo_shuffle(const uint8_t *in, size_t nbytes, int s, uint8_t *out);
void czo_unshuffle(const uint8_t *in, size_t nbytes, int s, uint8_t *out);
/* zero-RLE over 32-bit words (n a multiple of 4): tokens (u32 = literal words
 * | zero words << 16) then the literal words.  *nlit is in bytes.  Returns
 * bytes of tokens + literals, or < 0.                                         */
int64_t czo_rle_encode(const uint8_t *in, size_t n, uint32_t *tokens,
                       size_t tok_cap, size_t *ntok, uint8_t *lits,
                       size_t lit_cap, size_t *nlit);
int czo_rle_decode(const uint32_t *tokens, size_t ntok, const uint8_t *lits,
                   size_t nlit, uint8_t *out, size_t n);

/* ---- metrics (Sec. 3: CR includes metadata; PSNR has the factor 2) ------ */
double czo_psnr_f32(const float *R, const float *D, size_t n);
double czo_psnr_f64(const double *R, const double *D, size_t n);
double czo_linf_f32(const float *R, const float *D, size_t n);
double czo_linf_f64(const double *R, const double *D, size_t n);

/* ---- lifting-update weight of detail k on coarse node j (level with m
 *      coarse values); returns 0 and the exact fraction num/den, or -1 if d_k
 *      does not update node j.                                               */
int czo_update_weight(int m, int k, int j, int64_t *num, int64_t *den);

#ifdef __cplusplus
}
#endif
#endif
