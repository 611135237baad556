/*
 * czo.c -- CPU oracle for the CubismZ stage-1 wavelet codec.
 *
 * TEST INFRASTRUCTURE ONLY: called by the tests, the smoke check and the
 * benchmark's CPU-baseline leg; never by the GPU library.  Build with
 * -ffp-contract=off (no fused multiply-add).  See czo.h for the readings of
 * the paper that this file fixes.
 */
#include "czo.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define CAT2(a, b) a##b
#define CAT(a, b) CAT2(a, b)

static void czo_write_header(uint8_t *out, const czo_params *p, double t,
                             double mn, double mx, double range,
                             uint64_t data_bytes, uint64_t total);

/* --------------------------------------------------------------------------
 * W4 prediction rows as integers (Lagrange weights x 16).  Coarse nodes
 * j0..j0+3, odd sample at x = k + 1/2 in coarse units.  See czo_real.inc.
 * -------------------------------------------------------------------------- */
static void w4_row(int k, int m, int *j0, int w[4])
{
  static const int LEFT[4] = {5, 15, -5, 1};
  static const int MID[4] = {-1, 9, 9, -1};
  static const int RIGHT[4] = {1, -5, 15, 5};
  static const int EXTRAP[4] = {-5, 21, -35, 35};
  const int *r;
  if (k == 0) {
    r = LEFT;
    *j0 = 0;
  } else if (k <= m - 3) {
    r = MID;
    *j0 = k - 1;
  } else if (k == m - 2) {
    r = RIGHT;
    *j0 = m - 4;
  } else {
    r = EXTRAP;
    *j0 = m - 4;
  }
  for (int q = 0; q < 4; ++q) w[q] = r[q];
}

static int64_t gcd64(int64_t a, int64_t b)
{
  if (a < 0) a = -a;
  if (b < 0) b = -b;
  while (b) {
    int64_t t = a % b;
    a = b;
    b = t;
  }
  return a;
}

/* --------------------------------------------------------------------------
 * W4li update weights: the lifting scheme on the interval.
 *
 * The synthesis wavelet of detail k is psi_k = delta_{2k+1} - sum_j U_jk phi_j,
 * where phi_j is the predict-only synthesis scaling function of coarse node j
 * (1 at fine position 2j, the prediction weights of column j at the odd
 * positions).  The update gives psi_k two vanishing moments,
 *     sum_j U_jk M_j^p = (2k+1)^p,   p = 0, 1,   M_j^p = moment p of phi_j,
 * with the two coarse nodes nearest to the detail as its support: (k, k+1),
 * or (m-2, m-1) for the last detail, which lies past the last coarse node.
 * In the interior this gives the familiar U = 1/4 on both neighbours.  The
 * 2x2 system is solved exactly (Cramer's rule on integers, moments scaled
 * by 16).
 * -------------------------------------------------------------------------- */
int czo_update_weight(int m, int k, int j, int64_t *num, int64_t *den)
{
  if (m < 4 || m > 64 || k < 0 || k >= m || j < 0 || j >= m) return -1;
  int a = (k <= m - 2) ? k : m - 2;
  int b = a + 1;
  if (j != a && j != b) return -1;
  /* 16 * M_j^0 and 16 * M_j^1 for the two support nodes */
  int64_t A0[2] = {16, 16}, A1[2] = {16 * 2 * (int64_t)a, 16 * 2 * (int64_t)b};
  for (int r = 0; r < m; ++r) {
    int j0, w[4];
    w4_row(r, m, &j0, w);
    for (int q = 0; q < 4; ++q) {
      int col = j0 + q;
      for (int t = 0; t < 2; ++t)
        if (col == (t == 0 ? a : b)) {
          A0[t] += w[q];
          A1[t] += (int64_t)w[q] * (2 * r + 1);
        }
    }
  }
  int64_t rhs0 = 16, rhs1 = 16 * (int64_t)(2 * k + 1);
  int64_t det = A0[0] * A1[1] - A0[1] * A1[0];
  if (det == 0) return -1;
  int64_t n = (j == a) ? (rhs0 * A1[1] - A0[1] * rhs1) : (A0[0] * rhs1 - A1[0] * rhs0);
  int64_t d = det;
  if (d < 0) {
    d = -d;
    n = -n;
  }
  int64_t g = gcd64(n, d);
  if (g == 0) g = 1;
  *num = n / g;
  *den = d / g;
  return 0;
}

double czo_threshold(double eps, int eps_mode, double range)
{
  return eps_mode == CZO_EPS_ABS ? eps : eps * range;
}

/* see czo.h; every sum runs in increasing index order, in double */
double czo_synthesis_norm(int kind, int B)
{
  enum { MAXB = 64, MAXL = 4 };
  if (B < 8 || B > MAXB || (B & (B - 1))) return -1.0;
  int L = 0;
  while ((B >> L) > 4) ++L;
  if (L > MAXL) return -1.0;
  double R[MAXL][MAXB], E[MAXL][MAXB];
  for (int l = 0; l < L; ++l) {
    const int nl = B >> l;
    for (int x = 0; x < B; ++x) R[l][x] = E[l][x] = 0.0;
    for (int j = 0; j < nl; ++j) {
      /* column j of m_l: unit coefficient at local index j of level l,
         synthesised level by level down to the B fine samples */
      double w[MAXB] = {0};
      w[j] = 1.0;
      for (int k = l; k >= 0; --k) {
        const int nk = B >> k;
        if (czo_inv1d_f64(kind, w, nk, 1) != CZO_OK) return -1.0;
        if (k > 0) {
          double u[MAXB] = {0};
          for (int i = 0; i < nk; ++i) u[2 * i] = w[i];
          for (int i = 0; i < 2 * nk; ++i) w[i] = u[i];
        }
      }
      for (int x = 0; x < B; ++x) {
        const double a = fabs(w[x]);
        R[l][x] += a;
        if (!(j & 1)) E[l][x] += a;
      }
    }
  }
  double C = 0.0;
  for (int iz = 0; iz < B; ++iz)
    for (int iy = 0; iy < B; ++iy)
      for (int ix = 0; ix < B; ++ix) {
        double s = 0.0;
        for (int l = 0; l < L; ++l) s += (R[l][ix] * R[l][iy]) * R[l][iz] - (E[l][ix] * E[l][iy]) * E[l][iz];
        if (s > C) C = s;
      }
  return C;
}

/* --------------------------------------------------------------------------
 * Stage 2 (Sec. 2.3 "Lossless compression": shuffling of the whole output,
 * coefficients and masks together, with the element size of the data).
 * Shuffle: output plane b (b < s) holds byte b of every s-byte element.
 * -------------------------------------------------------------------------- */
void czo_shuffle(const uint8_t *in, size_t nbytes, int s, uint8_t *out)
{
  size_t E = nbytes / (size_t)s;
  for (size_t e = 0; e < E; ++e)
    for (int b = 0; b < s; ++b) out[(size_t)b * E + e] = in[e * (size_t)s + b];
  for (size_t q = E * (size_t)s; q < nbytes; ++q) out[q] = in[q]; /* tail */
}

void czo_unshuffle(const uint8_t *in, size_t nbytes, int s, uint8_t *out)
{
  size_t E = nbytes / (size_t)s;
  for (size_t e = 0; e < E; ++e)
    for (int b = 0; b < s; ++b) out[e * (size_t)s + b] = in[(size_t)b * E + e];
  for (size_t q = E * (size_t)s; q < nbytes; ++q) out[q] = in[q];
}

/* --------------------------------------------------------------------------
 * Zero run-length coding of the shuffled payload, in 32-bit words (the
 * payload is a whole number of words).  The word sequence is cut into pairs
 *   (literal run, zero run)
 * where every zero run is a maximal run of at least CZO_ZMIN_WORDS zero
 * words and the literal run is everything between it and the previous such
 * run; a final pair with zero run 0 carries trailing literals.  Each pair is
 * one token (u32: literal words in the low 16 bits, zero words in the high
 * 16 bits); a literal run longer than 65535 words first emits (65535, 0)
 * tokens, a zero run longer than 65535 emits (lit, 65535) and then
 * (0, rest).  The literal words follow the tokens.
 * -------------------------------------------------------------------------- */
static int emit_pair(size_t lit, size_t zr, uint32_t *tok, size_t cap, size_t *nt)
{
  while (lit > 65535) {
    if (*nt >= cap) return CZO_ERR_CAPACITY;
    tok[(*nt)++] = 65535u;
    lit -= 65535;
  }
  while (zr > 65535) {
    if (*nt >= cap) return CZO_ERR_CAPACITY;
    tok[(*nt)++] = (uint32_t)lit | (65535u << 16);
    lit = 0;
    zr -= 65535;
  }
  if (*nt >= cap) return CZO_ERR_CAPACITY;
  tok[(*nt)++] = (uint32_t)lit | ((uint32_t)zr << 16);
  return CZO_OK;
}

static uint32_t word_at(const uint8_t *in, size_t w)
{
  uint32_t v;
  memcpy(&v, in + 4 * w, 4);
  return v;
}

int64_t czo_rle_encode(const uint8_t *in, size_t n, uint32_t *tokens,
                       size_t tok_cap, size_t *ntok, uint8_t *lits,
                       size_t lit_cap, size_t *nlit)
{
  if (n % 4 != 0) return CZO_ERR_ARG;
  const size_t W = n / 4;
  size_t nt = 0, nl = 0, lit_start = 0, i = 0;
  while (i < W) {
    if (word_at(in, i) != 0) {
      ++i;
      continue;
    }
    size_t j = i;
    while (j < W && word_at(in, j) == 0) ++j;
    if (j - i >= CZO_ZMIN_WORDS) {
      size_t lit = i - lit_start;
      if (4 * (nl + lit) > lit_cap) return CZO_ERR_CAPACITY;
      memcpy(lits + 4 * nl, in + 4 * lit_start, 4 * lit);
      nl += lit;
      int r = emit_pair(lit, j - i, tokens, tok_cap, &nt);
      if (r) return r;
      lit_start = j;
    }
    i = j;
  }
  if (lit_start < W) {
    size_t lit = W - lit_start;
    if (4 * (nl + lit) > lit_cap) return CZO_ERR_CAPACITY;
    memcpy(lits + 4 * nl, in + 4 * lit_start, 4 * lit);
    nl += lit;
    int r = emit_pair(lit, 0, tokens, tok_cap, &nt);
    if (r) return r;
  }
  *ntok = nt;
  *nlit = 4 * nl;
  return (int64_t)(4 * nt + 4 * nl);
}

/* nlit and n in bytes (multiples of 4); token counts in words */
int czo_rle_decode(const uint32_t *tokens, size_t ntok, const uint8_t *lits,
                   size_t nlit, uint8_t *out, size_t n)
{
  if (n % 4 != 0) return CZO_ERR_CORRUPT;
  const size_t W = n / 4, NL = nlit / 4;
  size_t o = 0, l = 0;
  for (size_t q = 0; q < ntok; ++q) {
    size_t lit = tokens[q] & 0xFFFFu, zr = tokens[q] >> 16;
    if (l + lit > NL || o + lit + zr > W) return CZO_ERR_CORRUPT;
    memcpy(out + 4 * o, lits + 4 * l, 4 * lit);
    o += lit;
    l += lit;
    memset(out + 4 * o, 0, 4 * zr);
    o += zr;
  }
  return o == W ? CZO_OK : CZO_ERR_CORRUPT;
}

/* --------------------------------------------------------------------------
 * Stage 2 of one payload: byte shuffle with element size s, then the zero
 * run-length code.  The tokens and then the literal words go to out (cap
 * bytes); *ntok gets the token count.  Returns the bytes written or < 0.
 * -------------------------------------------------------------------------- */
static int64_t stage2_encode(const uint8_t *pay, size_t pbytes, int s, uint8_t *out,
                             size_t cap, uint32_t *ntok)
{
  uint8_t *sh = (uint8_t *)malloc(pbytes + 4);
  size_t tok_cap = pbytes / 4 + 16;
  uint32_t *tok = (uint32_t *)malloc(tok_cap * 4);
  uint8_t *lit = (uint8_t *)malloc(pbytes + 4);
  size_t nt = 0, nl = 0;
  int64_t r = CZO_ERR_ARG;
  if (sh && tok && lit) {
    czo_shuffle(pay, pbytes, s, sh);
    r = czo_rle_encode(sh, pbytes, tok, tok_cap, &nt, lit, pbytes, &nl);
    if (r >= 0) {
      if (4 * nt + nl > cap) {
        r = CZO_ERR_CAPACITY;
      } else {
        memcpy(out, tok, 4 * nt);
        memcpy(out + 4 * nt, lit, nl);
        *ntok = (uint32_t)nt;
        r = (int64_t)(4 * nt + nl);
      }
    }
  }
  free(sh);
  free(tok);
  free(lit);
  return r;
}

/* the inverse: ntok tokens then literal words in the n bytes at in -> the
 * pbytes of the payload */
static int stage2_decode(const uint8_t *in, size_t n, uint32_t ntok, int s, uint8_t *pay,
                         size_t pbytes)
{
  if ((size_t)ntok > n / 4 || n % 4 != 0) return CZO_ERR_CORRUPT;
  uint32_t *tok = (uint32_t *)malloc((size_t)ntok * 4 + 4);
  uint8_t *sh = (uint8_t *)malloc(pbytes + 4);
  int r = CZO_ERR_ARG;
  if (tok && sh) {
    memcpy(tok, in, (size_t)ntok * 4);
    r = czo_rle_decode(tok, ntok, in + (size_t)ntok * 4, n - (size_t)ntok * 4, sh, pbytes);
    if (r == CZO_OK) czo_unshuffle(sh, pbytes, s, pay);
  }
  free(tok);
  free(sh);
  return r;
}

int czo_group_blocks(int32_t flags)
{
  const int code = (flags & CZO_GROUP_MASK) >> 3;
  return code ? 2 << code : 1;
}

/* --------------------------------------------------------------------------
 * Stream header (little-endian, 128 bytes):
 *   0 u32 magic "CCZ1"   4 u16 version=1   6 u16 header bytes=128
 *   8 i32 nx  12 i32 ny  16 i32 nz
 *  20 u8 B  21 u8 dtype  22 u8 kind  23 u8 stage2  24 u8 eps_mode  25 u8 L
 *  26 u8 bound_mode  27 u8 flags (bit zeroing, group code)  28 u32 nblocks
 *  32 f64 eps  40 f64 t (threshold as used, widened)  48 f64 min  56 f64 max
 *  64 f64 range  72 u64 chunk-section bytes  80 u64 total stream bytes
 * Then (nchunks+1) u64 chunk offsets relative to the chunk section, which
 * starts at the next multiple of 16 bytes; nchunks = ceil(nblocks / G) with
 * G blocks per chunk (1 unless a group flag is set).
 * -------------------------------------------------------------------------- */
static void czo_write_header(uint8_t *out, const czo_params *p, double t,
                             double mn, double mx, double range,
                             uint64_t data_bytes, uint64_t total)
{
  uint32_t magic = CZO_MAGIC;
  uint16_t ver = 1, hb = CZO_HEADER_BYTES;
  int L = 0;
  while ((p->block >> L) > 4) ++L;
  uint32_t nb = (uint32_t)((p->nx / p->block) * (p->ny / p->block) * (p->nz / p->block));
  memset(out, 0, CZO_HEADER_BYTES);
  memcpy(out + 0, &magic, 4);
  memcpy(out + 4, &ver, 2);
  memcpy(out + 6, &hb, 2);
  memcpy(out + 8, &p->nx, 4);
  memcpy(out + 12, &p->ny, 4);
  memcpy(out + 16, &p->nz, 4);
  out[20] = (uint8_t)p->block;
  out[21] = (uint8_t)p->dtype;
  out[22] = (uint8_t)p->kind;
  out[23] = (uint8_t)p->stage2;
  out[24] = (uint8_t)p->eps_mode;
  out[25] = (uint8_t)L;
  out[26] = (uint8_t)p->bound_mode;
  out[27] = (uint8_t)(p->flags & (CZO_FLAG_ZERO4 | CZO_FLAG_ZERO8 | CZO_GROUP_MASK));
  memcpy(out + 28, &nb, 4);
  memcpy(out + 32, &p->eps, 8);
  memcpy(out + 40, &t, 8);
  memcpy(out + 48, &mn, 8);
  memcpy(out + 56, &mx, 8);
  memcpy(out + 64, &range, 8);
  memcpy(out + 72, &data_bytes, 8);
  memcpy(out + 80, &total, 8);
}

int czo_read_header(const uint8_t *in, size_t n, czo_params *p, double *t,
                    double *mn, double *mx, uint64_t *total)
{
  if (n < CZO_HEADER_BYTES) return CZO_ERR_CORRUPT;
  uint32_t magic;
  uint16_t ver, hb;
  memcpy(&magic, in, 4);
  memcpy(&ver, in + 4, 2);
  memcpy(&hb, in + 6, 2);
  if (magic != CZO_MAGIC || ver != 1 || hb != CZO_HEADER_BYTES) return CZO_ERR_CORRUPT;
  memset(p, 0, sizeof(*p));
  memcpy(&p->nx, in + 8, 4);
  memcpy(&p->ny, in + 12, 4);
  memcpy(&p->nz, in + 16, 4);
  p->block = in[20];
  p->dtype = in[21];
  p->kind = in[22];
  p->stage2 = in[23];
  p->eps_mode = in[24];
  p->bound_mode = in[26];
  p->flags = in[27] & (CZO_FLAG_ZERO4 | CZO_FLAG_ZERO8 | CZO_GROUP_MASK);
  memcpy(&p->eps, in + 32, 8);
  memcpy(t, in + 40, 8);
  memcpy(mn, in + 48, 8);
  memcpy(mx, in + 56, 8);
  memcpy(&p->range, in + 64, 8);
  memcpy(total, in + 80, 8);
  return CZO_OK;
}

/* ---- precision-generic part ---- */
#define T float
#define SFX _f32
#include "czo_real.inc"
#undef T
#undef SFX
#define T double
#define SFX _f64
#include "czo_real.inc"
#undef T
#undef SFX

static int check_params(const czo_params *p)
{
  int B = p->block;
  /* block edges of the paper's block-size study (Sec. 3, Exp. 3) */
  if (B != 8 && B != 16 && B != 32 && B != 64) return CZO_ERR_ARG;
  if (p->nx <= 0 || p->ny <= 0 || p->nz <= 0) return CZO_ERR_ARG;
  if (p->nx % B || p->ny % B || p->nz % B) return CZO_ERR_ARG;
  if (p->dtype != CZO_F32 && p->dtype != CZO_F64) return CZO_ERR_ARG;
  if (p->kind < CZO_W4 || p->kind > CZO_W3AI) return CZO_ERR_ARG;
  if (!(p->eps >= 0)) return CZO_ERR_ARG;
  if (p->bound_mode != CZO_BOUND_PAPER && p->bound_mode != CZO_BOUND_STRICT) return CZO_ERR_ARG;
  /* one zeroing width at most; the strict bound does not cover its error */
  const int z = p->flags & (CZO_FLAG_ZERO4 | CZO_FLAG_ZERO8);
  if (z == (CZO_FLAG_ZERO4 | CZO_FLAG_ZERO8)) return CZO_ERR_ARG;
  if (z && p->bound_mode == CZO_BOUND_STRICT) return CZO_ERR_ARG;
  /* aggregate chunks group the lossless substage's input */
  if ((p->flags & CZO_GROUP_MASK) && !p->stage2) return CZO_ERR_ARG;
  return CZO_OK;
}

int czo_compress_bound(const czo_params *p, size_t *bytes)
{
  if (check_params(p)) return CZO_ERR_ARG;
  size_t B = (size_t)p->block, s = p->dtype == CZO_F64 ? 8 : 4;
  size_t nb = (size_t)(p->nx / p->block) * (p->ny / p->block) * (p->nz / p->block);
  size_t pmax = 64 * s + B * B * B / 8 + (B * B * B - 64) * s;
  size_t chunk = 16 + pmax + 8 * ((pmax / 4 + 65534) / 65535);
  chunk = (chunk + 3) / 4 * 4;
  *bytes = (CZO_HEADER_BYTES + 8 * (nb + 1) + 15) / 16 * 16 + nb * chunk;
  return CZO_OK;
}

int czo_compress(const czo_params *p, const void *field, uint8_t *out,
                 size_t cap, size_t *out_bytes)
{
  if (check_params(p)) return CZO_ERR_ARG;
  if (p->dtype == CZO_F32) return compress_field_f32(p, (const float *)field, out, cap, out_bytes);
  return compress_field_f64(p, (const double *)field, out, cap, out_bytes);
}

int czo_decompress(const uint8_t *in, size_t n, void *field, size_t field_cap)
{
  czo_params p;
  double t, mn, mx;
  uint64_t total;
  int r = czo_read_header(in, n, &p, &t, &mn, &mx, &total);
  if (r) return r;
  if (check_params(&p)) return CZO_ERR_CORRUPT;
  size_t s = p.dtype == CZO_F64 ? 8 : 4;
  if ((size_t)p.nx * p.ny * p.nz * s > field_cap) return CZO_ERR_CAPACITY;
  if (total > n) return CZO_ERR_CORRUPT;
  if (p.dtype == CZO_F32) return decompress_field_f32(&p, in, n, (float *)field);
  return decompress_field_f64(&p, in, n, (double *)field);
}
