// cz_compress.cuh -- compression kernels.
//
// k_stage1 (persistent, static round-robin over blocks; register-resident):
// while the TMA unit fetches the next block's tile, the CTA transforms the
// current block, selects the significant details, and writes the block's
// slot in its own staging arena in global memory:
//   [nnz | 0 | 64 coarse values | mask row words | kept details in position order]
// which is already the finished chunk when stage 2 is off; the block table
// gets (slot offset, chunk bytes).  No CTA waits for another one.
//
// k_stage2 (static grid-stride; only with stage 2): the payload of a slot
// is scattered into byte-shuffled order (byte b of element e at b * E + e;
// element sizes are powers of two, so no division) in shared memory, the
// zero-word runs are found from a ballot bitmap with one block scan, and
// the chunk [nnz | ntok | tokens | literal words] replaces the slot's
// contents.  Small CTAs take the payloads of up to G2::SHCAP bytes, a
// second launch with large CTAs the rest.  With speculative thresholds the
// slots that may hold a detail below the exact threshold are tested too:
// inside a variant of k_stage2 for 32^3 blocks (k_stage2_refine then
// refines those that do), after the others by k_stage2_listed for 8^3 and
// 16^3 blocks (k_spec_list lists them first).
//
// k_place (one CTA per tile of 128 chunks, ticket order): chunk offsets by
// a block scan plus one decoupled look-back per tile, offset-table entries;
// the last tile writes the header.  k_copy (one warp per chunk) moves the
// chunks into the stream.
#pragma once

#include "cz_pair.cuh"

namespace czp {

struct S2Args {
  unsigned char *staging;
  unsigned long long *table;  // per block: slot offset, chunk bytes (~0: lost)
  const void *ws;             // header: count of large payloads (nbig), min / max keys
  const int *biglist;         // ids of the blocks with large payloads
  unsigned char *scratch;     // FP64 32^3: shuffled payloads, one G2::SCRATCH block per large CTA
  int nblocks;
  // speculative thresholds (spec): the stage kernel kept the details with
  // |d| >= t_lo, the threshold of the subsample's range (the header's
  // skmin / skmax), and marked in near[] the blocks that kept one below
  // near_threshold(t_lo); t comes from the final keys.  Slots go to rlist
  // (count in the header's nref): with block edges up to 16 those to test,
  // for k_stage2_listed; with 32 those holding a value below t, for
  // k_stage2_refine.
  int spec;
  const unsigned char *near;
  int *rlist;
  double eps;
  int eps_mode;
};

struct PlaceArgs {
  const unsigned char *staging;
  const unsigned long long *table;
  const unsigned long long *keys;  // batched: min/max keys, two per field
  unsigned long long *lbst;        // batched: look-back words, one per tile
  unsigned char *out;
  unsigned long long *out_bytes;  // may be null
  void *ws;
  unsigned long long out_cap, data0;
  double eps, range, cnorm;
  int nx, ny, nz, nblocks;  // nblocks: chunks (table entries)
  int hdr_nblocks;          // blocks of the field, for the header
  int block, levels, eps_mode, stage2, kind, dtype, bound_mode, flags;
};

// aggregate chunks (cz_group.cuh): the group coders' arguments
struct GroupArgs {
  const unsigned char *staging;       // block slots of the stage kernel: [nnz | 0 | payload]
  const unsigned long long *table;    // per block: slot offset, 8 + payload bytes (TB_LOST: lost)
  unsigned char *gstage;              // group slots, gslot bytes apart
  unsigned long long *gtable;         // per group: slot offset, chunk bytes | TB_FIN (TB_LOST: lost)
  void *ws;                           // header: status, count of the large groups (nbig)
  int *biglist;                       // ids of the large groups
  unsigned char *scratch;             // large groups: one shuffled buffer of hcap bytes per CTA
  unsigned long long gslot;
  int hcap;                           // bytes of the largest group payload (a multiple of 128)
  int nblocks, ngroups, G;
};

constexpr int PLACE_TILE = 128;  // chunks (and threads) per k_place CTA

// block table size words: ~0 = lost (staging overflow); bit 62 set = the
// size of a chunk that stage 2 has finished (so that the other stage-2
// launch, which classifies by size, leaves it alone)
constexpr unsigned long long TB_LOST = 0xFFFFFFFFFFFFFFFFull;
constexpr unsigned long long TB_FIN = 1ull << 62;
constexpr unsigned long long TB_SKIP = 1ull << 61;  // speculative thresholds: left to k_stage2_listed
__device__ __forceinline__ unsigned long long tb_size(unsigned long long cb) { return cb & ~TB_FIN; }

// ---- byte shuffle of payload words into SH: word k of raw (W words) holds
// bytes 0..3 of element e0 + 4k / ES at byte offset 4k % ES, and byte b of
// element e goes to b * E + e (element sizes are powers of two, so no
// division).  A payload that is one piece of a longer buffer (an aggregate
// chunk) passes its first element e0 and the buffer's element count E.
template <typename T, int NT, int OFF = 0>
__device__ __forceinline__ void shuffle_words(const unsigned *raw, int W, int e0, int E, unsigned char *SH)
{
  constexpr int ES = (int)sizeof(T), LGES = ES == 8 ? 3 : 2;
  const int tid = (int)threadIdx.x - OFF;
  for (int k0 = tid; k0 < W; k0 += 4 * NT) {
    unsigned wv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) wv[j] = k0 + j * NT < W ? raw[k0 + j * NT] : 0u;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = k0 + j * NT;
      if (k < W) {
        const int e = e0 + ((4 * k) >> LGES), b0 = (4 * k) & (ES - 1);
#pragma unroll
        for (int q = 0; q < 4; ++q) SH[(b0 + q) * E + e] = (unsigned char)(wv[j] >> (8 * q));
      }
    }
  }
}

// shuffle_words of a whole payload of W words (E elements) that, for
// FP32, also tests the value words from word vw0 on (one value each)
// against t: returns whether this thread met a value with |v| < t (a
// speculative slot to refine).  vw0 >= W tests nothing (FP64 always).
template <typename T, int NT>
__device__ __forceinline__ bool shuffle_check(const unsigned *raw, int W, int E, unsigned char *SH, int vw0, T t)
{
  constexpr int ES = (int)sizeof(T), LGES = ES == 8 ? 3 : 2;
  bool drop = false;
  for (int k0 = threadIdx.x; k0 < W; k0 += 4 * NT) {
    unsigned wv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) wv[j] = k0 + j * NT < W ? raw[k0 + j * NT] : 0u;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = k0 + j * NT;
      if (k < W) {
        if constexpr (ES == 4) {
          if (k >= vw0) drop |= fabsf(__uint_as_float(wv[j])) < (float)t;
        }
        const int e = (4 * k) >> LGES, b0 = (4 * k) & (ES - 1);
#pragma unroll
        for (int q = 0; q < 4; ++q) SH[(b0 + q) * E + e] = (unsigned char)(wv[j] >> (8 * q));
      }
    }
  }
  return drop;
}

// ---- zero-run code of a shuffled payload of pbytes (< 256 KiB: the run
// and word counts are packed in 16-bit halves) in SH: the zero-word runs
// are found from a ballot bitmap with one scan, and [ntok | tokens |
// literal words] are written from ch + 1 on (ch[0] is left alone).  Run by
// the NT threads OFF .. OFF + NT - 1 of a group that synchronises with
// barrier BAR (0: the whole CTA); AUX holds four bitmap arrays of `cap`
// words; s_u (>= 40 words) and s_i (>= 40) are the group's scan scratch.
// Four barriers.  Returns 8 + the bytes of tokens and literals (the same
// in every thread).
template <typename T, int NT, int BAR = 0, int OFF = 0>
__device__ __forceinline__ unsigned stage2_code(unsigned *ch, int pbytes, const unsigned char *SH, unsigned *AUX,
                                                int cap, unsigned *s_u, int *s_i)
{
  constexpr int NWP = NT / 32;
  const int tid = (int)threadIdx.x - OFF, lane = threadIdx.x & 31, wid = tid >> 5;
  const unsigned *SH32 = reinterpret_cast<const unsigned *>(SH);
  const int W = pbytes >> 2, NB = (W + 31) >> 5;
  unsigned *ZBM = AUX, *CM = AUX + cap, *EB = AUX + 2 * cap, *PRE = AUX + 3 * cap;
  for (int g = wid; g < NB; g += NWP) {
    const int w = g * 32 + lane;
    const unsigned bal = __ballot_sync(FULL, w < W && SH32[w] == 0u);
    if (lane == 0) ZBM[g] = bal;
  }
  group_sync<BAR, NT>();
  // coded words C: zero words with a zero neighbour; a run starts at an
  // S bit and ends before an Eb bit (or at W)
  const int KB = (NB + NT - 1) / NT;  // bitmap words per thread (contiguous)
  unsigned mine = 0;
  for (int q = 0; q < KB; ++q) {
    const int g = tid * KB + q;
    if (g < NB) {
      const unsigned Z = ZBM[g];
      const unsigned Zp = g > 0 ? ZBM[g - 1] : 0u, Zn = g + 1 < NB ? ZBM[g + 1] : 0u;
      const unsigned valid = (g == NB - 1 && (W & 31)) ? ((1u << (W & 31)) - 1u) : FULL;
      const unsigned C = Z & ((Z << 1) | (Zp >> 31) | (Z >> 1) | ((Zn & 1u) << 31)) & valid;
      // coded bit of the word before: zero with a zero neighbour
      const unsigned cin = g > 0 ? ((Zp >> 31) & (((Zp >> 30) & 1u) | (Z & 1u))) : 0u;
      CM[g] = C;
      EB[g] = ~C & ((C << 1) | cin) & valid;
      mine += (unsigned)__popc(C & ~((C << 1) | cin)) | ((unsigned)__popc(C) << 16);
    }
  }
  unsigned tot;
  unsigned run = block_exsum_nb<NT, BAR, OFF>(mine, s_u, tot);  // packed: runs | coded words << 16
  for (int q = 0; q < KB; ++q) {
    const int g = tid * KB + q;
    if (g < NB) {
      PRE[g] = run;
      const unsigned C = CM[g];
      const unsigned cin = g > 0 ? (CM[g - 1] >> 31) : 0u;
      run += (unsigned)__popc(C & ~((C << 1) | cin)) | ((unsigned)__popc(C) << 16);
    }
  }
  const unsigned ns_tot = tot & 0xFFFFu, nc_tot = tot >> 16;
  // the last word is coded iff it and the word before it are zero
  const int l = W - 1;
  const unsigned lastc =
      (((ZBM[l >> 5] >> (l & 31)) & 1u) && l > 0 && ((ZBM[(l - 1) >> 5] >> ((l - 1) & 31)) & 1u)) ? 1u : 0u;
  const unsigned ntok = ns_tot + (lastc ? 0u : 1u);
  const unsigned nlit = (unsigned)W - nc_tot;
  unsigned *tok = ch + 2;
  unsigned *lit = tok + ntok;
  // Run ends (Eb bits) around this thread's words: the last one before
  // them (group max-scan, 0 if none -- no run ends at position 0) and the
  // first one after them (group min-scan, W if none).
  int my_last = 0, my_first = W;
  for (int q = 0; q < KB; ++q) {
    const int g = tid * KB + q;
    if (g < NB && EB[g]) {
      my_last = max(my_last, g * 32 + 31 - (int)__clz(EB[g]));
      my_first = min(my_first, g * 32 + __ffs(EB[g]) - 1);
    }
  }
  // (its barrier also orders every thread's PRE words before the literal
  // loop reads them)
  int pe_words, ne_after;
  block_exmax_rexmin_nb<NT, BAR, OFF>(my_last, 0, my_first, W, s_i, pe_words, ne_after);
  // one token per run: (literal words since the previous run, run length);
  // a final (literals, 0) token when the payload does not end in a run
  for (int q = 0; q < KB; ++q) {
    const int g = tid * KB + q;
    if (g >= NB) break;
    const unsigned C = CM[g], Eb = EB[g];
    const unsigned cin = g > 0 ? (CM[g - 1] >> 31) : 0u;
    unsigned S = C & ~((C << 1) | cin);
    unsigned k = PRE[g] & 0xFFFFu;
    while (S) {
      const int b = __ffs(S) - 1;
      S &= S - 1u;
      const int p = g * 32 + b;
      // previous run's end (or 0), this run's end (or W)
      const unsigned below = Eb & ((1u << b) - 1u), above = Eb & ~((2u << b) - 1u);
      const int pe = below ? g * 32 + 31 - (int)__clz(below) : pe_words;
      int ne = ne_after;
      if (above) {
        ne = g * 32 + __ffs(above) - 1;
      } else {
        for (int h = q + 1; h < KB && tid * KB + h < NB; ++h)  // this thread's later words
          if (EB[tid * KB + h]) {
            ne = (tid * KB + h) * 32 + __ffs(EB[tid * KB + h]) - 1;
            break;
          }
      }
      tok[k] = (unsigned)(p - pe) | ((unsigned)(ne - p) << 16);
      if (k + 1 == ns_tot && !lastc) tok[k + 1] = (unsigned)(W - ne);
      ++k;
    }
    if (Eb) pe_words = g * 32 + 31 - (int)__clz(Eb);
  }
  if (tid == 0) {
    if (ns_tot == 0) tok[0] = (unsigned)W;  // no run at all
    ch[1] = ntok;
  }
  for (int w = tid; w < W; w += NT) {
    const int g = w >> 5, b = w & 31;
    const unsigned C = CM[g];
    if (!((C >> b) & 1u)) lit[(unsigned)w - ((PRE[g] >> 16) + __popc(C & ((1u << b) - 1u)))] = SH32[w];
  }
  group_sync<BAR, NT>();
  return 8u + 4u * ntok + 4u * nlit;
}

// ---- speculative thresholds: a slot that kept the details with |d| >=
// t_lo, a lower bound of the threshold t, drops those below t: the value
// list is checked (one barrier); only when some value is dropped are the
// values copied to SH (>= pbytes bytes), the mask bits of the dropped ones
// cleared and the rest moved down in place, and nnz rewritten (six more
// barriers).  The kept set is then exactly {|d| >= t}, the set a pass with
// t known from the start keeps.  AUX holds >= 2 ceil(nnz / 32) words; s_u
// is scan scratch.  All NT threads of the CTA; returns the payload bytes.
// (CHECKED: the caller has found a value to drop already)
template <typename T, int B, int NT, bool CHECKED = false>
__device__ __forceinline__ int refine_slot(unsigned *ch, int pbytes, T t, unsigned char *SH, unsigned *AUX,
                                           unsigned *s_u)
{
  using G = G2<T, B>;
  constexpr int ES = G::ES, NWP = NT / 32;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int nnz = (int)ch[0];
  unsigned char *P = reinterpret_cast<unsigned char *>(ch + 2);
  T *vals = reinterpret_cast<T *>(P + 64 * ES + G::MASKB);
  if constexpr (!CHECKED) {
    int drop = 0;
    for (int j = tid; j < nnz; j += NT) drop |= (fabs(vals[j]) < t) ? 1 : 0;
    if (!__syncthreads_or(drop)) return pbytes;
  }
  // keep bits (bit j % 32 of word j / 32), the values to SH
  const int NKW = (nnz + 31) >> 5;
  unsigned *KF = AUX, *KP = AUX + NKW;
  T *SV = reinterpret_cast<T *>(SH);
  for (int j0 = wid * 32; j0 < nnz; j0 += NT) {
    const int j = j0 + lane;
    T v = T(0);
    if (j < nnz) v = vals[j];
    const unsigned keep = __ballot_sync(FULL, j < nnz && !(fabs(v) < t));
    if (lane == 0) KF[j0 >> 5] = keep;
    if (j < nnz) SV[j] = v;
  }
  __syncthreads();
  // new index of each kept value: exclusive prefix of the keep counts
  {
    const int per = (NKW + NT - 1) / NT, w0 = tid * per;
    unsigned sum = 0;
    for (int q = 0; q < per; ++q)
      if (w0 + q < NKW) sum += __popc(KF[w0 + q]);
    unsigned tot;
    unsigned ex = block_exsum<NT>(sum, s_u, tot);
    for (int q = 0; q < per; ++q)
      if (w0 + q < NKW) {
        KP[w0 + q] = ex;
        ex += __popc(KF[w0 + q]);
      }
    if (tid == 0) ch[0] = tot;
  }
  __syncthreads();
  // mask rows: the j-th set bit (positions in stream order) is value j
  {
    unsigned *M = reinterpret_cast<unsigned *>(P + 64 * ES);
    constexpr int NMW = G::NMW, per = (NMW + NT - 1) / NT;
    const int m0 = tid * per;
    unsigned words[per], sum = 0;
#pragma unroll
    for (int q = 0; q < per; ++q) {
      words[q] = m0 + q < NMW ? M[m0 + q] : 0u;
      sum += __popc(words[q]);
    }
    unsigned tot;
    unsigned j = block_exsum<NT>(sum, s_u, tot);
#pragma unroll
    for (int q = 0; q < per; ++q) {
      unsigned wd = words[q], out = 0u;
      while (wd) {
        const int b = __ffs(wd) - 1;
        wd &= wd - 1u;
        if ((KF[j >> 5] >> (j & 31)) & 1u) out |= 1u << b;
        ++j;
      }
      if (m0 + q < NMW) M[m0 + q] = out;
    }
  }
  // the kept values, moved down (from the copy in SH)
  for (int j = tid; j < nnz; j += NT) {
    const unsigned kw = KF[j >> 5];
    if ((kw >> (j & 31)) & 1u) vals[KP[j >> 5] + __popc(kw & ((1u << (j & 31)) - 1u))] = SV[j];
  }
  __syncthreads();
  return 64 * ES + G::MASKB + (int)ch[0] * ES;
}

// ---- stage 2 of one slot, in place: [nnz | 0 | raw payload of pbytes]
// becomes [nnz | ntok | tokens | literal words] (shuffle into SH, then the
// zero-run code; five barriers).  Returns the chunk bytes.
template <typename T, int NT, int BAR = 0, int OFF = 0>
__device__ __forceinline__ unsigned stage2_chunk(unsigned *ch, int pbytes, unsigned char *SH, unsigned *AUX, int cap,
                                                 unsigned *s_u, int *s_i)
{
  constexpr int LGES = sizeof(T) == 8 ? 3 : 2;
  shuffle_words<T, NT, OFF>(ch + 2, pbytes >> 2, 0, pbytes >> LGES, SH);
  group_sync<BAR, NT>();  // the slot's payload is no longer needed
  return stage2_code<T, NT, BAR, OFF>(ch, pbytes, SH, AUX, cap, s_u, s_i);
}

// field of global block bid among the nf fields of a batched launch
template <int NF>
__device__ __forceinline__ int field_of(const StageMaps<NF> &maps, int nf, int bid)
{
  int f = 0;
  for (int q = 1; q < nf; ++q)
    if (maps.g[q].first <= bid) f = q;
  return f;
}

// NF = 1: one field described by a; NF > 1: up to NF fields of one group,
// their blocks numbered consecutively (field by field) in one index space
// ---- speculative thresholds: a warp's min / max (lo, hi; NaN never
// enters) into the header's keys where it extends the extremes this CTA
// has sent (s_kc; each is lowered / raised before the global atomic that
// carries it, so a warp that reads it and skips is covered by that atomic;
// the results are not waited for).
template <typename T>
__device__ __forceinline__ void send_extremes(T lo, T hi, unsigned long long *s_kc, WsHdr *ws)
{
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = min_nn(lo, __shfl_xor_sync(FULL, lo, o));
    hi = max_nn(hi, __shfl_xor_sync(FULL, hi, o));
  }
  if ((threadIdx.x & 31) == 0) {
    const unsigned long long kl = order_key(lo), kh = order_key(hi);
    if (kl < *(volatile unsigned long long *)&s_kc[0]) {
      atomicMin(&s_kc[0], kl);
      atomicMin(&ws->minkey, kl);
    }
    if (kh > *(volatile unsigned long long *)&s_kc[1]) {
      atomicMax(&s_kc[1], kh);
      atomicMax(&ws->maxkey, kh);
    }
  }
}

// SPEC (NF = 1): speculative thresholds (FwdArgs::spec).  At most 128
// registers a thread, whatever the block edge (enough CTAs per SM for the
// smaller edges: the speculative variant would otherwise take more)
template <typename T, int B, int KIND, int NF, bool SPEC = false>
__global__ void __launch_bounds__(B * B / 2, 65536 / (B * B / 2 * 128))
    k_stage1(const __grid_constant__ StageMaps<NF> maps, const FwdArgs a)
{
  using G = G2<T, B>;
  using T2 = typename V2T<T>::type;
  constexpr int NT = G::NT, ES = G::ES, Q = G::Q, ZH = G::ZH;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char *smem = align1024(smem_raw);
  unsigned char *PF = smem;                                   // tile [z][y][x], filled by TMA
  T2 *PL = reinterpret_cast<T2 *>(smem + G::TILE);            // level-0 plane
  T *CB = reinterpret_cast<T *>(smem + G::TILE);              // cube (start of the plane area)
  T2 *HX = reinterpret_cast<T2 *>(smem + G::TILE + G::PLC);   // level-0 halo
  // after the transform the halo area holds the row offsets and the mask
  // rows; the next block writes it only after its first barrier, so the
  // payload phase needs no barrier at its end
  unsigned *ROWOFF = reinterpret_cast<unsigned *>(smem + G::TILE + G::PLC);
  unsigned char *MASKU = smem + G::TILE + G::PLC + G::ROWB;  // mask rows (for placing values)
  __shared__ __align__(8) unsigned long long s_bar;
  __shared__ unsigned s_u[40];

  WsHdr *ws = reinterpret_cast<WsHdr *>(a.ws);
  const int tid = threadIdx.x, lane = tid & 31;
  int ap, k, h;
  quad_of<B>(tid, ap, k, h);
  const int seg = lane - ap;
  const int x0 = 2 * ap;
  const int zr = h * ZH + ap;  // z of this thread's two mask rows

  double mn, mx, range;
  T t;
  __shared__ T s_t[NF];
  static_assert(!SPEC || NF == 1, "speculative thresholds: one field");
  // speculative thresholds: the extremes this CTA's warps have sent to the
  // header's keys (send_extremes)
  __shared__ unsigned long long s_kc[2];
  if constexpr (SPEC) {
    if (tid == 0) {
      s_kc[0] = ~0ull;
      s_kc[1] = 0ull;
    }
  }
  __shared__ T s_thi;  // speculative thresholds: near_threshold(t_lo)
  if constexpr (NF == 1) {
    if constexpr (SPEC) {  // t_lo of the subsample's range, no larger than the field's threshold
      t = threshold_between<T>(a.eps, a.eps_mode, *(volatile const unsigned long long *)&ws->skmin,
                               *(volatile const unsigned long long *)&ws->skmax);
      if (tid == 0) s_thi = near_threshold(t);
    } else
      threshold_of<T>(a.eps, a.eps_mode, a.cnorm, a.range, ws, mn, mx, range, t);
  } else if (tid < a.nf) {
    T tf;
    threshold_keys<T>(maps.g[tid].eps, maps.g[tid].eps_mode, a.cnorm, maps.g[tid].range_in, a.keys + 2 * tid, mn,
                      mx, range, tf);
    s_t[tid] = tf;
  }
  const bool cE = (x0 % Q == 0) && ((2 * k) % Q == 0);  // column (x0, 2k) holds coarse values
  unsigned ccm = 0;                                      // their bits (2 zl) in the column word
#pragma unroll
  for (int zl = 0; zl < ZH; zl += Q) ccm |= 1u << (2 * zl);
  unsigned char *arena = a.staging + (size_t)blockIdx.x * a.arena_bytes;

  auto tile_of = [&](int bid) {
    int f = 0, lb = bid, nbx = a.nbx, nby = a.nby;
    if constexpr (NF > 1) {
      f = field_of<NF>(maps, a.nf, bid);
      lb = bid - maps.g[f].first;
      nbx = maps.g[f].nbx;
      nby = maps.g[f].nby;
    }
    const int bx = lb % nbx, by = (lb / nbx) % nby, bz = lb / (nbx * nby);
    tma_load_tile(&maps.tm[f], PF, &s_bar, bx * B, by * B, bz * B, G::TILE);
  };
  unsigned long long aoff = 0;  // bytes used in this CTA's staging arena (the same in every thread)
  __shared__ BlockWalk s_wk;  // the next tile's block (one field)
  // set by every thread whose wait for the tile gives up; read by all
  // threads only after a barrier, so the CTA decides as one
  __shared__ unsigned s_to;
  if (tid == 0) {
    s_wk.init(blockIdx.x + gridDim.x, gridDim.x, a.nbx, a.nby);
    mbar_init(&s_bar);
    s_to = 0;
    if ((int)blockIdx.x < a.nblocks) tile_of(blockIdx.x);
  }
  __syncthreads();
  unsigned phase = 0;

  for (int bid = blockIdx.x; bid < a.nblocks; bid += gridDim.x) {
    // a thread whose wait gives up records it and goes on with whatever the
    // tile holds (in-bounds arithmetic on it, nothing stored): no barrier
    // below waits for a thread that has left
    if (!mbar_wait(&s_bar, phase)) s_to = 1u;
    phase ^= 1u;
    if constexpr (SPEC) {
      if (tid == 0) a.near[bid] = 0;  // (set by the payload writes after the barriers below)
    }

    // ---- tile -> registers; the next tile is fetched after the
    // transform's first barrier, when every thread has read this one.
    // W4li (swizzled 128-byte rows): the finest x-level first, row by row in
    // the tile, then the pairs (two values of one 16-byte chunk) at their
    // swizzled places.
    constexpr bool RX = G::template rowx<KIND>();
    // speculative thresholds: the block's min / max into the header's keys,
    // from the pairs as they are loaded; the W4li row pass takes it from the
    // rows it reads
    if constexpr (RX) {
      if constexpr (SPEC) {
        T lo = (T)INFINITY, hi = (T)-INFINITY;
        x_rows<T, B, KIND, true, NT, true>(PF, lo, hi);
        send_extremes<T>(lo, hi, s_kc, ws);
      } else {
        x_rows<T, B, KIND, true, NT>(PF);
      }
      fence_async_smem();  // the next tile's copy overwrites these writes
      __syncthreads();
    }
    T2 v[2][ZH];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int zl = 0; zl < ZH; ++zl) {
        const unsigned o = (unsigned)((((h * ZH + zl) * B + 2 * k + r) * B + x0) * ES);
        v[r][zl] = *reinterpret_cast<const T2 *>(PF + (RX ? swz128(o) : o));
      }
    if constexpr (SPEC && !RX) {
      T lo = (T)INFINITY, hi = (T)-INFINITY;
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int zl = 0; zl < ZH; ++zl) {
          lo = min3_nn(lo, v[r][zl].x, v[r][zl].y);
          hi = max3_nn(hi, v[r][zl].x, v[r][zl].y);
        }
      send_extremes<T>(lo, hi, s_kc, ws);
    }
    const int nb = bid + (int)gridDim.x;

    // ---- forward transform
    auto prefetch = [&] {
      // (after a barrier: a timeout of this block's copy is visible here,
      // and then no further copy is started)
      if (tid == 0 && nb < a.nblocks && !*(volatile unsigned *)&s_to) {
        if constexpr (NF == 1) {
          tma_load_tile(&maps.tm[0], PF, &s_bar, s_wk.bx * B, s_wk.by * B, s_wk.bz * B, G::TILE);
          s_wk.next();
        } else {
          tile_of(nb);
        }
      }
    };
    fwd_all<T, B, KIND, !RX>(v, PL, HX, CB, ap, k, h, seg, prefetch);
    if constexpr (G::L == 1) __syncthreads();  // no cube: the halo's last reads were just now

    // ---- significance bits (bit 2 zl + p: column x0 + p at z = h B/2 + zl),
    // mask rows by bit transpose over the segment
    if constexpr (NF > 1) t = s_t[field_of<NF>(maps, a.nf, bid)];
    unsigned W[2] = {keep_bits<ZH>(v[0], t), keep_bits<ZH>(v[1], t)};
    if (cE) W[0] &= ~ccm;
    const unsigned R0 = seg_transpose<B>(W[0], ap), R1 = seg_transpose<B>(W[1], ap);  // rows (zr, 2k), (zr, 2k+1)
    ROWOFF[rpad<B>(zr, 2 * k)] = __popc(R0);
    ROWOFF[rpad<B>(zr, 2 * k + 1)] = __popc(R1);
    put_rowi<B>(MASKU, rpad<B>(zr, 2 * k), R0);
    put_rowi<B>(MASKU, rpad<B>(zr, 2 * k + 1), R1);
    __syncthreads();
    unsigned nnz;
    {
      constexpr int IPT = (B * B + NT - 1) / NT;
      unsigned loc[IPT], sum = 0;
#pragma unroll
      for (int q = 0; q < IPT; ++q) {
        loc[q] = ROWOFF[rpad_of<B>(tid * IPT + q)];
        sum += loc[q];
      }
      unsigned ex = block_exsum_nb<NT>(sum, s_u, nnz);
#pragma unroll
      for (int q = 0; q < IPT; ++q) {
        ROWOFF[rpad_of<B>(tid * IPT + q)] = ex;
        ex += loc[q];
      }
    }
    __syncthreads();
    if (*(volatile unsigned *)&s_to) {
      // the tile never arrived (in some thread's view): the whole CTA stops
      // here.  Wait once more, bounded, for the one copy in flight (no
      // later copy was started), and mark this block and the CTA's later
      // blocks lost, so that the stage-2 and placement kernels skip them.
      if (tid == 0) {
        atomicCAS(&ws->status, 0u, ST_TIMEOUT);
        mbar_wait(&s_bar, phase ^ 1u);
      }
      for (long long b = bid + (long long)tid * gridDim.x; b < a.nblocks; b += (long long)NT * gridDim.x)
        a.table[2 * b + 1] = TB_LOST;
      return;
    }

    // ---- slot [nnz | 0 | raw payload] -> this CTA's staging arena
    const int pbytes = 64 * ES + G::MASKB + (int)nnz * ES;
    const unsigned long long so = aoff;
    const unsigned long long slot = (unsigned long long)((pbytes + 12 + 15) & ~15);
    const bool ok = so + slot <= a.arena_bytes;
    if (ok) {
      unsigned char *P = arena + so + 8;
      // mask rows: a coalesced copy of the shared (padded) rows
      for (int i = tid; i < B * B; i += NT) put_rowi<B>(P + 64 * ES, i, get_rowi<B>(MASKU, rpad_of<B>(i)));
      if (cE) {
#pragma unroll
        for (int zl = 0; zl < ZH; zl += Q)
          reinterpret_cast<T *>(P)[(((h * ZH + zl) / Q) * 4 + (2 * k) / Q) * 4 + x0 / Q] = v[0][zl].x;
      }
      // kept details of this thread's columns (z unrolled: v stays in registers)
      T *VALS = reinterpret_cast<T *>(P + 64 * ES + G::MASKB);
      const unsigned lowE = (1u << x0) - 1u, lowO = (2u << x0) - 1u;
      if (W[0] | W[1]) {
        // speculative thresholds: whether a kept value lies below t_hi, a
        // little above t_lo (the block is then tested by stage 2)
        bool near = false;
        const T thi = SPEC ? s_thi : T(0);
#pragma unroll
        for (int zl = 0; zl < ZH; ++zl) {
          const int z = h * ZH + zl;
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            const unsigned b2 = (W[r] >> (2 * zl)) & 3u;
            if (b2) {
              const unsigned wd = get_rowi<B>(MASKU, rpad<B>(z, 2 * k + r));
              const unsigned base = ROWOFF[rpad<B>(z, 2 * k + r)];
              if (b2 & 1u) {
                VALS[base + __popc(wd & lowE)] = zero_low(v[r][zl].x, a.zbits);
                if constexpr (SPEC) near |= fabs(v[r][zl].x) < thi;
              }
              if (b2 & 2u) {
                VALS[base + __popc(wd & lowO)] = zero_low(v[r][zl].y, a.zbits);
                if constexpr (SPEC) near |= fabs(v[r][zl].y) < thi;
              }
            }
          }
        }
        if constexpr (SPEC) {
          if (near) a.near[bid] = 1;
        }
      }
    }
    if (tid == 0) {
      if (ok) {
        unsigned *hw = reinterpret_cast<unsigned *>(arena + so);
        hw[0] = nnz;
        hw[1] = 0u;
        if (a.stage2 && pbytes > G::SHCAP) a.biglist[atomicAdd(&ws->nbig, 1u)] = bid;  // for the large stage-2 launch
      } else {
        atomicCAS(&ws->status, 0u, ST_CAPACITY);
      }
      a.table[2 * bid] = (unsigned long long)(arena - a.staging) + so;
      a.table[2 * bid + 1] = ok ? 8ull + (unsigned long long)pbytes : TB_LOST;
    }
    if (ok) aoff = so + slot;
  }
}

// ---- speculative thresholds: the exact threshold t, and which slots are
// tested against it (0: none, t_lo is t; 1: those marked near, t lies
// within t_lo's near bound; 2: all)
template <typename T>
__device__ __forceinline__ int spec_mode(const S2Args &a, T &t)
{
  const WsHdr *h = reinterpret_cast<const WsHdr *>(a.ws);
  t = threshold_between<T>(a.eps, a.eps_mode, h->minkey, h->maxkey);
  const T tl = threshold_between<T>(a.eps, a.eps_mode, h->skmin, h->skmax);
  return t_bits(tl) == t_bits(t) ? 0 : t <= near_threshold(tl) ? 1 : 2;
}

// ---- speculative thresholds, before stage 2 (block edges up to 16): flag
// (TB_SKIP: the stage-2 launches pass over them) and list (rlist, count
// nref) the slots to test against t, those marked near in mode 1 and all
// in mode 2; k_stage2_listed takes them after the others
template <typename T>
__global__ void __launch_bounds__(256) k_spec_list(const S2Args a)
{
  T t;
  const int mode = spec_mode<T>(a, t);
  if (mode == 0) return;
  WsHdr *hw = reinterpret_cast<WsHdr *>(const_cast<void *>(a.ws));
  for (int b = blockIdx.x * 256 + threadIdx.x; b < a.nblocks; b += gridDim.x * 256) {
    if (mode == 1 && a.near[b] == 0) continue;
    const unsigned long long cb = a.table[2 * b + 1];
    if (cb == TB_LOST || (cb & TB_FIN)) continue;
    a.table[2 * b + 1] = cb | TB_SKIP;
    a.rlist[atomicAdd(&hw->nref, 1u)] = b;
  }
}

// ---- stage 2, in place, over the slots of all blocks.  SPEC (speculative
// thresholds, S2Args::spec, block edge 32; a variant of its own, so that
// the other keeps its registers): the slots to test (those marked near in
// mode 1, all in mode 2) are tested against t, for FP32 while the payload
// is shuffled, and one holding a value below t is listed (rlist, count
// nref) for k_stage2_refine, which spreads those over its CTAs.
template <typename T, int B, bool BIG, bool SPEC = false>
__global__ void __launch_bounds__(BIG ? 512 : 128, BIG ? 4 : sizeof(T) == 4 ? 16 : 12) k_stage2(const S2Args a)
{
  using G = G2<T, B>;
  constexpr int NT = BIG ? 512 : 128;
  constexpr int CAPB = BIG ? G::PMAX_AL : G::SHCAP;  // payload bytes in shared memory
  constexpr int cap = BIG ? G::NBWMAX : G::NBS;     // bitmap words
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ unsigned s_u[40];
  __shared__ int s_i[40];
  unsigned *AUX = reinterpret_cast<unsigned *>(smem + CAPB);

  // the small launch visits every block (and skips the large payloads and
  // those the stage kernel has coded already); the large launch visits
  // only the blocks the stage kernel listed
  const int count = BIG ? (int)reinterpret_cast<const WsHdr *>(a.ws)->nbig : a.nblocks;
  T t = T(0);
  int mode = 0;
  if constexpr (SPEC) mode = spec_mode<T>(a, t);
  for (int it = blockIdx.x; it < count; it += gridDim.x) {
    const int bid = BIG ? a.biglist[it] : it;
    const unsigned long long so = a.table[2 * bid], cb = a.table[2 * bid + 1];
    // (the mark is loaded with the table entry, so their latencies overlap)
    const bool test = SPEC && (mode == 2 || (mode == 1 && a.near[bid] != 0));
    // staging overflow, finished already, or left to k_stage2_listed
    if (cb == TB_LOST || (cb & (TB_FIN | TB_SKIP))) continue;
    const int pbytes = (int)cb - 8;
    if ((pbytes > G::SHCAP) != BIG) continue;  // the other launch's payload
    unsigned *ch = reinterpret_cast<unsigned *>(a.staging + so);
    unsigned cbytes;
    if (!test) {
      cbytes = stage2_chunk<T, NT>(ch, pbytes, smem, AUX, cap, s_u, s_i);
    } else if constexpr (SPEC) {
      bool drop;
      if constexpr (sizeof(T) == 4) {
        constexpr int VW0 = (64 * 4 + G::MASKB) / 4;
        drop = __syncthreads_or(shuffle_check<T, NT>(ch + 2, pbytes >> 2, pbytes >> 2, smem, VW0, t));
      } else {
        const T *vals = reinterpret_cast<const T *>(reinterpret_cast<const unsigned char *>(ch + 2) +
                                                    64 * G::ES + G::MASKB);
        bool d = false;
        for (int j = threadIdx.x; j < (int)ch[0]; j += NT) d |= fabs(vals[j]) < t;
        drop = __syncthreads_or(d);
        if (!drop) shuffle_words<T, NT>(ch + 2, pbytes >> 2, 0, pbytes >> 3, smem);
        __syncthreads();
      }
      if (drop) {  // the slot is left as it is (only SH holds the shuffle)
        if (threadIdx.x == 0)
          a.rlist[atomicAdd(&reinterpret_cast<WsHdr *>(const_cast<void *>(a.ws))->nref, 1u)] = bid;
        continue;
      }
      cbytes = stage2_code<T, NT>(ch, pbytes, smem, AUX, cap, s_u, s_i);
    }
    if (threadIdx.x == 0) a.table[2 * bid + 1] = TB_FIN | (unsigned long long)cbytes;
  }
}

// ---- speculative thresholds, block edges up to 16: stage 2 of the slots
// k_spec_list listed, CTAs and buffers as k_stage2's (BIG: the large
// payloads).  The values are tested against t (FP32: while the payload is
// shuffled); a slot holding one below t drops those first (refine_slot:
// SH holds its values, AUX its keep bits), then is coded.  (Tested inside
// k_stage2, the few slots to test made the common path of those small
// blocks' launches about a quarter longer in instructions.)
template <typename T, int B, bool BIG>
__global__ void __launch_bounds__(BIG ? 512 : 128, BIG ? 4 : 12) k_stage2_listed(const S2Args a)
{
  using G = G2<T, B>;
  constexpr int NT = BIG ? 512 : 128;
  constexpr int CAPB = BIG ? G::PMAX_AL : G::SHCAP;
  constexpr int cap = BIG ? G::NBWMAX : G::NBS;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ unsigned s_u[40];
  __shared__ int s_i[40];
  unsigned *AUX = reinterpret_cast<unsigned *>(smem + CAPB);
  const WsHdr *h = reinterpret_cast<const WsHdr *>(a.ws);
  const int count = (int)h->nref;
  if ((int)blockIdx.x >= count) return;
  const T t = threshold_between<T>(a.eps, a.eps_mode, h->minkey, h->maxkey);
  for (int it = blockIdx.x; it < count; it += gridDim.x) {
    const int bid = a.rlist[it];
    const unsigned long long so = a.table[2 * bid], cb = a.table[2 * bid + 1];
    int pbytes = (int)cb - 8;  // (the low half: TB_SKIP is a high bit)
    if ((pbytes > G::SHCAP) != BIG) continue;  // the other launch's payload
    unsigned *ch = reinterpret_cast<unsigned *>(a.staging + so);
    bool drop;
    if constexpr (sizeof(T) == 4) {
      constexpr int VW0 = (64 * 4 + G::MASKB) / 4;
      drop = __syncthreads_or(shuffle_check<T, NT>(ch + 2, pbytes >> 2, pbytes >> 2, smem, VW0, t));
    } else {
      const T *vals = reinterpret_cast<const T *>(reinterpret_cast<const unsigned char *>(ch + 2) + 64 * G::ES +
                                                  G::MASKB);
      bool d = false;
      for (int j = threadIdx.x; j < (int)ch[0]; j += NT) d |= fabs(vals[j]) < t;
      drop = __syncthreads_or(d);
      if (!drop) shuffle_words<T, NT>(ch + 2, pbytes >> 2, 0, pbytes >> 3, smem);
      __syncthreads();
    }
    unsigned cbytes;
    if (drop) {  // the slot is as the stage kernel left it (SH holds the shuffle)
      pbytes = refine_slot<T, B, NT, true>(ch, pbytes, t, smem, AUX, s_u);
      cbytes = stage2_chunk<T, NT>(ch, pbytes, smem, AUX, cap, s_u, s_i);
    } else {
      cbytes = stage2_code<T, NT>(ch, pbytes, smem, AUX, cap, s_u, s_i);
    }
    if (threadIdx.x == 0) a.table[2 * bid + 1] = TB_FIN | (unsigned long long)cbytes;
  }
}

// ---- speculative thresholds, block edge 32: the slots the stage-2 launches
// listed (they hold a value below the exact threshold t), one per CTA at a time: drop
// those values, then stage 2 as above.  512 threads, the payload buffer and
// the bitmaps of the large launch.
template <typename T, int B>
__global__ void __launch_bounds__(512) k_stage2_refine(const S2Args a)
{
  using G = G2<T, B>;
  constexpr int NT = 512, CAPB = G::PMAX_AL, cap = G::NBWMAX;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ unsigned s_u[40];
  __shared__ int s_i[40];
  unsigned *AUX = reinterpret_cast<unsigned *>(smem + CAPB);
  const WsHdr *h = reinterpret_cast<const WsHdr *>(a.ws);
  const int count = (int)*(volatile const unsigned *)&h->nref;
  if ((int)blockIdx.x >= count) return;
  const T t = threshold_between<T>(a.eps, a.eps_mode, h->minkey, h->maxkey);
  for (int it = blockIdx.x; it < count; it += gridDim.x) {
    const int bid = a.rlist[it];
    const unsigned long long so = a.table[2 * bid], cb = a.table[2 * bid + 1];
    unsigned *ch = reinterpret_cast<unsigned *>(a.staging + so);
    int pbytes = (int)cb - 8;
    pbytes = refine_slot<T, B, NT, true>(ch, pbytes, t, smem, AUX, s_u);
    const unsigned cbytes = stage2_chunk<T, NT>(ch, pbytes, smem, AUX, cap, s_u, s_i);
    if (threadIdx.x == 0) a.table[2 * bid + 1] = TB_FIN | (unsigned long long)cbytes;
  }
}

// ---- chunk offsets (tile scan + decoupled look-back), header
template <typename T>
__global__ void __launch_bounds__(PLACE_TILE) k_place(const PlaceArgs a)
{
  constexpr int PT = PLACE_TILE, NT = PLACE_TILE;
  __shared__ unsigned s_u[40];
  __shared__ int s_tile;
  __shared__ unsigned long long s_excl;
  WsHdr *ws = reinterpret_cast<WsHdr *>(a.ws);
  unsigned long long *lbst = reinterpret_cast<unsigned long long *>((char *)a.ws + WS_HDR);
  const int tid = threadIdx.x;
  if (tid == 0) s_tile = (int)atomicAdd(&ws->ticket, 1u);  // earlier tiles are resident or done
  __syncthreads();
  const int tile = s_tile, c0 = tile * PT;
  const int n = a.nblocks - c0 < PT ? a.nblocks - c0 : PT;
  unsigned long long cb = 0;
  if (tid < n) {
    cb = a.table[2 * (c0 + tid) + 1];
    if (cb == TB_LOST) {  // lost: leave an empty chunk
      atomicCAS(&ws->status, 0u, ST_CAPACITY);
      cb = 0;
    }
    cb = tb_size(cb);
  }
  unsigned ttot;
  const unsigned loc = block_exsum<NT>((unsigned)cb, s_u, ttot);  // < 2^32: 128 chunks of at most PMAX + 12 bytes
  if (tid < 32) {
    const unsigned long long ex = lookback(lbst, tile, ttot, &ws->status, (int)ST_TIMEOUT);
    if (tid == 0) s_excl = ex;
  }
  __syncthreads();
  const unsigned long long excl = s_excl;
  if (tid < n) {
    const unsigned long long off = excl + loc;
    st_le<unsigned long long>(a.out + HEADER_BYTES + 8ull * (c0 + tid), off);
    const bool fits = a.data0 + off + cb <= a.out_cap;
    if (!fits) atomicCAS(&ws->status, 0u, ST_CAPACITY);
  }
  if (tid == 0 && c0 + n == a.nblocks) {
    double mn, mx, range;
    T t;
    threshold_of<T>(a.eps, a.eps_mode, a.cnorm, a.range, ws, mn, mx, range, t);
    const unsigned long long data_bytes = excl + ttot, total = a.data0 + data_bytes;
    unsigned char *h = a.out;
    st_le<unsigned long long>(h + HEADER_BYTES + 8ull * a.nblocks, data_bytes);
    for (unsigned long long q = HEADER_BYTES + 8ull * (a.nblocks + 1); q < a.data0; ++q) h[q] = 0;
    for (int q = 0; q < HEADER_BYTES; ++q) h[q] = 0;
    st_le<unsigned>(h + 0, MAGIC);
    st_le<unsigned short>(h + 4, 1);
    st_le<unsigned short>(h + 6, HEADER_BYTES);
    st_le<int>(h + 8, a.nx);
    st_le<int>(h + 12, a.ny);
    st_le<int>(h + 16, a.nz);
    h[20] = (unsigned char)a.block;
    h[21] = (unsigned char)a.dtype;
    h[22] = (unsigned char)a.kind;
    h[23] = (unsigned char)a.stage2;
    h[24] = (unsigned char)a.eps_mode;
    h[25] = (unsigned char)a.levels;
    h[26] = (unsigned char)a.bound_mode;
    h[27] = (unsigned char)a.flags;
    st_le<unsigned>(h + 28, (unsigned)a.hdr_nblocks);
    st_le_f64(h + 32, a.eps);
    st_le_f64(h + 40, (double)t);
    st_le_f64(h + 48, mn);
    st_le_f64(h + 56, mx);
    st_le_f64(h + 64, range);
    st_le<unsigned long long>(h + 72, data_bytes);
    st_le<unsigned long long>(h + 80, total);
    ws->out_bytes = total;
    if (a.out_bytes) *a.out_bytes = total;
  }
}

// ---- one warp per chunk: staging slot -> its place in the stream
template <typename T>
__global__ void __launch_bounds__(256) k_copy(const PlaceArgs a)
{
  const int bid = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (bid >= a.nblocks) return;
  const unsigned long long so = a.table[2 * bid], cb0 = a.table[2 * bid + 1];
  if (cb0 == TB_LOST) return;
  const unsigned long long cb = tb_size(cb0);
  const unsigned long long off = *reinterpret_cast<const unsigned long long *>(a.out + HEADER_BYTES + 8ull * bid);
  if (a.data0 + off + cb > a.out_cap) return;
  const unsigned *__restrict__ src = reinterpret_cast<const unsigned *>(a.staging + so);
  unsigned *__restrict__ dst = reinterpret_cast<unsigned *>(a.out + a.data0 + off);
  const unsigned nw = (unsigned)(cb >> 2);
  constexpr int U = 8;
  for (unsigned q0 = lane; q0 < nw; q0 += 32 * U) {
    unsigned w[U];
#pragma unroll
    for (int j = 0; j < U; ++j) w[j] = q0 + 32 * j < nw ? src[q0 + 32 * j] : 0u;
#pragma unroll
    for (int j = 0; j < U; ++j)
      if (q0 + 32 * j < nw) dst[q0 + 32 * j] = w[j];
  }
}

// ---- batched placement: tiles of 128 chunks of one field; each field's
// look-back segment starts at its first tile, each field gets its own
// offset table and header
template <int NF>
__device__ __forceinline__ int field_of_tile(const BatchOut &bo, int tile)
{
  int f = 0;
  for (int q = 1; q < bo.nf; ++q)
    if (bo.f[q].tfirst <= tile) f = q;
  return f;
}

// PT chunks (and threads) per CTA: the scan granularity, a knob of the
// batch tuner (64, 128 or 256)
template <typename T, int PT>
__global__ void __launch_bounds__(PT) k_place_multi(const __grid_constant__ BatchOut bo, const PlaceArgs a)
{
  constexpr int NT = PT;
  __shared__ unsigned s_u[40];
  __shared__ int s_tile;
  __shared__ unsigned long long s_excl;
  WsHdr *ws = reinterpret_cast<WsHdr *>(a.ws);
  unsigned long long *lbst = a.lbst;
  const int tid = threadIdx.x;
  if (tid == 0) s_tile = (int)atomicAdd(&ws->ticket, 1u);  // earlier tiles are resident or done
  __syncthreads();
  const int tile = s_tile;
  const int f = field_of_tile<MAXF>(bo, tile);
  const FieldOut &fo = bo.f[f];
  const int c0 = fo.first + (tile - fo.tfirst) * PT;  // first global chunk of the tile
  const int cend = fo.first + fo.nblocks;
  const int n = cend - c0 < PT ? cend - c0 : PT;
  unsigned long long cb = 0;
  if (tid < n) {
    cb = a.table[2 * (c0 + tid) + 1];
    if (cb == TB_LOST) {  // lost: leave an empty chunk
      atomicCAS(&ws->status, 0u, ST_CAPACITY);
      cb = 0;
    }
    cb = tb_size(cb);
  }
  unsigned ttot;
  const unsigned loc = block_exsum<NT>((unsigned)cb, s_u, ttot);
  if (tid < 32) {
    const unsigned long long ex = lookback(lbst, tile, ttot, &ws->status, (int)ST_TIMEOUT, fo.tfirst);
    if (tid == 0) s_excl = ex;
  }
  __syncthreads();
  const unsigned long long excl = s_excl;
  if (tid < n) {
    const unsigned long long off = excl + loc;
    st_le<unsigned long long>(fo.out + HEADER_BYTES + 8ull * (c0 - fo.first + tid), off);
    if (fo.data0 + off + cb > fo.out_cap) atomicCAS(&ws->status, 0u, ST_CAPACITY);
  }
  if (tid == 0 && c0 + n == cend) {
    double mn, mx, range;
    T t;
    threshold_keys<T>(fo.eps, fo.eps_mode, a.cnorm, fo.range_in, a.keys + 2 * f, mn, mx, range, t);
    const unsigned long long data_bytes = excl + ttot, total = fo.data0 + data_bytes;
    unsigned char *h = fo.out;
    st_le<unsigned long long>(h + HEADER_BYTES + 8ull * fo.nblocks, data_bytes);
    for (unsigned long long q = HEADER_BYTES + 8ull * (fo.nblocks + 1); q < fo.data0; ++q) h[q] = 0;
    for (int q = 0; q < HEADER_BYTES; ++q) h[q] = 0;
    st_le<unsigned>(h + 0, MAGIC);
    st_le<unsigned short>(h + 4, 1);
    st_le<unsigned short>(h + 6, HEADER_BYTES);
    st_le<int>(h + 8, fo.nx);
    st_le<int>(h + 12, fo.ny);
    st_le<int>(h + 16, fo.nz);
    h[20] = (unsigned char)a.block;
    h[21] = (unsigned char)a.dtype;
    h[22] = (unsigned char)a.kind;
    h[23] = (unsigned char)a.stage2;
    h[24] = (unsigned char)fo.eps_mode;
    h[25] = (unsigned char)a.levels;
    h[26] = (unsigned char)a.bound_mode;
    h[27] = (unsigned char)a.flags;
    st_le<unsigned>(h + 28, (unsigned)fo.nblocks);
    st_le_f64(h + 32, fo.eps);
    st_le_f64(h + 40, (double)t);
    st_le_f64(h + 48, mn);
    st_le_f64(h + 56, mx);
    st_le_f64(h + 64, range);
    st_le<unsigned long long>(h + 72, data_bytes);
    st_le<unsigned long long>(h + 80, total);
    if (fo.out_bytes) *fo.out_bytes = total;
  }
}

// one warp per chunk of the batch: staging slot -> its field's stream
template <typename T>
__global__ void __launch_bounds__(256) k_copy_multi(const __grid_constant__ BatchOut bo, const PlaceArgs a)
{
  const int bid = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (bid >= a.nblocks) return;
  int f = 0;
  for (int q = 1; q < bo.nf; ++q)
    if (bo.f[q].first <= bid) f = q;
  const FieldOut &fo = bo.f[f];
  const unsigned long long so = a.table[2 * bid], cb0 = a.table[2 * bid + 1];
  if (cb0 == TB_LOST) return;
  const unsigned long long cb = tb_size(cb0);
  const unsigned long long off =
      *reinterpret_cast<const unsigned long long *>(fo.out + HEADER_BYTES + 8ull * (bid - fo.first));
  if (fo.data0 + off + cb > fo.out_cap) return;
  const unsigned *__restrict__ src = reinterpret_cast<const unsigned *>(a.staging + so);
  unsigned *__restrict__ dst = reinterpret_cast<unsigned *>(fo.out + fo.data0 + off);
  const unsigned nw = (unsigned)(cb >> 2);
  constexpr int U = 8;
  for (unsigned q0 = lane; q0 < nw; q0 += 32 * U) {
    unsigned w[U];
#pragma unroll
    for (int j = 0; j < U; ++j) w[j] = q0 + 32 * j < nw ? src[q0 + 32 * j] : 0u;
#pragma unroll
    for (int j = 0; j < U; ++j)
      if (q0 + 32 * j < nw) dst[q0 + 32 * j] = w[j];
  }
}

}  // namespace czp
