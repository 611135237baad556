// cz_group.cuh -- aggregate chunks: G consecutive blocks share one stage-2
// chunk (Sec. 3, Exp. 2 and 3: the stage-1 output of several blocks is
// concatenated and the lossless substage codes the concatenation as one
// buffer).
//
// Chunk of group k (blocks kG .. kG + g - 1, g = G but for the last group):
//   [u32 nnz of each block | u32 ntok | tokens | literal words]
// where the tokens and literals are the zero-run code of the byte shuffle
// (element size of the data) of the blocks' concatenated stage-1 payloads.
//
// Compression: the stage kernel writes raw slots as without stage 2; then
//   k_group2<0>  (persistent, 256 threads) gathers the payloads of a group
//                straight from their slots (one flat loop over the group's
//                words) into shuffled order in shared memory and codes them
//                with the single-payload coder into the group's slot, for
//                payloads up to 48 KiB, and lists the larger groups;
//   k_group2<1>  (512 threads) does the same for the listed groups up to
//                192 KiB, and lists the rest;
//   k_group_huge (512 threads) codes those, with the shuffled buffer in a
//                global scratch block per CTA (the slab lanes' large coder);
// and the placement and copy kernels run over the group table.
// Decompression: k_gunstage<0 / 1 / 2> (the same three tiers) decodes the
// tokens of a group into the shuffled buffer and unshuffles the payloads of
// the blocks it needs into their slots, in the layout the block decoders
// read without groups.
#pragma once

#include "cz_compress.cuh"
#include "cz_slab.cuh"

namespace czp {

constexpr int GROUP_MAXG = 16;
// largest group payload: its four bitmap arrays (one bit per word each)
// fill the large coder's shared memory
constexpr int GROUP_MAX_BYTES = 1792 * 1024;
constexpr int GROUP_HSMEM = GROUP_MAX_BYTES / 8;

// tiers of the group coder and decoder: threads and the payload bytes held
// in shared memory (tier 2: global scratch)
template <int TIER>
struct GT {
  static constexpr int NT = TIER == 0 ? 256 : 512;
  static constexpr int CAP = TIER == 0 ? 48 * 1024 : TIER == 1 ? 192 * 1024 : 0;
  static constexpr int CAPW = CAP / 128;                // bitmap words (one bit per payload word)
  static constexpr int SMEM = CAP + 4 * CAPW * 4;       // coder: payload + four bitmap arrays
  static constexpr int USMEM = CAP + 3 * NT * 4;        // decoder: payload + per-token words
};

// the payloads of group k, by warp 0: slot offsets and nnz of its g blocks
// and the words before each (s_w0[0..g], s_w0[g] = all words of the group);
// returns (in every lane of warp 0) whether a block of the group was lost
__device__ __forceinline__ bool group_slots(const GroupArgs &a, int k, int g, unsigned long long *s_so, int *s_w0,
                                            unsigned *s_nnz)
{
  const int lane = threadIdx.x & 31, b = k * a.G + lane;
  unsigned long long so = 0, cb = 0;
  if (lane < g) {
    so = a.table[2 * b];
    cb = a.table[2 * b + 1];
  }
  const bool lost = lane < g && cb == TB_LOST;
  const int w = (lane < g && !lost) ? (int)((cb - 8) >> 2) : 0;
  int inc = w;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int v = __shfl_up_sync(FULL, inc, d);
    if (lane >= d) inc += v;
  }
  if (lane < g) {
    s_so[lane] = so;
    s_nnz[lane] = lost ? 0u : *reinterpret_cast<const unsigned *>(a.staging + so);
  }
  if (lane <= g) s_w0[lane] = inc - w;
  return __ballot_sync(FULL, lost) != 0u;
}

// the block of a group's word k: the last i < g with s_w0[i] <= k (payloads
// are never empty, so s_w0 increases strictly)
__device__ __forceinline__ int block_of_word(const int *s_w0, int g, int k)
{
  int lo = 0, hi = g - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (s_w0[mid] <= k)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// the W words of a group's concatenated payloads, read from the blocks'
// slots, byte-shuffled into SH (E elements): word k is bytes 0..3 of
// element 4k / ES at byte offset 4k % ES (every payload is a whole number
// of elements, so the concatenation keeps element boundaries)
template <typename T, int NT>
__device__ __forceinline__ void shuffle_group(const unsigned char *staging, const unsigned long long *s_so,
                                              const int *s_w0, int g, int W, int E, unsigned char *SH)
{
  constexpr int ES = (int)sizeof(T), LGES = ES == 8 ? 3 : 2;
  for (int k0 = threadIdx.x; k0 < W; k0 += 4 * NT) {
    unsigned wv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = k0 + j * NT;
      wv[j] = 0u;
      if (k < W) {
        const int i = block_of_word(s_w0, g, k);
        wv[j] = reinterpret_cast<const unsigned *>(staging + s_so[i] + 8)[k - s_w0[i]];
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = k0 + j * NT;
      if (k < W) {
        const int e = (4 * k) >> LGES, b0 = (4 * k) & (ES - 1);
#pragma unroll
        for (int q = 0; q < 4; ++q) SH[(b0 + q) * E + e] = (unsigned char)(wv[j] >> (8 * q));
      }
    }
  }
}

// ---- coder tiers 0 and 1: the shuffled group payload in shared memory.
// Tier 0 visits every group and lists those above its capacity (biglist
// from 0, count nbig); tier 1 visits those and lists the rest (biglist from
// ngroups, count nbig2) for k_group_huge.
template <typename T, int B, int TIER>
__global__ void __launch_bounds__(GT<TIER>::NT) k_group2(const GroupArgs a)
{
  constexpr int NT = GT<TIER>::NT, CAPB = GT<TIER>::CAP, LGES = sizeof(T) == 8 ? 3 : 2;
  static_assert(TIER == 0 || TIER == 1, "shared-memory tiers only");
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ unsigned s_u[40];
  __shared__ int s_i[40];
  __shared__ unsigned long long s_so[GROUP_MAXG];
  __shared__ int s_w0[GROUP_MAXG + 1];
  __shared__ unsigned s_nnz[GROUP_MAXG];
  __shared__ int s_lost;
  unsigned *AUX = reinterpret_cast<unsigned *>(smem + CAPB);
  WsHdr *ws = reinterpret_cast<WsHdr *>(a.ws);
  const int tid = threadIdx.x;
  const int count = TIER == 0 ? a.ngroups : (int)*(volatile const unsigned *)&ws->nbig;
  for (int it = blockIdx.x; it < count; it += gridDim.x) {
    const int k = TIER == 0 ? it : a.biglist[it];
    const int g = min(a.G, a.nblocks - k * a.G);
    __syncthreads();  // the previous group's shared words are no longer read
    if (tid < 32) {
      const bool lost = group_slots(a, k, g, s_so, s_w0, s_nnz);
      if (tid == 0) s_lost = lost ? 1 : 0;
    }
    __syncthreads();
    const int W = s_w0[g], pbytes = 4 * W;
    if (s_lost || pbytes > CAPB) {
      if (tid == 0) {
        a.gtable[2 * k] = (unsigned long long)k * a.gslot;
        if (s_lost)
          a.gtable[2 * k + 1] = TB_LOST;
        else if (TIER == 0)
          a.biglist[atomicAdd(&ws->nbig, 1u)] = k;
        else
          a.biglist[a.ngroups + (int)atomicAdd(&ws->nbig2, 1u)] = k;
      }
      continue;
    }
    shuffle_group<T, NT>(a.staging, s_so, s_w0, g, W, pbytes >> LGES, smem);
    unsigned *gs = reinterpret_cast<unsigned *>(a.gstage + (unsigned long long)k * a.gslot);
    if (tid < g) gs[tid] = s_nnz[tid];
    __syncthreads();
    // [nnz_{g-1} | ntok | tokens | literals] from word g - 1 on
    const unsigned cb = stage2_code<T, NT>(gs + (g - 1), pbytes, smem, AUX, GT<TIER>::CAPW, s_u, s_i);
    if (tid == 0) {
      a.gtable[2 * k] = (unsigned long long)k * a.gslot;
      a.gtable[2 * k + 1] = TB_FIN | (4ull * (unsigned long long)(g - 1) + cb);
    }
  }
}

// ---- coder tier 2: the groups tier 1 listed, shuffled into a global
// scratch buffer of hcap bytes per CTA
template <typename T, int B>
__global__ void __launch_bounds__(512) k_group_huge(const GroupArgs a)
{
  constexpr int NT = 512, LGES = sizeof(T) == 8 ? 3 : 2;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ unsigned s_u[40];
  __shared__ int s_i[40];
  __shared__ int s_lastend;
  __shared__ unsigned long long s_so[GROUP_MAXG];
  __shared__ int s_w0[GROUP_MAXG + 1];
  __shared__ unsigned s_nnz[GROUP_MAXG];
  const int tid = threadIdx.x;
  if (tid == 0) s_lastend = 0;
  unsigned char *SH = a.scratch + (size_t)blockIdx.x * (size_t)a.hcap;
  const int count = (int)*(volatile const unsigned *)&reinterpret_cast<const WsHdr *>(a.ws)->nbig2;
  for (int it = blockIdx.x; it < count; it += gridDim.x) {
    const int k = a.biglist[a.ngroups + it];
    const int g = min(a.G, a.nblocks - k * a.G);
    __syncthreads();
    if (tid < 32) group_slots(a, k, g, s_so, s_w0, s_nnz);  // none lost: tier 0 listed it
    __syncthreads();
    const int W = s_w0[g], pbytes = 4 * W;
    if (pbytes > a.hcap) {  // cannot happen for a valid group; leave it lost
      if (tid == 0) {
        atomicCAS(&reinterpret_cast<WsHdr *>(a.ws)->status, 0u, ST_CAPACITY);
        a.gtable[2 * k + 1] = TB_LOST;
      }
      continue;
    }
    shuffle_group<T, NT>(a.staging, s_so, s_w0, g, W, pbytes >> LGES, SH);
    unsigned *gs = reinterpret_cast<unsigned *>(a.gstage + (unsigned long long)k * a.gslot);
    if (tid < g) gs[tid] = s_nnz[tid];
    __syncthreads();
    const unsigned long long cb = huge_code<NT>(gs + (g - 1), pbytes, SH, reinterpret_cast<unsigned *>(smem),
                                                a.hcap / 128, s_u, s_i, &s_lastend);
    if (tid == 0) a.gtable[2 * k + 1] = TB_FIN | (4ull * (unsigned long long)(g - 1) + cb);
  }
}

// ---- decompression: item it is group it (whole field), or the group of
// requested block ids[it] (random access: that block alone is unpacked).
// Tier 0 visits every item and lists those above its capacity (biglist
// from 0, count nbig); tier 1 visits those and lists the rest (biglist from
// `items`, count nbig2); tier 2 decodes those into global scratch.
template <typename T, int B, int TIER>
__global__ void __launch_bounds__(GT<TIER>::NT) k_gunstage(const UnArgs a)
{
  using G = G2<T, B>;
  constexpr int NT = GT<TIER>::NT, CAPB = GT<TIER>::CAP, ES = G::ES, LGES = G::LGES;
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char *P = TIER == 2 ? a.scratch + (size_t)blockIdx.x * (size_t)a.hcap : smem;
  unsigned *TL = reinterpret_cast<unsigned *>(smem + CAPB);
  unsigned *TO = TL + NT;
  unsigned *TK = TO + NT;
  __shared__ unsigned long long s_u64[NT / 32];
  __shared__ unsigned s_nnz[GROUP_MAXG];
  __shared__ int s_w0[GROUP_MAXG + 1];
  __shared__ unsigned s_ntok, s_bad;
  __shared__ int s_sel0, s_nsel, s_d0, s_g;
  __shared__ unsigned long long s_off, s_len;
  const int tid = threadIdx.x, lane = tid & 31;
  WsHdr *wsh = reinterpret_cast<WsHdr *>(a.ws);
  const int ngroups = (a.nchunks + a.group - 1) / a.group;
  const int items = a.ids ? a.nblocks : ngroups;
  const int count = TIER == 0 ? items
                              : (int)*(volatile const unsigned *)(TIER == 1 ? &wsh->nbig : &wsh->nbig2);
  const int cap = TIER == 2 ? a.hcap : CAPB;
  for (int it = blockIdx.x; it < count; it += gridDim.x) {
    const int item = TIER == 0 ? it : TIER == 1 ? a.biglist[it] : a.biglist[items + it];
    __syncthreads();  // the previous item's shared words are no longer read
    if (tid < 32) {
      // which group, which of its blocks, and where they go
      int grp = item, sel0 = 0, nsel = 0, d0 = item * a.group;
      unsigned bad = 0;
      if (a.ids) {
        int c = a.ids[item];
        if (c < 0 || c >= a.nchunks) {
          if (lane == 0) atomicCAS(&wsh->status, 0u, ST_ARG);
          c = 0;
          bad = 1;
        }
        grp = c / a.group;
        sel0 = c % a.group;
        nsel = 1;
        d0 = item;
      }
      const int g = min(a.group, a.nchunks - grp * a.group);
      if (!a.ids) nsel = g;
      const unsigned long long *tab = reinterpret_cast<const unsigned long long *>(a.in + HEADER_BYTES);
      const unsigned long long o0 = tab[grp], o1 = tab[grp + 1];
      const unsigned long long avail = a.in_bytes - a.data0;
      const unsigned long long hb = 4ull * (unsigned long long)g + 4ull;
      if (o0 > o1 || o1 > avail || o1 - o0 < hb || (o0 & 3) || ((o1 - o0) & 3)) bad = 1;
      const unsigned *c32 = reinterpret_cast<const unsigned *>(a.in + a.data0 + (bad ? 0ull : o0));
      const unsigned nnz = (!bad && lane < g) ? c32[lane] : 0u;
      if (lane < g && nnz > (unsigned)(G::NVOX - 64)) bad = 1;
      const int w = lane < g ? (64 * ES + G::MASKB + (int)(bad ? 0u : nnz) * ES) / 4 : 0;
      int inc = w;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int v = __shfl_up_sync(FULL, inc, d);
        if (lane >= d) inc += v;
      }
      bad = __ballot_sync(FULL, bad != 0u) ? 1u : 0u;
      const unsigned ntok = bad ? 0u : c32[g];
      if (!bad && (unsigned long long)ntok > (o1 - o0 - hb) / 4) bad = 1;
      if (lane < g) s_nnz[lane] = nnz;
      if (lane <= g) s_w0[lane] = inc - w;
      if (lane == 0) {
        s_bad = bad;
        s_ntok = ntok;
        s_off = o0;
        s_len = o1 - o0;
        s_sel0 = sel0;
        s_nsel = nsel;
        s_d0 = d0;
        s_g = g;
      }
    }
    __syncthreads();
    const int g = s_g, W = s_w0[g], pbytes = 4 * W;
    if (TIER < 2 && !s_bad && pbytes > CAPB) {  // a later tier's group
      if (tid == 0) {
        if (TIER == 0)
          a.biglist[atomicAdd(&wsh->nbig, 1u)] = item;
        else
          a.biglist[items + (int)atomicAdd(&wsh->nbig2, 1u)] = item;
      }
      continue;
    }
    // (a payload larger than the buffer: larger than any valid group of
    // this type)
    bool bad = s_bad != 0u || pbytes > cap;
    if (!bad) {
      const unsigned ntok = s_ntok;
      const unsigned long long hb = 4ull * (unsigned long long)g + 4ull;
      const unsigned long long nlit_avail = (s_len - hb - 4ull * ntok) / 4;
      const unsigned *tok = reinterpret_cast<const unsigned *>(a.in + a.data0 + s_off + hb);
      const unsigned *lit = tok + ntok;
      if (!untoken<NT>(tok, ntok, lit, nlit_avail, reinterpret_cast<unsigned *>(P), (unsigned)W, TL, TO, TK, s_u64))
        atomicOr(&s_bad, 1u);
      __syncthreads();
      bad = s_bad != 0u;
    }
    const int sel0 = s_sel0, nsel = s_nsel, d0 = s_d0;
    if (!bad) {
      // unshuffle the chosen blocks' words into their slots (one flat loop):
      // byte q of the group's raw word k is byte (4k + q) % ES of element
      // (4k + q) / ES
      const int E = pbytes >> LGES, k1 = s_w0[sel0 + nsel];
      for (int k = s_w0[sel0] + tid; k < k1; k += NT) {
        const int i = block_of_word(s_w0, g, k);
        const int e = (4 * k) >> LGES, b0 = (4 * k) & (ES - 1);
        unsigned wv = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) wv |= (unsigned)P[(b0 + q) * E + e] << (8 * q);
        reinterpret_cast<unsigned *>(a.staging + (size_t)(d0 + i - sel0) * a.slot)[k - s_w0[i]] = wv;
      }
    }
    if (tid < nsel) {
      const int d = d0 + tid;
      a.table[2 * d] = bad ? 0ull : (unsigned long long)s_nnz[sel0 + tid];
      a.table[2 * d + 1] = bad ? 1ull : 0ull;
    }
  }
}

}  // namespace czp
