// cz_compress.cuh -- compression kernels.
//
// k_stage1 (persistent, static round-robin over blocks): while the TMA unit
// fetches the next block's tile, the CTA transforms the current block in
// registers, selects significant details, and writes the block's payload
//   [64 coarse values | mask row words | kept details in position order]
// either raw or, with stage 2, directly in byte-shuffled order (byte b of
// payload element e at b * E + e; the element size is a power of two, so
// no division is needed).  The CTA then finds the zero-word runs of the
// shuffled payload from a ballot bitmap with one block scan, and the CTA
// writes the finished chunk [nnz | ntok | tokens | literal words] to its own
// staging arena and records (offset, bytes) in the block table.  No CTA
// ever waits for another one.
//
// k_place (one CTA per chunk, ticket order): exclusive prefix of the chunk
// sizes by decoupled look-back, copy of the chunk to its place in the
// stream, offset-table entry; the last chunk writes the stream header.
#pragma once

#include "cz_pair.cuh"

namespace czp {

struct PlaceArgs {
  const unsigned char *staging;
  const unsigned long long *table;
  unsigned char *out;
  unsigned long long *out_bytes;  // may be null
  void *ws;
  unsigned long long out_cap, data0;
  double eps, range;
  int nx, ny, nz, nblocks;
  int block, levels, eps_mode, stage2, kind, dtype;
};

template <typename T, int B, int KIND>
__global__ void __launch_bounds__(B * B / 2, 1) k_stage1(const __grid_constant__ CUtensorMap tmap, const FwdArgs a)
{
  using G = G2<T, B>;
  using T2 = typename V2T<T>::type;
  constexpr int NT = G::NT, ES = G::ES, Q = G::Q, LGES = G::LGES;
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char *PF = smem;
  unsigned char *R2 = smem + G::TILE;
  unsigned char *PS = R2 + G::R2C;
  T *X = reinterpret_cast<T *>(R2);
  T *AD = reinterpret_cast<T *>(R2 + G::XB);
  unsigned *ROWOFF = reinterpret_cast<unsigned *>(R2);
  unsigned char *MASKU = R2 + G::ROWB;  // unshuffled mask rows (for placing values)
  __shared__ __align__(8) unsigned long long s_bar;
  __shared__ unsigned s_u[40];
  __shared__ unsigned long long s_aoff;  // bytes used in this CTA's staging arena

  WsHdr *ws = reinterpret_cast<WsHdr *>(a.ws);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int ap = tid % G::HP, r = tid / G::HP;
  const int y = r < B / 2 ? 2 * r : 2 * (r - B / 2) + 1;
  const int seg = lane - ap;
  const int x0 = 2 * ap;

  double mn, mx, range;
  T t;
  threshold_of<T>(a.eps, a.eps_mode, a.range, ws, mn, mx, range, t);
  const auto tb = thr_bits(t);
  const bool cE = (x0 % Q == 0) && (y % Q == 0);  // this column pair holds coarse values (E)
  unsigned cmask = 0;
#pragma unroll
  for (int z = 0; z < B; z += Q) cmask |= 1u << z;
  unsigned char *arena = a.staging + (size_t)blockIdx.x * a.arena_bytes;

  auto tile_of = [&](int bid) {
    const int bx = bid % a.nbx, by = (bid / a.nbx) % a.nby, bz = bid / (a.nbx * a.nby);
    tma_load_tile(&tmap, PF, &s_bar, bx * B, by * B, bz * B, G::TILE);
  };
  if (tid == 0) {
    s_aoff = 0;
    mbar_init(&s_bar);
    if ((int)blockIdx.x < a.nblocks) tile_of(blockIdx.x);
  }
  __syncthreads();
  unsigned phase = 0;

  for (int bid = blockIdx.x; bid < a.nblocks; bid += gridDim.x) {
    if (!mbar_wait(&s_bar, phase)) {
      // the copy never completed: record, wait once more for it, stop
      if (tid == 0) atomicCAS(&ws->status, 0u, ST_TIMEOUT);
      mbar_wait(&s_bar, phase);
      break;
    }
    phase ^= 1u;

    // ---- a1: tile -> registers; start fetching the next tile
    T2 v[B];
#pragma unroll
    for (int z = 0; z < B; ++z) v[z] = *reinterpret_cast<const T2 *>(PF + ((z * B + y) * B + x0) * ES);
    __syncthreads();
    if (tid == 0 && bid + (int)gridDim.x < a.nblocks) tile_of(bid + gridDim.x);

    // ---- a2: forward transform
    fwd_all<T, B, KIND>(v, X, AD, ap, y, seg);

    // ---- a3: significance bits over z, mask row words by bit transpose
    unsigned me = 0, mo = 0;
#pragma unroll
    for (int z = 0; z < B; ++z) {
      me |= (unsigned)(magbits(v[z].x) >= tb) << z;
      mo |= (unsigned)(magbits(v[z].y) >= tb) << z;
    }
    if (cE) me &= ~cmask;
    unsigned w0 = me, w1 = mo;
    bit_transpose<B>(w0, w1, ap);  // row words of (z = 2ap, y) and (z = 2ap + 1, y)
    __syncthreads();               // planes free: row offsets and mask rows go there
    ROWOFF[(2 * ap) * B + y] = __popc(w0);
    ROWOFF[(2 * ap + 1) * B + y] = __popc(w1);
    put_row<B>(MASKU, 2 * ap, y, w0);
    put_row<B>(MASKU, 2 * ap + 1, y, w1);
    __syncthreads();
    unsigned nnz;
    {
      constexpr int IPT = (B * B + NT - 1) / NT;
      unsigned loc[IPT], sum = 0;
#pragma unroll
      for (int q = 0; q < IPT; ++q) {
        loc[q] = ROWOFF[tid * IPT + q];
        sum += loc[q];
      }
      unsigned ex = block_exsum<NT>(sum, s_u, nnz);
#pragma unroll
      for (int q = 0; q < IPT; ++q) {
        ROWOFF[tid * IPT + q] = ex;
        ex += loc[q];
      }
    }

    // ---- a4: payload, raw or byte-shuffled, in shared memory or (when it
    // does not fit) in this CTA's global scratch
    const int pbytes = 64 * ES + G::MASKB + (int)nnz * ES;
    const int E = pbytes >> LGES;  // elements of the payload
    const int W = pbytes >> 2;     // 32-bit words of the payload
    const int NB = (W + 31) >> 5;  // zero-bitmap words
    const bool in_smem = pbytes <= G::PCAP;
    unsigned char *scr = a.scratch + (size_t)blockIdx.x * a.scratch_per_cta;
    unsigned char *P = in_smem ? PS : scr;
    unsigned *AUX = in_smem ? reinterpret_cast<unsigned *>(MASKU + G::MASKB)
                            : reinterpret_cast<unsigned *>(scr + G::PMAX_AL);
    const int cap = in_smem ? G::NBWC : G::NBWMAX;
    unsigned *ZBM = AUX, *CM = AUX + cap, *EB = AUX + 2 * cap, *PRE = AUX + 3 * cap;
    const bool shuf = a.stage2 != 0;
    // payload byte p -> position (byte p % ES of element p / ES goes to
    // plane p % ES at index p / ES)
    auto put_byte = [&](int p, unsigned char b) {
      if (shuf)
        P[(p & (ES - 1)) * E + (p >> LGES)] = b;
      else
        P[p] = b;
    };
    auto put_val = [&](int e, T val) {  // element e of the payload
      if (shuf) {
        unsigned long long bits;
        if constexpr (ES == 8)
          bits = (unsigned long long)__double_as_longlong(val);
        else
          bits = __float_as_uint(val);
#pragma unroll
        for (int b = 0; b < ES; ++b) P[b * E + e] = (unsigned char)(bits >> (8 * b));
      } else {
        reinterpret_cast<T *>(P)[e] = val;
      }
    };
    {
      constexpr int RB = B / 8;  // bytes of one row word
      const int p0 = 64 * ES + ((2 * ap) * B + y) * B / 8, p1 = 64 * ES + ((2 * ap + 1) * B + y) * B / 8;
#pragma unroll
      for (int q = 0; q < RB; ++q) {
        put_byte(p0 + q, (unsigned char)(w0 >> (8 * q)));
        put_byte(p1 + q, (unsigned char)(w1 >> (8 * q)));
      }
    }
    if (cE) {
#pragma unroll
      for (int z = 0; z < B; z += Q) put_val(((z / Q) * 4 + y / Q) * 4 + x0 / Q, v[z].x);
    }
    {
      // kept details of this column pair, z by z (work grows with the count)
      const int VOFF = (64 * ES + G::MASKB) >> LGES;
      const unsigned lowE = (1u << x0) - 1u, lowO = (2u << x0) - 1u;
      unsigned bits = me | mo;
      while (bits) {
        const int z = __ffs(bits) - 1;
        bits &= bits - 1u;
        const T2 val = pick<B>(v, z);
        const unsigned wd = get_row<B>(MASKU, z, y);
        const unsigned base = ROWOFF[z * B + y];
        if ((me >> z) & 1u) put_val(VOFF + base + __popc(wd & lowE), val.x);
        if ((mo >> z) & 1u) put_val(VOFF + base + __popc(wd & lowO), val.y);
      }
    }
    __syncthreads();

    // ---- a6: zero-word runs of the shuffled payload.  Coded words C are
    // zero words with a zero neighbour; a run starts at S bits and ends
    // before an Eb bit (or at W).  One token per run: (literal words since
    // the previous run, run length); a final (literals, 0) token when the
    // payload does not end in a run.
    const unsigned *P32 = reinterpret_cast<const unsigned *>(P);
    unsigned ns_tot = 0, nc_tot = 0, lastc = 1;
    if (shuf) {
      for (int g = wid; g < NB; g += G::NW) {
        const int w = g * 32 + lane;
        const unsigned bal = __ballot_sync(FULL, w < W && P32[w] == 0u);
        if (lane == 0) ZBM[g] = bal;
      }
      __syncthreads();
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
          const unsigned S = C & ~((C << 1) | cin);
          CM[g] = C;
          EB[g] = ~C & ((C << 1) | cin) & valid;
          mine += (unsigned)__popc(S) | ((unsigned)__popc(C) << 16);
        }
      }
      unsigned tot;
      unsigned run = block_exsum<NT>(mine, s_u, tot);  // packed: runs | coded words << 16
      for (int q = 0; q < KB; ++q) {
        const int g = tid * KB + q;
        if (g < NB) {
          PRE[g] = run;
          const unsigned C = CM[g];
          const unsigned cin = g > 0 ? (CM[g - 1] >> 31) : 0u;
          run += (unsigned)__popc(C & ~((C << 1) | cin)) | ((unsigned)__popc(C) << 16);
        }
      }
      ns_tot = tot & 0xFFFFu;
      nc_tot = tot >> 16;
      lastc = (ZBM[NB - 1] >> ((W - 1) & 31)) & 1u;  // last word zero ...
      if (lastc) {                                     // ... and coded?
        const int l = W - 1;
        const bool prevz = l > 0 && ((ZBM[(l - 1) >> 5] >> ((l - 1) & 31)) & 1u);
        lastc = prevz ? 1u : 0u;
      }
      __syncthreads();
    }
    const unsigned ntok = shuf ? ns_tot + (lastc ? 0u : 1u) : 0u;
    const unsigned nlit = shuf ? (unsigned)W - nc_tot : 0u;
    const unsigned long long size = shuf ? 8ull + 4ull * ntok + 4ull * nlit : 8ull + (unsigned long long)pbytes;

    // ---- finished chunk -> this CTA's staging arena
    const unsigned long long so = s_aoff;
    const bool ok = so + size <= a.arena_bytes;
    if (tid == 0) {
      if (!ok) atomicCAS(&ws->status, 0u, ST_CAPACITY);
      a.table[2 * bid] = (unsigned long long)(arena - a.staging) + so;
      a.table[2 * bid + 1] = ok ? size : 0xFFFFFFFFFFFFFFFFull;
    }
    if (ok) {
      unsigned *ch = reinterpret_cast<unsigned *>(arena + so);
      if (tid == 0) {
        ch[0] = nnz;
        ch[1] = ntok;
      }
      if (shuf) {
        unsigned *tok = ch + 2;
        unsigned *lit = tok + ntok;
        const int KB = (NB + NT - 1) / NT;
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
            // previous run end (or 0) and this run's end (or W)
            int pe = 0, ne = W;
            const unsigned below = Eb & ((1u << b) - 1u), above = Eb & ~((2u << b) - 1u);
            if (below) {
              pe = g * 32 + 31 - __clz(below);
            } else {
              for (int h = g - 1; h >= 0; --h)
                if (EB[h]) {
                  pe = h * 32 + 31 - __clz(EB[h]);
                  break;
                }
            }
            if (above) {
              ne = g * 32 + __ffs(above) - 1;
            } else {
              for (int h = g + 1; h < NB; ++h)
                if (EB[h]) {
                  ne = h * 32 + __ffs(EB[h]) - 1;
                  break;
                }
            }
            tok[k] = (unsigned)(p - pe) | ((unsigned)(ne - p) << 16);
            if (k + 1 == ns_tot && !lastc) tok[k + 1] = (unsigned)(W - ne);  // trailing literals
            ++k;
          }
        }
        if (tid == 0 && ns_tot == 0) tok[0] = (unsigned)W;  // no run at all
        for (int w = tid; w < W; w += NT) {
          const int g = w >> 5, b = w & 31;
          const unsigned C = CM[g];
          if (!((C >> b) & 1u)) lit[(unsigned)w - ((PRE[g] >> 16) + __popc(C & ((1u << b) - 1u)))] = P32[w];
        }
      } else {
        for (int w = tid; w < W; w += NT) ch[2 + w] = P32[w];
      }
    }
    __syncthreads();
    if (tid == 0 && ok) s_aoff = so + ((size + 15) & ~15ull);
  }
}

// ---- chunk placement: offsets by decoupled look-back, copy, header
template <typename T>
__global__ void __launch_bounds__(128) k_place(const PlaceArgs a)
{
  __shared__ int s_bid;
  __shared__ unsigned long long s_excl;
  WsHdr *ws = reinterpret_cast<WsHdr *>(a.ws);
  unsigned long long *lbst = reinterpret_cast<unsigned long long *>((char *)a.ws + WS_HDR);
  const int tid = threadIdx.x;
  if (tid == 0) s_bid = (int)atomicAdd(&ws->ticket, 1u);  // predecessors are resident or done
  __syncthreads();
  const int bid = s_bid;
  const unsigned long long so = a.table[2 * bid], sz0 = a.table[2 * bid + 1];
  const bool lost = sz0 == 0xFFFFFFFFFFFFFFFFull;  // staging overflowed for this chunk
  const unsigned long long size = lost ? 0ull : sz0;
  if (tid < 32) {
    const unsigned long long ex = lookback(lbst, bid, size, &ws->status, (int)ST_TIMEOUT);
    if (tid == 0) s_excl = ex;
  }
  __syncthreads();
  const unsigned long long excl = s_excl;
  const bool fits = !lost && a.data0 + excl + size <= a.out_cap;
  if (tid == 0) {
    st_le<unsigned long long>(a.out + HEADER_BYTES + 8ull * bid, excl);
    if (!fits) atomicCAS(&ws->status, 0u, ST_CAPACITY);
    if (bid == a.nblocks - 1) {
      double mn, mx, range;
      T t;
      threshold_of<T>(a.eps, a.eps_mode, a.range, ws, mn, mx, range, t);
      const unsigned long long data_bytes = excl + size, total = a.data0 + data_bytes;
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
      st_le<unsigned>(h + 28, (unsigned)a.nblocks);
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
  if (fits) {
    const uint4 *src = reinterpret_cast<const uint4 *>(a.staging + so);
    unsigned *dst = reinterpret_cast<unsigned *>(a.out + a.data0 + excl);
    const unsigned nw = (unsigned)(size >> 2);
    // staging chunks are 16-byte aligned; destinations only 4-byte aligned
    for (unsigned q = tid; q < (nw >> 2); q += blockDim.x) {
      const uint4 u = src[q];
      dst[4 * q] = u.x;
      dst[4 * q + 1] = u.y;
      dst[4 * q + 2] = u.z;
      dst[4 * q + 3] = u.w;
    }
    const unsigned *s32 = reinterpret_cast<const unsigned *>(src);
    for (unsigned q = (nw & ~3u) + tid; q < nw; q += blockDim.x) dst[q] = s32[q];
  }
}

}  // namespace czp
