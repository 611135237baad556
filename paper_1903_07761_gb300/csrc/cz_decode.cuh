// cz_decode.cuh -- the block decoder with the next block's row offsets
// computed while the coarser levels run.
//
// k_decompress3 decodes one 32^3 FP32 block per CTA of B^2/2 threads, as
// k_decompress2 does, with the same arithmetic in the same order (fields
// are bit-identical to the oracle's).  The difference is the schedule: the
// inverse of the coarser levels takes one cube line per thread, which keeps
// only the first (B/2)^2 threads ("cube threads") busy.  Meanwhile the other
// threads ("row threads") wait for the NEXT block's payload, compute its
// row offsets (popcounts of its mask rows and one scan over the row
// threads) into the second of two row-offset tables, and flag its coarse
// positions; the cube passes synchronise with a named barrier over the cube
// threads only.  The next block then starts with its scatter: the row
// offsets and their scan, with their barriers, are off the critical path.
//
// Timeouts: a thread whose bounded wait for a payload gives up records it
// in s_to and does nothing with that payload; the CTA reads s_to only after
// a barrier that follows every such write, and stops as one.
#pragma once

#include "cz_pair.cuh"

namespace czp {

// exclusive prefix of v over the NTS threads of one group (whole warps,
// gtid = thread index within the group), one named barrier ID; tmp (>=
// NTS/32 words) must not be written again before the group's next barrier
template <int NTS, int ID, typename U>
__device__ __forceinline__ U group_exsum_nb(U v, U *tmp, U &total, int gtid)
{
  constexpr int NWP = NTS / 32;
  const int lane = gtid & 31, wid = gtid >> 5;
  const U inc = warp_incl_sum(v);
  if (lane == 31) tmp[wid] = inc;
  named_sync<ID, NTS>();
  const U t = lane < NWP ? tmp[lane] : U(0);
  const U ti = warp_incl_sum(t);
  const U before = __shfl_sync(FULL, ti - t, wid);
  total = __shfl_sync(FULL, ti, NWP - 1);
  return before + inc - v;
}

template <typename T, int B>
struct GD {
  using G = G2<T, B>;
  static constexpr int NT = G::NT;
  static constexpr int CT = (B / 2) * (B / 2);  // cube threads: one level-1 line each
  static constexpr int RT = NT - CT;            // row threads
  static constexpr int RPT = B * B / RT;        // mask rows per row thread
  static constexpr int ROWB_AL = (G::ROWB + 127) / 128 * 128;
  static constexpr int NPB = G::NPB;
  static constexpr int PBCAP = G::PBCAP;
  static constexpr int BUF_OFF = G::CUBE_AL + 2 * ROWB_AL;
  static constexpr int OT_OFF = BUF_OFF + NPB * PBCAP;
  static constexpr int OTB = (G::TILE > G::PLANE + G::HALO ? G::TILE : G::PLANE + G::HALO + 127) / 128 * 128;
  static constexpr int SMEM = OT_OFF + OTB;
};

template <typename T, int B, int KIND>
__global__ void __launch_bounds__(B * B / 2, 1) k_decompress3(const __grid_constant__ CUtensorMap omap,
                                                              const InvArgs a)
{
  using G = G2<T, B>;
  using D = GD<T, B>;
  using T2 = typename V2T<T>::type;
  static_assert(B == 32 && !G::SLAB, "the overlapped decoder serves register-resident 32^3 blocks");
  constexpr int NT = G::NT, ES = G::ES, Q = G::Q, ZH = G::ZH, N = B / 2;
  constexpr int CT = D::CT, RT = D::RT, RPT = D::RPT, NPB = D::NPB, PBCAP = D::PBCAP;
  static_assert(CT % 32 == 0 && RT % 32 == 0 && RT * RPT == B * B, "thread groups");
  constexpr int HEAD = 64 * ES + G::MASKB;  // coarse values + mask
  constexpr int RW = D::ROWB_AL / 4;         // words of one row-offset table
  extern __shared__ __align__(128) unsigned char smem[];
  T *CB = reinterpret_cast<T *>(smem);                               // cube of the coarser levels
  unsigned *ROWS = reinterpret_cast<unsigned *>(smem + G::CUBE_AL);  // two row-offset tables
  unsigned char *BUF0 = smem + D::BUF_OFF;                           // NPB payload buffers
  unsigned char *OT = smem + D::OT_OFF;                              // output tile [z][y][x]
  T2 *PL = reinterpret_cast<T2 *>(OT);  // level-0 plane and halo, inside the tile area
  T2 *HX = reinterpret_cast<T2 *>(OT + G::PLANE);
  __shared__ __align__(8) unsigned long long s_bar[NPB];
  __shared__ unsigned s_u[40];
  __shared__ unsigned s_nnz[NPB], s_bad[NPB], s_pend[NPB];
  __shared__ unsigned s_badx[2], s_to;

  WsHdr *ws = reinterpret_cast<WsHdr *>(a.ws);
  const int tid = threadIdx.x, lane = tid & 31;
  int ap, k, h;
  quad_of<B>(tid, ap, k, h);
  const int seg = lane - ap;
  const int x0 = 2 * ap;
  const int zr = h * ZH + ap;  // z of this thread's two mask rows
  const bool cE = (x0 % Q == 0) && ((2 * k) % Q == 0);  // column (x0, 2k) holds coarse values
  const bool pre = a.stage2 != 0;  // decoded payloads sit in 16-byte aligned slots
  constexpr int FT = NT - 32;      // lane 0 of the last warp (a row thread): fetches ahead
  const int G_ = (int)gridDim.x;

  // metadata of block b into buffer slot j, and (with stage 2) the start of
  // its payload copy; called by one thread with b's table entry
  __shared__ unsigned long long s_off[NPB];  // without stage 2: each buffer's chunk offset
  auto fetch = [&](int b, int j, unsigned long long t0, unsigned long long t1) {
    unsigned bad = 0, nnz = 0;
    unsigned long long o0 = 0;
    if (pre) {  // decoded (and checked) by k_unstage
      bad = t1 != 0;
      nnz = bad ? 0u : (unsigned)t0;
    } else {
      const unsigned long long *tab = reinterpret_cast<const unsigned long long *>(a.in + HEADER_BYTES);
      int c = a.ids ? a.ids[b] : b;  // the block's chunk in the stream
      if (c < 0 || c >= a.nchunks) {
        atomicCAS(&ws->status, 0u, ST_ARG);
        c = 0;
        bad = 1;
      }
      o0 = tab[c];
      const unsigned long long o1 = tab[c + 1];
      const unsigned long long avail = a.in_bytes - a.data0;
      if (bad || o0 > o1 || o1 > avail || o1 - o0 < 8 || (o0 & 3) || ((o1 - o0) & 3)) {
        bad = 1;
      } else {
        const unsigned *c32 = reinterpret_cast<const unsigned *>(a.in + a.data0 + o0);
        nnz = c32[0];
        if (nnz > (unsigned)(G::NVOX - 64)) bad = 1;
        const unsigned long long pb = 64ull * ES + G::MASKB + (unsigned long long)nnz * ES;
        if (!bad && (c32[1] != 0 || 8 + pb > o1 - o0)) bad = 1;
      }
    }
    s_bad[j] = bad;
    s_nnz[j] = bad ? 0u : nnz;
    s_off[j] = o0;
    if (pre && !bad) {
      const int pbytes = HEAD + (int)nnz * ES;
      const int cp = pbytes <= PBCAP ? pbytes : HEAD;
      s_pend[j] = 1u;
      bulk_load(BUF0 + j * PBCAP, a.staging + (size_t)b * a.slot, (unsigned)((cp + 15) & ~15), &s_bar[j]);
    }
  };

  unsigned phase = 0;  // bit j: parity of buffer j's next completion (the same in every thread)

  // row threads only: block b's payload (buffer jb; without stage 2 they
  // copy it there first), its row offsets into table `slot`, and its
  // coarse-position check into s_badx[slot]
  auto rows = [&](int b, int jb, int slot) {
    const int t = tid - CT;
    if (b >= a.nblocks || s_bad[jb]) return;  // the same in every row thread
    unsigned char *Pb = BUF0 + jb * PBCAP;
    const int pbytes = HEAD + (int)s_nnz[jb] * ES;
    if (pre) {
      // no phase flip here: every thread waits for this completion again
      // when block b comes (it has happened by then).  A thread that gives
      // up goes on (in-bounds work on whatever the buffer holds, so that the
      // named barrier below sees every row thread); block b is never used.
      if (!mbar_wait(&s_bar[jb], (phase >> jb) & 1u)) s_to = 1u;
    } else {
      const unsigned *c32 = reinterpret_cast<const unsigned *>(a.in + a.data0 + s_off[jb]);
      const int cp = pbytes <= PBCAP ? pbytes : HEAD;
      for (int w = t; w < cp / 4; w += RT) reinterpret_cast<unsigned *>(Pb)[w] = __ldg(c32 + 2 + w);
      named_sync<2, RT>();
    }
    const unsigned char *MASKb = Pb + 64 * ES;
    unsigned *RO = ROWS + slot * RW;
    unsigned loc[RPT], sum = 0;
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const int row = t * RPT + q;
      const unsigned wd = get_rowi<B>(MASKb, row);
      loc[q] = __popc(wd);
      sum += loc[q];
      if (((row / B) % Q) == 0 && ((row % B) % Q) == 0) {
        unsigned cm = 0;
#pragma unroll
        for (int x = 0; x < B; x += Q) cm |= 1u << x;
        if (wd & cm) atomicOr(&s_badx[slot], 1u);
      }
    }
    unsigned tot;
    unsigned ex = group_exsum_nb<RT, 2>(sum, s_u, tot, t);
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      RO[rpad_of<B>(t * RPT + q)] = ex;
      ex += loc[q];
    }
    if (t == 0 && tot != s_nnz[jb]) atomicOr(&s_badx[slot], 1u);
  };

  BlockWalk wk;  // coordinates of this CTA's current block (every thread keeps its own)
  wk.init(blockIdx.x, G_, a.nbx, a.nby);
  if (tid == 0) {
    for (int q = 0; q < NPB; ++q) {
      mbar_init(&s_bar[q]);
      s_pend[q] = 0;
    }
    s_to = 0;
    s_badx[0] = s_badx[1] = 0;
  }
  __syncthreads();
  if (tid == 0) {
    for (int q = 0; q < NPB - 1; ++q) {
      const int b = blockIdx.x + q * G_;
      if (b < a.nblocks) fetch(b, q, pre ? a.table[2 * b] : 0ull, pre ? a.table[2 * b + 1] : 0ull);
    }
  }
  __syncthreads();
  if (tid >= CT) rows(blockIdx.x, 0, 0);
  __syncthreads();
  __shared__ __align__(16) unsigned long long s_tab[2];  // a later block's table entry
  int j = 0, slot = 0;

  for (int bid = blockIdx.x; bid < a.nblocks; bid += G_, j = j + 1 < NPB ? j + 1 : 0, slot ^= 1) {
    unsigned char *P = BUF0 + j * PBCAP;
    const int nbid = bid + (NPB - 1) * G_;      // the block whose copy this one starts
    const int jn = j == 0 ? NPB - 1 : j - 1;    // its buffer: (j + NPB - 1) mod NPB
    const int j1 = j + 1 < NPB ? j + 1 : 0;     // the next block's buffer
    if (tid == FT && pre && nbid < a.nblocks) cp_async16(s_tab, a.table + 2 * nbid);
    if (tid == 0) s_badx[slot ^ 1] = 0;  // the next block's flags (last read in the previous block)
    const unsigned nnz = s_nnz[j];
    const int pbytes = HEAD + (int)nnz * ES;
    const bool bad0 = s_bad[j] != 0;
    bool mine = true;  // this thread has seen the payload complete
    if (pre && !bad0) {
      if (!mbar_wait(&s_bar[j], (phase >> j) & 1u)) {
        s_to = 1u;
        mine = false;
      } else if (tid == 0) {
        s_pend[j] = 0u;
      }
      phase ^= 1u << j;
    }
    // values beyond the buffer are read from global memory
    const T *VALS = pbytes <= PBCAP
                        ? reinterpret_cast<const T *>(P + HEAD)
                        : (pre ? reinterpret_cast<const T *>(a.staging + (size_t)bid * a.slot + HEAD)
                               : reinterpret_cast<const T *>(a.in + a.data0 + s_off[j] + 8 + HEAD));
    const unsigned char *MASK = P + 64 * ES;
    const unsigned *ROWOFF = ROWS + slot * RW;
    const bool bad = bad0 || s_badx[slot] != 0;  // written before the previous barrier
    if (bad && tid == 0) atomicCAS(&ws->status, 0u, ST_CORRUPT);

    // this thread's mask rows (z = zr at rows 2k, 2k + 1) and, transposed
    // over the segment's lanes (every lane takes part), its column bits
    unsigned R0 = 0, R1 = 0;
    if (!bad && mine) get_row_pair<B>(MASK, zr, 2 * k, R0, R1);
    const unsigned W[2] = {seg_transpose<B>(R0, ap), seg_transpose<B>(R1, ap)};
    T2 v[2][ZH];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int zl = 0; zl < ZH; ++zl) {
        v[r][zl].x = T(0);
        v[r][zl].y = T(0);
      }
    if (!bad && mine) {
      const unsigned lowE = (1u << x0) - 1u, lowO = (2u << x0) - 1u;
      if (W[0] | W[1]) {
#pragma unroll
        for (int zl = 0; zl < ZH; ++zl) {
          const int z = h * ZH + zl;
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            const unsigned b2 = (W[r] >> (2 * zl)) & 3u;
            if (b2) {
              const unsigned wd = get_row<B>(MASK, z, 2 * k + r);
              const unsigned base = ROWOFF[rpad<B>(z, 2 * k + r)];
              if (b2 & 1u) v[r][zl].x = VALS[base + __popc(wd & lowE)];
              if (b2 & 2u) v[r][zl].y = VALS[base + __popc(wd & lowO)];
            }
          }
        }
      }
      if (cE) {
        const T *COARSE = reinterpret_cast<const T *>(P);
#pragma unroll
        for (int zl = 0; zl < ZH; zl += Q) v[0][zl].x = COARSE[(((h * ZH + zl) / Q) * 4 + (2 * k) / Q) * 4 + x0 / Q];
      }
    }
    // the next block's payload copy (row thread FT) and row offsets (row
    // threads), after a barrier that follows every thread's use of this
    // block's s_badx slot's twin
    auto ahead = [&] {
      if (tid == FT && nbid < a.nblocks) {
        unsigned long long t0 = 0, t1 = 0;
        if (pre) {
          cp_async_wait_all();
          t0 = s_tab[0];
          t1 = s_tab[1];
        }
        fetch(nbid, jn, t0, t1);
      }
      rows(bid + G_, j1, slot ^ 1);
    };
    if (!bad) {
      to_cube<T, B>(v, CB, ap, k, h);
      __syncthreads();
      if (*(volatile unsigned *)&s_to) {
        // a payload copy never arrived (in some thread's view): the whole CTA
        // stops here, after waiting once more, bounded, for every copy it
        // started that has not been seen complete, and for its tile stores
        if (tid == 0) {
          atomicCAS(&ws->status, 0u, ST_TIMEOUT);
          for (int q = 0; q < NPB; ++q)
            if (s_pend[q]) mbar_wait(&s_bar[q], ((phase >> q) & 1u) ^ (q == j ? 1u : 0u));
          bulk_wait_all();
        }
        return;
      }
      if (tid < CT) {
        // the previous block's tile store has read the tile area (the plane
        // and halo are written after the barrier below)
        if (tid == 0) bulk_wait_read();
        cube_inv<T, N, KIND, CT, 1, CT>(CB);
      } else {
        ahead();
      }
      __syncthreads();
      from_cube<T, B>(v, CB, ap, k, h);
      z_inv<T, B, KIND>(v, HX, k, ap, h);
      y_inv<T, B, KIND>(v, PL, ap, k, h);
      x_inv<T, B, KIND>(v, ap, seg);
    } else {
      if (tid == 0) bulk_wait_read();
      __syncthreads();
      if (*(volatile unsigned *)&s_to) {
        if (tid == 0) {
          atomicCAS(&ws->status, 0u, ST_TIMEOUT);
          for (int q = 0; q < NPB; ++q)
            if (s_pend[q]) mbar_wait(&s_bar[q], ((phase >> q) & 1u) ^ (q == j ? 1u : 0u));
          bulk_wait_all();
        }
        return;
      }
      if (tid >= CT) ahead();
    }
    // block -> output tile -> TMA store, which drains while the next block
    // is decoded
    __syncthreads();  // the plane and the halo have been read
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int zl = 0; zl < ZH; ++zl)
        *reinterpret_cast<T2 *>(OT + (((h * ZH + zl) * B + 2 * k + r) * B + x0) * ES) = v[r][zl];
    fence_async_smem();
    __syncthreads();
    if (tid == 0) tma_store_tile(&omap, OT, wk.bx * B, wk.by * B, wk.bz * B);
    wk.next();
  }
  if (tid == 0) bulk_wait_all();
}

}  // namespace czp
