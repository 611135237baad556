// cz_half.cuh -- the block decoder as two independent CTAs per block.
//
// k_decompress_h decodes one z-half of a block per CTA ("unit" u = 2 b + h:
// block b, half h), two CTAs per SM, so that every barrier spans the
// B^2/4 threads of a half and the two CTAs on an SM hide each other's
// barrier waits.  The halves need nothing from each other:
//   * the inverse of the coarser levels works on the coarse cube (all
//     coordinates even), whose inputs are stored coefficients: each CTA
//     scatters its own half of the cube from its registers and reads the
//     other half straight from the payload, then inverts the whole cube;
//   * the level-0 inverse starts with the z-step, whose stencils reach at
//     most two pairs past the middle of a column; those inputs are again
//     stored coefficients (the payload) or level-0 coarse values (the
//     inverted cube), so each thread reads its few halo values itself
//     (W4: two z-planes, W3ai: one, W4li: three or four) and forms the
//     other half's W4li update removal with the same operations the other
//     half uses;
//   * the y- and x-steps stay within the half (a half plane and shuffles).
// Every value is produced by the same operation sequence as in the
// whole-block decoder, so fields are bit-identical to the oracle's.
// Each CTA stores its half tile (B x B x B/2) with one TMA tensor store.
#pragma once

#include "cz_pair.cuh"

namespace czp {

template <typename T, int B>
struct GH {
  using G = G2<T, B>;
  static constexpr int NT = B * B / 4;  // threads of a half CTA
  static constexpr int ES = G::ES, ZH = G::ZH, MH = G::MH, Q = G::Q;
  static constexpr int PLANE = ZH * G::NK * G::HP * 2 * ES;  // half plane
  static constexpr int TILE = B * B * ZH * ES;             // half output tile (holds the plane first)
  static_assert(PLANE <= TILE, "the half plane fits in the half tile");
  static constexpr int CUBE_OFF = TILE;
  static constexpr int ROW_OFF = CUBE_OFF + G::CUBE_AL;
  static constexpr int ROWB_AL = (G::ROWB + 127) / 128 * 128;
  // payload buffers: whole payloads of up to PBCAP bytes (most 32^3 FP32
  // payloads at eps = 1e-3); larger ones read their values from global memory
  static constexpr int PBCAP = G::PMAX_AL < 12288 ? G::PMAX_AL : 12288;
  static constexpr int NPB = 2;
  static constexpr int BUF_OFF = ROW_OFF + ROWB_AL;
  static constexpr int SMEM = BUF_OFF + NPB * PBCAP;
  static constexpr int IPT = B * B / NT;  // mask rows per thread in the row-offset scan
};

// thread (a, k) of a half CTA: x-pair a of row pair k (two row pairs per
// warp for B = 32, four for B = 16)
template <int B>
__device__ __forceinline__ void half_of(int tid, int &a, int &k)
{
  constexpr int HP = B / 2;
  const int w = tid >> 5, lane = tid & 31;
  k = w * (32 / HP) + lane / HP;
  a = lane % HP;
}

// ---- the level-0 inverse z-step of half H with the other half's values
// in registers.  hv[r][s] are the values zsrc<B, H> maps to slot s (the
// ones the whole-block decoder exchanges through its halo).
template <typename T, int B, int KIND, int H, typename T2>
__device__ __forceinline__ void zh_predict(T2 (&v)[2][B / 2], const T2 (&hv)[2][2])
{
  constexpr int MH = B / 4, m = B / 2, lo = H * MH;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    auto src = [&](int j) { return zsrc<B, H>(j, hv[r], [&](int jl) { return v[r][2 * jl]; }); };
    if constexpr (KIND == W3AI) {
      T2 e[MH], o[MH];
#pragma unroll
      for (int jl = 0; jl < MH; ++jl) {
        const AiRow rw = ai_row(lo + jl, m);
        e[jl] = add2(ai_predc<T2, T>(rw, v[r][2 * jl], src(rw.s1), src(rw.s2)), v[r][2 * jl + 1]);
        o[jl] = sub2(add2(v[r][2 * jl], v[r][2 * jl]), e[jl]);
      }
#pragma unroll
      for (int jl = 0; jl < MH; ++jl) {
        v[r][2 * jl] = e[jl];
        v[r][2 * jl + 1] = o[jl];
      }
    } else {
#pragma unroll
      for (int jl = 0; jl < MH; ++jl) {
        const W4Row rw = w4_row(lo + jl, m);
        v[r][2 * jl + 1] =
            add2(v[r][2 * jl + 1], pred4rp<T2, T>(rw, src(rw.j0), src(rw.j0 + 1), src(rw.j0 + 2), src(rw.j0 + 3)));
      }
    }
  }
}

// W4li: remove the update from the even values of half H; hd[r][s] are the
// other half's details zsrc<B, H> maps to slot s
template <typename T, int B, int H, typename T2>
__device__ __forceinline__ void zh_undo(T2 (&v)[2][B / 2], const T2 (&hd)[2][2])
{
  constexpr int MH = B / 4, m = B / 2, lo = H * MH;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    auto src = [&](int j) { return zsrc<B, H>(j, hd[r], [&](int jl) { return v[r][2 * jl + 1]; }); };
    T2 c[MH];
#pragma unroll
    for (int jl = 0; jl < MH; ++jl) {
      const int j = lo + jl;
      const LiSrc ls = li_src(j, m);
      const T uw[3] = {li_lookup<T>(m, j, 0), li_lookup<T>(m, j, 1), li_lookup<T>(m, j, 2)};
      const int k1 = ls.k0 + 1 < m ? ls.k0 + 1 : m - 1, k2 = ls.k0 + 2 < m ? ls.k0 + 2 : m - 1;
      c[jl] = sub2(v[r][2 * jl], li_accp<T2>(uw, ls.nt, src(ls.k0), src(k1), src(k2)));
    }
#pragma unroll
    for (int jl = 0; jl < MH; ++jl) v[r][2 * jl] = c[jl];
  }
}

// W4li: the other half's coarse value j with its update removed, formed as
// that half forms it (zh_undo of half 1 - H); d(i) returns detail i of the
// column (this half's from registers, the other half's from the payload)
template <typename T, int m, typename T2, typename D>
__device__ __forceinline__ T2 li_undone(int j, T2 c, D &&d)
{
  const LiSrc ls = li_src(j, m);
  const T uw[3] = {li_lookup<T>(m, j, 0), li_lookup<T>(m, j, 1), li_lookup<T>(m, j, 2)};
  const int k1 = ls.k0 + 1 < m ? ls.k0 + 1 : m - 1, k2 = ls.k0 + 2 < m ? ls.k0 + 2 : m - 1;
  return sub2(c, li_accp<T2>(uw, ls.nt, d(ls.k0), d(k1), d(k2)));
}

// z-planes of the other half that half H's z-step reads (W4li: details
// and coarse values; the others: coarse values), in the order of the
// `zp` array below, and how many there are
template <int B, int KIND, int H>
struct HaloPlanes {
  static constexpr int M = B / 2;  // the middle of the column
  // W4:   H0: c_{m/2}, c_{m/2+1} at z = M, M+2;   H1: c_{m/2-1} at z = M-2
  // W3ai: H0: a_{m/2} at z = M;                  H1: a_{m/2-1} at z = M-2
  // W4li: H0: z = M, M+1, M+2, M+3 (c, d, c, d);   H1: z = M-3, M-2, M-1 (d, c, d)
  static constexpr int N = KIND == W4LI ? (H == 0 ? 4 : 3) : (KIND == W4 && H == 0 ? 2 : 1);
  static constexpr int z(int q) { return KIND == W4LI ? (H == 0 ? M + q : M - 3 + q) : (H == 0 ? M + 2 * q : M - 2); }
};

template <typename T, int B, int KIND>
__global__ void __launch_bounds__(B * B / 4, 2) k_decompress_h(const __grid_constant__ CUtensorMap omap,
                                                                const InvArgs a)
{
  using G = G2<T, B>;
  using H2 = GH<T, B>;
  using T2 = typename V2T<T>::type;
  static_assert(B >= 16 && !G::SLAB, "half decoder: register-resident blocks of edge 16 or 32");
  constexpr int NT = H2::NT, ES = G::ES, Q = G::Q, ZH = G::ZH, MH = G::MH, N = B / 2;
  constexpr int HEAD = 64 * ES + G::MASKB;  // coarse values + mask
  constexpr int NPB = H2::NPB, PBCAP = H2::PBCAP;
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char *OT = smem;                                            // half output tile [z][y][x]
  T2 *PL = reinterpret_cast<T2 *>(smem);                               // half plane (level-0 y-step)
  T *CB = reinterpret_cast<T *>(smem + H2::CUBE_OFF);                  // cube of the coarser levels
  unsigned *ROWOFF = reinterpret_cast<unsigned *>(smem + H2::ROW_OFF);  // row offsets
  unsigned char *BUF0 = smem + H2::BUF_OFF;                            // NPB payload buffers
  __shared__ __align__(8) unsigned long long s_bar[NPB];
  __shared__ unsigned s_u[40];
  __shared__ unsigned s_nnz[NPB], s_bad[NPB], s_pend[NPB];
  __shared__ unsigned s_badx, s_to;

  WsHdr *ws = reinterpret_cast<WsHdr *>(a.ws);
  const int tid = threadIdx.x, lane = tid & 31;
  const int h = (int)(blockIdx.x & 1u);  // the grid is even: a CTA keeps its half
  int ap, k;
  half_of<B>(tid, ap, k);
  const int seg = lane - ap;
  const int x0 = 2 * ap;
  const int zr = h * ZH + ap;  // z of this thread's two mask rows
  const bool cE = (x0 % Q == 0) && ((2 * k) % Q == 0);  // column (x0, 2k) holds coarse values
  const bool pre = a.stage2 != 0;
  constexpr int FT = NT - 32;  // lane 0 of the last warp: fetches the next block
  const int ub = (int)(blockIdx.x >> 1), us = (int)(gridDim.x >> 1);  // first block, block stride

  // metadata of block b into buffer slot j, and (with stage 2) the start
  // of its payload copy; called by one thread with b's table entry
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
    if (pre && !bad) {
      const int pbytes = HEAD + (int)nnz * ES;
      const int cp = pbytes <= PBCAP ? pbytes : HEAD;
      s_pend[j] = 1u;
      bulk_load(BUF0 + j * PBCAP, a.staging + (size_t)b * a.slot, (unsigned)((cp + 15) & ~15), &s_bar[j]);
    }
    return o0;
  };

  BlockWalk wk;  // coordinates of this CTA's current block (every thread keeps its own)
  wk.init(ub, us, a.nbx, a.nby);
  __shared__ __align__(16) unsigned long long s_tab[2];  // a later block's table entry
  __shared__ unsigned long long s_off[NPB];  // without stage 2: each buffer's chunk offset
  if (tid == 0) {
    for (int q = 0; q < NPB; ++q) {
      mbar_init(&s_bar[q]);
      s_pend[q] = 0;
    }
    s_to = 0;
    s_badx = 0;  // reset again after each block's last read
  }
  __syncthreads();
  if (tid == 0) {
    for (int q = 0; q < NPB - 1; ++q) {
      const int b = ub + q * us;
      if (b < a.nblocks) s_off[q] = fetch(b, q, pre ? a.table[2 * b] : 0ull, pre ? a.table[2 * b + 1] : 0ull);
    }
  }
  __syncthreads();
  unsigned phase = 0;  // bit j: parity of buffer j's next completion
  int j = 0;

  for (int bid = ub; bid < a.nblocks; bid += us, j = j + 1 < NPB ? j + 1 : 0) {
    unsigned char *P = BUF0 + j * PBCAP;
    const int nbid = bid + (NPB - 1) * us;
    const int jn = j == 0 ? NPB - 1 : j - 1;  // (j + NPB - 1) mod NPB
    if (tid == FT && pre && nbid < a.nblocks) cp_async16(s_tab, a.table + 2 * nbid);
    const unsigned nnz = s_nnz[j];
    const int pbytes = HEAD + (int)nnz * ES;
    const bool bad0 = s_bad[j] != 0;
    if (pre) {
      if (!bad0) {
        // a thread whose wait gives up records it and goes on with whatever
        // the buffer holds (in-bounds work, nothing stored before the vote)
        if (!mbar_wait(&s_bar[j], (phase >> j) & 1u))
          s_to = 1u;
        else if (tid == 0)
          s_pend[j] = 0u;
        phase ^= 1u << j;
      }
    } else if (!bad0) {
      const unsigned *c32 = reinterpret_cast<const unsigned *>(a.in + a.data0 + s_off[j]);
      const int cp = pbytes <= PBCAP ? pbytes : HEAD;
      for (int w = tid; w < cp / 4; w += NT) reinterpret_cast<unsigned *>(P)[w] = __ldg(c32 + 2 + w);
      __syncthreads();
    }
    // values beyond the buffer are read from global memory
    const T *VALS = pbytes <= PBCAP
                        ? reinterpret_cast<const T *>(P + HEAD)
                        : (pre ? reinterpret_cast<const T *>(a.staging + (size_t)bid * a.slot + HEAD)
                               : reinterpret_cast<const T *>(a.in + a.data0 + s_off[j] + 8 + HEAD));
    const unsigned char *MASK = P + 64 * ES;
    const T *COARSE = reinterpret_cast<const T *>(P);

    // ---- row offsets of the whole block (rows in stream order, IPT per
    // thread); coarse positions carry no mask bit
    if (!bad0) {
      constexpr int IPT = H2::IPT;
      unsigned loc[IPT], sum = 0;
#pragma unroll
      for (int q = 0; q < IPT; ++q) {
        const int row = tid * IPT + q;
        const unsigned wd = get_rowi<B>(MASK, row);
        loc[q] = __popc(wd);
        sum += loc[q];
        if (((row / B) % Q) == 0 && ((row % B) % Q) == 0) {
          unsigned cm = 0;
#pragma unroll
          for (int x = 0; x < B; x += Q) cm |= 1u << x;
          if (wd & cm) atomicOr(&s_badx, 1u);
        }
      }
      unsigned tot;
      unsigned ex = block_exsum_nb<NT>(sum, s_u, tot);
#pragma unroll
      for (int q = 0; q < IPT; ++q) {
        ROWOFF[rpad_of<B>(tid * IPT + q)] = ex;
        ex += loc[q];
      }
      if (tid == 0 && tot != nnz) atomicOr(&s_badx, 1u);
    }
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
    const bool bad = bad0 || s_badx != 0;
    if (bad && tid == 0) atomicCAS(&ws->status, 0u, ST_CORRUPT);

    // the stored coefficient at block position (x, y, z): a coarse value,
    // a kept detail (mask bit set) or zero; for the pair (x, x + 1), x even
    auto coef2 = [&](int x, int y, int z) {
      const unsigned wd = get_row<B>(MASK, z, y);
      const unsigned base = ROWOFF[rpad<B>(z, y)];
      T2 c;
      c.x = ((wd >> x) & 1u) ? VALS[base + __popc(wd & ((1u << x) - 1u))] : T(0);
      c.y = ((wd >> (x + 1)) & 1u) ? VALS[base + __popc(wd & ((2u << x) - 1u))] : T(0);
      if ((x % Q) == 0 && (y % Q) == 0 && (z % Q) == 0) c.x = COARSE[((z / Q) * 4 + y / Q) * 4 + x / Q];
      return c;
    };

    T2 v[2][ZH];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int zl = 0; zl < ZH; ++zl) {
        v[r][zl].x = T(0);
        v[r][zl].y = T(0);
      }
    // the other half's planes that this half's z-step reads (stored
    // coefficients; the cube column's even entries are replaced by the
    // inverted cube below)
    using HP0 = HaloPlanes<B, KIND, 0>;
    using HP1 = HaloPlanes<B, KIND, 1>;
    constexpr int NHP = HP0::N > HP1::N ? HP0::N : HP1::N;
    T2 hz[2][NHP];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int q = 0; q < NHP; ++q) hz[r][q] = mk2(T(0));
    if (!bad) {
      // this thread's mask rows (z = zr at rows 2k, 2k + 1) transposed over
      // the segment's lanes: its own column bits (bit 2 zl + p: column
      // x0 + p at z = h B/2 + zl)
      unsigned R0, R1;
      get_row_pair<B>(MASK, zr, 2 * k, R0, R1);
      const unsigned W[2] = {seg_transpose<B>(R0, ap), seg_transpose<B>(R1, ap)};
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
#pragma unroll
        for (int zl = 0; zl < ZH; zl += Q) v[0][zl].x = COARSE[(((h * ZH + zl) / Q) * 4 + (2 * k) / Q) * 4 + x0 / Q];
      }
      if (h == 0) {
#pragma unroll
        for (int q = 0; q < HP0::N; ++q)
#pragma unroll
          for (int r = 0; r < 2; ++r) hz[r][q] = coef2(x0, 2 * k + r, HP0::z(q));
      } else {
#pragma unroll
        for (int q = 0; q < HP1::N; ++q)
#pragma unroll
          for (int r = 0; r < 2; ++r) hz[r][q] = coef2(x0, 2 * k + r, HP1::z(q));
      }
    }
    auto fetch_next = [&] {
      if (tid == FT && nbid < a.nblocks) {
        unsigned long long t0 = 0, t1 = 0;
        if (pre) {
          cp_async_wait_all();
          t0 = s_tab[0];
          t1 = s_tab[1];
        }
        s_off[jn] = fetch(nbid, jn, t0, t1);
      }
    };
    if (!bad) {
      // the cube: this half's coarse positions from the registers, the
      // other half's from the payload (column (x0, 2k) at the other half's
      // even z: one mask row word each, a value only where a bit is set)
      to_cube<T, B>(v, CB, ap, k, h);
      const unsigned lowE = (1u << x0) - 1u;
#pragma unroll
      for (int jl = 0; jl < MH; ++jl) {
        const int zc = (1 - h) * MH + jl, z = 2 * zc;
        const unsigned wd = get_row<B>(MASK, z, 2 * k);
        T c = T(0);
        if ((wd >> x0) & 1u) c = VALS[ROWOFF[rpad<B>(z, 2 * k)] + __popc(wd & lowE)];
        if (cE && (z % Q) == 0) c = COARSE[((z / Q) * 4 + (2 * k) / Q) * 4 + x0 / Q];
        CB[cidx<N>(ap, k, zc)] = c;
      }
      __syncthreads();
      if (tid == 0) {
        s_badx = 0;         // every thread has read it
        bulk_wait_read();   // the previous tile store has read the tile area (the plane's, after the cube's barriers)
      }
      fetch_next();
      cube_inv<T, N, KIND, NT>(CB);
      from_cube<T, B>(v, CB, ap, k, h);
      // the cube column's even halo entries: level-0 coarse values
#pragma unroll
      for (int q = 0; q < NHP; ++q) {
        const int zq = h == 0 ? HP0::z(q) : HP1::z(q);
        if (q < (h == 0 ? HP0::N : HP1::N) && (zq & 1) == 0) hz[0][q].x = CB[cidx<N>(ap, k, zq / 2)];
      }
      // ---- level 0: z (registers), y (half plane), x (shuffles)
      if (h == 0) {
        T2 hv[2][2];
        if constexpr (KIND == W4LI) {
          // slots of zsrc<B, 0>: j = m/2, m/2 + 1 (z = M, M + 2); the other
          // half's coarse values with their update removed
          constexpr int M = B / 2, m = B / 2;
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            // details of the column: this half's (odd slots, still
            // unchanged) and the other half's (z = M + 1, M + 3)
            auto d = [&](int i) {
              if (i < m / 2) return v[r][2 * (i - 0) + 1];
              return hz[r][i == m / 2 ? 1 : 3];
            };
            hv[r][0] = li_undone<T, m>(m / 2, hz[r][0], d);
            hv[r][1] = li_undone<T, m>(m / 2 + 1, hz[r][2], d);
            (void)M;
          }
          T2 hd[2][2];
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            hd[r][0] = hz[r][1];
            hd[r][1] = hz[r][3];
          }
          zh_undo<T, B, 0>(v, hd);
        } else if constexpr (KIND == W4) {
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            hv[r][0] = hz[r][0];
            hv[r][1] = hz[r][1];
          }
        } else {
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            hv[r][0] = hz[r][0];
            hv[r][1] = hz[r][0];  // (slot 1 is not read by half 0)
          }
        }
        zh_predict<T, B, KIND, 0>(v, hv);
      } else {
        T2 hv[2][2];
        if constexpr (KIND == W4LI) {
          // slots of zsrc<B, 1>: j = m/2 - 2, m/2 - 1 (z = M - 4, M - 2);
          // only m/2 - 1 is read.  hz: z = M - 3 (d), M - 2 (c), M - 1 (d)
          constexpr int m = B / 2;
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            auto d = [&](int i) {
              if (i >= m / 2) return v[r][2 * (i - m / 2) + 1];
              return hz[r][i == m / 2 - 2 ? 0 : 2];
            };
            hv[r][1] = li_undone<T, m>(m / 2 - 1, hz[r][1], d);
            hv[r][0] = hv[r][1];  // (slot 0 is not read by half 1)
          }
          T2 hd[2][2];
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            hd[r][0] = hz[r][0];
            hd[r][1] = hz[r][2];
          }
          zh_undo<T, B, 1>(v, hd);
        } else {
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            hv[r][1] = hz[r][0];
            hv[r][0] = hz[r][0];  // (slot 0 is not read by half 1)
          }
        }
        zh_predict<T, B, KIND, 1>(v, hv);
      }
      y_inv<T, B, KIND>(v, PL, ap, k, 0);
      x_inv<T, B, KIND>(v, ap, seg);
    } else {
      if (tid == 0) bulk_wait_read();  // the previous tile store has read the tile area
      __syncthreads();                 // every thread has read s_badx
      if (tid == 0) s_badx = 0;
      fetch_next();
    }
    // half block -> output tile -> TMA store, which drains while the next
    // block is decoded
    __syncthreads();  // the plane has been read
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int zl = 0; zl < ZH; ++zl)
        *reinterpret_cast<T2 *>(OT + ((zl * B + 2 * k + r) * B + x0) * ES) = v[r][zl];
    fence_async_smem();
    __syncthreads();
    if (tid == 0) tma_store_tile(&omap, OT, wk.bx * B, wk.by * B, wk.bz * B + h * ZH);
    wk.next();
  }
  if (tid == 0) bulk_wait_all();
}

}  // namespace czp
