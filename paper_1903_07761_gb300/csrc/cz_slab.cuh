// cz_slab.cuh -- blocks of 32^3 FP64 (256 KiB) and 64^3 FP32 (1 MiB):
// kernels whose block lives in global memory.
//
// Such a block holds more bytes than a CTA's shared memory and than the
// register file of an SM, so the register-resident kernels of cz_pair.cuh
// cannot take it.  Here a CTA works on a block held in global
// memory: its own scratch block when compressing (written by the first
// pass, which reads the field; L2-resident, one per CTA), the output block
// of the field itself when decompressing.  The transform is the same as
// everywhere else (Sec. 2.2, Eqs. 1-7; per level the x-, then y-, then
// z-lines of the current coarse cube): every pass gives one thread a whole
// line, which it transforms in registers with the line functions of
// cz_device.cuh (fwd_reg / inv_reg, the same rounded operations in the same
// order as the oracle), and writes back in place.  The last two levels
// (edges 16 and 8) move to a 16^3 cube in shared memory and take the cube
// passes of cz_pair.cuh.  Significance, mask rows and compaction go one warp per
// x-row (lane = x): a ballot is the row's mask word.
//
// GB300's FP64 pipe is far slower than its FP32 pipe, so FP64 blocks are
// bound by FP64 instructions, not by memory: the extra L2 traffic of the
// global block costs little.  64^3 blocks serve the block-size study
// (Sec. 3, Exp. 3).  Stage 2 of payloads too large for shared
// memory (k_stage2_huge, and k_unstage's large launch) shuffles in a
// global scratch block per CTA as well.
#pragma once

#include "cz_compress.cuh"
#include "cz_pair.cuh"

namespace czp {

template <typename T, int B>
struct SG {
  static constexpr int NT = 256;       // threads per CTA
  static constexpr int NW = NT / 32;   // warps
  static constexpr int ROWS = B * B;   // x-rows of a block
  static constexpr int RPT = ROWS / NT;  // rows per thread in the row scans
  static constexpr int MWPR = B / 32;  // 32-bit mask words per x-row
  static constexpr int Q = B / 4;      // spacing of the coarse values
  static constexpr int ES = (int)sizeof(T);
  static constexpr int HEAD = 64 * ES + B * B * B / 8;  // coarse values + mask
  // the last levels (edge 16 and 8) run on a 16^3 cube in shared memory,
  // the positions that are multiples of S0 = B / 16
  static constexpr int NC = 16, S0 = B / NC;
  static constexpr int CUBE = NC * NC * (NC + 1) * ES;
  static constexpr int CUBE_AL = (CUBE + 127) / 128 * 128;
  // shared memory: cube | mask words | row offsets
  static constexpr int SMEM = CUBE_AL + ROWS * MWPR * 4 + ROWS * 4;
  static constexpr int MINB = B == 64 ? 1 : 2;  // CTAs per SM (registers: a line of B values)
  // the warp-per-row loops take RB rows per round: their loads are all
  // issued before the first one is used (one memory round trip per RB rows)
  static constexpr int RB = 8;
  // (checked where a slab kernel is instantiated: whole 32-bit mask words
  // per row with the lanes on x, whole rows per thread)
  static constexpr bool OK = (B == 32 || B == 64) && ROWS % NT == 0;
  // global scratch per CTA of the stage kernel: the lane's scratch block
  // (room for the largest payload too) where the slab kernels are the
  // lane's own, one block otherwise (FP32 32^3, where the batch tuner may
  // pick them instead of the register-resident kernels)
  static constexpr size_t SCR = G2<T, B>::SLAB ? (size_t)G2<T, B>::SCRATCH : (size_t)B * B * B * ES;
};

// element (x, y, z) of a B^3 block inside a dense array
template <typename T>
struct BView {
  T *p;
  long long sy, sz;
  __device__ __forceinline__ T &at(int x, int y, int z) const { return p[z * sz + y * sy + x]; }
};

// ---- the finest x-lines (rows): read from src (the field, or the block
// itself), written to dst; rows are contiguous, so they move as 16-byte
// vectors
template <typename T, int B, int KIND, bool FWD, int NT>
__device__ __forceinline__ void slab_x(const T *src, long long ssy, long long ssz, const BView<T> &dst)
{
  using T2 = typename V2T<T>::type;
#pragma unroll 1
  for (int r = threadIdx.x; r < B * B; r += NT) {
    const int z = r / B, y = r % B;
    const T2 *s = reinterpret_cast<const T2 *>(src + z * ssz + y * ssy);
    T e[B];
#pragma unroll
    for (int i = 0; i < B / 2; ++i) {
      const T2 q = s[i];
      e[2 * i] = q.x;
      e[2 * i + 1] = q.y;
    }
    if constexpr (FWD)
      fwd_reg<T, KIND, B, 1>(e);
    else
      inv_reg<T, KIND, B, 1>(e);
    T2 *d = reinterpret_cast<T2 *>(&dst.at(0, y, z));
#pragma unroll
    for (int i = 0; i < B / 2; ++i) {
      T2 q;
      q.x = e[2 * i];
      q.y = e[2 * i + 1];
      d[i] = q;
    }
  }
}

// ---- one axis of the level of stride S (n = B / S points per line): one
// line per thread, lines dealt round robin; for y- and z-lines consecutive
// threads take consecutive x.  W4 changes only the odd points.
template <typename T, int B, int KIND, bool FWD, int NT, int AXIS, int S>
__device__ __forceinline__ void slab_pass(const BView<T> &v)
{
  constexpr int n = B / S;
  const long long st = AXIS == 0 ? S : (AXIS == 1 ? S * v.sy : S * v.sz);
#pragma unroll 1
  for (int r = threadIdx.x; r < n * n; r += NT) {
    const int f = (r % n) * S, g = (r / n) * S;  // the line's two other coordinates
    T *base = AXIS == 0 ? &v.at(0, f, g) : (AXIS == 1 ? &v.at(f, 0, g) : &v.at(f, g, 0));
    T e[n];
#pragma unroll
    for (int i = 0; i < n; ++i) e[i] = base[i * st];
    if constexpr (FWD)
      fwd_reg<T, KIND, n, 1>(e);
    else
      inv_reg<T, KIND, n, 1>(e);
#pragma unroll
    for (int i = 0; i < n; ++i)
      if (KIND != W4 || (i & 1)) base[i * st] = e[i];
  }
}

// the last levels: the 16^3 values at multiples of S -> shared-memory cube
// -> cube passes (edges 16 and 8) -> back
template <typename T, int B, int KIND, bool FWD, int NT, int S>
__device__ __forceinline__ void slab_cube(const BView<T> &v, T *C)
{
  constexpr int N = B / S;
  static_assert(N == 16, "the shared-memory cube holds the edge-16 level");
  for (int i = threadIdx.x; i < N * N * N; i += NT) {
    const int x = i % N, y = (i / N) % N, z = i / (N * N);
    C[cidx<N>(x, y, z)] = v.at(S * x, S * y, S * z);
  }
  __syncthreads();
  if constexpr (FWD)
    cube_fwd<T, N, KIND, NT>(C);
  else
    cube_inv<T, N, KIND, NT>(C);
  for (int i = threadIdx.x; i < N * N * N; i += NT) {
    const int x = i % N, y = (i / N) % N, z = i / (N * N);
    v.at(S * x, S * y, S * z) = C[cidx<N>(x, y, z)];
  }
  __syncthreads();
}

// levels of stride S and coarser (the finest x-lines already done when S = 1)
template <typename T, int B, int KIND, int NT, int S>
__device__ __forceinline__ void slab_fwd_from(const BView<T> &v, T *C)
{
  if constexpr (B / S > 16) {
    if constexpr (S > 1) {
      slab_pass<T, B, KIND, true, NT, 0, S>(v);
      __syncthreads();
    }
    slab_pass<T, B, KIND, true, NT, 1, S>(v);
    __syncthreads();
    slab_pass<T, B, KIND, true, NT, 2, S>(v);
    __syncthreads();
    slab_fwd_from<T, B, KIND, NT, 2 * S>(v, C);
  } else {
    slab_cube<T, B, KIND, true, NT, S>(v, C);
  }
}

template <typename T, int B, int KIND, int NT, int S>
__device__ __forceinline__ void slab_inv_from(const BView<T> &v, T *C)
{
  if constexpr (B / S > 16) {
    slab_inv_from<T, B, KIND, NT, 2 * S>(v, C);
    slab_pass<T, B, KIND, false, NT, 2, S>(v);
    __syncthreads();
    slab_pass<T, B, KIND, false, NT, 1, S>(v);
    __syncthreads();
    if constexpr (S == 1)
      slab_x<T, B, KIND, false, NT>(v.p, v.sy, v.sz, v);
    else
      slab_pass<T, B, KIND, false, NT, 0, S>(v);
    __syncthreads();
  } else {
    slab_cube<T, B, KIND, false, NT, S>(v, C);
  }
}

// whole forward transform: field block (src) -> v (every value rewritten);
// per level the x-, y- and z-lines (Sec. 2.2)
template <typename T, int B, int KIND, int NT>
__device__ __forceinline__ void slab_fwd(const T *src, long long ssy, long long ssz, const BView<T> &v, T *C)
{
  slab_x<T, B, KIND, true, NT>(src, ssy, ssz, v);
  __syncthreads();
  slab_fwd_from<T, B, KIND, NT, 1>(v, C);
}

// whole inverse transform in place (levels from the coarsest, axes z, y, x)
template <typename T, int B, int KIND, int NT>
__device__ __forceinline__ void slab_inv(const BView<T> &v, T *C)
{
  slab_inv_from<T, B, KIND, NT, 1>(v, C);
}

// ---- compression: the same slot as k_stage1 writes
//   [nnz | 0 | 64 coarse values | mask row words | kept details in position order]
// NF = 1: one field described by a; NF > 1: fields of one batched group
template <typename T, int B, int KIND, int NF>
__global__ void __launch_bounds__(SG<T, B>::NT, SG<T, B>::MINB) k_stage1_slab(
    const __grid_constant__ StageMaps<NF> maps, const FwdArgs a)
{
  static_assert(SG<T, B>::OK, "slab geometry: B = 32 or 64");
  using S = SG<T, B>;
  using G = G2<T, B>;
  constexpr int NT = S::NT, NW = S::NW, Q = S::Q, ES = S::ES, ROWS = S::ROWS, RPT = S::RPT, MWPR = S::MWPR,
                RB = S::RB;
  static_assert(ROWS % (NW * RB) == 0, "whole rounds of RB rows per warp");
  extern __shared__ __align__(128) unsigned char smem[];
  T *C = reinterpret_cast<T *>(smem);
  unsigned *MW = reinterpret_cast<unsigned *>(smem + S::CUBE_AL);  // mask words (MWPR per row)
  unsigned *RO = MW + ROWS * MWPR;                                   // row offsets
  __shared__ unsigned s_u[40];
  __shared__ T s_t[NF];

  WsHdr *ws = reinterpret_cast<WsHdr *>(a.ws);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  double mn, mx, range;
  T t;
  if constexpr (NF == 1) {
    threshold_of<T>(a.eps, a.eps_mode, a.cnorm, a.range, ws, mn, mx, range, t);
  } else if (tid < a.nf) {
    T tf;
    threshold_keys<T>(maps.g[tid].eps, maps.g[tid].eps_mode, a.cnorm, maps.g[tid].range_in, a.keys + 2 * tid, mn,
                      mx, range, tf);
    s_t[tid] = tf;
  }
  __syncthreads();
  const BView<T> v{reinterpret_cast<T *>(a.scratch + (size_t)blockIdx.x * S::SCR), B, (long long)B * B};
  unsigned char *arena = a.staging + (size_t)blockIdx.x * a.arena_bytes;
  unsigned long long aoff = 0;  // bytes used in this CTA's staging arena (the same in every thread)

  for (int bid = blockIdx.x; bid < a.nblocks; bid += gridDim.x) {
    // the block in its field
    const T *field = reinterpret_cast<const T *>(a.field);
    int lb = bid, nbx = a.nbx, nby = a.nby;
    if constexpr (NF > 1) {
      const int f = field_of<NF>(maps, a.nf, bid);
      field = reinterpret_cast<const T *>(maps.g[f].field);
      lb = bid - maps.g[f].first;
      nbx = maps.g[f].nbx;
      nby = maps.g[f].nby;
      t = s_t[f];
    }
    const long long nx = (long long)nbx * B, ny = (long long)nby * B;
    const int bx = lb % nbx, by = (lb / nbx) % nby, bz = lb / (nbx * nby);
    const T *src = field + ((long long)bz * B * ny + (long long)by * B) * nx + (long long)bx * B;

    slab_fwd<T, B, KIND, NT>(src, nx, nx * ny, v, C);

    // ---- mask rows (coarse positions carry no bit; word h of a row holds
    // x = 32 h + lane), row offsets; a warp takes RB consecutive rows a round
    for (int r0 = wid * RB; r0 < ROWS; r0 += NW * RB) {
      T d[RB][MWPR];
#pragma unroll
      for (int j = 0; j < RB; ++j)
#pragma unroll
        for (int h = 0; h < MWPR; ++h) d[j][h] = v.at(32 * h + lane, (r0 + j) % B, (r0 + j) / B);
#pragma unroll
      for (int j = 0; j < RB; ++j) {
        const int r = r0 + j, z = r / B, y = r % B;
#pragma unroll
        for (int h = 0; h < MWPR; ++h) {
          const int x = 32 * h + lane;
          const bool coarse = (x % Q == 0) && (y % Q == 0) && (z % Q == 0);
          const unsigned w = __ballot_sync(FULL, !coarse && keep(d[j][h], t));
          if (lane == 0) MW[r * MWPR + h] = w;
        }
      }
    }
    __syncthreads();
    unsigned nnz;
    {
      unsigned loc[RPT], sum = 0;
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        loc[q] = 0;
#pragma unroll
        for (int h = 0; h < MWPR; ++h) loc[q] += __popc(MW[(tid * RPT + q) * MWPR + h]);
        sum += loc[q];
      }
      unsigned ex = block_exsum<NT>(sum, s_u, nnz);
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        RO[tid * RPT + q] = ex;
        ex += loc[q];
      }
    }
    __syncthreads();

    // ---- slot [nnz | 0 | raw payload] -> this CTA's staging arena
    // (room for the finished stage-2 chunk: payload + 12 bytes + one split
    // token per 65535 words)
    const int pbytes = S::HEAD + (int)nnz * ES;
    const unsigned long long so = aoff;
    const unsigned long long slot = (unsigned long long)((pbytes + 12 + 4 * ((pbytes / 4) / 65535) + 15) & ~15);
    const bool ok = so + slot <= a.arena_bytes;
    if (ok) {
      unsigned char *P = arena + so + 8;
      unsigned *MASK = reinterpret_cast<unsigned *>(P + 64 * ES);
      for (int i = tid; i < ROWS * MWPR; i += NT) MASK[i] = MW[i];
      T *COARSE = reinterpret_cast<T *>(P);
      T *VALS = reinterpret_cast<T *>(P + S::HEAD);
      for (int r0 = wid * RB; r0 < ROWS; r0 += NW * RB) {
        // (rows without kept values or coarse values are not read:
        // warp-uniform)
        T d[RB][MWPR];
#pragma unroll
        for (int j = 0; j < RB; ++j) {
          const int r = r0 + j, z = r / B, y = r % B;
          const bool crow = (y % Q == 0) && (z % Q == 0);
#pragma unroll
          for (int h = 0; h < MWPR; ++h)
            d[j][h] = (MW[r * MWPR + h] != 0 || crow) ? v.at(32 * h + lane, y, z) : T(0);
        }
#pragma unroll
        for (int j = 0; j < RB; ++j) {
          const int r = r0 + j, z = r / B, y = r % B;
          const bool crow = (y % Q == 0) && (z % Q == 0);
          unsigned base = RO[r];
#pragma unroll
          for (int h = 0; h < MWPR; ++h) {
            const unsigned w = MW[r * MWPR + h];
            const int x = 32 * h + lane;
            if ((w >> lane) & 1u) VALS[base + __popc(w & ((1u << lane) - 1u))] = zero_low(d[j][h], a.zbits);
            if (crow && x % Q == 0) COARSE[((z / Q) * 4 + y / Q) * 4 + x / Q] = d[j][h];
            base += __popc(w);
          }
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
    __syncthreads();  // the scratch block, the mask words and the row offsets are free again
  }
}

// ---- decompression, in place in the output block (the field, or a tile of
// the random-access output)
template <typename T, int B, int KIND>
__global__ void __launch_bounds__(SG<T, B>::NT, SG<T, B>::MINB) k_decompress_slab(const InvArgs a)
{
  static_assert(SG<T, B>::OK, "slab geometry: B = 32 or 64");
  using S = SG<T, B>;
  using G = G2<T, B>;
  constexpr int NT = S::NT, NW = S::NW, Q = S::Q, ES = S::ES, ROWS = S::ROWS, RPT = S::RPT, MWPR = S::MWPR,
                RB = S::RB;
  static_assert(ROWS % (NW * RB) == 0, "whole rounds of RB rows per warp");
  extern __shared__ __align__(128) unsigned char smem[];
  T *C = reinterpret_cast<T *>(smem);
  unsigned *RO = reinterpret_cast<unsigned *>(smem + S::CUBE_AL);  // row offsets
  __shared__ unsigned s_u[40];
  __shared__ unsigned s_bad, s_nnz, s_badx;
  __shared__ const unsigned char *s_pay;

  WsHdr *ws = reinterpret_cast<WsHdr *>(a.ws);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const bool pre = a.stage2 != 0;  // decoded (and checked) payloads in staging slots
  T *out = reinterpret_cast<T *>(a.field);
  const long long nx = a.nx, ny = a.ny;

  for (int bid = blockIdx.x; bid < a.nblocks; bid += gridDim.x) {
    if (tid == 0) {
      unsigned bad = 0, nnz = 0;
      const unsigned char *pay = nullptr;
      if (pre) {
        bad = a.table[2 * bid + 1] != 0;
        nnz = bad ? 0u : (unsigned)a.table[2 * bid];
        pay = a.staging + (size_t)bid * a.slot;
      } else {
        const unsigned long long *tab = reinterpret_cast<const unsigned long long *>(a.in + HEADER_BYTES);
        int c = a.ids ? a.ids[bid] : bid;  // the block's chunk in the stream
        if (c < 0 || c >= a.nchunks) {
          atomicCAS(&ws->status, 0u, ST_ARG);
          c = 0;
          bad = 1;
        }
        const unsigned long long o0 = tab[c], o1 = tab[c + 1];
        const unsigned long long avail = a.in_bytes - a.data0;
        // chunks are whole numbers of elements (8-byte words for FP64)
        if (bad || o0 > o1 || o1 > avail || o1 - o0 < 8 || (o0 & (ES - 1)) || ((o1 - o0) & 3)) {
          bad = 1;
        } else {
          const unsigned *c32 = reinterpret_cast<const unsigned *>(a.in + a.data0 + o0);
          nnz = c32[0];
          if (nnz > (unsigned)(G::NVOX - 64)) bad = 1;
          const unsigned long long pb = (unsigned long long)S::HEAD + (unsigned long long)nnz * ES;
          if (!bad && (c32[1] != 0 || 8 + pb > o1 - o0)) bad = 1;
          pay = a.in + a.data0 + o0 + 8;
        }
      }
      s_bad = bad;
      s_nnz = bad ? 0u : nnz;
      s_pay = pay;
      s_badx = 0;
    }
    __syncthreads();
    const bool bad0 = s_bad != 0;
    const unsigned nnz = s_nnz;
    const unsigned char *P = s_pay;
    const unsigned *MASK = reinterpret_cast<const unsigned *>(P + 64 * ES);
    if (!bad0) {
      // row populations -> row offsets; coarse positions carry no mask bit
      // (cm: their bits within each of a row's words)
      unsigned loc[RPT], sum = 0;
      unsigned cm = 0;
#pragma unroll
      for (int x = 0; x < 32; x += Q) cm |= 1u << x;
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        const int r = tid * RPT + q, z = r / B, y = r % B;
        loc[q] = 0;
#pragma unroll
        for (int h = 0; h < MWPR; ++h) {
          const unsigned w = MASK[r * MWPR + h];
          if ((z % Q) == 0 && (y % Q) == 0 && (w & cm)) atomicOr(&s_badx, 1u);
          loc[q] += __popc(w);
        }
        sum += loc[q];
      }
      unsigned tot;
      unsigned ex = block_exsum<NT>(sum, s_u, tot);
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        RO[tid * RPT + q] = ex;
        ex += loc[q];
      }
      if (tid == 0 && tot != nnz) atomicOr(&s_badx, 1u);
    }
    __syncthreads();
    const bool bad = bad0 || s_badx != 0;
    if (bad && tid == 0) atomicCAS(&ws->status, 0u, ST_CORRUPT);

    const int bx = bid % a.nbx, by = (bid / a.nbx) % a.nby, bz = bid / (a.nbx * a.nby);
    const BView<T> v{out + ((long long)bz * B * ny + (long long)by * B) * nx + (long long)bx * B, nx, nx * ny};
    // coefficients (zeros where no bit) -> the output block; a bad block
    // decodes to zeros
    const T *COARSE = reinterpret_cast<const T *>(P);
    const T *VALS = reinterpret_cast<const T *>(P + S::HEAD);
    // a warp takes RB consecutive rows a round: their mask words, then all
    // their values, are loaded before any is used
    for (int r0 = wid * RB; r0 < ROWS; r0 += NW * RB) {
      unsigned w[RB][MWPR];
      T d[RB][MWPR];
#pragma unroll
      for (int j = 0; j < RB; ++j)
#pragma unroll
        for (int h = 0; h < MWPR; ++h) w[j][h] = bad ? 0u : MASK[(r0 + j) * MWPR + h];
#pragma unroll
      for (int j = 0; j < RB; ++j) {
        const int r = r0 + j, z = r / B, y = r % B;
        unsigned base = bad ? 0u : RO[r];
#pragma unroll
        for (int h = 0; h < MWPR; ++h) {
          const int x = 32 * h + lane;
          d[j][h] = T(0);
          if (!bad) {
            if ((w[j][h] >> lane) & 1u) d[j][h] = VALS[base + __popc(w[j][h] & ((1u << lane) - 1u))];
            if ((y % Q) == 0 && (z % Q) == 0 && (x % Q) == 0) d[j][h] = COARSE[((z / Q) * 4 + y / Q) * 4 + x / Q];
            base += __popc(w[j][h]);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < RB; ++j)
#pragma unroll
        for (int h = 0; h < MWPR; ++h) v.at(32 * h + lane, (r0 + j) % B, (r0 + j) / B) = d[j][h];
    }
    __syncthreads();
    if (!bad) slab_inv<T, B, KIND, NT>(v, C);
  }
}

// ---- dense transforms (test entry points): one CTA per block, in place in
// the destination block
template <typename T, int B, int KIND, bool FWD>
__global__ void __launch_bounds__(SG<T, B>::NT) k_dense_slab(const DenseArgs a)
{
  static_assert(SG<T, B>::OK, "slab geometry: B = 32 or 64");
  using S = SG<T, B>;
  constexpr int NT = S::NT, NW = S::NW, ROWS = S::ROWS;
  extern __shared__ __align__(128) unsigned char smem[];
  T *C = reinterpret_cast<T *>(smem);
  const int bid = blockIdx.x, lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int bx = bid % a.nbx, by = (bid / a.nbx) % a.nby, bz = bid / (a.nbx * a.nby);
  const long long nx = a.nx, ny = a.ny;
  const long long off = ((long long)bz * B * ny + (long long)by * B) * nx + (long long)bx * B;
  const T *src = reinterpret_cast<const T *>(a.src) + off;
  const BView<T> v{reinterpret_cast<T *>(a.dst) + off, nx, nx * ny};
  if constexpr (FWD) {
    slab_fwd<T, B, KIND, NT>(src, nx, nx * ny, v, C);
  } else {
    for (int r = wid; r < ROWS; r += NW)
      for (int x = lane; x < B; x += 32) v.at(x, r % B, r / B) = src[(r / B) * nx * ny + (r % B) * nx + x];
    __syncthreads();
    slab_inv<T, B, KIND, NT>(v, C);
  }
}

// ---- stage 2 of payloads too large for shared memory: the k_stage2 coder
// (byte shuffle, zero-word runs from a ballot bitmap, tokens and literal
// words in place of the slot) with the shuffled payload in a global scratch
// block per CTA.  Payloads here may exceed 65535 words, so a pair (literal
// words, zero run) longer than a token field splits as the stream format
// says: (65535, 0) tokens while more than 65535 literals remain, then
// (literals, 65535) and (0, 65535) tokens while more than 65535 zero words
// remain, then the rest.
__device__ __forceinline__ unsigned pair_tokens(unsigned lit, unsigned zr)
{
  return (lit > 65535u ? (lit - 1u) / 65535u : 0u) + (zr > 65535u ? (zr - 1u) / 65535u : 0u) + 1u;
}

__device__ __forceinline__ void put_pair(unsigned *tok, unsigned k, unsigned lit, unsigned zr)
{
  while (lit > 65535u) {
    tok[k++] = 65535u;
    lit -= 65535u;
  }
  while (zr > 65535u) {
    tok[k++] = lit | (65535u << 16);
    lit = 0u;
    zr -= 65535u;
  }
  tok[k] = lit | (zr << 16);
}

// ---- zero-run code of a shuffled payload of pbytes (any size) in global
// memory SH, by all NT = 512 threads of the CTA: [ntok | tokens | literal
// words] are written from ch + 1 on (ch[0] is left alone).  The four bitmap
// arrays of `cap` words (ZBM, CM, EB, PRC) live in shared memory at BM;
// s_u / s_i (>= 40 words) are scan scratch and *s_lastend an int that is 0
// on entry (and again on return).  Returns 8 + the bytes of tokens and
// literals (the same in every thread).
template <int NT>
__device__ __forceinline__ unsigned long long huge_code(unsigned *ch, int pbytes, const unsigned char *SH,
                                                        unsigned *BM, int cap, unsigned *s_u, int *s_i,
                                                        int *s_lastend)
{
  constexpr int NWP = NT / 32;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const unsigned *SH32 = reinterpret_cast<const unsigned *>(SH);
  unsigned *ZBM = BM, *CM = ZBM + cap, *EB = ZBM + 2 * cap, *PRC = ZBM + 3 * cap;  // PRC: coded words before
  const int W = pbytes >> 2, NB = (W + 31) >> 5;
  for (int g = wid; g < NB; g += NWP) {
    const int w = g * 32 + lane;
    const unsigned bal = __ballot_sync(FULL, w < W && SH32[w] == 0u);
    if (lane == 0) ZBM[g] = bal;
  }
  __syncthreads();
  // coded words C: zero words with a zero neighbour; a run starts at an S
  // bit and ends before an Eb bit (or at W)
  const int KB = (NB + NT - 1) / NT;  // bitmap words per thread (contiguous)
  unsigned mine_s = 0, mine_c = 0;
  for (int q = 0; q < KB; ++q) {
    const int g = tid * KB + q;
    if (g < NB) {
      const unsigned Z = ZBM[g];
      const unsigned Zp = g > 0 ? ZBM[g - 1] : 0u, Zn = g + 1 < NB ? ZBM[g + 1] : 0u;
      const unsigned valid = (g == NB - 1 && (W & 31)) ? ((1u << (W & 31)) - 1u) : FULL;
      const unsigned Cw = Z & ((Z << 1) | (Zp >> 31) | (Z >> 1) | ((Zn & 1u) << 31)) & valid;
      const unsigned cin = g > 0 ? ((Zp >> 31) & (((Zp >> 30) & 1u) | (Z & 1u))) : 0u;
      CM[g] = Cw;
      EB[g] = ~Cw & ((Cw << 1) | cin) & valid;
      mine_s += (unsigned)__popc(Cw & ~((Cw << 1) | cin));
      mine_c += (unsigned)__popc(Cw);
    }
  }
  unsigned ns_tot, nc_tot;
  block_exsum<NT>(mine_s, s_u, ns_tot);
  unsigned crun = block_exsum<NT>(mine_c, s_u, nc_tot);
  for (int q = 0; q < KB; ++q) {
    const int g = tid * KB + q;
    if (g < NB) {
      PRC[g] = crun;
      crun += (unsigned)__popc(CM[g]);
    }
  }
  // run ends around this thread's words: the last one before them (0 if
  // none) and the first one after them (W if none)
  int my_last = 0, my_first = W;
  for (int q = 0; q < KB; ++q) {
    const int g = tid * KB + q;
    if (g < NB && EB[g]) {
      my_last = max(my_last, g * 32 + 31 - (int)__clz(EB[g]));
      my_first = min(my_first, g * 32 + __ffs(EB[g]) - 1);
    }
  }
  const int pe0 = block_exmax<NT>(my_last, 0, s_i);
  const int ne_after = block_rexmin<NT>(my_first, W, s_i);
  const int l = W - 1;
  const bool lastc =
      (((ZBM[l >> 5] >> (l & 31)) & 1u) && l > 0 && ((ZBM[(l - 1) >> 5] >> ((l - 1) & 31)) & 1u));
  // visit this thread's runs in order: f(start, previous run's end, end)
  auto runs = [&](auto &&f) {
    int pe_words = pe0;
    for (int q = 0; q < KB; ++q) {
      const int g = tid * KB + q;
      if (g >= NB) break;
      const unsigned Cw = CM[g], Eb = EB[g];
      const unsigned cin = g > 0 ? (CM[g - 1] >> 31) : 0u;
      unsigned Sb = Cw & ~((Cw << 1) | cin);
      while (Sb) {
        const int b = __ffs(Sb) - 1;
        Sb &= Sb - 1u;
        const int p = g * 32 + b;
        const unsigned below = Eb & ((1u << b) - 1u), above = Eb & ~((2u << b) - 1u);
        const int pe = below ? g * 32 + 31 - (int)__clz(below) : pe_words;
        int ne = ne_after;
        if (above) {
          ne = g * 32 + __ffs(above) - 1;
        } else {
          for (int h = q + 1; h < KB && tid * KB + h < NB; ++h)
            if (EB[tid * KB + h]) {
              ne = (tid * KB + h) * 32 + __ffs(EB[tid * KB + h]) - 1;
              break;
            }
        }
        f(p, pe, ne);
      }
      if (Eb) pe_words = g * 32 + 31 - (int)__clz(Eb);
    }
  };
  unsigned mine_t = 0;
  runs([&](int p, int pe, int ne) { mine_t += pair_tokens((unsigned)(p - pe), (unsigned)(ne - p)); });
  unsigned run_tok;
  unsigned k = block_exsum<NT>(mine_t, s_u, run_tok);
  // the last run end in the payload (0 if none): the trailing pair holds
  // the literals after it, unless the payload ends in a run
  if (my_last > 0) atomicMax(s_lastend, my_last);
  __syncthreads();
  const unsigned tail = (unsigned)(W - *s_lastend);
  const unsigned ntok = run_tok + (lastc ? 0u : pair_tokens(tail, 0u));
  const unsigned nlit = (unsigned)W - nc_tot;
  unsigned *tok = ch + 2;
  unsigned *lit = tok + ntok;
  runs([&](int p, int pe, int ne) {
    put_pair(tok, k, (unsigned)(p - pe), (unsigned)(ne - p));
    k += pair_tokens((unsigned)(p - pe), (unsigned)(ne - p));
  });
  if (tid == 0) {
    if (!lastc) put_pair(tok, run_tok, tail, 0u);
    ch[1] = ntok;
  }
  for (int w = tid; w < W; w += NT) {
    const int g = w >> 5, b = w & 31;
    const unsigned Cw = CM[g];
    if (!((Cw >> b) & 1u)) lit[(unsigned)w - (PRC[g] + __popc(Cw & ((1u << b) - 1u)))] = SH32[w];
  }
  __syncthreads();  // the scratch block and the bitmaps are free again
  if (tid == 0) *s_lastend = 0;
  return 8ull + 4ull * ntok + 4ull * nlit;
}

template <typename T, int B>
__global__ void __launch_bounds__(512) k_stage2_huge(const S2Args a)
{
  using G = G2<T, B>;
  constexpr int NT = 512, LGES = G::LGES, cap = G::NBWMAX;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ unsigned s_u[40];
  __shared__ int s_i[40];
  __shared__ int s_lastend;
  const int tid = threadIdx.x;
  if (tid == 0) s_lastend = 0;  // ordered before its first use by the loop's barriers
  unsigned char *SH = a.scratch + (size_t)blockIdx.x * G::SCRATCH;

  const int count = (int)reinterpret_cast<const WsHdr *>(a.ws)->nbig;
  for (int it = blockIdx.x; it < count; it += gridDim.x) {
    const int bid = a.biglist[it];
    const unsigned long long so = a.table[2 * bid], cb = a.table[2 * bid + 1];
    if (cb == TB_LOST || (cb & TB_FIN)) continue;
    const int pbytes = (int)cb - 8;
    if (pbytes <= G::SHCAP) continue;  // the small launch's payload
    unsigned *ch = reinterpret_cast<unsigned *>(a.staging + so);
    // shuffle: payload word k holds bytes 0..3 of element 4k / ES at byte
    // offset 4k % ES
    const int W = pbytes >> 2;
    const unsigned *raw = ch + 2;
    for (int k = tid; k < W; k += NT) {
      const unsigned wv = raw[k];
      const int e = (4 * k) >> LGES, b0 = (4 * k) & (G::ES - 1);
#pragma unroll
      for (int q = 0; q < 4; ++q) SH[(b0 + q) * (pbytes >> LGES) + e] = (unsigned char)(wv >> (8 * q));
    }
    __syncthreads();  // the slot's payload is no longer needed
    const unsigned long long cbytes =
        huge_code<NT>(ch, pbytes, SH, reinterpret_cast<unsigned *>(smem), cap, s_u, s_i, &s_lastend);
    if (tid == 0) a.table[2 * bid + 1] = TB_FIN | cbytes;
  }
}

}  // namespace czp
