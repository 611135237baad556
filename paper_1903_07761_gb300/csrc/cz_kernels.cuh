// cz_kernels.cuh -- kernels of the GB300 wavelet codec.
//
// k_compress  : one CTA per cubic block: load the block (thread (x,y) keeps
//               its z-column in registers), L levels of the forward 3D
//               transform, threshold against t, one __ballot_sync per warp
//               and plane gives a mask word, a block scan of the word
//               populations places every kept detail, optional stage 2
//               (byte shuffle + zero-word run-length coding) in shared
//               memory, decoupled look-back for the chunk offset, write.
// k_decompress: one CTA per chunk: stage-2 decode into shared memory,
//               scatter coarse values and kept details into the register
//               columns, inverse levels, store.
// k_minmax    : range of the field for a relative threshold.
// k_fwd_dense / k_inv_dense: the transform alone (test access).
#pragma once

#include "cz_device.cuh"

namespace czk {
using namespace czd;

// numeric values of the public status codes
constexpr unsigned ST_CAPACITY = (unsigned)-2;
constexpr unsigned ST_CORRUPT = (unsigned)-3;
constexpr unsigned ST_TIMEOUT = (unsigned)-4;

constexpr int HEADER_BYTES = 128;
constexpr unsigned MAGIC = 0x315A4343u;

// workspace: this header, then one u64 look-back word per block
struct WsHdr {
  unsigned status;
  unsigned ticket;
  unsigned pad0, pad1;
  unsigned long long minkey, maxkey;
  unsigned long long out_bytes;
};
constexpr int WS_HDR = 256;

template <typename T, int B>
struct Geo {
  static constexpr int NT = B * B;         // threads per CTA
  static constexpr int NW = NT / 32;       // warps = mask words per z-plane
  static constexpr int L = (B == 8) ? 1 : (B == 16) ? 2 : 3;  // levels to 4^3
  static constexpr int Q = B / 4;          // coarse spacing
  static constexpr int S = (int)sizeof(T); // element bytes
  static constexpr int NMW = B * B * B / 32;  // mask words
  static constexpr int PMAX = 64 * S + NMW * 4 + (B * B * B - 64) * S;
  static constexpr int P_AL = (PMAX + 15) / 16 * 16;
  static constexpr int WMAX = PMAX / 4;    // shuffled words
  static constexpr int NBW = (WMAX + 31) / 32;  // zero-bitmap words
  static constexpr int ZB0 = 32768 / (B * B * S);
  static constexpr int ZB = ZB0 < B ? ZB0 : B;  // y-exchange planes per batch
  static constexpr int XBYTES = ZB * B * B * S;
  static constexpr int ENC_AUX = (NMW + 4 * NBW) * 4;
  static constexpr int DEC_AUX = (NMW + 3 * NT) * 4;
  static constexpr int R2 = XBYTES > ENC_AUX ? (XBYTES > DEC_AUX ? XBYTES : DEC_AUX)
                                             : (ENC_AUX > DEC_AUX ? ENC_AUX : DEC_AUX);
  static constexpr int SMEM = P_AL + (R2 + 15) / 16 * 16;
};

struct FwdArgs {
  const void *field;
  unsigned char *out;
  unsigned long long *out_bytes;  // may be null
  void *ws;
  unsigned long long out_cap, data0;
  double eps, range;
  int nx, ny, nz, nbx, nby, nbz, nblocks;
  int eps_mode, stage2, kind, dtype;
};

struct InvArgs {
  const unsigned char *in;
  void *field;
  void *ws;
  unsigned long long in_bytes, data0;
  int nx, ny, nz, nbx, nby, nbz, nblocks;
  int stage2;
};

struct DenseArgs {
  const void *src;
  void *dst;
  int nx, ny, nz, nbx, nby, nbz;
};

// ============================================================ levels
template <typename T, int B, int KIND, int LEV>
__device__ __forceinline__ void fwd_level(T (&v)[B], T *X, int x, int y)
{
  using G = Geo<T, B>;
  constexpr int S = 1 << LEV, n = B >> LEV, m = n / 2, NZ = B / S, ZB = G::ZB;
  const int lane = threadIdx.x & 31;
  const bool xact = (x & (S - 1)) == 0, yact = (y & (S - 1)) == 0;
  // ---- x: warp shuffles (a row is B consecutive lanes)
  {
    const Stencil<T> st = make_stencil<T, KIND>(x / S, m);
    const int seg = lane - x;
    if (B < 32 || yact) {
#pragma unroll
      for (int z = 0; z < B; z += S) {
        const T f = v[z];
        auto g = [&](int idx) { return shfl(f, seg + idx * S); };
        T r;
        if constexpr (KIND == W4) {
          r = fwd_predict(st, f, g);
        } else if constexpr (KIND == W4LI) {
          const T f1 = fwd_predict(st, f, g);
          r = fwd_update(st, f1, [&](int idx) { return shfl(f1, seg + idx * S); });
        } else {
          r = fwd_ai(st, f, g, [&](int idx, T a) { return shfl(a, seg + idx * S); });
        }
        if (xact && yact) v[z] = r;
      }
    }
  }
  // ---- y: shared-memory planes, ZB planes per batch
  {
    const Stencil<T> st = make_stencil<T, KIND>(y / S, m);
    const bool act = xact && yact;
#pragma unroll
    for (int zb = 0; zb < NZ; zb += ZB) {
#pragma unroll
      for (int q = 0; q < ZB; ++q)
        if (zb + q < NZ && act) X[(q * B + y) * B + x] = v[(zb + q) * S];
      __syncthreads();
#pragma unroll
      for (int q = 0; q < ZB; ++q) {
        if (zb + q < NZ && act) {
          T *Xq = X + q * B * B + x;
          auto g = [&](int idx) { return Xq[idx * S * B]; };
          const T f = v[(zb + q) * S];
          T r;
          if constexpr (KIND == W4) {
            r = fwd_predict(st, f, g);
          } else if constexpr (KIND == W4LI) {
            r = fwd_predict(st, f, g);
            if (st.i & 1) Xq[y * B] = r;  // odd rows now hold details
          } else {
            r = fwd_ai(st, f, g, [&](int idx, T) { return mulx(addx(g(idx), g(idx + 1)), (T)0.5); });
          }
          v[(zb + q) * S] = r;
        }
      }
      if constexpr (KIND == W4LI) {
        __syncthreads();
#pragma unroll
        for (int q = 0; q < ZB; ++q) {
          if (zb + q < NZ && act) {
            T *Xq = X + q * B * B + x;
            v[(zb + q) * S] = fwd_update(st, v[(zb + q) * S], [&](int idx) { return Xq[idx * S * B]; });
          }
        }
      }
      __syncthreads();
    }
  }
  // ---- z: registers
  if (xact && yact) fwd_reg<T, KIND, B, S>(v);
}

template <typename T, int B, int KIND, int LEV>
__device__ __forceinline__ void inv_level(T (&v)[B], T *X, int x, int y)
{
  using G = Geo<T, B>;
  constexpr int S = 1 << LEV, n = B >> LEV, m = n / 2, NZ = B / S, ZB = G::ZB;
  const int lane = threadIdx.x & 31;
  const bool xact = (x & (S - 1)) == 0, yact = (y & (S - 1)) == 0;
  // ---- z
  if (xact && yact) inv_reg<T, KIND, B, S>(v);
  // ---- y
  {
    const Stencil<T> st = make_stencil<T, KIND>(y / S, m);
    const bool act = xact && yact;
#pragma unroll
    for (int zb = 0; zb < NZ; zb += ZB) {
#pragma unroll
      for (int q = 0; q < ZB; ++q)
        if (zb + q < NZ && act) X[(q * B + y) * B + x] = v[(zb + q) * S];
      __syncthreads();
      if constexpr (KIND == W4LI) {
#pragma unroll
        for (int q = 0; q < ZB; ++q) {
          if (zb + q < NZ && act) {
            T *Xq = X + q * B * B + x;
            const T c = inv_update(st, v[(zb + q) * S], [&](int idx) { return Xq[idx * S * B]; });
            if (!(st.i & 1)) Xq[y * B] = c;  // even rows now hold coarse values
            v[(zb + q) * S] = c;
          }
        }
        __syncthreads();
      }
#pragma unroll
      for (int q = 0; q < ZB; ++q) {
        if (zb + q < NZ && act) {
          T *Xq = X + q * B * B + x;
          auto g = [&](int idx) { return Xq[idx * S * B]; };
          const T f = v[(zb + q) * S];
          if constexpr (KIND == W3AI)
            v[(zb + q) * S] = inv_ai(st, f, g);
          else
            v[(zb + q) * S] = inv_predict(st, f, g);
        }
      }
      __syncthreads();
    }
  }
  // ---- x
  {
    const Stencil<T> st = make_stencil<T, KIND>(x / S, m);
    const int seg = lane - x;
    if (B < 32 || yact) {
#pragma unroll
      for (int z = 0; z < B; z += S) {
        const T f = v[z];
        auto g = [&](int idx) { return shfl(f, seg + idx * S); };
        T r;
        if constexpr (KIND == W4) {
          r = inv_predict(st, f, g);
        } else if constexpr (KIND == W4LI) {
          const T f1 = inv_update(st, f, g);
          r = inv_predict(st, f1, [&](int idx) { return shfl(f1, seg + idx * S); });
        } else {
          r = inv_ai(st, f, g);
        }
        if (xact && yact) v[z] = r;
      }
    }
  }
}

template <typename T, int B, int KIND>
__device__ __forceinline__ void fwd_transform(T (&v)[B], T *X, int x, int y)
{
  fwd_level<T, B, KIND, 0>(v, X, x, y);
  if constexpr (Geo<T, B>::L > 1) fwd_level<T, B, KIND, 1>(v, X, x, y);
  if constexpr (Geo<T, B>::L > 2) fwd_level<T, B, KIND, 2>(v, X, x, y);
}

template <typename T, int B, int KIND>
__device__ __forceinline__ void inv_transform(T (&v)[B], T *X, int x, int y)
{
  if constexpr (Geo<T, B>::L > 2) inv_level<T, B, KIND, 2>(v, X, x, y);
  if constexpr (Geo<T, B>::L > 1) inv_level<T, B, KIND, 1>(v, X, x, y);
  inv_level<T, B, KIND, 0>(v, X, x, y);
}

// ============================================================ helpers
// word w of the byte-shuffled payload: shuffled byte j is byte (j / E) of
// element (j % E), E = payload bytes / element size
__device__ __forceinline__ unsigned shuffled_word(const unsigned char *P, int w, int E, int es)
{
  const int j = 4 * w;
  int b = j / E;
  int e = j - b * E;
  unsigned r = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (e == E) {
      e = 0;
      ++b;
    }
    r |= (unsigned)P[e * es + b] << (8 * q);
    ++e;
  }
  return r;
}

__device__ __forceinline__ void unshuffle_word(unsigned char *P, int w, unsigned val, int E, int es)
{
  const int j = 4 * w;
  int b = j / E;
  int e = j - b * E;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (e == E) {
      e = 0;
      ++b;
    }
    P[e * es + b] = (unsigned char)(val >> (8 * q));
    ++e;
  }
}

__device__ __forceinline__ unsigned tokcount(unsigned lit, unsigned zr)
{
  return 1u + (lit > 65535u ? (lit - 1u) / 65535u : 0u) + (zr > 65535u ? (zr - 1u) / 65535u : 0u);
}

__device__ __forceinline__ unsigned emit_tokens(unsigned *tok, unsigned idx, unsigned lit, unsigned zr)
{
  while (lit > 65535u) {
    tok[idx++] = 65535u;
    lit -= 65535u;
  }
  while (zr > 65535u) {
    tok[idx++] = lit | (65535u << 16);
    lit = 0;
    zr -= 65535u;
  }
  tok[idx++] = lit | (zr << 16);
  return idx;
}

template <typename U>
__device__ __forceinline__ void st_le(unsigned char *p, U v)
{
#pragma unroll
  for (int q = 0; q < (int)sizeof(U); ++q) p[q] = (unsigned char)((unsigned long long)v >> (8 * q));
}
__device__ __forceinline__ void st_le_f64(unsigned char *p, double v)
{
  st_le<unsigned long long>(p, (unsigned long long)__double_as_longlong(v));
}

// range and threshold exactly as the stream header records them
template <typename T>
__device__ __forceinline__ void threshold_of(const FwdArgs &a, const WsHdr *ws, double &mn, double &mx,
                                             double &range, T &t)
{
  if (a.range >= 0) {
    range = a.range;
    mn = mx = __longlong_as_double(0x7FF8000000000000LL);
  } else {
    const unsigned long long kmin = *(volatile const unsigned long long *)&ws->minkey;
    const unsigned long long kmax = *(volatile const unsigned long long *)&ws->maxkey;
    mn = key_value(kmin, T(0));
    mx = key_value(kmax, T(0));
    mn = (double)(T)((T)mn + (T)0);  // -0 reported as +0
    mx = (double)(T)((T)mx + (T)0);
    range = (mn <= mx) ? mx - mn : 0.0;
  }
  const double td = a.eps_mode == 1 ? a.eps : a.eps * range;
  t = (T)td;
}

// ============================================================ compress
template <typename T, int B, int KIND>
__global__ void __launch_bounds__(B * B) k_compress(const FwdArgs a)
{
  using G = Geo<T, B>;
  constexpr int NT = G::NT, NW = G::NW, Q = G::Q, ES = G::S, NMW = G::NMW;
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char *P = smem;
  T *X = reinterpret_cast<T *>(smem + G::P_AL);
  unsigned *WC = reinterpret_cast<unsigned *>(smem + G::P_AL);
  unsigned *ZBM = WC + NMW;
  unsigned *CMk = ZBM + G::NBW;
  unsigned *BDM = CMk + G::NBW;
  unsigned *LP = BDM + G::NBW;
  __shared__ unsigned s_u[40];
  __shared__ int s_i[40];
  __shared__ int s_bid;
  __shared__ unsigned long long s_excl;

  WsHdr *ws = reinterpret_cast<WsHdr *>(a.ws);
  unsigned long long *lbst = reinterpret_cast<unsigned long long *>((char *)a.ws + WS_HDR);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int x = tid % B, y = tid / B;

  // block ids in ticket order: every block waited on is already resident
  if (tid == 0) s_bid = (int)atomicAdd(&ws->ticket, 1u);
  __syncthreads();
  const int bid = s_bid;
  const int bx = bid % a.nbx, by = (bid / a.nbx) % a.nby, bz = bid / (a.nbx * a.nby);

  double mn, mx, range;
  T t;
  threshold_of<T>(a, ws, mn, mx, range, t);

  // ---- a1: load
  T v[B];
  {
    const size_t zs = (size_t)a.ny * a.nx;
    const T *src = reinterpret_cast<const T *>(a.field) + (size_t)(bz * B) * zs +
                   (size_t)(by * B + y) * a.nx + (size_t)(bx * B + x);
#pragma unroll
    for (int z = 0; z < B; ++z) v[z] = __ldcs(src + z * zs);
  }
  // ---- a2: forward transform
  fwd_transform<T, B, KIND>(v, X, x, y);
  __syncthreads();

  // ---- a3/a4: coarse values, mask words, compaction
  const bool xyq = (x % Q == 0) && (y % Q == 0);
  if (xyq) {
#pragma unroll
    for (int z = 0; z < B; z += Q) reinterpret_cast<T *>(P)[((z / Q) * 4 + y / Q) * 4 + x / Q] = v[z];
  }
  unsigned *MASK = reinterpret_cast<unsigned *>(P + 64 * ES);
#pragma unroll
  for (int z = 0; z < B; ++z) {
    const bool sig = !(absx(v[z]) < t) && !(xyq && (z % Q == 0));
    const unsigned bal = __ballot_sync(FULL, sig);
    if (lane == 0) {
      MASK[z * NW + wid] = bal;
      WC[z * NW + wid] = __popc(bal);
    }
  }
  __syncthreads();
  unsigned nnz;
  {
    constexpr int IPT = (NMW + NT - 1) / NT;
    unsigned loc[IPT];
    unsigned sum = 0;
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
      const int k = tid * IPT + q;
      loc[q] = k < NMW ? WC[k] : 0u;
      sum += loc[q];
    }
    unsigned ex = block_exsum<NT>(sum, s_u, nnz);
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
      const int k = tid * IPT + q;
      if (k < NMW) WC[k] = ex;
      ex += loc[q];
    }
  }
  __syncthreads();
  {
    T *VALS = reinterpret_cast<T *>(P + 64 * ES + NMW * 4);
    const unsigned ltm = (1u << lane) - 1u;
#pragma unroll
    for (int z = 0; z < B; ++z) {
      const bool sig = !(absx(v[z]) < t) && !(xyq && (z % Q == 0));
      const unsigned bal = __ballot_sync(FULL, sig);
      if (sig) VALS[WC[z * NW + wid] + __popc(bal & ltm)] = v[z];
    }
  }
  __syncthreads();
  const int pbytes = 64 * ES + NMW * 4 + (int)nnz * ES;

  // ---- a6: stage 2 sizes (byte shuffle + zero-word RLE)
  const int W = pbytes / 4, E = pbytes / ES, NB = (W + 31) / 32;
  constexpr int KB = (G::NBW + NT - 1) / NT;
  unsigned ntok = 0, nlit = 0, tokbase = 0;
  int prev_before = -1, next_after = W;
  if (a.stage2) {
    for (int wb = wid; wb < NB; wb += NW) {
      const int w = wb * 32 + lane;
      const bool zr = (w < W) && (shuffled_word(P, w, E, ES) == 0u);
      const unsigned bal = __ballot_sync(FULL, zr);
      if (lane == 0) ZBM[wb] = bal;
    }
    __syncthreads();
    int first_bd = W, last_bd = -1;
    unsigned my_lit = 0;
#pragma unroll
    for (int q = 0; q < KB; ++q) {
      const int i = tid * KB + q;
      if (i < NB) {
        const unsigned Z = ZBM[i];
        const unsigned pw = i > 0 ? ZBM[i - 1] : 0u;
        const unsigned nw = (i + 1 < NB) ? ZBM[i + 1] : 0u;
        // coded zero word: zero with a zero neighbour (runs of >= 2 words)
        unsigned C = Z & ((Z << 1) | (pw >> 31) | (Z >> 1) | ((nw & 1u) << 31));
        const unsigned cp = i > 0 ? ((pw >> 31) & (((pw >> 30) & 1u) | (Z & 1u))) : 0u;
        unsigned Bd = C ^ ((C << 1) | cp);
        if (i == 0) Bd |= 1u;
        const unsigned valid = (i == NB - 1 && (W & 31)) ? ((1u << (W & 31)) - 1u) : FULL;
        C &= valid;
        Bd &= valid;
        CMk[i] = C;
        BDM[i] = Bd;
        my_lit += __popc(~C & valid);
        if (Bd) {
          if (first_bd == W) first_bd = i * 32 + __ffs(Bd) - 1;
          last_bd = i * 32 + 31 - __clz(Bd);
        }
      }
    }
    const unsigned litbase = block_exsum<NT>(my_lit, s_u, nlit);
    prev_before = block_exmax<NT>(last_bd, -1, s_i);
    next_after = block_rexmin<NT>(first_bd, W, s_i);
    {
      unsigned run = litbase;
#pragma unroll
      for (int q = 0; q < KB; ++q) {
        const int i = tid * KB + q;
        if (i < NB) {
          const unsigned valid = (i == NB - 1 && (W & 31)) ? ((1u << (W & 31)) - 1u) : FULL;
          LP[i] = run;
          run += __popc(~CMk[i] & valid);
        }
      }
    }
    // token count of the pairs whose boundary lies in this thread's words
    unsigned my_tok = 0;
    {
      int prev = prev_before, cur = -1;
      auto handle = [&](int p, int pv, int nb) {
        if ((CMk[p >> 5] >> (p & 31)) & 1u)
          my_tok += tokcount(p == 0 ? 0u : (unsigned)(p - pv), (unsigned)(nb - p));
        else if (nb == W)
          my_tok += tokcount((unsigned)(W - p), 0u);
      };
#pragma unroll
      for (int q = 0; q < KB; ++q) {
        const int i = tid * KB + q;
        if (i < NB) {
          unsigned bd = BDM[i];
          while (bd) {
            const int p = i * 32 + __ffs(bd) - 1;
            bd &= bd - 1u;
            if (cur >= 0) {
              handle(cur, prev, p);
              prev = cur;
            }
            cur = p;
          }
        }
      }
      if (cur >= 0) handle(cur, prev, next_after);
    }
    tokbase = block_exsum<NT>(my_tok, s_u, ntok);
  }
  const unsigned long long size =
      a.stage2 ? 8ull + 4ull * ntok + 4ull * nlit : 8ull + (unsigned long long)pbytes;

  // ---- a5: chunk offset by decoupled look-back
  if (wid == 0) {
    const unsigned long long ex = lookback(lbst, bid, size, &ws->status, (int)ST_TIMEOUT);
    if (lane == 0) s_excl = ex;
  }
  __syncthreads();
  const unsigned long long excl = s_excl;
  const bool fits = a.data0 + excl + size <= a.out_cap;
  if (tid == 0) {
    st_le<unsigned long long>(a.out + HEADER_BYTES + 8ull * bid, excl);
    if (!fits) atomicCAS(&ws->status, 0u, ST_CAPACITY);
    if (bid == a.nblocks - 1) {
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
      h[20] = (unsigned char)B;
      h[21] = (unsigned char)a.dtype;
      h[22] = (unsigned char)a.kind;
      h[23] = (unsigned char)a.stage2;
      h[24] = (unsigned char)a.eps_mode;
      h[25] = (unsigned char)G::L;
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
  if (!fits) return;

  // ---- write the chunk
  unsigned char *ch = a.out + a.data0 + excl;
  unsigned *ch32 = reinterpret_cast<unsigned *>(ch);
  if (tid == 0) {
    ch32[0] = nnz;
    ch32[1] = a.stage2 ? ntok : 0u;
  }
  if (a.stage2) {
    unsigned *tok = ch32 + 2;
    {
      unsigned idx = tokbase;
      int prev = prev_before, cur = -1;
      auto handle = [&](int p, int pv, int nb) {
        if ((CMk[p >> 5] >> (p & 31)) & 1u)
          idx = emit_tokens(tok, idx, p == 0 ? 0u : (unsigned)(p - pv), (unsigned)(nb - p));
        else if (nb == W)
          idx = emit_tokens(tok, idx, (unsigned)(W - p), 0u);
      };
#pragma unroll
      for (int q = 0; q < KB; ++q) {
        const int i = tid * KB + q;
        if (i < NB) {
          unsigned bd = BDM[i];
          while (bd) {
            const int p = i * 32 + __ffs(bd) - 1;
            bd &= bd - 1u;
            if (cur >= 0) {
              handle(cur, prev, p);
              prev = cur;
            }
            cur = p;
          }
        }
      }
      if (cur >= 0) handle(cur, prev, next_after);
    }
    unsigned *lit = tok + ntok;
    for (int w = tid; w < W; w += NT) {
      const unsigned C = CMk[w >> 5];
      const int b = w & 31;
      if (!((C >> b) & 1u)) lit[LP[w >> 5] + __popc(~C & ((1u << b) - 1u))] = shuffled_word(P, w, E, ES);
    }
  } else {
    const unsigned *P32 = reinterpret_cast<const unsigned *>(P);
    for (int w = tid; w < pbytes / 4; w += NT) ch32[2 + w] = P32[w];
  }
}

// ============================================================ decompress
template <typename T, int B, int KIND>
__global__ void __launch_bounds__(B * B) k_decompress(const InvArgs a)
{
  using G = Geo<T, B>;
  constexpr int NT = G::NT, NW = G::NW, Q = G::Q, ES = G::S, NMW = G::NMW;
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char *P = smem;
  T *X = reinterpret_cast<T *>(smem + G::P_AL);
  unsigned *WC = reinterpret_cast<unsigned *>(smem + G::P_AL);
  unsigned *TL = WC + NMW;
  unsigned *TO = TL + NT;
  __shared__ unsigned s_u[40];
  __shared__ unsigned s_nnz, s_ntok, s_bad;
  __shared__ unsigned long long s_off, s_len;

  WsHdr *ws = reinterpret_cast<WsHdr *>(a.ws);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int x = tid % B, y = tid / B;
  const int bid = blockIdx.x;
  const int bx = bid % a.nbx, by = (bid / a.nbx) % a.nby, bz = bid / (a.nbx * a.nby);

  if (tid == 0) {
    unsigned bad = 0;
    const unsigned long long *tab = reinterpret_cast<const unsigned long long *>(a.in + HEADER_BYTES);
    const unsigned long long o0 = tab[bid], o1 = tab[bid + 1];
    const unsigned long long avail = a.in_bytes - a.data0;
    unsigned nnz = 0, ntok = 0;
    if (o0 > o1 || o1 > avail || o1 - o0 < 8 || (o0 & 3)) {
      bad = 1;
    } else {
      const unsigned *c32 = reinterpret_cast<const unsigned *>(a.in + a.data0 + o0);
      nnz = c32[0];
      ntok = c32[1];
      const unsigned long long len = o1 - o0;
      if (nnz > (unsigned)(B * B * B - 64)) bad = 1;
      const unsigned long long pb = 64ull * ES + NMW * 4ull + (unsigned long long)nnz * ES;
      if (!bad && !a.stage2 && (ntok != 0 || 8 + pb > len)) bad = 1;
      if (!bad && a.stage2 && (unsigned long long)ntok > (len - 8) / 4) bad = 1;
    }
    s_bad = bad;
    s_nnz = nnz;
    s_ntok = ntok;
    s_off = o0;
    s_len = o1 - o0;
  }
  __syncthreads();
  const unsigned nnz = s_nnz;
  const int pbytes = 64 * ES + NMW * 4 + (int)nnz * ES;
  const unsigned *c32 = reinterpret_cast<const unsigned *>(a.in + a.data0 + s_off);

  // ---- stage-2 inverse into the payload buffer P
  if (!s_bad) {
    if (a.stage2) {
      const int W = pbytes / 4, E = pbytes / ES;
      const unsigned ntok = s_ntok;
      const unsigned long long nlit_avail = (s_len - 8 - 4ull * ntok) / 4;
      const unsigned *tok = c32 + 2;
      const unsigned *lit = tok + ntok;
      unsigned *P32 = reinterpret_cast<unsigned *>(P);
      for (int w = tid; w < W; w += NT) P32[w] = 0u;
      __syncthreads();
      unsigned lit_carry = 0, out_carry = 0;
      bool bad = false;
      for (unsigned r0 = 0; r0 < ntok; r0 += NT) {
        const unsigned k = r0 + tid;
        const unsigned tk = k < ntok ? tok[k] : 0u;
        const unsigned nl = tk & 0xFFFFu, run = nl + (tk >> 16);
        unsigned tl, to_;
        const unsigned lp = block_exsum<NT>(nl, s_u, tl);
        const unsigned op = block_exsum<NT>(run, s_u, to_);
        TL[tid] = lit_carry + lp;
        TO[tid] = out_carry + op;
        __syncthreads();
        const unsigned cnt = (ntok - r0) < (unsigned)NT ? (ntok - r0) : (unsigned)NT;
        for (unsigned l = lit_carry + tid; l < lit_carry + tl; l += NT) {
          unsigned lo = 0, hi = cnt - 1;  // largest kk with TL[kk] <= l
          while (lo < hi) {
            const unsigned mid = (lo + hi + 1) >> 1;
            if (TL[mid] <= l) lo = mid; else hi = mid - 1;
          }
          const unsigned ow = TO[lo] + (l - TL[lo]);
          if (l < nlit_avail && ow < (unsigned)W) unshuffle_word(P, (int)ow, lit[l], E, ES);
          else bad = true;
        }
        lit_carry += tl;
        out_carry += to_;
        __syncthreads();
      }
      if (bad || out_carry != (unsigned)W || (unsigned long long)lit_carry > nlit_avail) atomicOr(&s_bad, 1u);
    } else {
      unsigned *P32 = reinterpret_cast<unsigned *>(P);
      for (int w = tid; w < pbytes / 4; w += NT) P32[w] = c32[2 + w];
    }
  }
  __syncthreads();

  // ---- mask words -> positions of kept details
  const unsigned *MASK = reinterpret_cast<const unsigned *>(P + 64 * ES);
  if (!s_bad) {
    constexpr int IPT = (NMW + NT - 1) / NT;
    unsigned loc[IPT];
    unsigned sum = 0;
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
      const int k = tid * IPT + q;
      loc[q] = k < NMW ? (unsigned)__popc(MASK[k]) : 0u;
      sum += loc[q];
    }
    unsigned tot;
    unsigned ex = block_exsum<NT>(sum, s_u, tot);
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
      const int k = tid * IPT + q;
      if (k < NMW) WC[k] = ex;
      ex += loc[q];
    }
    if (tid < 64) {  // coarse positions carry no mask bit
      const int cx = tid & 3, cy = (tid >> 2) & 3, cz = tid >> 4;
      const int li = ((cz * Q) * B + cy * Q) * B + cx * Q;
      if ((MASK[li >> 5] >> (li & 31)) & 1u) atomicOr(&s_bad, 1u);
    }
    if (tid == 0 && tot != nnz) atomicOr(&s_bad, 1u);
  }
  __syncthreads();
  const bool bad = s_bad != 0;
  if (bad && tid == 0) atomicCAS(&ws->status, 0u, ST_CORRUPT);

  // ---- a7: scatter, inverse transform, store
  T v[B];
  {
    const bool xyq = (x % Q == 0) && (y % Q == 0);
    const T *COARSE = reinterpret_cast<const T *>(P);
    const T *VALS = reinterpret_cast<const T *>(P + 64 * ES + NMW * 4);
    const unsigned ltm = (1u << lane) - 1u;
#pragma unroll
    for (int z = 0; z < B; ++z) {
      T r = T(0);
      if (!bad) {
        if (xyq && (z % Q == 0)) {
          r = COARSE[((z / Q) * 4 + y / Q) * 4 + x / Q];
        } else {
          const unsigned wd = MASK[z * NW + wid];
          if ((wd >> lane) & 1u) r = VALS[WC[z * NW + wid] + __popc(wd & ltm)];
        }
      }
      v[z] = r;
    }
  }
  __syncthreads();
  if (!bad) inv_transform<T, B, KIND>(v, X, x, y);
  {
    const size_t zs = (size_t)a.ny * a.nx;
    T *dst = reinterpret_cast<T *>(a.field) + (size_t)(bz * B) * zs + (size_t)(by * B + y) * a.nx +
             (size_t)(bx * B + x);
#pragma unroll
    for (int z = 0; z < B; ++z) __stcs(dst + z * zs, v[z]);
  }
}

// ============================================================ dense transforms
template <typename T, int B, int KIND, bool FWD>
__global__ void __launch_bounds__(B * B) k_dense(const DenseArgs a)
{
  using G = Geo<T, B>;
  extern __shared__ __align__(16) unsigned char smem[];
  T *X = reinterpret_cast<T *>(smem);
  const int tid = threadIdx.x, x = tid % B, y = tid / B;
  const int bid = blockIdx.x;
  const int bx = bid % a.nbx, by = (bid / a.nbx) % a.nby, bz = bid / (a.nbx * a.nby);
  const size_t zs = (size_t)a.ny * a.nx;
  const size_t off = (size_t)(bz * B) * zs + (size_t)(by * B + y) * a.nx + (size_t)(bx * B + x);
  const T *src = reinterpret_cast<const T *>(a.src) + off;
  T *dst = reinterpret_cast<T *>(a.dst) + off;
  T v[B];
#pragma unroll
  for (int z = 0; z < B; ++z) v[z] = src[z * zs];
  if constexpr (FWD)
    fwd_transform<T, B, KIND>(v, X, x, y);
  else
    inv_transform<T, B, KIND>(v, X, x, y);
#pragma unroll
  for (int z = 0; z < B; ++z) dst[z * zs] = v[z];
  (void)G::L;
}

// ============================================================ a0: min / max
template <typename T>
__global__ void __launch_bounds__(512) k_minmax(const T *__restrict__ xs, size_t n, WsHdr *ws)
{
  T lo = (T)INFINITY, hi = (T)-INFINITY;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if constexpr (sizeof(T) == 4) {
    const float4 *v4 = reinterpret_cast<const float4 *>(xs);
    const size_t n4 = n / 4;
    for (size_t k = i; k < n4; k += stride) {
      const float4 q = __ldcs(v4 + k);
      lo = q.x < lo ? q.x : lo; hi = q.x > hi ? q.x : hi;
      lo = q.y < lo ? q.y : lo; hi = q.y > hi ? q.y : hi;
      lo = q.z < lo ? q.z : lo; hi = q.z > hi ? q.z : hi;
      lo = q.w < lo ? q.w : lo; hi = q.w > hi ? q.w : hi;
    }
    for (size_t k = n4 * 4 + i; k < n; k += stride) {
      const T q = xs[k];
      lo = q < lo ? q : lo;
      hi = q > hi ? q : hi;
    }
  } else {
    const double2 *v2 = reinterpret_cast<const double2 *>(xs);
    const size_t n2 = n / 2;
    for (size_t k = i; k < n2; k += stride) {
      const double2 q = __ldcs(v2 + k);
      lo = q.x < lo ? q.x : lo; hi = q.x > hi ? q.x : hi;
      lo = q.y < lo ? q.y : lo; hi = q.y > hi ? q.y : hi;
    }
    for (size_t k = n2 * 2 + i; k < n; k += stride) {
      const T q = xs[k];
      lo = q < lo ? q : lo;
      hi = q > hi ? q : hi;
    }
  }
  // NaN never enters: every comparison with NaN is false
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const T l2 = __shfl_xor_sync(FULL, lo, o), h2 = __shfl_xor_sync(FULL, hi, o);
    lo = l2 < lo ? l2 : lo;
    hi = h2 > hi ? h2 : hi;
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&ws->minkey, order_key(lo));
    atomicMax(&ws->maxkey, order_key(hi));
  }
}

}  // namespace czk
