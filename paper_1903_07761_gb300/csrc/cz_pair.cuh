// cz_pair.cuh -- the codec kernels in the "pair quad" layout.
//
// A CTA owns one cubic B^3 block with B^2/2 threads.  Thread (a, k, h) keeps
// the z-columns at x = 2a, 2a + 1 of rows y = 2k, 2k + 1, over the half
// z = h B/2 .. h B/2 + B/2 - 1, in registers as packed pairs, so
//   * at the finest level the x-transform of a pair is local except for the
//     neighbouring pairs' values (warp shuffles over the B/2 lanes of a
//     segment), the y-transform of a row pair is local except for the
//     neighbouring row pairs' values (one shared-memory plane), and the
//     z-transform is register code except for the two pairs next to the
//     middle of the column (a small shared-memory halo);
//   * the half h is the same across a warp (B >= 16), so the z-steps'
//     compile-time stencils of the two halves never diverge within a warp;
//   * coarser levels live on the coarse values only, gathered in a
//     shared-memory cube and transformed one line per thread.
// Every value is produced by the same operation sequence as the reference
// definition of each wavelet step (explicitly rounded, never fused).
//
// Significance: a thread's bits over its half columns (bit 2 zl + p for column
// 2a + p) become the stream's row words (bit x of row (z, y)) by a bit
// transpose over the lanes of a segment.
//
// Compression runs as two kernels (cz_compress.cuh): a persistent stage
// kernel that turns blocks into finished chunks in workspace staging while
// the next tile arrives by TMA, and a placement kernel that computes chunk
// offsets with a decoupled look-back and copies the chunks into the stream.
#pragma once

#include <cuda.h>

#include <type_traits>

#include "cz_device.cuh"

namespace czp {
using namespace czd;

// numeric values of the public status codes
constexpr unsigned ST_ARG = (unsigned)-1;
constexpr unsigned ST_CAPACITY = (unsigned)-2;
constexpr unsigned ST_CORRUPT = (unsigned)-3;
constexpr unsigned ST_TIMEOUT = (unsigned)-4;
constexpr int HEADER_BYTES = 128;
constexpr unsigned MAGIC = 0x315A4343u;
constexpr int WS_HDR = 256;
constexpr unsigned WAIT_LIMIT = 1u << 24;

// workspace header (the look-back words, the block table, the overflow
// scratch and the chunk staging area follow it)
struct WsHdr {
  unsigned status;
  unsigned ticket;
  unsigned nbig;  // blocks whose payload exceeds the small stage-2 CTAs' capacity
  unsigned nbig2;  // aggregate chunks: groups beyond the second coder (or decoder) tier
  unsigned long long minkey, maxkey;
  unsigned long long out_bytes;
  unsigned long long bump;  // staging bytes handed out so far
  // speculative thresholds: min / max keys of a subsample of the field
  // (every 4th row of every 4th z-plane), a lower bound of the range, and
  // the count of the slots listed for refinement
  unsigned long long skmin, skmax;
  unsigned nref, pad2;
};

// ---- several fields in one launch (one group: same type, block, kind)
constexpr int MAXF = 32;  // fields per batched launch

// per-field geometry and threshold inputs of the stage kernel
struct FieldGeo {
  const void *field;    // the field (read directly by the slab kernels)
  int nbx, nby, first;  // block grid (x, y) and the field's first global block
  int eps_mode;
  double eps, range_in;  // range_in < 0: range from this field's min/max keys
};

// tensor maps (and geometry) of the fields of one launch, passed by value
template <int NF>
struct StageMaps {
  CUtensorMap tm[NF];
  FieldGeo g[NF];
};

// per-field output description of the placement and copy kernels
struct FieldOut {
  unsigned char *out;
  unsigned long long *out_bytes;  // device u64 or null
  unsigned long long out_cap, data0;
  double eps, range_in;
  int nx, ny, nz, nblocks, first, tfirst;  // blocks, first global block, first global tile
  int eps_mode;
};

struct BatchOut {
  FieldOut f[MAXF];
  int nf;
};

struct FwdArgs {
  const void *field;
  void *ws;
  int *biglist;  // ids of the blocks with large payloads (count in the header's nbig)
  unsigned long long *keys;  // batched: min/max keys, two per field
  unsigned char *staging;     // raw payloads, one arena per CTA
  unsigned long long *table;  // per block: staging offset, nnz
  unsigned long long arena_bytes;
  unsigned char *scratch;  // slab kernels: one G2::SCRATCH block per CTA
  double eps, range, cnorm;
  int nx, ny, nz, nbx, nby, nbz, nblocks, nf;
  int eps_mode, stage2, kind, dtype;
  int zbits;  // bit zeroing: 0, 4 or 8 least significant bits of each kept detail cleared
  // speculative thresholds (one field, range computed): the stage kernel
  // merges each warp's min / max into the header's keys and thresholds at
  // t_lo <= t, the threshold of a subsample's range (the header's skmin /
  // skmax); near[bid] = 1 where the block kept a value below
  // near_threshold(t_lo); stage 2 drops the details below the exact t
  int spec;
  unsigned char *near;
};

struct InvArgs {
  const unsigned char *in;
  void *field;
  void *ws;
  const unsigned char *staging;       // stage 2: decoded payloads, one slot per block
  const unsigned long long *table;    // stage 2: per block nnz, bad flag
  const int *ids;                     // random access: chunk of each decoded block (else the identity)
  int nchunks;                        // blocks in the stream
  unsigned long long in_bytes, data0, slot;
  int nx, ny, nz, nbx, nby, nbz, nblocks;
  int stage2;
  int decoder;  // host side: 0 = one CTA per block, 1 = two CTAs per block (half blocks)
};

// stage-2 decoding: chunk -> raw payload in a staging slot
struct UnArgs {
  const unsigned char *in;
  unsigned char *staging;
  unsigned long long *table;  // per block: nnz, bad flag
  void *ws;                   // header: count of large chunks (nbig)
  int *biglist;               // ids of the chunks with large payloads
  unsigned char *scratch;     // FP64 32^3: shuffled payloads, one G2::SCRATCH block per large CTA
  const int *ids;             // random access: chunk of each decoded block (else the identity)
  int nchunks;                // blocks in the stream
  unsigned long long in_bytes, data0, slot;
  int nblocks;
  int group;                  // blocks per aggregate chunk (1: one chunk per block)
  int hcap;                   // aggregate chunks: scratch bytes per CTA of the large launch
};

struct DenseArgs {
  const void *src;
  void *dst;
  int nx, ny, nz, nbx, nby, nbz;
};

// ------------------------------------------------------------ pairs
template <typename T>
struct V2T;
template <>
struct V2T<float> {
  using type = float2;
};
template <>
struct V2T<double> {
  using type = double2;
};

__device__ __forceinline__ float2 mk2(float s) { return make_float2(s, s); }
__device__ __forceinline__ double2 mk2(double s) { return make_double2(s, s); }
// Pair arithmetic.  FP32 sums and differences of pairs are one packed
// add.rn.f32x2 / sub.rn.f32x2 each: both round each lane exactly like the
// scalar operation (IEEE round to nearest, subnormals kept).  Products stay
// two explicitly rounded scalar multiplies: chained packed multiply -> add
// sequences were measured to differ from separately rounded scalar ops, so
// no packed product feeds a packed sum on the exact path.  FP64 pairs are
// scalar throughout.
#ifdef CZ_FAST
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return make_float2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ double2 add2(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 mul2(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 sub2(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
#else
__device__ __forceinline__ unsigned long long pk2(float2 a)
{
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
__device__ __forceinline__ float2 upk2(unsigned long long r)
{
  float2 a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
  return a;
}
__device__ __forceinline__ float2 add2(float2 a, float2 b)
{
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
  return upk2(d);
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b)
{
  return make_float2(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y));
}
__device__ __forceinline__ double2 add2(double2 a, double2 b)
{
  return make_double2(__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y));
}
__device__ __forceinline__ double2 mul2(double2 a, double2 b)
{
  return make_double2(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y));
}
// subtraction lane by lane (exactly a - b, signed zeros included)
__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
  return upk2(d);
}
__device__ __forceinline__ double2 sub2(double2 a, double2 b)
{
  return make_double2(__dsub_rn(a.x, b.x), __dsub_rn(a.y, b.y));
}
#endif

// significance: keep iff !(|d| < t) (ties kept; a NaN detail or a NaN
// threshold keeps the value)
__device__ __forceinline__ bool keep(float d, float t) { return !(fabsf(d) < t); }
__device__ __forceinline__ bool keep(double d, double t) { return !(fabs(d) < t); }

// the value with the zbits least significant bits of its pattern cleared
__device__ __forceinline__ float zero_low(float v, int zbits)
{
  return __uint_as_float(__float_as_uint(v) & ~((1u << zbits) - 1u));
}
__device__ __forceinline__ double zero_low(double v, int zbits)
{
  return __longlong_as_double(__double_as_longlong(v) & ~((1ll << zbits) - 1ll));
}

// Significance bits of a thread's half columns: bit 2 zl + p for component
// p of v[zl].  For FP32 the sign of |d| - t (explicitly rounded, subnormals
// kept) is the rule: negative iff |d| < t; +0 on a tie; NaN (positive, the
// canonical GPU NaN) for a NaN detail or threshold; one funnel shift per
// value collects the "dropped" sign bits.
template <int ZH>
__device__ __forceinline__ unsigned keep_bits(const float2 (&v)[ZH], float t)
{
  unsigned nk = 0;
#pragma unroll
  for (int zl = ZH - 1; zl >= 0; --zl) {
    nk = __funnelshift_l(__float_as_uint(__fsub_rn(fabsf(v[zl].y), t)), nk, 1);
    nk = __funnelshift_l(__float_as_uint(__fsub_rn(fabsf(v[zl].x), t)), nk, 1);
  }
  return ZH == 16 ? ~nk : (~nk & ((1u << (2 * ZH)) - 1u));
}

template <int ZH>
__device__ __forceinline__ unsigned keep_bits(const double2 (&v)[ZH], double t)
{
  unsigned w = 0;
#pragma unroll
  for (int zl = 0; zl < ZH; ++zl)
    w |= ((unsigned)keep(v[zl].x, t) << (2 * zl)) | ((unsigned)keep(v[zl].y, t) << (2 * zl + 1));
  return w;
}

// ------------------------------------------------------------ geometry
template <typename T, int B>
struct G2 {
  static constexpr int NT = B * B / 2;
  static constexpr int NW = NT / 32;
  static constexpr int HP = B / 2;  // lanes of a segment: the x-pairs of a row
  static constexpr int NK = B / 2;  // row pairs (y = 2k, 2k + 1)
  static constexpr int ZH = B / 2;  // z-values of one half column
  static constexpr int MH = B / 4;  // z-pairs of one half column
  static constexpr int L = (B == 8) ? 1 : (B == 16) ? 2 : (B == 32) ? 3 : 4;
  // FP64 32^3 blocks (256 KiB) and 64^3 blocks (1 MiB FP32) fit neither
  // the registers nor the shared memory of one CTA: they take the slab
  // kernels (cz_slab.cuh), whose block lives in global memory (a scratch
  // block per CTA, L2-resident), and large stage-2 payloads are shuffled in
  // global scratch too
  static constexpr bool SLAB = (sizeof(T) == 8 && B == 32) || B == 64;
  // W4li with FP32 32^3 blocks runs the finest x-level row by row in shared
  // memory (rowx), on tiles the TMA copies with the 128-byte swizzle (their
  // rows are 128 bytes): its x-step with shuffles costs more than the extra
  // shared-memory traffic (measured: compression -12 %, decompression
  // -16 %), while W4 and W3ai are faster with the shuffles on plain tiles.
  template <int KIND>
  static constexpr bool rowx() { return sizeof(T) == 4 && B == 32 && KIND == W4LI; }
  static constexpr int Q = B / 4;
  static constexpr int ES = (int)sizeof(T);
  static constexpr int LGES = ES == 8 ? 3 : 2;
  static constexpr int NVOX = B * B * B;
  static constexpr int NMW = NVOX / 32;
  static constexpr int MASKB = NVOX / 8;
  static constexpr int PMAX = 64 * ES + MASKB + (NVOX - 64) * ES;
  static constexpr int WMAX = PMAX / 4;
  static constexpr int NBWMAX = (WMAX + 31) / 32;
  static constexpr int TILE = NVOX * ES;
  // level-0 exchange areas: the y plane holds one pair value per (z, k, a),
  // the z halo two pair values per (step, half, row, k, a)
  static constexpr int PLANE = B * NK * HP * 2 * ES;
  static constexpr int HALO = 2 * 2 * 2 * 2 * NK * HP * 2 * ES;
  // cube of the coarser levels: (B/2)^2 rows of B/2 + 1 elements
  static constexpr int CUBE = L > 1 ? (B / 2) * (B / 2) * (B / 2 + 1) * ES : 0;
  static constexpr int CUBE_AL = (CUBE + 127) / 128 * 128;
  // row offsets and mask rows in shared memory: B + 1 rows per z, so that
  // the rows of one y over consecutive z fall in distinct banks
  static constexpr int ROWB = B * (B + 1) * 4;
  static constexpr int MASKBP = B * (B + 1) * B / 8;
  static constexpr int PMAX_AL = (PMAX + 127) / 128 * 128;
  // stage kernel: tile | plane area (the cube at its start) | halo area
  // (after the transform: the row offsets and the mask rows)
  static constexpr int PLC0 = PLANE > CUBE_AL ? PLANE : CUBE_AL;
  static constexpr int PLC = (PLC0 + 127) / 128 * 128;
  // (+ 1 KiB: the kernels align their shared memory to 1024 bytes, the
  // period of the 128-byte swizzle)
  static constexpr int SMEM_C = TILE + PLC + HALO + 1024;
  // staging slot of one block: [nnz | 0 | raw payload]; the finished
  // stage-2 chunk replaces it in place and is at most 12 bytes longer than
  // the payload (every coded run of >= 2 zero words saves at least one
  // word; one trailing token), plus one token per 65535 literal words that
  // a payload of more than 65535 words may split off (slab lanes only), so
  // a slot holds payload + 12 + 4 * (words / 65535) bytes
  static constexpr int PSLOT = (PMAX + 12 + 4 * (WMAX / 65535) + 15) / 16 * 16;
  // stage-2 kernels: the shuffled payload lives in shared memory; payloads
  // of up to SHCAP bytes go to small CTAs, larger ones to large CTAs
  static constexpr int SHCAP = PMAX_AL < 16384 ? PMAX_AL : 16384;
  static constexpr int NBS = (SHCAP / 4 + 31) / 32;
  static constexpr int SMEM_S2 = SHCAP + 4 * NBS * 4;
  static constexpr bool HAS_BIG = SHCAP < PMAX;
  static constexpr int SMEM_S2B = PMAX_AL + 4 * NBWMAX * 4;
  // stage-2 inverse kernels: payload + three per-token arrays
  static constexpr int SMEM_U = SHCAP + 3 * 128 * 4;
  static constexpr int SMEM_UB = (SLAB ? 0 : PMAX_AL) + 3 * 512 * 4;
  // dense kernels: cube | plane | halo
  static constexpr int SMEM_DN0 = CUBE_AL + PLANE + HALO;
  // decompress: cube | row offsets | payload buffers | output tile, which
  // holds the plane and the halo while level 0 runs
  static constexpr int R2D = CUBE_AL + (ROWB + 127) / 128 * 128;
  // decompress payload buffer: whole payloads of up to PBCAP bytes (with
  // 32^3 blocks most payloads, the rest read their values from global memory)
  static constexpr int PBCAP = B == 32 ? (PMAX_AL < 16384 ? PMAX_AL : 16384) : PMAX_AL;
  // payload buffers: with 32^3 blocks (one CTA per SM) a copy is issued two
  // blocks ahead; smaller blocks keep two buffers and more CTAs per SM
  static constexpr int NPB = B == 32 ? 3 : 2;
  static constexpr int OTB0 = TILE > PLANE + HALO ? TILE : PLANE + HALO;
  static constexpr int OTB = (OTB0 + 127) / 128 * 128;
  static constexpr int SMEM_D = OTB + R2D + NPB * PBCAP + 1024;
  static constexpr int SCRATCH = SLAB ? (PMAX_AL > TILE ? PMAX_AL : TILE) : 0;  // per CTA
  static_assert(HP == NK && NK == ZH && NT == HP * NK * 2, "thread grid");
  static_assert(HALO >= ROWB + MASKBP, "row offsets and mask rows fit the halo area");
  static_assert(SLAB || SMEM_C <= 227 * 1024 - 512, "stage kernel shared memory");
  static_assert(SLAB || SMEM_D <= 227 * 1024 - 512, "decompress shared memory");
  static_assert(SLAB || SMEM_S2B <= 227 * 1024 - 1024, "stage-2 shared memory");
  static_assert(SLAB || WMAX < 65536, "zero-RLE tokens hold run lengths below 65536 words");
};

// ------------------------------------------------------------ TMA / mbarrier
__device__ __forceinline__ unsigned smem_u32(const void *p)
{
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar)
{
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void tma_load_tile(const CUtensorMap *tm, void *dst, unsigned long long *bar,
                                              int x, int y, int z, unsigned bytes)
{
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(tm)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// 1D bulk copy global -> shared (addresses 16-byte aligned, bytes a
// multiple of 16) completing on the mbarrier
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, unsigned long long *bar)
{
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(reinterpret_cast<unsigned long long>(src)), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// tiled 3D store shared -> global of one box, in the CTA's bulk group
// (callers fence the generic writes to the tile and synchronise first)
__device__ __forceinline__ void tma_store_tile(const CUtensorMap *tm, const void *src, int x, int y, int z)
{
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
                   reinterpret_cast<unsigned long long>(tm)),
               "r"(smem_u32(src)), "r"(x), "r"(y), "r"(z)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// 16-byte asynchronous copy global -> shared (no register waits on it)
__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n\tcp.async.commit_group;" ::"r"(smem_u32(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// the CTA's bulk stores have finished reading shared memory
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

// the CTA's bulk stores are complete
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// generic-proxy writes to shared memory, made visible to the async proxy
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// bounded wait for the mbarrier phase with the given parity; false on
// timeout.  A timeout is one thread's view: the kernels record it in a
// shared flag and decide at their next barrier, all threads together,
// whether the CTA gives up (so no thread is left waiting at a barrier for
// threads that have gone).
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, unsigned limit = WAIT_LIMIT)
{
  const unsigned addr = smem_u32(bar);
  for (unsigned it = 0; it < limit; ++it) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// the dynamic shared memory rounded up to 1024 bytes (the period of the
// 128-byte TMA swizzle); the kernels allocate 1 KiB more
__device__ __forceinline__ unsigned char *align1024(unsigned char *p)
{
  return p + ((1024u - (smem_u32(p) & 1023u)) & 1023u);
}

// byte offset o of a tile of 128-byte rows as the 128-byte TMA swizzle
// places it: 16-byte chunk c of row r lands at chunk c ^ (r mod 8)
__device__ __forceinline__ unsigned swz128(unsigned o) { return o ^ ((o >> 3) & 0x70u); }

// ------------------------------------------------------------ thread grid
// Thread tid holds x-pair a of row pair k over z-half h.  With B >= 16 the
// warps alternate between the halves, so the warps holding the boundary row
// pairs (whose y-step takes the longer general form) land on four different
// schedulers; the half stays the same across a warp.
template <int B>
__device__ __forceinline__ void quad_of(int tid, int &a, int &k, int &h)
{
  constexpr int HP = B / 2, NT = B * B / 2;
  if constexpr (NT >= 64) {
    const int w = tid >> 5, lane = tid & 31;
    h = w & 1;
    k = (w >> 1) * (32 / HP) + lane / HP;
    a = lane % HP;
  } else {
    a = tid % HP;
    k = (tid / HP) % (B / 2);
    h = tid / (NT / 2);
  }
}

// ------------------------------------------------------------ block walk
// Block coordinates of bid, bid + step, bid + 2 step, ... of an nbx x nby x
// nbz block grid, advanced without divisions: step's digits are added with
// one carry per axis.  Kept in shared memory and used by one thread.
struct BlockWalk {
  int bx, by, bz, sx, sy, sz, nbx, nby;
  __device__ __forceinline__ void init(int bid, int step, int nbx_, int nby_)
  {
    nbx = nbx_;
    nby = nby_;
    bx = bid % nbx;
    by = (bid / nbx) % nby;
    bz = bid / (nbx * nby);
    sx = step % nbx;
    sy = (step / nbx) % nby;
    sz = step / (nbx * nby);
  }
  __device__ __forceinline__ void next()
  {
    int x = bx + sx, c = x >= nbx;
    bx = c ? x - nbx : x;
    int y = by + sy + c;
    c = y >= nby;
    by = c ? y - nby : y;
    bz += sz + c;
  }
};

// ------------------------------------------------------------ bit transpose
// Over the B/2 lanes of a segment: lane a holds w with bit 2i + p = entry
// (x = 2a + p, i) of a B x (B/2) bit matrix; afterwards lane a holds the word
// of i = a, bit x.  The same steps map such words back.  Recursive block
// swap (Hacker's Delight 7-3) in which word bit distance j pairs with lane
// distance j/2.
template <int B>
__device__ __forceinline__ unsigned seg_transpose(unsigned w, int a)
{
#pragma unroll
  for (int j = B / 2; j >= 2; j >>= 1) {
    const unsigned m = j == 16 ? 0x0000FFFFu : j == 8 ? 0x00FF00FFu : j == 4 ? 0x0F0F0F0Fu : 0x33333333u;
    const int ld = j >> 1;
    const unsigned p = __shfl_xor_sync(FULL, w, ld);
    if (!(a & ld))
      w ^= (((w >> j) ^ p) & m) << j;
    else
      w ^= ((p >> j) ^ w) & m;
  }
  return w;
}

// ============================================================ level 0 (pairs)
// per-lane stencil of the finest x-level: pair a holds coarse node a (E)
// and detail a (O) of its row
template <typename T>
struct XSt {
  int src[4];  // W4: lanes of the four coarse sources
  T w[4];
  int usrc[3];  // W4li: lanes of the update details
  T uw[3];
  int nt;
  int s1, s2;  // W3ai: lanes of the two average sources
  T aw[3];
  bool bnd;
};

template <typename T, int KIND>
__device__ __forceinline__ XSt<T> make_xst(int a, int m, int seg)
{
  XSt<T> s;
  if (KIND == W4 || KIND == W4LI) {
    const W4Row r = w4_row(a, m);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      s.src[q] = seg + r.j0 + q;
      s.w[q] = (T)r.w[q];
    }
  }
  if (KIND == W4LI) {
    const LiSrc ls = li_src(a, m);
    s.nt = ls.nt;
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      int kk = ls.k0 + t;
      kk = kk < m ? kk : m - 1;
      s.usrc[t] = seg + kk;
      s.uw[t] = li_lookup<T>(m, a, t);
    }
  }
  if (KIND == W3AI) {
    const AiRow r = ai_row(a, m);
    s.s1 = seg + r.s1;
    s.s2 = seg + r.s2;
    s.aw[0] = (T)r.w0;
    s.aw[1] = (T)r.w1;
    s.aw[2] = (T)r.w2;
    s.bnd = r.bnd;
  }
  return s;
}

template <typename T>
__device__ __forceinline__ T pred4s(const T (&w)[4], T c0, T c1, T c2, T c3)
{
  T p = mulx(w[0], c0);
  p = addx(p, mulx(w[1], c1));
  p = addx(p, mulx(w[2], c2));
  p = addx(p, mulx(w[3], c3));
  return mulx(p, (T)0.0625);
}

template <typename T>
__device__ __forceinline__ T ai_preds(T a, T a1, T a2, T w0, T w1, T w2, bool bnd)
{
  const T x0 = bnd ? a : a1, x1 = bnd ? a1 : a2;
  T q = addx(mulx(w0, x0), mulx(w1, x1));
  if (bnd) q = addx(q, mulx(w2, a2));
  return addx(a, mulx(q, (T)0.125));
}

template <typename T, int KIND, typename T2>
__device__ __forceinline__ void x0_fwd(const XSt<T> &s, T2 &v)
{
  T E = v.x, O = v.y;
  if constexpr (KIND == W4 || KIND == W4LI) {
    const T c0 = shfl(E, s.src[0]), c1 = shfl(E, s.src[1]), c2 = shfl(E, s.src[2]), c3 = shfl(E, s.src[3]);
    O = subx(O, pred4s(s.w, c0, c1, c2, c3));
    if constexpr (KIND == W4LI) {
      const T d0 = shfl(O, s.usrc[0]), d1 = shfl(O, s.usrc[1]), d2 = shfl(O, s.usrc[2]);
      T acc = mulx(s.uw[0], d0);
      if (s.nt > 1) acc = addx(acc, mulx(s.uw[1], d1));
      if (s.nt > 2) acc = addx(acc, mulx(s.uw[2], d2));
      E = addx(E, acc);
    }
  } else {
    const T a = mulx(addx(E, O), (T)0.5);
    const T a1 = shfl(a, s.s1), a2 = shfl(a, s.s2);
    O = subx(E, ai_preds(a, a1, a2, s.aw[0], s.aw[1], s.aw[2], s.bnd));
    E = a;
  }
  v.x = E;
  v.y = O;
}

template <typename T, int KIND, typename T2>
__device__ __forceinline__ void x0_inv(const XSt<T> &s, T2 &v)
{
  T E = v.x, O = v.y;
  if constexpr (KIND == W4 || KIND == W4LI) {
    if constexpr (KIND == W4LI) {
      const T d0 = shfl(O, s.usrc[0]), d1 = shfl(O, s.usrc[1]), d2 = shfl(O, s.usrc[2]);
      T acc = mulx(s.uw[0], d0);
      if (s.nt > 1) acc = addx(acc, mulx(s.uw[1], d1));
      if (s.nt > 2) acc = addx(acc, mulx(s.uw[2], d2));
      E = subx(E, acc);
    }
    const T c0 = shfl(E, s.src[0]), c1 = shfl(E, s.src[1]), c2 = shfl(E, s.src[2]), c3 = shfl(E, s.src[3]);
    O = addx(O, pred4s(s.w, c0, c1, c2, c3));
  } else {
    const T a1 = shfl(E, s.s1), a2 = shfl(E, s.s2);
    const T f0 = addx(ai_preds(E, a1, a2, s.aw[0], s.aw[1], s.aw[2], s.bnd), O);
    O = subx(mulx((T)2, E), f0);
    E = f0;
  }
  v.x = E;
  v.y = O;
}

// ---- packed forms for the y- and z-levels of the pairs (both columns)
template <typename T2, typename T>
__device__ __forceinline__ T2 pred4p(const T (&w)[4], T2 c0, T2 c1, T2 c2, T2 c3)
{
  T2 p = mul2(mk2(w[0]), c0);
  p = add2(p, mul2(mk2(w[1]), c1));
  p = add2(p, mul2(mk2(w[2]), c2));
  p = add2(p, mul2(mk2(w[3]), c3));
  return mul2(p, mk2((T)0.0625));
}

template <typename T2, typename T>
__device__ __forceinline__ T2 ai_predp(T2 a, T2 a1, T2 a2, T w0, T w1, T w2, bool bnd)
{
  const T2 x0 = bnd ? a : a1, x1 = bnd ? a1 : a2;
  T2 q = add2(mul2(mk2(w0), x0), mul2(mk2(w1), x1));
  if (bnd) q = add2(q, mul2(mk2(w2), a2));
  return add2(a, mul2(q, mk2((T)0.125)));
}

// packed interior W4 row (weights -1, 9, 9, -1; see pred4i)
template <typename T2, typename T>
__device__ __forceinline__ T2 pred4ip(T2 c0, T2 c1, T2 c2, T2 c3)
{
  T2 p = sub2(mul2(mk2((T)9), c1), c0);
  p = add2(p, mul2(mk2((T)9), c2));
  p = sub2(p, c3);
  return mul2(p, mk2((T)0.0625));
}

// packed compile-time W4 row
template <typename T2, typename T>
__device__ __forceinline__ T2 pred4rp(const W4Row &r, T2 c0, T2 c1, T2 c2, T2 c3)
{
  if (r.w[0] == -1 && r.w[1] == 9 && r.w[2] == 9 && r.w[3] == -1) return pred4ip<T2, T>(c0, c1, c2, c3);
  const T w[4] = {(T)r.w[0], (T)r.w[1], (T)r.w[2], (T)r.w[3]};
  return pred4p<T2>(w, c0, c1, c2, c3);
}

// packed interior W3ai row (weights 1, -1)
template <typename T2, typename T>
__device__ __forceinline__ T2 ai_predip(T2 a, T2 a1, T2 a2)
{
  return add2(a, mul2(sub2(a1, a2), mk2((T)0.125)));
}

// the same with a compile-time row: interior rows (weights 1, -1) as one
// subtraction, which rounds exactly like the two exact products and the sum
template <typename T2, typename T>
__device__ __forceinline__ T2 ai_predc(const AiRow &r, T2 a, T2 a1, T2 a2)
{
  if (!r.bnd) return ai_predip<T2, T>(a, a1, a2);
  return ai_predp<T2>(a, a1, a2, (T)r.w0, (T)r.w1, (T)r.w2, true);
}

// ---- finest y-level: row pairs exchange one pair value per (z, k, a)
// through the plane P[z][k][a]
template <typename T>
struct YP {
  int e[4];  // W4: row pairs whose even rows predict
  T w[4];
  int d[3];  // W4li: row pairs whose details update
  T uw[3];
  int nt;
  int k1, k2;  // W3ai: row pairs of the two source averages
  T aw[3];
  bool bnd;
};

template <typename T, int KIND>
__device__ __forceinline__ YP<T> make_yp(int k, int m)
{
  YP<T> s;
  if (KIND == W4 || KIND == W4LI) {
    const W4Row r = w4_row(k, m);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      s.e[q] = r.j0 + q;
      s.w[q] = (T)r.w[q];
    }
  }
  if (KIND == W4LI) {
    const LiSrc ls = li_src(k, m);
    s.nt = ls.nt;
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      int kk = ls.k0 + t;
      kk = kk < m ? kk : m - 1;
      s.d[t] = kk;
      s.uw[t] = li_lookup<T>(m, k, t);
    }
  }
  if (KIND == W3AI) {
    const AiRow r = ai_row(k, m);
    s.k1 = r.s1;
    s.k2 = r.s2;
    s.aw[0] = (T)r.w0;
    s.aw[1] = (T)r.w1;
    s.aw[2] = (T)r.w2;
    s.bnd = r.bnd;
  }
  return s;
}

template <typename T2, typename T>
__device__ __forceinline__ T2 li_accp(const T (&uw)[3], int nt, T2 d0, T2 d1, T2 d2)
{
  T2 acc = mul2(mk2(uw[0]), d0);
  if (nt > 1) acc = add2(acc, mul2(mk2(uw[1]), d1));
  if (nt > 2) acc = add2(acc, mul2(mk2(uw[2]), d2));
  return acc;
}

// ============================================================ level 0
// Thread (a, k, h) holds v[r][zl] = (f(2a, 2k + r, z), f(2a + 1, 2k + r, z))
// for z = h B/2 + zl: an x-pair of both rows of a row pair over one half of
// the z-columns.  The x-step is local to a pair except for the neighbouring
// pairs' values (shuffles within the B/2-lane segment); the y-step is local
// to the row pair except for the neighbouring row pairs' values (the plane);
// the z-step is local to the half column except for two pairs next to the
// middle (the halo).  Every step evaluates the same rounded operations in
// the same order as the 1D definition of its wavelet.

template <int B, typename T2>
__device__ __forceinline__ T2 &plane_at(T2 *pl, int z, int k, int a)
{
  return pl[(z * (B / 2) + k) * (B / 2) + a];
}

// halo slot: step (0: predict inputs, 1: W4li update inputs), the half that
// wrote it, slot s, row r
template <int B, typename T2>
__device__ __forceinline__ T2 &halo_at(T2 *hx, int step, int half, int s, int r, int k, int a)
{
  return hx[((((step * 2 + half) * 2 + s) * 2 + r) * (B / 2) + k) * (B / 2) + a];
}

// ---- x
template <typename T, int B, int KIND, typename T2>
__device__ __forceinline__ void x_fwd(T2 (&v)[2][B / 2], int a, int seg)
{
  const XSt<T> s = make_xst<T, KIND>(a, B / 2, seg);
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int zl = 0; zl < B / 2; ++zl) x0_fwd<T, KIND>(s, v[r][zl]);
}

template <typename T, int B, int KIND, typename T2>
__device__ __forceinline__ void x_inv(T2 (&v)[2][B / 2], int a, int seg)
{
  const XSt<T> s = make_xst<T, KIND>(a, B / 2, seg);
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int zl = 0; zl < B / 2; ++zl) x0_inv<T, KIND>(s, v[r][zl]);
}

// ---- y (first_sync runs right after the first barrier).  A warp whose
// row pairs are all interior takes the interior forms of its rows (the same
// roundings); barriers stay outside the warp-uniform branches.
template <int KIND>
__device__ __forceinline__ bool y_interior(int k, int m)
{
  return KIND == W3AI ? (k >= 1 && k <= m - 2) : (k >= 1 && k <= m - 3);
}

template <typename T, int B, int KIND, typename T2, typename F>
__device__ __forceinline__ void y_fwd(T2 (&v)[2][B / 2], T2 *pl, int a, int k, int h, F &&first_sync)
{
  constexpr int ZH = B / 2, m = B / 2;
  const YP<T> s = make_yp<T, KIND>(k, m);
  const bool wint = __all_sync(FULL, y_interior<KIND>(k, m));
  const int z0 = h * ZH;
  if constexpr (KIND == W3AI) {
    // the odd row's slot takes the pair average
#pragma unroll
    for (int zl = 0; zl < ZH; ++zl) {
      v[1][zl] = mul2(add2(v[0][zl], v[1][zl]), mk2((T)0.5));
      plane_at<B>(pl, z0 + zl, k, a) = v[1][zl];
    }
    __syncthreads();
    first_sync();
    if (wint) {
#pragma unroll
      for (int zl = 0; zl < ZH; ++zl) {
        const T2 av = v[1][zl];
        const T2 a1 = plane_at<B>(pl, z0 + zl, k - 1, a), a2 = plane_at<B>(pl, z0 + zl, k + 1, a);
        v[1][zl] = sub2(v[0][zl], ai_predip<T2, T>(av, a1, a2));
        v[0][zl] = av;
      }
    } else {
#pragma unroll
      for (int zl = 0; zl < ZH; ++zl) {
        const T2 av = v[1][zl];
        const T2 a1 = plane_at<B>(pl, z0 + zl, s.k1, a), a2 = plane_at<B>(pl, z0 + zl, s.k2, a);
        v[1][zl] = sub2(v[0][zl], ai_predp<T2>(av, a1, a2, s.aw[0], s.aw[1], s.aw[2], s.bnd));
        v[0][zl] = av;
      }
    }
  } else {
#pragma unroll
    for (int zl = 0; zl < ZH; ++zl) plane_at<B>(pl, z0 + zl, k, a) = v[0][zl];
    __syncthreads();
    first_sync();
    if (wint) {
#pragma unroll
      for (int zl = 0; zl < ZH; ++zl) {
        const int z = z0 + zl;
        v[1][zl] = sub2(v[1][zl], pred4ip<T2, T>(plane_at<B>(pl, z, k - 1, a), plane_at<B>(pl, z, k, a),
                                                  plane_at<B>(pl, z, k + 1, a), plane_at<B>(pl, z, k + 2, a)));
      }
    } else {
#pragma unroll
      for (int zl = 0; zl < ZH; ++zl) {
        const int z = z0 + zl;
        v[1][zl] = sub2(v[1][zl], pred4p<T2>(s.w, plane_at<B>(pl, z, s.e[0], a), plane_at<B>(pl, z, s.e[1], a),
                                              plane_at<B>(pl, z, s.e[2], a), plane_at<B>(pl, z, s.e[3], a)));
      }
    }
    if constexpr (KIND == W4LI) {
      __syncthreads();
#pragma unroll
      for (int zl = 0; zl < ZH; ++zl) plane_at<B>(pl, z0 + zl, k, a) = v[1][zl];
      __syncthreads();
      if (wint) {  // two update terms: details k - 1 and k
#pragma unroll
        for (int zl = 0; zl < ZH; ++zl) {
          const int z = z0 + zl;
          const T2 acc = add2(mul2(mk2(s.uw[0]), plane_at<B>(pl, z, k - 1, a)),
                              mul2(mk2(s.uw[1]), plane_at<B>(pl, z, k, a)));
          v[0][zl] = add2(v[0][zl], acc);
        }
      } else {
#pragma unroll
        for (int zl = 0; zl < ZH; ++zl) {
          const int z = z0 + zl;
          v[0][zl] = add2(v[0][zl], li_accp<T2>(s.uw, s.nt, plane_at<B>(pl, z, s.d[0], a),
                                                 plane_at<B>(pl, z, s.d[1], a), plane_at<B>(pl, z, s.d[2], a)));
        }
      }
    }
  }
}

template <typename T, int B, int KIND, typename T2>
__device__ __forceinline__ void y_inv(T2 (&v)[2][B / 2], T2 *pl, int a, int k, int h)
{
  constexpr int ZH = B / 2, m = B / 2;
  const YP<T> s = make_yp<T, KIND>(k, m);
  const bool wint = __all_sync(FULL, y_interior<KIND>(k, m));
  const int z0 = h * ZH;
  if constexpr (KIND == W3AI) {
#pragma unroll
    for (int zl = 0; zl < ZH; ++zl) plane_at<B>(pl, z0 + zl, k, a) = v[0][zl];
    __syncthreads();
    if (wint) {
#pragma unroll
      for (int zl = 0; zl < ZH; ++zl) {
        const T2 a1 = plane_at<B>(pl, z0 + zl, k - 1, a), a2 = plane_at<B>(pl, z0 + zl, k + 1, a);
        const T2 f0 = add2(ai_predip<T2, T>(v[0][zl], a1, a2), v[1][zl]);
        v[1][zl] = sub2(add2(v[0][zl], v[0][zl]), f0);
        v[0][zl] = f0;
      }
    } else {
#pragma unroll
      for (int zl = 0; zl < ZH; ++zl) {
        const T2 a1 = plane_at<B>(pl, z0 + zl, s.k1, a), a2 = plane_at<B>(pl, z0 + zl, s.k2, a);
        const T2 f0 = add2(ai_predp<T2>(v[0][zl], a1, a2, s.aw[0], s.aw[1], s.aw[2], s.bnd), v[1][zl]);
        v[1][zl] = sub2(add2(v[0][zl], v[0][zl]), f0);
        v[0][zl] = f0;
      }
    }
  } else {
    if constexpr (KIND == W4LI) {
#pragma unroll
      for (int zl = 0; zl < ZH; ++zl) plane_at<B>(pl, z0 + zl, k, a) = v[1][zl];
      __syncthreads();
      if (wint) {
#pragma unroll
        for (int zl = 0; zl < ZH; ++zl) {
          const int z = z0 + zl;
          const T2 acc = add2(mul2(mk2(s.uw[0]), plane_at<B>(pl, z, k - 1, a)),
                              mul2(mk2(s.uw[1]), plane_at<B>(pl, z, k, a)));
          v[0][zl] = sub2(v[0][zl], acc);
        }
      } else {
#pragma unroll
        for (int zl = 0; zl < ZH; ++zl) {
          const int z = z0 + zl;
          v[0][zl] = sub2(v[0][zl], li_accp<T2>(s.uw, s.nt, plane_at<B>(pl, z, s.d[0], a),
                                                 plane_at<B>(pl, z, s.d[1], a), plane_at<B>(pl, z, s.d[2], a)));
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int zl = 0; zl < ZH; ++zl) plane_at<B>(pl, z0 + zl, k, a) = v[0][zl];
    __syncthreads();
    if (wint) {
#pragma unroll
      for (int zl = 0; zl < ZH; ++zl) {
        const int z = z0 + zl;
        v[1][zl] = add2(v[1][zl], pred4ip<T2, T>(plane_at<B>(pl, z, k - 1, a), plane_at<B>(pl, z, k, a),
                                                  plane_at<B>(pl, z, k + 1, a), plane_at<B>(pl, z, k + 2, a)));
      }
    } else {
#pragma unroll
      for (int zl = 0; zl < ZH; ++zl) {
        const int z = z0 + zl;
        v[1][zl] = add2(v[1][zl], pred4p<T2>(s.w, plane_at<B>(pl, z, s.e[0], a), plane_at<B>(pl, z, s.e[1], a),
                                              plane_at<B>(pl, z, s.e[2], a), plane_at<B>(pl, z, s.e[3], a)));
      }
    }
  }
}

// ---- z: half H of each column holds the pairs lo = H m/2 .. lo + m/2 - 1
// (m = B/2).  Every stencil reaches at most two pairs past the middle, so a
// half exports its two pairs next to the middle and reads the other half's.
template <int B, int H, typename T2>
__device__ __forceinline__ void halo_put(T2 *hx, int step, int r, int k, int a, const T2 &p0, const T2 &p1)
{
  halo_at<B>(hx, step, H, 0, r, k, a) = p0;
  halo_at<B>(hx, step, H, 1, r, k, a) = p1;
}

// local z-pair of the first exported pair
template <int B, int H>
constexpr int halo_first()
{
  return H == 0 ? B / 4 - 2 : 0;
}

// the value of pair j of the column: local pairs from loc(jl), the two pairs
// past the middle from the halo
template <int B, int H, typename T2, typename F>
__device__ __forceinline__ T2 zsrc(int j, const T2 (&hv)[2], F &&loc)
{
  constexpr int MH = B / 4, lo = H * MH;
  if (j >= lo && j < lo + MH) return loc(j - lo);
  const int s = H == 0 ? j - MH : j - (MH - 2);
  return hv[s < 0 ? 0 : (s > 1 ? 1 : s)];
}

template <typename T, int B, int KIND, int H, typename T2>
__device__ __forceinline__ void zf_a(T2 (&v)[2][B / 2], T2 *hx, int k, int a)
{
  constexpr int MH = B / 4, f = halo_first<B, H>();
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    if constexpr (KIND == W3AI) {
      // the odd slot takes the pair average
#pragma unroll
      for (int jl = 0; jl < MH; ++jl) v[r][2 * jl + 1] = mul2(add2(v[r][2 * jl], v[r][2 * jl + 1]), mk2((T)0.5));
      halo_put<B, H>(hx, 0, r, k, a, v[r][2 * f + 1], v[r][2 * f + 3]);
    } else {
      halo_put<B, H>(hx, 0, r, k, a, v[r][2 * f], v[r][2 * f + 2]);
    }
  }
}

template <typename T, int B, int KIND, int H, typename T2>
__device__ __forceinline__ void zf_b(T2 (&v)[2][B / 2], T2 *hx, int k, int a)
{
  constexpr int MH = B / 4, m = B / 2, lo = H * MH, f = halo_first<B, H>();
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const T2 hv[2] = {halo_at<B>(hx, 0, 1 - H, 0, r, k, a), halo_at<B>(hx, 0, 1 - H, 1, r, k, a)};
    T2 d[MH];
    if constexpr (KIND == W3AI) {
      auto src = [&](int j) { return zsrc<B, H>(j, hv, [&](int jl) { return v[r][2 * jl + 1]; }); };
#pragma unroll
      for (int jl = 0; jl < MH; ++jl) {
        const AiRow rw = ai_row(lo + jl, m);
        d[jl] = sub2(v[r][2 * jl], ai_predc<T2, T>(rw, v[r][2 * jl + 1], src(rw.s1), src(rw.s2)));
      }
#pragma unroll
      for (int jl = 0; jl < MH; ++jl) {
        v[r][2 * jl] = v[r][2 * jl + 1];
        v[r][2 * jl + 1] = d[jl];
      }
    } else {
      auto src = [&](int j) { return zsrc<B, H>(j, hv, [&](int jl) { return v[r][2 * jl]; }); };
#pragma unroll
      for (int jl = 0; jl < MH; ++jl) {
        const W4Row rw = w4_row(lo + jl, m);
        d[jl] = sub2(v[r][2 * jl + 1], pred4rp<T2, T>(rw, src(rw.j0), src(rw.j0 + 1), src(rw.j0 + 2), src(rw.j0 + 3)));
      }
#pragma unroll
      for (int jl = 0; jl < MH; ++jl) v[r][2 * jl + 1] = d[jl];
      if constexpr (KIND == W4LI) halo_put<B, H>(hx, 1, r, k, a, d[f], d[f + 1]);
    }
  }
}

// W4li: update of the even values from the new details
template <typename T, int B, int H, typename T2>
__device__ __forceinline__ void zf_c(T2 (&v)[2][B / 2], T2 *hx, int k, int a)
{
  constexpr int MH = B / 4, m = B / 2, lo = H * MH;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const T2 hv[2] = {halo_at<B>(hx, 1, 1 - H, 0, r, k, a), halo_at<B>(hx, 1, 1 - H, 1, r, k, a)};
    auto src = [&](int j) { return zsrc<B, H>(j, hv, [&](int jl) { return v[r][2 * jl + 1]; }); };
    T2 sn[MH];
#pragma unroll
    for (int jl = 0; jl < MH; ++jl) {
      const int j = lo + jl;
      const LiSrc ls = li_src(j, m);
      const T uw[3] = {li_lookup<T>(m, j, 0), li_lookup<T>(m, j, 1), li_lookup<T>(m, j, 2)};
      const int k1 = ls.k0 + 1 < m ? ls.k0 + 1 : m - 1, k2 = ls.k0 + 2 < m ? ls.k0 + 2 : m - 1;
      sn[jl] = add2(v[r][2 * jl], li_accp<T2>(uw, ls.nt, src(ls.k0), src(k1), src(k2)));
    }
#pragma unroll
    for (int jl = 0; jl < MH; ++jl) v[r][2 * jl] = sn[jl];
  }
}

template <typename T, int B, int KIND, typename T2>
__device__ __forceinline__ void z_fwd(T2 (&v)[2][B / 2], T2 *hx, int k, int a, int h)
{
  if (h == 0)
    zf_a<T, B, KIND, 0>(v, hx, k, a);
  else
    zf_a<T, B, KIND, 1>(v, hx, k, a);
  __syncthreads();
  if (h == 0)
    zf_b<T, B, KIND, 0>(v, hx, k, a);
  else
    zf_b<T, B, KIND, 1>(v, hx, k, a);
  if constexpr (KIND == W4LI) {
    __syncthreads();
    if (h == 0)
      zf_c<T, B, 0>(v, hx, k, a);
    else
      zf_c<T, B, 1>(v, hx, k, a);
  }
}

// inverse: W4li first removes the update (halo step 1: details), then every
// kind exports its predict inputs (step 0: coarse values) and predicts
template <typename T, int B, int H, typename T2>
__device__ __forceinline__ void zi_undo(T2 (&v)[2][B / 2], T2 *hx, int k, int a)
{
  constexpr int MH = B / 4, m = B / 2, lo = H * MH, f = halo_first<B, H>();
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const T2 hv[2] = {halo_at<B>(hx, 1, 1 - H, 0, r, k, a), halo_at<B>(hx, 1, 1 - H, 1, r, k, a)};
    auto src = [&](int j) { return zsrc<B, H>(j, hv, [&](int jl) { return v[r][2 * jl + 1]; }); };
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
    halo_put<B, H>(hx, 0, r, k, a, v[r][2 * f], v[r][2 * f + 2]);
  }
}

template <typename T, int B, int KIND, int H, typename T2>
__device__ __forceinline__ void zi_a(T2 (&v)[2][B / 2], T2 *hx, int k, int a)
{
  constexpr int f = halo_first<B, H>();
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    if constexpr (KIND == W4LI)
      halo_put<B, H>(hx, 1, r, k, a, v[r][2 * f + 1], v[r][2 * f + 3]);
    else
      halo_put<B, H>(hx, 0, r, k, a, v[r][2 * f], v[r][2 * f + 2]);
  }
}

template <typename T, int B, int KIND, int H, typename T2>
__device__ __forceinline__ void zi_b(T2 (&v)[2][B / 2], T2 *hx, int k, int a)
{
  constexpr int MH = B / 4, m = B / 2, lo = H * MH;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const T2 hv[2] = {halo_at<B>(hx, 0, 1 - H, 0, r, k, a), halo_at<B>(hx, 0, 1 - H, 1, r, k, a)};
    auto src = [&](int j) { return zsrc<B, H>(j, hv, [&](int jl) { return v[r][2 * jl]; }); };
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

template <typename T, int B, int KIND, typename T2>
__device__ __forceinline__ void z_inv(T2 (&v)[2][B / 2], T2 *hx, int k, int a, int h)
{
  if (h == 0)
    zi_a<T, B, KIND, 0>(v, hx, k, a);
  else
    zi_a<T, B, KIND, 1>(v, hx, k, a);
  __syncthreads();
  if constexpr (KIND == W4LI) {
    if (h == 0)
      zi_undo<T, B, 0>(v, hx, k, a);
    else
      zi_undo<T, B, 1>(v, hx, k, a);
    __syncthreads();
  }
  if (h == 0)
    zi_b<T, B, KIND, 0>(v, hx, k, a);
  else
    zi_b<T, B, KIND, 1>(v, hx, k, a);
}

// ============================================================ coarser levels
// After level 0 the coarse values (all coordinates even) form an N^3 cube,
// N = B/2, held in v[0][2 jl].x of every thread (to_cube).  Levels 1.. are
// the same transform on that cube, run in shared memory by up to NT threads:
// C(x, y, z) = C[(z N + y)(N + 1) + x] (rows padded by one element, so that
// lines along x, taken y-fastest across threads, hit distinct banks).
template <int N>
__device__ __forceinline__ int cidx(int x, int y, int z)
{
  return (z * N + y) * (N + 1) + x;
}

// line `li` of pass AXIS at level stride S: base index and step along it
// (consecutive lines start in distinct banks)
template <int N, int S, int AXIS>
__device__ __forceinline__ void cube_line(int li, int &base, int &step)
{
  constexpr int n = N / S;
  const int f = li % n, g = li / n;  // fast, slow line coordinates (units of S)
  if (AXIS == 0) {  // lines along x, y fastest
    base = cidx<N>(0, f * S, g * S);
    step = S;
  } else if (AXIS == 1) {  // along y, x fastest
    base = cidx<N>(f * S, 0, g * S);
    step = S * (N + 1);
  } else {  // along z, x fastest
    base = cidx<N>(f * S, g * S, 0);
    step = S * N * (N + 1);
  }
}

// one axis of one level: a thread per line, the line in registers
// (compile-time stencils), written back in place.  Along x and along y,
// thread li gets a line of z-slice li / n, so the two passes of a level
// touch each slice from one warp (n divides 32 or is a multiple of 16):
// between them a warp barrier orders the accesses (WARP_ONLY).
// barrier of the NTH threads that use barrier ID (a multiple of 32 threads,
// whole warps; ID 0 is __syncthreads')
template <int ID, int NTH>
__device__ __forceinline__ void named_sync()
{
  asm volatile("bar.sync %0, %1;" ::"n"(ID), "n"(NTH) : "memory");
}

// NB > 0: the passes' barriers span only threads 0..NB-1 (named barrier 1),
// so that other warps of the CTA can do other work meanwhile
template <typename T, int N, int KIND, int NT, int S, int AXIS, bool FWD, bool WARP_ONLY, int NB = 0>
__device__ __forceinline__ void cube_pass(T *C)
{
  constexpr int n = N / S, LINES = n * n;
  static_assert(LINES <= NT, "one line per thread");
  static_assert(!WARP_ONLY || AXIS < 2, "only x and y lines share slices by warp");
  static_assert(32 % n == 0 || n % 16 == 0, "a z-slice's lines lie in one warp");
  const int tid = threadIdx.x;
  if (tid < LINES) {
    int base, step;
    cube_line<N, S, AXIS>(tid, base, step);
    T e[n];
#pragma unroll
    for (int i = 0; i < n; ++i) e[i] = C[base + i * step];
    if constexpr (FWD)
      fwd_reg<T, KIND, n, 1>(e);
    else
      inv_reg<T, KIND, n, 1>(e);
#pragma unroll
    for (int i = 0; i < n; ++i)
      if (KIND != W4 || (i & 1)) C[base + i * step] = e[i];  // W4 changes only the odd points
  }
  if constexpr (WARP_ONLY)
    __syncwarp();
  else if constexpr (NB > 0)
    named_sync<1, NB>();
  else
    __syncthreads();
}

// all levels of the N^3 cube down to 4^3 (x, y, z per level)
template <typename T, int N, int KIND, int NT, int S = 1, int NB = 0>
__device__ __forceinline__ void cube_fwd(T *C)
{
  if constexpr (N / S >= 8) {
    cube_pass<T, N, KIND, NT, S, 0, true, true, NB>(C);
    cube_pass<T, N, KIND, NT, S, 1, true, false, NB>(C);
    cube_pass<T, N, KIND, NT, S, 2, true, false, NB>(C);
    cube_fwd<T, N, KIND, NT, 2 * S, NB>(C);
  }
}

template <typename T, int N, int KIND, int NT, int S = 1, int NB = 0>
__device__ __forceinline__ void cube_inv(T *C)
{
  if constexpr (N / S >= 8) {
    cube_inv<T, N, KIND, NT, 2 * S, NB>(C);
    cube_pass<T, N, KIND, NT, S, 2, false, false, NB>(C);
    cube_pass<T, N, KIND, NT, S, 1, false, true, NB>(C);
    cube_pass<T, N, KIND, NT, S, 0, false, false, NB>(C);
  }
}

// coarse values of level 0 <-> the cube: pair jl of row 0 of thread
// (a, k, h) holds the coarse value at cube position (a, k, h B/4 + jl)
template <typename T, int B, typename T2>
__device__ __forceinline__ void to_cube(const T2 (&v)[2][B / 2], T *C, int a, int k, int h)
{
  constexpr int N = B / 2, MH = B / 4;
#pragma unroll
  for (int jl = 0; jl < MH; ++jl) C[cidx<N>(a, k, h * MH + jl)] = v[0][2 * jl].x;
}

template <typename T, int B, typename T2>
__device__ __forceinline__ void from_cube(T2 (&v)[2][B / 2], const T *C, int a, int k, int h)
{
  constexpr int N = B / 2, MH = B / 4;
#pragma unroll
  for (int jl = 0; jl < MH; ++jl) v[0][2 * jl].x = C[cidx<N>(a, k, h * MH + jl)];
}

// ---- the finest x-level row by row in a swizzled tile of 128-byte rows
// (FP32 32^3 blocks): thread t takes rows t, t + NT, ... (consecutive lanes
// take consecutive rows, so the eight 16-byte chunks of a quarter warp fall
// in distinct bank groups), holds a row in registers and transforms it with
// compile-time stencils (fwd_reg / inv_reg: the same rounded operations in
// the same order as the pair kernels' x-step), and writes it back in place.
// With MM, lo / hi also take the min / max of the rows' values as read
// (NaN never enters).
template <typename T, int B, int KIND, bool FWD, int NT, bool MM = false>
__device__ __forceinline__ void x_rows(unsigned char *tile, T &lo, T &hi)
{
  static_assert(sizeof(T) == 4 && B == 32 && (B * B) % (2 * NT) == 0, "128-byte FP32 rows, two per round");
#pragma unroll 1
  for (int r0 = threadIdx.x; r0 < B * B; r0 += 2 * NT) {
    T e[2][B];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int row = r0 + q * NT;
      const unsigned char *rp = tile + row * 128;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const float4 w = *reinterpret_cast<const float4 *>(rp + ((c ^ (row & 7)) << 4));
        e[q][4 * c] = w.x;
        e[q][4 * c + 1] = w.y;
        e[q][4 * c + 2] = w.z;
        e[q][4 * c + 3] = w.w;
        if constexpr (MM) {
          lo = min3_nn(min3_nn(lo, w.x, w.y), w.z, w.w);
          hi = max3_nn(max3_nn(hi, w.x, w.y), w.z, w.w);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if constexpr (FWD)
        fwd_reg<T, KIND, B, 1>(e[q]);
      else
        inv_reg<T, KIND, B, 1>(e[q]);
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int row = r0 + q * NT;
      unsigned char *rp = tile + row * 128;
#pragma unroll
      for (int c = 0; c < 8; ++c)
        *reinterpret_cast<float4 *>(rp + ((c ^ (row & 7)) << 4)) =
            make_float4(e[q][4 * c], e[q][4 * c + 1], e[q][4 * c + 2], e[q][4 * c + 3]);
    }
  }
}

template <typename T, int B, int KIND, bool FWD, int NT>
__device__ __forceinline__ void x_rows(unsigned char *tile)
{
  T lo = T(0), hi = T(0);
  x_rows<T, B, KIND, FWD, NT, false>(tile, lo, hi);
}

// Whole forward transform.  The plane area and the cube may overlap (the
// cube is written after the plane's last read); the halo is separate.
// first_sync runs right after the first barrier (every thread has read its
// input by then).  Ends without a barrier: from_cube's reads of the cube
// are ordered by the caller's next barrier.
// side() runs after the barrier that follows the level-0 steps (at the end
// without coarser levels), while the coarser levels' first pass keeps
// half of the threads or fewer busy.
template <typename T, int B, int KIND, bool XSTEP = true, typename T2, typename F, typename F2>
__device__ __forceinline__ void fwd_all(T2 (&v)[2][B / 2], T2 *pl, T2 *hx, T *cube, int a, int k, int h, int seg,
                                        F &&first_sync, F2 &&side)
{
  if constexpr (XSTEP) x_fwd<T, B, KIND>(v, a, seg);
  y_fwd<T, B, KIND>(v, pl, a, k, h, first_sync);
  z_fwd<T, B, KIND>(v, hx, k, a, h);
  if constexpr (G2<T, B>::L > 1) {
    to_cube<T, B>(v, cube, a, k, h);
    __syncthreads();
    side();
    cube_fwd<T, B / 2, KIND, G2<T, B>::NT>(cube);
    from_cube<T, B>(v, cube, a, k, h);
  } else {
    side();
  }
}

template <typename T, int B, int KIND, bool XSTEP = true, typename T2, typename F>
__device__ __forceinline__ void fwd_all(T2 (&v)[2][B / 2], T2 *pl, T2 *hx, T *cube, int a, int k, int h, int seg,
                                        F &&first_sync)
{
  fwd_all<T, B, KIND, XSTEP>(v, pl, hx, cube, a, k, h, seg, first_sync, [] {});
}

// Whole inverse transform.  The cube must not overlap the plane or the
// halo; the caller orders the plane's and the halo's previous uses by a
// barrier before the call, and their last reads by one after it.  side()
// runs after the first barrier (at the start without coarser levels).
template <typename T, int B, int KIND, bool XSTEP = true, typename T2, typename F>
__device__ __forceinline__ void inv_all(T2 (&v)[2][B / 2], T2 *pl, T2 *hx, T *cube, int a, int k, int h, int seg,
                                        F &&side)
{
  if constexpr (G2<T, B>::L > 1) {
    to_cube<T, B>(v, cube, a, k, h);
    __syncthreads();
    side();
    cube_inv<T, B / 2, KIND, G2<T, B>::NT>(cube);
    from_cube<T, B>(v, cube, a, k, h);
  } else {
    side();
  }
  z_inv<T, B, KIND>(v, hx, k, a, h);
  y_inv<T, B, KIND>(v, pl, a, k, h);
  if constexpr (XSTEP) x_inv<T, B, KIND>(v, a, seg);
}

// ============================================================ stream helpers
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

// B-bit row word number m of a mask (bit offset m*B)
template <int B>
__device__ __forceinline__ void put_rowi(unsigned char *mask, int m, unsigned w)
{
  if constexpr (B == 32)
    reinterpret_cast<unsigned *>(mask)[m] = w;
  else if constexpr (B == 16)
    reinterpret_cast<unsigned short *>(mask)[m] = (unsigned short)w;
  else
    mask[m] = (unsigned char)w;
}

template <int B>
__device__ __forceinline__ unsigned get_rowi(const unsigned char *mask, int m)
{
  if constexpr (B == 32)
    return reinterpret_cast<const unsigned *>(mask)[m];
  else if constexpr (B == 16)
    return reinterpret_cast<const unsigned short *>(mask)[m];
  else
    return mask[m];
}

// row (z, y) of a stream mask (row z*B + y)
template <int B>
__device__ __forceinline__ void put_row(unsigned char *mask, int z, int y, unsigned w)
{
  put_rowi<B>(mask, z * B + y, w);
}

template <int B>
__device__ __forceinline__ unsigned get_row(const unsigned char *mask, int z, int y)
{
  return get_rowi<B>(mask, z * B + y);
}

// rows (z, y) and (z, y + 1), y even, in one load (they are adjacent)
template <int B>
__device__ __forceinline__ void get_row_pair(const unsigned char *mask, int z, int y, unsigned &r0, unsigned &r1)
{
  const int m = z * B + y;
  if constexpr (B == 32) {
    const uint2 w = reinterpret_cast<const uint2 *>(mask)[m >> 1];
    r0 = w.x;
    r1 = w.y;
  } else if constexpr (B == 16) {
    const unsigned w = reinterpret_cast<const unsigned *>(mask)[m >> 1];
    r0 = w & 0xFFFFu;
    r1 = w >> 16;
  } else {
    const unsigned w = reinterpret_cast<const unsigned short *>(mask)[m >> 1];
    r0 = w & 0xFFu;
    r1 = w >> 8;
  }
}

// index of row (z, y) in the padded shared-memory tables (B + 1 rows per z)
template <int B>
__device__ __forceinline__ int rpad(int z, int y)
{
  return z * (B + 1) + y;
}

// row offset table entry of scan position p (rows in stream order)
template <int B>
__device__ __forceinline__ int rpad_of(int p)
{
  return rpad<B>(p / B, p % B);
}

template <typename T>
__device__ __forceinline__ void threshold_keys(double eps, int eps_mode, double cnorm, double range_in,
                                               const unsigned long long *keys, double &mn, double &mx,
                                               double &range, T &t)
{
  if (range_in >= 0) {
    range = range_in;
    mn = mx = __longlong_as_double(0x7FF8000000000000LL);
  } else {
    const unsigned long long kmin = *(volatile const unsigned long long *)&keys[0];
    const unsigned long long kmax = *(volatile const unsigned long long *)&keys[1];
    mn = key_value(kmin, T(0));
    mx = key_value(kmax, T(0));
    mn = (double)(T)((T)mn + (T)0);  // -0 reported as +0
    mx = (double)(T)((T)mx + (T)0);
    range = (mn <= mx) ? mx - mn : 0.0;
  }
  // cnorm = 1 (paper bound) or the synthesis norm C (strict bound)
  const double td = (eps_mode == 1 ? eps : eps * range) / cnorm;
  t = (T)td;
}

template <typename T>
__device__ __forceinline__ void threshold_of(double eps, int eps_mode, double cnorm, double range_in,
                                             const WsHdr *ws, double &mn, double &mx, double &range, T &t)
{
  threshold_keys<T>(eps, eps_mode, cnorm, range_in, &ws->minkey, mn, mx, range, t);
}

// the threshold of the range between two order keys, formed exactly as
// threshold_keys does with the paper bound (divisor 1); monotonic in the
// range, so the keys of any subset of the field give a threshold no larger
// than the whole field's
template <typename T>
__device__ __forceinline__ T threshold_between(double eps, int eps_mode, unsigned long long kmin,
                                               unsigned long long kmax)
{
  double mn = key_value(kmin, T(0)), mx = key_value(kmax, T(0));
  mn = (double)(T)((T)mn + (T)0);
  mx = (double)(T)((T)mx + (T)0);
  const double range = (mn <= mx) ? mx - mn : 0.0;
  return (T)(eps_mode == 1 ? eps : eps * range);
}

// speculative thresholds: a bound a little above t_lo (by 2^-10 of it).
// Where the exact threshold t is at most this bound, only the blocks that
// kept a value below it can hold one below t.
template <typename T>
__device__ __forceinline__ T near_threshold(T tlo)
{
  return tlo * (T)(1.0 + 1.0 / 1024.0);
}

// bits of a threshold, for comparing two of them exactly
__device__ __forceinline__ unsigned long long t_bits(float t) { return __float_as_uint(t); }
__device__ __forceinline__ unsigned long long t_bits(double t) { return (unsigned long long)__double_as_longlong(t); }

// ============================================================ decompress
// ---- stage-2 inverse of one chunk's tokens, by all NT threads of the CTA:
// block scans of (literal words, output words) per round of NT tokens place
// every token; a warp per token copies its literals and writes its zero run
// into the W words of the shuffled payload at SH32.  TL, TO, TK are NT
// words each of shared memory, s_u64 NT / 32 words.  Returns false (in
// some thread) when a token would read past the nlit_avail literal words or
// write past the payload, or the tokens do not fill it exactly; such
// tokens write nothing.
template <int NT>
__device__ __forceinline__ bool untoken(const unsigned *tok, unsigned ntok, const unsigned *lit,
                                        unsigned long long nlit_avail, unsigned *SH32, unsigned W, unsigned *TL,
                                        unsigned *TO, unsigned *TK, unsigned long long *s_u64)
{
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  unsigned lit_carry = 0, out_carry = 0;
  bool bad = false;
  for (unsigned r0 = 0; r0 < ntok; r0 += NT) {
    const unsigned k = r0 + tid;
    const unsigned tk = k < ntok ? __ldg(tok + k) : 0u;
    const unsigned nl = tk & 0xFFFFu, run = nl + (tk >> 16);
    // both prefixes in one scan (one barrier): literal words in the low
    // half, output words in the high half (each sum stays below 2^32)
    unsigned long long tot2;
    const unsigned long long ex2 =
        block_exsum_nb<NT>((unsigned long long)nl | ((unsigned long long)run << 32), s_u64, tot2);
    const unsigned lp = (unsigned)ex2, op = (unsigned)(ex2 >> 32);
    const unsigned tl = (unsigned)tot2, to_ = (unsigned)(tot2 >> 32);
    TL[tid] = lit_carry + lp;
    TO[tid] = out_carry + op;
    TK[tid] = tk;
    __syncthreads();
    const unsigned cnt = (ntok - r0) < (unsigned)NT ? (ntok - r0) : (unsigned)NT;
    for (unsigned i = wid; i < cnt; i += NT / 32) {
      const unsigned t = TK[i], l0 = TL[i], o0 = TO[i], n = t & 0xFFFFu, z = t >> 16;
      if ((unsigned long long)l0 + n > nlit_avail || (unsigned long long)o0 + n + z > (unsigned long long)W) {
        bad = true;
        continue;
      }
      for (unsigned q = lane; q < n; q += 32) SH32[o0 + q] = __ldg(lit + l0 + q);
      for (unsigned q = lane; q < z; q += 32) SH32[o0 + n + q] = 0u;
    }
    lit_carry += tl;
    out_carry += to_;
    __syncthreads();
  }
  return !(bad || out_carry != W || (unsigned long long)lit_carry > nlit_avail);
}

// ---- stage-2 inverse, one chunk at a time: block scans of (literal
// words, output words) per token place every token; a warp per token copies
// its literals and writes its zero run into the shuffled payload in shared
// memory, which is then unshuffled into the block's staging slot.  Small CTAs take the payloads of up
// to G2::SHCAP bytes (and the malformed chunks), a second launch with large
// CTAs the rest.
template <typename T, int B, bool BIG>
__global__ void __launch_bounds__(BIG ? 512 : 128) k_unstage(const UnArgs a)
{
  using G = G2<T, B>;
  constexpr int NT = BIG ? 512 : 128, ES = G::ES;
  // FP64 32^3: the large launch's shuffled payload lives in a global
  // scratch block per CTA (it does not fit in shared memory)
  constexpr bool GP = BIG && G::SLAB;
  constexpr int CAPB = BIG ? (GP ? 0 : G::PMAX_AL) : G::SHCAP;
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char *P = GP ? a.scratch + (size_t)blockIdx.x * G::SCRATCH : smem;
  unsigned *TL = reinterpret_cast<unsigned *>(smem + CAPB);  // per token of a round: first literal,
  unsigned *TO = TL + NT;                                      // first output word,
  unsigned *TK = TO + NT;                                      // the token
  __shared__ unsigned long long s_u64[NT / 32];
  __shared__ unsigned s_nnz, s_ntok, s_bad;
  __shared__ unsigned long long s_off, s_len;
  const int tid = threadIdx.x;

  WsHdr *wsh = reinterpret_cast<WsHdr *>(a.ws);
  // the small launch visits every chunk and lists the large ones, which the
  // large launch then visits alone
  const int count = BIG ? (int)*(volatile const unsigned *)&wsh->nbig : a.nblocks;
  for (int it = blockIdx.x; it < count; it += gridDim.x) {
    const int bid = BIG ? a.biglist[it] : it;  // the decoded block (its staging slot and table entry)
    if (tid == 0) {
      unsigned bad = 0;
      const unsigned long long *tab = reinterpret_cast<const unsigned long long *>(a.in + HEADER_BYTES);
      int c = a.ids ? a.ids[bid] : bid;  // its chunk in the stream
      if (c < 0 || c >= a.nchunks) {
        atomicCAS(&wsh->status, 0u, ST_ARG);
        c = 0;
        bad = 1;
      }
      const unsigned long long o0 = tab[c], o1 = tab[c + 1];
      const unsigned long long avail = a.in_bytes - a.data0;
      unsigned nnz = 0, ntok = 0;
      if (bad || o0 > o1 || o1 > avail || o1 - o0 < 8 || (o0 & 3) || ((o1 - o0) & 3)) {
        bad = 1;
      } else {
        const unsigned *c32 = reinterpret_cast<const unsigned *>(a.in + a.data0 + o0);
        nnz = c32[0];
        ntok = c32[1];
        if (nnz > (unsigned)(G::NVOX - 64)) bad = 1;
        if (!bad && (unsigned long long)ntok > (o1 - o0 - 8) / 4) bad = 1;
      }
      s_bad = bad;
      s_nnz = bad ? 0u : nnz;
      s_ntok = ntok;
      s_off = o0;
      s_len = o1 - o0;
    }
    __syncthreads();
    const unsigned nnz = s_nnz;
    const int pbytes = 64 * ES + G::MASKB + (int)nnz * ES;
    if (!BIG && !s_bad && pbytes > G::SHCAP) {  // the large launch's chunk
      if (tid == 0) a.biglist[atomicAdd(&wsh->nbig, 1u)] = bid;
      __syncthreads();
      continue;
    }
    if (!s_bad) {
      const int W = pbytes / 4, E = pbytes >> G::LGES;
      const unsigned ntok = s_ntok;
      const unsigned long long nlit_avail = (s_len - 8 - 4ull * ntok) / 4;
      const unsigned *c32 = reinterpret_cast<const unsigned *>(a.in + a.data0 + s_off);
      const unsigned *tok = c32 + 2;
      const unsigned *lit = tok + ntok;
      if (!untoken<NT>(tok, ntok, lit, nlit_avail, reinterpret_cast<unsigned *>(P), (unsigned)W, TL, TO, TK, s_u64))
        atomicOr(&s_bad, 1u);
      __syncthreads();
      if (!s_bad) {
        // unshuffle straight into the slot: byte q of raw word k is byte
        // (4k + q) % ES of element (4k + q) / ES, found at plane offset
        unsigned *dst = reinterpret_cast<unsigned *>(a.staging + (size_t)bid * a.slot);
        for (int k = tid; k < W; k += NT) {
          const int e = (4 * k) >> G::LGES, b0 = (4 * k) & (ES - 1);
          unsigned wv = 0;
#pragma unroll
          for (int q = 0; q < 4; ++q) wv |= (unsigned)P[(b0 + q) * E + e] << (8 * q);
          dst[k] = wv;
        }
      }
    }
    if (tid == 0) {
      a.table[2 * bid] = s_bad ? 0ull : (unsigned long long)nnz;
      a.table[2 * bid + 1] = s_bad ? 1ull : 0ull;
    }
    __syncthreads();
  }
}

template <typename T, int B, int KIND>
__global__ void __launch_bounds__(B * B / 2, 1) k_decompress2(const __grid_constant__ CUtensorMap omap,
                                                              const InvArgs a)
{
  using G = G2<T, B>;
  using T2 = typename V2T<T>::type;
  constexpr int NT = G::NT, ES = G::ES, Q = G::Q;
  constexpr int HEAD = 64 * ES + G::MASKB;  // coarse values + mask
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char *smem = align1024(smem_raw);
  constexpr int ZH = G::ZH;
  unsigned char *OT = smem;  // output tile [z][y][x] (swizzled 128-byte rows for FP32 32^3 W4li)
  constexpr bool RX = G::template rowx<KIND>();  // the finest x-level row by row in the tile
  T *CB = reinterpret_cast<T *>(smem + G::OTB);                                 // cube of the coarser levels
  unsigned *ROWOFF = reinterpret_cast<unsigned *>(smem + G::OTB + G::CUBE_AL);  // row offsets
  constexpr int NPB = G::NPB;
  unsigned char *BUF0 = smem + G::OTB + G::R2D;  // NPB payload buffers of G::PBCAP bytes
  T2 *PL = reinterpret_cast<T2 *>(OT);  // level-0 plane and halo, inside the tile area
  T2 *HX = reinterpret_cast<T2 *>(OT + G::PLANE);
  __shared__ __align__(8) unsigned long long s_bar[NPB];
  __shared__ unsigned s_u[40];
  __shared__ unsigned s_nnz[NPB], s_bad[NPB];
  __shared__ unsigned s_badx;
  // s_pend[j]: a payload copy into buffer j was started and not yet seen
  // complete; s_to: some thread's wait for a copy gave up (read by all
  // threads only after a barrier, so the CTA decides as one)
  __shared__ unsigned s_pend[NPB], s_to;

  WsHdr *ws = reinterpret_cast<WsHdr *>(a.ws);
  const int tid = threadIdx.x, lane = tid & 31;
  int ap, k, h;
  quad_of<B>(tid, ap, k, h);
  const int seg = lane - ap;
  const int x0 = 2 * ap;
  const int zr = h * ZH + ap;  // z of this thread's two mask rows
  const bool cE = (x0 % Q == 0) && ((2 * k) % Q == 0);  // column (x0, 2k) holds coarse values
  const bool pre = a.stage2 != 0;  // decoded payloads sit in 16-byte aligned slots
  constexpr int FT = NT - 32;      // lane 0 of the last warp: fetches the next block

  // metadata of block b into buffer slot j, and (with stage 2) the start
  // of its payload copy; called by thread 0 with b's table entry (t0, t1)
  // loaded ahead
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
      const int cp = pbytes <= G::PBCAP ? pbytes : HEAD;
      s_pend[j] = 1u;
      bulk_load(BUF0 + j * G::PBCAP, a.staging + (size_t)b * a.slot, (unsigned)((cp + 15) & ~15), &s_bar[j]);
    }
    return o0;
  };

  __shared__ BlockWalk s_wk;  // coordinates of this CTA's current block
  __shared__ __align__(16) unsigned long long s_tab[2];  // a later block's table entry
  __shared__ unsigned long long s_off[NPB];  // without stage 2: each buffer's chunk offset
  if (tid == 0) {
    for (int q = 0; q < NPB; ++q) {
      mbar_init(&s_bar[q]);
      s_pend[q] = 0;
    }
    s_to = 0;
    s_badx = 0;  // reset again after each block's last read
    s_wk.init(blockIdx.x, gridDim.x, a.nbx, a.nby);
  }
  __syncthreads();
  if (tid == 0) {
    // the first NPB - 1 blocks' copies
    for (int q = 0; q < NPB - 1; ++q) {
      const int b = blockIdx.x + q * gridDim.x;
      if (b < a.nblocks) s_off[q] = fetch(b, q, pre ? a.table[2 * b] : 0ull, pre ? a.table[2 * b + 1] : 0ull);
    }
  }
  __syncthreads();
  unsigned phase = 0;  // bit j: parity of buffer j's next completion (a register, not an indexed array)
  int j = 0;

  for (int bid = blockIdx.x; bid < a.nblocks; bid += gridDim.x, j = j + 1 < NPB ? j + 1 : 0) {
    unsigned char *P = BUF0 + j * G::PBCAP;
    // the table entry of the block NPB - 1 ahead, fetched now
    // (asynchronously, into shared memory) by the thread that later starts
    // its payload copy into the buffer this block frees
    const int nbid = bid + (NPB - 1) * (int)gridDim.x;
    const int jn = j == 0 ? NPB - 1 : j - 1;  // (j + NPB - 1) mod NPB
    if (tid == FT && pre && nbid < a.nblocks) cp_async16(s_tab, a.table + 2 * nbid);
    const unsigned nnz = s_nnz[j];
    const int pbytes = HEAD + (int)nnz * ES;
    bool bad0 = s_bad[j] != 0;
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
      const int cp = pbytes <= G::PBCAP ? pbytes : HEAD;
      for (int w = tid; w < cp / 4; w += NT) reinterpret_cast<unsigned *>(P)[w] = __ldg(c32 + 2 + w);
      __syncthreads();
    }
    // values beyond the buffer are read from global memory
    const T *VALS = pbytes <= G::PBCAP
                        ? reinterpret_cast<const T *>(P + HEAD)
                        : (pre ? reinterpret_cast<const T *>(a.staging + (size_t)bid * a.slot + HEAD)
                               : reinterpret_cast<const T *>(a.in + a.data0 + s_off[j] + 8 + HEAD));
    const unsigned char *MASK = P + 64 * ES;
    // this thread's mask rows (z = zr at rows 2k, 2k + 1) and, transposed
    // over the segment's lanes, its own column bits (bit 2 zl + p: column
    // x0 + p at z = h B/2 + zl)
    unsigned R0 = 0, R1 = 0;
    if (!bad0) get_row_pair<B>(MASK, zr, 2 * k, R0, R1);
    const unsigned W[2] = {seg_transpose<B>(R0, ap), seg_transpose<B>(R1, ap)};
    if (!bad0) {
      // row populations (rows in stream order, IPT per thread, straight
      // from the mask) -> row offsets; coarse positions carry no mask bit
      constexpr int IPT = B * B / NT;
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
      // stops here.  Before leaving, wait once more, bounded, for every
      // copy it started that has not been seen complete (this block's and
      // the one issued ahead), and for its tile stores.
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

    T2 v[2][ZH];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int zl = 0; zl < ZH; ++zl) {
        v[r][zl].x = T(0);
        v[r][zl].y = T(0);
      }
    if (!bad) {
      // kept values of this thread's columns (z unrolled: v stays in
      // registers; threads whose columns keep nothing skip the rows)
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
    // the next block's metadata and payload copy, issued by a thread of the
    // last warp (idle in the first passes of the coarser levels), after a
    // barrier that follows every thread's read of s_badx; thread 0 waits
    // until the previous block's tile store has read the tile area, which
    // the level-0 exchange uses next (other threads write it only after a
    // later barrier)
    auto fetch_next = [&] {
      if (tid == 0) {
        s_badx = 0;
        bulk_wait_read();
      }
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
    if (!bad && G::L > 1) {
      // fetch_next runs after the cube's first barrier; the cube passes'
      // barriers follow it
      inv_all<T, B, KIND, !RX>(v, PL, HX, CB, ap, k, h, seg, fetch_next);
    } else {
      if (tid == 0) bulk_wait_read();
      __syncthreads();
      fetch_next();
      if (!bad) inv_all<T, B, KIND, !RX>(v, PL, HX, CB, ap, k, h, seg, [] {});
    }
    // block -> output tile -> TMA store, which drains while the next block
    // is decoded.  W4li (swizzled 128-byte rows): the pairs go to their
    // swizzled places, then the finest x-level runs row by row in the tile
    // (a bad block's zeros stay zeros).
    __syncthreads();  // the plane and the halo have been read
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int zl = 0; zl < ZH; ++zl) {
        const unsigned o = (unsigned)((((h * ZH + zl) * B + 2 * k + r) * B + x0) * ES);
        *reinterpret_cast<T2 *>(OT + (RX ? swz128(o) : o)) = v[r][zl];
      }
    if constexpr (RX) {
      __syncthreads();
      if (!bad) x_rows<T, B, KIND, false, NT>(OT);
    }
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tma_store_tile(&omap, OT, s_wk.bx * B, s_wk.by * B, s_wk.bz * B);
      s_wk.next();
    }
  }
  if (tid == 0) bulk_wait_all();
}

// ============================================================ dense transforms
template <typename T, int B, int KIND, bool FWD>
__global__ void __launch_bounds__(B * B / 2) k_dense2(const DenseArgs a)
{
  using G = G2<T, B>;
  using T2 = typename V2T<T>::type;
  constexpr int ZH = G::ZH;
  extern __shared__ __align__(128) unsigned char smem[];
  T *CB = reinterpret_cast<T *>(smem);
  T2 *PL = reinterpret_cast<T2 *>(smem + G::CUBE_AL);
  T2 *HX = reinterpret_cast<T2 *>(smem + G::CUBE_AL + G::PLANE);
  const int tid = threadIdx.x, lane = tid & 31;
  int ap, k, h;
  quad_of<B>(tid, ap, k, h);
  const int seg = lane - ap;
  const int bid = blockIdx.x;
  const int bx = bid % a.nbx, by = (bid / a.nbx) % a.nby, bz = bid / (a.nbx * a.nby);
  const size_t zs = (size_t)a.ny * a.nx;
  const size_t base = (size_t)(bz * B + h * ZH) * zs + (size_t)(by * B + 2 * k) * a.nx + (size_t)(bx * B + 2 * ap);
  const T *src = reinterpret_cast<const T *>(a.src) + base;
  T *dst = reinterpret_cast<T *>(a.dst) + base;
  T2 v[2][ZH];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int zl = 0; zl < ZH; ++zl) v[r][zl] = *reinterpret_cast<const T2 *>(src + zl * zs + r * a.nx);
  if constexpr (FWD)
    fwd_all<T, B, KIND>(v, PL, HX, CB, ap, k, h, seg, [] {});
  else
    inv_all<T, B, KIND>(v, PL, HX, CB, ap, k, h, seg, [] {});
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int zl = 0; zl < ZH; ++zl) *reinterpret_cast<T2 *>(dst + zl * zs + r * a.nx) = v[r][zl];
}

// ============================================================ a0: min / max
// min / max of xs[i], xs[i + stride], ... (< n), NaN never enters (every
// comparison with NaN is false); lanes then combine and commit with atomics
template <typename T>
__device__ __forceinline__ void minmax_part(const T *__restrict__ xs, size_t n, size_t i, size_t stride,
                                            unsigned long long *kmin, unsigned long long *kmax)
{
  T lo = (T)INFINITY, hi = (T)-INFINITY;
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
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const T l2 = __shfl_xor_sync(FULL, lo, o), h2 = __shfl_xor_sync(FULL, hi, o);
    lo = l2 < lo ? l2 : lo;
    hi = h2 > hi ? h2 : hi;
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(kmin, order_key(lo));
    atomicMax(kmax, order_key(hi));
  }
}

template <typename T>
__global__ void __launch_bounds__(512) k_minmax(const T *__restrict__ xs, size_t n, WsHdr *ws)
{
  minmax_part<T>(xs, n, (size_t)blockIdx.x * blockDim.x + threadIdx.x, (size_t)gridDim.x * blockDim.x,
                 &ws->minkey, &ws->maxkey);
}

// batched: field blockIdx.y, chunk blockIdx.x of MM_CHUNK elements (an
// even count, so vector loads stay aligned); keys[2f], keys[2f+1]
constexpr size_t MM_CHUNK = 1u << 20;
struct MinmaxArgs {
  const void *field[MAXF];
  unsigned long long n[MAXF];
  unsigned long long *keys;
};

template <typename T>
__global__ void __launch_bounds__(512) k_minmax_multi(const __grid_constant__ MinmaxArgs a)
{
  const int f = blockIdx.y;
  const size_t b0 = (size_t)blockIdx.x * MM_CHUNK;
  if (b0 >= a.n[f]) return;
  const size_t len = a.n[f] - b0 < MM_CHUNK ? a.n[f] - b0 : MM_CHUNK;
  minmax_part<T>(reinterpret_cast<const T *>(a.field[f]) + b0, len, threadIdx.x, blockDim.x, &a.keys[2 * f],
                 &a.keys[2 * f + 1]);
}

// min / max of the subsample of speculative thresholds: every 4th row (y)
// of every 4th z-plane, whole rows (16-byte vectors; a row is a multiple of
// 8 elements), one warp per row; the keys go to the header's skmin / skmax
template <typename T>
__global__ void __launch_bounds__(512) k_minmax_sample(const T *__restrict__ xs, int nx, int ny, int nz, WsHdr *ws)
{
  constexpr int V = sizeof(T) == 4 ? 4 : 2;  // elements per 16-byte vector
  using VT = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  const int lane = threadIdx.x & 31;
  const long long rows_y = (ny + 3) / 4, rows = rows_y * ((nz + 3) / 4);
  const long long w0 = (long long)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const long long ws_ = (long long)gridDim.x * (blockDim.x / 32);
  T lo = (T)INFINITY, hi = (T)-INFINITY;
  const int nv = nx / V;
  for (long long r = w0; r < rows; r += ws_) {
    const long long z = 4 * (r / rows_y), y = 4 * (r % rows_y);
    const VT *row = reinterpret_cast<const VT *>(xs + (z * ny + y) * (long long)nx);
    for (int q = lane; q < nv; q += 32) {
      const VT v = __ldcs(row + q);
      if constexpr (V == 4) {
        lo = v.x < lo ? v.x : lo; hi = v.x > hi ? v.x : hi;
        lo = v.y < lo ? v.y : lo; hi = v.y > hi ? v.y : hi;
        lo = v.z < lo ? v.z : lo; hi = v.z > hi ? v.z : hi;
        lo = v.w < lo ? v.w : lo; hi = v.w > hi ? v.w : hi;
      } else {
        lo = v.x < lo ? v.x : lo; hi = v.x > hi ? v.x : hi;
        lo = v.y < lo ? v.y : lo; hi = v.y > hi ? v.y : hi;
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const T l2 = __shfl_xor_sync(FULL, lo, o), h2 = __shfl_xor_sync(FULL, hi, o);
    lo = l2 < lo ? l2 : lo;
    hi = h2 > hi ? h2 : hi;
  }
  if (lane == 0) {
    atomicMin(&ws->skmin, order_key(lo));
    atomicMax(&ws->skmax, order_key(hi));
  }
}

}  // namespace czp
