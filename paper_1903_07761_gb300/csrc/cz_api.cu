// cz_api.cu -- host side of the C ABI declared in include/cz.h.
//
// Validates parameters, lays out the workspace, builds the TMA tensor map of
// the field, enqueues the min/max pass (a0) and the per-block codec kernels
// on the caller's stream, and parses stream headers.  No device memory is
// allocated here.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <cctype>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/cz.h"
#include "cz_compress.cuh"
#include "cz_launch.h"
#include "cz_pair.cuh"

using namespace czp;

namespace {

// an NVTX range around one host entry point (a no-op unless a profiler
// attaches an NVTX tool), so that profiles can be cut by call
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

struct Shape {
  int nbx, nby, nbz, nblocks, L, es;
  int G, nchunks;  // blocks per chunk (1, or 4 / 8 / 16 with aggregate chunks) and chunks
  unsigned long long data0;
};

constexpr int GROUP_FLAGS = CZ_FLAG_GROUP16;  // the two-bit group field

// blocks per chunk of a flags word: 1, 4, 8 or 16
int group_of(int flags)
{
  const int code = (flags & GROUP_FLAGS) >> 3;
  return code ? 2 << code : 1;
}

// bytes of the largest stage-1 payload of one block
size_t pmax_bytes(int block, int es)
{
  const size_t v = (size_t)block * block * block;
  return 64 * (size_t)es + v / 8 + (v - 64) * (size_t)es;
}

int check(const cz_params *p, Shape *sh)
{
  if (!p) return CZ_ERR_ARG;
  const int B = p->block;
  if (B != 8 && B != 16 && B != 32 && B != 64) return CZ_ERR_ARG;
  if (p->dtype != CZ_F32 && p->dtype != CZ_F64) return CZ_ERR_ARG;
  if (B == 64 && p->dtype != CZ_F32) return CZ_ERR_ARG;  // 64^3 blocks: FP32 only
  if (p->kind < CZ_W4 || p->kind > CZ_W3AI) return CZ_ERR_ARG;
  if (p->eps_mode != CZ_EPS_REL && p->eps_mode != CZ_EPS_ABS) return CZ_ERR_ARG;
  if (p->stage2 != 0 && p->stage2 != 1) return CZ_ERR_ARG;
  if (p->bound_mode != CZ_BOUND_PAPER && p->bound_mode != CZ_BOUND_STRICT) return CZ_ERR_ARG;
  if (p->flags & ~(CZ_FLAG_FAST | CZ_FLAG_ZERO4 | CZ_FLAG_ZERO8 | GROUP_FLAGS)) return CZ_ERR_ARG;
  // the fast build keeps the PSNR of the exact build within 0.01 dB only for
  // W3ai; W4 and W4li (extrapolating rows with weights up to 35/16) are
  // refused with it
  if ((p->flags & CZ_FLAG_FAST) && p->kind != CZ_W3AI) return CZ_ERR_ARG;
  const int zf = p->flags & (CZ_FLAG_ZERO4 | CZ_FLAG_ZERO8);
  if (zf == (CZ_FLAG_ZERO4 | CZ_FLAG_ZERO8)) return CZ_ERR_ARG;  // one zeroing width at most
  if (zf && p->bound_mode == CZ_BOUND_STRICT) return CZ_ERR_ARG;  // the strict bound excludes zeroing
  // aggregate chunks group the input of stage 2, and a group's payload
  // must fit the large group coder's buffer
  const int G = group_of(p->flags);
  if (G > 1 && (!p->stage2 || (size_t)G * pmax_bytes(B, p->dtype == CZ_F64 ? 8 : 4) > CZ_GROUP_MAX_BYTES))
    return CZ_ERR_ARG;
  if (!(p->eps >= 0) || std::isinf(p->eps)) return CZ_ERR_ARG;
  if (std::isnan(p->range)) return CZ_ERR_ARG;
  if (p->nx <= 0 || p->ny <= 0 || p->nz <= 0) return CZ_ERR_ARG;
  if (p->nx % B || p->ny % B || p->nz % B) return CZ_ERR_ARG;
  const long long nb = (long long)(p->nx / B) * (p->ny / B) * (p->nz / B);
  if (nb > (1ll << 30)) return CZ_ERR_ARG;
  if (sh) {
    sh->nbx = p->nx / B;
    sh->nby = p->ny / B;
    sh->nbz = p->nz / B;
    sh->nblocks = (int)nb;
    sh->L = B == 8 ? 1 : (B == 16 ? 2 : (B == 32 ? 3 : 4));
    sh->es = p->dtype == CZ_F64 ? 8 : 4;
    sh->G = G;
    sh->nchunks = (int)((nb + G - 1) / G);
    sh->data0 = (HEADER_BYTES + 8ull * (sh->nchunks + 1) + 15) / 16 * 16;
  }
  return CZ_OK;
}

// ---- strict error bound (host, fp64, every sum in increasing index order)
// One level of the 1D inverse transform on f[0..n): the same steps as the
// kernels (undo the W4li update, add back the W4 prediction; W3ai: even
// sample A_k + d_k, odd sample 2 a_k minus it).
void inv1d_host(int kind, double *f, int n)
{
  const int m = n / 2;
  double c[32], d[32], o[32];
  for (int k = 0; k < m; ++k) {
    c[k] = f[2 * k];
    d[k] = f[2 * k + 1];
  }
  if (kind == CZ_W4 || kind == CZ_W4LI) {
    if (kind == CZ_W4LI) {
      double e[32];
      for (int j = 0; j < m; ++j) {
        const czd::LiSrc ls = czd::li_src(j, m);
        double acc = czd::li_weight<double>(m, j, 0) * d[ls.k0];
        for (int t = 1; t < ls.nt; ++t) acc = acc + czd::li_weight<double>(m, j, t) * d[ls.k0 + t];
        e[j] = c[j] - acc;
      }
      for (int j = 0; j < m; ++j) c[j] = e[j];
    }
    for (int k = 0; k < m; ++k) {
      const czd::W4Row r = czd::w4_row(k, m);
      double pr = (double)r.w[0] * c[r.j0];
      pr = pr + (double)r.w[1] * c[r.j0 + 1];
      pr = pr + (double)r.w[2] * c[r.j0 + 2];
      pr = pr + (double)r.w[3] * c[r.j0 + 3];
      o[k] = d[k] + pr * 0.0625;
    }
  } else {
    double e[32];
    for (int k = 0; k < m; ++k) {
      double q;
      if (k == 0) {
        q = 3.0 * c[0];
        q = q - 4.0 * c[1];
        q = q + c[2];
      } else if (k == m - 1) {
        q = -3.0 * c[m - 1];
        q = q + 4.0 * c[m - 2];
        q = q - c[m - 3];
      } else {
        q = c[k - 1] - c[k + 1];
      }
      e[k] = (c[k] + q * 0.125) + d[k];
    }
    for (int k = 0; k < m; ++k) o[k] = 2.0 * c[k] - e[k];
    for (int k = 0; k < m; ++k) c[k] = e[k];
  }
  for (int k = 0; k < m; ++k) {
    f[2 * k] = c[k];
    f[2 * k + 1] = o[k];
  }
}

// C = max over the positions i of a block of sum_j |S_ij| over the detail
// columns j of the block synthesis S.  A level-l detail is rebuilt by the
// syntheses of levels l..0 only, whose composition is the Kronecker cube of
// a B x (B >> l) matrix; its columns' row sums are products of the 1D row
// sums over all columns (R) and over the even (coarse) columns (E).
double synthesis_norm_uncached(int kind, int B)
{
  int L = 0;
  while ((B >> L) > 4) ++L;
  double R[4][64], E[4][64];
  for (int l = 0; l < L; ++l) {
    const int nl = B >> l;
    for (int x = 0; x < B; ++x) R[l][x] = E[l][x] = 0.0;
    for (int j = 0; j < nl; ++j) {
      double w[64] = {0};
      w[j] = 1.0;
      for (int k = l; k >= 0; --k) {
        const int nk = B >> k;
        inv1d_host(kind, w, nk);
        if (k > 0) {
          double u[64] = {0};
          for (int i = 0; i < nk; ++i) u[2 * i] = w[i];
          for (int i = 0; i < 2 * nk; ++i) w[i] = u[i];
        }
      }
      for (int x = 0; x < B; ++x) {
        const double a = std::fabs(w[x]);
        R[l][x] += a;
        if (!(j & 1)) E[l][x] += a;
      }
    }
  }
  double C = 0.0;
  for (int iz = 0; iz < B; ++iz)
    for (int iy = 0; iy < B; ++iy)
      for (int ix = 0; ix < B; ++ix) {
        double sum = 0.0;
        for (int l = 0; l < L; ++l) sum += (R[l][ix] * R[l][iy]) * R[l][iz] - (E[l][ix] * E[l][iy]) * E[l][iz];
        if (sum > C) C = sum;
      }
  return C;
}

// divisor of the threshold for p: 1 (paper bound) or C (strict bound),
// computed once per (kind, B)
double threshold_divisor(const cz_params *p)
{
  if (p->bound_mode != CZ_BOUND_STRICT) return 1.0;
  static std::mutex mu;
  static double cache[3][4] = {{0}};
  const int bi = p->block == 8 ? 0 : (p->block == 16 ? 1 : (p->block == 32 ? 2 : 3));
  std::lock_guard<std::mutex> lock(mu);
  double &c = cache[p->kind][bi];
  if (c == 0.0) c = synthesis_norm_uncached(p->kind, p->block);
  return c;
}

struct Lanes {
  cudaError_t (*compress)(int, const CUtensorMap *, const FwdArgs *, const S2Args *, const PlaceArgs *, int, int,
                          int, const GroupArgs *, const int *, const cudaEvent_t *, cudaStream_t);
  cudaError_t (*compress_batch)(int, const StageMaps<MAXF> *, const FwdArgs *, const S2Args *, const BatchOut *,
                                const PlaceArgs *, int, int, int, int, int, int, cudaStream_t);
  cudaError_t (*decompress)(int, const CUtensorMap *, const InvArgs *, const UnArgs *, int, const int *,
                            const cudaEvent_t *, cudaStream_t);
  cudaError_t (*dense)(int, int, const DenseArgs *, int, cudaStream_t);
  int (*occupancy)(int, int);
  int (*slot_bytes)();
  int (*group_occupancy)(int, int);  // the group kernels (coder tiers 0-2, decoder tiers 0-2)
  int (*scratch_bytes)();  // global scratch per CTA (FP64 32^3 only)
  int (*alt_scratch_bytes)();  // per CTA of the batched slab stage kernel where the tuner may pick it
};

#define CZ_LANES(sfx)                                                                                      \
  Lanes                                                                                                    \
  {                                                                                                        \
    czl_compress_##sfx, czl_compress_batch_##sfx, czl_decompress_##sfx, czl_dense_##sfx, czl_occupancy_##sfx, \
        czl_slot_bytes_##sfx, czl_group_occupancy_##sfx, czl_scratch_bytes_##sfx, czl_alt_scratch_bytes_##sfx \
  }

Lanes lanes_for(const cz_params &p)
{
  const bool fast = (p.flags & CZ_FLAG_FAST) != 0;
  if (p.dtype == CZ_F32) {
    if (p.block == 8) return fast ? CZ_LANES(f32_b8_fast) : CZ_LANES(f32_b8);
    if (p.block == 16) return fast ? CZ_LANES(f32_b16_fast) : CZ_LANES(f32_b16);
    if (p.block == 32) return fast ? CZ_LANES(f32_b32_fast) : CZ_LANES(f32_b32);
    return fast ? CZ_LANES(f32_b64_fast) : CZ_LANES(f32_b64);
  }
  if (p.block == 8) return fast ? CZ_LANES(f64_b8_fast) : CZ_LANES(f64_b8);
  if (p.block == 16) return fast ? CZ_LANES(f64_b16_fast) : CZ_LANES(f64_b16);
  return fast ? CZ_LANES(f64_b32_fast) : CZ_LANES(f64_b32);
}

int sm_count()
{
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  return sms > 0 ? sms : 1;
}

// decoder choice (a test and measurement hook): 0 = one CTA per block (the
// default; measured the faster), 1 = the half-block decoder where the lane
// has one
int g_decoder_mode = 0;

// the half-block decoder (two CTAs per block, one per z-half) decodes p's
// blocks
bool use_half(const cz_params &p)
{
  if (__atomic_load_n(&g_decoder_mode, __ATOMIC_RELAXED) != 1) return false;
  return lanes_for(p).occupancy(p.kind, 6) > 0;
}

// the decoder InvArgs::decoder names for p
int decoder_of(const cz_params &p) { return use_half(p) ? 1 : 0; }

// persistent grids: one CTA per resident slot, at most one per block (per
// half block for the half-block decoder, whose grid is even so that a CTA
// keeps its half)
int grid_for(const cz_params *p, const Shape &sh, int which)
{
  const Lanes L = lanes_for(*p);
  if (which == 1 && use_half(*p)) {
    const long long g = (long long)sm_count() * L.occupancy(p->kind, 6);
    long long c = g < 2ll * sh.nblocks ? g : 2ll * sh.nblocks;
    c &= ~1ll;
    return (int)(c < 2 ? 2 : c);
  }
  int occ = L.occupancy(p->kind, which);
  // kernels that hold a block or a large payload in global scratch (one
  // scratch block per CTA): at most two CTAs per SM, which bounds the
  // scratch of the large stage-2 kernels
  if (L.scratch_bytes() && (which == 3 || which == 5) && occ > 2) occ = 2;
  const long long g = (long long)sm_count() * (occ > 0 ? occ : 1);
  return (int)(g < sh.nblocks ? g : sh.nblocks);
}

// workspace: header | one u64 look-back word per block | block table
// (slot offset, chunk bytes) | staging (one arena per stage CTA, room for
// the largest slot of each of its blocks)
size_t lb_bytes(const Shape &sh) { return (8ull * sh.nblocks + 255) / 256 * 256; }
size_t table_bytes(const Shape &sh) { return (16ull * sh.nblocks + 255) / 256 * 256; }

struct WsLayout {
  size_t lb, table, big, near, rlist, staging, scratch, total, arena;
  int grid, grid2, grid3;
  // aggregate chunks: group table, group slots and the large group coder's
  // scratch (one buffer of hcap bytes per CTA); zero sizes without groups
  size_t gtable, gstage, gscratch;
  unsigned long long gslot;
  int hcap;
  int ggrid[3];  // grids of the three coder tiers
};

// aggregate chunks: bytes of the largest group payload (a multiple of 128)
// and of a group slot, which holds the finished chunk: the nnz words, ntok,
// and at most the payload plus one trailing token plus one token per 65535
// literal words split off
int group_hcap(const cz_params *p, const Shape &sh)
{
  const size_t h = (size_t)sh.G * pmax_bytes(p->block, sh.es);
  return (int)((h + 127) / 128 * 128);
}

unsigned long long group_slot(const Shape &sh, int hcap)
{
  return (4ull * sh.G + 16ull + (unsigned long long)hcap + 4ull * ((unsigned long long)hcap / 262140ull + 1ull) +
          15ull) / 16ull * 16ull;
}

// grid of a group kernel over `items` (which: coder tiers 0, 1, 2, decoder
// tiers 3, 4, 5); the last tiers hold an hcap buffer in global scratch per
// CTA, so they run one CTA per SM
int group_grid(const cz_params *p, int which, int hcap, long long items)
{
  int occ = 1;
  if (which != 2 && which != 5) occ = lanes_for(*p).group_occupancy(which, hcap);
  const long long g = (long long)sm_count() * (occ > 0 ? occ : 1);
  const long long n = items > 0 ? items : 1;
  return (int)(g < n ? g : n);
}

size_t big_bytes(long long nblocks) { return (4ull * nblocks + 255) / 256 * 256; }

// global scratch of the FP64 32^3 kernels: one block per CTA of the stage
// kernel, the large stage-2 kernel and the large stage-2 inverse kernel
// (the largest of their grids; 0 bytes for every other lane)
size_t scratch_need(const cz_params *p, const Shape &sh, int grid, int grid3)
{
  const size_t per = (size_t)lanes_for(*p).scratch_bytes();
  if (!per) return 0;
  int n = grid > grid3 ? grid : grid3;
  const int gu = grid_for(p, sh, 5);
  n = n > gu ? n : gu;
  return per * (size_t)n;
}

// offset of the decoded blocks' slots in the decompress workspace, after
// the header, the block table and the list of the large chunks (aggregate
// chunks: two lists of groups, for the decoder tiers)
size_t dec_slots_off(const Shape &dsh)
{
  return WS_HDR + table_bytes(dsh) + big_bytes((dsh.G > 1 ? 2ll : 1ll) * dsh.nblocks);
}

// workspace of decompress_impl for the decoded blocks dsh: header | block
// table | list of the large chunks | one staging slot per decoded block
// (stage 2 only) | scratch of the large stage-2 inverse kernel (FP64 32^3)
size_t dec_ws_need(const cz_params *p, const Shape &dsh, size_t *scratch_off)
{
  if (!p->stage2) {
    if (scratch_off) *scratch_off = 0;
    return WS_HDR;
  }
  const Lanes L = lanes_for(*p);
  const size_t off = dec_slots_off(dsh) + (size_t)dsh.nblocks * L.slot_bytes();
  if (scratch_off) *scratch_off = off;
  if (dsh.G > 1) {  // the last decoder tier's buffers
    const int hcap = group_hcap(p, dsh);
    return off + (size_t)hcap * (size_t)group_grid(p, 5, hcap, dsh.nblocks);
  }
  const size_t per = (size_t)L.scratch_bytes();
  return off + (per ? per * (size_t)grid_for(p, dsh, 5) : 0);
}

// bit zeroing width of the kept details (0, 4 or 8)
int zero_bits(const cz_params &p)
{
  return (p.flags & CZ_FLAG_ZERO8) ? 8 : (p.flags & CZ_FLAG_ZERO4) ? 4 : 0;
}

WsLayout ws_layout(const cz_params *p, const Shape &sh)
{
  const Lanes L = lanes_for(*p);
  WsLayout w;
  w.grid = grid_for(p, sh, 0);
  w.grid2 = grid_for(p, sh, 2);
  w.grid3 = grid_for(p, sh, 3);
  w.lb = WS_HDR;
  w.table = w.lb + lb_bytes(sh);
  w.big = w.table + table_bytes(sh);
  // speculative thresholds: one byte per block, and the list of the slots
  // to refine
  w.near = w.big + big_bytes(sh.nblocks);
  w.rlist = w.near + ((size_t)sh.nblocks + 255) / 256 * 256;
  w.staging = w.rlist + big_bytes(sh.nblocks);
  // blocks are dealt round robin to the stage CTAs
  w.arena = (((size_t)sh.nblocks + w.grid - 1) / w.grid) * (size_t)L.slot_bytes();
  w.scratch = w.staging + w.arena * (size_t)w.grid;
  w.total = w.scratch + scratch_need(p, sh, w.grid, w.grid3);
  w.gtable = w.gstage = w.gscratch = 0;
  w.gslot = 0;
  w.hcap = 0;
  w.ggrid[0] = w.ggrid[1] = w.ggrid[2] = 0;
  if (sh.G > 1) {
    w.hcap = group_hcap(p, sh);
    w.gslot = group_slot(sh, w.hcap);
    for (int t = 0; t < 3; ++t) w.ggrid[t] = group_grid(p, t, w.hcap, sh.nchunks);
    w.gtable = (w.total + 255) / 256 * 256;
    w.gstage = w.gtable + (16ull * sh.nchunks + 255) / 256 * 256;
    w.gscratch = (w.gstage + (size_t)sh.nchunks * w.gslot + 255) / 256 * 256;
    w.total = w.gscratch + (size_t)w.hcap * (size_t)w.ggrid[2];
    // cz_workspace_size covers decompression too, whose large-group decoder
    // may run more CTAs (one per block, up to one per SM)
    const size_t dec = dec_ws_need(p, sh, nullptr);
    w.total = w.total > dec ? w.total : dec;
  }
  return w;
}

size_t ws_need(const cz_params *p, const Shape &sh) { return ws_layout(p, sh).total; }

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
  }
  return fn;
}

// 3D tiled tensor map over the field, one B^3 box per block; FP32 32^3
// W4li boxes (128-byte rows) take the 128-byte swizzle (the stage kernel and
// the one-CTA-per-block decoder address their W4li tiles that way); half =
// true: a B x B x B/2 box without swizzle (the half-block decoder's stores)
bool make_tile_map(CUtensorMap *tm, const cz_params *p, const void *d_field, bool half = false)
{
  auto enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t es = p->dtype == CZ_F64 ? 8 : 4;
  const cuuint64_t dims[3] = {(cuuint64_t)p->nx, (cuuint64_t)p->ny, (cuuint64_t)p->nz};
  const cuuint64_t strides[2] = {(cuuint64_t)p->nx * es, (cuuint64_t)p->nx * p->ny * es};
  // (the kernels of FP64 32^3 and of 64^3 blocks address the field directly
  // and do not use the map: a box of 8 z-planes keeps it within the
  // encoder's limits)
  const cuuint32_t bz = ((p->dtype == CZ_F64 && p->block == 32) || p->block == 64) ? 8u
                        : half                                                   ? (cuuint32_t)p->block / 2
                                                                                 : (cuuint32_t)p->block;
  const cuuint32_t box[3] = {(cuuint32_t)p->block, (cuuint32_t)p->block, bz};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r =
      enc(tm, p->dtype == CZ_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
          const_cast<void *>(d_field), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
          (p->dtype == CZ_F32 && p->block == 32 && p->kind == CZ_W4LI && !half) ? CU_TENSOR_MAP_SWIZZLE_128B
                                                                                : CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// the subsample of speculative thresholds (every 4th row of every 4th
// z-plane): one warp per row, at most four 512-thread CTAs per SM
template <typename T>
cudaError_t run_minmax_sample(const cz_params *p, const void *field, WsHdr *ws, cudaStream_t s)
{
  const long long rows = (long long)((p->ny + 3) / 4) * ((p->nz + 3) / 4);
  long long blocks = (rows + 15) / 16;
  const long long cap = (long long)sm_count() * 4;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  k_minmax_sample<T><<<(unsigned)blocks, 512, 0, s>>>(reinterpret_cast<const T *>(field), p->nx, p->ny, p->nz, ws);
  return cudaGetLastError();
}

// speculative thresholds for p: the range is computed (one field, stage 2
// on, the paper bound, no bit zeroing, no aggregate chunks, a
// register-resident stage kernel); the stage kernel then merges the
// blocks' min / max itself and stage 2 drops the details below the exact
// threshold
bool speculative(const cz_params *p, const Shape &sh)
{
  return p->range < 0 && p->stage2 && p->bound_mode == CZ_BOUND_PAPER && zero_bits(*p) == 0 && sh.G == 1 &&
         lanes_for(*p).scratch_bytes() == 0;
}

template <typename T>
cudaError_t run_minmax(const void *field, size_t n, WsHdr *ws, cudaStream_t s)
{
  size_t blocks = (n / (sizeof(T) == 4 ? 4 : 2) + 511) / 512;
  const size_t cap = (size_t)sm_count() * 4;
  if (blocks > cap) blocks = cap;
  if (blocks == 0) blocks = 1;
  k_minmax<T><<<(unsigned)blocks, 512, 0, s>>>(reinterpret_cast<const T *>(field), n, ws);
  return cudaGetLastError();
}

__global__ void k_fp64_probe(int iters, double *sink)
{
  double a[8];
  const double m = 1.0 + 1e-9 * threadIdx.x, c = 1e-12;
#pragma unroll
  for (int q = 0; q < 8; ++q) a[q] = 1.0 + q * 1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = fma(a[q], m, c);
  }
  double s = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) s += a[q];
  if (s == 0.0) *sink = s;  // never true; keeps the chains live
}

// Drives the codec's bounded waits past a short limit (tests of the
// timeout paths; nothing faults and nothing waits without bound).
//  which 0: the look-back of the chunk-offset scan.  One warp per tile;
//    tile `skip` never publishes its aggregate, so the tiles after it spin
//    until `limit`, then record ST_TIMEOUT and return.  out[t] = exclusive
//    prefix seen by tile t (t for the tiles before `skip`: aggregates of 1).
//  which 1: an mbarrier armed for 16 bytes that no copy delivers.  Every
//    thread waits until `limit`; the CTA decides at one barrier, as the
//    codec kernels do, and thread 0 records ST_TIMEOUT.  out[tid] = the
//    CTA's decision (1: gave up) as each thread saw it.
__global__ void k_wait_probe(int which, int skip, unsigned limit, unsigned *status, unsigned long long *state,
                             unsigned long long *out)
{
  if (which == 0) {
    const int tile = blockIdx.x;
    if (tile == skip) return;
    const unsigned long long ex = lookback(state, tile, 1ull, status, (int)ST_TIMEOUT, 0, limit);
    if (threadIdx.x == 0) out[tile] = ex;
    return;
  }
  __shared__ __align__(8) unsigned long long bar;
  __shared__ unsigned s_to;
  if (threadIdx.x == 0) {
    mbar_init(&bar);
    s_to = 0;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&bar)), "r"(16u)
                 : "memory");
  }
  __syncthreads();
  if (!mbar_wait(&bar, 0u, limit)) s_to = 1u;
  __syncthreads();
  const unsigned gave_up = *(volatile unsigned *)&s_to;
  if (threadIdx.x == 0 && gave_up) atomicCAS(status, 0u, ST_TIMEOUT);
  out[threadIdx.x] = gave_up;
}

// ---- batched compression
// fields of one launch: same element type, block, kind, stage 2 and bound
// mode, at most MAXF, in the order the caller gave them
struct Group {
  std::vector<int> idx;
};

std::vector<Group> plan_batch(int n, const cz_params *p)
{
  std::vector<Group> out;
  std::vector<int> open;  // index in `out` of the last group of each signature
  auto same = [&](const cz_params &a, const cz_params &b) {
    return a.dtype == b.dtype && a.block == b.block && a.kind == b.kind && a.stage2 == b.stage2 &&
           a.bound_mode == b.bound_mode && a.flags == b.flags;
  };
  for (int i = 0; i < n; ++i) {
    int g = -1;
    for (int q : open)
      if (same(p[out[q].idx[0]], p[i]) && (int)out[q].idx.size() < MAXF) g = q;
    if (g < 0) {
      out.push_back(Group{});
      g = (int)out.size() - 1;
      open.push_back(g);
    }
    out[g].idx.push_back(i);
  }
  return out;
}

// knobs chosen by cz_batch_tune for a group of fields (one launch)
struct BatchKnobs {
  int s1_balanced;  // stage grid: fewest CTAs with the same number of rounds
  int s2_div;       // stage-2 CTAs: resident slots / s2_div
  int place_tile;   // scan granularity: chunks per look-back tile (64, 128, 256)
  int slab;         // stage kernel: 0 = register-resident pair quads, 1 = slab kernel (block in global scratch)
};

constexpr BatchKnobs DEFAULT_KNOBS{0, 1, 128, 0};

// the knob settings the tuner tries for a group whose first field is p0
std::vector<BatchKnobs> knob_candidates(const cz_params &p0)
{
  std::vector<BatchKnobs> c;
  const bool alt = lanes_for(p0).alt_scratch_bytes() > 0;
  for (int slab = 0; slab <= (alt ? 1 : 0); ++slab)
    for (int b = 0; b <= 1; ++b)
      for (int d = 1; d <= 2; ++d)
        for (int pt : {64, 128, 256}) c.push_back(BatchKnobs{b, d, pt, slab});
  return c;
}

struct BatchLayout {
  size_t keys, lb, table, big, staging, scratch, total, arena;
  int grid, grid2, grid3, tiles, nblocks;
};

BatchLayout batch_layout(const Group &g, const cz_params *p, const BatchKnobs &kn)
{
  const cz_params &p0 = p[g.idx[0]];
  const int PT = kn.place_tile;
  BatchLayout w{};
  w.nblocks = 0;
  w.tiles = 0;
  for (int i : g.idx) {
    Shape sh;
    check(&p[i], &sh);
    w.nblocks += sh.nblocks;
    w.tiles += (sh.nblocks + PT - 1) / PT;
  }
  Shape all{};
  all.nblocks = w.nblocks;
  const Lanes L = lanes_for(p0);
  const bool slab = kn.slab && L.alt_scratch_bytes() > 0;
  if (slab) {
    const long long gs = (long long)sm_count() * (L.occupancy(p0.kind, 7) > 0 ? L.occupancy(p0.kind, 7) : 1);
    w.grid = (int)(gs < w.nblocks ? gs : w.nblocks);
  } else {
    w.grid = grid_for(&p0, all, 0);
  }
  if (kn.s1_balanced) {
    const int rounds = (w.nblocks + w.grid - 1) / w.grid;
    w.grid = (w.nblocks + rounds - 1) / rounds;
  }
  w.grid2 = grid_for(&p0, all, 2) / (kn.s2_div > 0 ? kn.s2_div : 1);
  w.grid3 = grid_for(&p0, all, 3) / (kn.s2_div > 0 ? kn.s2_div : 1);
  if (w.grid2 < 1) w.grid2 = 1;
  if (w.grid3 < 1) w.grid3 = 1;
  w.keys = WS_HDR;
  w.lb = w.keys + 16 * MAXF;
  w.table = w.lb + (8ull * w.tiles + 255) / 256 * 256;
  w.big = w.table + (16ull * w.nblocks + 255) / 256 * 256;
  w.staging = w.big + big_bytes(w.nblocks);
  w.arena = (((size_t)w.nblocks + w.grid - 1) / w.grid) * (size_t)L.slot_bytes();
  w.scratch = w.staging + w.arena * (size_t)w.grid;
  size_t scr = scratch_need(&p0, all, w.grid, w.grid3);
  if (slab) {
    const size_t alt = (size_t)L.alt_scratch_bytes() * (size_t)w.grid;
    scr = alt > scr ? alt : scr;
  }
  w.total = w.scratch + scr;
  return w;
}

std::mutex g_knob_mu;
std::vector<std::pair<unsigned long long, BatchKnobs>> g_knobs;

// signature of a group of fields: the parameters of every field of the
// group (not the pointers)
unsigned long long group_signature(const Group &g, const cz_params *p)
{
  unsigned long long h = 1469598103934665603ull;
  auto mix = [&](unsigned long long v) { h = (h ^ v) * 1099511628211ull; };
  mix((unsigned long long)g.idx.size());
  for (int i : g.idx) {
    mix((unsigned long long)p[i].nx);
    mix((unsigned long long)p[i].ny);
    mix((unsigned long long)p[i].nz);
    mix((unsigned long long)(p[i].block | p[i].dtype << 8 | p[i].kind << 12 | p[i].stage2 << 16 |
                             p[i].bound_mode << 20 | p[i].flags << 24));
  }
  return h;
}

BatchKnobs knobs_for(const Group &g, const cz_params *p)
{
  const unsigned long long sig = group_signature(g, p);
  std::lock_guard<std::mutex> lock(g_knob_mu);
  for (auto &e : g_knobs)
    if (e.first == sig) {
      BatchKnobs k = e.second;
      if (k.slab && lanes_for(p[g.idx[0]]).alt_scratch_bytes() == 0) k.slab = 0;  // not this lane's choice
      return k;
    }
  return DEFAULT_KNOBS;
}

void set_knobs(const Group &g, const cz_params *p, const BatchKnobs &k)
{
  const unsigned long long sig = group_signature(g, p);
  std::lock_guard<std::mutex> lock(g_knob_mu);
  for (auto &e : g_knobs)
    if (e.first == sig) {
      e.second = k;
      return;
    }
  g_knobs.push_back({sig, k});
}

// workspace for every group under its stored knobs, or under every
// candidate setting (all = true: room for whatever the tuner picks).  The
// largest layouts are those with the most look-back tiles (64 chunks) and
// the full stage-2 grid, so only those candidates are laid out.
size_t batch_ws_need(int n, const cz_params *p, bool all)
{
  size_t need = WS_HDR;
  for (const Group &g : plan_batch(n, p)) {
    std::vector<BatchKnobs> ks;
    if (all) {
      for (const BatchKnobs &k : knob_candidates(p[g.idx[0]]))
        if (k.place_tile == 64 && k.s2_div == 1) ks.push_back(k);
    } else {
      ks.push_back(knobs_for(g, p));
    }
    for (const BatchKnobs &kn : ks) {
      const BatchLayout w = batch_layout(g, p, kn);
      need = w.total > need ? w.total : need;
    }
  }
  return need;
}

// one group's launches (its fields share dtype, block, kind, stage 2, bound
// mode and flags) with knobs kn; the workspace is the group's alone
int compress_group(const Group &g, const cz_params *p, const void *const *d_fields, void *const *d_outs,
                   const size_t *out_caps, uint64_t *d_out_bytes, unsigned char *wsb, cudaStream_t s,
                   const BatchKnobs &kn)
{
  const cz_params &p0 = p[g.idx[0]];
  const BatchLayout w = batch_layout(g, p, kn);
  const int nf = (int)g.idx.size();
  // ticket, min/max keys (min keys all ones) and look-back words
  if (cudaMemsetAsync(wsb + 4, 0, w.table - 4, s) != cudaSuccess) return CZ_ERR_CUDA;
  if (cudaMemset2DAsync(wsb + w.keys, 16, 0xFF, 8, nf, s) != cudaSuccess) return CZ_ERR_CUDA;
  unsigned long long *keys = reinterpret_cast<unsigned long long *>(wsb + w.keys);
  MinmaxArgs mm{};
  mm.keys = keys;
  unsigned long long maxn = 0;
  StageMaps<MAXF> maps{};
  BatchOut bo{};
  bo.nf = nf;
  int first = 0, tfirst = 0;
  for (int f = 0; f < nf; ++f) {
    const int i = g.idx[f];
    Shape sh;
    check(&p[i], &sh);
    const bool need_range = p[i].range < 0 && p[i].eps_mode == CZ_EPS_REL;
    mm.field[f] = d_fields[i];
    mm.n[f] = need_range ? (unsigned long long)p[i].nx * p[i].ny * p[i].nz : 0ull;
    maxn = mm.n[f] > maxn ? mm.n[f] : maxn;
    if (!make_tile_map(&maps.tm[f], &p[i], d_fields[i])) return CZ_ERR_CUDA;
    maps.g[f] = FieldGeo{d_fields[i], sh.nbx, sh.nby, first, p[i].eps_mode, p[i].eps, p[i].range};
    FieldOut &fo = bo.f[f];
    fo.out = reinterpret_cast<unsigned char *>(d_outs[i]);
    fo.out_bytes = d_out_bytes ? reinterpret_cast<unsigned long long *>(d_out_bytes + i) : nullptr;
    fo.out_cap = out_caps[i];
    fo.data0 = sh.data0;
    fo.eps = p[i].eps;
    fo.range_in = p[i].range;
    fo.nx = p[i].nx;
    fo.ny = p[i].ny;
    fo.nz = p[i].nz;
    fo.nblocks = sh.nblocks;
    fo.first = first;
    fo.tfirst = tfirst;
    fo.eps_mode = p[i].eps_mode;
    first += sh.nblocks;
    tfirst += (sh.nblocks + kn.place_tile - 1) / kn.place_tile;
  }
  if (maxn > 0) {
    const dim3 grid((unsigned)((maxn + MM_CHUNK - 1) / MM_CHUNK), (unsigned)nf);
    if (p0.dtype == CZ_F32)
      k_minmax_multi<float><<<grid, 512, 0, s>>>(mm);
    else
      k_minmax_multi<double><<<grid, 512, 0, s>>>(mm);
    if (cudaGetLastError() != cudaSuccess) return CZ_ERR_CUDA;
  }
  FwdArgs a{};
  a.ws = wsb;
  a.keys = keys;
  a.biglist = reinterpret_cast<int *>(wsb + w.big);
  a.staging = wsb + w.staging;
  a.arena_bytes = w.arena;
  a.scratch = wsb + w.scratch;
  a.table = reinterpret_cast<unsigned long long *>(wsb + w.table);
  a.cnorm = threshold_divisor(&p0);
  a.nblocks = w.nblocks;
  a.nf = nf;
  a.stage2 = p0.stage2;
  a.kind = p0.kind;
  a.zbits = zero_bits(p0);
  a.dtype = p0.dtype;
  S2Args sa{};
  sa.staging = a.staging;
  sa.table = a.table;
  sa.ws = wsb;
  sa.biglist = a.biglist;
  sa.scratch = a.scratch;
  sa.nblocks = w.nblocks;
  PlaceArgs pa{};
  pa.staging = a.staging;
  pa.table = a.table;
  pa.keys = keys;
  pa.lbst = reinterpret_cast<unsigned long long *>(wsb + w.lb);
  pa.ws = wsb;
  pa.cnorm = a.cnorm;
  pa.nblocks = w.nblocks;
  pa.block = p0.block;
  pa.levels = p0.block == 8 ? 1 : (p0.block == 16 ? 2 : (p0.block == 32 ? 3 : 4));
  pa.stage2 = p0.stage2;
  pa.kind = p0.kind;
  pa.dtype = p0.dtype;
  pa.bound_mode = p0.bound_mode;
  pa.flags = p0.flags;
  const Lanes L = lanes_for(p0);
  const int slab = kn.slab && L.alt_scratch_bytes() > 0 ? 1 : 0;
  if (L.compress_batch(p0.kind, &maps, &a, &sa, &bo, &pa, w.grid, w.grid2, w.grid3, w.tiles, kn.place_tile, slab,
                       s) != cudaSuccess)
    return CZ_ERR_CUDA;
  return CZ_OK;
}

int batch_check(int n, const cz_params *p, const void *const *d_fields, void *const *d_outs, const size_t *out_caps,
                const void *d_ws)
{
  if (n < 0 || (n > 0 && (!p || !d_fields || !d_outs || !out_caps)) || !d_ws) return CZ_ERR_ARG;
  if ((uintptr_t)d_ws % 16) return CZ_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    Shape sh;
    const int r = check(&p[i], &sh);
    if (r != CZ_OK) return r;
    if (sh.G > 1) return CZ_ERR_ARG;  // batched launches take no aggregate chunks
    if (!d_fields[i] || !d_outs[i] || ((uintptr_t)d_fields[i] % 16) || ((uintptr_t)d_outs[i] % 16))
      return CZ_ERR_ARG;
    if (out_caps[i] < sh.data0) return CZ_ERR_CAPACITY;
  }
  return CZ_OK;
}

// every group with its stored knobs (the tuner's choices, else the
// defaults), or with `force` for every group
int compress_batch_impl(int n, const cz_params *p, const void *const *d_fields, void *const *d_outs,
                        const size_t *out_caps, uint64_t *d_out_bytes, void *d_ws, size_t ws_bytes,
                        cudaStream_t s, const BatchKnobs *force = nullptr)
{
  const NvtxRange nvtx("cz_compress_batch");
  const int r = batch_check(n, p, d_fields, d_outs, out_caps, d_ws);
  if (r != CZ_OK) return r;
  if (ws_bytes < batch_ws_need(n, p, force != nullptr)) return CZ_ERR_CAPACITY;
  unsigned char *wsb = reinterpret_cast<unsigned char *>(d_ws);
  if (cudaMemsetAsync(d_ws, 0, 4, s) != cudaSuccess) return CZ_ERR_CUDA;  // status, once for the batch
  for (const Group &g : plan_batch(n, p)) {
    BatchKnobs kn = force ? *force : knobs_for(g, p);
    if (kn.slab && lanes_for(p[g.idx[0]]).alt_scratch_bytes() == 0) kn.slab = 0;  // not this lane's choice
    const int rg = compress_group(g, p, d_fields, d_outs, out_caps, d_out_bytes, wsb, s, kn);
    if (rg != CZ_OK) return rg;
  }
  return CZ_OK;
}

unsigned long long rd64(const unsigned char *p)
{
  unsigned long long v;
  std::memcpy(&v, p, 8);
  return v;
}

}  // namespace

extern "C" {

int cz_compress_bound(const cz_params *p, size_t *bytes)
{
  Shape sh;
  const int r = check(p, &sh);
  if (r != CZ_OK || !bytes) return r ? r : CZ_ERR_ARG;
  const size_t B = (size_t)p->block, s = (size_t)sh.es;
  const size_t pmax = 64 * s + B * B * B / 8 + (B * B * B - 64) * s;
  // raw chunk: 8 + pmax; stage-2 chunk: 8 + 4 * tokens + literal words,
  // where every token but the last and the splits removes >= 2 zero words
  size_t chunk = 16 + pmax + 8 * ((pmax / 4 + 65534) / 65535);
  chunk = (chunk + 3) / 4 * 4;
  *bytes = (size_t)sh.data0 + (size_t)sh.nblocks * chunk;
  return CZ_OK;
}

int cz_workspace_size(const cz_params *p, size_t *bytes)
{
  Shape sh;
  const int r = check(p, &sh);
  if (r != CZ_OK || !bytes) return r ? r : CZ_ERR_ARG;
  *bytes = ws_need(p, sh);
  return CZ_OK;
}

namespace {

int compress_impl(const cz_params *p, const void *d_field, void *d_out, size_t out_cap,
                  uint64_t *d_out_bytes, void *d_ws, size_t ws_bytes, void *stream,
                  const cudaEvent_t *marks)
{
  const NvtxRange nvtx("cz_compress");
  Shape sh;
  int r = check(p, &sh);
  if (r != CZ_OK) return r;
  if (!d_field || !d_out || !d_ws) return CZ_ERR_ARG;
  if (((uintptr_t)d_field % 16) || ((uintptr_t)d_out % 16) || ((uintptr_t)d_ws % 16)) return CZ_ERR_ARG;
  const WsLayout wl = ws_layout(p, sh);
  if (out_cap < sh.data0 || ws_bytes < wl.total) return CZ_ERR_CAPACITY;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  WsHdr *ws = reinterpret_cast<WsHdr *>(d_ws);
  unsigned char *wsb = reinterpret_cast<unsigned char *>(d_ws);
  if (cudaMemsetAsync(d_ws, 0, wl.table, s) != cudaSuccess) return CZ_ERR_CUDA;
  const bool spec = speculative(p, sh);
  if (p->range < 0) {
    if (cudaMemsetAsync(&ws->minkey, 0xFF, 8, s) != cudaSuccess) return CZ_ERR_CUDA;
    cudaError_t e;
    if (spec) {  // the subsample only; the stage kernel merges the blocks' min / max
      if (cudaMemsetAsync(&ws->skmin, 0xFF, 8, s) != cudaSuccess) return CZ_ERR_CUDA;
      e = p->dtype == CZ_F32 ? run_minmax_sample<float>(p, d_field, ws, s)
                             : run_minmax_sample<double>(p, d_field, ws, s);
    } else {
      const size_t n = (size_t)p->nx * p->ny * p->nz;
      e = p->dtype == CZ_F32 ? run_minmax<float>(d_field, n, ws, s) : run_minmax<double>(d_field, n, ws, s);
    }
    if (e != cudaSuccess) return CZ_ERR_CUDA;
  }
  const Lanes L = lanes_for(*p);
  FwdArgs a{};
  a.field = d_field;
  a.ws = d_ws;
  a.biglist = reinterpret_cast<int *>(wsb + wl.big);
  a.staging = wsb + wl.staging;
  a.arena_bytes = wl.arena;
  a.scratch = wsb + wl.scratch;
  a.table = reinterpret_cast<unsigned long long *>(wsb + wl.table);
  a.eps = p->eps;
  a.range = p->range;
  a.cnorm = threshold_divisor(p);
  a.nx = p->nx;
  a.ny = p->ny;
  a.nz = p->nz;
  a.nbx = sh.nbx;
  a.nby = sh.nby;
  a.nbz = sh.nbz;
  a.nblocks = sh.nblocks;
  a.eps_mode = p->eps_mode;
  a.stage2 = sh.G > 1 ? 0 : p->stage2;  // aggregate chunks: raw slots, the group coders do stage 2
  a.kind = p->kind;
  a.zbits = zero_bits(*p);
  a.dtype = p->dtype;
  a.spec = spec ? 1 : 0;
  a.near = spec ? wsb + wl.near : nullptr;
  S2Args sa{};
  sa.staging = a.staging;
  sa.table = a.table;
  sa.ws = d_ws;
  sa.biglist = a.biglist;
  sa.scratch = a.scratch;
  sa.nblocks = sh.nblocks;
  sa.spec = a.spec;
  sa.near = a.near;
  sa.rlist = spec ? reinterpret_cast<int *>(wsb + wl.rlist) : nullptr;
  sa.eps = p->eps;
  sa.eps_mode = p->eps_mode;
  PlaceArgs pa{};
  pa.staging = a.staging;
  pa.table = a.table;
  pa.out = reinterpret_cast<unsigned char *>(d_out);
  pa.out_bytes = reinterpret_cast<unsigned long long *>(d_out_bytes);
  pa.ws = d_ws;
  pa.out_cap = out_cap;
  pa.data0 = sh.data0;
  pa.eps = p->eps;
  pa.range = p->range;
  pa.cnorm = a.cnorm;
  pa.bound_mode = p->bound_mode;
  pa.flags = p->flags;
  pa.nx = p->nx;
  pa.ny = p->ny;
  pa.nz = p->nz;
  pa.nblocks = sh.nblocks;
  pa.hdr_nblocks = sh.nblocks;
  pa.block = p->block;
  pa.levels = sh.L;
  pa.eps_mode = p->eps_mode;
  pa.stage2 = p->stage2;
  pa.kind = p->kind;
  pa.dtype = p->dtype;
  GroupArgs ga{};
  if (sh.G > 1) {
    // the group coders read the block slots and table and fill the group
    // slots and table, over which placement and copy then run
    ga.staging = a.staging;
    ga.table = a.table;
    ga.gstage = wsb + wl.gstage;
    ga.gtable = reinterpret_cast<unsigned long long *>(wsb + wl.gtable);
    ga.ws = d_ws;
    ga.biglist = a.biglist;
    ga.scratch = wsb + wl.gscratch;
    ga.gslot = wl.gslot;
    ga.hcap = wl.hcap;
    ga.nblocks = sh.nblocks;
    ga.ngroups = sh.nchunks;
    ga.G = sh.G;
    pa.staging = ga.gstage;
    pa.table = ga.gtable;
    pa.nblocks = sh.nchunks;
  }
  CUtensorMap tm;
  if (!make_tile_map(&tm, p, d_field)) return CZ_ERR_CUDA;
  return L.compress(p->kind, &tm, &a, &sa, &pa, wl.grid, wl.grid2, wl.grid3, sh.G > 1 ? &ga : nullptr, wl.ggrid,
                    marks, s) == cudaSuccess
             ? CZ_OK
             : CZ_ERR_CUDA;
}

}  // namespace

int cz_compress(const cz_params *p, const void *d_field, void *d_out, size_t out_cap,
                uint64_t *d_out_bytes, void *d_ws, size_t ws_bytes, void *stream)
{
  return compress_impl(p, d_field, d_out, out_cap, d_out_bytes, d_ws, ws_bytes, stream, nullptr);
}

int cz_batch_workspace_size(int n, const cz_params *p, size_t *bytes)
{
  if (n < 0 || !bytes || (n > 0 && !p)) return CZ_ERR_ARG;
  for (int i = 0; i < n; ++i)
    if (check(&p[i], nullptr) != CZ_OK || group_of(p[i].flags) > 1) return CZ_ERR_ARG;
  *bytes = batch_ws_need(n, p, true);  // room for every knob setting the tuner may pick
  return CZ_OK;
}

int cz_compress_batch(int n, const cz_params *p, const void *const *d_fields, void *const *d_outs,
                      const size_t *out_caps, uint64_t *d_out_bytes, void *d_ws, size_t ws_bytes, void *stream)
{
  return compress_batch_impl(n, p, d_fields, d_outs, out_caps, d_out_bytes, d_ws, ws_bytes,
                             reinterpret_cast<cudaStream_t>(stream));
}

int cz_batch_tune(int n, const cz_params *p, const void *const *d_fields, void *const *d_outs,
                  const size_t *out_caps, uint64_t *d_out_bytes, void *d_ws, size_t ws_bytes, void *stream,
                  int reps)
{
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int r = batch_check(n, p, d_fields, d_outs, out_caps, d_ws);
  if (r != CZ_OK) return r;
  if (ws_bytes < batch_ws_need(n, p, true)) return CZ_ERR_CAPACITY;
  unsigned char *wsb = reinterpret_cast<unsigned char *>(d_ws);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return CZ_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return CZ_ERR_CUDA;
  }
  // every group on its own: each candidate once to warm up, then `reps`
  // timed launches; the fastest is kept for the group's signature
  for (const Group &g : plan_batch(n, p)) {
    const std::vector<BatchKnobs> cand = knob_candidates(p[g.idx[0]]);
    int best = -1;
    float best_ms = 0;
    for (size_t c = 0; c < cand.size() && r == CZ_OK; ++c) {
      if (cudaMemsetAsync(wsb, 0, 4, s) != cudaSuccess) r = CZ_ERR_CUDA;
      if (r == CZ_OK) r = compress_group(g, p, d_fields, d_outs, out_caps, d_out_bytes, wsb, s, cand[c]);
      if (r != CZ_OK) break;
      if (cudaEventRecord(e0, s) != cudaSuccess) r = CZ_ERR_CUDA;
      for (int q = 0; q < (reps > 0 ? reps : 3) && r == CZ_OK; ++q)
        r = compress_group(g, p, d_fields, d_outs, out_caps, d_out_bytes, wsb, s, cand[c]);
      if (r != CZ_OK) break;
      if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
        r = CZ_ERR_CUDA;
        break;
      }
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (best < 0 || ms < best_ms) {
        best = (int)c;
        best_ms = ms;
      }
    }
    if (r != CZ_OK) break;
    if (best >= 0) set_knobs(g, p, cand[best]);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return r;
}

// ---- quantities of a cell-struct array: de-interleave, then one batched
// compression of the chosen components
extern "C++" {
namespace {

struct AosPick {
  int n;
  int comp[MAXF];
  void *out[MAXF];
};

// one cell per thread (grid-stride): its chosen components go to their
// dense fields; consecutive threads read consecutive cells and write
// consecutive elements of every field
template <typename T>
__global__ void __launch_bounds__(256) k_deinterleave(const T *cells, int ncomp, const AosPick pick,
                                                      unsigned long long ncells)
{
  for (unsigned long long i = blockIdx.x * 256ull + threadIdx.x; i < ncells; i += (unsigned long long)gridDim.x * 256)
    for (int q = 0; q < pick.n; ++q) reinterpret_cast<T *>(pick.out[q])[i] = cells[i * ncomp + pick.comp[q]];
}

size_t aos_field_bytes(const cz_params &p)
{
  return ((size_t)p.nx * p.ny * p.nz * (p.dtype == CZ_F64 ? 8 : 4) + 255) / 256 * 256;
}

int aos_check(int n, const cz_params *p)
{
  if (n < 1 || n > MAXF || !p) return CZ_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    if (check(&p[i], nullptr) != CZ_OK || group_of(p[i].flags) > 1) return CZ_ERR_ARG;
    if (p[i].nx != p[0].nx || p[i].ny != p[0].ny || p[i].nz != p[0].nz || p[i].dtype != p[0].dtype)
      return CZ_ERR_ARG;
  }
  return CZ_OK;
}

}  // namespace
}  // extern "C++"

int cz_aos_workspace_size(int n, const cz_params *p, size_t *bytes)
{
  if (!bytes) return CZ_ERR_ARG;
  const int r = aos_check(n, p);
  if (r != CZ_OK) return r;
  size_t b = 0;
  const int rb = cz_batch_workspace_size(n, p, &b);
  if (rb != CZ_OK) return rb;
  *bytes = (b + 255) / 256 * 256 + (size_t)n * aos_field_bytes(p[0]);
  return CZ_OK;
}

int cz_compress_aos(int n, const cz_params *p, const void *d_cells, int ncomp, const int32_t *comps,
                    void *const *d_outs, const size_t *out_caps, uint64_t *d_out_bytes, void *d_ws,
                    size_t ws_bytes, void *stream)
{
  int r = aos_check(n, p);
  if (r != CZ_OK) return r;
  if (!d_cells || !comps || !d_outs || !out_caps || !d_ws || ncomp < 1 || ncomp > 4096) return CZ_ERR_ARG;
  const size_t es = p[0].dtype == CZ_F64 ? 8 : 4;
  if ((uintptr_t)d_cells % es || (uintptr_t)d_ws % 16) return CZ_ERR_ARG;
  for (int i = 0; i < n; ++i)
    if (comps[i] < 0 || comps[i] >= ncomp) return CZ_ERR_ARG;
  size_t need = 0;
  if ((r = cz_aos_workspace_size(n, p, &need)) != CZ_OK) return r;
  if (ws_bytes < need) return CZ_ERR_CAPACITY;
  // workspace: the batched compression's (its status word first) | the n
  // dense fields
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  unsigned char *wsb = reinterpret_cast<unsigned char *>(d_ws);
  const size_t fb = aos_field_bytes(p[0]);
  const size_t f0 = need - (size_t)n * fb;
  AosPick pick{};
  pick.n = n;
  std::vector<const void *> fields(n);
  for (int i = 0; i < n; ++i) {
    pick.comp[i] = comps[i];
    pick.out[i] = wsb + f0 + (size_t)i * fb;
    fields[i] = pick.out[i];
  }
  const unsigned long long ncells = (unsigned long long)p[0].nx * p[0].ny * p[0].nz;
  unsigned long long blocks = (ncells + 255) / 256;
  const unsigned long long cap = (unsigned long long)sm_count() * 8;
  if (blocks > cap) blocks = cap;
  if (es == 8)
    k_deinterleave<double><<<(unsigned)blocks, 256, 0, s>>>(reinterpret_cast<const double *>(d_cells), ncomp, pick,
                                                            ncells);
  else
    k_deinterleave<float><<<(unsigned)blocks, 256, 0, s>>>(reinterpret_cast<const float *>(d_cells), ncomp, pick,
                                                           ncells);
  if (cudaGetLastError() != cudaSuccess) return CZ_ERR_CUDA;
  return compress_batch_impl(n, p, fields.data(), d_outs, out_caps, d_out_bytes, wsb, f0, s);
}

// ---- the tuner's choices as JSON text
int cz_batch_knobs_export(char *buf, size_t cap, size_t *len)
{
  if (!len) return CZ_ERR_ARG;
  std::string out = "{\"format\": \"cz-batch-knobs\", \"version\": 2, \"entries\": [";
  {
    std::lock_guard<std::mutex> lock(g_knob_mu);
    for (size_t i = 0; i < g_knobs.size(); ++i) {
      char e[224];
      const BatchKnobs &k = g_knobs[i].second;
      std::snprintf(e, sizeof e,
                    "%s{\"signature\": \"%016llx\", \"s1_balanced\": %d, \"s2_div\": %d, \"place_tile\": %d, "
                    "\"slab\": %d}",
                    i ? ", " : "", g_knobs[i].first, k.s1_balanced, k.s2_div, k.place_tile, k.slab);
      out += e;
    }
  }
  out += "]}";
  *len = out.size() + 1;
  if (!buf) return CZ_OK;
  if (cap < out.size() + 1) return CZ_ERR_CAPACITY;
  std::memcpy(buf, out.c_str(), out.size() + 1);
  return CZ_OK;
}

int cz_batch_knobs_import(const char *json)
{
  if (!json) return CZ_ERR_ARG;
  const std::string t(json);
  auto ws = [&](size_t i) {
    while (i < t.size() && (t[i] == ' ' || t[i] == '\n' || t[i] == '\r' || t[i] == '\t')) ++i;
    return i;
  };
  // the value after "key": in t[b, e): a string's contents or a number's text
  auto value = [&](size_t b, size_t e, const char *key, std::string &v) {
    const std::string k = std::string("\"") + key + "\"";
    const size_t at = t.find(k, b);
    if (at == std::string::npos || at >= e) return false;
    size_t i = ws(at + k.size());
    if (i >= e || t[i] != ':') return false;
    i = ws(i + 1);
    if (i >= e) return false;
    if (t[i] == '"') {
      const size_t q = t.find('"', i + 1);
      if (q == std::string::npos || q >= e) return false;
      v = t.substr(i + 1, q - i - 1);
    } else {
      size_t j = i;
      while (j < e && (std::isdigit((unsigned char)t[j]) || t[j] == '-')) ++j;
      if (j == i) return false;
      v = t.substr(i, j - i);
    }
    return true;
  };
  std::string v;
  if (!value(0, t.size(), "format", v) || v != "cz-batch-knobs") return CZ_ERR_ARG;
  if (!value(0, t.size(), "version", v) || (v != "1" && v != "2")) return CZ_ERR_ARG;
  const bool v2 = v == "2";  // version 1 entries: look-back tiles of 128 chunks, register-resident kernels
  size_t i = t.find("\"entries\"");
  if (i == std::string::npos) return CZ_ERR_ARG;
  i = ws(i + 9);
  if (i >= t.size() || t[i] != ':') return CZ_ERR_ARG;
  i = ws(i + 1);
  if (i >= t.size() || t[i] != '[') return CZ_ERR_ARG;
  std::vector<std::pair<unsigned long long, BatchKnobs>> got;
  i = ws(i + 1);
  while (i < t.size() && t[i] != ']') {
    if (t[i] != '{') return CZ_ERR_ARG;
    const size_t e = t.find('}', i);
    if (e == std::string::npos) return CZ_ERR_ARG;
    std::string sig, s1, s2, spt = "128", ssl = "0";
    if (!value(i, e, "signature", sig) || !value(i, e, "s1_balanced", s1) || !value(i, e, "s2_div", s2))
      return CZ_ERR_ARG;
    if (v2 && (!value(i, e, "place_tile", spt) || !value(i, e, "slab", ssl))) return CZ_ERR_ARG;
    if (sig.empty() || sig.size() > 16 || sig.find_first_not_of("0123456789abcdefABCDEF") != std::string::npos)
      return CZ_ERR_ARG;
    const int b1 = std::atoi(s1.c_str()), d2 = std::atoi(s2.c_str()), pt = std::atoi(spt.c_str());
    if ((s1 != "0" && s1 != "1") || d2 < 1 || d2 > 64 || s2 != std::to_string(d2)) return CZ_ERR_ARG;
    if ((spt != "64" && spt != "128" && spt != "256") || (ssl != "0" && ssl != "1")) return CZ_ERR_ARG;
    got.push_back({std::stoull(sig, nullptr, 16), BatchKnobs{b1, d2, pt, ssl == "1" ? 1 : 0}});
    i = ws(e + 1);
    if (i < t.size() && t[i] == ',') i = ws(i + 1);
  }
  if (i >= t.size()) return CZ_ERR_ARG;  // no closing bracket
  std::lock_guard<std::mutex> lock(g_knob_mu);
  for (const auto &g : got) {
    bool found = false;
    for (auto &k : g_knobs)
      if (k.first == g.first) {
        k.second = g.second;
        found = true;
      }
    if (!found) g_knobs.push_back(g);
  }
  return CZ_OK;
}

int cz_stream_concat(int n, const void *const *h_streams, const size_t *sizes, void *h_out, size_t out_cap,
                     size_t *out_bytes)
{
  if (n < 1 || !h_streams || !sizes || !out_bytes) return CZ_ERR_ARG;
  cz_params p0{}, pr{};
  double t0 = 0, tr = 0;
  unsigned long long nz = 0, nblocks = 0, nchunks = 0, data = 0;
  double mn = 0, mx = 0;
  for (int r = 0; r < n; ++r) {
    if (!h_streams[r]) return CZ_ERR_ARG;
    const unsigned char *h = reinterpret_cast<const unsigned char *>(h_streams[r]);
    const int e = cz_read_header(h, sizes[r], r ? &pr : &p0, r ? &tr : &t0);
    if (e != CZ_OK) return e;
    const cz_params &q = r ? pr : p0;
    Shape sh;
    check(&q, &sh);
    const unsigned long long total = rd64(h + 80), db = rd64(h + 72);
    if (total > sizes[r] || sh.data0 + db != total) return CZ_ERR_CORRUPT;
    const unsigned char *h0 = reinterpret_cast<const unsigned char *>(h_streams[0]);
    if (r) {  // slabs of one field: everything but nz must agree, eps and the threshold included
      if (pr.nx != p0.nx || pr.ny != p0.ny || pr.block != p0.block || pr.dtype != p0.dtype || pr.kind != p0.kind ||
          pr.stage2 != p0.stage2 || pr.eps_mode != p0.eps_mode || pr.bound_mode != p0.bound_mode ||
          pr.flags != p0.flags ||
          std::memcmp(&tr, &t0, 8) != 0 || std::memcmp(h + 32, h0 + 32, 8) != 0 ||
          std::memcmp(h + 64, h0 + 64, 8) != 0)
        return CZ_ERR_ARG;
    }
    // min / max over the slabs (NaN, when the range was supplied, only if
    // no slab has a value)
    double a, b;
    std::memcpy(&a, h + 48, 8);
    std::memcpy(&b, h + 56, 8);
    if (r == 0) {
      mn = a;
      mx = b;
    } else {
      if (std::isnan(mn) || (!std::isnan(a) && a < mn)) mn = a;
      if (std::isnan(mx) || (!std::isnan(b) && b > mx)) mx = b;
    }
    // aggregate chunks: a slab's last group must be full unless it is the
    // last slab (the joined stream's groups are the slabs' groups)
    if (sh.G > 1 && r + 1 < n && sh.nblocks % sh.G) return CZ_ERR_ARG;
    nz += (unsigned long long)q.nz;
    nblocks += (unsigned long long)sh.nblocks;
    nchunks += (unsigned long long)sh.nchunks;
    data += db;
  }
  if (nz > 0x7FFFFFFFull || nblocks > (1ull << 30)) return CZ_ERR_ARG;
  const unsigned long long data0 = (HEADER_BYTES + 8ull * (nchunks + 1) + 15) / 16 * 16, total = data0 + data;
  *out_bytes = (size_t)total;
  if (!h_out) return CZ_OK;  // size query
  if (out_cap < total) return CZ_ERR_CAPACITY;
  unsigned char *o = reinterpret_cast<unsigned char *>(h_out);
  std::memset(o, 0, (size_t)data0);
  std::memcpy(o, h_streams[0], HEADER_BYTES);
  const int nz32 = (int)nz;
  const unsigned nb32 = (unsigned)nblocks;
  std::memcpy(o + 16, &nz32, 4);
  std::memcpy(o + 28, &nb32, 4);
  std::memcpy(o + 48, &mn, 8);
  std::memcpy(o + 56, &mx, 8);
  std::memcpy(o + 72, &data, 8);
  std::memcpy(o + 80, &total, 8);
  // offsets rebased by the data bytes of the slabs before (the exclusive
  // scan of per-rank sizes), chunks appended in rank order
  unsigned long long base = 0, chk = 0;
  for (int r = 0; r < n; ++r) {
    const unsigned char *h = reinterpret_cast<const unsigned char *>(h_streams[r]);
    cz_params q;
    double tq;
    cz_read_header(h, sizes[r], &q, &tq);
    Shape sh;
    check(&q, &sh);
    const unsigned long long db = rd64(h + 72);
    for (int b = 0; b < sh.nchunks; ++b) {
      const unsigned long long off = rd64(h + HEADER_BYTES + 8ull * b) + base;
      std::memcpy(o + HEADER_BYTES + 8ull * (chk + b), &off, 8);
    }
    std::memcpy(o + data0 + base, h + sh.data0, (size_t)db);
    base += db;
    chk += (unsigned long long)sh.nchunks;
  }
  std::memcpy(o + HEADER_BYTES + 8ull * nchunks, &base, 8);
  return CZ_OK;
}

// Not part of the ABI: FP64 throughput probe for the roofline of the FP64
// path.  Every thread runs `iters` rounds of 8 independent fused multiply-
// adds (one DFMA instruction each); the result goes to *d_sink so nothing
// is optimised away.  DFMA instructions = grid * threads * iters * 8.
int czi_fp64_probe(int grid, int threads, int iters, double *d_sink, void *stream)
{
  if (grid < 1 || threads < 32 || threads > 1024 || iters < 1 || !d_sink) return CZ_ERR_ARG;
  k_fp64_probe<<<grid, threads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(iters, d_sink);
  return cudaGetLastError() == cudaSuccess ? CZ_OK : CZ_ERR_CUDA;
}

// Not part of the ABI: runs k_wait_probe (see there) on `stream`.
// which 0: `tiles` (1..1024) warps, d_state = `tiles` zeroed u64 words,
// d_out = `tiles` u64; which 1: one CTA of `tiles` (32..1024, a multiple
// of 32) threads, d_out = `tiles` u64.  d_status: a zeroed u32.
int czi_wait_probe(int which, int tiles, int skip, unsigned limit, void *d_status, void *d_state, void *d_out,
                   void *stream)
{
  if ((which != 0 && which != 1) || !d_status || !d_out || limit < 1 || limit > (1u << 20)) return CZ_ERR_ARG;
  if (which == 0 && (tiles < 1 || tiles > 1024 || !d_state)) return CZ_ERR_ARG;
  if (which == 1 && (tiles < 32 || tiles > 1024 || tiles % 32)) return CZ_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (which == 0)
    k_wait_probe<<<tiles, 32, 0, s>>>(0, skip, limit, reinterpret_cast<unsigned *>(d_status),
                                      reinterpret_cast<unsigned long long *>(d_state),
                                      reinterpret_cast<unsigned long long *>(d_out));
  else
    k_wait_probe<<<1, tiles, 0, s>>>(1, skip, limit, reinterpret_cast<unsigned *>(d_status), nullptr,
                                     reinterpret_cast<unsigned long long *>(d_out));
  return cudaGetLastError() == cudaSuccess ? CZ_OK : CZ_ERR_CUDA;
}

// Not part of the ABI: the host link's copy rate as plain cudaMemcpyAsync
// calls see it (context for the end-to-end figure).  `reps` copies of
// `bytes` between the host buffer h (pinned by the caller) and the device
// buffer d, host to device (dir 0) or device to host (dir 1), timed with
// events on `stream`; *ms receives the total time.  Synchronises.
int czi_link_probe(void *h, void *d, size_t bytes, int reps, int dir, void *stream, float *ms)
{
  if (!h || !d || !ms || bytes == 0 || reps < 1 || (dir != 0 && dir != 1)) return CZ_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return CZ_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return CZ_ERR_CUDA;
  }
  int r = CZ_OK;
  if (cudaEventRecord(e0, s) != cudaSuccess) r = CZ_ERR_CUDA;
  for (int i = 0; i < reps && r == CZ_OK; ++i) {
    const cudaError_t e = dir == 0 ? cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, s)
                                   : cudaMemcpyAsync(h, d, bytes, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) r = CZ_ERR_CUDA;
  }
  if (r == CZ_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
    r = CZ_ERR_CUDA;
  if (r == CZ_OK && cudaEventElapsedTime(ms, e0, e1) != cudaSuccess) r = CZ_ERR_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return r;
}

// Not part of the ABI: which decoder later calls use (tests and timing
// compare the two): 0 = one CTA per block everywhere (the default), 1 = the
// half-block decoder where the lane has one (FP32, blocks of edge 16 and 32).
int czi_set_decoder(int mode)
{
  if (mode != 0 && mode != 1) return CZ_ERR_ARG;
  __atomic_store_n(&g_decoder_mode, mode, __ATOMIC_RELAXED);
  return CZ_OK;
}

// Not part of the ABI: cz_compress_batch with one knob setting forced on
// every group (tests: streams must not depend on it): s1_balanced (0, 1),
// s2_div (1, 2), place_tile (64, 128, 256), slab (0, 1; ignored where the
// lane has no slab alternative).  d_ws as for cz_compress_batch.
int czi_compress_batch_knobs(int n, const cz_params *p, const void *const *d_fields, void *const *d_outs,
                             const size_t *out_caps, uint64_t *d_out_bytes, void *d_ws, size_t ws_bytes,
                             void *stream, int s1_balanced, int s2_div, int place_tile, int slab)
{
  if ((s1_balanced != 0 && s1_balanced != 1) || (s2_div != 1 && s2_div != 2) ||
      (place_tile != 64 && place_tile != 128 && place_tile != 256) || (slab != 0 && slab != 1))
    return CZ_ERR_ARG;
  const BatchKnobs kn{s1_balanced, s2_div, place_tile, slab};
  return compress_batch_impl(n, p, d_fields, d_outs, out_caps, d_out_bytes, d_ws, ws_bytes,
                             reinterpret_cast<cudaStream_t>(stream), &kn);
}

// Not part of the ABI: the strict-bound divisor C of (kind, B), for tests.
double czi_synthesis_norm(int kind, int block)
{
  if (kind < CZ_W4 || kind > CZ_W3AI || (block != 8 && block != 16 && block != 32 && block != 64)) return -1.0;
  cz_params p{};
  p.kind = kind;
  p.block = block;
  p.bound_mode = CZ_BOUND_STRICT;
  return threshold_divisor(&p);
}

// Not part of the ABI: cz_compress with four CUDA events recorded on
// `stream` around its kernels (before the stage kernel, after it, after
// stage 2, after the chunk copy), for timing the kernels one by one.
int czi_compress_marked(const cz_params *p, const void *d_field, void *d_out, size_t out_cap,
                        uint64_t *d_out_bytes, void *d_ws, size_t ws_bytes, void *stream,
                        void *const *events)
{
  if (!events) return CZ_ERR_ARG;
  cudaEvent_t ev[4];
  for (int i = 0; i < 4; ++i) {
    if (!events[i]) return CZ_ERR_ARG;
    ev[i] = reinterpret_cast<cudaEvent_t>(events[i]);
  }
  return compress_impl(p, d_field, d_out, out_cap, d_out_bytes, d_ws, ws_bytes, stream, ev);
}

int cz_read_header(const void *h_in, size_t n, cz_params *p, double *t_used)
{
  if (!h_in || !p || n < (size_t)HEADER_BYTES) return CZ_ERR_ARG;
  const unsigned char *h = reinterpret_cast<const unsigned char *>(h_in);
  unsigned magic;
  unsigned short ver, hb;
  std::memcpy(&magic, h, 4);
  std::memcpy(&ver, h + 4, 2);
  std::memcpy(&hb, h + 6, 2);
  if (magic != MAGIC || ver != 1 || hb != HEADER_BYTES) return CZ_ERR_CORRUPT;
  cz_params q{};
  std::memcpy(&q.nx, h + 8, 4);
  std::memcpy(&q.ny, h + 12, 4);
  std::memcpy(&q.nz, h + 16, 4);
  q.block = h[20];
  q.dtype = h[21];
  q.kind = h[22];
  q.stage2 = h[23];
  q.eps_mode = h[24];
  q.bound_mode = h[26];
  q.flags = h[27] & (CZ_FLAG_FAST | CZ_FLAG_ZERO4 | CZ_FLAG_ZERO8 | GROUP_FLAGS);
  std::memcpy(&q.eps, h + 32, 8);
  std::memcpy(&q.range, h + 64, 8);
  if (std::isnan(q.range)) return CZ_ERR_CORRUPT;
  if (check(&q, nullptr) != CZ_OK) return CZ_ERR_CORRUPT;
  unsigned nb;
  std::memcpy(&nb, h + 28, 4);
  if ((long long)nb != (long long)(q.nx / q.block) * (q.ny / q.block) * (q.nz / q.block)) return CZ_ERR_CORRUPT;
  *p = q;
  if (t_used) std::memcpy(t_used, h + 40, 8);
  return CZ_OK;
}

namespace {

// Decompress the whole field (ids == nullptr) or the n blocks ids[0..n) into
// n consecutive B^3 tiles.  The decoded blocks are numbered 0..n-1 in the
// workspace; with tiles the block grid is 1 x 1 x n, so block i lands at
// z = i B of the B x B x nB tile array.
int decompress_impl(const void *d_in, size_t in_bytes, const void *h_header, const int32_t *ids, int n,
                    void *d_out, size_t out_cap, void *d_ws, size_t ws_bytes, void *stream,
                    const cudaEvent_t *marks = nullptr)
{
  const NvtxRange nvtx(ids ? "cz_decompress_blocks" : "cz_decompress");
  if (!d_in || !d_out || !d_ws) return CZ_ERR_ARG;
  if (((uintptr_t)d_in % 16) || ((uintptr_t)d_out % 16) || ((uintptr_t)d_ws % 16)) return CZ_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  unsigned char hb[HEADER_BYTES];
  if (in_bytes < (size_t)HEADER_BYTES) return CZ_ERR_CORRUPT;
  if (h_header) {
    std::memcpy(hb, h_header, HEADER_BYTES);
  } else {
    if (cudaMemcpyAsync(hb, d_in, HEADER_BYTES, cudaMemcpyDeviceToHost, s) != cudaSuccess) return CZ_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return CZ_ERR_CUDA;
  }
  cz_params p;
  int r = cz_read_header(hb, HEADER_BYTES, &p, nullptr);
  if (r != CZ_OK) return r;
  Shape sh;
  check(&p, &sh);
  const unsigned long long total = rd64(hb + 80), data_bytes = rd64(hb + 72);
  if (total > in_bytes || sh.data0 + data_bytes != total) return CZ_ERR_CORRUPT;
  const int nchunks = sh.nblocks;
  // the decoded blocks: the whole grid, or n tiles stacked along z
  cz_params q = p;
  Shape dsh = sh;
  if (ids) {
    if (n < 0) return CZ_ERR_ARG;
    if (n == 0) return CZ_OK;
    if ((long long)n * p.block > INT32_MAX) return CZ_ERR_ARG;
    q.nx = q.ny = p.block;
    q.nz = n * p.block;
    dsh.nbx = dsh.nby = 1;
    dsh.nbz = n;
    dsh.nblocks = n;
  }
  if ((size_t)q.nx * q.ny * q.nz * sh.es > out_cap) return CZ_ERR_CAPACITY;
  const Lanes L = lanes_for(p);
  // workspace: header | block table (nnz, bad flag) | list of the large
  // chunks | one staging slot per decoded block for the stage-2 payloads
  // (within cz_workspace_size)
  const size_t slot = (size_t)L.slot_bytes();
  size_t scr = 0;
  const size_t need = dec_ws_need(&p, dsh, &scr);
  if (ws_bytes < need) return CZ_ERR_CAPACITY;
  if (cudaMemsetAsync(d_ws, 0, WS_HDR, s) != cudaSuccess) return CZ_ERR_CUDA;
  unsigned char *wsb = reinterpret_cast<unsigned char *>(d_ws);
  InvArgs a{};
  a.in = reinterpret_cast<const unsigned char *>(d_in);
  a.field = d_out;
  a.ws = d_ws;
  a.in_bytes = total;
  a.data0 = sh.data0;
  a.nx = q.nx;
  a.ny = q.ny;
  a.nz = q.nz;
  a.nbx = dsh.nbx;
  a.nby = dsh.nby;
  a.nbz = dsh.nbz;
  a.nblocks = dsh.nblocks;
  a.stage2 = p.stage2;
  a.ids = ids;
  a.nchunks = nchunks;
  a.table = reinterpret_cast<const unsigned long long *>(wsb + WS_HDR);
  a.staging = wsb + dec_slots_off(dsh);
  a.slot = slot;
  UnArgs ua{};
  ua.in = a.in;
  ua.staging = wsb + dec_slots_off(dsh);
  ua.ws = d_ws;
  ua.biglist = reinterpret_cast<int *>(wsb + WS_HDR + table_bytes(dsh));
  ua.scratch = wsb + scr;
  ua.table = reinterpret_cast<unsigned long long *>(wsb + WS_HDR);
  ua.ids = ids;
  ua.nchunks = nchunks;
  ua.in_bytes = total;
  ua.data0 = sh.data0;
  ua.slot = slot;
  ua.nblocks = dsh.nblocks;
  ua.group = sh.G;
  int ugrid[3];
  if (sh.G > 1) {
    // the group decoder tiers: one item per group (whole field) or per
    // requested block
    ua.hcap = group_hcap(&p, sh);
    const long long items = ids ? n : sh.nchunks;
    ugrid[0] = group_grid(&p, 3, ua.hcap, items);
    ugrid[1] = group_grid(&p, 4, ua.hcap, items);
    ugrid[2] = group_grid(&p, 5, ua.hcap, dsh.nblocks);  // as dec_ws_need sized the scratch
  } else {
    ugrid[0] = grid_for(&p, dsh, 4);
    ugrid[1] = grid_for(&p, dsh, 5);
    ugrid[2] = 0;
  }
  a.decoder = decoder_of(p);
  CUtensorMap om;
  if (!make_tile_map(&om, &q, d_out, a.decoder == 1)) return CZ_ERR_CUDA;
  return L.decompress(p.kind, &om, &a, &ua, grid_for(&p, dsh, 1), ugrid, marks, s) == cudaSuccess
             ? CZ_OK
             : CZ_ERR_CUDA;
}

}  // namespace

// Not part of the ABI: cz_decompress with one CUDA event recorded right before the decode kernel
// (after the stage-2 inverse launches), for timing the kernels one by one.
int czi_decompress_marked(const void *d_in, size_t in_bytes, const void *h_header, void *d_field, size_t field_cap,
                          void *d_ws, size_t ws_bytes, void *stream, void *const *events)
{
  if (!events || !events[0]) return CZ_ERR_ARG;
  cudaEvent_t ev[1] = {reinterpret_cast<cudaEvent_t>(events[0])};
  return decompress_impl(d_in, in_bytes, h_header, nullptr, 0, d_field, field_cap, d_ws, ws_bytes, stream, ev);
}


int cz_decompress(const void *d_in, size_t in_bytes, const void *h_header, void *d_field,
                  size_t field_cap, void *d_ws, size_t ws_bytes, void *stream)
{
  return decompress_impl(d_in, in_bytes, h_header, nullptr, 0, d_field, field_cap, d_ws, ws_bytes, stream);
}

int cz_decompress_blocks_workspace_size(const cz_params *p, int n, size_t *bytes)
{
  Shape sh;
  const int r = check(p, &sh);
  if (r != CZ_OK || !bytes || n < 0) return r ? r : CZ_ERR_ARG;
  sh.nbx = sh.nby = 1;
  sh.nbz = n;
  sh.nblocks = n;
  *bytes = dec_ws_need(p, sh, nullptr);
  return CZ_OK;
}

int cz_decompress_blocks(const void *d_in, size_t in_bytes, const void *h_header, const int32_t *d_ids, int n,
                         void *d_tiles, size_t tiles_cap, void *d_ws, size_t ws_bytes, void *stream)
{
  if (!d_ids && n > 0) return CZ_ERR_ARG;
  if (!d_ids) return n == 0 ? CZ_OK : CZ_ERR_ARG;
  return decompress_impl(d_in, in_bytes, h_header, d_ids, n, d_tiles, tiles_cap, d_ws, ws_bytes, stream);
}

int cz_status(const void *d_ws, void *stream)
{
  if (!d_ws) return CZ_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  unsigned st = 0;
  if (cudaMemcpyAsync(&st, d_ws, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess) return CZ_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return CZ_ERR_CUDA;
  return (int)st;
}

const char *cz_strerror(int code)
{
  switch (code) {
    case CZ_OK: return "ok";
    case CZ_ERR_ARG: return "invalid argument or unsupported combination";
    case CZ_ERR_CAPACITY: return "buffer too small";
    case CZ_ERR_CORRUPT: return "corrupt or inconsistent stream";
    case CZ_ERR_TIMEOUT: return "device-side wait timed out";
    case CZ_ERR_CUDA: return "CUDA runtime error";
    case CZ_ERR_BUDGET: return "request exceeds the memory budget";
    default: return "unknown error";
  }
}

static int dense(const cz_params *p, const void *src, void *dst, int fwd, void *stream)
{
  Shape sh;
  const int r = check(p, &sh);
  if (r != CZ_OK) return r;
  if (!src || !dst) return CZ_ERR_ARG;
  if (((uintptr_t)src % 16) || ((uintptr_t)dst % 16)) return CZ_ERR_ARG;
  DenseArgs a{};
  a.src = src;
  a.dst = dst;
  a.nx = p->nx;
  a.ny = p->ny;
  a.nz = p->nz;
  a.nbx = sh.nbx;
  a.nby = sh.nby;
  a.nbz = sh.nbz;
  const Lanes L = lanes_for(*p);
  return L.dense(p->kind, fwd, &a, sh.nblocks, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess
             ? CZ_OK
             : CZ_ERR_CUDA;
}

int cz_forward_dense(const cz_params *p, const void *d_field, void *d_coef, void *stream)
{
  return dense(p, d_field, d_coef, 1, stream);
}

int cz_inverse_dense(const cz_params *p, const void *d_coef, void *d_field, void *stream)
{
  return dense(p, d_coef, d_field, 0, stream);
}

}  // extern "C"
