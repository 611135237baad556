// cz_inst.cu -- kernel instantiations for one (element type, block edge).
// Built once per combination with -DCZ_T=float|double -DCZ_TNAME=f32|f64
// -DCZ_B=8|16|32|64 (and once more with -DCZ_FAST for the contracting
// build, which serves W3ai only) so the heavily unrolled kernels compile in
// parallel.
#include <cuda.h>
#include <cuda_runtime.h>

#include "cz_compress.cuh"
#include "cz_group.cuh"
#include "cz_half.cuh"
#include "cz_launch.h"
#include "cz_pair.cuh"
#include "cz_slab.cuh"

#ifndef CZ_T
#error "CZ_T must be defined"
#endif
#ifndef CZ_B
#error "CZ_B must be defined"
#endif

using namespace czp;

namespace {

using G = G2<CZ_T, CZ_B>;
using SGi = SG<CZ_T, CZ_B>;  // slab geometry (used only when G::SLAB)
// lanes with the half-block decoder (FP32 blocks of edge 16 and 32)
constexpr bool HAS_HALF = sizeof(CZ_T) == 4 && (CZ_B == 16 || CZ_B == 32);
// lanes where the batched stage kernel can also be the slab kernel (the
// block in global scratch) instead of the register-resident one: the tuner
// picks (FP32 32^3)
constexpr bool HAS_SLAB_ALT = !G::SLAB && SGi::OK;

// raise the dynamic shared-memory limit of kernel KERN once per device
template <auto KERN>
cudaError_t prepare(int smem)
{
  static unsigned long long done_mask = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (__atomic_load_n(&done_mask, __ATOMIC_ACQUIRE) & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(KERN, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) __atomic_fetch_or(&done_mask, bit, __ATOMIC_ACQ_REL);
  return e;
}

// one stage-2 launch (BIG: the large payloads, 512-thread CTAs); KIND 0:
// k_stage2, 1: its speculative variant, 2: k_stage2_listed
template <auto KERN, bool BIG>
cudaError_t stage2_go(const S2Args &sa, int grid, cudaStream_t s)
{
  constexpr int sm = BIG ? G::SMEM_S2B : G::SMEM_S2;
  cudaError_t e = prepare<KERN>(sm);
  if (e != cudaSuccess) return e;
  KERN<<<grid, BIG ? 512 : 128, sm, s>>>(sa);
  return cudaGetLastError();
}
template <bool BIG, int KIND>
cudaError_t stage2_one(const S2Args &sa, int grid, cudaStream_t s)
{
  if constexpr (KIND == 2)
    return stage2_go<k_stage2_listed<CZ_T, CZ_B, BIG>, BIG>(sa, grid, s);
  else
    return stage2_go<k_stage2<CZ_T, CZ_B, BIG, KIND == 1>, BIG>(sa, grid, s);
}

// stage 2 on every slot (small and large payloads).  SPEC (speculative
// thresholds): with block edges up to 16 the slots to test are listed
// first and taken after the others by k_stage2_listed; with 32 they are
// tested within k_stage2, and the listed slots that hold a value to drop
// are refined after.  (Each measured the faster for its block edges.)
template <bool SPEC>
cudaError_t stage2_launch(const S2Args &sa, int grid2, int grid3, cudaStream_t s)
{
  constexpr bool LIST = SPEC && CZ_B <= 16;
  constexpr int K = SPEC && !LIST ? 1 : 0;
  if constexpr (LIST) {
    const int gl = (sa.nblocks + 255) / 256 < grid2 ? (sa.nblocks + 255) / 256 : grid2;
    k_spec_list<CZ_T><<<gl, 256, 0, s>>>(sa);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = stage2_one<false, K>(sa, grid2, s);
  if (e != cudaSuccess) return e;
  if constexpr (G::SLAB) {
    constexpr int sm = 4 * G::NBWMAX * 4;
    e = prepare<k_stage2_huge<CZ_T, CZ_B>>(sm);
    if (e != cudaSuccess) return e;
    k_stage2_huge<CZ_T, CZ_B><<<grid3, 512, sm, s>>>(sa);
    e = cudaGetLastError();
  } else {
    if constexpr (G::HAS_BIG) {
      if ((e = stage2_one<true, K>(sa, grid3, s)) != cudaSuccess) return e;
    }
    if constexpr (LIST) {
      if ((e = stage2_one<false, 2>(sa, grid2, s)) != cudaSuccess) return e;
      if constexpr (G::HAS_BIG) e = stage2_one<true, 2>(sa, grid3, s);
    } else if constexpr (SPEC) {
      e = prepare<k_stage2_refine<CZ_T, CZ_B>>(G::SMEM_S2B);
      if (e != cudaSuccess) return e;
      k_stage2_refine<CZ_T, CZ_B><<<grid3, 512, G::SMEM_S2B, s>>>(sa);
      e = cudaGetLastError();
    }
  }
  return e;
}

// stage 2, when enabled (a template, so that only the kernels of this lane
// are instantiated); the speculative variant exists only for the lanes
// whose stage kernel keeps the block in registers
template <int = 0>
cudaError_t stage2_k(const S2Args &sa, int stage2, int grid2, int grid3, cudaStream_t s)
{
  if (!stage2) return cudaSuccess;
  if constexpr (!G::SLAB) {
    if (sa.spec) return stage2_launch<true>(sa, grid2, grid3, s);
  }
  return stage2_launch<false>(sa, grid2, grid3, s);
}

// aggregate chunks: the three tiers of the group coder over the raw slots
// (ggrid: their grids)
template <int = 0>
cudaError_t group_k(const GroupArgs &ga, const int *ggrid, cudaStream_t s)
{
  if (ga.hcap <= 0 || ga.hcap > GROUP_MAX_BYTES || ga.hcap % 128) return cudaErrorInvalidValue;
  cudaError_t e = prepare<k_group2<CZ_T, CZ_B, 0>>(GT<0>::SMEM);
  if (e != cudaSuccess) return e;
  k_group2<CZ_T, CZ_B, 0><<<ggrid[0], GT<0>::NT, GT<0>::SMEM, s>>>(ga);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = prepare<k_group2<CZ_T, CZ_B, 1>>(GT<1>::SMEM)) != cudaSuccess) return e;
  k_group2<CZ_T, CZ_B, 1><<<ggrid[1], GT<1>::NT, GT<1>::SMEM, s>>>(ga);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = prepare<k_group_huge<CZ_T, CZ_B>>(GROUP_HSMEM)) != cudaSuccess) return e;
  k_group_huge<CZ_T, CZ_B><<<ggrid[2], 512, ga.hcap / 8, s>>>(ga);  // four bitmap arrays of hcap / 128 words
  return cudaGetLastError();
}

// ga: aggregate chunks (the stage kernel then writes raw slots, the group
// coders replace stage 2, and pa describes the group table); else null
template <int KIND>
cudaError_t compress_k(const CUtensorMap &tm, const FwdArgs &a, const S2Args &sa, const PlaceArgs &pa, int grid,
                       int grid2, int grid3, const GroupArgs *ga, const int *ggrid, const cudaEvent_t *marks,
                       cudaStream_t s)
{
  cudaError_t e;
  StageMaps<1> maps{};
  maps.tm[0] = tm;
  if constexpr (G::SLAB) {
    e = prepare<k_stage1_slab<CZ_T, CZ_B, KIND, 1>>(SGi::SMEM);
    if (e != cudaSuccess) return e;
    if (marks && (e = cudaEventRecord(marks[0], s)) != cudaSuccess) return e;
    k_stage1_slab<CZ_T, CZ_B, KIND, 1><<<grid, SGi::NT, SGi::SMEM, s>>>(maps, a);
  } else if (a.spec) {  // speculative thresholds
    e = prepare<k_stage1<CZ_T, CZ_B, KIND, 1, true>>(G::SMEM_C);
    if (e != cudaSuccess) return e;
    if (marks && (e = cudaEventRecord(marks[0], s)) != cudaSuccess) return e;
    k_stage1<CZ_T, CZ_B, KIND, 1, true><<<grid, G::NT, G::SMEM_C, s>>>(maps, a);
  } else {
    e = prepare<k_stage1<CZ_T, CZ_B, KIND, 1>>(G::SMEM_C);
    if (e != cudaSuccess) return e;
    if (marks && (e = cudaEventRecord(marks[0], s)) != cudaSuccess) return e;
    k_stage1<CZ_T, CZ_B, KIND, 1><<<grid, G::NT, G::SMEM_C, s>>>(maps, a);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (marks && (e = cudaEventRecord(marks[1], s)) != cudaSuccess) return e;
  if (ga)
    e = group_k(*ga, ggrid, s);
  else
    e = stage2_k(sa, pa.stage2, grid2, grid3, s);
  if (e != cudaSuccess) return e;
  if (marks && (e = cudaEventRecord(marks[2], s)) != cudaSuccess) return e;
  const int tiles = (pa.nblocks + PLACE_TILE - 1) / PLACE_TILE;
  k_place<CZ_T><<<tiles, PLACE_TILE, 0, s>>>(pa);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_copy<CZ_T><<<(pa.nblocks + 7) / 8, 256, 0, s>>>(pa);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (marks && (e = cudaEventRecord(marks[3], s)) != cudaSuccess) return e;
  return cudaGetLastError();
}

// place_tile: chunks per look-back tile (64, 128 or 256); slab: the slab
// stage kernel where the lane also has the register-resident one
template <int KIND>
cudaError_t compress_batch_k(const StageMaps<MAXF> &maps, const FwdArgs &a, const S2Args &sa, const BatchOut &bo,
                             const PlaceArgs &pa, int grid, int grid2, int grid3, int tiles, int place_tile, int slab,
                             cudaStream_t s)
{
  cudaError_t e;
  if (place_tile != 64 && place_tile != 128 && place_tile != 256) return cudaErrorInvalidValue;
  if (slab && !G::SLAB && !HAS_SLAB_ALT) return cudaErrorInvalidValue;
  if constexpr (G::SLAB || HAS_SLAB_ALT) {
    if (G::SLAB || slab) {
      e = prepare<k_stage1_slab<CZ_T, CZ_B, KIND, MAXF>>(SGi::SMEM);
      if (e != cudaSuccess) return e;
      k_stage1_slab<CZ_T, CZ_B, KIND, MAXF><<<grid, SGi::NT, SGi::SMEM, s>>>(maps, a);
    }
  }
  if constexpr (!G::SLAB) {
    if (!slab) {
      e = prepare<k_stage1<CZ_T, CZ_B, KIND, MAXF>>(G::SMEM_C);
      if (e != cudaSuccess) return e;
      k_stage1<CZ_T, CZ_B, KIND, MAXF><<<grid, G::NT, G::SMEM_C, s>>>(maps, a);
    }
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if ((e = stage2_k(sa, pa.stage2, grid2, grid3, s)) != cudaSuccess) return e;
  if (place_tile == 64)
    k_place_multi<CZ_T, 64><<<tiles, 64, 0, s>>>(bo, pa);
  else if (place_tile == 128)
    k_place_multi<CZ_T, 128><<<tiles, 128, 0, s>>>(bo, pa);
  else
    k_place_multi<CZ_T, 256><<<tiles, 256, 0, s>>>(bo, pa);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_copy_multi<CZ_T><<<(pa.nblocks + 7) / 8, 256, 0, s>>>(bo, pa);
  return cudaGetLastError();
}

// marks (optional): marks[0] is recorded right before the decode kernel
template <int KIND>
cudaError_t decompress_k(const CUtensorMap &om, const InvArgs &a, const UnArgs &ua, int grid, const int *ugrid,
                         const cudaEvent_t *marks, cudaStream_t s)
{
  const int gridu = ugrid[0], gridub = ugrid[1];
  cudaError_t e;
  if (a.stage2 && ua.group > 1) {
    // aggregate chunks: the three tiers of the group decoder
    e = prepare<k_gunstage<CZ_T, CZ_B, 0>>(GT<0>::USMEM);
    if (e != cudaSuccess) return e;
    k_gunstage<CZ_T, CZ_B, 0><<<ugrid[0], GT<0>::NT, GT<0>::USMEM, s>>>(ua);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = prepare<k_gunstage<CZ_T, CZ_B, 1>>(GT<1>::USMEM)) != cudaSuccess) return e;
    k_gunstage<CZ_T, CZ_B, 1><<<ugrid[1], GT<1>::NT, GT<1>::USMEM, s>>>(ua);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_gunstage<CZ_T, CZ_B, 2><<<ugrid[2], GT<2>::NT, GT<2>::USMEM, s>>>(ua);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  } else if (a.stage2) {
    e = prepare<k_unstage<CZ_T, CZ_B, false>>(G::SMEM_U);
    if (e != cudaSuccess) return e;
    k_unstage<CZ_T, CZ_B, false><<<gridu, 128, G::SMEM_U, s>>>(ua);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if constexpr (G::HAS_BIG) {
      e = prepare<k_unstage<CZ_T, CZ_B, true>>(G::SMEM_UB);
      if (e != cudaSuccess) return e;
      k_unstage<CZ_T, CZ_B, true><<<gridub, 512, G::SMEM_UB, s>>>(ua);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  if constexpr (G::SLAB) {
    e = prepare<k_decompress_slab<CZ_T, CZ_B, KIND>>(SGi::SMEM);
    if (e != cudaSuccess) return e;
    if (marks && (e = cudaEventRecord(marks[0], s)) != cudaSuccess) return e;
    k_decompress_slab<CZ_T, CZ_B, KIND><<<grid, SGi::NT, SGi::SMEM, s>>>(a);
  } else if constexpr (HAS_HALF) {
    if (a.decoder == 1) {
      using GHi = GH<CZ_T, CZ_B>;
      if (grid < 2 || (grid & 1)) return cudaErrorInvalidValue;  // a CTA keeps its half: an even grid
      e = prepare<k_decompress_h<CZ_T, CZ_B, KIND>>(GHi::SMEM);
      if (e != cudaSuccess) return e;
      if (marks && (e = cudaEventRecord(marks[0], s)) != cudaSuccess) return e;
      k_decompress_h<CZ_T, CZ_B, KIND><<<grid, GHi::NT, GHi::SMEM, s>>>(om, a);
    } else {
      e = prepare<k_decompress2<CZ_T, CZ_B, KIND>>(G::SMEM_D);
      if (e != cudaSuccess) return e;
      if (marks && (e = cudaEventRecord(marks[0], s)) != cudaSuccess) return e;
      k_decompress2<CZ_T, CZ_B, KIND><<<grid, G::NT, G::SMEM_D, s>>>(om, a);
    }
  } else {
    e = prepare<k_decompress2<CZ_T, CZ_B, KIND>>(G::SMEM_D);
    if (e != cudaSuccess) return e;
    if (marks && (e = cudaEventRecord(marks[0], s)) != cudaSuccess) return e;
    k_decompress2<CZ_T, CZ_B, KIND><<<grid, G::NT, G::SMEM_D, s>>>(om, a);
  }
  return cudaGetLastError();
}

template <int KIND, bool FWD>
cudaError_t dense_k(const DenseArgs &a, int nblocks, cudaStream_t s)
{
  cudaError_t e;
  if constexpr (G::SLAB) {
    e = prepare<k_dense_slab<CZ_T, CZ_B, KIND, FWD>>(SGi::SMEM);
    if (e != cudaSuccess) return e;
    k_dense_slab<CZ_T, CZ_B, KIND, FWD><<<nblocks, SGi::NT, SGi::SMEM, s>>>(a);
  } else {
    e = prepare<k_dense2<CZ_T, CZ_B, KIND, FWD>>(G::SMEM_DN0);
    if (e != cudaSuccess) return e;
    k_dense2<CZ_T, CZ_B, KIND, FWD><<<nblocks, G::NT, G::SMEM_DN0, s>>>(a);
  }
  return cudaGetLastError();
}

template <int KIND>
int occupancy_c()
{
  int n = 0;
  if constexpr (G::SLAB) {
    if (prepare<k_stage1_slab<CZ_T, CZ_B, KIND, 1>>(SGi::SMEM) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_stage1_slab<CZ_T, CZ_B, KIND, 1>, SGi::NT,
                                                      SGi::SMEM) != cudaSuccess)
      return 0;
  } else {
    if (prepare<k_stage1<CZ_T, CZ_B, KIND, 1>>(G::SMEM_C) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_stage1<CZ_T, CZ_B, KIND, 1>, G::NT, G::SMEM_C) !=
        cudaSuccess)
      return 0;
  }
  return n;
}

template <bool BIG>
int occupancy_s2()
{
  if constexpr (BIG && G::SLAB) {
    constexpr int sm = 4 * G::NBWMAX * 4;
    if (prepare<k_stage2_huge<CZ_T, CZ_B>>(sm) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_stage2_huge<CZ_T, CZ_B>, 512, sm) != cudaSuccess)
      return 0;
    return n;
  } else {
    constexpr int sm = BIG ? G::SMEM_S2B : G::SMEM_S2;
    if (prepare<k_stage2<CZ_T, CZ_B, BIG>>(sm) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_stage2<CZ_T, CZ_B, BIG>, BIG ? 512 : 128, sm) !=
        cudaSuccess)
      return 0;
    return n;
  }
}

template <bool BIG>
int occupancy_u()
{
  constexpr int sm = BIG ? G::SMEM_UB : G::SMEM_U;
  if (prepare<k_unstage<CZ_T, CZ_B, BIG>>(sm) != cudaSuccess) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_unstage<CZ_T, CZ_B, BIG>, BIG ? 512 : 128, sm) !=
      cudaSuccess)
    return 0;
  return n;
}

// group kernels (which): coder tiers 0, 1, 2 (0, 1, 2), decoder tiers 0,
// 1, 2 (3, 4, 5); hcap bytes of the largest group payload
template <auto KERN>
int occ_of(int nt, int smem, bool raise)
{
  int n = 0;
  if (raise && prepare<KERN>(smem) != cudaSuccess) return 0;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, KERN, nt, smem) == cudaSuccess ? n : 0;
}

int occupancy_g(int which, int hcap)
{
  switch (which) {
    case 0: return occ_of<k_group2<CZ_T, CZ_B, 0>>(GT<0>::NT, GT<0>::SMEM, true);
    case 1: return occ_of<k_group2<CZ_T, CZ_B, 1>>(GT<1>::NT, GT<1>::SMEM, true);
    case 2:
      if (prepare<k_group_huge<CZ_T, CZ_B>>(GROUP_HSMEM) != cudaSuccess) return 0;
      return occ_of<k_group_huge<CZ_T, CZ_B>>(512, hcap / 8, false);
    case 3: return occ_of<k_gunstage<CZ_T, CZ_B, 0>>(GT<0>::NT, GT<0>::USMEM, true);
    case 4: return occ_of<k_gunstage<CZ_T, CZ_B, 1>>(GT<1>::NT, GT<1>::USMEM, true);
    default: return occ_of<k_gunstage<CZ_T, CZ_B, 2>>(GT<2>::NT, GT<2>::USMEM, false);
  }
}

template <int KIND>
int occupancy_slab_alt()
{
  if constexpr (HAS_SLAB_ALT) {
    int n = 0;
    if (prepare<k_stage1_slab<CZ_T, CZ_B, KIND, MAXF>>(SGi::SMEM) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_stage1_slab<CZ_T, CZ_B, KIND, MAXF>, SGi::NT,
                                                      SGi::SMEM) != cudaSuccess)
      return 0;
    return n;
  } else {
    return 0;
  }
}

template <int KIND>
int occupancy_h()
{
  if constexpr (HAS_HALF) {
    using GHi = GH<CZ_T, CZ_B>;
    int n = 0;
    if (prepare<k_decompress_h<CZ_T, CZ_B, KIND>>(GHi::SMEM) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_decompress_h<CZ_T, CZ_B, KIND>, GHi::NT, GHi::SMEM) !=
        cudaSuccess)
      return 0;
    return n;
  } else {
    return 0;
  }
}

template <int KIND>
int occupancy_d()
{
  int n = 0;
  if constexpr (G::SLAB) {
    if (prepare<k_decompress_slab<CZ_T, CZ_B, KIND>>(SGi::SMEM) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_decompress_slab<CZ_T, CZ_B, KIND>, SGi::NT,
                                                      SGi::SMEM) != cudaSuccess)
      return 0;
    return n;
  } else {
    if (prepare<k_decompress2<CZ_T, CZ_B, KIND>>(G::SMEM_D) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_decompress2<CZ_T, CZ_B, KIND>, G::NT, G::SMEM_D) !=
        cudaSuccess)
      return 0;
    return n;
  }
}

}  // namespace

#define CZ_CAT2(a, b) a##b
#define CZ_CAT(a, b) CZ_CAT2(a, b)
#ifdef CZ_FAST
#define CZ_SUFFIX CZ_CAT(CZ_CAT(CZ_CAT(CZ_TNAME, _b), CZ_B), _fast)
#else
#define CZ_SUFFIX CZ_CAT(CZ_CAT(CZ_TNAME, _b), CZ_B)
#endif

extern "C" cudaError_t CZ_CAT(czl_compress_, CZ_SUFFIX)(int kind, const CUtensorMap *tm, const FwdArgs *a,
                                                         const S2Args *sa, const PlaceArgs *pa, int grid,
                                                         int grid2, int grid3, const GroupArgs *ga,
                                                         const int *ggrid, const cudaEvent_t *marks, cudaStream_t s)
{
#ifdef CZ_FAST
  if (kind != W3AI) return cudaErrorInvalidValue;
  return compress_k<W3AI>(*tm, *a, *sa, *pa, grid, grid2, grid3, ga, ggrid, marks, s);
#else
  switch (kind) {
    case W4: return compress_k<W4>(*tm, *a, *sa, *pa, grid, grid2, grid3, ga, ggrid, marks, s);
    case W4LI: return compress_k<W4LI>(*tm, *a, *sa, *pa, grid, grid2, grid3, ga, ggrid, marks, s);
    default: return compress_k<W3AI>(*tm, *a, *sa, *pa, grid, grid2, grid3, ga, ggrid, marks, s);
  }
#endif
}

extern "C" cudaError_t CZ_CAT(czl_compress_batch_, CZ_SUFFIX)(int kind, const StageMaps<MAXF> *maps,
                                                               const FwdArgs *a, const S2Args *sa,
                                                               const BatchOut *bo, const PlaceArgs *pa, int grid,
                                                               int grid2, int grid3, int tiles, int place_tile,
                                                               int slab, cudaStream_t s)
{
#ifdef CZ_FAST
  if (kind != W3AI) return cudaErrorInvalidValue;
  return compress_batch_k<W3AI>(*maps, *a, *sa, *bo, *pa, grid, grid2, grid3, tiles, place_tile, slab, s);
#else
  switch (kind) {
    case W4: return compress_batch_k<W4>(*maps, *a, *sa, *bo, *pa, grid, grid2, grid3, tiles, place_tile, slab, s);
    case W4LI: return compress_batch_k<W4LI>(*maps, *a, *sa, *bo, *pa, grid, grid2, grid3, tiles, place_tile, slab, s);
    default: return compress_batch_k<W3AI>(*maps, *a, *sa, *bo, *pa, grid, grid2, grid3, tiles, place_tile, slab, s);
  }
#endif
}

extern "C" cudaError_t CZ_CAT(czl_decompress_, CZ_SUFFIX)(int kind, const CUtensorMap *om, const InvArgs *a,
                                                           const UnArgs *ua, int grid, const int *ugrid,
                                                           const cudaEvent_t *marks, cudaStream_t s)
{
#ifdef CZ_FAST
  if (kind != W3AI) return cudaErrorInvalidValue;
  return decompress_k<W3AI>(*om, *a, *ua, grid, ugrid, marks, s);
#else
  switch (kind) {
    case W4: return decompress_k<W4>(*om, *a, *ua, grid, ugrid, marks, s);
    case W4LI: return decompress_k<W4LI>(*om, *a, *ua, grid, ugrid, marks, s);
    default: return decompress_k<W3AI>(*om, *a, *ua, grid, ugrid, marks, s);
  }
#endif
}

extern "C" cudaError_t CZ_CAT(czl_dense_, CZ_SUFFIX)(int kind, int fwd, const DenseArgs *a, int nblocks,
                                                      cudaStream_t s)
{
#ifdef CZ_FAST
  if (kind != W3AI) return cudaErrorInvalidValue;
  return fwd ? dense_k<W3AI, true>(*a, nblocks, s) : dense_k<W3AI, false>(*a, nblocks, s);
#else
  if (fwd) {
    switch (kind) {
      case W4: return dense_k<W4, true>(*a, nblocks, s);
      case W4LI: return dense_k<W4LI, true>(*a, nblocks, s);
      default: return dense_k<W3AI, true>(*a, nblocks, s);
    }
  }
  switch (kind) {
    case W4: return dense_k<W4, false>(*a, nblocks, s);
    case W4LI: return dense_k<W4LI, false>(*a, nblocks, s);
    default: return dense_k<W3AI, false>(*a, nblocks, s);
  }
#endif
}

// CTAs per SM of the stage kernel (which = 0), the decompress kernel
// (which = 1), the small (2) or large (3) stage-2 kernel, the small (4) or
// large (5) stage-2 inverse kernel, the half-block decoder (6; 0 where the
// lane has none), the batched slab stage kernel where the lane's own is the
// register-resident one (7; 0 where it has none)
static int occupancy_query(int kind, int which);

// cached per device: later calls (e.g. inside a stream capture) make no
// CUDA call but cudaGetDevice
extern "C" int CZ_CAT(czl_occupancy_, CZ_SUFFIX)(int kind, int which)
{
  static int cache[64][3][8];  // device, kind, which; 0 = not yet known
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64 || kind < 0 || kind > 2 || which < 0 ||
      which > 7)
    return occupancy_query(kind, which);
  int v = __atomic_load_n(&cache[dev][kind][which], __ATOMIC_ACQUIRE);
  if (v > 0) return v;
  v = occupancy_query(kind, which);
  if (v > 0) __atomic_store_n(&cache[dev][kind][which], v, __ATOMIC_RELEASE);
  return v;
}

static int occupancy_query(int kind, int which)
{
  if (which == 2) return occupancy_s2<false>();
  if (which == 3) return G::HAS_BIG ? occupancy_s2<true>() : 1;
  if (which == 4) return occupancy_u<false>();
  if (which == 5) return G::HAS_BIG ? occupancy_u<true>() : 1;
#ifdef CZ_FAST
  if (kind != W3AI) return 0;
  if (which == 6) return occupancy_h<W3AI>();
  if (which == 7) return occupancy_slab_alt<W3AI>();
  return which == 0 ? occupancy_c<W3AI>() : occupancy_d<W3AI>();
#else
  if (which == 6) {
    switch (kind) {
      case W4: return occupancy_h<W4>();
      case W4LI: return occupancy_h<W4LI>();
      default: return occupancy_h<W3AI>();
    }
  }
  if (which == 7) {
    switch (kind) {
      case W4: return occupancy_slab_alt<W4>();
      case W4LI: return occupancy_slab_alt<W4LI>();
      default: return occupancy_slab_alt<W3AI>();
    }
  }
  if (which == 0) {
    switch (kind) {
      case W4: return occupancy_c<W4>();
      case W4LI: return occupancy_c<W4LI>();
      default: return occupancy_c<W3AI>();
    }
  }
  switch (kind) {
    case W4: return occupancy_d<W4>();
    case W4LI: return occupancy_d<W4LI>();
    default: return occupancy_d<W3AI>();
  }
#endif
}

// bytes of the staging slot of the largest payload
extern "C" int CZ_CAT(czl_slot_bytes_, CZ_SUFFIX)() { return G::PSLOT; }

// CTAs per SM of a group kernel (see occupancy_g; 0 on error)
extern "C" int CZ_CAT(czl_group_occupancy_, CZ_SUFFIX)(int which, int hcap)
{
  if (which < 0 || which > 5 || hcap <= 0 || hcap > GROUP_MAX_BYTES || hcap % 128) return 0;
  return occupancy_g(which, hcap);
}

// global scratch per CTA of the stage kernel, the large stage-2 kernel and
// the large stage-2 inverse kernel (FP64 32^3 only; 0 otherwise)
extern "C" int CZ_CAT(czl_scratch_bytes_, CZ_SUFFIX)() { return G::SCRATCH; }

// global scratch per CTA of the batched slab stage kernel where the tuner
// may pick it instead of the register-resident one (one block; 0 where the
// lane has no such choice)
extern "C" int CZ_CAT(czl_alt_scratch_bytes_, CZ_SUFFIX)() { return HAS_SLAB_ALT ? (int)SGi::SCR : 0; }
