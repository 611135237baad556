// cz_launch.h -- internal launchers, one set per (element type, block edge).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

namespace czp {
struct FwdArgs;
struct InvArgs;
struct UnArgs;
struct DenseArgs;
struct S2Args;
struct PlaceArgs;
struct GroupArgs;
struct BatchOut;
template <int NF>
struct StageMaps;
}  // namespace czp

#define CZ_DECLARE_LAUNCHERS(sfx)                                                                    \
  extern "C" cudaError_t czl_compress_##sfx(int kind, const CUtensorMap *tm, const czp::FwdArgs *a, \
                                            const czp::S2Args *sa, const czp::PlaceArgs *pa,        \
                                            int grid, int grid2, int grid3,                         \
                                            const czp::GroupArgs *ga, const int *ggrid,             \
                                            const cudaEvent_t *marks, cudaStream_t s);              \
  extern "C" cudaError_t czl_compress_batch_##sfx(                                                   \
      int kind, const czp::StageMaps<32> *maps, const czp::FwdArgs *a, const czp::S2Args *sa,          \
      const czp::BatchOut *bo, const czp::PlaceArgs *pa, int grid, int grid2, int grid3, int tiles,    \
      int place_tile, int slab, cudaStream_t s);                                                        \
  extern "C" cudaError_t czl_decompress_##sfx(int kind, const CUtensorMap *om, const czp::InvArgs *a,  \
                                              const czp::UnArgs *ua, int grid, const int *ugrid,      \
                                              const cudaEvent_t *marks, cudaStream_t s);              \
  extern "C" cudaError_t czl_dense_##sfx(int kind, int fwd, const czp::DenseArgs *a, int nblocks,   \
                                         cudaStream_t s);                                           \
  extern "C" int czl_occupancy_##sfx(int kind, int which);                                         \
  extern "C" int czl_slot_bytes_##sfx();                                                           \
  extern "C" int czl_group_occupancy_##sfx(int which, int hcap);                                   \
  extern "C" int czl_scratch_bytes_##sfx();                                                        \
  extern "C" int czl_alt_scratch_bytes_##sfx();

CZ_DECLARE_LAUNCHERS(f32_b8)
CZ_DECLARE_LAUNCHERS(f32_b16)
CZ_DECLARE_LAUNCHERS(f32_b32)
CZ_DECLARE_LAUNCHERS(f32_b64)
CZ_DECLARE_LAUNCHERS(f64_b8)
CZ_DECLARE_LAUNCHERS(f64_b16)
CZ_DECLARE_LAUNCHERS(f64_b32)
CZ_DECLARE_LAUNCHERS(f32_b8_fast)
CZ_DECLARE_LAUNCHERS(f32_b16_fast)
CZ_DECLARE_LAUNCHERS(f32_b32_fast)
CZ_DECLARE_LAUNCHERS(f32_b64_fast)
CZ_DECLARE_LAUNCHERS(f64_b8_fast)
CZ_DECLARE_LAUNCHERS(f64_b16_fast)
CZ_DECLARE_LAUNCHERS(f64_b32_fast)
