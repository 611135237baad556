// cz_launch.h -- internal launchers, one set per (element type, block edge).
#pragma once
#include <cuda_runtime.h>

namespace czk {
struct FwdArgs;
struct InvArgs;
struct DenseArgs;
}  // namespace czk

#define CZ_DECLARE_LAUNCHERS(sfx)                                                                \
  extern "C" cudaError_t czl_compress_##sfx(int kind, const czk::FwdArgs *a, cudaStream_t s);   \
  extern "C" cudaError_t czl_decompress_##sfx(int kind, const czk::InvArgs *a, cudaStream_t s); \
  extern "C" cudaError_t czl_dense_##sfx(int kind, int fwd, const czk::DenseArgs *a, int nblocks, \
                                         cudaStream_t s);                                       \
  extern "C" int czl_smem_##sfx(void);

CZ_DECLARE_LAUNCHERS(f32_b8)
CZ_DECLARE_LAUNCHERS(f32_b16)
CZ_DECLARE_LAUNCHERS(f32_b32)
CZ_DECLARE_LAUNCHERS(f64_b8)
CZ_DECLARE_LAUNCHERS(f64_b16)
