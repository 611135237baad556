// cz_inst.cu -- kernel instantiations for one (element type, block edge).
// Built once per combination with -DCZ_T=float|double -DCZ_B=8|16|32 so the
// heavily unrolled kernels compile in parallel.  Exposes plain launchers.
#include <cuda_runtime.h>

#include "cz_kernels.cuh"
#include "cz_launch.h"

#ifndef CZ_T
#error "CZ_T must be defined"
#endif
#ifndef CZ_B
#error "CZ_B must be defined"
#endif

using namespace czk;

namespace {

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

template <int KIND>
cudaError_t compress_k(const FwdArgs &a, cudaStream_t s)
{
  using G = Geo<CZ_T, CZ_B>;
  cudaError_t e = prepare<k_compress<CZ_T, CZ_B, KIND>>(G::SMEM);
  if (e != cudaSuccess) return e;
  k_compress<CZ_T, CZ_B, KIND><<<a.nblocks, G::NT, G::SMEM, s>>>(a);
  return cudaGetLastError();
}

template <int KIND>
cudaError_t decompress_k(const InvArgs &a, cudaStream_t s)
{
  using G = Geo<CZ_T, CZ_B>;
  cudaError_t e = prepare<k_decompress<CZ_T, CZ_B, KIND>>(G::SMEM);
  if (e != cudaSuccess) return e;
  k_decompress<CZ_T, CZ_B, KIND><<<a.nblocks, G::NT, G::SMEM, s>>>(a);
  return cudaGetLastError();
}

template <int KIND, bool FWD>
cudaError_t dense_k(const DenseArgs &a, int nblocks, cudaStream_t s)
{
  using G = Geo<CZ_T, CZ_B>;
  cudaError_t e = prepare<k_dense<CZ_T, CZ_B, KIND, FWD>>(G::XBYTES);
  if (e != cudaSuccess) return e;
  k_dense<CZ_T, CZ_B, KIND, FWD><<<nblocks, G::NT, G::XBYTES, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

#define CZ_CAT2(a, b) a##b
#define CZ_CAT(a, b) CZ_CAT2(a, b)
#define CZ_SUFFIX CZ_CAT(CZ_CAT(CZ_TNAME, _b), CZ_B)

extern "C" cudaError_t CZ_CAT(czl_compress_, CZ_SUFFIX)(int kind, const FwdArgs *a, cudaStream_t s)
{
  switch (kind) {
    case W4: return compress_k<W4>(*a, s);
    case W4LI: return compress_k<W4LI>(*a, s);
    default: return compress_k<W3AI>(*a, s);
  }
}

extern "C" cudaError_t CZ_CAT(czl_decompress_, CZ_SUFFIX)(int kind, const InvArgs *a, cudaStream_t s)
{
  switch (kind) {
    case W4: return decompress_k<W4>(*a, s);
    case W4LI: return decompress_k<W4LI>(*a, s);
    default: return decompress_k<W3AI>(*a, s);
  }
}

extern "C" cudaError_t CZ_CAT(czl_dense_, CZ_SUFFIX)(int kind, int fwd, const DenseArgs *a, int nblocks,
                                                      cudaStream_t s)
{
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
}

extern "C" int CZ_CAT(czl_smem_, CZ_SUFFIX)(void) { return Geo<CZ_T, CZ_B>::SMEM; }
