// cz_noalloc.cu -- cz_compress with a workspace that the library owns.
//
// The workspace is a fixed array in this module's device memory.  Its
// address is looked up once per device, the first time the entry point is
// called with that device current; later calls reuse it.  No call here
// allocates or frees device memory.  The module (and so the array) is
// loaded by the CUDA runtime the first time its symbol is looked up.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/cz.h"

namespace {

static __device__ __align__(256) unsigned char g_ws[CZ_NOALLOC_WS_BYTES];

constexpr int MAX_DEVICES = 64;
void *g_ws_ptr[MAX_DEVICES];  // device address of g_ws per device, null until looked up
std::mutex g_ws_mutex;

// address of g_ws on the current device, or null on a CUDA error
void *workspace_of_current_device()
{
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return nullptr;
  void *p = __atomic_load_n(&g_ws_ptr[dev], __ATOMIC_ACQUIRE);
  if (p) return p;
  std::lock_guard<std::mutex> lock(g_ws_mutex);
  p = g_ws_ptr[dev];
  if (!p) {
    if (cudaGetSymbolAddress(&p, g_ws) != cudaSuccess || !p) return nullptr;
    __atomic_store_n(&g_ws_ptr[dev], p, __ATOMIC_RELEASE);
  }
  return p;
}

}  // namespace

int cz_compress_noalloc(const cz_params *p, const void *d_field, void *d_out, size_t out_cap,
                        uint64_t *d_out_bytes, void *stream)
{
  // the caller's buffers are checked as cz_compress checks them, before
  // any CUDA call (the workspace lookup below is one)
  if (!d_field || !d_out || ((uintptr_t)d_field % 16) || ((uintptr_t)d_out % 16)) return CZ_ERR_ARG;
  size_t need = 0;
  const int r = cz_workspace_size(p, &need);
  if (r != CZ_OK) return r;
  if (need > (size_t)CZ_NOALLOC_WS_BYTES) return CZ_ERR_CAPACITY;
  void *ws = workspace_of_current_device();
  if (!ws) return CZ_ERR_CUDA;
  // cz_compress clears the parts of the workspace that must start at zero
  // (status word, ticket, min/max keys, look-back words) on `stream` before
  // its kernels run; the rest is written before it is read.
  return cz_compress(p, d_field, d_out, out_cap, d_out_bytes, ws, (size_t)CZ_NOALLOC_WS_BYTES, stream);
}

int cz_noalloc_status(void *stream)
{
  // the status word is the first word of the workspace
  void *ws = workspace_of_current_device();
  if (!ws) return CZ_ERR_CUDA;
  return cz_status(ws, stream);
}
