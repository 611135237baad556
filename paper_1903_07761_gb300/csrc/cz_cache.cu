// cz_cache.cu -- decoded-block cache for random access (Sec. 2.3, "Data
// decompression": recently decompressed blocks are kept and served again
// without decompressing).
//
// The cache is a device array of `capacity` decoded B^3 tiles plus as many
// staging tiles, and a host-side map from block id to slot with a
// least-recently-used order.  A fetch plans on the host which requested
// blocks are cached and which slots the missing ones replace, decodes the
// missing blocks (each once) into the staging tiles with
// cz_decompress_blocks, and then runs one copy kernel: staging -> the
// replaced slots, and for every request slot or staging -> its output tile.
// No copy reads a tile that another copy of the same launch writes (hits
// are never replaced in their own call), so the copies are independent.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <list>
#include <new>
#include <unordered_map>
#include <vector>

#include "../../include/cz.h"

namespace {

struct TileCopy {
  const unsigned char *src;
  unsigned char *dst;
};

// one CTA per tile, 16-byte vectors (tiles are whole multiples of 16 bytes)
__global__ void __launch_bounds__(256) k_tile_copy(const TileCopy *plan, int ntiles, unsigned long long tile_bytes)
{
  const int k = blockIdx.x;
  if (k >= ntiles) return;
  const uint4 *s = reinterpret_cast<const uint4 *>(plan[k].src);
  uint4 *d = reinterpret_cast<uint4 *>(plan[k].dst);
  const unsigned long long n = tile_bytes / 16;
  for (unsigned long long i = threadIdx.x; i < n; i += blockDim.x) d[i] = s[i];
}

}  // namespace

struct cz_cache {
  int cap = 0, block = 0, dtype = 0;
  size_t tile = 0;
  unsigned char *slots = nullptr, *stage = nullptr;
  // device copies of the plan (room for 2 * cap copies) and the ids (cap),
  // and pinned host buffers they are uploaded from: a ring of NUP, so that
  // the host may run up to NUP calls ahead of the device (a ring entry is
  // free again once its event, recorded after its uploads, has completed)
  static constexpr int NUP = 4;
  TileCopy *d_plan[NUP] = {};
  int32_t *d_ids[NUP] = {};
  TileCopy *h_plan[NUP] = {};
  int32_t *h_ids[NUP] = {};
  cudaEvent_t uploaded[NUP] = {};
  int next = 0;
  // the stream the cached blocks come from
  const void *src = nullptr;
  size_t src_bytes = 0;
  unsigned char hdr[CZ_HEADER_BYTES] = {0};
  // block id -> slot; slot -> block id (-1: empty); slots by recency (front:
  // most recent; empty slots at the back)
  std::unordered_map<int, int> where;
  std::vector<int> owner;
  std::list<int> lru;
  std::vector<std::list<int>::iterator> pos;
  long long hits = 0, misses = 0;

  void clear()
  {
    where.clear();
    lru.clear();
    for (int q = 0; q < cap; ++q) {
      owner[q] = -1;
      pos[q] = lru.insert(lru.end(), q);
    }
  }
  void touch(int slot)
  {
    lru.erase(pos[slot]);
    pos[slot] = lru.insert(lru.begin(), slot);
  }
};

extern "C" {

int cz_cache_create(int capacity, int block, int dtype, cz_cache **out)
{
  if (!out) return CZ_ERR_ARG;
  *out = nullptr;
  if (capacity < 1 || capacity > (1 << 20)) return CZ_ERR_ARG;
  if (block != 8 && block != 16 && block != 32 && block != 64) return CZ_ERR_ARG;
  if (dtype != CZ_F32 && dtype != CZ_F64) return CZ_ERR_ARG;
  cz_cache *c = new (std::nothrow) cz_cache;
  if (!c) return CZ_ERR_CUDA;
  c->cap = capacity;
  c->block = block;
  c->dtype = dtype;
  c->tile = (size_t)block * block * block * (dtype == CZ_F64 ? 8 : 4);
  c->owner.assign(capacity, -1);
  c->pos.resize(capacity);
  bool ok = cudaMalloc(&c->slots, c->tile * capacity) == cudaSuccess &&
            cudaMalloc(&c->stage, c->tile * capacity) == cudaSuccess;
  for (int u = 0; u < cz_cache::NUP && ok; ++u)
    ok = cudaMalloc(&c->d_plan[u], sizeof(TileCopy) * 2 * (size_t)capacity) == cudaSuccess &&
         cudaMalloc(&c->d_ids[u], sizeof(int32_t) * (size_t)capacity) == cudaSuccess &&
         cudaMallocHost(&c->h_plan[u], sizeof(TileCopy) * 2 * (size_t)capacity) == cudaSuccess &&
         cudaMallocHost(&c->h_ids[u], sizeof(int32_t) * (size_t)capacity) == cudaSuccess &&
         cudaEventCreateWithFlags(&c->uploaded[u], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cz_cache_destroy(c);
    return CZ_ERR_CUDA;
  }
  c->clear();
  *out = c;
  return CZ_OK;
}

void cz_cache_destroy(cz_cache *c)
{
  if (!c) return;
  cudaFree(c->slots);
  cudaFree(c->stage);
  for (int u = 0; u < cz_cache::NUP; ++u) {
    cudaFree(c->d_plan[u]);
    cudaFree(c->d_ids[u]);
    cudaFreeHost(c->h_plan[u]);
    cudaFreeHost(c->h_ids[u]);
    if (c->uploaded[u]) cudaEventDestroy(c->uploaded[u]);
  }
  delete c;
}

int cz_cache_clear(cz_cache *c)
{
  if (!c) return CZ_ERR_ARG;
  c->clear();
  return CZ_OK;
}

int cz_cache_stats(const cz_cache *c, int *held, long long *hits, long long *misses)
{
  if (!c) return CZ_ERR_ARG;
  if (held) *held = (int)c->where.size();
  if (hits) *hits = c->hits;
  if (misses) *misses = c->misses;
  return CZ_OK;
}

int cz_cache_fetch(cz_cache *c, const void *d_in, size_t in_bytes, const void *h_header, const int32_t *h_ids,
                   int n, void *d_tiles, size_t tiles_cap, void *d_ws, size_t ws_bytes, void *stream, int *h_hits)
{
  if (h_hits) *h_hits = 0;
  if (!c || !d_in || n < 0 || (n > 0 && (!h_ids || !d_tiles))) return CZ_ERR_ARG;
  if (n > c->cap) return CZ_ERR_ARG;
  if (n == 0) return CZ_OK;
  if ((uintptr_t)d_tiles % 16) return CZ_ERR_ARG;
  if ((size_t)n * c->tile > tiles_cap) return CZ_ERR_CAPACITY;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  unsigned char hb[CZ_HEADER_BYTES];
  if (in_bytes < (size_t)CZ_HEADER_BYTES) return CZ_ERR_CORRUPT;
  if (h_header) {
    std::memcpy(hb, h_header, CZ_HEADER_BYTES);
  } else {
    if (cudaMemcpyAsync(hb, d_in, CZ_HEADER_BYTES, cudaMemcpyDeviceToHost, s) != cudaSuccess) return CZ_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return CZ_ERR_CUDA;
  }
  cz_params p;
  int r = cz_read_header(hb, CZ_HEADER_BYTES, &p, nullptr);
  if (r != CZ_OK) return r;
  if (p.block != c->block || p.dtype != c->dtype) return CZ_ERR_ARG;
  const long long nblocks = (long long)(p.nx / p.block) * (p.ny / p.block) * (p.nz / p.block);
  for (int i = 0; i < n; ++i)
    if (h_ids[i] < 0 || h_ids[i] >= nblocks) return CZ_ERR_ARG;
  // another stream: the cached blocks are not its blocks
  if (d_in != c->src || in_bytes != c->src_bytes || std::memcmp(hb, c->hdr, CZ_HEADER_BYTES) != 0) c->clear();

  // plan: the blocks held now (pinned for this call), the missing ones in
  // order of first request, each with the slot it replaces
  std::unordered_map<int, int> miss_at;  // missing block id -> index in `miss`
  std::vector<int32_t> miss;
  std::vector<char> pinned(c->cap, 0);
  int hits = 0;
  for (int i = 0; i < n; ++i) {
    const auto it = c->where.find(h_ids[i]);
    if (it != c->where.end()) {
      pinned[it->second] = 1;
      ++hits;
    } else if (miss_at.find(h_ids[i]) == miss_at.end()) {
      miss_at.emplace(h_ids[i], (int)miss.size());
      miss.push_back(h_ids[i]);
    }
  }
  const int nm = (int)miss.size();
  std::vector<int> victim;
  victim.reserve(nm);
  for (auto it = c->lru.rbegin(); it != c->lru.rend() && (int)victim.size() < nm; ++it)
    if (!pinned[*it]) victim.push_back(*it);
  if ((int)victim.size() < nm) return CZ_ERR_ARG;  // cannot happen: distinct blocks <= n <= capacity

  // this call's ring entry: free once the uploads of the call NUP calls ago
  // have completed
  const int u = c->next;
  if (cudaEventSynchronize(c->uploaded[u]) != cudaSuccess) return CZ_ERR_CUDA;
  TileCopy *hp = c->h_plan[u];
  int np = 0;
  for (int m = 0; m < nm; ++m) hp[np++] = {c->stage + (size_t)m * c->tile, c->slots + (size_t)victim[m] * c->tile};
  unsigned char *out = reinterpret_cast<unsigned char *>(d_tiles);
  for (int i = 0; i < n; ++i) {
    const auto it = c->where.find(h_ids[i]);
    const unsigned char *src = it != c->where.end() ? c->slots + (size_t)it->second * c->tile
                                                    : c->stage + (size_t)miss_at[h_ids[i]] * c->tile;
    hp[np++] = {src, out + (size_t)i * c->tile};
  }

  // enqueue: decode the missing blocks into the staging tiles, then the
  // copies
  // the status word of d_ws reports this call: cz_decompress_blocks resets
  // it when there are blocks to decode, a call served wholly from the cache
  // resets it here
  if (nm == 0 && d_ws && cudaMemsetAsync(d_ws, 0, sizeof(unsigned), s) != cudaSuccess) return CZ_ERR_CUDA;
  if (nm > 0) {
    std::memcpy(c->h_ids[u], miss.data(), sizeof(int32_t) * nm);
    if (cudaMemcpyAsync(c->d_ids[u], c->h_ids[u], sizeof(int32_t) * nm, cudaMemcpyHostToDevice, s) != cudaSuccess)
      return CZ_ERR_CUDA;
    r = cz_decompress_blocks(d_in, in_bytes, hb, c->d_ids[u], nm, c->stage, (size_t)nm * c->tile, d_ws, ws_bytes,
                             stream);
    if (r != CZ_OK) return r;
  }
  if (cudaMemcpyAsync(c->d_plan[u], hp, sizeof(TileCopy) * np, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return CZ_ERR_CUDA;
  if (cudaEventRecord(c->uploaded[u], s) != cudaSuccess) return CZ_ERR_CUDA;
  c->next = (u + 1) % cz_cache::NUP;
  k_tile_copy<<<(unsigned)np, 256, 0, s>>>(c->d_plan[u], np, (unsigned long long)c->tile);
  if (cudaGetLastError() != cudaSuccess) return CZ_ERR_CUDA;

  // commit: the decoded blocks take their slots; this call's blocks become
  // the most recent, the last request the most recent of all
  for (int m = 0; m < nm; ++m) {
    const int q = victim[m];
    if (c->owner[q] >= 0) c->where.erase(c->owner[q]);
    c->owner[q] = miss[m];
    c->where[miss[m]] = q;
  }
  for (int i = 0; i < n; ++i) c->touch(c->where[h_ids[i]]);
  c->src = d_in;
  c->src_bytes = in_bytes;
  std::memcpy(c->hdr, hb, CZ_HEADER_BYTES);
  c->hits += hits;
  c->misses += nm;
  if (h_hits) *h_hits = hits;
  return CZ_OK;
}

}  // extern "C"
