/*
 * cz.h -- C ABI of the GB300 wavelet codec for block-structured 3D fields.
 *
 * The codec is the first compression substage of CubismZ (Hadjidoukas and
 * Wermelinger, arXiv 1903.07761): every cubic block of a 3D float field
 * (Sec. 2.1: constant-size cubic blocks, power-of-two edge) goes through a
 * full dyadic 3D interpolating-wavelet transform on the interval (Sec. 2.3
 * "Wavelet-based compression" and "Wavelet types": W4, W4li, W3ai), its
 * detail coefficients are thresholded against eps, and the block is stored
 * as a bit-set mask plus the significant coefficients (Sec. 2.3).  An
 * optional second substage byte-shuffles each block's output with the
 * element size of the data (Sec. 2.3 "Lossless compression") and applies
 * zero run-length coding.  Offsets of the per-block chunks come from an
 * exclusive prefix sum (Sec. 2.2, the paper's MPI scan of file offsets),
 * here a single-pass scan on the device.  Decompression reverses the steps
 * block by block (Sec. 2.3 "Data decompression").
 *
 * Conventions
 *  - Pointers named d_* are CUDA device pointers, h_* are host pointers.
 *  - `stream` is a cudaStream_t passed as void*; NULL is the legacy stream.
 *  - All work is enqueued asynchronously on `stream`; the calls themselves
 *    never allocate device memory and never synchronise unless stated.
 *  - The caller owns every buffer.  Fields are dense C-order arrays
 *    field[z][y][x] (x fastest) of float (CZ_F32) or double (CZ_F64).
 *  - Return values: CZ_OK or a negative CZ_ERR_* code for errors found on
 *    the host.  Errors found on the device (capacity, corrupt stream,
 *    look-back timeout) are written to a status word in the workspace and
 *    read with cz_status().  Kernels never trap.
 *
 * Stream layout (little-endian), produced and consumed only by this library:
 *   header (128 B) | (nblocks+1) u64 chunk offsets | pad to 16 | chunks
 *   chunk  = [u32 nnz][u32 ntok][ntok u32 tokens][literal words]  (stage 2)
 *          = [u32 nnz][u32 0][payload]                            (no stage 2)
 *   payload = 64 coarse values | B^3/32 u32 mask words | nnz values
 * Blocks are numbered x fastest over the block grid.
 */
#ifndef CZ_H
#define CZ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* wavelet kinds (Sec. 2.3 "Wavelet types") */
enum { CZ_W4 = 0, CZ_W4LI = 1, CZ_W3AI = 2 };
/* element types: the paper's precision option (float, double) */
enum { CZ_F32 = 0, CZ_F64 = 1 };
/* threshold: t = eps * (max - min) of the whole field, or t = eps */
enum { CZ_EPS_REL = 0, CZ_EPS_ABS = 1 };
/* error bound: CZ_BOUND_PAPER drops details below t (Sec. 2.3: decimation
 * error "not larger than" the threshold, which holds per level and axis);
 * CZ_BOUND_STRICT drops details below t / C, C the largest row sum of
 * |synthesis| over the detail columns of a block, so that the decoded error
 * never exceeds t (C: 127 / 1572 / 5331 for W4 at B = 8 / 16 / 32, 19 / 100 /
 * 249 for W3ai, 51 / 1229 / 4637 for W4li) */
enum { CZ_BOUND_PAPER = 0, CZ_BOUND_STRICT = 1 };
/* flags: CZ_FLAG_FAST selects the fast build of the kernels, which lets the
 * compiler fuse multiply-adds (one rounding instead of two): coefficients
 * move by a few ulps, so a detail next to the threshold may be kept or
 * dropped differently and streams are no longer bit-identical to the exact
 * build's.  It keeps every coefficient within 2^-20 of the field range of
 * the exact one and the PSNR within 0.01 dB.  W3ai only: with W4 or W4li
 * (whose extrapolating rows carry weights up to 35/16) the flag is refused
 * with CZ_ERR_ARG.  The flag is recorded in the stream header;
 * decompression uses the build the stream was made with. */
enum { CZ_FLAG_FAST = 1 };
/* flags: CZ_FLAG_ZERO4 / CZ_FLAG_ZERO8 zero the 4 / 8 least significant
 * bits of every kept detail coefficient before the lossless substage (bit
 * zeroing "Z4" / "Z8", Sec. 3 Exp. 2): more zero bytes for stage 2 at a
 * small loss of precision; the mask and the coarse values are untouched.
 * At most one of the two; not with CZ_BOUND_STRICT (whose bound does not
 * cover the zeroing error).  Recorded in the stream header. */
enum { CZ_FLAG_ZERO4 = 2, CZ_FLAG_ZERO8 = 4 };
/* flags: aggregate chunks (Sec. 3, Exp. 2 and 3: the stage-1 output of
 * several blocks is concatenated and the lossless substage codes the
 * concatenation as one buffer).  CZ_FLAG_GROUP4 / 8 / 16 put G = 4 / 8 / 16
 * consecutive blocks (x-fastest block order; the last group may hold fewer)
 * in one chunk with one offset-table entry: the chunk is [u32 nnz of each
 * block | u32 ntok | tokens | literal words], the zero-run code of the byte
 * shuffle of the blocks' concatenated payloads.  The stream then carries
 * ceil(nblocks / G) + 1 offsets.  Stage 2 only, and only where G times the
 * largest block payload is at most CZ_GROUP_MAX_BYTES (FP32 32^3 blocks:
 * G <= 8; FP64 32^3: G = 4; FP32 64^3: none); otherwise CZ_ERR_ARG.
 * cz_compress, cz_compress_noalloc, cz_decompress, cz_decompress_blocks
 * (which decodes the whole group of each requested block) and
 * cz_stream_concat (slabs whose block counts are multiples of G, but the
 * last) take such streams; cz_compress_batch, cz_compress_aos and the server
 * refuse the flag.  Recorded in the stream header. */
enum { CZ_FLAG_GROUP4 = 8, CZ_FLAG_GROUP8 = 16, CZ_FLAG_GROUP16 = 24 };
#define CZ_GROUP_MAX_BYTES (1792u * 1024u)

enum {
  CZ_OK = 0,
  CZ_ERR_ARG = -1,      /* invalid parameter or unsupported combination   */
  CZ_ERR_CAPACITY = -2, /* output or workspace buffer too small           */
  CZ_ERR_CORRUPT = -3,  /* stream header, offsets or chunk inconsistent   */
  CZ_ERR_TIMEOUT = -4,  /* a bounded device-side wait gave up             */
  CZ_ERR_CUDA = -5,     /* a CUDA runtime call failed                     */
  CZ_ERR_BUDGET = -6    /* request refused by a memory budget             */
};

#define CZ_HEADER_BYTES 128

typedef struct cz_params {
  int32_t nx, ny, nz; /* field dims in elements; each a multiple of block   */
  int32_t block;      /* cubic block edge B: 8, 16, 32 or 64 (64: F32 only) */
  int32_t dtype;      /* CZ_F32 or CZ_F64                                   */
  int32_t kind;       /* CZ_W4, CZ_W4LI or CZ_W3AI                          */
  int32_t eps_mode;   /* CZ_EPS_REL (default) or CZ_EPS_ABS                 */
  int32_t stage2;     /* 1: byte shuffle + zero-RLE each chunk; 0: raw      */
  int32_t bound_mode; /* CZ_BOUND_PAPER (default) or CZ_BOUND_STRICT        */
  int32_t flags;      /* CZ_FLAG_FAST, CZ_FLAG_ZERO4 / CZ_FLAG_ZERO8,
                         CZ_FLAG_GROUP4 / 8 / 16 (or'ed), or 0            */
  double eps;         /* tolerance, >= 0                                    */
  double range;       /* >= 0: max - min supplied by the caller (skips the
                         min/max pass); < 0: computed on the device        */
} cz_params;

/* Worst-case stream size for p.  Returns CZ_OK or CZ_ERR_ARG. */
int cz_compress_bound(const cz_params *p, size_t *bytes);

/* Device workspace needed by cz_compress / cz_decompress for p: a status
 * word, the min/max keys, one u64 look-back word per block, a block table
 * (16 bytes per block), a mark byte and a list entry per block (the
 * single-read compression of cz_compress), and the staging slots the
 * chunks are built in (room for the largest chunk of every block, about
 * the size of the field; aggregate chunks add as much again).  FP64
 * with 32^3 blocks and FP32 with 64^3 blocks add one scratch block per CTA
 * (260 KiB / 1.03 MiB) of the kernels that hold a block or a large payload
 * in global memory.
 * Needs the current device (it sizes the persistent grids by its SM count). */
int cz_workspace_size(const cz_params *p, size_t *bytes);

/* Compress d_field into d_out (capacity out_cap bytes).
 * Steps: the field's min / max when range < 0; a persistent kernel that
 * loads each block with TMA, transforms it, thresholds it and writes
 * mask + compacted values to a staging slot; optional stage 2 on every
 * slot; chunk offsets by a decoupled look-back over tiles of chunks; a copy
 * of the chunks into the stream.  With range < 0, stage 2 on, the paper
 * bound, no bit zeroing and no aggregate chunks (FP32 blocks of edge 8 to
 * 32, FP64 of edge 8 and 16), the field is read once: a min / max pass over
 * every 4th row of every 4th z-plane gives a threshold t_lo <= t, the stage
 * kernel thresholds at t_lo and merges every block's min / max into the
 * header's, and stage 2 drops the details below the exact t from the
 * (few) slots that kept one.  The stream is the same byte for byte as with
 * t known first.  Otherwise a min / max pass reads the whole field first.
 * *d_out_bytes (device u64, may be NULL) receives the stream length; if it
 * exceeds out_cap the status word is CZ_ERR_CAPACITY and the stream is
 * incomplete.  d_ws must hold cz_workspace_size() bytes; it is overwritten.
 * Host-side errors: CZ_ERR_ARG, CZ_ERR_CAPACITY (out_cap below the fixed
 * header+table size, ws too small), CZ_ERR_CUDA. */
int cz_compress(const cz_params *p, const void *d_field, void *d_out,
                size_t out_cap, uint64_t *d_out_bytes, void *d_ws,
                size_t ws_bytes, void *stream);

/* Decompress the stream d_in (in_bytes long) into d_field (field_cap bytes).
 * The parameters come from the stream header: pass a host copy of its first
 * CZ_HEADER_BYTES bytes in h_header, or NULL to have the call copy it from
 * the device (one synchronous 128-byte copy on `stream`).  Chunk offsets and
 * chunk contents are validated on the device; a bad chunk sets the status
 * word to CZ_ERR_CORRUPT and its block is written as zeros. */
int cz_decompress(const void *d_in, size_t in_bytes, const void *h_header,
                  void *d_field, size_t field_cap, void *d_ws, size_t ws_bytes,
                  void *stream);

/* Random access (the paper's per-block decompression, Sec. 2.3: blocks are
 * compressed independently): decode the blocks d_ids[0..n) of the stream
 * d_in into n consecutive B^3 tiles at d_tiles (tile i holds block d_ids[i],
 * x fastest, then y, then z; tiles_cap >= n * B^3 * element bytes).  d_ids
 * is a device array of n int32 block indices in the stream's x-fastest
 * block order; they may repeat.  The workspace needs room for n blocks
 * (cz_decompress_blocks_workspace_size; cz_workspace_size of the stream's
 * parameters suffices for n <= nblocks).  An index outside the stream sets the status word to
 * CZ_ERR_ARG and a bad chunk CZ_ERR_CORRUPT; such tiles are zeros.  n = 0
 * is a no-op.  Header handling as for cz_decompress. */
int cz_decompress_blocks(const void *d_in, size_t in_bytes, const void *h_header, const int32_t *d_ids, int n,
                         void *d_tiles, size_t tiles_cap, void *d_ws, size_t ws_bytes, void *stream);

/* Workspace bytes cz_decompress_blocks needs to decode n blocks of a stream
 * made with parameters p.  Returns CZ_OK or CZ_ERR_ARG. */
int cz_decompress_blocks_workspace_size(const cz_params *p, int n, size_t *bytes);

/* ---- decoded-block cache for random access (Sec. 2.3, "Data
 * decompression": recently decompressed blocks are kept, and later requests
 * for them are served without decompressing again) --------------------------
 * A cache owns device memory for `capacity` decoded B^3 tiles of one
 * element type and block edge (and as many tiles of staging for the blocks
 * a call decodes), allocated by cz_cache_create on the current device.
 * It serves one stream at a time: a call with another stream (other device
 * address, length or header) empties it first; a stream rewritten in place
 * with the same length and header is not noticed, so clear the cache then.  Not thread-safe: one host
 * thread uses a cache at a time, with one CUDA stream. */
typedef struct cz_cache cz_cache;

/* Create a cache of `capacity` (>= 1) tiles for blocks of edge `block` and
 * element type `dtype` (CZ_F32 / CZ_F64).  CZ_ERR_ARG for bad arguments,
 * CZ_ERR_CUDA if the memory cannot be allocated. */
int cz_cache_create(int capacity, int block, int dtype, cz_cache **out);
void cz_cache_destroy(cz_cache *c);

/* Fetch blocks h_ids[0..n) (a HOST array; ids may repeat) of the stream
 * d_in into n consecutive B^3 tiles at d_tiles, as cz_decompress_blocks
 * does.  A block held by the cache is copied from it; the others (each
 * once) are decoded with cz_decompress_blocks into the staging tiles, then
 * take the cache slots of the least recently used blocks that this call
 * does not request.  All copies are one kernel on `stream`; nothing is
 * synchronised.  n <= capacity; every id must lie in the stream (checked on
 * the host: CZ_ERR_ARG before anything is enqueued); the stream's block
 * edge and type must match the cache's.  d_ws / ws_bytes as for
 * cz_decompress_blocks with n blocks.  *h_hits (may be NULL) receives the
 * number of requests served from the cache (blocks it held when the call
 * began).  Header handling as for cz_decompress.  The call resets the
 * status word of d_ws (also when every request is served from the cache);
 * device-side errors (a corrupt chunk) go to it, as for
 * cz_decompress_blocks; the block is then cached as the zeros it decoded
 * to, so after a call that set the status word, empty the cache
 * (cz_cache_clear). */
int cz_cache_fetch(cz_cache *c, const void *d_in, size_t in_bytes, const void *h_header, const int32_t *h_ids,
                   int n, void *d_tiles, size_t tiles_cap, void *d_ws, size_t ws_bytes, void *stream, int *h_hits);

/* Forget every cached block (the memory stays allocated). */
int cz_cache_clear(cz_cache *c);

/* Blocks the cache holds now, and the cumulative counts of requests served
 * from it (hits) and blocks it decoded (misses). */
int cz_cache_stats(const cz_cache *c, int *held, long long *hits, long long *misses);

/* Size of the workspace that cz_compress_noalloc uses: 64 MiB. */
#define CZ_NOALLOC_WS_BYTES (64u << 20)

/* cz_compress for callers that cannot allocate device memory.  The paper
 * has no counterpart; this entry point exists for the in-situ use the paper
 * describes, where a solver that has committed the device's memory
 * compresses its fields between time steps.  Such callers cannot make
 * cudaMalloc/cudaFree calls there: the memory may not be free, the calls
 * can synchronise the device, and caching allocators (PyTorch's included)
 * may hold what is free.  Instead of a caller-supplied d_ws this call uses
 * a CZ_NOALLOC_WS_BYTES array that the library owns in device memory, so
 * it works only for fields whose cz_workspace_size() is at most
 * CZ_NOALLOC_WS_BYTES; larger fields return CZ_ERR_CAPACITY before
 * anything is enqueued.  The workspace size depends on the device's SM
 * count (it holds one staging arena per CTA of the persistent stage
 * kernel): on a 152-SM GB300 the limit is 456 blocks of 32^3 FP32 (e.g. a
 * 128^3 field of 64 blocks fits, a 256^3 field of 512 blocks does not).
 *  - The first call on a device looks up the array's address with that
 *    device current (the CUDA runtime loads the library's module then).
 *    Make that first call before any stream capture begins.
 *  - There is one array per device: calls whose work may overlap on the
 *    device (different streams, or different host threads) race on it and
 *    corrupt each other's output.  Calls enqueued on one stream run one
 *    after the other and are safe.
 *  - The device status word of a call (CZ_ERR_CAPACITY when the output did
 *    not fit, CZ_ERR_TIMEOUT, ...) stays in the array until the next call:
 *    read it with cz_noalloc_status().
 * Other arguments and host-side errors are those of cz_compress (null or
 * misaligned buffers: CZ_ERR_ARG before any CUDA call). */
int cz_compress_noalloc(const cz_params *p, const void *d_field, void *d_out,
                        size_t out_cap, uint64_t *d_out_bytes, void *stream);

/* Synchronise `stream` and return the device status word of the last
 * cz_compress_noalloc call on the current device (CZ_OK or a CZ_ERR_* code
 * set by a kernel).  Calls that overlap on the device share the word as
 * they share the array.  CZ_ERR_CUDA if the array cannot be reached. */
int cz_noalloc_status(void *stream);

/* ---- many fields in one call (the paper compresses many blocks of many
 * quantities per node, Sec. 2.2; here whole fields are batched) ----------
 * Fields with the same dtype, block, kind, stage2, bound_mode and flags (at
 * most 32 at a time, in the order given) share one persistent launch of each
 * kernel: their blocks form one index space, each block finds its field,
 * and every field still gets its own stream, identical byte for byte to the
 * one cz_compress would write.  Field i is d_fields[i] (parameters p[i]),
 * its stream goes to d_outs[i] (capacity out_caps[i], length to
 * d_out_bytes[i], a device array of n u64, may be NULL).  The call makes no
 * allocation and no synchronisation; with its parameters fixed it can be
 * captured in a CUDA graph once a call outside the capture has set up the
 * kernels.  Errors as for cz_compress; the status word is shared.
 * Host-side: d_ws must hold cz_batch_workspace_size() bytes (the largest
 * group's workspace under any tuner setting; groups run one after another
 * and reuse it).  Each group uses the tuner's choices for its fields'
 * parameters (cz_batch_tune), else the defaults. */
int cz_batch_workspace_size(int n, const cz_params *p, size_t *bytes);
int cz_compress_batch(int n, const cz_params *p, const void *const *d_fields,
                      void *const *d_outs, const size_t *out_caps,
                      uint64_t *d_out_bytes, void *d_ws, size_t ws_bytes,
                      void *stream);

/* Autotuner of the batched launch: for every group of the batch (the
 * fields that share one launch) it times the group's launches on these very
 * arguments under each candidate setting of four knobs, `reps` timed calls
 * each after one warm-up, and keeps the fastest for later calls with the
 * same field parameters:
 *  - the lifting tile shape of the stage kernel: the block in registers
 *    (pair quads, one CTA of B^2/2 threads per block) or, where a lane has
 *    both (FP32 32^3), the slab kernel (the block in a global scratch block,
 *    one 256-thread CTA per block, two per SM);
 *  - the block-to-CTA mapping: one CTA per resident slot, or the fewest CTAs
 *    that keep the same number of rounds (blocks per CTA);
 *  - the stage-2 grid: all resident CTAs, or half;
 *  - the scan granularity: 64, 128 or 256 chunks per look-back tile.
 * Streams are identical under every setting.  Synchronises `stream`.  The
 * outputs are overwritten.  d_ws must hold cz_batch_workspace_size() bytes. */
int cz_batch_tune(int n, const cz_params *p, const void *const *d_fields,
                  void *const *d_outs, const size_t *out_caps,
                  uint64_t *d_out_bytes, void *d_ws, size_t ws_bytes,
                  void *stream, int reps);

/* The tuner's choices as JSON text, so that they outlive the process:
 *   {"format": "cz-batch-knobs", "version": 2, "entries": [
 *     {"signature": "<16 hex digits>", "s1_balanced": 0|1, "s2_div": 1..64,
 *      "place_tile": 64|128|256, "slab": 0|1}, ...]}
 * A signature identifies a group of fields by their parameters (not by their
 * buffers).  The choices are those of the device they were tuned on.
 * Version 1 texts (without place_tile and slab) are read with 128 and 0.
 * Export: *len receives the text length + 1; with buf NULL only the size is
 * returned, otherwise buf (cap bytes) receives the NUL-terminated text or
 * CZ_ERR_CAPACITY.  Import: merges the entries of such a text (an entry
 * replaces the one with its signature); CZ_ERR_ARG, and nothing changes,
 * if the text is not of this form.  Host only: no CUDA call. */
int cz_batch_knobs_export(char *buf, size_t cap, size_t *len);
int cz_batch_knobs_import(const char *json);

/* ---- quantities of a cell-struct array (the paper's solver stores all
 * quantities of a cell together and compresses chosen quantities from that
 * storage, Sec. 2.1 / 2.2) ---------------------------------------------------
 * d_cells holds nz*ny*nx cells of ncomp elements of one type, C order
 * [nz][ny][nx][ncomp].  Quantity i of the call is component comps[i]
 * (a host array; 0 <= comps[i] < ncomp) and is compressed with parameters
 * p[i] (all with the same nx, ny, nz and dtype; kind, block, eps, stage 2
 * and flags may differ) into d_outs[i] (capacity out_caps[i], length to
 * d_out_bytes[i], a device array of n u64, may be NULL).  One kernel reads
 * every cell once and writes the n chosen components as dense fields into
 * the workspace; a cz_compress_batch call then compresses them, so every
 * stream is identical to cz_compress of that component alone.  Errors as
 * for cz_compress_batch; d_ws must hold cz_aos_workspace_size() bytes. */
int cz_aos_workspace_size(int n, const cz_params *p, size_t *bytes);
int cz_compress_aos(int n, const cz_params *p, const void *d_cells, int ncomp, const int32_t *comps,
                    void *const *d_outs, const size_t *out_caps, uint64_t *d_out_bytes, void *d_ws,
                    size_t ws_bytes, void *stream);

/* ---- request server (the paper compresses in situ, while the simulation
 * runs, Sec. 2.2; here requests of mixed sizes and precisions arrive at any
 * time and share the device) ----------------------------------------------
 * The server allocates one device pool of budget_bytes when it is created
 * (the HBM budget; every admitted request takes its workspace from it) and
 * `streams` CUDA streams, and runs a worker thread that admits waiting
 * requests in arrival order as streams and pool memory free up.  Compress
 * requests that wait together and share dtype, block, kind, stage2,
 * bound_mode and flags are launched as one cz_compress_batch call.  Requests keep
 * their buffers (caller-owned, on the device) until they are done; results
 * are identical to cz_compress / cz_decompress on the same inputs.  Latency
 * is measured from submission to the worker seeing the request's work
 * finished. */
enum { CZ_OP_COMPRESS = 0, CZ_OP_DECOMPRESS = 1 };
enum { CZ_REQ_QUEUED = 0, CZ_REQ_RUNNING = 1, CZ_REQ_DONE = 2 };

typedef struct cz_request {
  int32_t op;          /* CZ_OP_COMPRESS or CZ_OP_DECOMPRESS                  */
  int32_t reserved;
  cz_params params;    /* compress: the field's parameters                    */
  const void *d_in;    /* compress: field; decompress: stream                 */
  size_t in_bytes;     /* decompress: stream bytes                            */
  unsigned char h_header[CZ_HEADER_BYTES]; /* decompress: host copy of the
                                              stream's header                 */
  void *d_out;         /* compress: stream buffer; decompress: field buffer   */
  size_t out_cap;      /* bytes of d_out                                      */
  uint64_t *d_out_bytes; /* compress: device u64 for the stream length, or NULL */
} cz_request;

/* Create a server on the current device.  CZ_ERR_CUDA if the pool cannot be
 * allocated. */
int cz_server_create(size_t budget_bytes, int streams, void **server);
/* Queue a request (copied); returns its ticket.  CZ_ERR_BUDGET if its
 * workspace can never fit the budget, else the host-side errors of the
 * corresponding call. */
int cz_server_submit(void *server, const cz_request *req, uint64_t *ticket);
/* State (CZ_REQ_*), result (CZ_OK or a CZ_ERR_* code from the host call or
 * the device status word) and latency in ms (-1 until done).  A done ticket
 * is reported once, then forgotten. */
int cz_server_poll(void *server, uint64_t ticket, int *state, int *result,
                   double *latency_ms);
/* Block until the ticket is done; then as cz_server_poll.  CZ_ERR_ARG for
 * an unknown ticket, or one that another thread's poll or wait reported (and
 * so forgot) while this call waited.  submit, poll and wait may be called
 * from several host threads at once. */
int cz_server_wait(void *server, uint64_t ticket, int *result, double *latency_ms);
/* Finish all queued and running work, then free the server. */
int cz_server_destroy(void *server);

/* ---- several GPUs: slabs of one field -----------------------------------
 * Blocks are independent (Sec. 2.2), so a field cut into z-slabs of whole
 * block planes can be compressed slab by slab (one GPU or rank each) with
 * the same parameters and the same supplied range (so that the threshold is
 * the same everywhere).  This host-side call joins the slab streams, given
 * in z order as host buffers, into the stream of the whole field: header
 * with the summed nz, offsets rebased by the exclusive prefix sum of the
 * slabs' data bytes (the paper's scan of per-rank sizes), chunks appended.
 * The result equals, byte for byte, the stream cz_compress writes for the
 * whole field with that range.  With h_out == NULL only *out_bytes is set.
 * CZ_ERR_ARG if the slabs disagree on anything but nz, CZ_ERR_CORRUPT for
 * a malformed stream, CZ_ERR_CAPACITY if out_cap is too small. */
int cz_stream_concat(int n, const void *const *h_streams, const size_t *sizes,
                     void *h_out, size_t out_cap, size_t *out_bytes);

/* Parse a host copy of a stream header into *p (and the threshold used). */
int cz_read_header(const void *h_in, size_t n, cz_params *p, double *t_used);

/* Synchronise `stream` and return the device status word of d_ws
 * (CZ_OK or a CZ_ERR_* code set by a kernel). */
int cz_status(const void *d_ws, void *stream);

/* Human-readable text of a CZ_* code (static storage). */
const char *cz_strerror(int code);

/* Dense coefficients, for testing the transform alone: the forward
 * transform of every block of d_field written in place of the field layout
 * to d_coef (same shape and type), or the inverse of d_coef into d_field. */
int cz_forward_dense(const cz_params *p, const void *d_field, void *d_coef,
                     void *stream);
int cz_inverse_dense(const cz_params *p, const void *d_coef, void *d_field,
                     void *stream);

#ifdef __cplusplus
}
#endif
#endif
