// cz_serve.cu -- a request server over the codec: compress and decompress
// requests arrive at any time, are admitted as device memory and streams
// free up, and overlap on the GPU.
//
// The server owns one device pool of `budget` bytes, allocated once, from
// which every admitted request (or group of requests) takes its workspace;
// the requests' own buffers are the caller's and stay on the device.  A
// worker thread loops: it retires finished work (an event per stream),
// then admits waiting requests in arrival order while a stream and pool
// memory are free.  Compress requests that wait together and share element
// type, block, kind, stage 2 and bound mode are launched as one batched call
// (continuous batching: arrivals join the next launch instead of queueing
// one by one).  A request that waits behind one that does not fit may be
// admitted before it, unless the waiting one has waited longer than the
// starvation limit, after which admission waits for it.
//
// The worker owns a host core while the server is active: with work in
// flight, or within IDLE_SPIN of the last request, it polls the streams'
// events and an arrival flag without sleeping (a sleep and a wake-up cost
// tens of microseconds each, more than a small request takes on the GPU);
// it blocks on the condition variable only after that.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <list>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/cz.h"

namespace {

using Clock = std::chrono::steady_clock;
constexpr int MAX_GROUP = 32;                             // requests per batched launch
constexpr auto STARVE_LIMIT = std::chrono::milliseconds(50);
constexpr auto IDLE_SPIN = std::chrono::milliseconds(50);   // polling without sleep after the last activity

struct Req {
  uint64_t ticket = 0;
  cz_request r{};
  cz_params p{};   // compress: r.params; decompress: from the header copy
  size_t ws = 0;   // workspace bytes when run alone
  Clock::time_point t_submit{}, t_done{};
  int state = CZ_REQ_QUEUED;
  int result = CZ_OK;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  unsigned *h_status = nullptr;  // pinned copy of the workspace status word
  bool busy = false;
  std::vector<uint64_t> tickets;
  size_t ws_off = 0, ws_len = 0;
};

// first-fit allocator of [offset, length) ranges of the pool, 256-byte units
class Ranges {
 public:
  explicit Ranges(size_t n) { free_[0] = n; }
  bool take(size_t len, size_t *off)
  {
    len = (len + 255) / 256 * 256;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= len) {
        *off = it->first;
        const size_t rest = it->second - len, at = it->first + len;
        free_.erase(it);
        if (rest) free_[at] = rest;
        return true;
      }
    }
    return false;
  }
  void give(size_t off, size_t len)
  {
    len = (len + 255) / 256 * 256;
    auto it = free_.emplace(off, len).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }

 private:
  std::map<size_t, size_t> free_;
};

bool same_group(const cz_params &a, const cz_params &b)
{
  return a.dtype == b.dtype && a.block == b.block && a.kind == b.kind && a.stage2 == b.stage2 &&
         a.bound_mode == b.bound_mode && a.flags == b.flags;
}

class Server {
 public:
  int init(size_t budget, int nslots)
  {
    if (cudaGetDevice(&dev_) != cudaSuccess) return CZ_ERR_CUDA;
    budget_ = (budget + 255) / 256 * 256;
    if (cudaMalloc(&pool_, budget_) != cudaSuccess) return CZ_ERR_CUDA;
    ranges_ = new Ranges(budget_);
    slots_.resize(nslots);
    for (Slot &s : slots_) {
      if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess) return CZ_ERR_CUDA;
      if (cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess) return CZ_ERR_CUDA;
      if (cudaMallocHost(&s.h_status, sizeof(unsigned)) != cudaSuccess) return CZ_ERR_CUDA;
    }
    worker_ = std::thread([this] { loop(); });
    return CZ_OK;
  }

  ~Server()
  {
    {
      std::lock_guard<std::mutex> lock(mu_);
      stop_ = true;
    }
    cv_.notify_all();
    if (worker_.joinable()) worker_.join();
    for (Slot &s : slots_) {
      if (s.stream) cudaStreamSynchronize(s.stream);
      if (s.stream) cudaStreamDestroy(s.stream);
      if (s.done) cudaEventDestroy(s.done);
      if (s.h_status) cudaFreeHost(s.h_status);
    }
    if (pool_) cudaFree(pool_);
    delete ranges_;
  }

  int submit(const cz_request *r, uint64_t *ticket)
  {
    Req q;
    q.r = *r;
    if (r->op == CZ_OP_COMPRESS) {
      q.p = r->params;
      // compressions run as batched launches, which take no aggregate chunks
      if (q.p.flags & (CZ_FLAG_GROUP4 | CZ_FLAG_GROUP8 | CZ_FLAG_GROUP16)) return CZ_ERR_ARG;
    } else if (r->op == CZ_OP_DECOMPRESS) {
      double t;
      const int e = cz_read_header(r->h_header, CZ_HEADER_BYTES, &q.p, &t);
      if (e != CZ_OK) return e;
    } else {
      return CZ_ERR_ARG;
    }
    int e;
    {
      // workspace sizes depend on the device: query it from this thread
      // with the server's device current
      int cur = 0;
      cudaGetDevice(&cur);
      if (cur != dev_) cudaSetDevice(dev_);
      e = cz_workspace_size(&q.p, &q.ws);
      if (cur != dev_) cudaSetDevice(cur);
    }
    if (e != CZ_OK) return e;
    if (q.ws + 512 > budget_) return CZ_ERR_BUDGET;  // never fits
    std::lock_guard<std::mutex> lock(mu_);
    q.ticket = ++next_;
    q.t_submit = Clock::now();
    *ticket = q.ticket;
    reqs_[q.ticket] = q;
    queue_.push_back(q.ticket);
    arrived_.store(true, std::memory_order_release);
    cv_.notify_all();
    return CZ_OK;
  }

  int poll(uint64_t ticket, int *state, int *result, double *latency_ms)
  {
    std::lock_guard<std::mutex> lock(mu_);
    auto it = reqs_.find(ticket);
    if (it == reqs_.end()) return CZ_ERR_ARG;
    report(it->second, state, result, latency_ms);
    if (it->second.state == CZ_REQ_DONE) reqs_.erase(it);  // reported once
    return CZ_OK;
  }

  int wait(uint64_t ticket, int *result, double *latency_ms)
  {
    std::unique_lock<std::mutex> lock(mu_);
    auto it = reqs_.find(ticket);
    if (it == reqs_.end()) return CZ_ERR_ARG;
    // find, never operator[]: a ticket that another thread reported (and so
    // removed) meanwhile must not come back as a fresh, never-done entry
    done_cv_.wait(lock, [&] {
      const auto j = reqs_.find(ticket);
      return j == reqs_.end() || j->second.state == CZ_REQ_DONE;
    });
    it = reqs_.find(ticket);
    if (it == reqs_.end()) return CZ_ERR_ARG;  // reported to another caller
    int st;
    report(it->second, &st, result, latency_ms);
    reqs_.erase(it);
    return CZ_OK;
  }

 private:
  static void report(const Req &q, int *state, int *result, double *latency_ms)
  {
    if (state) *state = q.state;
    if (result) *result = q.result;
    if (latency_ms)
      *latency_ms = q.state == CZ_REQ_DONE
                        ? std::chrono::duration<double, std::milli>(q.t_done - q.t_submit).count()
                        : -1.0;
  }

  // retire finished slots (mu_ held)
  bool retire()
  {
    bool any = false;
    for (Slot &s : slots_) {
      if (!s.busy) continue;
      const cudaError_t e = cudaEventQuery(s.done);
      if (e == cudaErrorNotReady) continue;
      const Clock::time_point now = Clock::now();
      const int res = e == cudaSuccess ? (int)*s.h_status : CZ_ERR_CUDA;
      for (uint64_t t : s.tickets) {
        Req &q = reqs_[t];
        q.state = CZ_REQ_DONE;
        q.result = res;
        q.t_done = now;
      }
      ranges_->give(s.ws_off, s.ws_len);
      s.busy = false;
      s.tickets.clear();
      any = true;
    }
    if (any) done_cv_.notify_all();
    return any;
  }

  // run requests `ts` (one, or several compress requests of one group) on
  // slot s with workspace [off, off + len) of the pool (mu_ held)
  void launch(Slot &s, const std::vector<uint64_t> &ts, size_t off, size_t len)
  {
    unsigned char *ws = reinterpret_cast<unsigned char *>(pool_) + off;
    int r = CZ_OK;
    Req &q0 = reqs_[ts[0]];
    if (ts.size() == 1 && q0.r.op == CZ_OP_COMPRESS) {
      r = cz_compress(&q0.p, q0.r.d_in, q0.r.d_out, q0.r.out_cap, q0.r.d_out_bytes, ws, len, s.stream);
    } else if (ts.size() == 1) {
      r = cz_decompress(q0.r.d_in, q0.r.in_bytes, q0.r.h_header, q0.r.d_out, q0.r.out_cap, ws, len, s.stream);
    } else {
      const int n = (int)ts.size();
      std::vector<cz_params> ps(n);
      std::vector<const void *> in(n);
      std::vector<void *> out(n);
      std::vector<size_t> cap(n);
      for (int i = 0; i < n; ++i) {
        Req &q = reqs_[ts[i]];
        ps[i] = q.p;
        in[i] = q.r.d_in;
        out[i] = q.r.d_out;
        cap[i] = q.r.out_cap;
      }
      // stream lengths land in the first 256 bytes of the range, then go
      // to each request's own counter
      uint64_t *lens = reinterpret_cast<uint64_t *>(ws);
      r = cz_compress_batch(n, ps.data(), in.data(), out.data(), cap.data(), lens, ws + 256, len - 256, s.stream);
      for (int i = 0; i < n && r == CZ_OK; ++i) {
        Req &q = reqs_[ts[i]];
        if (q.r.d_out_bytes &&
            cudaMemcpyAsync(q.r.d_out_bytes, lens + i, 8, cudaMemcpyDeviceToDevice, s.stream) != cudaSuccess)
          r = CZ_ERR_CUDA;
      }
      ws += 256;
    }
    if (r == CZ_OK && cudaMemcpyAsync(s.h_status, ws, 4, cudaMemcpyDeviceToHost, s.stream) != cudaSuccess)
      r = CZ_ERR_CUDA;
    if (r == CZ_OK && cudaEventRecord(s.done, s.stream) != cudaSuccess) r = CZ_ERR_CUDA;
    if (r != CZ_OK) {  // nothing (more) runs for these: finish them now
      cudaStreamSynchronize(s.stream);
      for (uint64_t t : ts) {
        Req &q = reqs_[t];
        q.state = CZ_REQ_DONE;
        q.result = r;
        q.t_done = Clock::now();
      }
      ranges_->give(off, len);
      done_cv_.notify_all();
      return;
    }
    for (uint64_t t : ts) reqs_[t].state = CZ_REQ_RUNNING;
    s.busy = true;
    s.tickets = ts;
    s.ws_off = off;
    s.ws_len = len;
  }

  // admit waiting requests in arrival order (mu_ held)
  bool admit()
  {
    bool any = false;
    bool blocked = false;  // an old request is waiting for memory: no overtaking
    for (auto it = queue_.begin(); it != queue_.end();) {
      Slot *free_slot = nullptr;
      for (Slot &s : slots_)
        if (!s.busy) {
          free_slot = &s;
          break;
        }
      if (!free_slot) break;
      Req &q = reqs_[*it];
      std::vector<uint64_t> group{q.ticket};
      size_t len = q.ws;
      if (q.r.op == CZ_OP_COMPRESS) {
        // continuous batching: later compress requests of the same group
        std::vector<cz_params> ps{q.p};
        for (auto jt = std::next(it); jt != queue_.end() && (int)group.size() < MAX_GROUP; ++jt) {
          Req &o = reqs_[*jt];
          if (o.r.op != CZ_OP_COMPRESS || !same_group(o.p, q.p)) continue;
          ps.push_back(o.p);
          size_t need = 0;
          if (cz_batch_workspace_size((int)ps.size(), ps.data(), &need) != CZ_OK || need + 256 > budget_ / 2) {
            ps.pop_back();
            break;
          }
          group.push_back(o.ticket);
        }
        if (group.size() > 1) {
          size_t need = 0;
          cz_batch_workspace_size((int)ps.size(), ps.data(), &need);
          len = need + 256;
        }
      }
      size_t off = 0;
      bool ok = !blocked && ranges_->take(len, &off);
      if (!ok && group.size() > 1) {  // try it alone
        group.resize(1);
        len = q.ws;
        ok = !blocked && ranges_->take(len, &off);
      }
      if (!ok) {
        if (Clock::now() - q.t_submit > STARVE_LIMIT) blocked = true;
        ++it;
        continue;
      }
      // remove the launched requests from the queue
      for (size_t g = 1; g < group.size(); ++g) {
        for (auto jt = std::next(it); jt != queue_.end(); ++jt)
          if (*jt == group[g]) {
            queue_.erase(jt);
            break;
          }
      }
      it = queue_.erase(it);
      launch(*free_slot, group, off, len);
      any = true;
    }
    return any;
  }

  void loop()
  {
    cudaSetDevice(dev_);
    std::unique_lock<std::mutex> lock(mu_);
    Clock::time_point active = Clock::now();  // the last admission, retirement or arrival
    for (;;) {
      arrived_.store(false, std::memory_order_relaxed);
      const bool r = retire();
      const bool a = admit();
      bool busy = false;
      for (Slot &s : slots_) busy |= s.busy;
      if (stop_ && !busy && queue_.empty()) break;
      const Clock::time_point now = Clock::now();
      if (r || a) active = now;
      if (r || a) continue;
      if (busy || now - active < IDLE_SPIN) {
        // poll: let submitters and pollers take the lock, then look again
        // (events, arrivals) without sleeping
        lock.unlock();
        for (int i = 0; i < 64 && !arrived_.load(std::memory_order_acquire); ++i) std::this_thread::yield();
        lock.lock();
        if (arrived_.load(std::memory_order_relaxed)) active = Clock::now();
      } else {
        cv_.wait_for(lock, std::chrono::milliseconds(5));  // idle: sleep until a submit
        active = Clock::now();
      }
    }
  }

  int dev_ = 0;
  size_t budget_ = 0;
  void *pool_ = nullptr;
  Ranges *ranges_ = nullptr;
  std::vector<Slot> slots_;
  std::thread worker_;
  std::mutex mu_;
  std::condition_variable cv_, done_cv_;
  bool stop_ = false;
  std::atomic<bool> arrived_{false};  // a submit since the worker last looked
  uint64_t next_ = 0;
  std::unordered_map<uint64_t, Req> reqs_;
  std::list<uint64_t> queue_;  // arrival order; erasing one entry keeps the others' iterators
};

}  // namespace

int cz_server_create(size_t budget_bytes, int streams, void **server)
{
  if (!server || streams < 1 || streams > 64 || budget_bytes < (1u << 20)) return CZ_ERR_ARG;
  Server *s = new Server();
  const int r = s->init(budget_bytes, streams);
  if (r != CZ_OK) {
    delete s;
    return r;
  }
  *server = s;
  return CZ_OK;
}

int cz_server_submit(void *server, const cz_request *req, uint64_t *ticket)
{
  if (!server || !req || !ticket) return CZ_ERR_ARG;
  return static_cast<Server *>(server)->submit(req, ticket);
}

int cz_server_poll(void *server, uint64_t ticket, int *state, int *result, double *latency_ms)
{
  if (!server) return CZ_ERR_ARG;
  return static_cast<Server *>(server)->poll(ticket, state, result, latency_ms);
}

int cz_server_wait(void *server, uint64_t ticket, int *result, double *latency_ms)
{
  if (!server) return CZ_ERR_ARG;
  return static_cast<Server *>(server)->wait(ticket, result, latency_ms);
}

int cz_server_destroy(void *server)
{
  if (!server) return CZ_ERR_ARG;
  delete static_cast<Server *>(server);
  return CZ_OK;
}
