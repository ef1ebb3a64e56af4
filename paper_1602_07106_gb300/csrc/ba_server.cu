// ba_server.cu -- serving edge-range requests with continuous batching.
//
// Output buffers come from one device arena of `memory_budget_bytes`, handed out
// first-fit; a queued request is admitted (FIFO) when max_active allows and its
// 16*(edge_end-edge_begin) bytes fit in the arena.  A scheduler thread runs ticks: each
// tick packs the next chunk (<= chunk_edges) of every admitted request into one batched
// launch per position path (the k_generate_refill<..., Batched> kernel, output offsets
// pointing into the arena), so requests that arrive while others run join the next tick
// and their work overlaps on the device.  Up to max_inflight_ticks ticks are enqueued
// ahead of the GPU.  A host callback at the end of each tick marks the requests whose last
// chunk it carried as DONE and stamps their completion time.  A request's edge i is a
// pure function of (seed, n, d, n0, i), so its bits equal those of a plain call whatever
// else shares its ticks.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ba_internal.h"

using namespace ba;

namespace {

uint64_t now_ns() {
  return static_cast<uint64_t>(std::chrono::duration_cast<std::chrono::nanoseconds>(
                                   std::chrono::steady_clock::now().time_since_epoch())
                                   .count());
}

// First-fit allocator over [0, capacity) edges of the arena, coalescing on free.
class Arena {
 public:
  void reset(uint64_t cap) {
    free_.clear();
    if (cap) free_[0] = cap;
    used_ = 0;
  }
  bool alloc(uint64_t len, uint64_t *off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= len) {
        *off = it->first;
        const uint64_t rest = it->second - len;
        const uint64_t at = it->first + len;
        free_.erase(it);
        if (rest) free_[at] = rest;
        used_ += len;
        return true;
      }
    }
    return false;
  }
  void release(uint64_t off, uint64_t len) {
    used_ -= len;
    auto it = free_.emplace(off, len).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }
  uint64_t used() const { return used_; }

 private:
  std::map<uint64_t, uint64_t> free_;
  uint64_t used_ = 0;
};

struct Request {
  ba_graph_desc desc{};
  uint64_t len = 0;
  uint64_t cursor = 0;  // edges already issued
  uint64_t arena_off = 0;
  int32_t state = BA_REQ_QUEUED;
  bool admitted = false;
  uint64_t t_submit = 0, t_done = 0;
};

struct TickSlot {
  bool busy = false;
  GraphDev *host_tab = nullptr;  // pinned: 2 tables of max_active graphs
  uint64_t *host_prefix = nullptr;
  GraphDev *dev_tab = nullptr;
  uint64_t *dev_prefix = nullptr;
  unsigned long long *dev_counter = nullptr;
  std::vector<uint64_t> completing;  // tickets whose last chunk is in this tick
  struct ba_server *server = nullptr;
};

}  // namespace

struct ba_server {
  ba_server_config cfg{};
  int device = 0;
  cudaStream_t stream = nullptr;
  int64_t *arena_base = nullptr;
  uint64_t arena_edges = 0;
  Arena arena;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Request> reqs;
  std::vector<uint64_t> running;  // admitted, chunks left to issue
  std::vector<TickSlot> slots;
  int inflight = 0;
  uint64_t next_ticket = 1;
  bool stop = false;
  bool failed = false;
  ba_server_stats stats{};
  std::thread worker;
};

namespace {

void CUDART_CB on_tick_done(void *arg) {
  TickSlot *slot = static_cast<TickSlot *>(arg);
  ba_server *s = slot->server;
  const uint64_t t = now_ns();
  {
    std::lock_guard<std::mutex> lock(s->mu);
    for (uint64_t ticket : slot->completing) {
      auto it = s->reqs.find(ticket);
      if (it == s->reqs.end()) continue;
      it->second.state = BA_REQ_DONE;
      it->second.t_done = t;
      s->stats.completed++;
    }
    slot->completing.clear();
    slot->busy = false;
    s->inflight--;
  }
  s->cv.notify_all();
}

// Admits queued requests in FIFO order while slots and arena space allow.  Holds mu.
void admit(ba_server *s) {
  while (!s->queue.empty() && static_cast<int>(s->running.size()) < s->cfg.max_active) {
    Request &r = s->reqs[s->queue.front()];
    uint64_t off = 0;
    if (!s->arena.alloc(r.len, &off)) break;
    r.arena_off = off;
    r.admitted = true;
    r.state = BA_REQ_RUNNING;
    s->running.push_back(s->queue.front());
    s->queue.pop_front();
    s->stats.admitted++;
  }
}

// Packs the next chunk of every running request into the slot's pinned tables.  Holds mu.
struct TickPlan {
  int cnt[2] = {0, 0};
  bool seed[2] = {false, false};
  Shape shape[2];
};

void prepare_tick(ba_server *s, TickSlot &slot, TickPlan &plan) {
  const int cap = s->cfg.max_active;
  GraphDev *tab[2] = {slot.host_tab, slot.host_tab + cap};
  uint64_t *pre[2] = {slot.host_prefix, slot.host_prefix + (cap + 1)};
  pre[0][0] = pre[1][0] = 0;
  plan.shape[0] = shape_for(BA_KIND_BATCH, true);
  plan.shape[1] = shape_for(BA_KIND_BATCH, false);
  // With a tick budget, the requests with the least work left go first and the budget is
  // handed out in that order (the first always gets work); the rest wait for a later tick.
  // The budget holds only while no request waits for admission: it bounds the tick a short
  // request arriving at a light load waits behind, and when requests queue up (a saturated
  // server) full ticks keep the per-tick overhead small.
  const bool budgeted = s->cfg.tick_edges > 0 && s->queue.empty();
  if (budgeted)
    std::stable_sort(s->running.begin(), s->running.end(), [&](uint64_t x, uint64_t y) {
      const Request &rx = s->reqs[x], &ry = s->reqs[y];
      return rx.len - rx.cursor < ry.len - ry.cursor;
    });
  std::vector<uint64_t> take(s->running.size(), 0);  // edges of each request in this tick
  uint64_t budget = budgeted ? s->cfg.tick_edges : ~0ull;
  for (size_t k = 0; k < s->running.size() && budget > 0; ++k) {
    const Request &r = s->reqs[s->running[k]];
    take[k] = std::min({r.len - r.cursor, s->cfg.chunk_edges, budget});
    budget -= take[k];
  }
  // This tick's work per position path, then tiles sized to it (a light tick still spreads
  // over the GPU; see adapt_tile).
  uint64_t work[2] = {0, 0};
  for (size_t k = 0; k < s->running.size(); ++k) {
    if (take[k] == 0) continue;
    const Request &r = s->reqs[s->running[k]];
    const uint64_t a = r.desc.edge_begin + r.cursor;
    work[a + take[k] <= (1ull << 31) ? 0 : 1] += take[k];
  }
  plan.shape[0].tile = adapt_tile(work[0], plan.shape[0]);
  plan.shape[1].tile = adapt_tile(work[1], plan.shape[1]);
  const uint64_t tiles[2] = {static_cast<uint64_t>(plan.shape[0].tile),
                             static_cast<uint64_t>(plan.shape[1].tile)};
  std::vector<uint64_t> still;
  slot.completing.clear();
  uint64_t edges = 0;
  for (size_t k = 0; k < s->running.size(); ++k) {
    const uint64_t ticket = s->running[k];
    Request &r = s->reqs[ticket];
    if (take[k] == 0) {  // no budget left in this tick
      still.push_back(ticket);
      continue;
    }
    const uint64_t a = r.desc.edge_begin + r.cursor;
    const uint64_t b = a + take[k];
    const int path = b <= (1ull << 31) ? 0 : 1;
    GraphDev g = make_graph_dev(r.desc.seed, r.desc.n, r.desc.d, r.desc.n0, a, b);
    g.out_edge = r.arena_off + r.cursor;
    const int c = plan.cnt[path]++;
    g.tile0 = pre[path][c];
    tab[path][c] = g;
    pre[path][c + 1] = pre[path][c] + (b - a + tiles[path] - 1) / tiles[path];
    plan.seed[path] |= g.m0 > 0;
    r.cursor += b - a;
    edges += b - a;
    if (r.cursor == r.len) slot.completing.push_back(ticket);
    else still.push_back(ticket);
  }
  s->running.swap(still);
  slot.busy = true;
  s->inflight++;
  s->stats.ticks++;
  s->stats.edges_done += edges;
}

// Enqueues a prepared tick: table uploads, one batched launch per position path and the
// completion callback.  Called WITHOUT mu (the callback takes it).
ba_status enqueue_tick(ba_server *s, TickSlot &slot, const TickPlan &plan) {
  const int cap = s->cfg.max_active;
  for (int path = 0; path < 2; ++path) {
    const int cnt = plan.cnt[path];
    if (cnt == 0) continue;
    GraphDev *htab = slot.host_tab + path * cap;
    uint64_t *hpre = slot.host_prefix + path * (cap + 1);
    GraphDev *dtab = slot.dev_tab + path * cap;
    uint64_t *dpre = slot.dev_prefix + path * (cap + 1);
    cudaError_t e;
    if ((e = cudaMemcpyAsync(dtab, htab, cnt * sizeof(GraphDev), cudaMemcpyHostToDevice,
                             s->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(dpre, hpre, (cnt + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice,
                             s->stream)) != cudaSuccess)
      return cuda_fail(e, "cudaMemcpyAsync");
    BatchTable bt{dtab, dpre, cnt};
    ba_status st = launch_batch(bt, hpre[cnt], path == 0, plan.seed[path], s->arena_base,
                                plan.shape[path], slot.dev_counter + path * 32,
                                s->stream);
    if (st != BA_OK) return st;
  }
  cudaError_t e = cudaLaunchHostFunc(s->stream, on_tick_done, &slot);
  if (e != cudaSuccess) return cuda_fail(e, "cudaLaunchHostFunc");
  return BA_OK;
}

void worker_loop(ba_server *s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop) {
    admit(s);
    TickSlot *free_slot = nullptr;
    if (!s->running.empty() && s->inflight < s->cfg.max_inflight_ticks) {
      for (auto &slot : s->slots)
        if (!slot.busy) {
          free_slot = &slot;
          break;
        }
    }
    if (free_slot && !s->failed) {
      TickPlan plan;
      prepare_tick(s, *free_slot, plan);
      lk.unlock();
      const ba_status st = enqueue_tick(s, *free_slot, plan);
      lk.lock();
      if (st != BA_OK) {
        s->failed = true;  // mark everything still pending as failed
        for (auto &kv : s->reqs)
          if (kv.second.state == BA_REQ_RUNNING || kv.second.state == BA_REQ_QUEUED)
            kv.second.state = BA_REQ_FAILED;
        s->running.clear();
        s->queue.clear();
        s->cv.notify_all();
      }
      continue;
    }
    s->cv.wait_for(lk, std::chrono::milliseconds(5));
  }
}

}  // namespace

extern "C" {

ba_status ba_server_create(const ba_server_config *cfg, ba_server **server) {
  set_error("");
  if (!server) {
    set_error("server output pointer is NULL");
    return BA_ERR_INVALID_ARG;
  }
  *server = nullptr;
  ba_server *s = new (std::nothrow) ba_server();
  if (!s) return BA_ERR_NOMEM;
  if (cfg) s->cfg = *cfg;
  if (s->cfg.max_active > 65536 || s->cfg.max_inflight_ticks > 64 || s->cfg.max_queued < 0) {
    delete s;
    set_error("server config: max_active <= 65536, max_inflight_ticks <= 64, max_queued >= 0");
    return BA_ERR_INVALID_ARG;
  }
  if (s->cfg.device < 0) cudaGetDevice(&s->device); else s->device = s->cfg.device;
  if (s->cfg.chunk_edges == 0) s->cfg.chunk_edges = 1ull << 24;
  if (s->cfg.max_active <= 0) s->cfg.max_active = 256;
  if (s->cfg.max_inflight_ticks <= 0) s->cfg.max_inflight_ticks = 2;
  cudaError_t e = cudaSetDevice(s->device);
  if (e != cudaSuccess) {
    delete s;
    return cuda_fail(e, "cudaSetDevice");
  }
  if (s->cfg.memory_budget_bytes == 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    s->cfg.memory_budget_bytes = fr / 2;
  }
  s->arena_edges = s->cfg.memory_budget_bytes / 16;
  ba_status st = BA_OK;
  if ((count_device_allocation(), e = cudaMalloc(&s->arena_base, std::max<uint64_t>(s->arena_edges, 1) * 16)) != cudaSuccess) {
    st = e == cudaErrorMemoryAllocation ? BA_ERR_NOMEM : cuda_fail(e, "cudaMalloc(arena)");
  } else if ((e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking)) != cudaSuccess) {
    st = cuda_fail(e, "cudaStreamCreateWithFlags");
  }
  s->arena.reset(s->arena_edges);
  const int cap = s->cfg.max_active;
  s->slots.resize(s->cfg.max_inflight_ticks);
  for (auto &slot : s->slots) {
    slot.server = s;
    if (st != BA_OK) break;
    if ((e = cudaMallocHost(&slot.host_tab, 2 * cap * sizeof(GraphDev))) != cudaSuccess ||
        (e = cudaMallocHost(&slot.host_prefix, 2 * (cap + 1) * sizeof(uint64_t))) != cudaSuccess ||
        (count_device_allocation(), e = cudaMalloc(&slot.dev_tab, 2 * cap * sizeof(GraphDev))) != cudaSuccess ||
        (count_device_allocation(), e = cudaMalloc(&slot.dev_prefix, 2 * (cap + 1) * sizeof(uint64_t))) != cudaSuccess ||
        (count_device_allocation(), e = cudaMalloc(&slot.dev_counter, 512)) != cudaSuccess)
      st = e == cudaErrorMemoryAllocation ? BA_ERR_NOMEM : cuda_fail(e, "server tick tables");
  }
  if (st != BA_OK) {
    ba_server_destroy(s);
    return st;
  }
  s->worker = std::thread(worker_loop, s);
  *server = s;
  return BA_OK;
}

ba_status ba_server_submit(ba_server *s, const ba_graph_desc *req, uint64_t *ticket) {
  set_error("");
  if (!s || !req || !ticket) {
    set_error("NULL server, request or ticket");
    return BA_ERR_INVALID_ARG;
  }
  uint64_t m = 0;
  ba_status st = validate_graph(req->n, req->d, req->n0, &m);
  if (st != BA_OK) return st;
  if (req->edge_begin > req->edge_end || req->edge_end > m) {
    set_error("request edge range outside 0..m");
    return BA_ERR_RANGE;
  }
  const uint64_t len = req->edge_end - req->edge_begin;
  if (len > s->arena_edges) {
    set_error("request larger than the server's memory budget");
    return BA_ERR_NOMEM;
  }
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->failed) {
      set_error("server stopped after a CUDA error");
      return BA_ERR_CUDA;
    }
    if (len > 0 && s->cfg.max_queued > 0 && s->queue.size() >= static_cast<size_t>(s->cfg.max_queued)) {
      s->stats.rejected_busy++;
      set_error("admission queue full (max_queued)");
      return BA_ERR_BUSY;
    }
    const uint64_t t = s->next_ticket++;
    Request r;
    r.desc = *req;
    r.len = len;
    r.t_submit = now_ns();
    if (len == 0) {
      r.state = BA_REQ_DONE;
      r.t_done = r.t_submit;
      s->stats.completed++;
    }
    s->reqs.emplace(t, r);
    if (len > 0) s->queue.push_back(t);
    s->stats.submitted++;
    *ticket = t;
  }
  s->cv.notify_all();
  return BA_OK;
}

ba_status ba_server_poll(ba_server *s, uint64_t ticket, int32_t *state, uint64_t *latency_ns) {
  if (!s || !state) {
    set_error("NULL server or state");
    return BA_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) {
    set_error("unknown ticket");
    return BA_ERR_NOT_FOUND;
  }
  *state = it->second.state;
  if (latency_ns)
    *latency_ns = it->second.state == BA_REQ_DONE ? it->second.t_done - it->second.t_submit : 0;
  return BA_OK;
}

ba_status ba_server_wait(ba_server *s, uint64_t ticket, int64_t timeout_ms) {
  if (!s) {
    set_error("NULL server");
    return BA_ERR_INVALID_ARG;
  }
  std::unique_lock<std::mutex> lk(s->mu);
  // clamped so that the deadline cannot overflow the clock (2^40 ms is 35 years)
  const int64_t ms = std::min<int64_t>(std::max<int64_t>(timeout_ms, 0), int64_t{1} << 40);
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(ms);
  for (;;) {
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) {
      set_error("unknown ticket");
      return BA_ERR_NOT_FOUND;
    }
    if (it->second.state == BA_REQ_DONE) return BA_OK;
    if (it->second.state == BA_REQ_FAILED) {
      set_error("request failed");
      return BA_ERR_CUDA;
    }
    if (s->cv.wait_until(lk, deadline) == std::cv_status::timeout) {
      auto again = s->reqs.find(ticket);
      if (again != s->reqs.end() && again->second.state == BA_REQ_DONE) return BA_OK;
      set_error("wait timed out");
      return BA_ERR_TIMEOUT;
    }
  }
}

ba_status ba_server_result(ba_server *s, uint64_t ticket, const int64_t **out_dev, uint64_t *n_edges) {
  if (!s || !out_dev || !n_edges) {
    set_error("NULL argument");
    return BA_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) {
    set_error("unknown ticket");
    return BA_ERR_NOT_FOUND;
  }
  if (it->second.state != BA_REQ_DONE) {
    set_error("request not done");
    return BA_ERR_BUSY;
  }
  *n_edges = it->second.len;
  *out_dev = it->second.len ? s->arena_base + 2 * it->second.arena_off : nullptr;
  return BA_OK;
}

ba_status ba_server_copy_result(ba_server *s, uint64_t ticket, int64_t *dst, void *stream) {
  const int64_t *src = nullptr;
  uint64_t k = 0;
  ba_status st = ba_server_result(s, ticket, &src, &k);
  if (st != BA_OK) return st;
  if (k == 0) return BA_OK;
  if (!dst) {
    set_error("NULL destination");
    return BA_ERR_INVALID_ARG;
  }
  cudaError_t e = cudaMemcpyAsync(dst, src, k * 16, cudaMemcpyDefault, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? BA_OK : cuda_fail(e, "cudaMemcpyAsync");
}

ba_status ba_server_release(ba_server *s, uint64_t ticket) {
  if (!s) {
    set_error("NULL server");
    return BA_ERR_INVALID_ARG;
  }
  {
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) {
      set_error("unknown ticket");
      return BA_ERR_NOT_FOUND;
    }
    if (it->second.state != BA_REQ_DONE && it->second.state != BA_REQ_FAILED) {
      set_error("request still queued or running");
      return BA_ERR_BUSY;
    }
    if (it->second.admitted) s->arena.release(it->second.arena_off, it->second.len);
    s->reqs.erase(it);
    s->stats.released++;
  }
  s->cv.notify_all();
  return BA_OK;
}

ba_status ba_server_cancel(ba_server *s, uint64_t ticket) {
  if (!s) {
    set_error("NULL server");
    return BA_ERR_INVALID_ARG;
  }
  {
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) {
      set_error("unknown ticket");
      return BA_ERR_NOT_FOUND;
    }
    if (it->second.state != BA_REQ_QUEUED) {
      set_error(it->second.state == BA_REQ_RUNNING
                    ? "request already admitted: wait for it, then release it"
                    : "request finished: release it");
      return BA_ERR_BUSY;
    }
    // a QUEUED request holds no arena space and has no work on the device
    for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
      if (*q == ticket) {
        s->queue.erase(q);
        break;
      }
    s->reqs.erase(it);
    s->stats.cancelled++;
  }
  s->cv.notify_all();
  return BA_OK;
}

ba_status ba_server_stats_get(ba_server *s, ba_server_stats *out) {
  if (!s || !out) {
    set_error("NULL argument");
    return BA_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(s->mu);
  *out = s->stats;
  out->bytes_in_use = s->arena.used() * 16;
  out->queue_depth = s->queue.size();
  out->active = s->running.size();
  return BA_OK;
}

ba_status ba_server_destroy(ba_server *s) {
  if (!s) return BA_OK;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (auto &slot : s->slots) {
    if (slot.host_tab) cudaFreeHost(slot.host_tab);
    if (slot.host_prefix) cudaFreeHost(slot.host_prefix);
    if (slot.dev_tab) cudaFree(slot.dev_tab);
    if (slot.dev_prefix) cudaFree(slot.dev_prefix);
    if (slot.dev_counter) cudaFree(slot.dev_counter);
  }
  if (s->arena_base) cudaFree(s->arena_base);
  if (s->stream) cudaStreamDestroy(s->stream);
  delete s;
  return BA_OK;
}

}  // extern "C"
