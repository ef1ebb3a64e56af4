// ba_api.cu -- the C ABI of libba (include/ba.h): argument checks, per-call scratch and
// the launches of the plain entry points.
#include <atomic>
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "ba_draw.cuh"
#include "ba_internal.h"

namespace ba {

namespace {
thread_local std::string g_last_error;

// Per-call scratch from the stream-ordered allocator: freed on the same stream once the
// work enqueued before the free has run, so concurrent calls never share it.
// libba's own stream-ordered pool, one per device, created on first use and kept: it holds
// on to up to 64 MB between calls (the default pool returns everything at each
// synchronisation, and mapping it again costs more than a small call's kernel).
std::mutex g_pool_mutex;
std::vector<cudaMemPool_t> g_pools;

cudaError_t library_pool(cudaMemPool_t *out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_pool_mutex);
  if (g_pools.size() <= static_cast<size_t>(dev)) g_pools.resize(dev + 1, nullptr);
  if (g_pools[dev] == nullptr) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    e = cudaMemPoolCreate(&pool, &props);
    if (e != cudaSuccess) return e;
    uint64_t keep = 64ull << 20;
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) {
      cudaMemPoolDestroy(pool);
      return e;
    }
    g_pools[dev] = pool;
  }
  *out = g_pools[dev];
  return cudaSuccess;
}

struct StreamScratch {
  void *ptr = nullptr;
  cudaStream_t stream = nullptr;
  ba_status alloc(size_t bytes, cudaStream_t s) {
    stream = s;
    return pool_alloc(&ptr, bytes, s);
  }
  void release() {
    if (ptr) cudaFreeAsync(ptr, stream);
    ptr = nullptr;
  }
  ~StreamScratch() { release(); }
};

std::mutex g_sm_mutex;
std::vector<int> g_sm_counts;
}  // namespace

void set_error(const char *msg) { g_last_error = msg ? msg : ""; }

ba_status pool_alloc(void **ptr, size_t bytes, cudaStream_t s) {
  *ptr = nullptr;
  count_device_allocation();
  cudaMemPool_t pool = nullptr;
  cudaError_t e = library_pool(&pool);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemPoolCreate");
  e = cudaMallocFromPoolAsync(ptr, bytes, pool, s);
  if (e != cudaSuccess) {
    *ptr = nullptr;
    if (e != cudaErrorMemoryAllocation) return cuda_fail(e, "cudaMallocFromPoolAsync");
    set_error("cudaMallocFromPoolAsync: out of memory");
    return BA_ERR_NOMEM;
  }
  return BA_OK;
}

namespace {
std::atomic<unsigned long long> g_device_allocations{0};
}

void count_device_allocation() { g_device_allocations.fetch_add(1, std::memory_order_relaxed); }

int adapt_tile(uint64_t total_edges, const Shape &s) {
  const uint64_t warps = static_cast<uint64_t>(sm_count()) * std::max(s.ctas_per_sm, 1) *
                         std::max(s.block / 32, 1);
  int t = s.tile;
  while (t > 256 && total_edges / static_cast<uint64_t>(t) < 4 * warps) t >>= 1;
  return t;
}

ba_status cuda_fail(cudaError_t e, const char *where) {
  g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
  return BA_ERR_CUDA;
}

int sm_count() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  std::lock_guard<std::mutex> lock(g_sm_mutex);
  if (dev >= static_cast<int>(g_sm_counts.size())) g_sm_counts.resize(dev + 1, 0);
  if (g_sm_counts[dev] == 0) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    g_sm_counts[dev] = std::max(n, 1);
  }
  return g_sm_counts[dev];
}

ba_status validate_graph(uint64_t n, uint32_t d, uint64_t n0, uint64_t *m_out) {
  if (n == 0 || d == 0 || n0 > n) {
    set_error("graph parameters need n >= 1, d >= 1 and n0 <= n");
    return BA_ERR_INVALID_ARG;
  }
  const unsigned __int128 m0 = n0 > 0 ? (static_cast<unsigned __int128>(n0) * (n0 - 1)) / 2 : 0;
  const unsigned __int128 m = m0 + static_cast<unsigned __int128>(n - n0) * d;
  if (m > (static_cast<unsigned __int128>(1) << 62)) {
    set_error("m exceeds 2^62 edges: positions 2m would not fit 64 bits");
    return BA_ERR_OVERFLOW;
  }
  *m_out = static_cast<uint64_t>(m);
  return BA_OK;
}

GraphDev make_graph_dev(uint64_t seed, uint64_t n, uint32_t d, uint64_t n0, uint64_t begin,
                        uint64_t end) {
  GraphDev g{};
  g.seed = seed;
  g.seed_pre = seed_premix(seed);
  g.n = n;
  g.n0 = n0;
  g.m0 = n0 > 0 ? n0 * (n0 - 1) / 2 : 0;
  g.two_m0 = 2 * g.m0;
  g.begin = begin;
  g.end = end;
  g.out_edge = 0;
  g.tile0 = 0;
  g.d = d;
  const uint32_t l = d == 1 ? 0 : 32 - __builtin_clz(d - 1);  // ceil(log2 d)
  const unsigned __int128 one = 1;
  g.div.l = l;
  g.div.m64 = static_cast<uint64_t>(((one << (62 + l)) + d - 1) / d);
  g.div.m32 = static_cast<uint32_t>(((one << (31 + l)) + d - 1) / d);
  g.div.pow2 = (d & (d - 1)) == 0 ? 1u : 0u;
  return g;
}

}  // namespace ba

using namespace ba;

namespace {

ba_status check_range(uint64_t n, uint32_t d, uint64_t n0, uint64_t begin, uint64_t end,
                      uint64_t *m) {
  ba_status st = validate_graph(n, d, n0, m);
  if (st != BA_OK) return st;
  if (begin > end || end > *m) {
    set_error("edge range must satisfy edge_begin <= edge_end <= m");
    return BA_ERR_RANGE;
  }
  return BA_OK;
}

}  // namespace

extern "C" {

const char *ba_status_string(int status) {
  switch (status) {
    case BA_OK: return "ok";
    case BA_ERR_INVALID_ARG: return "invalid argument";
    case BA_ERR_RANGE: return "edge range outside 0..m";
    case BA_ERR_OVERFLOW: return "graph too large (m > 2^62)";
    case BA_ERR_CUDA: return "CUDA error";
    case BA_ERR_NOMEM: return "out of memory";
    case BA_ERR_TIMEOUT: return "timed out";
    case BA_ERR_BUSY: return "busy";
    case BA_ERR_NOT_FOUND: return "not found";
    default: return "unknown status";
  }
}

const char *ba_last_error_message(void) { return g_last_error.c_str(); }

int ba_version(void) { return 10000; }

uint64_t ba_device_allocations(void) { return g_device_allocations.load(std::memory_order_relaxed); }

uint64_t ba_num_edges(uint64_t n, uint32_t d, uint64_t n0) {
  uint64_t m = 0;
  std::string saved = g_last_error;
  ba_status st = validate_graph(n, d, n0, &m);
  g_last_error = saved;
  return st == BA_OK ? m : 0;
}

ba_status ba_generate_edges(uint64_t seed, uint64_t n, uint32_t d, uint64_t n0,
                            uint64_t edge_begin, uint64_t edge_end, int64_t *out_dev,
                            void *stream) {
  set_error("");
  uint64_t m = 0;
  ba_status st = check_range(n, d, n0, edge_begin, edge_end, &m);
  if (st != BA_OK) return st;
  if (edge_begin == edge_end) return BA_OK;
  if (out_dev == nullptr || (reinterpret_cast<uintptr_t>(out_dev) & 15) != 0) {
    set_error("out must be a non-NULL, 16-byte aligned device pointer");
    return BA_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const GraphDev g = make_graph_dev(seed, n, d, n0, edge_begin, edge_end);
  const Shape shape = shape_for(BA_KIND_GENERATE, edge_end <= (1ull << 31));
  StreamScratch scratch;
  if (shape.refill != 0) {
    st = scratch.alloc(sizeof(unsigned long long), s);
    if (st != BA_OK) return st;
  }
  return launch_generate(g, out_dev, shape, static_cast<unsigned long long *>(scratch.ptr), s);
}

ba_status ba_generate_edges_checked(uint64_t seed, uint64_t n, uint32_t d, uint64_t n0,
                                    uint64_t edge_begin, uint64_t edge_end, int64_t *out_dev,
                                    uint64_t out_capacity_edges, uint64_t *status_dev,
                                    void *stream) {
  set_error("");
  uint64_t m = 0;
  ba_status st = check_range(n, d, n0, edge_begin, edge_end, &m);
  if (st != BA_OK) return st;
  if (status_dev == nullptr || (reinterpret_cast<uintptr_t>(status_dev) & 7) != 0) {
    set_error("status must be a non-NULL, 8-byte aligned device pointer");
    return BA_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(status_dev, 0xff, sizeof(uint64_t), s);  // no violation yet
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  if (edge_begin == edge_end) return BA_OK;
  if (out_dev == nullptr || (reinterpret_cast<uintptr_t>(out_dev) & 15) != 0) {
    set_error("out must be a non-NULL, 16-byte aligned device pointer");
    return BA_ERR_INVALID_ARG;
  }
  const GraphDev g = make_graph_dev(seed, n, d, n0, edge_begin, edge_end);
  const Shape shape = shape_for(BA_KIND_GENERATE, edge_end <= (1ull << 31));
  StreamScratch scratch;
  st = scratch.alloc(sizeof(unsigned long long), s);
  if (st != BA_OK) return st;
  return launch_generate_checked(g, out_dev, out_capacity_edges,
                                 reinterpret_cast<unsigned long long *>(status_dev), shape,
                                 static_cast<unsigned long long *>(scratch.ptr), s);
}

ba_status ba_check_status(const uint64_t *status_dev, void *stream) {
  set_error("");
  if (status_dev == nullptr) {
    set_error("NULL status");
    return BA_ERR_INVALID_ARG;
  }
  uint64_t v = 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(&v, status_dev, sizeof v, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "reading the check status");
  if (v == ~0ull) return BA_OK;
  set_error(("device check: a store to output slot " + std::to_string(v) +
             " (edge offset from the start of out) was beyond the declared capacity; "
             "it and every later slot were skipped").c_str());
  return BA_ERR_CUDA;
}

ba_status ba_generate_edges32(uint64_t seed, uint64_t n, uint32_t d, uint64_t n0,
                              uint64_t edge_begin, uint64_t edge_end, int32_t *out_dev,
                              void *stream) {
  set_error("");
  uint64_t m = 0;
  ba_status st = check_range(n, d, n0, edge_begin, edge_end, &m);
  if (st != BA_OK) return st;
  if (n > (1ull << 31)) {
    set_error("int32 output needs every node ID below 2^31 (n <= 2^31)");
    return BA_ERR_INVALID_ARG;
  }
  if (edge_begin == edge_end) return BA_OK;
  if (out_dev == nullptr || (reinterpret_cast<uintptr_t>(out_dev) & 7) != 0) {
    set_error("out must be a non-NULL, 8-byte aligned device pointer");
    return BA_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const GraphDev g = make_graph_dev(seed, n, d, n0, edge_begin, edge_end);
  const Shape shape = shape_for(BA_KIND_GENERATE, edge_end <= (1ull << 31));
  StreamScratch scratch;
  if (shape.refill != 0) {
    st = scratch.alloc(sizeof(unsigned long long), s);
    if (st != BA_OK) return st;
  }
  return launch_generate(g, reinterpret_cast<int64_t *>(out_dev), shape,
                         static_cast<unsigned long long *>(scratch.ptr), s, true);
}

ba_status ba_degree_count_range(uint64_t seed, uint64_t n, uint32_t d, uint64_t n0,
                                uint64_t edge_begin, uint64_t edge_end, uint64_t node_limit,
                                uint64_t *counts_dev, int accumulate, void *stream) {
  set_error("");
  uint64_t m = 0;
  ba_status st = check_range(n, d, n0, edge_begin, edge_end, &m);
  if (st != BA_OK) return st;
  if (node_limit == 0) return BA_OK;
  if (counts_dev == nullptr || (reinterpret_cast<uintptr_t>(counts_dev) & 7) != 0) {
    set_error("counts must be a non-NULL, 8-byte aligned device pointer");
    return BA_ERR_INVALID_ARG;
  }
  if (node_limit > (1ull << 40)) {
    set_error("node_limit above 2^40 counters");
    return BA_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const GraphDev g = make_graph_dev(seed, n, d, n0, edge_begin, edge_end);
  const Shape shape = shape_for(BA_KIND_DEGREE, edge_end <= (1ull << 31));
  StreamScratch scratch;
  st = scratch.alloc(sizeof(unsigned long long), s);
  if (st != BA_OK) return st;
  return launch_degree(g, node_limit, counts_dev, accumulate, shape,
                       static_cast<unsigned long long *>(scratch.ptr), s);
}

ba_status ba_degree_count(uint64_t seed, uint64_t n, uint32_t d, uint64_t node_limit,
                          uint64_t *counts_dev, void *stream) {
  uint64_t m = 0;
  ba_status st = validate_graph(n, d, 0, &m);
  if (st != BA_OK) return st;
  return ba_degree_count_range(seed, n, d, 0, 0, m, node_limit, counts_dev, 0, stream);
}

// Checks the variant flags against the graph: known bits only, a seed edge for the
// self-loop-free rule, and the limits of the rejection of parallel edges.
static ba_status check_variant(uint32_t variant, uint32_t d, uint64_t n0) {
  if ((variant & ~static_cast<uint32_t>(BA_VARIANT_CRC_HASH | BA_VARIANT_NO_SELF_LOOPS |
                                        BA_VARIANT_NO_PARALLEL_EDGES)) != 0) {
    set_error("unknown variant flag");
    return BA_ERR_INVALID_ARG;
  }
  if ((variant & BA_VARIANT_NO_SELF_LOOPS) && n0 < 2) {
    set_error("the self-loop-free graph needs a seed graph with an edge (n0 >= 2)");
    return BA_ERR_INVALID_ARG;
  }
  if ((variant & BA_VARIANT_NO_PARALLEL_EDGES) && ((variant & BA_VARIANT_CRC_HASH) || d > 1024)) {
    set_error("rejecting parallel edges needs d <= 1024 and the SplitMix64 hash");
    return BA_ERR_INVALID_ARG;
  }
  return BA_OK;
}

// Edges per chunk of the degree count without parallel edges (16 bytes each of scratch).
constexpr uint64_t kRejectCountChunk = 1ull << 27;

static_assert(BA_VARIANT_CRC_HASH == kVariantCrc && BA_VARIANT_NO_SELF_LOOPS == kVariantNoLoop,
              "public variant flags and kernel policies disagree");

// Section 4's graph without parallel edges through the fold (d a power of two <= 32): the
// generate kernel with the detecting chunk flush, then the exact pass over the nodes it
// listed.  Edge lists: one launch over the range, writing edge c at slot c - begin of out,
// with a list of (range >> 6) + 2^20 entries at most; should more nodes be listed, the
// exact pass takes every node instead.  Counting (out == nullptr): launches of at most
// 2^25 nodes' edges, each with a list that holds all of its nodes, since the flush has
// already counted the nodes it did not list.
static ba_status fold_range(uint64_t seed, uint64_t n, uint32_t d, uint64_t n0, uint64_t begin,
                            uint64_t end, int64_t *out, uint64_t *counts, uint64_t node_limit,
                            bool no_loops, cudaStream_t s) {
  const uint64_t m0 = n0 > 0 ? n0 * (n0 - 1) / 2 : 0;
  const uint64_t span = out ? end - begin : (1ull << 25) * d;
  const uint64_t nodes = std::min(end - begin, span) / d + 2;  // nodes a launch can list
  const uint64_t cap = out ? std::min<uint64_t>(nodes, ((end - begin) >> 6) + (1ull << 20)) : nodes;
  Shape shape = shape_for(BA_KIND_GENERATE, end <= (1ull << 31));
  shape.refill = 1;
  StreamScratch list, count, counter;
  ba_status st;
  if ((st = list.alloc(cap * sizeof(uint32_t), s)) != BA_OK) return st;
  if ((st = count.alloc(sizeof(unsigned long long), s)) != BA_OK) return st;
  if ((st = counter.alloc(sizeof(unsigned long long), s)) != BA_OK) return st;
  uint32_t *lst = static_cast<uint32_t *>(list.ptr);
  unsigned long long *cnt = static_cast<unsigned long long *>(count.ptr);
  for (uint64_t c0 = begin; c0 < end; c0 += span) {
    const uint64_t c1 = std::min(end, c0 + span);
    GraphDev gc = make_graph_dev(seed, n, d, n0, c0, c1);
    gc.out_edge = c0 - begin;
    const uint64_t lo = std::max(c0, m0);  // the launch's first node edge
    const uint64_t q0 = lo < c1 ? (lo - m0) / d : 0;
    const uint64_t q_hi = lo < c1 ? (c1 - 1 - m0) / d : 0;
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    st = launch_generate_fold(gc, out, shape, static_cast<unsigned long long *>(counter.ptr), s,
                              no_loops, lst, cnt, q0, cap, counts, node_limit);
    if (st != BA_OK) return st;
    if (lo >= c1) continue;  // seed-clique edges only: no node to finish
    st = launch_reject_listed(gc, out, counts, node_limit, lst, cnt, cap, q0, q_hi, s, no_loops);
    if (st != BA_OK) return st;
  }
  return BA_OK;
}

ba_status ba_generate_edges_variant(uint64_t seed, uint64_t n, uint32_t d, uint64_t n0,
                                    uint64_t edge_begin, uint64_t edge_end, uint32_t variant,
                                    int64_t *out_dev, void *stream) {
  set_error("");
  uint64_t m = 0;
  ba_status st = check_range(n, d, n0, edge_begin, edge_end, &m);
  if (st != BA_OK) return st;
  st = check_variant(variant, d, n0);
  if (st != BA_OK) return st;
  if (edge_begin == edge_end) return BA_OK;
  if (out_dev == nullptr || (reinterpret_cast<uintptr_t>(out_dev) & 15) != 0) {
    set_error("out must be a non-NULL, 16-byte aligned device pointer");
    return BA_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((variant & BA_VARIANT_NO_PARALLEL_EDGES) && fold_supported(d))
    return fold_range(seed, n, d, n0, edge_begin, edge_end, out_dev, nullptr, 0,
                      (variant & BA_VARIANT_NO_SELF_LOOPS) != 0, s);
  const GraphDev g = make_graph_dev(seed, n, d, n0, edge_begin, edge_end);
  Shape shape = shape_for(BA_KIND_GENERATE, edge_end <= (1ull << 31));
  shape.refill = 1;  // the variant draws run on the refill kernel only
  StreamScratch scratch;
  st = scratch.alloc(sizeof(unsigned long long), s);
  if (st != BA_OK) return st;
  const uint32_t draw_flags = variant & (BA_VARIANT_CRC_HASH | BA_VARIANT_NO_SELF_LOOPS);
  st = launch_generate_variant(g, out_dev, shape, static_cast<unsigned long long *>(scratch.ptr), s,
                               draw_flags);
  if (st != BA_OK || !(variant & BA_VARIANT_NO_PARALLEL_EDGES)) return st;
  return launch_reject_duplicates(g, out_dev, s, (variant & BA_VARIANT_NO_SELF_LOOPS) != 0);
}

ba_status ba_degree_count_variant(uint64_t seed, uint64_t n, uint32_t d, uint64_t n0,
                                  uint64_t edge_begin, uint64_t edge_end, uint64_t node_limit,
                                  uint32_t variant, uint64_t *counts_dev, int accumulate,
                                  void *stream) {
  set_error("");
  uint64_t m = 0;
  ba_status st = check_range(n, d, n0, edge_begin, edge_end, &m);
  if (st != BA_OK) return st;
  st = check_variant(variant, d, n0);
  if (st != BA_OK) return st;
  if (node_limit == 0) return BA_OK;
  if (counts_dev == nullptr || (reinterpret_cast<uintptr_t>(counts_dev) & 7) != 0) {
    set_error("counts must be a non-NULL, 8-byte aligned device pointer");
    return BA_ERR_INVALID_ARG;
  }
  if (node_limit > (1ull << 40)) {
    set_error("node_limit above 2^40 counters");
    return BA_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const GraphDev g = make_graph_dev(seed, n, d, n0, edge_begin, edge_end);
  const uint32_t draw_flags = variant & (BA_VARIANT_CRC_HASH | BA_VARIANT_NO_SELF_LOOPS);
  if (!(variant & BA_VARIANT_NO_PARALLEL_EDGES) || d == 1) {  // d = 1: nothing to reject
    Shape shape = shape_for(BA_KIND_DEGREE, edge_end <= (1ull << 31));
    shape.refill = 1;
    StreamScratch scratch;
    st = scratch.alloc(sizeof(unsigned long long), s);
    if (st != BA_OK) return st;
    return launch_degree_variant(g, node_limit, counts_dev, accumulate, shape,
                                 static_cast<unsigned long long *>(scratch.ptr), s, draw_flags);
  }
  // Without parallel edges: the sources in closed form, then chunk by chunk the array's
  // targets written by the generate kernel into library scratch and each edge's final
  // target (after section 4's rejections) counted by the rejection pass -- every chain
  // runs once, in the refill scheduler.
  st = launch_degree_sources(g, node_limit, counts_dev, accumulate, s);
  if (st != BA_OK) return st;
  const uint64_t a = std::max(edge_begin, g.m0);
  if (a >= edge_end) return BA_OK;
  if (fold_supported(d))  // no edge stored: the fold counts as it generates
    return fold_range(seed, n, d, n0, a, edge_end, nullptr, counts_dev, node_limit,
                      (variant & BA_VARIANT_NO_SELF_LOOPS) != 0, s);
  const uint64_t chunk = std::min<uint64_t>(edge_end - a, kRejectCountChunk);
  StreamScratch pairs, counter;
  if ((st = pairs.alloc(chunk * 16, s)) != BA_OK) return st;
  if ((st = counter.alloc(sizeof(unsigned long long), s)) != BA_OK) return st;
  const Shape gshape = shape_for(BA_KIND_GENERATE, edge_end <= (1ull << 31));
  int64_t *buf = static_cast<int64_t *>(pairs.ptr);
  for (uint64_t c0 = a; c0 < edge_end; c0 += chunk) {
    const uint64_t c1 = std::min(edge_end, c0 + chunk);
    const GraphDev gc = make_graph_dev(seed, n, d, n0, c0, c1);
    if ((st = launch_generate_variant(gc, buf, gshape,
                                      static_cast<unsigned long long *>(counter.ptr), s,
                                      draw_flags)) != BA_OK ||
        (st = launch_count_rejections(gc, buf, node_limit, counts_dev, s,
                                      (variant & BA_VARIANT_NO_SELF_LOOPS) != 0)) != BA_OK)
      return st;
  }
  return BA_OK;
}

ba_status ba_generate_edges_host(uint64_t seed, uint64_t n, uint32_t d, uint64_t n0,
                                 uint64_t edge_begin, uint64_t edge_end, int64_t *host_out,
                                 void *stream) {
  set_error("");
  uint64_t m = 0;
  ba_status st = check_range(n, d, n0, edge_begin, edge_end, &m);
  if (st != BA_OK) return st;
  if (edge_begin == edge_end) return BA_OK;
  if (host_out == nullptr) {
    set_error("host_out must be non-NULL");
    return BA_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const uint64_t total = edge_end - edge_begin;
  const uint64_t chunk = std::min<uint64_t>(total, 1ull << 25);  // 512 MB of pairs
  const int nbuf = total > chunk ? 2 : 1;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t produced[2] = {nullptr, nullptr}, copied[2] = {nullptr, nullptr};
  StreamScratch bufs[2];
  auto cleanup = [&]() {
    for (int b = 0; b < 2; ++b) {
      if (produced[b]) cudaEventDestroy(produced[b]);
      if (copied[b]) cudaEventDestroy(copied[b]);
    }
    if (copy_stream) cudaStreamDestroy(copy_stream);
  };
  cudaError_t e = cudaStreamCreateWithFlags(&copy_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreateWithFlags");
  for (int b = 0; b < nbuf; ++b) {
    if ((e = cudaEventCreateWithFlags(&produced[b], cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&copied[b], cudaEventDisableTiming)) != cudaSuccess) {
      cleanup();
      return cuda_fail(e, "cudaEventCreateWithFlags");
    }
    st = bufs[b].alloc(chunk * 2 * sizeof(int64_t), s);
    if (st != BA_OK) {
      cleanup();
      return st;
    }
  }
  const Shape shape = shape_for(BA_KIND_GENERATE, edge_end <= (1ull << 31));
  StreamScratch counter;
  if ((st = counter.alloc(sizeof(unsigned long long), s)) != BA_OK) {
    cleanup();
    return st;
  }
  uint64_t k = 0;
  for (uint64_t a = edge_begin; a < edge_end; a += chunk, ++k) {
    const int b = static_cast<int>(k % nbuf);
    const uint64_t end = std::min(edge_end, a + chunk);
    if (k >= static_cast<uint64_t>(nbuf)) cudaStreamWaitEvent(s, copied[b], 0);  // buffer free
    const GraphDev g = make_graph_dev(seed, n, d, n0, a, end);
    st = launch_generate(g, static_cast<int64_t *>(bufs[b].ptr), shape,
                         static_cast<unsigned long long *>(counter.ptr), s);
    if (st != BA_OK) break;
    cudaEventRecord(produced[b], s);
    cudaStreamWaitEvent(copy_stream, produced[b], 0);
    e = cudaMemcpyAsync(host_out + 2 * (a - edge_begin), bufs[b].ptr, (end - a) * 2 * sizeof(int64_t),
                        cudaMemcpyDeviceToHost, copy_stream);
    if (e != cudaSuccess) {
      st = cuda_fail(e, "cudaMemcpyAsync");
      break;
    }
    cudaEventRecord(copied[b], copy_stream);
  }
  e = cudaStreamSynchronize(copy_stream);
  if (st == BA_OK && e != cudaSuccess) st = cuda_fail(e, "cudaStreamSynchronize");
  // buffers are freed on `s` after the copies finished
  for (int b = 0; b < nbuf; ++b) cudaStreamWaitEvent(s, copied[b], 0);
  bufs[0].release();
  bufs[1].release();
  e = cudaStreamSynchronize(s);
  if (st == BA_OK && e != cudaSuccess) st = cuda_fail(e, "cudaStreamSynchronize");
  cleanup();
  return st;
}

}  // extern "C"
