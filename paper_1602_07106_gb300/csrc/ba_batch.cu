// ba_batch.cu -- batched generation: many graphs of uneven size in one persistent launch.
//
// The host validates the descriptors, lays the graphs' tiles end to end (graph g owns
// global tiles [prefix[g], prefix[g+1])) and uploads the table once.  The kernel
// (k_generate_refill<..., Batched=true>) maps each tile to its graph by binary search and
// runs the same warp-refill loop as the plain entry point, with the graph's constants
// staged in shared memory, so every graph's bits equal those of a plain call.  A plan
// captures its launch (counter reset + kernel) into a CUDA graph and replays it.
#include <algorithm>
#include <new>
#include <vector>

#include "ba_internal.h"

using namespace ba;

struct ba_batch_plan {
  int device = 0;
  int32_t G = 0;
  std::vector<GraphDev> graphs;  // host copy with out_edge / tile0 filled in
  std::vector<int64_t> offsets;  // G+1 output offsets in edges
  std::vector<uint64_t> prefix;  // G+1 tile prefix
  uint64_t total_edges = 0;
  bool r32 = true;
  bool has_seed = false;
  Shape shape;
  GraphDev *d_graphs = nullptr;
  uint64_t *d_prefix = nullptr;
  unsigned long long *d_counter = nullptr;
  cudaStream_t capture_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t *graph_out = nullptr;
};

namespace {

// Fills graphs/offsets/prefix of a plan from host descriptors; shape.tile is adapted to
// the total work first (adapt_tile), and the launch must use the adapted shape.
ba_status build_tables(const ba_graph_desc *descs, int32_t G, const int64_t *out_offsets,
                       Shape &shape, ba_batch_plan *p) {
  if (G < 0 || (G > 0 && descs == nullptr)) {
    set_error("batch needs G >= 0 descriptors");
    return BA_ERR_INVALID_ARG;
  }
  p->G = G;
  p->graphs.resize(G);
  p->offsets.assign(G + 1, 0);
  p->prefix.assign(G + 1, 0);
  p->r32 = true;
  p->has_seed = false;
  uint64_t total = 0;  // valid ranges only; the loop below rejects the rest
  for (int32_t g = 0; g < G; ++g)
    if (descs[g].edge_end > descs[g].edge_begin) total += descs[g].edge_end - descs[g].edge_begin;
  shape.tile = adapt_tile(total, shape);
  const uint64_t T = static_cast<uint64_t>(shape.tile);
  for (int32_t g = 0; g < G; ++g) {
    const ba_graph_desc &d = descs[g];
    uint64_t m = 0;
    ba_status st = validate_graph(d.n, d.d, d.n0, &m);
    if (st != BA_OK) return st;
    if (d.edge_begin > d.edge_end || d.edge_end > m) {
      set_error("a batch descriptor's edge range is outside 0..m");
      return BA_ERR_RANGE;
    }
    GraphDev gd = make_graph_dev(d.seed, d.n, d.d, d.n0, d.edge_begin, d.edge_end);
    const uint64_t len = d.edge_end - d.edge_begin;
    if (out_offsets) {
      if (out_offsets[g] < 0 || out_offsets[g + 1] < out_offsets[g] ||
          static_cast<uint64_t>(out_offsets[g + 1] - out_offsets[g]) < len) {
        set_error("out_offsets must be non-decreasing and leave room for every graph's range");
        return BA_ERR_INVALID_ARG;
      }
      p->offsets[g] = out_offsets[g];
      p->offsets[g + 1] = out_offsets[g + 1];
    } else {
      p->offsets[g + 1] = p->offsets[g] + static_cast<int64_t>(len);
    }
    gd.out_edge = static_cast<uint64_t>(p->offsets[g]);
    gd.tile0 = p->prefix[g];
    p->prefix[g + 1] = p->prefix[g] + (len + T - 1) / T;
    p->graphs[g] = gd;
    if (d.edge_end > (1ull << 31)) p->r32 = false;
    if (gd.m0 > 0) p->has_seed = true;
  }
  p->total_edges = static_cast<uint64_t>(p->offsets[G]);
  return BA_OK;
}

// Launch shape of a batch: the caller's, else the tuned one for its position path.
ba_status batch_shape(const ba_graph_desc *descs, int32_t G, const ba_tuning *tune, Shape *out) {
  if (tune) return shape_from_public(BA_KIND_BATCH, tune, out);
  bool r32 = true;
  for (int32_t g = 0; g < G && descs; ++g)
    if (descs[g].edge_end > (1ull << 31)) r32 = false;
  *out = shape_for(BA_KIND_BATCH, r32);
  return BA_OK;
}

}  // namespace

extern "C" {

ba_status ba_batch_plan_create(const ba_graph_desc *descs, int32_t G, const int64_t *out_offsets,
                               const ba_tuning *tune, ba_batch_plan **plan) {
  set_error("");
  if (plan == nullptr) {
    set_error("plan output pointer is NULL");
    return BA_ERR_INVALID_ARG;
  }
  *plan = nullptr;
  ba_batch_plan *p = new (std::nothrow) ba_batch_plan();
  if (!p) return BA_ERR_NOMEM;
  cudaGetDevice(&p->device);
  ba_status st = batch_shape(descs, G, tune, &p->shape);
  if (st == BA_OK) st = build_tables(descs, G, out_offsets, p->shape, p);
  if (st != BA_OK) {
    delete p;
    return st;
  }
  cudaError_t e;
  if ((count_device_allocation(), e = cudaMalloc(&p->d_graphs, std::max<size_t>(1, p->graphs.size()) * sizeof(GraphDev))) != cudaSuccess ||
      (count_device_allocation(), e = cudaMalloc(&p->d_prefix, p->prefix.size() * sizeof(uint64_t))) != cudaSuccess ||
      (count_device_allocation(), e = cudaMalloc(&p->d_counter, 256)) != cudaSuccess ||
      (e = cudaMemcpy(p->d_graphs, p->graphs.data(), p->graphs.size() * sizeof(GraphDev),
                      cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(p->d_prefix, p->prefix.data(), p->prefix.size() * sizeof(uint64_t),
                      cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&p->capture_stream, cudaStreamNonBlocking)) != cudaSuccess) {
    st = (e == cudaErrorMemoryAllocation) ? BA_ERR_NOMEM : cuda_fail(e, "batch plan set-up");
    ba_batch_plan_destroy(p);
    return st;
  }
  *plan = p;
  return BA_OK;
}

uint64_t ba_batch_plan_total_edges(const ba_batch_plan *plan) {
  return plan ? plan->total_edges : 0;
}

ba_status ba_batch_plan_offsets(const ba_batch_plan *plan, int64_t *host_offsets) {
  if (!plan || !host_offsets) {
    set_error("NULL plan or offsets");
    return BA_ERR_INVALID_ARG;
  }
  std::copy(plan->offsets.begin(), plan->offsets.end(), host_offsets);
  return BA_OK;
}

ba_status ba_batch_plan_launch(ba_batch_plan *p, int64_t *out_dev, void *stream) {
  set_error("");
  if (!p) {
    set_error("NULL plan");
    return BA_ERR_INVALID_ARG;
  }
  if (p->total_edges == 0) return BA_OK;
  if (out_dev == nullptr || (reinterpret_cast<uintptr_t>(out_dev) & 15) != 0) {
    set_error("out must be a non-NULL, 16-byte aligned device pointer");
    return BA_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (p->exec == nullptr || p->graph_out != out_dev) {
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    p->exec = nullptr;
    p->graph = nullptr;
    // Capture on the plan's own stream (the caller's may be the legacy default stream).
    cudaError_t e = cudaStreamBeginCapture(p->capture_stream, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    BatchTable tab{p->d_graphs, p->d_prefix, p->G};
    ba_status st = launch_batch(tab, p->prefix.back(), p->r32, p->has_seed, out_dev, p->shape,
                                p->d_counter, p->capture_stream);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(p->capture_stream, &graph);
    if (st != BA_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&p->exec, graph, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(graph);
      return cuda_fail(e, "cudaGraphInstantiate");
    }
    p->graph = graph;
    p->graph_out = out_dev;
  }
  cudaError_t e = cudaGraphLaunch(p->exec, s);
  return e == cudaSuccess ? BA_OK : cuda_fail(e, "cudaGraphLaunch");
}

ba_status ba_batch_plan_destroy(ba_batch_plan *p) {
  if (!p) return BA_OK;
  // cudaFree waits for the device work that may still read the tables.
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->d_graphs) cudaFree(p->d_graphs);
  if (p->d_prefix) cudaFree(p->d_prefix);
  if (p->d_counter) cudaFree(p->d_counter);
  if (p->capture_stream) cudaStreamDestroy(p->capture_stream);
  delete p;
  return BA_OK;
}

ba_status ba_generate_batch(const ba_graph_desc *descs, int32_t G, const int64_t *offsets_host,
                            int64_t *out_dev, const ba_tuning *tune, void *stream) {
  set_error("");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ba_batch_plan p;
  Shape shape;
  ba_status st = batch_shape(descs, G, tune, &shape);
  if (st == BA_OK) st = build_tables(descs, G, offsets_host, shape, &p);
  if (st != BA_OK) return st;
  if (p.total_edges == 0) return BA_OK;
  if (out_dev == nullptr || (reinterpret_cast<uintptr_t>(out_dev) & 15) != 0) {
    set_error("out must be a non-NULL, 16-byte aligned device pointer");
    return BA_ERR_INVALID_ARG;
  }
  // Stream-ordered tables: freed on `s` after the launch has read them.
  const size_t gbytes = p.graphs.size() * sizeof(GraphDev);
  const size_t bytes = gbytes + p.prefix.size() * sizeof(uint64_t) + 256;
  void *mem = nullptr;
  st = pool_alloc(&mem, bytes, s);
  if (st != BA_OK) return st;
  cudaError_t e;
  char *base = static_cast<char *>(mem);
  GraphDev *dg = reinterpret_cast<GraphDev *>(base);
  uint64_t *dp = reinterpret_cast<uint64_t *>(base + gbytes);
  unsigned long long *dc = reinterpret_cast<unsigned long long *>(base + bytes - 256);
  if ((e = cudaMemcpyAsync(dg, p.graphs.data(), gbytes, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(dp, p.prefix.data(), p.prefix.size() * sizeof(uint64_t),
                           cudaMemcpyHostToDevice, s)) != cudaSuccess) {
    cudaFreeAsync(mem, s);
    return cuda_fail(e, "cudaMemcpyAsync");
  }
  BatchTable tab{dg, dp, p.G};
  st = launch_batch(tab, p.prefix.back(), p.r32, p.has_seed, out_dev, shape, dc, s);
  cudaFreeAsync(mem, s);
  // the host tables of `p` must outlive the pageable H2D copies above
  e = cudaStreamSynchronize(s);
  if (st == BA_OK && e != cudaSuccess) st = cuda_fail(e, "cudaStreamSynchronize");
  return st;
}

}  // extern "C"
