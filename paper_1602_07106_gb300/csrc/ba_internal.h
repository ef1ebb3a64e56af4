// ba_internal.h -- host-side interfaces shared by libba's translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "ba.h"  // include/ba.h, on the include path of the build
#include "ba_device.cuh"

namespace ba {

// Persistent-scheduler parameters of one launch.
struct SchedParams {
  uint64_t num_tiles;            // tiles of 2^tile_shift edges over the whole launch
  unsigned long long *counter;   // zeroed before the launch; tiles past the first wave
  uint32_t tile_shift;
  uint32_t total_warps;          // warps in the grid (first tile of warp w is w)
  uint32_t hist_agg;             // degree kernel: warp-aggregate histogram increments
  uint32_t pad;
  // checked launches only: output slots [0, out_cap) exist; a store to a slot beyond them
  // is skipped and the lowest such slot is kept in *status (atomicMin)
  uint64_t out_cap;
  unsigned long long *status;
  // fold launches only (ba_fold.cu): the nodes that the chunk flush hands on to the exact
  // pass of section 4's rejection, as offsets from fold_q0 (at most fold_cap of them,
  // *fold_count of them written), and, when counting, the counters below fold_limit
  uint32_t *fold_list;
  unsigned long long *fold_count;
  uint64_t fold_q0;
  uint64_t fold_cap;
  unsigned long long *fold_counts;
  uint64_t fold_limit;
};

// Graph table of a batched launch (device pointers).
struct BatchTable {
  const GraphDev *graphs;        // G entries
  const uint64_t *tile_prefix;   // G+1 entries: graph g owns tiles [tile_prefix[g], [g+1])
  int32_t G;
};

struct Shape {
  int block = 0;
  int ctas_per_sm = 0;
  int tile = 0;
  int refill = 1;
  int hist_bins = 0;
  int hist_agg = 0;
  int chains = 1;  // hash chains per lane in the generate / batched refill kernels
};

// ---- host helpers (ba_api.cu)
void set_error(const char *msg);
ba_status cuda_fail(cudaError_t e, const char *where);
GraphDev make_graph_dev(uint64_t seed, uint64_t n, uint32_t d, uint64_t n0, uint64_t begin,
                        uint64_t end);
ba_status validate_graph(uint64_t n, uint32_t d, uint64_t n0, uint64_t *m_out);
int sm_count();
// Stream-ordered scratch from libba's own pool on the current device (kept mapped up to
// 64 MB between calls); release with cudaFreeAsync on the same stream.
ba_status pool_alloc(void **ptr, size_t bytes, cudaStream_t s);
// Counts one device allocation (pool_alloc does; so does every cudaMalloc of the library).
void count_device_allocation();
// Tile size for a batched launch of `total_edges` edges with shape s: the shape's tile,
// halved (down to 256) until every warp of a full grid has about four tiles, as plain
// calls do, so that small batches and light serving ticks still spread over the GPU.
int adapt_tile(uint64_t total_edges, const Shape &s);

// ---- tuner cache (ba_tune.cu)
Shape shape_for(int kind, bool r32);
ba_status shape_from_public(int kind, const ba_tuning *t, Shape *out);  // validates
void shape_store(int kind, bool r32, const Shape &s);

// ---- kernel launchers (ba_kernels.cu).  All enqueue on `stream` and return BA_OK or
// BA_ERR_CUDA.  `counter` must point to >= 8 bytes of device memory; it is zeroed here.
// narrow: write (source, target) as two int32 (8 bytes per edge) instead of two int64.
ba_status launch_generate(const GraphDev &g, int64_t *out, const Shape &s,
                          unsigned long long *counter, cudaStream_t stream, bool narrow = false);
ba_status launch_degree(const GraphDev &g, uint64_t node_limit, uint64_t *counts,
                        int accumulate, const Shape &s, unsigned long long *counter,
                        cudaStream_t stream);
// Variant draws (BA_VARIANT_* flags; 0 = the plain graph): int64 output.  The caller has
// checked the flags and that the self-loop-free rule has a seed graph (n0 >= 2).
ba_status launch_generate_variant(const GraphDev &g, int64_t *out, const Shape &s,
                                  unsigned long long *counter, cudaStream_t stream,
                                  uint32_t variant);
ba_status launch_degree_variant(const GraphDev &g, uint64_t node_limit, uint64_t *counts,
                                int accumulate, const Shape &s, unsigned long long *counter,
                                cudaStream_t stream, uint32_t variant);
// Section 4's rejection of a node's duplicate targets over an output that the generate
// kernel (plain, or self-loop-free with no_loops) has already written; d <= 1024.
ba_status launch_reject_duplicates(const GraphDev &g, int64_t *out, cudaStream_t stream,
                                   bool no_loops);
// The same rejections for a degree count: `pairs` holds edges [g.begin, g.end) of the
// array without rejection as the generate kernel wrote them (g.out_edge = 0); counts[]
// (below node_limit) gets one per edge of the range at its final target.  d <= 1024.
ba_status launch_count_rejections(const GraphDev &g, const int64_t *pairs, uint64_t node_limit,
                                  uint64_t *counts, cudaStream_t stream, bool no_loops);
// counts[j] (j < node_limit) = (accumulate ? counts[j] : 0) + the end points at node j of
// the edges in [g.begin, g.end) that section 4's graph fixes without a draw: the source of
// every non-seed edge and both ends of every seed-clique edge (k_degree_init).
ba_status launch_degree_sources(const GraphDev &g, uint64_t node_limit, uint64_t *counts,
                                int accumulate, cudaStream_t stream);
// ---- section 4's rejection folded into the generate kernel (ba_fold.cu), for d a power of
// two in 2..32.  Generates edges [g.begin, g.end) with the array's targets (written to out,
// or, with out == nullptr, counted: one per target below node_limit of a node the pass
// settles) and lists in list[] (offsets from node q0, at most cap entries, the number at
// *list_count, zeroed by the caller) every node that holds a repeated target or is cut by a
// chunk; launch_reject_listed then finishes the listed nodes.  no_loops: the self-loop-free
// draw.  counter: >= 8 bytes of device memory.
bool fold_supported(uint32_t d);
ba_status launch_generate_fold(const GraphDev &g, int64_t *out, const Shape &s,
                               unsigned long long *counter, cudaStream_t stream, bool no_loops,
                               uint32_t *list, unsigned long long *list_count, uint64_t q0,
                               uint64_t cap, uint64_t *counts, uint64_t node_limit);
// The exact pass of the rejection for the listed nodes only (ba_simple.cu): out == nullptr
// counts final targets below node_limit (recomputing every target; the list must then hold
// every listed node: list_cap >= the nodes q0..q_hi), else writes changed targets back
// (and takes every node q0..q_hi when more than list_cap were listed).  q0, q_hi: the
// nodes the list may name.
ba_status launch_reject_listed(const GraphDev &g, int64_t *out, uint64_t *counts,
                               uint64_t node_limit, const uint32_t *list,
                               const unsigned long long *list_count, uint64_t list_cap,
                               uint64_t q0, uint64_t q_hi, cudaStream_t stream, bool no_loops);
// launch_generate with every output store checked against out_cap (edges): see SchedParams.
ba_status launch_generate_checked(const GraphDev &g, int64_t *out, uint64_t out_cap,
                                  unsigned long long *status, const Shape &s,
                                  unsigned long long *counter, cudaStream_t stream);
ba_status launch_batch(const BatchTable &tab, uint64_t total_tiles, bool r32, bool has_seed,
                       int64_t *out, const Shape &s, unsigned long long *counter,
                       cudaStream_t stream);

// Number of CUDA kernels the last launch_* call on this thread enqueued (for the
// benchmark's launch count).
int last_kernel_count();

}  // namespace ba
