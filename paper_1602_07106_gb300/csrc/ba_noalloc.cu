// ba_noalloc.cu -- ba_generate_batch_noalloc: the batched launch without any allocation.
//
// ba_generate_batch takes its scratch (the per-graph constant table, the tile prefix and the
// tile counter of the persistent scheduler) from the stream-ordered allocator.  Some callers
// cannot allocate device memory at the point where they want edges: code that runs while
// another framework's caching allocator holds all device memory, hosts with a fixed device
// memory budget that forbid hidden allocations, and code that must not risk an allocation
// failure or the implicit synchronisation an allocation can cause in the middle of its
// stream.  For them this entry point keeps the scratch in one file-scope device array of a
// fixed size, reserved when the library's module is loaded on a GPU and held until exit.
//
// Host code never hands the array's name to a kernel (in host code the name is only a
// host-side stand-in): the array's device address is looked up with cudaGetSymbolAddress
// once per device, with that device current, on the first call made on it.
#include <mutex>

#include "ba_internal.h"

using namespace ba;

namespace {

struct NoAllocScratch {
  GraphDev graphs[BA_NOALLOC_MAX_GRAPHS];
  uint64_t tile_prefix[BA_NOALLOC_MAX_GRAPHS + 1];
  unsigned long long counter[32];
};

// The shared scratch: one per GPU that loads the library, ~114 KB.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (looked up once per device).
ba_status scratch_address(NoAllocScratch **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device ordinal beyond the no-allocation set-up table (64 devices)");
    return BA_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (g_scratch_addr[dev] == nullptr) {
    void *ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || ptr == nullptr) return cuda_fail(e, "cudaGetSymbolAddress");
    g_scratch_addr[dev] = ptr;
  }
  *out = static_cast<NoAllocScratch *>(g_scratch_addr[dev]);
  return BA_OK;
}

}  // namespace

extern "C" ba_status ba_generate_batch_noalloc(const ba_graph_desc *descs, int32_t G,
                                               const int64_t *offsets_host, int64_t *out_dev,
                                               void *stream) {
  set_error("");
  if (G < 0 || (G > 0 && descs == nullptr)) {
    set_error("batch needs G >= 0 descriptors");
    return BA_ERR_INVALID_ARG;
  }
  if (G > BA_NOALLOC_MAX_GRAPHS) {
    set_error("batch has more graphs than the no-allocation scratch table holds "
              "(BA_NOALLOC_MAX_GRAPHS = 1024); split it or use ba_generate_batch");
    return BA_ERR_INVALID_ARG;
  }
  // Pass 1: validate every descriptor and find the launch's position path, without storage.
  bool r32 = true;
  bool has_seed = false;
  uint64_t total_edges = 0;
  for (int32_t g = 0; g < G; ++g) {
    const ba_graph_desc &d = descs[g];
    uint64_t m = 0;
    ba_status st = validate_graph(d.n, d.d, d.n0, &m);
    if (st != BA_OK) return st;
    if (d.edge_begin > d.edge_end || d.edge_end > m) {
      set_error("a batch descriptor's edge range is outside 0..m");
      return BA_ERR_RANGE;
    }
    const uint64_t len = d.edge_end - d.edge_begin;
    if (offsets_host) {
      if (offsets_host[g] < 0 || offsets_host[g + 1] < offsets_host[g] ||
          static_cast<uint64_t>(offsets_host[g + 1] - offsets_host[g]) < len) {
        set_error("out_offsets must be non-decreasing and leave room for every graph's range");
        return BA_ERR_INVALID_ARG;
      }
    }
    total_edges += len;
    if (d.edge_end > (1ull << 31)) r32 = false;
    if (d.n0 > 1) has_seed = true;
  }
  if (total_edges == 0) return BA_OK;
  if (out_dev == nullptr || (reinterpret_cast<uintptr_t>(out_dev) & 15) != 0) {
    set_error("out must be a non-NULL, 16-byte aligned device pointer");
    return BA_ERR_INVALID_ARG;
  }
  NoAllocScratch *scratch = nullptr;
  ba_status st = scratch_address(&scratch);
  if (st != BA_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Shape shape = shape_for(BA_KIND_BATCH, r32);
  const uint64_t T = static_cast<uint64_t>(shape.tile);

  // Pass 2: build the tables in small stack blocks and copy each into the scratch.  A copy
  // from pageable memory returns once its source has been staged, so the block can be reused.
  constexpr int kBlock = 32;
  GraphDev gblock[kBlock];
  uint64_t pblock[kBlock + 1];
  uint64_t prefix = 0;
  int64_t off = 0;
  for (int32_t g0 = 0; g0 < G; g0 += kBlock) {
    const int cnt = G - g0 < kBlock ? G - g0 : kBlock;
    for (int k = 0; k < cnt; ++k) {
      const ba_graph_desc &d = descs[g0 + k];
      GraphDev gd = make_graph_dev(d.seed, d.n, d.d, d.n0, d.edge_begin, d.edge_end);
      const uint64_t len = d.edge_end - d.edge_begin;
      gd.out_edge = static_cast<uint64_t>(offsets_host ? offsets_host[g0 + k] : off);
      off += static_cast<int64_t>(len);
      gd.tile0 = prefix;
      pblock[k] = prefix;
      prefix += (len + T - 1) / T;
      gblock[k] = gd;
    }
    pblock[cnt] = prefix;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(scratch->graphs + g0, gblock, cnt * sizeof(GraphDev),
                             cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(scratch->tile_prefix + g0, pblock, (cnt + 1) * sizeof(uint64_t),
                             cudaMemcpyHostToDevice, s)) != cudaSuccess)
      return cuda_fail(e, "cudaMemcpyAsync");
  }
  // launch_batch zeroes the tile counter before the kernel (the scratch keeps the previous
  // call's contents; the tables above were rewritten in full for this call's G graphs).
  BatchTable tab{scratch->graphs, scratch->tile_prefix, G};
  return launch_batch(tab, prefix, r32, has_seed, out_dev, shape, scratch->counter, s);
}
