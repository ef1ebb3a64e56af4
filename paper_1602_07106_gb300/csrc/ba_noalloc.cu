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
// host-side stand-in): the array's device address is looked up with cudaGetSymbolAddress,
// with the device current, on the first call made on it (and again after its context was
// reset).
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
unsigned long long g_scratch_ctx[kMaxDevices] = {};  // context the address belongs to

// ID of the current CUDA context (unique for the process's lifetime, so a context created
// again after a reset gets a new one), through the driver's entry points; false when no
// context is current or the driver does not offer the calls.
bool current_context_id(unsigned long long *id) {
  using GetCurrent = int (*)(void **);
  using GetId = int (*)(void *, unsigned long long *);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    looked_up = true;
    void *f = nullptr, *g = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q1) ==
            cudaSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &g, 12000, cudaEnableDefault, &q2) ==
            cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
      get_current = reinterpret_cast<GetCurrent>(f);
      get_id = reinterpret_cast<GetId>(g);
    }
    cudaGetLastError();
  }
  if (get_current == nullptr || get_id == nullptr) return false;
  void *ctx = nullptr;
  if (get_current(&ctx) != 0 || ctx == nullptr) return false;
  return get_id(ctx, id) == 0;
}

// Device address of g_noalloc_scratch on the current device.  Looked up (with that device
// current) on the first call made on the device, and again whenever the current context
// is not the one the cached address came from (after a reset the module is loaded anew and
// the array may have moved).  Without the driver's context IDs it is looked up every call.
ba_status scratch_address(NoAllocScratch **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device ordinal beyond the no-allocation set-up table (64 devices)");
    return BA_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_setup_mu);
  unsigned long long id = 0;
  const bool known = current_context_id(&id);
  if (g_scratch_addr[dev] == nullptr || !known || id != g_scratch_ctx[dev]) {
    void *ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || ptr == nullptr) return cuda_fail(e, "cudaGetSymbolAddress");
    g_scratch_addr[dev] = ptr;
    g_scratch_ctx[dev] = current_context_id(&id) ? id : 0;  // the lookup made one current
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
  // the same launch shape as ba_generate_batch: the tuned tile, shrunk for small batches
  Shape shape = shape_for(BA_KIND_BATCH, r32);
  shape.tile = adapt_tile(total_edges, shape);
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
