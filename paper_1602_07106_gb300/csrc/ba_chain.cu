// ba_chain.cu -- the work bound of section 2 measured on the device: a histogram of the
// chain lengths of Fig. 1 (draws made for edge i's second end point, from position 2i+1
// until the position is even or inside the seed clique; 0 for a seed edge).
//
// One thread per edge (grid-stride), the plain C form of the hash, counts kept in a
// per-CTA shared histogram and added to the caller's counters once per CTA.  It is a
// counter, not a hot path: it exists so that the device's chain lengths can be compared
// with the oracle's, edge for edge, and their mean with the exact expectation.
#include <algorithm>

#include "ba_internal.h"

namespace ba {
namespace {

constexpr int kChainThreads = 256;

template <class RT, bool HasSeed>
__global__ void __launch_bounds__(kChainThreads)
k_chain_lengths(const GraphDev g, uint32_t bins, unsigned long long *__restrict__ hist) {
  extern __shared__ unsigned long long local[];  // bins counters
  for (uint32_t k = threadIdx.x; k < bins; k += blockDim.x) local[k] = 0;
  __syncthreads();
  const RT two_m0 = seed_limit<RT>(g.two_m0);
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t i = g.begin + static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
       i < g.end; i += stride) {
    uint32_t len = 0;
    if (!(HasSeed && i < g.m0)) {  // a seed edge's end point is in the clique: no draw
      RT r = static_cast<RT>(2 * i + 1);
      do {
        r = hash_pos<RT>(g.seed, r);
        ++len;
      } while (!chain_stops<RT, HasSeed>(r, two_m0));
    }
    atomicAdd(local + min(len, bins - 1), 1ull);
  }
  __syncthreads();
  for (uint32_t k = threadIdx.x; k < bins; k += blockDim.x)
    if (local[k]) atomicAdd(hist + k, local[k]);
}

template <class RT, bool HasSeed>
ba_status chain_t(const GraphDev &g, uint32_t bins, unsigned long long *hist, cudaStream_t s) {
  const size_t smem = static_cast<size_t>(bins) * sizeof(unsigned long long);
  int occ = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &occ, k_chain_lengths<RT, HasSeed>, kChainThreads, smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  const uint64_t len = g.end - g.begin;
  const uint64_t want = (len + kChainThreads - 1) / kChainThreads;
  const int grid = static_cast<int>(
      std::max<uint64_t>(1, std::min<uint64_t>(want, static_cast<uint64_t>(sm_count()) * std::max(occ, 1))));
  k_chain_lengths<RT, HasSeed><<<grid, kChainThreads, smem, s>>>(g, bins, hist);
  e = cudaGetLastError();
  return e == cudaSuccess ? BA_OK : cuda_fail(e, "k_chain_lengths");
}

}  // namespace
}  // namespace ba

using namespace ba;

extern "C" ba_status ba_chain_lengths(uint64_t seed, uint64_t n, uint32_t d, uint64_t n0,
                                      uint64_t edge_begin, uint64_t edge_end, uint32_t bins,
                                      uint64_t *hist_dev, int accumulate, void *stream) {
  set_error("");
  uint64_t m = 0;
  ba_status st = validate_graph(n, d, n0, &m);
  if (st != BA_OK) return st;
  if (edge_begin > edge_end || edge_end > m) {
    set_error("edge range outside 0..m");
    return BA_ERR_RANGE;
  }
  if (bins < 2 || bins > 1024) {
    set_error("bins must be 2..1024");
    return BA_ERR_INVALID_ARG;
  }
  if (hist_dev == nullptr || (reinterpret_cast<uintptr_t>(hist_dev) & 7) != 0) {
    set_error("hist must be a non-NULL, 8-byte aligned device pointer");
    return BA_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!accumulate) {
    cudaError_t e = cudaMemsetAsync(hist_dev, 0, static_cast<size_t>(bins) * 8, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  }
  if (edge_begin == edge_end) return BA_OK;
  const GraphDev g = make_graph_dev(seed, n, d, n0, edge_begin, edge_end);
  unsigned long long *hist = reinterpret_cast<unsigned long long *>(hist_dev);
  const bool r32 = edge_end <= (1ull << 31);
  if (g.m0 > 0)
    return r32 ? chain_t<uint32_t, true>(g, bins, hist, s) : chain_t<uint64_t, true>(g, bins, hist, s);
  return r32 ? chain_t<uint32_t, false>(g, bins, hist, s) : chain_t<uint64_t, false>(g, bins, hist, s);
}
