// ba_probe.cu -- roofline probes: the integer floor of the hash chain and the HBM write
// bandwidth, measured on the GPU the library runs on.
//
//   k_probe_hash   the algorithmic integer work of generateEdge (paper Fig. 1) with no
//                  scheduling, no stop test and no stores: every "edge" costs exactly two
//                  draws h(r) (the expected chain length, section 2's work bound), the
//                  second keyed by the first result made odd.  C independent chains per
//                  thread keep the multiplies' latency hidden, so the rate is that of the
//                  integer pipes alone.  The draw is the PTX form the kernels use.
//                  Positions start at 2*base+1: base = 0 takes the 32-bit-position
//                  hash, base >= 2^31 the 64-bit one.
//   k_probe_write  16-byte streaming stores over a buffer, nothing read: the write side
//                  of the generate kernel's roofline (16 bytes per edge).
#include <algorithm>

#include "ba_internal.h"

namespace ba {
namespace {

constexpr uint32_t kFullMask = 0xffffffffu;

// The fastest form of h(r) the kernels use (the PTX one).
__device__ __forceinline__ uint32_t hash_ptx(uint64_t seed_pre, uint32_t r) {
  return hash_r32_pre_ptx(seed_pre, r);
}
__device__ __forceinline__ uint64_t hash_ptx(uint64_t seed_pre, uint64_t r) {
  return hash_r64_pre_ptx(seed_pre, r);
}

template <class RT, int C>
__global__ void __launch_bounds__(256)
k_probe_hash(uint64_t seed_pre, uint64_t base, uint64_t edges, unsigned long long *sink) {
  const uint64_t tid = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  uint64_t acc = 0;
  for (uint64_t e0 = tid * C; e0 < edges; e0 += stride * C) {
    RT r[C];
#pragma unroll
    for (int c = 0; c < C; ++c) r[c] = static_cast<RT>(2 * (base + e0 + c) + 1);
#pragma unroll
    for (int c = 0; c < C; ++c) r[c] = hash_ptx(seed_pre, r[c]);
#pragma unroll
    for (int c = 0; c < C; ++c) r[c] = hash_ptx(seed_pre, r[c] | 1);
#pragma unroll
    for (int c = 0; c < C; ++c)
      if (e0 + c < edges) acc ^= static_cast<uint64_t>(r[c]);
  }
  // one atomic per warp keeps the results live without a store per thread
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc ^= __shfl_xor_sync(kFullMask, acc, o);
  if ((threadIdx.x & 31) == 0) atomicXor(sink, static_cast<unsigned long long>(acc));
}

__global__ void __launch_bounds__(256) k_probe_write(int4 *__restrict__ dst, uint64_t n16) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  const int4 v = make_int4(static_cast<int>(threadIdx.x), 0, static_cast<int>(blockIdx.x), 0);
  for (uint64_t k = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; k < n16; k += stride)
    __stcs(dst + k, v);
}

template <class K>
int full_grid(K kernel, int block) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, block, 0) != cudaSuccess || occ < 1)
    occ = 1;
  return sm_count() * occ;
}

template <class RT, int C>
ba_status probe_hash_t(uint64_t seed_pre, uint64_t base, uint64_t edges, unsigned long long *sink,
                       cudaStream_t s) {
  const int block = 256;
  const int grid = static_cast<int>(std::min<uint64_t>(
      full_grid(k_probe_hash<RT, C>, block), (edges + block * C - 1) / (block * C)));
  k_probe_hash<RT, C><<<std::max(grid, 1), block, 0, s>>>(seed_pre, base, edges, sink);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? BA_OK : cuda_fail(e, "k_probe_hash");
}

}  // namespace
}  // namespace ba

using namespace ba;

extern "C" {

ba_status ba_probe_hash(uint64_t seed, uint64_t base, uint64_t edges, int32_t chains,
                        uint64_t *sink_dev, void *stream) {
  set_error("");
  if (sink_dev == nullptr || (reinterpret_cast<uintptr_t>(sink_dev) & 7) != 0) {
    set_error("sink must be a non-NULL, 8-byte aligned device pointer");
    return BA_ERR_INVALID_ARG;
  }
  if (chains != 1 && chains != 2 && chains != 4) {
    set_error("chains must be 1, 2 or 4");
    return BA_ERR_INVALID_ARG;
  }
  if (edges > (1ull << 60) || base > (1ull << 60) - edges) {
    set_error("base + edges must stay below 2^60");
    return BA_ERR_RANGE;
  }
  if (edges == 0) return BA_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned long long *sink = reinterpret_cast<unsigned long long *>(sink_dev);
  const uint64_t sp = seed_premix(seed);
  const bool r32 = base + edges <= (1ull << 31);
  if (r32) {
    switch (chains) {
      case 1: return probe_hash_t<uint32_t, 1>(sp, base, edges, sink, s);
      case 2: return probe_hash_t<uint32_t, 2>(sp, base, edges, sink, s);
      default: return probe_hash_t<uint32_t, 4>(sp, base, edges, sink, s);
    }
  }
  switch (chains) {
    case 1: return probe_hash_t<uint64_t, 1>(sp, base, edges, sink, s);
    case 2: return probe_hash_t<uint64_t, 2>(sp, base, edges, sink, s);
    default: return probe_hash_t<uint64_t, 4>(sp, base, edges, sink, s);
  }
}

ba_status ba_probe_write(void *dst_dev, uint64_t bytes, void *stream) {
  set_error("");
  if (bytes == 0) return BA_OK;
  if (dst_dev == nullptr || (reinterpret_cast<uintptr_t>(dst_dev) & 15) != 0 || (bytes & 15) != 0) {
    set_error("dst must be a non-NULL, 16-byte aligned device pointer and bytes a multiple of 16");
    return BA_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int block = 256;
  const uint64_t n16 = bytes / 16;
  const int grid = static_cast<int>(std::min<uint64_t>(full_grid(k_probe_write, block),
                                                       (n16 + block - 1) / block));
  k_probe_write<<<std::max(grid, 1), block, 0, s>>>(static_cast<int4 *>(dst_dev), n16);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? BA_OK : cuda_fail(e, "k_probe_write");
}

}  // extern "C"
