// Device check of the hash_crc remainder (Fig. 3) on 32-bit positions, built and run by
// tests/test_gpu_remainder.py.  It compares
//   * recip_word(d) with floor((2^64 - 1) / d) - 2^32 for every normalised divisor
//     d in [2^31, 2^32), the definition of the 2-by-1 reciprocal;
//   * mod_64by32(x, r) with x % r on 2^32 pseudo-random pairs whose divisors spread over
//     every magnitude from 1 to 2^32 - 1 (so every normalisation shift occurs).
// Exit status 0 when nothing differs.  Every thread only reads its own index and adds to
// three counters.
#include <cstdint>
#include <cstdio>

#include <cuda_runtime.h>

#include "ba_draw.cuh"

namespace {

__global__ void check_reciprocal(unsigned long long *mismatches, unsigned long long *first) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t t = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < (1ull << 31);
       t += stride) {
    const uint32_t d = static_cast<uint32_t>((1ull << 31) + t);
    const uint32_t want = static_cast<uint32_t>(0xFFFFFFFFFFFFFFFFull / d - 0x100000000ull);
    if (ba::recip_word(d) != want) {
      atomicAdd(mismatches, 1ull);
      atomicMin(first, static_cast<unsigned long long>(d));
    }
  }
}

// SplitMix64 of a counter: the pairs' bits.
__device__ __forceinline__ uint64_t bits(uint64_t c) {
  uint64_t z = c * 0x9E3779B97F4A7C15ull + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void check_remainder(uint64_t pairs, unsigned long long *mismatches) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t t = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < pairs;
       t += stride) {
    const uint64_t x = bits(2 * t);
    const uint64_t q = bits(2 * t + 1);
    uint32_t r = static_cast<uint32_t>(q >> (32 + (q & 31)));  // below 2^(32 - (q mod 32))
    if (r == 0) r = 1;
    if (ba::mod_64by32(x, r) != static_cast<uint32_t>(x % r)) atomicAdd(mismatches, 1ull);
  }
}

}  // namespace

int main() {
  unsigned long long *dev = nullptr;
  if (cudaMalloc(&dev, 3 * sizeof(unsigned long long)) != cudaSuccess) return 2;
  const unsigned long long init[3] = {0ull, ~0ull, 0ull};
  cudaMemcpy(dev, init, sizeof init, cudaMemcpyHostToDevice);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  check_reciprocal<<<sms * 8, 256>>>(dev, dev + 1);
  check_remainder<<<sms * 8, 256>>>(1ull << 32, dev + 2);
  const cudaError_t e = cudaDeviceSynchronize();
  unsigned long long got[3] = {0, 0, 0};
  cudaMemcpy(got, dev, sizeof got, cudaMemcpyDeviceToHost);
  cudaFree(dev);
  std::printf("%s: reciprocal mismatches %llu (first divisor %llu), remainder mismatches %llu\n",
              cudaGetErrorString(e), got[0], got[1], got[2]);
  return (e == cudaSuccess && got[0] == 0 && got[2] == 0) ? 0 : 1;
}
