// ba_simple.cu -- section 4's graph without parallel edges.
//
// The paper keeps the targets already generated for a node in a table of at most d
// entries and rejects a duplicate.  Here the generate kernel first writes every edge with
// the target of the array without rejection (the array every chain follows: the
// recursion of Fig. 1 cannot see rejections made while another node was generated).
// k_reject_duplicates then walks the nodes that own edges in range, one lane per edge of a
// node (d <= 32, so a warp holds 32/d whole nodes):
//   1. each lane holds its edge's target (read back from the output, or recomputed for
//      the edges of the first node that lie before the range);
//   2. __match_any_sync on (target) and on (node) finds the lanes whose target an earlier
//      edge of the same node already has; a warp without such a lane is done;
//   3. otherwise the node's edges are taken in order from the first duplicate on: while an
//      edge's candidate is one of the targets accepted before it (a ballot over the node's
//      lanes), j < reach(u) and fewer than kRedrawCap redraws were made, its lane redraws:
//      the plain draw's range and key 2i+1 with the SplitMix64 bits of
//      seed ^ k * kRedrawSalt, then the array's chain from the drawn position.
// Only changed targets are written back.  Sources and seed-clique edges never change.
#include <algorithm>

#include "ba_draw.cuh"
#include "ba_internal.h"

namespace ba {
namespace {

constexpr uint32_t kAll = 0xffffffffu;
constexpr uint64_t kRedrawSalt = 0xD6E8FEB86659FD93ull;
constexpr uint32_t kRedrawCap = 65536u;

// E[x] of the array without rejection: the chain of Fig. 1 (and section 4's seed test)
// from position x.
template <class RT, bool HasSeed, class Draw>
__device__ uint64_t array_value(RT x, const GraphDev &g, const Draw &draw, RT l2m0) {
  while (!chain_stops<RT, HasSeed>(x, l2m0)) x = draw(x);
  return target_of<RT, HasSeed>(x, g);
}

// Candidate k >= 1 for edge i: a draw over the plain draw's range keyed by 2i+1 with the
// salted seed, resolved through the array.
template <class RT, bool HasSeed, class Draw>
__device__ uint64_t redraw(uint64_t i, uint32_t k, const GraphDev &g, const Draw &draw, RT l2m0) {
  Draw salted = draw;
  salted.spre = seed_premix(g.seed ^ (static_cast<uint64_t>(k) * kRedrawSalt));
  return array_value<RT, HasSeed>(salted(static_cast<RT>(2 * i + 1)), g, draw, l2m0);
}

// Warp items of npw consecutive nodes n0 + q, q in [q_lo, q_hi]; lane = slot * d + j.
template <class RT, bool HasSeed, class Draw, bool NoLoop>
__global__ void __launch_bounds__(256)
k_reject_duplicates(const GraphDev g, int64_t *__restrict__ out, uint64_t q_lo, uint64_t q_hi,
                    uint32_t npw) {
  Draw draw;
  draw.setup(g, nullptr, sizeof(RT) == 4);
  draw.bind(g);
  const RT l2m0 = seed_limit<RT>(g.two_m0);
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t d = g.d;
  const uint32_t slot = lane / d;
  const uint32_t j = lane - slot * d;
  const uint32_t lt = (1u << lane) - 1u;
  const uint64_t items = (q_hi - q_lo) / npw + 1;
  const uint64_t warps = static_cast<uint64_t>(gridDim.x) * (blockDim.x >> 5);
  for (uint64_t item = static_cast<uint64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
       item < items; item += warps) {
    const uint64_t q = q_lo + item * npw + slot;
    const uint64_t i = g.m0 + q * d + j;
    const bool part = slot < npw && q <= q_hi && i < g.end;  // the edge or an earlier sibling is in range
    const bool in_out = part && i >= g.begin;
    long long *dst = reinterpret_cast<long long *>(out) + 2 * (in_out ? g.out_edge + (i - g.begin) : 0) + 1;
    uint64_t t = 0;
    if (in_out) t = static_cast<uint64_t>(__ldcs(dst));
    else if (part) t = array_value<RT, HasSeed>(draw(static_cast<RT>(2 * i + 1)), g, draw, l2m0);
    // node IDs are below 2^62, so the idle lanes' keys match nothing real
    const uint32_t same_t = __match_any_sync(kAll, part ? t : ~0ull - lane);
    const uint32_t same_node = __match_any_sync(kAll, part ? slot : 32u + lane);
    const uint64_t node = g.n0 + q;
    const uint64_t reach = NoLoop ? node : (g.n0 == 1 ? node : node + 1);
    const bool dup = part && j < reach && (same_t & same_node & lt) != 0;
    uint32_t dups = __ballot_sync(kAll, dup);
    if (dups == 0) continue;
    const uint32_t parts = __ballot_sync(kAll, part);
    uint64_t acc = t;
    while (dups) {  // nodes with a duplicate, one at a time, edges in order
      const uint32_t first = __ffs(dups) - 1;
      const uint32_t base = (first / d) * d;
      const uint32_t node_lanes = (d == 32 ? kAll : ((1u << d) - 1u)) << base;
      const uint64_t reach_l = __shfl_sync(kAll, reach, first);
      for (uint32_t L = first; L < base + d && ((parts >> L) & 1u); ++L) {
        const uint64_t iL = __shfl_sync(kAll, i, L);
        uint64_t cand = __shfl_sync(kAll, acc, L);
        uint32_t k = 0;
        for (;;) {
          const bool taken = __ballot_sync(kAll, lane >= base && lane < L && acc == cand) != 0;
          if (!taken || L - base >= reach_l || k >= kRedrawCap) break;
          ++k;
          uint64_t v = 0;
          if (lane == L) v = redraw<RT, HasSeed>(iL, k, g, draw, l2m0);
          cand = __shfl_sync(kAll, v, L);
        }
        if (lane == L) acc = cand;
      }
      dups &= ~node_lanes;
    }
    if (in_out && acc != t) __stcs(dst, static_cast<long long>(acc));
  }
}

template <class RT, bool HasSeed, class Draw, bool NoLoop>
ba_status launch_t(const GraphDev &g, int64_t *out, uint64_t q_lo, uint64_t q_hi, uint32_t npw,
                   cudaStream_t stream) {
  auto kernel = k_reject_duplicates<RT, HasSeed, Draw, NoLoop>;
  constexpr int kBlock = 256;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, 0);
  if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  const uint64_t items = (q_hi - q_lo) / npw + 1;
  const uint64_t want = (items + kBlock / 32 - 1) / (kBlock / 32);
  const int grid = static_cast<int>(std::min<uint64_t>(
      want, static_cast<uint64_t>(sm_count()) * static_cast<uint64_t>(std::max(per_sm, 1))));
  kernel<<<grid, kBlock, 0, stream>>>(g, out, q_lo, q_hi, npw);
  e = cudaGetLastError();
  return e == cudaSuccess ? BA_OK : cuda_fail(e, "k_reject_duplicates");
}

}  // namespace

ba_status launch_reject_duplicates(const GraphDev &g, int64_t *out, cudaStream_t stream,
                                   bool no_loops) {
  if (g.d <= 1 || g.d > 32) return g.d <= 1 ? BA_OK : BA_ERR_INVALID_ARG;
  const uint64_t a = std::max(g.begin, g.m0);
  if (a >= g.end) return BA_OK;  // only seed-clique edges in range
  const uint64_t q_lo = (a - g.m0) / g.d;
  const uint64_t q_hi = (g.end - 1 - g.m0) / g.d;
  const uint32_t npw = 32u / g.d;
  const bool r32 = g.end <= (1ull << 31);
  if (no_loops) {  // needs a seed edge, so a seed clique
    using D = DrawVariant<false, true>;
    return r32 ? launch_t<uint32_t, true, D, true>(g, out, q_lo, q_hi, npw, stream)
               : launch_t<uint64_t, true, D, true>(g, out, q_lo, q_hi, npw, stream);
  }
  if (g.m0 > 0)
    return r32 ? launch_t<uint32_t, true, DrawPlain, false>(g, out, q_lo, q_hi, npw, stream)
               : launch_t<uint64_t, true, DrawPlain, false>(g, out, q_lo, q_hi, npw, stream);
  return r32 ? launch_t<uint32_t, false, DrawPlain, false>(g, out, q_lo, q_hi, npw, stream)
             : launch_t<uint64_t, false, DrawPlain, false>(g, out, q_lo, q_hi, npw, stream);
}

}  // namespace ba
