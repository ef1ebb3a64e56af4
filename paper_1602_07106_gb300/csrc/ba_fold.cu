// ba_fold.cu -- section 4's rejection of parallel edges folded into the generate kernel.
//
// The rejection needs, for every node, whether two of its d targets repeat.  The refill
// generate kernel (ba_refill.cuh) already holds a chunk's targets in the warp's staging
// ring when it writes the chunk out, so for d a power of two <= 32 its chunk flush here
// also looks for repeats: it lays the chunk's edges out so that a node's d edges sit in d
// consecutive lanes of one row, and each lane compares its target's low 32 bits with those
// of the next d/2 lanes of its node, cyclically (a shuffle within d-lane segments), which
// compares every pair of the node once.  The few nodes with a repeat (a few thousand of the
// 2^27 nodes of the large workload), and the nodes a chunk boundary cuts, go to a list;
// launch_reject_listed (ba_simple.cu) then runs the exact accept/redraw pass of the
// rejection over the listed nodes only.  The separate pass over every node reads the whole
// output back (16 bytes an edge); this one reads nothing.
//
// Counting (section 3's streaming analysis of this graph): the flush writes nothing and
// adds each target of a node it settles (whole in the chunk, no repeat) to its counter;
// the listed nodes are counted by the exact pass.
#include "ba_refill.cuh"

namespace ba {
namespace {

template <bool CountOnly>
struct FoldDetect {
  static constexpr bool kActive = true;

  // The chunk's edges [e0, e0 + len) in rows of 32 lanes, lane l of row k on chunk edge
  // 32k + l - delta, delta = the place of e0 in its node (edge m0 + q*D starts node q), so
  // that a node's edges are lanes [s*D, s*D + D) of a row.  With d = D = 2^kLog the
  // divisions are shifts; on 32-bit positions every edge index fits 32 bits.
  template <uint32_t D, class RT, bool HasSeed>
  __device__ __forceinline__ static void rows(const RT *stage, uint64_t e0, uint32_t len,
                                              const GraphDev &g, int64_t *__restrict__ out,
                                              const SchedParams &sp) {
    using IT = RT;  // edge indices: < 2^31 on the 32-bit-position path
    constexpr uint32_t kLog = D == 2 ? 1 : D == 4 ? 2 : D == 8 ? 3 : D == 16 ? 4 : 5;
    constexpr uint32_t kGroup = D == 32 ? 0xffffffffu : (1u << D) - 1u;
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t gm = kGroup << (lane & ~(D - 1));  // the lanes of this lane's node
    const bool leader = (lane & (D - 1)) == 0;
    const int next = static_cast<int>(lane + 1);  // the cyclic successor within the node
    const IT ei = static_cast<IT>(e0);
    const IT m0 = static_cast<IT>(g.m0);
    const IT n0 = static_cast<IT>(g.n0);
    const RT two_m0 = seed_limit<RT>(g.two_m0);
    const uint32_t delta = static_cast<uint32_t>(e0 - g.m0) & (D - 1);
    int64_t *const dst = CountOnly ? nullptr : out + 2 * (g.out_edge + (e0 - g.begin));
    const bool first_chunk = e0 == g.begin;
    // rows [k_lo, k_hi) hold only edges of the chunk that belong to nodes (no seed-clique
    // edge, no lane outside the chunk): every node there is whole
    const uint32_t nrows = (len + delta + 31) >> 5;
    uint32_t k_lo = delta > 0 ? 1 : 0;
    if (HasSeed && ei < m0) k_lo = nrows;  // the graph's first chunk: the general rows
    const uint32_t k_hi = (len + delta) >> 5;
    auto edge = [&](int32_t j, IT i, IT &u, IT &v) {  // the pair of chunk edge j (a node edge)
      const RT r = stage[j];
      u = n0 + ((i - m0) >> kLog);
      v = n0 + ((static_cast<IT>(r >> 1) - m0) >> kLog);
      if (HasSeed && __any_sync(kFull, r < two_m0)) {  // a chain that ended in the clique
        if (r < two_m0) v = static_cast<IT>(clique_position(r));
      }
    };
    // Another lane of the node holds the same key: the keys of lanes 1..D/2 places on,
    // cyclically, in independent chains of at most four one-place rotations (shorter
    // dependent shuffle chains), chain c starting 4c + 1 places on.
    auto repeat = [&](uint32_t key) {
      constexpr uint32_t kOffsets = D / 2;
      constexpr uint32_t kLen = kOffsets < 4 ? kOffsets : 4;
      bool seen = false;
#pragma unroll
      for (uint32_t c = 0; c < kOffsets / kLen; ++c) {
        uint32_t rot = __shfl_sync(kFull, key, static_cast<int>(lane + 1 + 4 * c), D);
        seen |= rot == key;
#pragma unroll
        for (uint32_t o = 1; o < kLen; ++o) {
          rot = __shfl_sync(kFull, rot, next, D);
          seen |= rot == key;
        }
      }
      return seen;
    };
    auto append = [&](bool list_it, IT i) {  // warp-collective: list the flagged nodes
      const uint32_t lb = __ballot_sync(kFull, list_it);
      if (lb != 0) {
        unsigned long long at = 0;
        if (lane == 0) at = atomicAdd(sp.fold_count, static_cast<unsigned long long>(__popc(lb)));
        at = __shfl_sync(kFull, at, 0) + __popc(lb & lt);
        if (list_it && at < sp.fold_cap)
          sp.fold_list[at] = static_cast<uint32_t>(((i - m0) >> kLog) - sp.fold_q0);
      }
    };
    for (uint32_t k = 0; k < nrows; ++k) {
      const int32_t j = static_cast<int32_t>(32 * k + lane) - static_cast<int32_t>(delta);
      const IT i = ei + static_cast<IT>(j);
      if (k >= k_lo && k < k_hi) {  // every lane on an edge of a whole node
        IT u, v;
        edge(j, i, u, v);
        if constexpr (!CountOnly) store_edge(dst, static_cast<uint32_t>(j), u, v);
        // a repeat among the node's targets (low 32 bits: equal halves of different
        // targets only send the node to the exact pass)
        const uint32_t sb = __ballot_sync(kFull, repeat(static_cast<uint32_t>(v)));
        if constexpr (CountOnly) {
          if ((sb & gm) == 0 && v < sp.fold_limit) atomicAdd(sp.fold_counts + v, 1ull);
        }
        if (sb != 0) append(leader && (sb & gm) != 0, i);
        continue;
      }
      // The general row: lanes outside the chunk, or seed-clique edges (part of no node).
      const bool in = j >= 0 && j < static_cast<int32_t>(len);
      const bool node_edge = in && (!HasSeed || i >= m0);
      IT v = 0;
      if (in) {
        IT u;
        if (HasSeed && i < m0) {
          u = static_cast<IT>(clique_position(2 * static_cast<uint64_t>(i)));
          v = static_cast<IT>(clique_position(2 * static_cast<uint64_t>(i) + 1));
        } else {
          const RT r = stage[j];
          u = n0 + ((i - m0) >> kLog);
          if (HasSeed && r < two_m0) v = static_cast<IT>(clique_position(r));
          else v = n0 + ((static_cast<IT>(r >> 1) - m0) >> kLog);
        }
        if constexpr (!CountOnly) store_edge(dst, static_cast<uint32_t>(j), u, v);
      }
      const bool seen = repeat(static_cast<uint32_t>(v));
      const uint32_t nb = __ballot_sync(kFull, node_edge);
      const uint32_t sb = __ballot_sync(kFull, node_edge && seen);
      const bool whole = (nb & gm) == gm;
      const bool settled = whole && (sb & gm) == 0;
      if constexpr (CountOnly) {
        if (node_edge && settled && v < sp.fold_limit) atomicAdd(sp.fold_counts + v, 1ull);
      }
      // To the list: a whole node with a repeat; a node cut by the chunk's ends, from the
      // chunk that holds its first edge, or from the range's first chunk when the node
      // starts before the range.  (The groups of seed-clique edges have no node edge.)
      append(leader && (nb & gm) != 0 && !settled && (whole || j >= 0 || first_chunk), i);
    }
  }

  template <class RT, bool HasSeed>
  __device__ __forceinline__ static void chunk(const RT *stage, uint64_t e0, uint32_t len,
                                               const GraphDev &g, int64_t *__restrict__ out,
                                               const SchedParams &sp) {
    __syncwarp();
    switch (g.d) {
      case 2: rows<2, RT, HasSeed>(stage, e0, len, g, out, sp); break;
      case 4: rows<4, RT, HasSeed>(stage, e0, len, g, out, sp); break;
      case 8: rows<8, RT, HasSeed>(stage, e0, len, g, out, sp); break;
      case 16: rows<16, RT, HasSeed>(stage, e0, len, g, out, sp); break;
      default: rows<32, RT, HasSeed>(stage, e0, len, g, out, sp); break;
    }
    __syncwarp();
  }
};

template <class RT, bool HasSeed, class Draw, bool CountOnly>
ba_status fold_t(const GraphDev &g, int64_t *out, const Shape &s, unsigned long long *counter,
                 cudaStream_t stream, SchedParams sp) {
  const uint64_t len = g.end - g.begin;
  // at most 256 threads a CTA: the flush takes the kernel to 64 registers, so larger CTAs
  // hold no more warps per SM (measured 1 % slower with 512)
  const int block = std::min(s.block, 256);
  const int warps = block / 32;
  const size_t smem = static_cast<size_t>(warps) * kRing * sizeof(RT);
  auto kernel = k_generate_refill<RT, HasSeed, false, false, Draw, 2, false, FoldDetect<CountOnly>>;
  ba_status st = set_smem(kernel, smem);
  if (st != BA_OK) return st;
  int grid = 0;
  st = persistent_grid(kernel, block, smem, s.ctas_per_sm, ~0ull, &grid);
  if (st != BA_OK) return st;
  uint32_t shift = static_cast<uint32_t>(floor_log2(static_cast<uint32_t>(s.tile)));
  const uint64_t all_warps = static_cast<uint64_t>(grid) * warps;
  while (shift > 8 && (len >> shift) < 4 * all_warps) --shift;  // as for generate
  sp.num_tiles = (len + (1ull << shift) - 1) >> shift;
  sp.counter = counter;
  sp.tile_shift = shift;
  grid = static_cast<int>(std::min<uint64_t>(grid, (sp.num_tiles + warps - 1) / warps));
  sp.total_warps = static_cast<uint32_t>(grid) * warps;
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  kernel<<<grid, block, smem, stream>>>(g, BatchTable{}, sp, out);
  return check_launch("k_generate_refill<fold>");
}

template <bool CountOnly>
ba_status fold_draw(const GraphDev &g, int64_t *out, const Shape &s, unsigned long long *counter,
                    cudaStream_t stream, bool no_loops, const SchedParams &sp) {
  const bool r32 = g.end <= (1ull << 31);
  if (no_loops) {  // needs a seed edge, so a seed clique
    using D = DrawVariant<false, true>;
    return r32 ? fold_t<uint32_t, true, D, CountOnly>(g, out, s, counter, stream, sp)
               : fold_t<uint64_t, true, D, CountOnly>(g, out, s, counter, stream, sp);
  }
  if (g.m0 > 0)
    return r32 ? fold_t<uint32_t, true, DrawPlainPtx, CountOnly>(g, out, s, counter, stream, sp)
               : fold_t<uint64_t, true, DrawPlainPtx, CountOnly>(g, out, s, counter, stream, sp);
  return r32 ? fold_t<uint32_t, false, DrawPlainPtx, CountOnly>(g, out, s, counter, stream, sp)
             : fold_t<uint64_t, false, DrawPlainPtx, CountOnly>(g, out, s, counter, stream, sp);
}

}  // namespace

bool fold_supported(uint32_t d) { return d >= 2 && d <= 32 && (d & (d - 1)) == 0; }

ba_status launch_generate_fold(const GraphDev &g, int64_t *out, const Shape &s,
                               unsigned long long *counter, cudaStream_t stream, bool no_loops,
                               uint32_t *list, unsigned long long *list_count, uint64_t q0,
                               uint64_t cap, uint64_t *counts, uint64_t node_limit) {
  if (!fold_supported(g.d)) return BA_ERR_INVALID_ARG;
  if (g.end == g.begin) return BA_OK;
  SchedParams sp{};
  sp.fold_list = list;
  sp.fold_count = list_count;
  sp.fold_q0 = q0;
  sp.fold_cap = cap;
  sp.fold_counts = reinterpret_cast<unsigned long long *>(counts);
  sp.fold_limit = node_limit;
  Shape shape = s;
  shape.chains = 2;
  if (out == nullptr) return fold_draw<true>(g, out, shape, counter, stream, no_loops, sp);
  return fold_draw<false>(g, out, shape, counter, stream, no_loops, sp);
}

}  // namespace ba
