// ba_simple.cu -- section 4's graph without parallel edges.
//
// The paper keeps the targets already generated for a node in a table of at most d
// entries and rejects a duplicate.  Here the generate kernel first writes every edge with
// the target of the array without rejection (the array every chain follows: the
// recursion of Fig. 1 cannot see rejections made while another node was generated).
// k_reject_duplicates then walks the nodes that own edges in range, one lane per edge of a
// node (d <= 32, so an item of a warp holds 32/d whole nodes; a warp takes kGroup items
// per pass, their loads in flight together; k_reject_duplicates_wide below takes nodes of
// 33..1024 edges, one warp per node):
//   1. each lane holds its edge's target (read back from the output, or recomputed for
//      the edges of the first node that lie before the range);
//   2. each lane compares its target (low 32 bits) with those of the next d/2 edges of its
//      node, cyclically, through shared memory; a pass without a repeat is done;
//   3. otherwise the flagged nodes' edges are taken in order: while an edge's candidate
//      is one of the targets accepted before it (a ballot over the node's lanes),
//      j < reach(u) and fewer than kRedrawCap redraws were made, its lane redraws: the
//      plain draw's range and key 2i+1 with the SplitMix64 bits of seed ^ k * kRedrawSalt,
//      then the array's chain from the drawn position.
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
// from position x.  Out of line, like redraw: both run for a few edges in 10^4 and would
// otherwise hold registers in the common path.
template <class RT, bool HasSeed, class Draw>
__device__ __noinline__ uint64_t array_value(RT x, const GraphDev &g, const Draw &draw, RT l2m0) {
  while (!chain_stops<RT, HasSeed>(x, l2m0)) x = draw(x);
  return target_of<RT, HasSeed>(x, g);
}

// Candidate k >= 1 for edge i: a draw over the plain draw's range keyed by 2i+1 with the
// salted seed, resolved through the array.
template <class RT, bool HasSeed, class Draw>
__device__ __noinline__ uint64_t redraw(uint64_t i, uint32_t k, const GraphDev &g, const Draw &draw, RT l2m0) {
  Draw salted = draw;
  salted.spre = seed_premix(g.seed ^ (static_cast<uint64_t>(k) * kRedrawSalt));
  return array_value<RT, HasSeed>(salted(static_cast<RT>(2 * i + 1)), g, draw, l2m0);
}

constexpr int kThreads = 256;
constexpr int kGroup = 4;  // items per pass of a warp's loop
constexpr uint32_t kNoKey = 0xffffffffu;

// Warp items of npw nodes n0 + q: item x holds the nodes of index x*npw + slot of the
// node sequence, lane = slot*d + j on edge m0 + q*d + j.  The sequence is q_lo..q_hi, or,
// Listed, q_lo + list[0 .. *list_count) (the nodes a fold launch handed on, each once),
// unless more than list_cap were handed on: then the list is incomplete and every node
// q_lo..q_hi is taken (the fold wrote the array's targets, so that is the full pass).
// Count: nothing is written back, and instead every edge's final target below node_limit
// is counted (section 3's streaming analysis of this graph: the sources are counted in
// closed form by the caller); the array's targets are read from `out`, scratch that the
// generate kernel has just filled with this range's edges, or, Recompute, recomputed.
template <class RT, bool HasSeed, class Draw, bool NoLoop, bool Count, bool Listed = false,
          bool Recompute = false>
__global__ void __launch_bounds__(kThreads)
k_reject_duplicates(const GraphDev g, int64_t *__restrict__ out,
                    unsigned long long *__restrict__ counts, uint64_t node_limit, uint64_t q_lo,
                    uint64_t q_hi, uint32_t npw, const uint32_t *__restrict__ list,
                    const unsigned long long *__restrict__ list_count, uint64_t list_cap) {
  // per warp: the low 32 bits of each node's targets, written twice in a row (entries j
  // and j + d) so that lane j reads entry j + o for every offset o without a wrap; node s's
  // row starts at word s * (d + 64), so the lanes of one read hit distinct banks (d >= 2:
  // at most 16 rows, the last ending below word 1024)
  __shared__ uint32_t key_rows[kThreads / 32][1024];
  Draw draw;
  draw.setup(g, nullptr, sizeof(RT) == 4);
  draw.bind(g);
  const RT l2m0 = seed_limit<RT>(g.two_m0);
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t d = g.d;
  const uint32_t W = npw * d;
  const uint32_t slot = lane / d;  // < 16 since d >= 2
  const uint32_t j = lane - slot * d;
  uint32_t *row = key_rows[threadIdx.x >> 5] + slot * (d + 64) + j;  // used by lanes < W
  const uint32_t half = d / 2;
  uint64_t nodes = q_hi - q_lo + 1;
  bool use_list = false;
  if constexpr (Listed) {
    const uint64_t listed = *list_count;
    if (listed <= list_cap) {
      nodes = min(nodes, listed);
      use_list = true;
    }
  }
  const uint64_t items = (nodes + npw - 1) / npw;
  const uint64_t groups = (items + kGroup - 1) / kGroup;
  const uint64_t warps = static_cast<uint64_t>(gridDim.x) * (kThreads / 32);
  long long *const tgt =  // targets: stride 2 (no output when recomputing)
      Recompute ? nullptr : reinterpret_cast<long long *>(out) + 1;
  for (uint64_t grp = static_cast<uint64_t>(blockIdx.x) * (kThreads / 32) + (threadIdx.x >> 5);
       grp < groups; grp += warps) {
    // This lane's node in item k of the group (q_lo + the sequence index; ~0 for none) and
    // its edge there.
    auto node_of = [&](int k) -> uint64_t {
      const uint64_t x = (grp * kGroup + k) * npw + slot;
      if (lane >= W || x >= nodes) return ~0ull;
      return use_list ? q_lo + list[x] : q_lo + x;
    };
    auto edge_of = [&](uint64_t q) { return q == ~0ull ? ~0ull : g.m0 + q * d + j; };
    // kGroup items per pass of the loop: their loads in flight together
    uint64_t t[kGroup];
#pragma unroll
    for (int k = 0; k < kGroup; ++k) {
      const uint64_t ik = edge_of(node_of(k));
      t[k] = 0;
      if (ik < g.end) {  // only the range's first node can start before it
        if (ik >= g.begin && !Recompute)
          t[k] = static_cast<uint64_t>(__ldcs(tgt + 2 * (g.out_edge + (ik - g.begin))));
        else
          t[k] = array_value<RT, HasSeed>(draw(static_cast<RT>(2 * ik + 1)), g, draw, l2m0);
      }
    }
    // Does another edge of the node have the same target?  Lane j compares its key (low
    // 32 bits) with the keys d/2 places after it, cyclically within the node, so every
    // pair is compared once; a key equal to the empty marker raises the flag too.  A false
    // alarm only sends the node through the exact pass below.  (__match_any_sync
    // serialises over the distinct values of the warp; a hash table with shared-memory
    // atomicCAS and a count over the whole row were slower than this.)
    uint32_t flags = 0;
#pragma unroll
    for (int k = 0; k < kGroup; ++k) {
      const bool part = edge_of(node_of(k)) < g.end;  // the edge matters to its node
      const uint32_t key = static_cast<uint32_t>(t[k]);
      __syncwarp();
      if (lane < W) row[0] = row[d] = part ? key : kNoKey;
      __syncwarp();
      bool seen = key == kNoKey;
      if (lane < W) {
#pragma unroll 4
        for (uint32_t o = 1; o <= half; ++o) seen |= row[o] == key;
      }
      flags |= (part && seen) ? 1u << k : 0u;
    }
    // Count: an edge of the range whose final target is a counted node adds one to it
    auto count = [&](uint64_t i, uint64_t target) {
      if constexpr (Count) {
        if (i < g.end && i >= g.begin && target < node_limit) atomicAdd(counts + target, 1ull);
      }
    };
    if (__ballot_sync(kAll, flags != 0) == 0) {
      if constexpr (Count) {
#pragma unroll
        for (int k = 0; k < kGroup; ++k) count(edge_of(node_of(k)), t[k]);
      }
      continue;
    }
    // Exact pass, node by node, edges in order: an edge whose candidate one of the node's
    // earlier edges has accepted draws again while a new target exists and redraws are left.
#pragma unroll 1
    for (int k = 0; k < kGroup; ++k) {
      uint32_t dups = __ballot_sync(kAll, (flags >> k) & 1u);
      const uint64_t q_k = node_of(k);
      const uint64_t i = edge_of(q_k);
      if (dups == 0) {
        if constexpr (Count) count(i, k == 0 ? t[0] : k == 1 ? t[1] : k == 2 ? t[2] : t[3]);
        continue;
      }
      const bool part = i < g.end;
      const uint32_t parts = __ballot_sync(kAll, part);
      const uint64_t t_k = k == 0 ? t[0] : k == 1 ? t[1] : k == 2 ? t[2] : t[3];
      uint64_t acc = t_k;
      while (dups) {
        const uint32_t base = ((__ffs(dups) - 1) / d) * d;
        const uint32_t node_lanes = (d == 32 ? kAll : ((1u << d) - 1u)) << base;
        const uint64_t node = g.n0 + __shfl_sync(kAll, q_k, base);
        const uint64_t reach = NoLoop ? node : (g.n0 == 1 ? node : node + 1);
        for (uint32_t L = base + 1; L < base + d && ((parts >> L) & 1u); ++L) {
          const uint64_t iL = i - lane + L;
          uint64_t cand = __shfl_sync(kAll, acc, L);
          uint32_t r = 0;
          for (;;) {
            const bool taken = __ballot_sync(kAll, lane >= base && lane < L && acc == cand) != 0;
            if (!taken || L - base >= reach || r >= kRedrawCap) break;
            ++r;
            uint64_t v = 0;
            if (lane == L) v = redraw<RT, HasSeed>(iL, r, g, draw, l2m0);
            cand = __shfl_sync(kAll, v, L);
          }
          if (lane == L) acc = cand;
        }
        dups &= ~node_lanes;
      }
      if constexpr (Count) {
        count(i, acc);
      } else if (part && i >= g.begin && acc != t_k) {
        __stcs(tgt + 2 * (g.out_edge + (i - g.begin)), static_cast<long long>(acc));
      }
    }
  }
}

// ---------------------------------------------------------------- wide nodes, d > 32 --
//
// One warp per node: the node's targets (read back, or recomputed for the edges of the
// range's first node that lie before it) go to the warp's shared row 32 at a time, and
// each lane inserts (low 32 bits of its target, its index) into the warp's open-addressing
// table (2d..4d slots, linear probing, 64-bit atomicCAS).  A lane that finds its key
// already there flags both itself and the index stored with it, so every edge whose target
// repeats another edge's is flagged (a false alarm, equal low halves, only costs work).
// The exact pass then takes just the flagged edges, in order, as the narrow kernel takes
// all of them: while the candidate is among the targets accepted before it (a warp-wide
// scan of the row), j < reach(u) and redraws are left, lane 0 redraws.  A changed target
// can make a later, unflagged edge collide, so a change flags every later edge holding the
// new value.  An edge never flagged keeps its target, as the full in-order pass would:
// nothing accepted before it can equal its target without one of the two flags above.
constexpr int kWideThreads = 128;
constexpr uint32_t kWideMaxD = 1024;
constexpr unsigned long long kNoEntry = ~0ull;

__host__ __device__ constexpr uint32_t wide_table_bits(uint32_t d) {
  uint32_t b = 6;  // at least 64 slots
  while ((1u << b) < 2 * d) ++b;
  return b;
}
// Per warp: the row (d targets), the table (8 bytes a slot) and the flags (1 bit an edge).
__host__ __device__ constexpr size_t wide_warp_bytes(uint32_t d) {
  return static_cast<size_t>(d) * 8 + (static_cast<size_t>(8) << wide_table_bits(d)) +
         static_cast<size_t>(kWideMaxD / 32) * 4;
}

template <class RT, bool HasSeed, class Draw, bool NoLoop, bool Count>
__global__ void __launch_bounds__(kWideThreads)
k_reject_duplicates_wide(const GraphDev g, int64_t *__restrict__ out,
                         unsigned long long *__restrict__ counts, uint64_t node_limit,
                         uint64_t q_lo, uint64_t q_hi) {
  extern __shared__ __align__(16) unsigned char wide_smem[];
  const uint32_t d = g.d;
  const uint32_t bits = wide_table_bits(d);
  const uint32_t P = 1u << bits;
  const uint32_t words = (d + 31) / 32;
  unsigned char *mine = wide_smem + static_cast<size_t>(threadIdx.x >> 5) * wide_warp_bytes(d);
  uint64_t *tt = reinterpret_cast<uint64_t *>(mine);                      // the node's targets
  unsigned long long *tab =
      reinterpret_cast<unsigned long long *>(mine + static_cast<size_t>(d) * 8);  // P entries
  uint32_t *flag = reinterpret_cast<uint32_t *>(mine + static_cast<size_t>(d) * 8 +
                                                (static_cast<size_t>(8) << bits));  // words
  Draw draw;
  draw.setup(g, nullptr, sizeof(RT) == 4);
  draw.bind(g);
  const RT l2m0 = seed_limit<RT>(g.two_m0);
  const uint32_t lane = threadIdx.x & 31;
  long long *const tgt = reinterpret_cast<long long *>(out) + 1;  // targets: stride 2
  const uint64_t warps = static_cast<uint64_t>(gridDim.x) * (kWideThreads / 32);
  auto mark = [&](uint32_t j) { atomicOr(flag + (j >> 5), 1u << (j & 31)); };
  for (uint64_t q = q_lo + static_cast<uint64_t>(blockIdx.x) * (kWideThreads / 32) + (threadIdx.x >> 5);
       q <= q_hi; q += warps) {
    const uint64_t node = g.n0 + q;
    const uint64_t first = g.m0 + q * d;
    const uint32_t cnt = static_cast<uint32_t>(min(static_cast<uint64_t>(d), g.end - first));
    __syncwarp();  // the previous node's row, table and flags are no longer read
    for (uint32_t k = lane; k < P; k += 32) tab[k] = kNoEntry;
    if (lane < words) flag[lane] = 0;
    __syncwarp();
    for (uint32_t j0 = 0; j0 < cnt; j0 += 32) {
      const uint32_t j = j0 + lane;
      if (j < cnt) {
        const uint64_t i = first + j;
        uint64_t t;
        if (i >= g.begin)
          t = static_cast<uint64_t>(__ldcs(tgt + 2 * (g.out_edge + (i - g.begin))));
        else
          t = array_value<RT, HasSeed>(draw(static_cast<RT>(2 * i + 1)), g, draw, l2m0);
        tt[j] = t;
        const uint32_t key = static_cast<uint32_t>(t);
        if (key == kNoKey) {
          mark(j);  // the key of an empty slot: every such edge flags itself
        } else {
          const unsigned long long entry = (static_cast<unsigned long long>(key) << 32) | j;
          uint32_t h = (key * 0x9E3779B1u) >> (32 - bits);
          for (;;) {  // at most d keys in >= 2d slots: an empty slot always exists
            const unsigned long long old = atomicCAS(tab + h, kNoEntry, entry);
            if (old == kNoEntry) break;
            if (static_cast<uint32_t>(old >> 32) == key) {
              mark(j);
              mark(static_cast<uint32_t>(old));
              break;
            }
            h = (h + 1) & (P - 1);
          }
        }
      }
    }
    __syncwarp();
    // Count: every edge of the range adds one to its final target if that is counted
    auto count_node = [&]() {
      if constexpr (Count) {
        __syncwarp();
        for (uint32_t j = lane; j < cnt; j += 32) {
          const uint64_t t = tt[j];
          if (first + j >= g.begin && t < node_limit) atomicAdd(counts + t, 1ull);
        }
      }
    };
    if (!__any_sync(kAll, lane < words && flag[lane] != 0)) {
      count_node();
      continue;
    }
    const uint64_t reach = NoLoop ? node : (g.n0 == 1 ? node : node + 1);
    for (uint32_t w = 0; w < words; ++w) {
      uint32_t pending = flag[w];
      while (pending) {
        const uint32_t b = __ffs(pending) - 1;
        const uint32_t j = 32 * w + b;
        if (j > 0 && j < cnt) {  // edge 0 has nothing accepted before it
          const uint64_t orig = tt[j];
          uint64_t cand = orig;
          uint32_t r = 0;
          for (;;) {
            bool taken = false;
            for (uint32_t l = lane; l < j; l += 32) taken |= tt[l] == cand;
            if (!__any_sync(kAll, taken) || j >= reach || r >= kRedrawCap) break;
            ++r;
            uint64_t v = 0;
            if (lane == 0) v = redraw<RT, HasSeed>(first + j, r, g, draw, l2m0);
            cand = __shfl_sync(kAll, v, 0);
          }
          if (cand != orig) {
            const uint64_t i = first + j;
            if (lane == 0) {
              tt[j] = cand;
              if (!Count && i >= g.begin)
                __stcs(tgt + 2 * (g.out_edge + (i - g.begin)), static_cast<long long>(cand));
            }
            // a later edge holding the new value now collides with it
            for (uint32_t k = j + 1 + lane; k < cnt; k += 32)
              if (tt[k] == cand) mark(k);
            __syncwarp();
          }
        }
        // the flags above b, read again: the forward scan may have set some
        pending = flag[w] & ((~0u << b) << 1);
      }
    }
    count_node();
  }
}

template <class RT, bool HasSeed, class Draw, bool NoLoop, bool Count>
ba_status launch_wide_t(const GraphDev &g, int64_t *out, unsigned long long *counts,
                        uint64_t node_limit, uint64_t q_lo, uint64_t q_hi, cudaStream_t stream) {
  auto kernel = k_reject_duplicates_wide<RT, HasSeed, Draw, NoLoop, Count>;
  const size_t smem = (kWideThreads / 32) * wide_warp_bytes(g.d);
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kWideThreads, smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  const uint64_t nodes = q_hi - q_lo + 1;
  const uint64_t want = (nodes + kWideThreads / 32 - 1) / (kWideThreads / 32);
  const int grid = static_cast<int>(std::min<uint64_t>(
      want, static_cast<uint64_t>(sm_count()) * static_cast<uint64_t>(std::max(per_sm, 1))));
  kernel<<<grid, kWideThreads, smem, stream>>>(g, out, counts, node_limit, q_lo, q_hi);
  e = cudaGetLastError();
  return e == cudaSuccess ? BA_OK : cuda_fail(e, "k_reject_duplicates_wide");
}

template <class RT, bool HasSeed, class Draw, bool NoLoop, bool Count>
ba_status launch_t(const GraphDev &g, int64_t *out, unsigned long long *counts,
                   uint64_t node_limit, uint64_t q_lo, uint64_t q_hi, uint32_t npw,
                   cudaStream_t stream) {
  auto kernel = k_reject_duplicates<RT, HasSeed, Draw, NoLoop, Count>;
  constexpr int kBlock = kThreads;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, 0);
  if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  const uint64_t items = (q_hi - q_lo) / npw + 1;
  const uint64_t groups = (items + kGroup - 1) / kGroup;
  const uint64_t want = (groups + kBlock / 32 - 1) / (kBlock / 32);
  const int grid = static_cast<int>(std::min<uint64_t>(
      want, static_cast<uint64_t>(sm_count()) * static_cast<uint64_t>(std::max(per_sm, 1))));
  kernel<<<grid, kBlock, 0, stream>>>(g, out, counts, node_limit, q_lo, q_hi, npw, nullptr,
                                      nullptr, 0);
  e = cudaGetLastError();
  return e == cudaSuccess ? BA_OK : cuda_fail(e, "k_reject_duplicates");
}

// The listed nodes only: the list's length is on the device, so the grid is the
// persistent one and the warps stride over the items.
template <class RT, bool HasSeed, class Draw, bool NoLoop, bool Count>
ba_status launch_listed_t(const GraphDev &g, int64_t *out, unsigned long long *counts,
                          uint64_t node_limit, uint64_t q_lo, uint64_t q_hi, uint32_t npw,
                          const uint32_t *list, const unsigned long long *list_count,
                          uint64_t list_cap, cudaStream_t stream) {
  auto kernel = k_reject_duplicates<RT, HasSeed, Draw, NoLoop, Count, true, Count>;
  constexpr int kBlock = kThreads;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, 0);
  if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  const uint64_t items = (q_hi - q_lo) / npw + 1;  // at most this many
  const uint64_t groups = (items + kGroup - 1) / kGroup;
  const uint64_t want = (groups + kBlock / 32 - 1) / (kBlock / 32);
  const int grid = static_cast<int>(std::min<uint64_t>(
      want, static_cast<uint64_t>(sm_count()) * static_cast<uint64_t>(std::max(per_sm, 1))));
  kernel<<<grid, kBlock, 0, stream>>>(g, out, counts, node_limit, q_lo, q_hi, npw, list,
                                      list_count, list_cap);
  e = cudaGetLastError();
  return e == cudaSuccess ? BA_OK : cuda_fail(e, "k_reject_duplicates<listed>");
}

// The nodes with edges in [g.begin, g.end), then the launch for the draw family.
template <bool Count>
ba_status reject_range(const GraphDev &g, int64_t *out, unsigned long long *counts,
                       uint64_t node_limit, cudaStream_t stream, bool no_loops) {
  if (g.d <= 1 || g.d > kWideMaxD) return g.d <= 1 ? BA_OK : BA_ERR_INVALID_ARG;
  const uint64_t a = std::max(g.begin, g.m0);
  if (a >= g.end) return BA_OK;  // only seed-clique edges in range
  const uint64_t q_lo = (a - g.m0) / g.d;
  const uint64_t q_hi = (g.end - 1 - g.m0) / g.d;
  const bool r32 = g.end <= (1ull << 31);
  if (g.d > 32) {  // one warp per node
    if (no_loops) {
      using D = DrawVariant<false, true>;
      return r32 ? launch_wide_t<uint32_t, true, D, true, Count>(g, out, counts, node_limit, q_lo, q_hi, stream)
                 : launch_wide_t<uint64_t, true, D, true, Count>(g, out, counts, node_limit, q_lo, q_hi, stream);
    }
    if (g.m0 > 0)
      return r32 ? launch_wide_t<uint32_t, true, DrawPlain, false, Count>(g, out, counts, node_limit, q_lo, q_hi, stream)
                 : launch_wide_t<uint64_t, true, DrawPlain, false, Count>(g, out, counts, node_limit, q_lo, q_hi, stream);
    return r32 ? launch_wide_t<uint32_t, false, DrawPlain, false, Count>(g, out, counts, node_limit, q_lo, q_hi, stream)
               : launch_wide_t<uint64_t, false, DrawPlain, false, Count>(g, out, counts, node_limit, q_lo, q_hi, stream);
  }
  const uint32_t npw = 32u / g.d;
  if (no_loops) {  // needs a seed edge, so a seed clique
    using D = DrawVariant<false, true>;
    return r32 ? launch_t<uint32_t, true, D, true, Count>(g, out, counts, node_limit, q_lo, q_hi, npw, stream)
               : launch_t<uint64_t, true, D, true, Count>(g, out, counts, node_limit, q_lo, q_hi, npw, stream);
  }
  if (g.m0 > 0)
    return r32 ? launch_t<uint32_t, true, DrawPlain, false, Count>(g, out, counts, node_limit, q_lo, q_hi, npw, stream)
               : launch_t<uint64_t, true, DrawPlain, false, Count>(g, out, counts, node_limit, q_lo, q_hi, npw, stream);
  return r32 ? launch_t<uint32_t, false, DrawPlain, false, Count>(g, out, counts, node_limit, q_lo, q_hi, npw, stream)
             : launch_t<uint64_t, false, DrawPlain, false, Count>(g, out, counts, node_limit, q_lo, q_hi, npw, stream);
}

// The listed nodes of a fold launch, for the draw family (Count: the fold wrote nothing,
// so the targets are recomputed).
template <bool Count>
ba_status reject_listed(const GraphDev &g, int64_t *out, unsigned long long *counts,
                        uint64_t node_limit, const uint32_t *list,
                        const unsigned long long *list_count, uint64_t list_cap, uint64_t q_lo,
                        uint64_t q_hi, cudaStream_t stream, bool no_loops) {
  const uint32_t npw = 32u / g.d;
  const bool r32 = g.end <= (1ull << 31);
  if (no_loops) {
    using D = DrawVariant<false, true>;
    return r32 ? launch_listed_t<uint32_t, true, D, true, Count>(g, out, counts, node_limit, q_lo, q_hi, npw, list, list_count, list_cap, stream)
               : launch_listed_t<uint64_t, true, D, true, Count>(g, out, counts, node_limit, q_lo, q_hi, npw, list, list_count, list_cap, stream);
  }
  if (g.m0 > 0)
    return r32 ? launch_listed_t<uint32_t, true, DrawPlain, false, Count>(g, out, counts, node_limit, q_lo, q_hi, npw, list, list_count, list_cap, stream)
               : launch_listed_t<uint64_t, true, DrawPlain, false, Count>(g, out, counts, node_limit, q_lo, q_hi, npw, list, list_count, list_cap, stream);
  return r32 ? launch_listed_t<uint32_t, false, DrawPlain, false, Count>(g, out, counts, node_limit, q_lo, q_hi, npw, list, list_count, list_cap, stream)
             : launch_listed_t<uint64_t, false, DrawPlain, false, Count>(g, out, counts, node_limit, q_lo, q_hi, npw, list, list_count, list_cap, stream);
}

}  // namespace

ba_status launch_reject_listed(const GraphDev &g, int64_t *out, uint64_t *counts,
                               uint64_t node_limit, const uint32_t *list,
                               const unsigned long long *list_count, uint64_t list_cap,
                               uint64_t q0, uint64_t q_hi, cudaStream_t stream, bool no_loops) {
  if (g.d < 2 || g.d > 32 || q_hi < q0) return BA_ERR_INVALID_ARG;
  if (out == nullptr)
    return reject_listed<true>(g, nullptr, reinterpret_cast<unsigned long long *>(counts),
                               node_limit, list, list_count, list_cap, q0, q_hi, stream,
                               no_loops);
  return reject_listed<false>(g, out, nullptr, 0, list, list_count, list_cap, q0, q_hi, stream,
                              no_loops);
}

ba_status launch_reject_duplicates(const GraphDev &g, int64_t *out, cudaStream_t stream,
                                   bool no_loops) {
  return reject_range<false>(g, out, nullptr, 0, stream, no_loops);
}

ba_status launch_count_rejections(const GraphDev &g, const int64_t *pairs, uint64_t node_limit,
                                  uint64_t *counts, cudaStream_t stream, bool no_loops) {
  return reject_range<true>(g, const_cast<int64_t *>(pairs),  // read only in this mode
                            reinterpret_cast<unsigned long long *>(counts), node_limit, stream,
                            no_loops);
}

}  // namespace ba
