// ba_refill.cuh -- the refill generate kernel (paper Fig. 1 over a range of edge IDs) and
// the launch helpers it shares between translation units: ba_kernels.cu launches it for
// the edge lists, the batched tables and the variant draws; ba_fold.cu launches it with a
// chunk flush that also looks for section 4's parallel edges (the Fold policy).
#pragma once
#include <algorithm>
#include <type_traits>

#include "ba_draw.cuh"
#include "ba_internal.h"

namespace ba {
namespace {

constexpr uint32_t kFull = 0xffffffffu;

// One (source, target) pair: two int64 (16 bytes) or, with Narrow, two int32 (8 bytes).
template <bool Narrow>
__device__ __forceinline__ void store_pair(int64_t *out, uint64_t k, uint64_t u, uint64_t v) {
  if constexpr (Narrow)
    __stcs(reinterpret_cast<int2 *>(out) + k, make_int2(static_cast<int>(u), static_cast<int>(v)));
  else
    store_edge(out, k, u, v);
}

// ------------------------------------------------------------ warp tile scheduling --

// Takes the warp's next tile index: the first one is the warp's own index, later ones
// come from the global counter.  Warp-collective.
__device__ __forceinline__ uint64_t next_tile(const SchedParams &sp, bool &first,
                                              uint64_t gwarp) {
  if (first) {
    first = false;
    return gwarp;
  }
  unsigned long long t = 0;
  if ((threadIdx.x & 31) == 0) t = atomicAdd(sp.counter, 1ull);
  return __shfl_sync(kFull, t, 0) + sp.total_warps;
}

// Graph that owns global tile t of a batched launch (binary search in the tile prefix).
__device__ __forceinline__ int graph_of_tile(const BatchTable &tab, uint64_t t) {
  int lo = 0, hi = tab.G;  // tile_prefix[lo] <= t < tile_prefix[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (tab.tile_prefix[mid] <= t) lo = mid; else hi = mid;
  }
  return lo;
}

// Warp-collective copy of one GraphDev into shared memory.
__device__ __forceinline__ void copy_graph(GraphDev *dst, const GraphDev *src) {
  constexpr int kWords = sizeof(GraphDev) / 8;
  static_assert(sizeof(GraphDev) % 8 == 0, "GraphDev must be a whole number of words");
  const int lane = threadIdx.x & 31;
  if (lane < kWords)
    reinterpret_cast<uint64_t *>(dst)[lane] = reinterpret_cast<const uint64_t *>(src)[lane];
  __syncwarp();
}

// Writes the finished chunk [base, base+len) of the staging ring: lane j of the warp
// handles edges base+j, base+j+32, ... so each warp store covers 512 contiguous bytes (256
// with Narrow int32 pairs).
// Checked: a store to slot out_cap or beyond is skipped and the lowest such slot is kept in
// *status (the checked launch; the slot bound comes from the caller, not from the range).
template <class RT, bool HasSeed, bool Narrow = false, bool Checked = false, bool Full = false>
__device__ __forceinline__ void flush_tile(const RT *stage, uint64_t base, uint32_t len,
                                           const GraphDev &g, int64_t *__restrict__ out,
                                           uint64_t out_cap = 0,
                                           unsigned long long *status = nullptr) {
  __syncwarp();
  const uint64_t out0 = g.out_edge + (base - g.begin);
  // fn(j, k) for the lane's edges j = lane + 32k < len; Full: len is 256 (8 per lane)
  auto each = [&](auto fn) {
    if constexpr (Full) {
#pragma unroll
      for (uint32_t k = 0; k < 8; ++k) fn((threadIdx.x & 31) + 32 * k, k);
    } else {
      uint32_t k = 0;
      for (uint32_t j = threadIdx.x & 31; j < len; j += 32, ++k) fn(j, k);
    }
  };
  // false (and the slot recorded) when slot k does not exist
  [[maybe_unused]] auto slot_ok = [&](uint64_t k) {
    if constexpr (Checked) {
      if (k >= out_cap) {
        atomicMin(status, static_cast<unsigned long long>(k));
        return false;
      }
    }
    return true;
  };
  if constexpr (sizeof(RT) == 4) {
    // 32-bit positions: i < 2^31 and every node ID < 2^32, so the pairs are built from
    // 32-bit words (high words zero).
    // The graph's constants in registers (in a batched launch `g` lives in shared memory).
    const uint32_t n0 = static_cast<uint32_t>(g.n0);
    const uint32_t m0 = static_cast<uint32_t>(g.m0);
    const uint32_t seed_m0 = g.m0 > 0xffffffffull ? 0xffffffffu : static_cast<uint32_t>(g.m0);
    const uint32_t two_m0 = seed_limit<uint32_t>(g.two_m0);
    const FastDiv dv = g.div;
    const uint32_t b32 = static_cast<uint32_t>(base);
    int4 *dst = reinterpret_cast<int4 *>(out) + out0;
    int2 *dst2 = reinterpret_cast<int2 *>(out) + out0;
    // d a power of two (d = 2^l): the divisions are shifts.
    auto body = [&](auto pow2_tag) {
      constexpr bool Pow2 = decltype(pow2_tag)::value;
      // d not a power of two: d >= 3, so l >= 2 and the multiply-high path always applies
      const uint32_t np2_shift = dv.l - 1;
      auto div = [&](uint32_t x) -> uint32_t {
        if constexpr (Pow2) return x >> dv.l;
        else return __umulhi(x, dv.m32) >> np2_shift;
      };
      auto put = [&](uint32_t j, uint32_t u, uint32_t v) {
        if (!slot_ok(out0 + j)) return;
        if constexpr (Narrow)
          __stcs(dst2 + j, make_int2(static_cast<int>(u), static_cast<int>(v)));
        else
          __stcs(dst + j, make_int4(static_cast<int>(u), 0, static_cast<int>(v), 0));
      };
      if (n0 == 0) {  // also the unseeded graphs of a batched launch that has seeded ones
        // Empty seed graph: source i/d, target (r/2)/d; with d = 2^l both are one shift.
        const uint32_t l1 = dv.l + 1;
        each([&](uint32_t j, uint32_t) {
          const uint32_t r = stage[j];
          if constexpr (Pow2) put(j, (b32 + j) >> dv.l, r >> l1);
          else put(j, div(b32 + j), div(r >> 1));
        });
      } else {
        // A chain that stopped inside the seed names a clique node (a few in 10^4 chains:
        // the seed nodes' share of all end points).  Bit k of `fix` marks the lane's k-th
        // edge of the chunk as one; those few pairs are rewritten afterwards.
        [[maybe_unused]] uint32_t fix = 0;
        each([&](uint32_t j, uint32_t k) {
          const uint32_t i = b32 + j;
          const uint32_t r = stage[j];
          if constexpr (HasSeed) fix |= r < two_m0 ? 1u << k : 0u;
          put(j, n0 + div(i - m0), n0 + div((r >> 1) - m0));
        });
        if constexpr (HasSeed) {
          if (__any_sync(kFull, fix != 0)) {
            while (fix) {  // by the lane that wrote the pair
              const uint32_t j = (threadIdx.x & 31) + 32u * (__ffs(fix) - 1);
              fix &= fix - 1;
              put(j, n0 + div(b32 + j - m0), static_cast<uint32_t>(clique_position(stage[j])));
            }
          }
        }
      }
      if constexpr (HasSeed) {
        // The seed edges themselves (the graph's first m0) sit in its first chunks only.
        if (b32 < seed_m0) {
          for (uint32_t j = threadIdx.x & 31; j < len; j += 32) {
            const uint32_t i = b32 + j;
            if (i < seed_m0)
              put(j, static_cast<uint32_t>(clique_position(2 * static_cast<uint64_t>(i))),
                  static_cast<uint32_t>(clique_position(2 * static_cast<uint64_t>(i) + 1)));
          }
        }
      }
    };
    if (dv.pow2) body(std::true_type{});
    else body(std::false_type{});
  } else if (g.n0 == 0 && g.div.pow2) {
    // Empty seed graph, d = 2^l (every request of a typical serving mix): one shift each
    // instead of two 64-bit multiply-highs.
    const uint32_t l = g.div.l;
    each([&](uint32_t j, uint32_t) {
      if (slot_ok(out0 + j))
        store_pair<Narrow>(out, out0 + j, (base + j) >> l, static_cast<uint64_t>(stage[j]) >> (l + 1));
    });
  } else {
    each([&](uint32_t j, uint32_t) {
      const uint64_t i = base + j;
      uint64_t u, v;
      if (HasSeed && i < g.m0) {
        u = clique_position(2 * i);
        v = clique_position(2 * i + 1);
      } else {
        u = source_of<RT, HasSeed>(i, g);
        v = target_of<RT, HasSeed>(stage[j], g);
      }
      if (slot_ok(out0 + j)) store_pair<Narrow>(out, out0 + j, u, v);
    });
  }
  __syncwarp();
}

// ----------------------------------------------------------- refill generate kernel --

// Per-warp staging ring: the final position r of edge (tile offset) o is parked at
// ring[o mod kRing] until the 256-edge chunk that holds it is complete and written out.
constexpr uint32_t kRing = 1024;
constexpr uint32_t kChunk = 256;

// One fast step's bookkeeping for one chain as predicated PTX: the stop test of Fig. 1
// (r even, or inside the seed clique), the parked store of a final r into the staging ring,
// the warp's ballot and the hand-out of the next IDs of the tile (rank among the stopped
// lanes).  r, o and hoff are updated in place; ring_s is the ring's shared-space address.
template <bool Seed>
__device__ __forceinline__ void park_and_refill(uint32_t &r, uint32_t &o, uint32_t &hoff,
                                                uint32_t lt, uint32_t r0, uint32_t two_m0,
                                                uint32_t ring_s) {
  if constexpr (Seed) {
    asm volatile(
        "{\n\t"
        ".reg .pred p;\n\t"
        ".reg .u32 t, a, fm, x;\n\t"
        "and.b32 t, %0, 1;\n\t"
        "setp.eq.u32 p, t, 0;\n\t"
        "setp.lt.or.u32 p, %0, %6, p;\n\t"
        "and.b32 a, %1, 1023;\n\t"
        "shl.b32 a, a, 2;\n\t"
        "add.u32 a, a, %5;\n\t"
        "@p st.shared.u32 [a], %0;\n\t"
        "vote.sync.ballot.b32 fm, p, 0xffffffff;\n\t"
        "and.b32 x, fm, %3;\n\t"
        "popc.b32 x, x;\n\t"
        "@p add.u32 %1, %2, x;\n\t"
        "@p mad.lo.u32 %0, %1, 2, %4;\n\t"
        "popc.b32 x, fm;\n\t"
        "add.u32 %2, %2, x;\n\t"
        "}"
        : "+r"(r), "+r"(o), "+r"(hoff)
        : "r"(lt), "r"(r0), "r"(ring_s), "r"(two_m0)
        : "memory");
  } else {
    asm volatile(
        "{\n\t"
        ".reg .pred p;\n\t"
        ".reg .u32 t, a, fm, x;\n\t"
        "and.b32 t, %0, 1;\n\t"
        "setp.eq.u32 p, t, 0;\n\t"
        "and.b32 a, %1, 1023;\n\t"
        "shl.b32 a, a, 2;\n\t"
        "add.u32 a, a, %5;\n\t"
        "@p st.shared.u32 [a], %0;\n\t"
        "vote.sync.ballot.b32 fm, p, 0xffffffff;\n\t"
        "and.b32 x, fm, %3;\n\t"
        "popc.b32 x, x;\n\t"
        "@p add.u32 %1, %2, x;\n\t"
        "@p mad.lo.u32 %0, %1, 2, %4;\n\t"
        "popc.b32 x, fm;\n\t"
        "add.u32 %2, %2, x;\n\t"
        "}"
        : "+r"(r), "+r"(o), "+r"(hoff)
        : "r"(lt), "r"(r0), "r"(ring_s)
        : "memory");
  }
}
// 64-bit positions: the next ID's position r0 + 2o is handed out on the two 32-bit halves
// as a predicated carry chain (a predicated 64-bit multiply-add measured 1.7 % slower).
template <bool Seed>
__device__ __forceinline__ void park_and_refill(uint64_t &r, uint32_t &o, uint32_t &hoff,
                                                uint32_t lt, uint64_t r0, uint64_t two_m0,
                                                uint32_t ring_s) {
  if constexpr (Seed) {
    asm volatile(
        "{\n\t"
        ".reg .pred p;\n\t"
        ".reg .u32 t, a, fm, x, rl, rh, nl, nh;\n\t"
        "cvt.u32.u64 t, %0;\n\t"
        "and.b32 t, t, 1;\n\t"
        "setp.eq.u32 p, t, 0;\n\t"
        "setp.lt.or.u64 p, %0, %6, p;\n\t"
        "and.b32 a, %1, 1023;\n\t"
        "shl.b32 a, a, 3;\n\t"
        "add.u32 a, a, %5;\n\t"
        "@p st.shared.u64 [a], %0;\n\t"
        "vote.sync.ballot.b32 fm, p, 0xffffffff;\n\t"
        "and.b32 x, fm, %3;\n\t"
        "popc.b32 x, x;\n\t"
        "@p add.u32 %1, %2, x;\n\t"
        "mov.b64 {rl, rh}, %4;\n\t"
        "mov.b64 {nl, nh}, %0;\n\t"
        "@p mad.lo.cc.u32 nl, %1, 2, rl;\n\t"
        "@p addc.u32 nh, rh, 0;\n\t"
        "mov.b64 %0, {nl, nh};\n\t"
        "popc.b32 x, fm;\n\t"
        "add.u32 %2, %2, x;\n\t"
        "}"
        : "+l"(r), "+r"(o), "+r"(hoff)
        : "r"(lt), "l"(r0), "r"(ring_s), "l"(two_m0)
        : "memory");
  } else {
    asm volatile(
        "{\n\t"
        ".reg .pred p;\n\t"
        ".reg .u32 t, a, fm, x, rl, rh, nl, nh;\n\t"
        "cvt.u32.u64 t, %0;\n\t"
        "and.b32 t, t, 1;\n\t"
        "setp.eq.u32 p, t, 0;\n\t"
        "and.b32 a, %1, 1023;\n\t"
        "shl.b32 a, a, 3;\n\t"
        "add.u32 a, a, %5;\n\t"
        "@p st.shared.u64 [a], %0;\n\t"
        "vote.sync.ballot.b32 fm, p, 0xffffffff;\n\t"
        "and.b32 x, fm, %3;\n\t"
        "popc.b32 x, x;\n\t"
        "@p add.u32 %1, %2, x;\n\t"
        "mov.b64 {rl, rh}, %4;\n\t"
        "mov.b64 {nl, nh}, %0;\n\t"
        "@p mad.lo.cc.u32 nl, %1, 2, rl;\n\t"
        "@p addc.u32 nh, rh, 0;\n\t"
        "mov.b64 %0, {nl, nh};\n\t"
        "popc.b32 x, fm;\n\t"
        "add.u32 %2, %2, x;\n\t"
        "}"
        : "+l"(r), "+r"(o), "+r"(hoff)
        : "r"(lt), "l"(r0), "r"(ring_s)
        : "memory");
  }
}

// The chunk flush's policy: NoFold writes the pairs (flush_tile); a policy with kActive
// supplies its own chunk(stage, first edge, edges, graph, out, sched params) instead.
struct NoFold {
  static constexpr bool kActive = false;
};

// K chains per lane: lane l runs the chains of virtual lanes l, l+32, ..., l+32(K-1), so
// each lane has K independent hash chains in flight.  The hash is one long dependency
// chain of integer multiplies and shifts; a second chain per lane hides its latency.
template <class RT, bool HasSeed, bool Batched, bool Narrow = false, class Draw = DrawPlainPtx,
          int K = 1, bool Checked = false, class Fold = NoFold>
__global__ void __launch_bounds__(1024)
k_generate_refill(const GraphDev g0, const BatchTable tab, const SchedParams sp,
                  int64_t *__restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const uint32_t shift = sp.tile_shift;
  const uint32_t T = 1u << shift;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int warps = blockDim.x >> 5;
  RT *ring = reinterpret_cast<RT *>(smem_raw) + static_cast<size_t>(wib) * kRing;
  const uint32_t ring_s = static_cast<uint32_t>(__cvta_generic_to_shared(ring));
  GraphDev *sg = nullptr;
  if constexpr (Batched)
    sg = reinterpret_cast<GraphDev *>(smem_raw + static_cast<size_t>(warps) * kRing * sizeof(RT)) + wib;
  Draw draw;  // tables (if any) after the rings
  draw.setup(g0, reinterpret_cast<uint32_t *>(smem_raw + static_cast<size_t>(warps) * kRing * sizeof(RT)),
             sizeof(RT) == 4);
  const uint32_t lt = (1u << lane) - 1u;
  const uint64_t gwarp = static_cast<uint64_t>(blockIdx.x) * warps + wib;
  constexpr uint32_t kLanes = 32u * K;  // virtual lanes of the warp
  constexpr uint32_t kSteps = 2;  // fast steps per loop iteration
  bool first = true;

  for (;;) {  // one tile of up to T edges at a time (section 2: batches of edge IDs)
    const uint64_t t = next_tile(sp, first, gwarp);
    if (t >= sp.num_tiles) break;
    uint64_t base;
    if constexpr (Batched) {
      copy_graph(sg, tab.graphs + graph_of_tile(tab, t));
      base = sg->begin + ((t - sg->tile0) << shift);
    } else {
      base = g0.begin + (t << shift);
    }
    const GraphDev &g = Batched ? *sg : g0;
    const uint32_t len = static_cast<uint32_t>(min(static_cast<uint64_t>(T), g.end - base));
    draw.bind(g);
    const RT l2m0 = seed_limit<RT>(g.two_m0);
    const RT r0 = static_cast<RT>(2 * base + 1);
    auto flush = [&](uint32_t from, uint32_t count) {
      // ring entries from..from+count-1 are contiguous: a chunk never wraps the ring
      if constexpr (Fold::kActive)
        Fold::template chunk<RT, HasSeed>(ring + (from & (kRing - 1)), base + from, count, g,
                                          out, sp);
      else
        flush_tile<RT, HasSeed, Narrow, Checked>(ring + (from & (kRing - 1)), base + from,
                                                 count, g, out, sp.out_cap, sp.status);
    };
    auto flush_full = [&](uint32_t from) {  // a whole chunk: a fixed trip count per lane
      if constexpr (Fold::kActive)
        flush(from, kChunk);
      else
        flush_tile<RT, HasSeed, Narrow, Checked, true>(ring + (from & (kRing - 1)), base + from,
                                                       kChunk, g, out, sp.out_cap, sp.status);
    };

    // Chain c of this lane: edge base+o[c] at position r[c] while busy[c].
    uint32_t hoff = min(kLanes, len);
    uint32_t o[K];
    RT r[K];
    bool busy[K];
#pragma unroll
    for (int c = 0; c < K; ++c) {
      o[c] = 32u * c + lane;
      busy[c] = o[c] < hoff;
      r[c] = r0 + 2 * static_cast<RT>(o[c]);
    }
    uint32_t flushed = 0;  // edges [0, flushed) of the tile are written out
    bool all_busy = hoff == kLanes;

    // Fast steps: every chain busy and >= kSteps*kLanes IDs may still be handed out before
    // the ring is full or the tile ends; a chain that stops parks r and starts the next ID.
    // The bookkeeping is predicated PTX (park_and_refill): no branch per step.
    auto in_flight_below = [&](uint32_t edge) {  // any chain of the warp on an edge < edge?
      bool any = false;
#pragma unroll
      for (int c = 0; c < K; ++c) any |= busy[c] && o[c] < edge;
      return __any_sync(kFull, any);
    };
    auto fast_loop = [&](auto seed_tag) {
      constexpr bool Seed = decltype(seed_tag)::value;
      uint32_t last = min(len, flushed + kRing) - kSteps * kLanes;
      for (;;) {
#pragma unroll
        for (uint32_t u = 0; u < kSteps; ++u) {
#pragma unroll
          for (int c = 0; c < K; ++c) r[c] = draw(r[c]);
#pragma unroll
          for (int c = 0; c < K; ++c) park_and_refill<Seed>(r[c], o[c], hoff, lt, r0, l2m0, ring_s);
        }
        if (hoff <= last) continue;
        // The ring is nearly full (or the tile nearly used up): write the oldest chunk out
        // without leaving the fast steps when the ring is the limit and the chunk is done.
        if (flushed + kRing >= len || in_flight_below(flushed + kChunk)) break;
        flush_full(flushed);
        flushed += kChunk;
        last = min(len, flushed + kRing) - kSteps * kLanes;
        if (hoff > last) break;
      }
    };

    for (;;) {
      if (all_busy && hoff + kSteps * kLanes <= min(len, flushed + kRing)) {
        if (HasSeed && l2m0 != 0) fast_loop(std::true_type{});
        else fast_loop(std::false_type{});
      }
      // Make room: write out the oldest chunks whose edges are all done.
      bool made_room = false;
      while (flushed + kChunk <= hoff && !in_flight_below(flushed + kChunk)) {
        flush_full(flushed);
        flushed += kChunk;
        made_room = true;
      }
      // Every chain still busy and room again: back to the fast steps directly.
      if (made_room && all_busy && hoff + kSteps * kLanes <= min(len, flushed + kRing)) continue;
      if (hoff == len && !in_flight_below(len)) break;  // tile done
      // General step: some chains idle, or the ring or the tile is nearly used up.
      uint32_t room = min(len, flushed + kRing) - hoff;
      bool idle = false;
#pragma unroll
      for (int c = 0; c < K; ++c) {
        if (busy[c]) {
          r[c] = draw(r[c]);
          if (chain_stops<RT, HasSeed>(r[c], l2m0)) {
            ring[o[c] & (kRing - 1)] = r[c];
            busy[c] = false;
          }
        }
        const uint32_t fm = __ballot_sync(kFull, !busy[c]);
        const uint32_t k = min(room, static_cast<uint32_t>(__popc(fm)));
        const uint32_t rank = __popc(fm & lt);
        if (!busy[c] && rank < k) {
          o[c] = hoff + rank;
          r[c] = r0 + 2 * static_cast<RT>(o[c]);
          busy[c] = true;
        }
        hoff += k;
        room -= k;
        idle |= !busy[c];
      }
      all_busy = __ballot_sync(kFull, idle) == 0;
    }
    while (flushed < len) {  // the rest, chunk by chunk (a chunk never wraps the ring)
      const uint32_t c = min(kChunk, len - flushed);
      flush(flushed, c);
      flushed += c;
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------------ launch helpers --

int floor_log2(uint32_t x) { return 31 - __builtin_clz(x); }

constexpr size_t kMaxSmemPerCta = 227 * 1024;  // sm_100-class opt-in limit per CTA

template <class K>
ba_status set_smem(K kernel, size_t smem) {
  if (smem > kMaxSmemPerCta) {
    set_error("launch shape needs more shared memory per CTA than an SM offers "
              "(lower block or tile)");
    return BA_ERR_INVALID_ARG;
  }
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) cudaGetLastError();  // not sticky: clear it so later checks stay exact
  return e == cudaSuccess ? BA_OK : cuda_fail(e, "cudaFuncSetAttribute");
}

// Persistent grid: min(SMs x CTAs/SM (capped by occupancy), CTAs that have a tile).
template <class K>
ba_status persistent_grid(K kernel, int block, size_t smem, int ctas_per_sm, uint64_t work_ctas,
                          int *grid) {
  int occ = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, block, smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  if (occ < 1) {
    set_error("launch shape does not fit on an SM (block size / shared memory)");
    return BA_ERR_INVALID_ARG;
  }
  const uint64_t cap = static_cast<uint64_t>(sm_count()) * std::min(occ, std::max(ctas_per_sm, 1));
  *grid = static_cast<int>(std::max<uint64_t>(1, std::min(cap, work_ctas)));
  return BA_OK;
}

ba_status check_launch(const char *what) {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? BA_OK : cuda_fail(e, what);
}

}  // namespace
}  // namespace ba
